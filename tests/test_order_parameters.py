"""Restriction to a subgroup's sector (ed_restrict) and the four- and six-spin
order parameters built on it: the nematic N (Eq. nematicorderparameter) and
the chirality correlation X (Eq. chiralityorderparameter).

CPU (oracle): products of two local operators are pinned to closed forms,
(S_a.S_b)^2 = 3/16 - 1/2 S_a.S_b for spin 1/2 and <(S_0.S_1)(S_2.S_3)> = 9/16
on two singlets; chi^2 = e^2 in the single-triangle chirality eigenstates
(-e^2 with one orientation reversed).  The oracle's restriction of a ground
state is an eigenvector, with the same energy, of the subgroup sector's matrix
(and of the unsymmetrised fixed-Sz matrix for the trivial group); restrictions
of two irreps of one momentum are orthogonal.  The translation-sum identity
the library uses, sum_t <O t O t^-1> = <B^2>/|T|, is checked against the
oracle's term-by-term sums.

GPU: ed_restrict against the oracle's V_H^dagger V_G x element by element
(real, complex, FP32, several vectors, the trivial group), its argument
checks, and N and X of the library against the oracle's on the same GPU
ground state; at the 24-site triangular workload (T24 x C2v) properties that
hold at any size: the restricted ground state has the same Rayleigh quotient
and the same residual under the translation sector's H, <B>/|T| equals the correlation
computed in the full symmetric sector, and <B^2> - <B>^2 >= 0.
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Problem, Sector, Terms
from edinputs.vectors import state_vector

EPS64 = np.finfo(np.float64).eps


def _sub(sector, idx):
    idx = [0] + [int(e) for e in idx if int(e) != 0]
    return Sector(sector.n_sites, sector.n_up, np.asarray(sector.perm)[idx], np.asarray(sector.spinflip)[idx],
                  np.asarray(sector.chi)[idx], sector.n_sublat)


def _trivial(sector):
    return _sub(sector, [0])


def _ground(p):
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    w, v = np.linalg.eigh(H.toarray())
    return w[0], v[:, 0]


def _orbit(perm, tr, sites):
    return [tuple(int(perm[t][s]) for s in sites) for t in tr]


def _tri12():
    return C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, n_up=6)


# ---------------------------------------------------------------- oracle pins
def test_oracle_bond_square_closed_form():
    p = C.chain(12, 1.0, 0.3, translations=True)
    e0, psi = _ground(p)
    Cm = oracle.correlation_matrix(p.sector, psi)
    for a, b in ((0, 1), (2, 5), (3, 9)):
        v = oracle.product_expectation(p.sector, psi, ("bond", (a, b)), ("bond", (a, b)))
        assert v.real == pytest.approx(3 / 16 - 0.5 * Cm[a, b], abs=1e-12) and abs(v.imag) < 1e-12


def test_oracle_two_singlets():
    s = Sector(4, 2, np.array([[0, 1, 2, 3]], np.int32), np.zeros(1, np.uint8), np.ones(1, complex), 1)
    # product basis 0011, 0101, 0110, 1001, 1010, 1100 (site 0 = MSB): singlet(0,1) x singlet(2,3)
    psi = np.array([0.0, 0.5, -0.5, -0.5, 0.5, 0.0])
    v = oracle.product_expectation(s, psi, ("bond", (0, 1)), ("bond", (2, 3)))
    assert v == pytest.approx(9 / 16, abs=1e-14)
    assert oracle.product_expectation(s, psi, ("bond", (0, 1)), ("bond", (0, 1))) == pytest.approx(9 / 16)
    # the nematic sum over the single bond (2, 3) is connected: 9/16 - (3/4)^2 = 0
    assert abs(oracle.nematic(s, psi, (0, 1), [(2, 3)])) < 1e-14


def test_oracle_chirality_square_in_eigenstates():
    s = Sector(3, 1, np.array([[0, 1, 2]], np.int32), np.zeros(1, np.uint8), np.ones(1, complex), 1)
    t = Terms(np.zeros((0, 2), np.int32), np.zeros(0), np.array([[0, 1, 2]], np.int32), np.ones(1))
    Hd, _ = oracle.dense_sz(Problem("tri", s, t))
    w, v = np.linalg.eigh(Hd)
    for e, vec in zip(w, v.T):
        a = oracle.product_expectation(s, vec, ("tri", (0, 1, 2)), ("tri", (0, 1, 2)))
        b = oracle.product_expectation(s, vec, ("tri", (0, 1, 2)), ("tri", (1, 0, 2)))
        assert a.real == pytest.approx(e * e, abs=1e-14) and b.real == pytest.approx(-e * e, abs=1e-14)
        assert oracle.chirality_sum(s, vec, (0, 1, 2), [(0, 1, 2), (2, 0, 1)]).real == pytest.approx(2 * e * e)


def test_oracle_restriction_is_an_eigenvector():
    p = _tri12()
    e0, psi = _ground(p)
    T = _sub(p.sector, p.meta["translations"])
    psi_t = oracle.restrict(p.sector, psi, T)
    assert np.linalg.norm(psi_t) == pytest.approx(1.0, abs=1e-12)
    Ht = oracle.csr(Problem("t", T, p.terms))
    assert np.linalg.norm(Ht @ psi_t - e0 * psi_t) < 1e-10
    phi = oracle.restrict(p.sector, psi, _trivial(p.sector))
    Hd, _ = oracle.dense_sz(p)
    assert len(phi) == oracle.binom(12, 6) and np.linalg.norm(Hd @ phi - e0 * phi) < 1e-10
    # another irrep at the same momentum restricts to an orthogonal vector of the same sector
    q = C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, n_up=6, irrep="B1")
    _, chi_q = _ground(q)
    chi_t = oracle.restrict(q.sector, chi_q, _sub(q.sector, q.meta["translations"]))
    assert abs(np.vdot(psi_t, chi_t)) < 1e-12


def test_oracle_translation_sum_identity():
    """sum over the translates of <O_0 O_t> equals <B^2>/|T| with B the
    translation sum, <B^2> = |B psi_T|^2 in the translation sector."""
    p = _tri12()
    e0, psi = _ground(p)
    tr = p.meta["translations"]
    T = _sub(p.sector, tr)
    psi_t = oracle.restrict(p.sector, psi, T)
    bond = tuple(int(v) for v in p.terms.bonds[0])
    bonds = _orbit(p.sector.perm, tr, bond)
    Bt = oracle.csr(Problem("b", T, Terms(np.array(bonds, np.int32), np.ones(len(bonds)), np.zeros((0, 3), np.int32),
                                          np.zeros(0))))
    b1 = np.vdot(psi_t, Bt @ psi_t).real
    b2 = np.linalg.norm(Bt @ psi_t) ** 2
    n = oracle.nematic(p.sector, psi, bond, bonds)
    assert abs(n.imag) < 1e-12
    assert n.real == pytest.approx((b2 - b1 * b1) / len(tr), abs=1e-12)
    tri = tuple(p.meta["triangles"][0])
    tris = _orbit(p.sector.perm, tr, tri)
    Xt = oracle.csr(Problem("x", T, Terms(np.zeros((0, 2), np.int32), np.zeros(0), np.array(tris, np.int32),
                                          np.ones(len(tris)))))
    x = oracle.chirality_sum(p.sector, psi, tri, tris)
    assert abs(x.imag) < 1e-12
    assert x.real == pytest.approx(np.linalg.norm(Xt @ psi_t) ** 2 / len(tr), abs=1e-12)


# ---------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


CASES = {
    "triangular12_A1_translations": (_tri12, "translations"),
    "triangular12_A1_trivial": (_tri12, "trivial"),
    "kagome12_E1_translations": (lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"), "translations"),
    "chain12_flip_translations": (lambda: C.chain(12, 1.0, 0.3, translations=True, spinflip=-1), "translations"),
}


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32", "c128", "c64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_gpu_restrict_matches_oracle(P, name, dtype):
    import torch
    make, which = CASES[name]
    p = make()
    if dtype in ("f64", "f32") and not p.sector.is_real:
        pytest.skip("complex characters need a complex dtype")
    sub = _trivial(p.sector) if which == "trivial" else _sub(p.sector, p.meta["translations"])
    b = P.Basis(p.sector)
    bs = P.Basis(sub)
    reps, _ = b.export()
    cplx = dtype in ("c128", "c64")
    nvec = 2
    X = np.stack([state_vector(31 + v, reps, complex_=cplx) for v in range(nvec)])
    tdt = {"f64": torch.float64, "f32": torch.float32, "c128": torch.complex128, "c64": torch.complex64}[dtype]
    x = torch.tensor(X, dtype=tdt, device="cuda")
    y = b.restrict_to(bs, x)
    torch.cuda.synchronize()
    Y = y.cpu().numpy().astype(complex)
    Xin = x.cpu().numpy().astype(complex)       # the values the kernel read (rounded for FP32)
    tol = 64 * EPS64 if dtype in ("f64", "c128") else 4 * np.finfo(np.float32).eps
    for v in range(nvec):
        ref = oracle.restrict(p.sector, Xin[v], sub)
        assert ref.shape == Y[v].shape
        scale = np.abs(Xin[v]).max()
        assert np.all(np.abs(Y[v] - ref) <= tol * scale), np.abs(Y[v] - ref).max()
        assert np.linalg.norm(Y[v]) == pytest.approx(np.linalg.norm(Xin[v]), rel=10 * tol)
    # one vector gives the first row of the two-vector call
    y1 = b.restrict_to(bs, x[0].contiguous())
    assert torch.equal(y1, y[0])


@pytest.mark.gpu
def test_gpu_restrict_argument_checks(P):
    import torch
    p = C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1")
    sub = _sub(p.sector, p.meta["translations"])
    b, bs = P.Basis(p.sector), P.Basis(sub)
    x = torch.zeros(b.dim, dtype=torch.complex128, device="cuda")
    xs = torch.zeros(bs.dim, dtype=torch.complex128, device="cuda")
    with pytest.raises(P.EdError) as e:             # the group is not a subgroup of its translations
        bs.restrict_to(b, xs)
    assert e.value.name == "ED_ERR_ARG"
    # same group (the translations of a 12-site chain), characters of another momentum
    k1 = C.chain(12, 1.0, 0.3, translations=True, k=1)
    k2 = C.chain(12, 1.0, 0.3, translations=True, k=2)
    b1, b2 = P.Basis(k1.sector), P.Basis(k2.sector)
    with pytest.raises(P.EdError) as e:
        b1.restrict_to(b2, torch.zeros(b1.dim, dtype=torch.complex128, device="cuda"))
    assert e.value.name == "ED_ERR_ARG"
    with pytest.raises(P.EdError) as e:             # complex characters, real vectors
        b.restrict_to(bs, torch.zeros(b.dim, dtype=torch.float64, device="cuda"))
    assert e.value.name == "ED_ERR_ARG"


def _gpu_ground(P, p):
    import torch
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    tdt = torch.float64 if h.is_real else torch.complex128
    ev = torch.zeros((1, b.dim), dtype=tdt, device="cuda")
    vals, _ = h.lanczos(n_eig=1, tol=1e-12, max_iter=300, evecs=ev)
    return b, h, float(vals[0]), ev[0].contiguous()


@pytest.mark.gpu
def test_gpu_order_parameters_triangular12(P):
    from paper_2210_03511_gb300.observables import TranslationSector, chirality_correlation, nematic
    p = _tri12()
    b, h, e0, psi = _gpu_ground(P, p)
    ts = TranslationSector(b, p.sector, p.meta["translations"])
    psi_h = psi.cpu().numpy()
    tr = p.meta["translations"]
    for bond in (tuple(int(v) for v in p.terms.bonds[0]), tuple(int(v) for v in p.terms.bonds[-1])):
        ng = nematic(ts, psi, bond)
        no = oracle.nematic(p.sector, psi_h, bond, _orbit(p.sector.perm, tr, bond))
        assert ng == pytest.approx(no.real, abs=1e-10)
    for tri in (tuple(p.meta["triangles"][0]), tuple(p.meta["triangles"][-1])):
        xg = chirality_correlation(ts, psi, tri)
        xo = oracle.chirality_sum(p.sector, psi_h, tri, _orbit(p.sector.perm, tr, tri))
        assert xg == pytest.approx(xo.real, abs=1e-10)
    ts.close()


@pytest.mark.gpu
def test_gpu_order_parameters_triangular24_properties(P):
    import torch
    from paper_2210_03511_gb300.observables import TranslationSector, chirality_correlation, correlations, nematic
    p = C.triangular24()
    b, h, e0, psi = _gpu_ground(P, p)
    ts = TranslationSector(b, p.sector, p.meta["translations"])
    assert ts.n_trans == 24
    psi_t = b.restrict_to(ts.sub, psi)
    assert float(torch.linalg.vector_norm(psi_t)) == pytest.approx(float(torch.linalg.vector_norm(psi)), rel=1e-13)
    # the restriction is an isometry that commutes with H: the Ritz pair's
    # residual is the same in both sectors (it is ~1e-6, set by the Lanczos
    # tolerance on the eigenvalue, not by the restriction)
    ht = P.Hamiltonian(ts.sub, p.terms)
    r = torch.empty_like(psi_t)
    ht.apply(psi_t, r)
    rg = torch.empty_like(psi)
    h.apply(psi, rg)
    res_t = float(torch.linalg.vector_norm(r - e0 * psi_t))
    res_g = float(torch.linalg.vector_norm(rg - e0 * psi))
    assert res_g < 1e-4 and abs(res_t - res_g) < 1e-10, (res_t, res_g)
    assert np.real(ht.expectation(psi_t)[0]) == pytest.approx(e0, abs=1e-9)
    bond = tuple(int(v) for v in p.terms.bonds[0])
    from paper_2210_03511_gb300.observables import _Bonds
    bonds = ts.orbit_bonds(bond)
    b1, b2 = ts.moments(psi, _Bonds(bonds, np.ones(len(bonds)), np.zeros((0, 3), np.int32), np.zeros(0)))
    Cm = correlations(b, p.sector, psi)
    assert b1 / 24 == pytest.approx(Cm[bond[0], bond[1]], abs=1e-10)
    assert nematic(ts, psi, bond) == pytest.approx((b2 - b1 * b1) / 24, abs=1e-12)
    assert b2 - b1 * b1 >= -1e-9
    assert chirality_correlation(ts, psi, tuple(p.meta["triangles"][0])) >= 0.0
    ht.close()
    ts.close()


# ---------------------------------------------------------------- host logic (CPU)
def test_subgroup_sector_host():
    """The subgroup sector keeps the identity first, the restricted characters
    and the sublattice blocks; a subgroup without the identity is refused."""
    from paper_2210_03511_gb300.observables import subgroup_sector
    p = C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1")
    tr = p.meta["translations"]
    sub = subgroup_sector(p.sector, list(reversed(tr)))
    assert np.array_equal(sub.perm[0], np.arange(p.sector.n_sites))
    assert sorted(map(tuple, sub.perm.tolist())) == sorted(tuple(p.sector.perm[t].tolist()) for t in tr)
    for g, row in enumerate(sub.perm):
        e = [t for t in tr if np.array_equal(p.sector.perm[t], row)][0]
        assert sub.chi[g] == p.sector.chi[e] and sub.spinflip[g] == p.sector.spinflip[e]
    assert sub.n_sublat == p.sector.n_sublat
    with pytest.raises(ValueError):
        subgroup_sector(p.sector, [t for t in tr if t != 0])


def test_translation_elements_form_the_translation_group():
    """meta["translations"] of each workload: |T| = number of unit cells, closed
    under composition, no spin flips, each a fixed-point-free permutation but the
    identity."""
    for p in (_tri12(), C.triangular24(), C.kagome36(), C.square32()):
        tr = p.meta["translations"]
        perm = np.asarray(p.sector.perm)
        assert len(tr) == p.meta["n_cells"]
        rows = {tuple(perm[t].tolist()) for t in tr}
        for a in tr:
            assert not p.sector.spinflip[a]
            if a != 0:
                assert np.all(perm[a] != np.arange(len(perm[a])))
            for b in tr:
                assert tuple(perm[a][perm[b]].tolist()) in rows
