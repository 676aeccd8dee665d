"""Dynamical spin structure factor by the continued-fraction expansion:
S^z sums between sectors (ed_apply_sz) and the Lanczos recursion from a given
vector (ed_lanczos_tridiag).

CPU (oracle): the oracle's poles and weights (dense eigendecomposition of the
fixed-Sz matrix) are pinned to the two-site closed form (the singlet's
staggered S^z has weight 1/2 at w = J, the uniform one none), to the
static sum rule sum_n w_n = S(q)/3 of a singlet ground state with S(q) from
the oracle's spin correlations, and to the f-sum rule
sum_n (E_n - E_0) w_n = -(2/(3N)) sum_b J_b (1 - cos q.d_b) <S_i.S_j>.
The host logic that finds the target sector is checked against the same
condition on the oracle side (the operator's phases under every element).

GPU: ed_apply_sz against the oracle's V_to^dagger O V_from x (momentum
transfer, spin-flip parity change, the translation sector of a point-group
sector; every dtype, two vectors), its argument checks; the continued
fraction with full reorthogonalisation against the oracle's Lorentzians on a
frequency grid, and the plain recursion's moments e_1^T T^k e_1 against the
oracle's sum_n w_n (E_n)^k; at the 24-site triangular workload the static and
f-sum rules with the GPU's own correlations.
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Cluster, Problem, Sector, allowed_momenta, triangular_lattice
from edinputs.vectors import state_vector

EPS64 = np.finfo(np.float64).eps


def _lam(sector, c):
    """lambda(g) with s_g c_{g^-1(j)} = lambda(g) c_j (the oracle side's own statement)."""
    N = sector.n_sites
    out = []
    for g in range(sector.n_sym):
        p = np.asarray(sector.perm[g])
        inv = np.empty(N, int)
        inv[p] = np.arange(N)
        sg = -1.0 if sector.spinflip[g] else 1.0
        j0 = int(np.argmax(np.abs(c)))
        lam = sg * c[inv[j0]] / c[j0]
        assert np.allclose(sg * c[inv], lam * c, atol=1e-12)
        out.append(lam)
    return np.array(out)


def _target(sector, c):
    chi = _lam(sector, c) * np.asarray(sector.chi)
    chi = np.where(np.abs(chi.imag) < 1e-12, chi.real + 0j, chi)
    return Sector(sector.n_sites, sector.n_up, np.asarray(sector.perm), np.asarray(sector.spinflip), chi,
                  sector.n_sublat)


def _sub(sector, idx):
    idx = [0] + [int(e) for e in idx if int(e) != 0]
    return Sector(sector.n_sites, sector.n_up, np.asarray(sector.perm)[idx], np.asarray(sector.spinflip)[idx],
                  np.asarray(sector.chi)[idx], sector.n_sublat)


def _coef(positions, q):
    r = np.asarray(positions, dtype=float)
    return np.exp(1j * (r @ np.asarray(q, dtype=float))) / np.sqrt(len(r))


def _ground(p):
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    w, v = np.linalg.eigh(H.toarray())
    return w[0], v[:, 0]


def _chain(**kw):
    return C.chain(12, 1.0, 0.3, translations=True, **kw)


def _qchain(n):
    return np.array([2 * np.pi * n / 12, 0.0])


def _fsum(p, C_, q):
    """-(2/(3N)) sum_b J_b (1 - cos q.d_b) C_ij for an SU(2) singlet."""
    r = np.asarray(p.meta["positions"], dtype=float)
    N = len(r)
    tot = 0.0
    for (i, j), J in zip(p.terms.bonds, p.terms.J):
        tot += J * (1 - np.cos(np.asarray(q) @ (r[i] - r[j]))) * C_[i, j]
    return -2.0 * tot / (3 * N)


def _sq(C_, positions, q):
    r = np.asarray(positions, dtype=float)
    ph = np.exp(1j * (r @ np.asarray(q, dtype=float)))
    return float(np.real(np.conj(ph) @ C_ @ ph)) / len(r)


# ---------------------------------------------------------------- oracle pins
def test_oracle_two_site_singlet():
    from edinputs.lattice import Terms
    s = Sector(2, 1, np.array([[0, 1]], np.int32), np.zeros(1, np.uint8), np.ones(1, complex), 1)
    t = Terms(np.array([[0, 1]], np.int32), np.array([1.0]), np.zeros((0, 3), np.int32), np.zeros(0))
    p = Problem("two", s, t)
    singlet = np.array([1.0, -1.0]) / np.sqrt(2)       # basis |01>, |10>
    poles, w, e0 = oracle.sz_spectrum(p, singlet, np.array([1.0, -1.0]) / np.sqrt(2))
    assert e0 == pytest.approx(-0.75)
    k = np.argmax(w)
    assert poles[k] == pytest.approx(1.0) and w[k] == pytest.approx(0.5) and w.sum() == pytest.approx(0.5)
    _, w0, _ = oracle.sz_spectrum(p, singlet, np.array([1.0, 1.0]) / np.sqrt(2))
    assert w0.sum() < 1e-30
    om = np.linspace(-1, 3, 9)
    L = oracle.lorentzians([1.0], [0.5], om, 0.2)
    assert np.allclose(L, 0.5 * 0.2 / np.pi / ((om - 1.0) ** 2 + 0.04))


@pytest.mark.parametrize("n", [1, 3, 6])
def test_oracle_sum_rules_chain12(n):
    p = _chain()
    e0, psi = _ground(p)
    Cm = oracle.correlation_matrix(p.sector, psi)
    q = _qchain(n)
    c = _coef(p.meta["positions"], q)
    poles, w, e = oracle.sz_spectrum(p, psi, c)
    assert e == pytest.approx(e0, abs=1e-12)
    assert w.sum() == pytest.approx(_sq(Cm, p.meta["positions"], q) / 3, abs=1e-12)
    assert (poles * w).sum() == pytest.approx(_fsum(p, Cm, q), abs=1e-12)
    assert poles[w > 1e-12].min() > -1e-10                       # excitations above the ground state


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


def _tri12():
    return C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, n_up=6)


def _tri_q(P_, index):
    qs = allowed_momenta(Cluster(triangular_lattice(), P_))
    return np.asarray(qs[index], dtype=float)


def _case(name):
    """(source sector, coefficients, positions) for each transfer case."""
    if name == "chain12_k0_q3":
        p = _chain()
        return p, p.sector, _coef(p.meta["positions"], _qchain(3))
    if name == "chain12_k1_q5":
        p = _chain(k=1)
        return p, p.sector, _coef(p.meta["positions"], _qchain(5))
    if name == "chain12_flip_qpi":
        p = _chain(spinflip=1)
        return p, p.sector, np.real(_coef(p.meta["positions"], _qchain(6))).astype(complex)
    if name == "triangular12_T_q":
        p = _tri12()
        return p, _sub(p.sector, p.meta["translations"]), _coef(p.meta["positions"], _tri_q([[2, 2], [-2, 4]], 3))
    raise KeyError(name)


CASES = ["chain12_k0_q3", "chain12_k1_q5", "chain12_flip_qpi", "triangular12_T_q"]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32", "c128", "c64"])
@pytest.mark.parametrize("name", CASES)
def test_gpu_apply_sz_matches_oracle(P, name, dtype):
    import torch
    p, src, c = _case(name)
    tgt = _target(src, c)
    real_ok = np.all(np.abs(c.imag) < 1e-12) and src.is_real and tgt.is_real
    if dtype in ("f64", "f32") and not real_ok:
        pytest.skip("complex coefficients or characters need a complex dtype")
    bf, bt = P.Basis(src), P.Basis(tgt)
    reps, _ = bf.export()
    cplx = dtype in ("c128", "c64")
    X = np.stack([state_vector(41 + v, reps, complex_=cplx) for v in range(2)])
    tdt = {"f64": torch.float64, "f32": torch.float32, "c128": torch.complex128, "c64": torch.complex64}[dtype]
    x = torch.tensor(X, dtype=tdt, device="cuda")
    y = bf.apply_sz(bt, c, x)
    torch.cuda.synchronize()
    Y = y.cpu().numpy().astype(complex)
    Xin = x.cpu().numpy().astype(complex)
    N = src.n_sites
    states = oracle.sz_states(N, src.n_up)
    fz = np.array([sum(c[i] * (0.5 if (int(s) >> (N - 1 - i)) & 1 else -0.5) for i in range(N)) for s in states])
    Vt, _ = oracle.projector_matrix(tgt, states)
    tol = 64 * EPS64 if dtype in ("f64", "c128") else 8 * np.finfo(np.float32).eps
    for v in range(2):
        phi, _ = oracle.plain_state(src, Xin[v])
        ref = Vt.conj().T @ (fz * phi)
        scale = np.abs(Xin[v]).max() * np.abs(c).sum()
        assert np.all(np.abs(Y[v] - ref) <= tol * scale), np.abs(Y[v] - ref).max()


@pytest.mark.gpu
def test_gpu_apply_sz_argument_checks(P):
    import torch
    p = _chain()
    bf = P.Basis(p.sector)
    x = torch.zeros(bf.dim, dtype=torch.complex128, device="cuda")
    c = _coef(p.meta["positions"], _qchain(3))
    bt = P.Basis(_target(p.sector, c))
    with pytest.raises(P.EdError) as e:             # the source sector is not where S^z(q) maps to
        bf.apply_sz(bf, c, x)
    assert e.value.name == "ED_ERR_ARG"
    bad = np.exp(1j * 0.37 * np.arange(12)) / np.sqrt(12)   # not a momentum of the ring
    with pytest.raises(P.EdError) as e:
        bf.apply_sz(bt, bad, x)
    assert e.value.name == "ED_ERR_ARG"
    with pytest.raises(P.EdError) as e:             # complex coefficients, real vectors
        bf.apply_sz(bt, c, torch.zeros(bf.dim, dtype=torch.float64, device="cuda"))
    assert e.value.name == "ED_ERR_ARG"
    with pytest.raises(P.EdError) as e:
        bf.apply_sz(bt, np.zeros(12, complex), x)
    assert e.value.name == "ED_ERR_ARG"


def _gpu_ground(P, basis, terms):
    import torch
    h = P.Hamiltonian(basis, terms)
    tdt = torch.float64 if h.is_real else torch.complex128
    ev = torch.zeros((1, basis.dim), dtype=tdt, device="cuda")
    vals, _ = h.lanczos(n_eig=1, tol=1e-12, max_iter=300, evecs=ev)
    return h, float(vals[0]), ev[0].contiguous()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [3, 6])
def test_gpu_continued_fraction_chain12(P, n):
    import torch
    from paper_2210_03511_gb300.observables import continued_fraction, dynamical_structure_factor
    p = _chain()
    b = P.Basis(p.sector)
    h, e0, psi = _gpu_ground(P, b, p.terms)
    c = _coef(p.meta["positions"], _qchain(n))
    tgt = _target(p.sector, c)
    bt = P.Basis(tgt)
    ht = P.Hamiltonian(bt, p.terms)
    phi = b.apply_sz(bt, c, psi.to(torch.complex128))
    poles, w, e_o = oracle.sz_spectrum(p, psi.cpu().numpy(), c)
    assert e_o == pytest.approx(e0, abs=1e-9)
    om = np.linspace(-0.5, 4.0, 91)
    eta = 0.1
    S, a, bb, n2 = dynamical_structure_factor(ht, phi, om, e0, eta, m=400, reorth=True)
    assert n2 == pytest.approx(w.sum(), rel=1e-12)
    assert len(a) <= bt.dim
    So = oracle.lorentzians(poles, w, om, eta)
    assert np.allclose(S, So, rtol=0, atol=1e-8 * So.max()), np.abs(S - So).max()
    # the plain recursion: its first moments are exact
    a2, b2, n22 = ht.lanczos_tridiag(phi, 12, reorth=False)
    k = len(a2)
    T = np.diag(a2) + np.diag(b2[:k - 1], 1) + np.diag(b2[:k - 1], -1)
    e1 = np.zeros(k)
    e1[0] = 1.0
    v = e1.copy()
    for mom in range(6):
        ref = float((w * (poles + e0) ** mom).sum())
        assert n22 * (e1 @ v) == pytest.approx(ref, rel=1e-9, abs=1e-12)
        v = T @ v
    # far from the spectrum the fraction is |phi|^2 / z (1 + alpha_0 / z + ...)
    z = 1.0e4
    G = continued_fraction(a2, b2, n22, np.array([z + 0j]))
    assert G[0].real * z == pytest.approx(n22 * (1 + a2[0] / z), rel=1e-6)


@pytest.mark.gpu
def test_gpu_structure_factor_triangular12_via_translation_sector(P):
    """Point-group sector -> translation sector (ed_restrict) -> S^z(q) (ed_apply_sz)
    -> continued fraction, against the oracle's dense spectrum of the same state."""
    import torch
    from paper_2210_03511_gb300.observables import TranslationSector, dynamical_structure_factor, sz_target_sector
    p = _tri12()
    b = P.Basis(p.sector)
    h, e0, psi = _gpu_ground(P, b, p.terms)
    ts = TranslationSector(b, p.sector, p.meta["translations"])
    psi_t = b.restrict_to(ts.sub, psi.to(torch.complex128))
    q = _tri_q([[2, 2], [-2, 4]], 3)
    c = _coef(p.meta["positions"], q)
    tgt = sz_target_sector(ts.sector, c)
    bt = P.Basis(tgt)
    ht = P.Hamiltonian(bt, p.terms)
    phi = ts.sub.apply_sz(bt, c, psi_t)
    om = np.linspace(-0.5, 5.0, 111)
    S, a, bb, n2 = dynamical_structure_factor(ht, phi, om, e0, 0.1, m=400, reorth=True)
    poles, w, _ = oracle.sz_spectrum(p, psi.cpu().numpy(), c)
    So = oracle.lorentzians(poles, w, om, 0.1)
    assert n2 == pytest.approx(w.sum(), rel=1e-10)
    assert np.allclose(S, So, rtol=0, atol=1e-8 * So.max()), np.abs(S - So).max()
    ts.close()


@pytest.mark.gpu
def test_gpu_sum_rules_triangular24(P):
    """24-site triangular workload (T24 x C2v ground state): the static sum rule
    |S^z(q)|0>|^2 = S(q)/3 and the f-sum rule (alpha_0 - E_0)|phi|^2, with S(q)
    and the bond correlations from the GPU's own orbit-averaged correlations."""
    import torch
    from paper_2210_03511_gb300.observables import (TranslationSector, correlations, dynamical_structure_factor,
                                                    sz_target_sector)
    p = C.triangular24()
    b = P.Basis(p.sector)
    h, e0, psi = _gpu_ground(P, b, p.terms)
    Cm = correlations(b, p.sector, psi)
    ts = TranslationSector(b, p.sector, p.meta["translations"])
    psi_t = b.restrict_to(ts.sub, psi.to(torch.complex128))
    for index in (1, 5):
        q = _tri_q([[5, 1], [4, -4]], index)
        c = _coef(p.meta["positions"], q)
        bt = P.Basis(sz_target_sector(ts.sector, c))
        ht = P.Hamiltonian(bt, p.terms)
        phi = ts.sub.apply_sz(bt, c, psi_t)
        S, a, bb, n2 = dynamical_structure_factor(ht, phi, np.array([0.0]), e0, 0.1, m=30, reorth=False)
        # both rules hold exactly for an SU(2) singlet; the Ritz vector (residual
        # ~1e-6 at the Lanczos tolerance) carries S = 2 admixtures that enter to
        # first order (3e-8 relative was seen), hence the looser bounds
        assert n2 == pytest.approx(_sq(Cm, p.meta["positions"], q) / 3, rel=1e-6)
        assert (a[0] - e0) * n2 == pytest.approx(_fsum(p, Cm, q), rel=1e-5)
        ht.close()
        bt.close()
    ts.close()


# ---------------------------------------------------------------- host logic (CPU)
def test_continued_fraction_is_the_resolvent():
    """norm2 / (z - a0 - b0^2/(z - a1 - ...)) = norm2 [(z - T)^-1]_00 for the tridiagonal T."""
    from paper_2210_03511_gb300.observables import continued_fraction
    rng = np.random.default_rng(4)
    for m in (1, 2, 7, 30):
        a = rng.normal(size=m)
        b = np.abs(rng.normal(size=m)) + 0.1
        T = np.diag(a) + np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
        z = np.array([0.3 + 0.05j, -1.7 + 0.2j, 4.0 + 1e-3j])
        G = continued_fraction(a, b, 2.5, z)
        ref = [2.5 * np.linalg.inv(zz * np.eye(m) - T)[0, 0] for zz in z]
        assert np.allclose(G, ref, rtol=1e-10, atol=0)


def test_sz_target_sector_host():
    """The target sector of S^z(q) on a ring: characters exp(i (k - q) t); a phase
    pattern that is not a momentum of the ring is refused."""
    from paper_2210_03511_gb300.observables import sz_target_sector, szq_coefficients
    p = _chain(k=1)
    pos = np.asarray(p.meta["positions"])
    q = _qchain(5)
    c = szq_coefficients(pos, q)
    assert np.allclose(c, _coef(pos, q))
    tgt = sz_target_sector(p.sector, c)
    ref = _chain(k=(1 - 5) % 12)
    assert np.array_equal(np.asarray(tgt.perm), np.asarray(ref.sector.perm))
    assert np.allclose(tgt.chi, ref.sector.chi, atol=1e-12)
    assert np.allclose(tgt.chi, _target(p.sector, c).chi, atol=1e-12)
    with pytest.raises(ValueError):
        sz_target_sector(p.sector, np.exp(1j * 0.37 * np.arange(12)))
    # spin flip: S^z changes the flip parity
    pf = _chain(spinflip=1)
    tf = sz_target_sector(pf.sector, np.real(_coef(pf.meta["positions"], _qchain(6))).astype(complex))
    perm = np.asarray(pf.sector.perm)
    g = [e for e in range(len(perm)) if pf.sector.spinflip[e] and np.array_equal(perm[e], np.arange(12))][0]
    assert tf.chi[g] == pytest.approx(-pf.sector.chi[g])
