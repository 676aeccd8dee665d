"""Ground-state observables: spin correlations <S_i.S_j>, the static structure
factor (Eq. structurefactor) and scalar chiralities <S_i.(S_j x S_k)>.

CPU (oracle and host logic): the oracle's correlation matrix is pinned to the
two-site singlet/triplet, the four-site ring (ground state -2: nearest
neighbours -1/2, diagonal +1/4), the energy identity E = sum_b J_b <S_i.S_j>,
total spin zero of a singlet (sum_ij C_ij = 0) and translation invariance; the
pair orbits partition all pairs; the structure factor obeys its sum rule; the
oracle's triangle chirality is the eigenvalue in the chirality's eigenstates.

GPU: the library's correlations (ed_expectation on orbit-averaged bond
and triangle operators) against the oracle's, computed from the same GPU
ground state, and the energy identity with the chirality terms.
Tolerance 1e-10: both are FP64 sums of O(N^2 |terms|) products of unit-size
numbers.
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Sector


def _ground(p):
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    w, v = np.linalg.eigh(H.toarray())
    return w[0], v[:, 0], reps


def test_oracle_two_site_singlet_and_triplet():
    s = Sector(2, 1, np.array([[0, 1]], np.int32), np.zeros(1, np.uint8), np.ones(1, complex), 1)
    singlet = np.array([1.0, -1.0]) / np.sqrt(2)      # basis order |01>, |10>
    triplet = np.array([1.0, 1.0]) / np.sqrt(2)
    Cs = oracle.correlation_matrix(s, singlet)
    Ct = oracle.correlation_matrix(s, triplet)
    assert Cs[0, 1] == pytest.approx(-0.75) and Ct[0, 1] == pytest.approx(0.25)
    assert Cs[0, 0] == pytest.approx(0.75)


def test_oracle_four_site_ring():
    p = C.chain(4, 1.0, 0.0, translations=True)
    e0, psi, _ = _ground(p)
    assert e0 == pytest.approx(-2.0)
    Cm = oracle.correlation_matrix(p.sector, psi)
    assert Cm[0, 1] == pytest.approx(-0.5) and Cm[0, 2] == pytest.approx(0.25)


def test_oracle_chain12_identities():
    p = C.chain(12, 1.0, 0.0, translations=True)
    e0, psi, _ = _ground(p)
    Cm = oracle.correlation_matrix(p.sector, psi)
    e = sum(J * Cm[i, j] for (i, j), J in zip(p.terms.bonds, p.terms.J))
    assert e == pytest.approx(e0, abs=1e-10)
    assert abs(Cm.sum()) < 1e-10                       # singlet: S_tot^2 = 0
    pos = np.asarray(p.meta["positions"])[:, 0]
    for i in range(12):
        for j in range(12):
            d = int(round(pos[j] - pos[i])) % 12
            i0 = int(np.argmin(np.abs(pos - 0.0)))
            j0 = int(np.argmin(np.abs(pos - d)))
            assert Cm[i, j] == pytest.approx(Cm[i0, j0], abs=1e-12)


def test_pair_orbits_partition():
    from paper_2210_03511_gb300.observables import pair_orbits
    for p in (C.chain(12, 1.0, 0.0, translations=True), C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
              C.square32()):
        N = p.sector.n_sites
        orbs = pair_orbits(p.sector)
        allp = np.concatenate(orbs)
        assert len(allp) == N * (N - 1) // 2
        assert len({(int(a), int(b)) for a, b in allp}) == len(allp)


def test_structure_factor_sum_rule():
    from paper_2210_03511_gb300.observables import structure_factor
    p = C.chain(12, 1.0, 0.0, translations=True)
    e0, psi, _ = _ground(p)
    Cm = oracle.correlation_matrix(p.sector, psi)
    pos = np.asarray(p.meta["positions"])
    ks = np.array([[2 * np.pi * n / 12, 0.0] for n in range(12)])
    S = structure_factor(Cm, pos, ks)
    assert S.sum() == pytest.approx(0.75 * 12, abs=1e-10)   # sum over the allowed momenta
    assert np.argmax(S) == 6                                 # antiferromagnetic peak at k = pi
    # direct form of the definition with reference site 0
    i0 = int(np.argmin(np.linalg.norm(pos, axis=1)))
    for n, k in enumerate(ks):
        direct = sum(np.exp(1j * k @ (pos[j] - pos[i0])) * Cm[j, i0] for j in range(12)).real
        assert S[n] == pytest.approx(direct, abs=1e-10)


SECTORS = {
    "chain12": lambda: C.chain(12, 1.0, 0.3, translations=True),
    "kagome12_E1": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
    "triangular12_A1": lambda: C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, n_up=6),
}


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(SECTORS))
def test_gpu_correlations_match_oracle(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as P
    from paper_2210_03511_gb300.observables import correlations
    p = SECTORS[name]()
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    tdt = torch.complex128 if cplx else torch.float64
    ev = torch.zeros((1, b.dim), dtype=tdt, device="cuda")
    vals, rep = h.lanczos(n_eig=1, tol=1e-12, max_iter=300, evecs=ev)
    psi = ev[0].contiguous()
    Cg = correlations(b, p.sector, psi)
    Co = oracle.correlation_matrix(p.sector, psi.cpu().numpy())
    assert np.allclose(Cg, Co, rtol=0, atol=1e-10), np.abs(Cg - Co).max()
    # the bond energy of the state is its eigenvalue (to the residual of the Ritz pair)
    e = sum(J * Cg[i, j] for (i, j), J in zip(p.terms.bonds, p.terms.J))
    if not len(p.terms.tris):
        assert e == pytest.approx(vals[0], abs=1e-8)
    # <x|H|x> of the full Hamiltonian is the Ritz value
    assert np.real(h.expectation(psi)[0]) == pytest.approx(vals[0], abs=1e-8)


def test_oracle_triangle_chirality_eigenstates():
    """Three sites, one up spin: the chirality S_0.(S_1 x S_2) has eigenvalues 0 and
    +-sqrt(3)/4 there; in each eigenstate the expectation is the eigenvalue."""
    from edinputs.lattice import Terms
    s = Sector(3, 1, np.array([[0, 1, 2]], np.int32), np.zeros(1, np.uint8), np.ones(1, complex), 1)
    t = Terms(np.zeros((0, 2), np.int32), np.zeros(0), np.array([[0, 1, 2]], np.int32), np.ones(1))

    class Prob:
        sector, terms = s, t
    Hd, states = oracle.dense_sz(Prob)
    w, v = np.linalg.eigh(Hd)
    assert np.allclose(sorted(w), [-np.sqrt(3) / 4, 0, np.sqrt(3) / 4])
    # without symmetry the symmetric basis is the product basis in increasing order
    for e, vec in zip(w, v.T):
        assert oracle.triangle_expectation(s, vec, (0, 1, 2)) == pytest.approx(e, abs=1e-12)
        assert oracle.triangle_expectation(s, vec, (1, 0, 2)) == pytest.approx(-e, abs=1e-12)


@pytest.mark.gpu
def test_gpu_chiralities_and_energy_kagome12():
    """Chiral kagome (J_chi = 0.3): GPU triangle chiralities against the oracle's on the
    same GPU ground state, and E = sum_b J_b <S_i.S_j> + sum_t J_chi <chi_t>."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as P
    from paper_2210_03511_gb300.observables import chiralities, correlations
    p = SECTORS["kagome12_E1"]()
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    ev = torch.zeros((1, b.dim), dtype=torch.complex128, device="cuda")
    vals, rep = h.lanczos(n_eig=1, tol=1e-12, max_iter=300, evecs=ev)
    psi = ev[0].contiguous()
    chi_g = chiralities(b, p.sector, psi, p.terms.tris)
    psi_h = psi.cpu().numpy()
    chi_o = np.array([oracle.triangle_expectation(p.sector, psi_h, t) for t in p.terms.tris])
    assert np.allclose(chi_g, chi_o, rtol=0, atol=1e-10), np.abs(chi_g - chi_o).max()
    Cg = correlations(b, p.sector, psi)
    e = sum(J * Cg[i, j] for (i, j), J in zip(p.terms.bonds, p.terms.J)) + float(np.dot(p.terms.Jchi, chi_g))
    assert e == pytest.approx(vals[0], abs=1e-8)
