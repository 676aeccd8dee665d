"""Pins of the CPU oracle against closed forms, the thesis's worked examples,
invariants and brute force (no GPU).

Each test names the passage or the mathematics it checks.  A plausible slip in
the oracle (a dropped term, a wrong sign, a transposed operand, chi instead of
conj(chi), a wrong norm) breaks at least one of them.
"""
import json
import os
from math import comb, sqrt

import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Problem, Sector, Terms
from edinputs.vectors import splitmix64, state_vector

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _chain6_sector(site_positions):
    """Six-site ring, translations T_n: x -> x+n, sites numbered by the given positions."""
    pos = list(site_positions)
    site_of = {x: i for i, x in enumerate(pos)}
    perm = np.array([[site_of[(pos[i] + n) % 6] for i in range(6)] for n in range(6)], dtype=np.int32)
    return Sector(6, 3, perm, np.zeros(6, np.uint8), np.ones(6, complex), 1)


def _bits(s):
    return int(s, 2)


# ---------------------------------------------------------------- local operators
def test_two_site_singlet_triplet():
    """Eq. twositeheisenbergeigenstates: singlet -3/4, triplet +1/4."""
    B = oracle.bond_matrix()
    w = np.linalg.eigvalsh(B)
    assert np.allclose(w, [-0.75, 0.25, 0.25, 0.25], atol=1e-14)
    singlet = np.zeros(4)
    singlet[0b10] = 1 / sqrt(2)   # |up down>
    singlet[0b01] = -1 / sqrt(2)  # |down up>
    assert np.allclose(B @ singlet, -0.75 * singlet)
    for v in (0b11, 0b00):  # |up up>, |down down>
        e = np.zeros(4)
        e[v] = 1
        assert np.allclose(B @ e, 0.25 * e)


def test_exchange_matrix_element_13_to_11():
    """Eq. exchangeapplyspin / exchangespinmatelement: <11|S_2.S_3|13> = 1/2 (sites 2,3 of four)."""
    sec = Sector(4, 3, np.arange(4, dtype=np.int32)[None], np.zeros(1, np.uint8), np.ones(1, complex), 1)
    terms = Terms(np.array([[1, 2]], np.int32), np.array([1.0]), np.zeros((0, 3), np.int32), np.zeros(0))
    H, st = oracle.dense_sz(Problem("four", sec, terms))
    idx = {int(s): i for i, s in enumerate(st)}
    assert H[idx[11], idx[13]] == pytest.approx(0.5)
    assert H[idx[13], idx[11]] == pytest.approx(0.5)
    # Ising part on 13 = |up up down up>: sites 2,3 antiparallel -> -1/4
    assert H[idx[13], idx[13]].real == pytest.approx(-0.25)


def test_chirality_single_triangle_spectrum():
    """S_i.(S_j x S_k) on one triangle: eigenvalues 0 (x4) and +-sqrt(3)/4 (x2 each).

    Closed form: the operator vanishes on the spin-3/2 quartet and is
    +-sqrt(3)/4 on the two chiral spin-1/2 doublets."""
    Cm = oracle.chirality_matrix()
    assert np.allclose(Cm, Cm.conj().T)
    w = np.sort(np.linalg.eigvalsh(Cm))
    s = sqrt(3) / 4
    assert np.allclose(w, [-s, -s, 0, 0, 0, 0, s, s], atol=1e-14)


def test_chirality_antisymmetric_and_su2():
    """Swapping two sites reverses the orientation (sign flip); the operator commutes with total S."""
    Cm = oracle.chirality_matrix()
    # swap sites j and k in the local basis
    P = np.zeros((8, 8))
    for a in range(8):
        i, j, k = (a >> 2) & 1, (a >> 1) & 1, a & 1
        P[(i << 2) | (k << 1) | j, a] = 1
    assert np.allclose(P @ Cm @ P.T, -Cm)
    from oracle.ops import SPIN, _kron
    I = np.eye(2)
    for S in SPIN:
        Stot = _kron(S, I, I) + _kron(I, S, I) + _kron(I, I, S)
        assert np.allclose(Stot @ Cm, Cm @ Stot, atol=1e-14)


def test_four_site_ring_ground_state():
    """H = (S1+S3).(S2+S4) = [S_tot^2 - S_13^2 - S_24^2]/2 has E0 = -2."""
    p = C.chain(4, 1.0)
    H, _ = oracle.dense_sz(p)
    assert np.linalg.eigvalsh(H)[0] == pytest.approx(-2.0, abs=1e-13)


def test_majumdar_ghosh_point():
    """J2 = J1/2 ring of even length: E0 = -3N/8, twofold degenerate (dimer product states)."""
    p = C.chain(12, 1.0, 0.5)
    H, _ = oracle.dense_sz(p)
    w = np.linalg.eigvalsh(H)
    assert w[0] == pytest.approx(-4.5, abs=1e-12)
    assert w[1] == pytest.approx(-4.5, abs=1e-12)
    assert w[2] > -4.5 + 1e-3


def test_complete_graph_spectrum():
    """All-to-all J=1 on N sites: H = [S_tot^2 - 3N/4]/2, spectrum from total spin only."""
    N = 6
    bonds = np.array([(i, j) for i in range(N) for j in range(i + 1, N)], np.int32)
    sec = Sector(N, 3, np.arange(N, dtype=np.int32)[None], np.zeros(1, np.uint8), np.ones(1, complex), 1)
    terms = Terms(bonds, np.ones(len(bonds)), np.zeros((0, 3), np.int32), np.zeros(0))
    H, st = oracle.dense_sz(Problem("K6", sec, terms))
    w = np.sort(np.linalg.eigvalsh(H))
    # multiplicities of total spin S in Sz=0 for six spins: S=0:5, S=1:9, S=2:5, S=3:1
    expect = sorted([0.5 * (S * (S + 1) - 4.5) for S, m in ((0, 5), (1, 9), (2, 5), (3, 1)) for _ in range(m)])
    assert np.allclose(w, expect, atol=1e-12)


# ---------------------------------------------------------------- worked examples
@pytest.mark.parametrize("which", ["two_sublattice", "three_sublattice"])
def test_worked_example_representative(which):
    """Both sublattice-coding examples: representative and minimising translation."""
    ex = json.load(open(os.path.join(GOLD, "worked_examples.json")))[which]
    sec = _chain6_sector(ex["site_positions"])
    r, g, nstab, stabsum = oracle.rep(sec, _bits(ex["state"]))
    assert r == _bits(ex["rep"])
    assert f"T{g}" == ex["g"]
    assert nstab == 1
    if which == "three_sublattice":
        assert oracle.apply(sec, 2, _bits(ex["state"])) == _bits(ex["T2_image"])
        assert oracle.apply(sec, 5, _bits(ex["state"])) == _bits(ex["T5_image"])


def test_group_action_is_active_translation():
    """T1 on the real-space chain moves the spin at x to x+1 (both examples imply this)."""
    sec = _chain6_sector(range(6))
    assert oracle.apply(sec, 1, 0b100000) == 0b010000
    assert oracle.apply(sec, 1, 0b000001) == 0b100000


# ---------------------------------------------------------------- basis and dimensions
def test_dimensions_character_formula_vs_enumeration():
    """Basis size from brute-force enumeration equals the character formula (Eq. characterformula)."""
    probs = [C.chain(12, translations=True, k=k) for k in range(4)]
    probs += [C.chain(12, translations=True, reflection=True, spinflip=s) for s in (1, -1)]
    probs += [C.square([[4, 0], [0, 4]], 1.0, 0.5, irrep=ir, spinflip=1) for ir in ("A1", "A2", "B1", "B2")]
    probs += [C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep=ir) for ir in ("A", "B", "E1", "E2")]
    probs += [C.triangular([[2, 2], [-2, 4]], 1.0, 0.2, irrep=ir) for ir in ("A1", "B2")]
    for p in probs:
        reps, stab = oracle.basis(p.sector)
        assert len(reps) == oracle.sector_dim_formula(p.sector), p.name
        assert np.all(np.diff(reps.astype(np.int64)) > 0)
        assert np.all(p.sector.n_sym % stab == 0)


def test_abelian_sectors_partition_the_sz_space():
    """For T_N x Z2 (abelian) the sector dimensions over all 1-D irreps sum to C(N, N/2)."""
    N = 12
    tot = 0
    for k in range(N):
        for s in (1, -1):
            tot += len(oracle.basis(C.chain(N, translations=True, k=k, spinflip=s).sector)[0])
    assert tot == comb(N, N // 2)


# ---------------------------------------------------------------- symmetric-basis matrix
PROJECTION_CASES = [
    lambda: C.chain(10, 1.0, 0.3, translations=True, reflection=True, spinflip=-1, irrep="A2"),
    lambda: C.chain(12, 1.0, 0.0, translations=True, k=5),
    lambda: C.chain(12, 1.0, 0.0, translations=True, k=3, spinflip=1),
    lambda: C.square([[4, 0], [0, 4]], 1.0, 0.5, irrep="B1", spinflip=-1, n_up=8),
    lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
    lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.0, -0.7, irrep="B", spinflip=1),
    lambda: C.triangular([[2, 2], [-2, 4]], 1.0, 0.2, irrep="A1", n_up=5),
]


@pytest.mark.parametrize("case", range(len(PROJECTION_CASES)))
def test_csr_equals_projected_dense(case):
    """O3: V^H H V with V the explicit projections sum_g conj(chi(g)) g|sigma> equals the oracle matrix.

    This pins the conj(chi(g_tau)) reading of Eq. matrixelementrepresentatives,
    the norm ratio sqrt(|Stab_tau|/|Stab_sigma|), and the choice of basis."""
    p = PROJECTION_CASES[case]()
    if p.sector.n_sites > 16:
        pytest.skip("too large for dense projection")
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab).toarray()
    Hd, st = oracle.dense_sz(p)
    V, kept = oracle.projector_matrix(p.sector, st)
    assert np.array_equal(np.array(kept, dtype=np.uint64), reps)
    assert np.abs(V.conj().T @ Hd @ V - H).max() < 1e-12
    assert np.abs(H - H.conj().T).max() < 1e-13


def test_sector_spectra_reproduce_full_spectrum():
    """Union of all momentum-sector spectra equals the unsymmetrized fixed-Sz spectrum."""
    N = 10
    p0 = C.chain(N, 1.0, 0.35)
    Hd, _ = oracle.dense_sz(p0)
    full = np.sort(np.linalg.eigvalsh(Hd))
    parts = []
    for k in range(N):
        p = C.chain(N, 1.0, 0.35, translations=True, k=k)
        parts.append(np.linalg.eigvalsh(oracle.csr(p).toarray()))
    assert np.allclose(np.sort(np.concatenate(parts)), full, atol=1e-12)


def test_su2_multiplets_and_marshall():
    """Every Sz=1 level appears at Sz=0 (SU(2)); bipartite J2=0 ground state is a singlet (Marshall)."""
    p0 = C.square([[4, 0], [0, 4]], 1.0, 0.0, point="none", translations=True, k=(0, 0), irrep="A")
    p1 = C.square([[4, 0], [0, 4]], 1.0, 0.0, point="none", translations=True, k=(0, 0), irrep="A", n_up=9)
    e0 = oracle.lowest_eigs(oracle.csr(p0), 6)
    e1 = oracle.lowest_eigs(oracle.csr(p1), 4)
    for e in e1:
        assert np.min(np.abs(e0 - e)) < 1e-9 or e > e0[-1]
    assert e0[0] < e1[0] - 1e-3


def test_chirality_sign_reversal_keeps_spectrum():
    """Jchi -> -Jchi conjugates H (time reversal); the spectrum of the Gamma sector is unchanged."""
    a = np.linalg.eigvalsh(oracle.csr(C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.4)).toarray())
    b = np.linalg.eigvalsh(oracle.csr(C.kagome([[2, 0], [0, 2]], 1.0, 0.2, -0.4)).toarray())
    assert np.allclose(a, b, atol=1e-12)


# ---------------------------------------------------------------- matrix-free rows, eigensolver
@pytest.mark.parametrize("cplx", [False, True])
def test_rows_equal_csr_times_x(cplx):
    p = C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1") if cplx else C.chain(14, 1.0, 0.4, translations=True,
                                                                                   reflection=True, spinflip=1)
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    x = state_vector(7, reps, complex_=True)
    if not cplx:
        x = x.real
    y = H @ x
    ysample = oracle.rows(p, reps, 7, cplx)
    assert np.abs(ysample - y).max() < 1e-12


def test_arpack_matches_dense():
    p = C.chain(16, 1.0, 0.2, translations=True, k=0)
    H = oracle.csr(p)
    assert H.shape[0] > 800
    dense = np.linalg.eigvalsh(H.toarray())[:3]
    import scipy.sparse.linalg as sla
    w = np.sort(sla.eigsh(H, k=3, which="SA", tol=1e-14, return_eigenvectors=False))
    assert np.allclose(w, dense, atol=1e-11)


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0: first outputs as published with the generator."""
    z = np.array([0, 0x9E3779B97F4A7C15, 2 * 0x9E3779B97F4A7C15 % (1 << 64)], dtype=np.uint64)
    out = splitmix64(z)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4
    assert int(out[2]) == 0x06C45D188009454F
