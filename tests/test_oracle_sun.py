"""The SU(N) oracle (d-ary encoding, exchange operators P_ij) pinned to closed
forms, invariants and the spin-1/2 oracle (CPU only)."""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Problem, SectorSUN, Terms

sun = oracle.sun


def _trivial(N, d, counts, bonds, J):
    sec = SectorSUN(N, d, np.asarray(counts, np.int32), np.arange(N, dtype=np.int32)[None, :],
                    np.ones(1, complex), 1)
    return Problem("t", sec, Terms(np.asarray(bonds, np.int32).reshape(-1, 2), np.asarray(J, float),
                                   np.zeros((0, 3), np.int32), np.zeros(0)))


def test_encoding_and_order():
    """Eq. numberforspinconfig with d = 3: (2,0,1) -> 2*9 + 0*3 + 1 = 19; the colourings come
    in increasing order, and the library's packed form (2 bits a site) keeps that order."""
    assert sun.integer([2, 0, 1], 3) == 19 and sun.digits(19, 3, 3) == [2, 0, 1]
    st = sun.states(6, 3, [2, 2, 2])
    assert len(st) == sun.multinomial([2, 2, 2]) == 90
    assert all(a < b for a, b in zip(st, st[1:]))
    pk = [sun.packed(s, 6, 3) for s in st]
    assert all(a < b for a, b in zip(pk, pk[1:]))
    assert sun.packed(19, 3, 3) == 0b100001


def test_two_sites():
    """P_12 on two sites: eigenvalue +1 on symmetric, -1 on antisymmetric colour pairs."""
    H, _ = sun.dense(_trivial(2, 3, [1, 1, 0], [[0, 1]], [1.0]))
    assert np.allclose(np.linalg.eigvalsh(H), [-1, 1])
    H, _ = sun.dense(_trivial(2, 3, [2, 0, 0], [[0, 1]], [1.0]))
    assert np.allclose(H, [[1.0]])


def test_complete_graph_contents():
    """sum_{i<j} P_ij on the complete graph acts on the S_N irrep of Young diagram lambda as
    the sum of its contents (column - row); one site of each colour is the regular
    representation: K3 -> {3, 0 x4, -3}, K4 -> {6, 2 x9, 0 x4, -2 x9, -6}."""
    pairs3 = [[0, 1], [0, 2], [1, 2]]
    H, _ = sun.dense(_trivial(3, 3, [1, 1, 1], pairs3, [1.0] * 3))
    assert np.allclose(np.linalg.eigvalsh(H), [-3, 0, 0, 0, 0, 3])
    pairs4 = [[i, j] for i in range(4) for j in range(i + 1, 4)]
    H, _ = sun.dense(_trivial(4, 4, [1, 1, 1, 1], pairs4, [1.0] * 6))
    ref = [-6] + [-2] * 9 + [0] * 4 + [2] * 9 + [6]
    assert np.allclose(np.linalg.eigvalsh(H), ref)


def test_su2_is_the_spin_model():
    """With two colours, P_ij = 2 S_i.S_j + 1/2: the d-ary (binary) matrix equals twice the
    spin-1/2 oracle's fixed-S^z matrix plus sum_b J_b / 2, element by element (colour 1 is
    spin up in both encodings)."""
    spin = C.chain(8, 1.0, 0.3)
    t = spin.terms
    p2 = _trivial(8, 2, [4, 4], t.bonds, t.J)
    Hs, st_s = oracle.dense_sz(spin)
    Hu, st_u = sun.dense(p2)
    assert [int(a) for a in st_s] == list(st_u)
    assert np.allclose(Hu, 2 * Hs.real + 0.5 * np.sum(t.J) * np.eye(len(st_u)), atol=1e-13)


def test_dimensions_and_momentum_spectra():
    """SU(3) chain of 7 sites, counts (3, 2, 2), translations: the character-formula
    dimensions equal the enumerated ones, add up to the multinomial, and the union of the
    momentum sectors' spectra is the spectrum without symmetry."""
    counts = [3, 2, 2]
    full = None
    dims, spec = 0, []
    for k in range(7):
        p = C.sun_chain(7, 3, counts, 1.0, 0.4, k=k, n_sublat=7)
        reps, stab = sun.basis(p.sector)
        assert len(reps) == sun.sector_dim_formula(p.sector)
        dims += len(reps)
        spec.extend(np.linalg.eigvalsh(sun.csr(p, reps, stab).toarray()))
        if full is None:
            full = np.linalg.eigvalsh(sun.dense(p)[0])
    assert dims == sun.multinomial(counts) == len(full)
    assert np.allclose(np.sort(spec), full, atol=1e-10)


@pytest.mark.parametrize("k", [0, 2])
def test_symmetric_matrix_equals_projection(k):
    """The symmetric-basis matrix (conj(chi) reading, sqrt of stabiliser ratios) equals V^H H V
    for the explicit projections V (k = 0 with the reflection odd; complex characters at k = 2)."""
    p = C.sun_chain(6, 3, [2, 2, 2], 1.0, 0.3, k=k, reflection=True, n_sublat=3, irrep="A2") if k == 0 else \
        C.sun_chain(6, 3, [2, 2, 2], 1.0, 0.3, k=k, n_sublat=3)
    Hd, st = sun.dense(p)
    V, kept = sun.projector_matrix(p.sector, st)
    reps, stab = sun.basis(p.sector)
    assert kept == list(reps)
    assert np.allclose(V.conj().T @ Hd @ V, sun.csr(p, reps, stab).toarray(), atol=1e-12)
