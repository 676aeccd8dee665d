"""Shared-memory staging plans and launch sizes.

An H.x block keeps as many table sections in shared memory as the share of
the SM left by its resident blocks allows and reads the others from global
memory; tables larger than any SM (blocks of 16 sites) are read from global
memory by every kernel.  None of this may change a result: every row is
computed by one thread in a fixed order, so y must be bit-identical for
every resident-block count, and equal to the oracle within the FP64 bound.
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.vectors import state_vector

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


def _bound(H, x):
    return 64 * EPS64 * (abs(H) @ np.abs(x)) + 1e-300


def _apply(P, h, X, tdt):
    import torch
    x = torch.tensor(X, dtype=tdt, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_sixteen_site_block_tables_in_global_memory(P):
    """One block of 16 sites: Rep/Sym/SymmetryAction tables of several hundred KB, read from
    global memory by the basis build, the representative kernel and H.x."""
    import torch
    p = C.square([[4, 0], [0, 4]], 1.0, 0.5, n_sublat=1, max_table_bytes=1 << 30)
    assert p.sector.n_sublat == 1
    reps, stab = oracle.basis(p.sector)
    b = P.Basis(p.sector)
    greps, gstab = b.export()
    assert np.array_equal(greps, reps) and np.array_equal(gstab.astype(np.int32), stab)
    rng = np.random.default_rng(3)
    states = rng.integers(0, 1 << 16, size=300, dtype=np.uint64)
    rep, g, ns, cp = P.representatives(p.sector, states)
    for i, st in enumerate(states):
        r0, g0, n0, ssum = oracle.rep(p.sector, int(st))
        assert int(rep[i]) == r0 and ns[i] == n0 and bool(cp[i]) == (abs(ssum) > 1e-9)
    H = oracle.csr(p, reps, stab)
    h = P.Hamiltonian(b, p.terms)
    X = state_vector(4, reps)
    Y = _apply(P, h, X, torch.float64)
    assert np.all(np.abs(Y - H @ X) <= _bound(H, X))


def test_eight_site_blocks_square32(P):
    """square32 with 4 blocks of 8 sites (its whole 53 KB image fits shared memory; the
    default uses 2 blocks of 16 sites): sampled rows against the oracle."""
    import torch
    p = C.square32(n_sublat=4)
    assert p.sector.n_sublat == 4
    b = P.Basis(p.sector)
    assert b.dim == oracle.sector_dim_formula(p.sector)
    reps, _ = b.export()
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(b.dim, size=300, replace=False))
    h = P.Hamiltonian(b, p.terms)
    X = state_vector(9, reps)
    Y = _apply(P, h, X, torch.float64)
    yo = oracle.rows(p, reps[idx], 9, False)
    R = np.sum(np.abs(p.terms.J)) * (0.25 + 0.5 * np.sqrt(p.sector.n_sym))
    assert np.all(np.abs(Y[idx] - yo.real) <= 64 * EPS64 * R)


@pytest.mark.parametrize("which", ["real", "complex"])
def test_results_identical_for_every_block_count(P, which):
    """A 24-site triangular sector (98 KB of tables): at 3 or more resident blocks the Rep
    and Sym sections stay in global memory, at 1-2 they are staged.  Bit-identical y for every
    count, the autotuner's choice included, and oracle parity."""
    import torch
    secs = C.triangular24_sectors()
    real = [q for q in secs if q.sector.is_real and q.terms.is_real]
    cplx = [q for q in secs if not q.sector.is_real]
    p = real[0] if which == "real" else cplx[0]
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    is_c = which == "complex"
    tdt = torch.complex128 if is_c else torch.float64
    edt = P.ED_C128 if is_c else P.ED_F64
    X = state_vector(21, reps, complex_=is_c)
    top = 1
    while True:
        try:
            h.set_blocks(edt, 1, top + 1)
        except P.EdError:
            break
        top += 1
    assert top == (2 if is_c else 6)          # 32-bit states: 6 real, 2 complex FP64
    outs = []
    for nb in range(1, top + 1):
        h.set_blocks(edt, 1, nb)
        outs.append(_apply(P, h, X, tdt))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert np.all(np.abs(outs[0] - H @ X) <= _bound(H, X))
    x = torch.tensor(X, dtype=tdt, device="cuda")
    y = torch.empty_like(x)
    nb = h.autotune(x, y)
    assert 1 <= nb <= top
    assert np.array_equal(_apply(P, h, X, tdt), outs[0])
    h.set_blocks(edt, 1, 0)
    assert np.array_equal(_apply(P, h, X, tdt), outs[0])
    with pytest.raises(P.EdError) as e:
        h.set_blocks(edt, 1, top + 1)
    assert e.value.name == "ED_ERR_ARG"
