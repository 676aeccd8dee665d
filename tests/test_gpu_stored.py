"""Stored structure of H (ed_hamiltonian_store): parity with the oracle and
with the matrix-free kernel.

The stored path holds the same elements in the same order as the matrix-free
kernel; with one column segment and real vectors it must give bit-identical
y.  With several segments (forced small here so that small sectors have many)
the summation order changes, and y is checked against the oracle's sparse
matrix with the bound of test_gpu_parity: 64 eps (|H| |x|)_i (FP32 vectors:
eps_32, times 4 for the rounding of x).  At full size (square32, kagome36,
square40) y is compared with the matrix-free kernel over the whole vector and
with the oracle's matrix-free rows on sampled representatives.
"""
import math

import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.vectors import state_vector

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


SMALL = {
    "chain12_T_k5": lambda: C.chain(12, 1.0, 0.3, translations=True, k=5),
    "chain14_TRZ2_odd": lambda: C.chain(14, 1.0, 0.4, translations=True, reflection=True, spinflip=-1, irrep="A2"),
    "chain16_nosym": lambda: C.chain16(),
    "chain13_nup5": lambda: C.chain(13, 1.0, 0.2, translations=True, k=2, n_up=5),
    "square16_B1_odd": lambda: C.square([[4, 0], [0, 4]], 1.0, 0.5, irrep="B1", spinflip=-1),
    "square20_n1": lambda: C.square([[4, 2], [-2, 4]], 1.0, 0.5, spinflip=1, irrep="A", point="rot", n_sublat=4),
    "kagome12_E1": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
    "kagome18_A": lambda: C.kagome([[3, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="A", point="none"),
    "triangular12_E": lambda: C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, k=(4 * np.pi / 3, 0), irrep="A",
                                           point="none"),
    "chain34_nup3": lambda: C.chain(34, 1.0, 0.3, translations=True, reflection=True, n_up=3),
    "square40_nup3": lambda: C.square([[6, 2], [-2, 6]], 1.0, 0.55, n_up=3, irrep="A"),
    "kagome36_nup3_k": lambda: C.kagome([[2, 2], [-2, 4]], 1.0, 0.2, 0.3, n_up=3, irrep="E1"),
    "triangular18_Gamma": lambda: C.triangular([[3, 3], [-3, 3]], 1.0, 0.125, irrep="A1", spinflip=1,
                                               max_table_bytes=160 * 1024),
}

_cache = {}


def _oracle(name):
    if name not in _cache:
        p = SMALL[name]()
        reps, stab = oracle.basis(p.sector)
        H = oracle.csr(p, reps, stab)
        _cache[name] = (p, reps, stab, H)
    return _cache[name]


def _bound(H, x, eps):
    return 64 * eps * (abs(H) @ np.abs(x)) + 1e-300


def _many_segments(D):
    """Segment bits giving about 8 segments (at least 32 rows each)."""
    return max(5, int(math.ceil(math.log2(max(D, 2) / 8))))


def _vectors(reps, cplx, nvec, seed):
    return np.stack([state_vector(seed + v, reps, complex_=cplx) for v in range(nvec)])


@pytest.mark.parametrize("name", sorted(SMALL))
def test_stored_one_segment_equals_matrix_free(P, name):
    """One segment: FP64/complex-FP64 y equal to the matrix-free kernel's (bit for bit for real
    vectors) and within the bound of the oracle's matrix; the counters agree."""
    import torch
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    tdt = torch.complex128 if cplx else torch.float64
    X = _vectors(reps, cplx, 3, 21)
    x = torch.tensor(X, dtype=tdt, device="cuda")
    y_free = torch.empty_like(x)
    h.apply(x, y_free)
    g_free, s_free = h.counters()
    nbytes = h.store()
    info = h.store_info()
    assert info["segments"] == 1 and info["bytes"] == nbytes > 0
    assert info["entries"] == g_free
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    assert h.counters() == (g_free, s_free)
    if not cplx:
        assert torch.equal(y, y_free)
    Y = y.cpu().numpy()
    for v in range(3):
        assert np.all(np.abs(Y[v] - H @ X[v]) <= _bound(H, X[v], EPS64)), (name, v)
    h.store_free()
    assert h.store_info()["segments"] == 0
    y2 = torch.empty_like(x)
    h.apply(x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y2, y_free)


@pytest.mark.parametrize("name", sorted(SMALL))
def test_stored_many_segments_vs_oracle(P, name):
    """About 8 column segments (one pass each, partial sums carried in y): FP64 and FP32 vectors
    against the oracle's matrix, 1 and 5 vectors."""
    import torch
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    h.store(seg_log2=_many_segments(b.dim))
    info = h.store_info()
    assert info["segments"] == -(-b.dim // (1 << _many_segments(b.dim)))
    for nvec in (1, 5):
        X = _vectors(reps, cplx, nvec, 40 + nvec)
        for single in (False, True):
            if single:
                Xd = X.astype(np.complex64 if cplx else np.float32)
                tdt = torch.complex64 if cplx else torch.float32
                eps, fac = EPS32, 4
            else:
                Xd = X
                tdt = torch.complex128 if cplx else torch.float64
                eps, fac = EPS64, 1
            x = torch.tensor(Xd if nvec > 1 else Xd[0], dtype=tdt, device="cuda")
            y = torch.empty_like(x)
            h.apply(x, y)
            torch.cuda.synchronize()
            Y = y.cpu().numpy().reshape(nvec, -1).astype(np.complex128)
            for v in range(nvec):
                xv = Xd[v].astype(np.complex128)
                err = np.abs(Y[v] - H @ xv)
                assert np.all(err <= _bound(H, xv, eps) * fac), (name, nvec, single, v, err.max())


# Complex vectors on Hamiltonians whose stored coefficients are each real or purely
# imaginary (the two-multiply-add path of the pass kernel): a real Hamiltonian with complex
# vectors (all codes real), and a chirality-only kagome model at Gamma (all off-diagonal
# codes imaginary).  kagome12 with J1 and J_chi together has general complex codes.
AXIS = {
    "chain14_TRZ2_odd": lambda: C.chain(14, 1.0, 0.4, translations=True, reflection=True, spinflip=-1, irrep="A2"),
    "kagome12_chirality_only": lambda: C.kagome([[2, 0], [0, 2]], 0.0, 0.0, 0.3, irrep="A", point="none"),
    "kagome12_general": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.0, 0.3, irrep="A", point="none"),
}


@pytest.mark.parametrize("name", sorted(AXIS))
def test_stored_complex_vectors_axis_codes(P, name):
    """Complex FP64 and FP32 vectors, one and about eight segments, 1 and 5 vectors: y
    against the oracle's matrix within the bound of the other stored tests."""
    import torch
    p = AXIS[name]()
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    assert h.is_real == (name == "chain14_TRZ2_odd")
    for seg in (0, _many_segments(b.dim)):
        for single in (False, True):
            tdt = torch.complex64 if single else torch.complex128
            h.store(P.ED_C64 if single else P.ED_C128, seg_log2=seg)
            for nvec in (1, 5):
                X = _vectors(reps, True, nvec, 60 + nvec)
                Xd = X.astype(np.complex64) if single else X
                eps, fac = (EPS32, 4) if single else (EPS64, 1)
                x = torch.tensor(Xd if nvec > 1 else Xd[0], dtype=tdt, device="cuda")
                y = torch.empty_like(x)
                h.apply(x, y)
                torch.cuda.synchronize()
                Y = y.cpu().numpy().reshape(nvec, -1).astype(np.complex128)
                for v in range(nvec):
                    xv = Xd[v].astype(np.complex128)
                    err = np.abs(Y[v] - H @ xv)
                    assert np.all(err <= _bound(H, xv, eps) * fac), (name, seg, single, nvec, v, err.max())
            h.store_free()


LANES_CASES = ["chain16_nosym", "square16_B1_odd", "kagome12_E1", "kagome18_A", "square40_nup3", "chain14_TRZ2_odd"]


@pytest.mark.parametrize("name", LANES_CASES)
def test_stored_lanes_per_row_vs_oracle(P, name):
    """One-vector pass with 2, 4 and 8 lanes per row (ed_hamiltonian_store_set_lanes), one and
    about eight segments, FP64 and FP32 kinds (complex vectors on the real chain too): y
    against the oracle's matrix within the bound of the other stored tests; several vectors
    keep one lane per row; the schedule query reports the setting."""
    import torch
    if name in SMALL:
        p, reps, stab, H = _oracle(name)
    else:
        p = AXIS[name]()
        reps, stab = oracle.basis(p.sector)
        H = oracle.csr(p, reps, stab)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real or name == "chain14_TRZ2_odd"
    kinds = [(torch.complex128, P.ED_C128, EPS64, 1), (torch.complex64, P.ED_C64, EPS32, 4)] if cplx else \
        [(torch.float64, P.ED_F64, EPS64, 1), (torch.float32, P.ED_F32, EPS32, 4)]
    X = _vectors(reps, cplx, 3, 77)
    for seg in (0, _many_segments(b.dim)):
        for tdt, edt, eps, fac in kinds:
            h.store(edt, seg_log2=seg)
            assert h.store_schedule()["lanes_per_row"] == 1
            npdt = {torch.complex64: np.complex64, torch.float32: np.float32}.get(tdt)
            Xd = X.astype(npdt) if npdt else X
            for lanes in (2, 4, 8):
                h.store_set_lanes(lanes)
                assert h.store_schedule()["lanes_per_row"] == lanes
                x = torch.tensor(Xd, dtype=tdt, device="cuda")
                y = torch.empty_like(x)
                for v in range(3):  # one vector at a time: the lanes schedule
                    h.apply(x[v], y[v])
                y3 = torch.empty_like(x)
                h.apply(x, y3)  # several vectors: one lane per row
                torch.cuda.synchronize()
                for yy in (y, y3):
                    Y = yy.cpu().numpy().astype(np.complex128)
                    for v in range(3):
                        xv = Xd[v].astype(np.complex128)
                        err = np.abs(Y[v] - H @ xv)
                        assert np.all(err <= _bound(H, xv, eps) * fac), (name, seg, edt, lanes, v, err.max())
            h.store_free()
            assert h.store_schedule() == dict(seg_log2=0, lanes_per_row=0)


def test_stored_lanes_errors(P):
    """ed_hamiltonian_store_set_lanes: ED_ERR_ARG without a stored structure and for counts
    other than 1, 2, 4, 8."""
    p, reps, stab, H = _oracle("chain16_nosym")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    with pytest.raises(P.EdError) as e:
        h.store_set_lanes(2)
    assert e.value.name == "ED_ERR_ARG"
    h.store()
    for bad in (0, 3, 16, -1):
        with pytest.raises(P.EdError) as e:
            h.store_set_lanes(bad)
        assert e.value.name == "ED_ERR_ARG"
    assert h.store_schedule()["lanes_per_row"] == 1


def test_stored_fp32_one_segment_bitexact(P):
    """Real FP32 vectors with one segment: bit-identical to the matrix-free kernel."""
    import torch
    for name in ("square16_B1_odd", "chain16_nosym", "square40_nup3"):
        p, reps, stab, H = _oracle(name)
        b = P.Basis(p.sector)
        h = P.Hamiltonian(b, p.terms)
        x = torch.tensor(state_vector(7, reps), dtype=torch.float32, device="cuda")
        y0, y1 = torch.empty_like(x), torch.empty_like(x)
        h.apply(x, y0)
        h.store(P.ED_F32)
        h.apply(x, y1)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1), name


@pytest.mark.parametrize("name", ["chain14_TRZ2_odd", "kagome12_E1", "square20_n1", "triangular18_Gamma"])
def test_stored_lanczos_vs_oracle(P, name):
    """ed_lanczos on the stored structure (several segments): lowest eigenvalues within 1e-10
    relative of the oracle's dense spectrum; FP32 vectors with refinement likewise."""
    p, reps, stab, H = _oracle(name)
    ref = np.linalg.eigvalsh(H.toarray())[:2]
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    h.store(seg_log2=_many_segments(b.dim))
    ev, rep = h.lanczos(n_eig=2, tol=1e-12, max_iter=300)
    assert np.all(np.abs(ev - ref) <= 1e-10 * np.abs(ref)), (ev, ref)
    dt = P.ED_F32 if h.is_real else P.ED_C64
    ev, rep = h.lanczos(n_eig=1, tol=1e-10, max_iter=300, dtype=dt, refine=True)
    assert abs(ev[0] - ref[0]) <= 1e-10 * abs(ref[0]), (ev, ref)


def test_stored_limit_refused(P):
    """A byte limit below the structure's size keeps nothing (ED_ERR_NOMEM) and ed_apply stays
    matrix-free and correct."""
    import torch
    p, reps, stab, H = _oracle("square16_B1_odd")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    with pytest.raises(P.EdError) as e:
        h.store(max_bytes=1000)
    assert e.value.name == "ED_ERR_NOMEM"
    assert h.store_info() == dict(entries=0, segments=0, codes=0, bytes=0)
    X = state_vector(3, reps)
    x = torch.tensor(X, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    assert np.all(np.abs(y.cpu().numpy() - H @ X) <= _bound(H, X, EPS64))
    with pytest.raises(P.EdError) as e:
        h.store(seg_log2=3)
    assert e.value.name == "ED_ERR_ARG"


def test_stored_autotune(P):
    """The autotuner keeps one of its segment candidates (half, one and two times the
    default of 2^24 complex-FP32 elements; one segment for this small sector) and one of
    the lanes-per-row schedules, and the kept structure gives the oracle's H x."""
    import torch
    p, reps, stab, H = _oracle("kagome18_A")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    seg, nbytes = h.store_autotune(P.ED_C64)
    assert seg in (23, 24, 25) and nbytes == h.store_info()["bytes"] > 0
    sch = h.store_schedule()
    assert sch["seg_log2"] == seg and sch["lanes_per_row"] in (1, 2, 4, 8)
    X = state_vector(5, reps, complex_=True)
    x = torch.tensor(X, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    assert np.all(np.abs(y.cpu().numpy() - H @ X) <= _bound(H, X, EPS64))


def test_stored_edge_sectors(P):
    """One-state sectors and a Hamiltonian without off-diagonal terms."""
    import torch
    for n_up in (0, 10):
        p = C.chain(10, 1.0, 0.3, translations=True, n_up=n_up)
        b = P.Basis(p.sector)
        h = P.Hamiltonian(b, p.terms)
        h.store()
        x = torch.ones(1, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        h.apply(x, y)
        torch.cuda.synchronize()
        assert y.item() == pytest.approx(10 * 0.25 + 10 * 0.3 * 0.25)
    p = C.chain(12, 0.0, 0.0, translations=True)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    h.store(seg_log2=5)
    x = torch.ones(b.dim, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, 7.0)
    h.apply(x, y)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0


# ------------------------------------------------------------------ full-size workloads
def _random_reps(problem, n, seed):
    rng = np.random.default_rng(seed)
    s = problem.sector
    out = []
    while len(out) < n:
        bits = np.zeros(s.n_sites, dtype=np.int64)
        bits[rng.choice(s.n_sites, s.n_up, replace=False)] = 1
        r, g, ns, ssum = oracle.rep(s, int("".join(map(str, bits)), 2))
        if abs(ssum) > 1e-9:
            out.append(r)
    return np.array(sorted(set(out)), dtype=np.uint64)


def _row_bound(problem, eps):
    G = problem.sector.n_sym
    R = np.sum(np.abs(problem.terms.J)) * (0.25 + 0.5 * np.sqrt(G))
    if len(problem.terms.tris):
        R += np.sum(np.abs(problem.terms.Jchi)) * 3 * 0.25 * np.sqrt(G)
    return 64 * eps * R


def _full_size(P, problem, dtypes, n_sample, seed, bitexact, lanes=1):
    import torch
    b = P.Basis(problem.sector)
    reps, _ = b.export()
    drawn = _random_reps(problem, n_sample, seed)
    pos = np.searchsorted(reps, drawn)
    assert np.array_equal(reps[pos], drawn)
    h = P.Hamiltonian(b, problem.terms)
    cplx = not h.is_real
    X = state_vector(9, reps, complex_=cplx)
    for tdt, edt in dtypes:
        x = torch.tensor(X, device="cuda").to(tdt)
        y_free = torch.empty_like(x)
        h.apply(x, y_free)
        g_free, _ = h.counters()
        h.store(edt)
        if lanes > 1:
            h.store_set_lanes(lanes)
        info = h.store_info()
        assert info["entries"] == g_free
        y = torch.empty_like(x)
        h.apply(x, y)
        torch.cuda.synchronize()
        single = tdt in (torch.float32, torch.complex64)
        eps = EPS32 if single else EPS64
        if bitexact and info["segments"] == 1 and not cplx and lanes == 1:
            assert torch.equal(y, y_free)
        else:
            d = (y - y_free).abs().max().item()
            assert d <= 2 * _row_bound(problem, eps) * (4 if single else 1), d
        yg = y[torch.tensor(pos.astype(np.int64), device="cuda")].cpu().numpy().astype(np.complex128)
        yo = oracle.rows(problem, drawn, 9, cplx)
        err = np.abs(yg - yo)
        assert np.all(err <= _row_bound(problem, eps) * (4 if single else 1)), err.max()
        h.store_free()
        del x, y, y_free
        torch.cuda.empty_cache()


def test_stored_square32_bench_config(P):
    """The 32-site workload (one segment): FP64 and FP32 bit-identical to matrix-free over all
    2.36e6 rows, and equal to the oracle's rows on sampled representatives."""
    import torch
    _full_size(P, C.square32(), [(torch.float64, P.ED_F64), (torch.float32, P.ED_F32)], 600, 3, True)


def test_stored_square32_lanes(P):
    """The 32-site workload with two lanes per row (the schedule the autotuner picks there):
    FP64 and FP32 within the summation-order bound of the matrix-free kernel over all rows
    and of the oracle's rows on sampled representatives."""
    import torch
    _full_size(P, C.square32(), [(torch.float64, P.ED_F64), (torch.float32, P.ED_F32)], 400, 5, True, lanes=2)


def test_stored_kagome36(P):
    """Complex chiral Hamiltonian, 64-bit words, several segments (complex FP32 and FP64)."""
    import torch
    _full_size(P, C.kagome36(), [(torch.complex64, P.ED_C64), (torch.complex128, P.ED_C128)], 300, 5, False)


def test_stored_square40(P):
    """The 40-site workload (D = 4.3e8, tens of segments), FP32 and FP64 vectors."""
    import torch
    _full_size(P, C.square40(), [(torch.float32, P.ED_F32), (torch.float64, P.ED_F64)], 200, 7, False)
