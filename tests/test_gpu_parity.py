"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances.  FP64: each output y_i is a sum of at most ~2 n_terms products,
so |y_gpu - y_oracle|_i <= 64 eps_64 (|H| |x|)_i with |H| the entrywise
absolute matrix (a standard bound for a dot product of that length, with a
safety factor).  FP32 vectors: the same with eps_32 plus the rounding of x to
FP32.  Basis, representatives, indices and stabilizer orders: bit-exact.
Eigenvalues (FP64): 1e-10 relative.
"""
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
    "chain12_T_k0": lambda: C.chain(12, 1.0, 0.3, translations=True),
    "chain12_T_k5": lambda: C.chain(12, 1.0, 0.3, translations=True, k=5),
    "chain14_TRZ2_odd": lambda: C.chain(14, 1.0, 0.4, translations=True, reflection=True, spinflip=-1, irrep="A2"),
    "chain16_nosym": lambda: C.chain16(),
    "chain13_nup5": lambda: C.chain(13, 1.0, 0.2, translations=True, k=2, n_up=5),
    "square16_B1_odd": lambda: C.square([[4, 0], [0, 4]], 1.0, 0.5, irrep="B1", spinflip=-1),
    "square16_M_A2": lambda: C.square([[4, 0], [0, 4]], 1.0, 0.5, k=(np.pi, np.pi), irrep="A2"),
    "square16_X": lambda: C.square([[4, 0], [0, 4]], 1.0, 0.3, k=(np.pi, 0), irrep="A", point="none"),
    "square20_n1": lambda: C.square([[4, 2], [-2, 4]], 1.0, 0.5, spinflip=1, irrep="A", point="rot", n_sublat=4),
    "kagome12_E1": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
    "kagome12_B_even": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.0, -0.7, irrep="B", spinflip=1),
    "kagome18_A": lambda: C.kagome([[3, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="A", point="none"),
    "triangular12_A1": lambda: C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, n_up=5),
    "triangular12_E": lambda: C.triangular([[2, 2], [-2, 4]], 1.0, 0.125, k=(4 * np.pi / 3, 0), irrep="A",
                                           point="none"),
    # 64-bit state words (N > 32) on sparse sectors the oracle enumerates quickly
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


@pytest.mark.parametrize("name", sorted(SMALL))
def test_basis_bitexact(P, name):
    p, reps, stab, _ = _oracle(name)
    b = P.Basis(p.sector)
    assert b.dim == len(reps) == oracle.sector_dim_formula(p.sector)
    greps, gstab = b.export()
    assert np.array_equal(greps, reps)
    assert np.array_equal(gstab.astype(np.int32), stab)


@pytest.mark.parametrize("name", sorted(SMALL))
def test_representatives_vs_oracle(P, name):
    """Alg. 2 on the device (ed_representatives) against the oracle's brute-force orbit minimum,
    on random states of every popcount: representative bit-exact, |Stab| exact, membership exact,
    and the returned element maps the state onto its representative."""
    p = SMALL[name]()
    s = p.sector
    rng = np.random.default_rng(5)
    N = s.n_sites
    states = rng.integers(0, 1 << min(N, 62), size=400, dtype=np.uint64)
    if N > 62:
        states |= rng.integers(0, 4, size=400, dtype=np.uint64) << np.uint64(62)
    rep, g, ns, cp = P.representatives(s, states)
    for i, st in enumerate(states):
        r0, g0, n0, ssum = oracle.rep(s, int(st))
        assert int(rep[i]) == r0, (name, int(st))
        assert ns[i] == n0
        assert bool(cp[i]) == (abs(ssum) > 1e-9)
        assert oracle.apply(s, int(g[i]), int(st)) == r0


def _bound(H, x, eps):
    return 64 * eps * (abs(H) @ np.abs(x)) + 1e-300


@pytest.mark.parametrize("name", sorted(SMALL))
def test_hx_fp64_parity(P, name):
    import torch
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    assert cplx == (not (p.sector.is_real and p.terms.is_real))
    nvec = 3
    X = np.stack([state_vector(11 + v, reps, complex_=cplx) for v in range(nvec)])
    tdt = torch.complex128 if cplx else torch.float64
    x = torch.tensor(X, dtype=tdt, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    Y = y.cpu().numpy()
    for v in range(nvec):
        ref = H @ X[v]
        err = np.abs(Y[v] - ref)
        assert np.all(err <= _bound(H, X[v], EPS64)), (name, v, err.max())
    g, skipped = h.counters()
    assert g > 0 or H.nnz == np.count_nonzero(H.diagonal())


@pytest.mark.parametrize("name", ["chain14_TRZ2_odd", "square16_B1_odd", "kagome12_E1", "triangular12_E"])
def test_hx_fp32_parity(P, name):
    import torch
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    X = state_vector(5, reps, complex_=cplx)
    X32 = X.astype(np.complex64 if cplx else np.float32)
    x = torch.tensor(X32, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    ref = H @ X32.astype(np.complex128)
    err = np.abs(y.cpu().numpy().astype(np.complex128) - ref)
    assert np.all(err <= _bound(H, X32, EPS32) * 4), err.max()


def test_fp64_dtype_rejected_for_complex(P):
    import torch
    p, reps, stab, H = _oracle("kagome12_E1")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    x = torch.zeros(b.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(P.EdError) as e:
        h.apply(x, torch.empty_like(x))
    assert e.value.name == "ED_ERR_ARG"


def test_edge_sectors(P):
    import torch
    # fully polarised sectors: one state
    for n_up in (0, 10):
        p = C.chain(10, 1.0, 0.3, translations=True, n_up=n_up)
        b = P.Basis(p.sector)
        assert b.dim == 1
        h = P.Hamiltonian(b, p.terms)
        x = torch.ones(1, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        h.apply(x, y)
        torch.cuda.synchronize()
        assert y.item() == pytest.approx(10 * 0.25 + 10 * 0.3 * 0.25)
    # an empty sector: momentum pi with a single up spin on 10 sites has dimension 1,
    # but the all-down state is invisible at k != 0
    p = C.chain(10, 1.0, 0.0, translations=True, k=3, n_up=0)
    with pytest.raises(P.EdError) as e:
        P.Basis(p.sector)
    assert e.value.name == "ED_ERR_EMPTY_SECTOR"
    # no terms at all: H = 0
    p = C.chain(12, 0.0, 0.0, translations=True)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    x = torch.ones(b.dim, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, 7.0)
    h.apply(x, y)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0


def test_nvec_eight(P):
    import torch
    p, reps, stab, H = _oracle("square16_B1_odd")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    X = np.stack([state_vector(100 + v, reps) for v in range(8)])
    x = torch.tensor(X, device="cuda")
    y = torch.empty_like(x)
    h.apply(x, y)
    torch.cuda.synchronize()
    for v in range(8):
        assert np.all(np.abs(y[v].cpu().numpy() - H @ X[v]) <= _bound(H, X[v], EPS64))


# ---------------------------------------------------------------- Lanczos
@pytest.mark.parametrize("name", ["chain16_nosym", "square16_B1_odd", "kagome12_E1", "triangular18_Gamma"])
def test_lanczos_fp64(P, name):
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    k = 3
    ev, rep = h.lanczos(n_eig=k, tol=1e-12, max_iter=min(400, b.dim), reorth=True)
    ref = np.linalg.eigvalsh(H.toarray()) if H.shape[0] <= 6000 else oracle.lowest_eigs(H, 8)
    # single-vector Lanczos sees each degenerate level once: compare with distinct levels
    distinct = [ref[0]]
    for e in ref[1:]:
        if e - distinct[-1] > 1e-8:
            distinct.append(e)
    assert rep.converged
    for i in range(min(k, len(distinct))):
        assert abs(ev[i] - distinct[i]) <= 1e-10 * max(1.0, abs(distinct[i])), (i, ev, distinct[:k])


@pytest.mark.parametrize("name", ["square16_B1_odd", "kagome12_E1"])
def test_lanczos_mixed_refined(P, name):
    """FP32/complex-FP32 vectors, FP64 reductions and FP64 Rayleigh-quotient refinement."""
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    dt = P.ED_F32 if h.is_real else P.ED_C64
    ev, rep = h.lanczos(n_eig=1, tol=1e-10, max_iter=300, dtype=dt, reorth=True, refine=True)
    e0 = np.linalg.eigvalsh(H.toarray())[0]
    assert abs(rep.ritz[0] - e0) < 1e-5 * abs(e0)
    assert abs(ev[0] - e0) <= 1e-10 * abs(e0), (ev[0], e0, rep.ritz[0])


def test_lanczos_eigenvectors(P):
    import torch
    p, reps, stab, H = _oracle("chain14_TRZ2_odd")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    ev = torch.zeros((2, b.dim), dtype=torch.float64, device="cuda")
    vals, rep = h.lanczos(n_eig=2, tol=1e-12, max_iter=300, evecs=ev)
    V = ev.cpu().numpy()
    ref = np.linalg.eigvalsh(H.toarray())
    for k in range(2):
        r = H @ V[k] - vals[k] * V[k]
        # eigenvectors are converged to a residual of sqrt(tol) * max(1, |E|)
        assert np.linalg.norm(r) <= 1e-6 * max(1.0, abs(vals[k])) * 1.01
        assert abs(np.linalg.norm(V[k]) - 1) < 1e-10
        assert abs(vals[k] - ref[k]) < 1e-10 * abs(ref[k])
    assert abs(np.vdot(V[0], V[1])) < 1e-8


def _distinct(ref, k):
    out = [ref[0]]
    for e in ref[1:]:
        if e - out[-1] > 1e-8:
            out.append(e)
    return out[:k]


@pytest.mark.parametrize("name", ["chain16_nosym", "kagome12_E1", "triangular18_Gamma"])
def test_lanczos_plain_recursion(P, name):
    """The three-term recursion without reorthogonalisation (the memory regime of the
    largest sectors): long enough for spurious copies of the lowest levels to appear;
    after the Cullum-Willoughby filter the 4 lowest distinct levels match to 1e-10."""
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    k = 4
    ev, rep = h.lanczos(n_eig=k, tol=1e-12, max_iter=min(800, b.dim), reorth=False)
    ref = np.linalg.eigvalsh(H.toarray()) if H.shape[0] <= 6000 else oracle.lowest_eigs(H, 12)
    distinct = _distinct(ref, k)
    assert rep.converged
    for i in range(len(distinct)):
        assert abs(ev[i] - distinct[i]) <= 1e-10 * max(1.0, abs(distinct[i])), (i, ev, distinct)


def test_lanczos_plain_recursion_eigenvectors(P):
    """Ritz vectors of the plain recursion from its second pass (the vectors are
    regenerated from the recorded alpha, beta)."""
    import torch
    p, reps, stab, H = _oracle("chain14_TRZ2_odd")
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    ev = torch.zeros((2, b.dim), dtype=torch.float64, device="cuda")
    vals, rep = h.lanczos(n_eig=2, tol=1e-12, max_iter=300, reorth=False, evecs=ev)
    V = ev.cpu().numpy()
    ref = _distinct(np.linalg.eigvalsh(H.toarray()), 2)
    assert rep.converged
    for k in range(2):
        r = H @ V[k] - vals[k] * V[k]
        assert np.linalg.norm(r) <= 1e-5 * max(1.0, abs(vals[k]))
        assert abs(np.linalg.norm(V[k]) - 1) < 1e-10
        assert abs(vals[k] - ref[k]) < 1e-10 * abs(ref[k])
    assert abs(np.vdot(V[0], V[1])) < 1e-5


@pytest.mark.parametrize("name", ["square16_B1_odd", "kagome12_E1"])
def test_lanczos_mixed_plain_recursion_refined(P, name):
    """FP32 vectors without reorthogonalisation, refined in FP64 from the second-pass
    Ritz vectors: the two lowest levels to 1e-10."""
    p, reps, stab, H = _oracle(name)
    b = P.Basis(p.sector)
    h = P.Hamiltonian(b, p.terms)
    dt = P.ED_F32 if h.is_real else P.ED_C64
    ev, rep = h.lanczos(n_eig=2, tol=1e-10, max_iter=400, dtype=dt, reorth=False, refine=True)
    ref = _distinct(np.linalg.eigvalsh(H.toarray()), 2)
    for i in range(2):
        assert abs(rep.ritz[i] - ref[i]) < 1e-5 * abs(ref[i])
        assert abs(ev[i] - ref[i]) <= 1e-10 * abs(ref[i]), (i, ev[:2], ref, list(rep.ritz[:2]))
