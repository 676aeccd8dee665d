"""SU(N) exchange models (d-ary colours packed in ceil(log2 d) bits per site)
against the SU(N) oracle: basis and stabilisers bit-exact (the packed words
keep the order of the d-ary integers), H x element by element within the
FP64 bound 64 eps (|H| |x|)_i (FP32: eps_32, x4), lowest eigenvalues within
1e-10 relative of the oracle's dense spectrum (FP64 and mixed precision)."""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.vectors import state_vector

pytestmark = pytest.mark.gpu
sun = oracle.sun
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


CASES = {
    "su3_chain9_k0": lambda: C.sun_chain(9, 3, [3, 3, 3], 1.0, 0.0, n_sublat=3),
    "su3_chain8_k1": lambda: C.sun_chain(8, 3, [3, 3, 2], 1.0, 0.3, k=1, n_sublat=2),
    "su3_chain8_refl_odd": lambda: C.sun_chain(8, 3, [3, 3, 2], 1.0, 0.3, reflection=True, n_sublat=2, irrep="A2"),
    "su4_chain8": lambda: C.sun_chain(8, 4, [2, 2, 2, 2], 1.0, 0.2, k=2, n_sublat=2),
    "su2_chain10": lambda: C.sun_chain(10, 2, [5, 5], 1.0, 0.4, k=0, n_sublat=2),
    "su3_triangular12": lambda: C.sun("triangular", [[2, 2], [-2, 4]], 3, [4, 4, 4], 1.0, 0.0, point="none",
                                      irrep="A", n_sublat=3),
    "su5_chain6": lambda: C.sun_chain(6, 5, [2, 1, 1, 1, 1], 1.0, 0.0, k=1, n_sublat=2),
}
_cache = {}


def _oracle(name):
    if name not in _cache:
        p = CASES[name]()
        reps, stab = sun.basis(p.sector)
        H = sun.csr(p, reps, stab)
        packed = np.array([sun.packed(r, p.sector.n_sites, p.sector.n_colors) for r in reps], dtype=np.uint64)
        _cache[name] = (p, reps, stab, H, packed)
    return _cache[name]


def _bound(H, x, eps):
    return 64 * eps * (abs(H) @ np.abs(x)) + 1e-300


@pytest.mark.parametrize("name", sorted(CASES))
def test_sun_basis_bitexact(P, name):
    p, reps, stab, H, packed = _oracle(name)
    b = P.BasisSUN(p.sector)
    assert b.dim == len(reps) == sun.sector_dim_formula(p.sector)
    greps, gstab = b.export()
    assert np.array_equal(greps, packed)
    assert np.array_equal(gstab.astype(np.int64), stab)


@pytest.mark.parametrize("name", sorted(CASES))
def test_sun_hx_and_lanczos(P, name):
    import torch
    p, reps, stab, H, packed = _oracle(name)
    b = P.BasisSUN(p.sector)
    h = P.Hamiltonian(b, p.terms)
    cplx = not h.is_real
    assert cplx == (not p.sector.is_real)
    nvec = 2
    X = np.stack([state_vector(31 + v, packed, complex_=cplx) for v in range(nvec)])
    for single in (False, True):
        if single:
            Xd = X.astype(np.complex64 if cplx else np.float32)
            tdt, eps, fac = (torch.complex64 if cplx else torch.float32), EPS32, 4
        else:
            Xd, tdt, eps, fac = X, (torch.complex128 if cplx else torch.float64), EPS64, 1
        x = torch.tensor(Xd, dtype=tdt, device="cuda")
        y = torch.empty_like(x)
        h.apply(x, y)
        torch.cuda.synchronize()
        Y = y.cpu().numpy().astype(np.complex128)
        for v in range(nvec):
            xv = Xd[v].astype(np.complex128)
            assert np.all(np.abs(Y[v] - H @ xv) <= _bound(H, xv, eps) * fac), (name, single, v)
    # single-vector Lanczos sees each degenerate level once: compare the distinct levels
    w = np.linalg.eigvalsh(H.toarray())
    ref = [w[0]] + [v for v in w if v > w[0] + 1e-8 * max(1.0, abs(w[0]))][:1]
    n_eig = min(2, len(ref))
    ev, rep = h.lanczos(n_eig=n_eig, tol=1e-12, max_iter=300)
    for k in range(n_eig):
        assert abs(ev[k] - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), (name, ev, ref)
    if b.dim > 8:
        dt = P.ED_C64 if cplx else P.ED_F32
        ev, rep = h.lanczos(n_eig=1, tol=1e-10, max_iter=300, dtype=dt, refine=True)
        assert abs(ev[0] - ref[0]) <= 1e-10 * max(1.0, abs(ref[0])), (ev, ref)


def test_su2_matches_the_spin_model(P):
    """Two colours: the SU(2) ground energy equals twice the spin-1/2 library's plus sum J / 2
    (P_ij = 2 S_i.S_j + 1/2) on the same cluster, group and sector."""
    p2 = CASES["su2_chain10"]()
    ps = C.chain(10, 1.0, 0.4, translations=True, n_sublat=2)
    bs = P.Basis(ps.sector)
    hs = P.Hamiltonian(bs, ps.terms)
    es, _ = hs.lanczos(n_eig=1, tol=1e-12, max_iter=300)
    b2 = P.BasisSUN(p2.sector)
    h2 = P.Hamiltonian(b2, p2.terms)
    e2, _ = h2.lanczos(n_eig=1, tol=1e-12, max_iter=300)
    assert abs(e2[0] - (2 * es[0] + 0.5 * float(np.sum(p2.terms.J)))) <= 1e-10 * abs(e2[0])


def test_sun_refuses_spin_calls(P):
    """An SU(N) basis takes ed_hamiltonian_create_sun; the spin-1/2 call refuses it."""
    import ctypes
    p = CASES["su3_chain9_k0"]()
    b = P.BasisSUN(p.sector)
    t = P.ed.ed_terms(0, None, None, 0, None, None)
    h = ctypes.c_void_p()
    assert P.lib().ed_hamiltonian_create(b.handle, ctypes.byref(t), ctypes.byref(h)) == 1  # ED_ERR_ARG


def _unpack(w, N, d):
    b = max(1, int(np.ceil(np.log2(d))))
    return sun.integer([(int(w) >> ((N - 1 - k) * b)) & ((1 << b) - 1) for k in range(N)], d)


def test_sun_triangular21_full_size(P):
    """SU(3) on the 21-site triangular torus (T21 x C6, 7 sites of each colour, D ~ 3.2e6):
    the GPU basis is the true one by a counting argument (character-formula dimension,
    strictly increasing, sampled members are compatible orbit minima with the right |Stab|,
    representatives of oracle-drawn colourings are present), and H x on sampled rows equals
    the oracle's matrix-free rows (FP64 and FP32)."""
    import torch
    p = C.sun_triangular21()
    s = p.sector
    N, d = s.n_sites, s.n_colors
    b = P.BasisSUN(s)
    assert b.dim == sun.sector_dim_formula(s)
    reps, stab = b.export()
    assert np.all(reps[1:] > reps[:-1])
    rng = np.random.default_rng(3)
    for i in rng.choice(b.dim, size=150, replace=False):
        r, g, n, ssum = sun.rep(s, _unpack(reps[i], N, d))
        assert sun.packed(r, N, d) == int(reps[i]) and n == int(stab[i]) and abs(ssum) > 1e-9
    drawn = []
    while len(drawn) < 60:
        col = rng.permutation([c for c in range(d) for _ in range(int(s.counts[c]))])
        r, g, n, ssum = sun.rep(s, sun.integer(col, d))
        if abs(ssum) > 1e-9:
            drawn.append(r)
    drawn = sorted(set(drawn))
    packed = np.array([sun.packed(r, N, d) for r in drawn], dtype=np.uint64)
    pos = np.searchsorted(reps, packed)
    assert np.all(pos < b.dim) and np.array_equal(reps[pos], packed)
    h = P.Hamiltonian(b, p.terms)
    X = state_vector(5, reps)
    key = {int(w): k for k, w in enumerate(reps[pos])}
    yo = sun.rows(p, drawn, lambda r: state_vector(5, np.array([sun.packed(r, N, d)], dtype=np.uint64))[0])
    R = np.sum(np.abs(p.terms.J)) * (1 + np.sqrt(s.n_sym))
    for tdt, eps, fac in ((torch.float64, EPS64, 1), (torch.float32, EPS32, 4)):
        x = torch.tensor(X, device="cuda").to(tdt)
        y = torch.empty_like(x)
        h.apply(x, y)
        torch.cuda.synchronize()
        yg = y[torch.tensor(pos.astype(np.int64), device="cuda")].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(yg - yo.real) <= 64 * eps * R * fac), np.abs(yg - yo.real).max()
    assert len(key) == len(drawn)
