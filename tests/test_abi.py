"""C ABI checks that need no GPU: the library loads, exports every function of
include/ed.h, validates sectors, and builds the sublattice-coding tables of
Alg. "Preparation of lookup tables for sublattice coding algorithm" as the
thesis's two worked examples state them."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

from edinputs import configs as C
from edinputs.lattice import Sector

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


def test_exports_every_declared_function(P):
    hdr = open(os.path.join(ROOT, "include", "ed.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(ed_[a-z_0-9]+)\s*\(", hdr))
    assert {"ed_basis_build", "ed_apply", "ed_lanczos"} <= names
    L = ctypes.CDLL(P.ed.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n


def _chain6(site_positions, chi=None, flip=None):
    pos = list(site_positions)
    site_of = {x: i for i, x in enumerate(pos)}
    perm = np.array([[site_of[(pos[i] + n) % 6] for i in range(6)] for n in range(6)], dtype=np.int32)
    chi = np.ones(6, complex) if chi is None else chi
    flip = np.zeros(6, np.uint8) if flip is None else flip
    return perm, chi, flip


def _bits(s):
    return int(s, 2)


def _sym_set(t, X, s):
    off = t["sym_off"]
    return sorted(int(g) for g in t["sym_ids"][off[X, s]:off[X, s + 1]])


def test_worked_example_two_sublattices(P):
    """Tables of the two-sublattice example: G_A, G_B, Rep_A, Rep_B, Sym_B."""
    ex = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_examples.json")))["two_sublattice"]
    perm, chi, flip = _chain6(ex["site_positions"])
    t = P.sector_tables(Sector(6, 3, perm, flip, chi, 2))
    assert t["m"] == 3
    # G_X = elements mapping block X onto block 0 (A)
    GA = [g for g in range(6) if t["dest"][g, 0] == 0]
    GB = [g for g in range(6) if t["dest"][g, 1] == 0]
    name = lambda g: "Id" if g == 0 else f"T{g}"
    assert [name(g) for g in GA] == ex["G_A"] and [name(g) for g in GB] == ex["G_B"]
    sA, sB = _bits(ex["substate_A"]), _bits(ex["substate_B"])
    assert t["rep"][0, sA] == ex["Rep_A"]
    assert t["rep"][1, sB] == ex["Rep_B"]
    assert [name(g) for g in _sym_set(t, 1, sB)] == ex["Sym_B"]


def test_worked_example_three_sublattices(P):
    """Tables of the three-sublattice example: Rep_A/B/C and Sym_A/B/C."""
    ex = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_examples.json")))["three_sublattice"]
    perm, chi, flip = _chain6(ex["site_positions"])
    t = P.sector_tables(Sector(6, 3, perm, flip, chi, 3))
    name = lambda g: "Id" if g == 0 else f"T{g}"
    for X, lab in enumerate("ABC"):
        s = _bits(ex[f"substate_{lab}"])
        assert t["rep"][X, s] == ex[f"Rep_{lab}"], lab
        assert [name(g) for g in _sym_set(t, X, s)] == ex[f"Sym_{lab}"], lab
    # SymmetryAction composes T2 sigma = 000111 block by block
    st = _bits(ex["state"])
    sub = [(st >> (2 * (2 - X))) & 3 for X in range(3)]
    img = [0, 0, 0]
    for X in range(3):
        img[t["dest"][2, X]] = t["sa"][2, X, sub[X]]
    assert (img[0] << 4) | (img[1] << 2) | img[2] == _bits(ex["T2_image"])


def test_tables_match_definitions_bruteforce(P):
    """Rep_X(s) = min over G_X of SymmetryAction_X(g, s); Sym_X(s) = its argmin set (Eqs. sublatrepdef, repsymdef)."""
    p = C.square([[4, 0], [0, 4]], 1.0, 0.5, spinflip=1)
    s = p.sector
    t = P.sector_tables(s)
    m, n_sub, G = t["m"], s.n_sublat, s.n_sym
    N = s.n_sites
    for X in range(n_sub):
        for sub in range(1 << m):
            vals = {}
            for g in range(G):
                Z = int(t["dest"][g, X])
                # direct action on the full state restricted to block X
                img = 0
                for l in range(m):
                    bit = (sub >> (m - 1 - l)) & 1
                    if s.spinflip[g]:
                        bit ^= 1
                    if bit:
                        img |= 1 << (m - 1 - (int(s.perm[g][X * m + l]) - Z * m))
                assert t["sa"][g, X, sub] == img
                if Z == 0:
                    vals[g] = img
            best = min(vals.values())
            assert t["rep"][X, sub] == best
            assert _sym_set(t, X, sub) == sorted(g for g, v in vals.items() if v == best)


def test_validation_errors(P):
    base = C.chain(8, translations=True)
    s = base.sector

    def err(sec):
        with pytest.raises(P.EdError) as e:
            P.sector_tables(sec)
        return e.value.name

    bad = Sector(s.n_sites, s.n_up, s.perm[::-1].copy(), s.spinflip, s.chi, s.n_sublat)
    assert err(bad) == "ED_ERR_NOT_GROUP"  # identity not first
    assert err(Sector(s.n_sites, s.n_up, s.perm[:3].copy(), s.spinflip[:3], s.chi[:3], s.n_sublat)) == "ED_ERR_NOT_GROUP"
    chi = s.chi.copy()
    chi[1] *= -1
    assert err(Sector(s.n_sites, s.n_up, s.perm, s.spinflip, chi, s.n_sublat)) == "ED_ERR_CHAR_NOT_HOMOMORPHISM"
    chi = s.chi.copy() * 1.1
    chi[0] = 1
    assert err(Sector(s.n_sites, s.n_up, s.perm, s.spinflip, chi, s.n_sublat)) == "ED_ERR_CHAR_NOT_HOMOMORPHISM"
    pf = C.chain(8, translations=True, spinflip=1).sector
    assert err(Sector(8, 3, pf.perm, pf.spinflip, pf.chi, pf.n_sublat)) == "ED_ERR_SPINFLIP_SZ"
    # translations by one site split the 2-block partition {0..3},{4..7} of a chain numbered in order
    perm = np.array([[(i + n) % 8 for i in range(8)] for n in range(8)], np.int32)
    assert err(Sector(8, 4, perm, np.zeros(8, np.uint8), np.ones(8, complex), 2)) == "ED_ERR_NOT_SUBLATTICE_STABLE"
    assert err(Sector(8, 4, perm, np.zeros(8, np.uint8), np.ones(8, complex), 3)) == "ED_ERR_ARG"
    perm2 = perm.copy()
    perm2[3] = perm2[2]
    assert err(Sector(8, 4, perm2, np.zeros(8, np.uint8), np.ones(8, complex), 1)) == "ED_ERR_NOT_GROUP"
    assert err(Sector(70, 35, np.arange(70, dtype=np.int32)[None], np.zeros(1, np.uint8), np.ones(1, complex), 1)) \
        == "ED_ERR_ARG"


def test_workload_tables_fit_shared_memory(P):
    """With blocks of at most 12 sites the table image stays below 200 KB (whole-image staging
    by the basis kernels): Rep and Sym tables plus SymmetryAction stored once per distinct local
    block map.  (square32's default 16-site blocks keep their 1.7 MB image in global memory.)"""
    for make in (lambda: C.square32(n_sublat=4), C.kagome36, C.triangular24, C.square40):
        s = make().sector
        t = P.sector_tables(s)
        m, n_sub, G = t["m"], s.n_sublat, s.n_sym
        maps = set()
        for g in range(G):
            for X in range(n_sub):
                Z = int(t["dest"][g, X])
                maps.add((tuple(int(s.perm[g][X * m + l]) - Z * m for l in range(m)), int(s.spinflip[g])))
        per_map = (1 << m) if m <= 8 else 2 * ((1 << (m - m // 2)) + (1 << (m // 2)))
        total = (len(maps) * per_map + t["rep"].size * 2 + t["sym_off"].size * 4 + len(t["sym_ids"]) * 2
                 + G * n_sub * 4 + G * 40)
        assert total <= 200 * 1024, (make.__name__, total)


def _plain_lanczos(A, n, dt, seed):
    """Three-term Lanczos recursion without reorthogonalisation, vectors stored in dt."""
    rng = np.random.default_rng(seed)
    D = A.shape[0]
    v = rng.uniform(-1, 1, D)
    v = (v / np.linalg.norm(v)).astype(dt)
    vp = np.zeros(D, dt)
    a, b, beta = [], [], 0.0
    for _ in range(n):
        w = A @ v.astype(np.float64)
        al = float(v.astype(np.float64) @ w)
        w = w - al * v.astype(np.float64) - beta * vp.astype(np.float64)
        beta = float(np.linalg.norm(w))
        a.append(al)
        b.append(beta)
        vp, v = v, (w / beta).astype(dt)
    return np.array(a), np.array(b)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_tridiag_ghost_filter(P, dt):
    """Plain Lanczos on a matrix with a known spectrum runs long enough for the lowest
    eigenvalues to reappear as spurious copies; the unfiltered T-matrix solve lists them
    repeatedly, the filtered one lists each distinct eigenvalue once."""
    D = 300
    rng = np.random.default_rng(2)
    lam = np.sort(np.concatenate([[-5.0, -4.6, -4.1, -3.9], rng.uniform(-3.5, 3.0, D - 4)]))
    Q, _ = np.linalg.qr(rng.normal(size=(D, D)))
    A = (Q * lam) @ Q.T
    a, b = _plain_lanczos(A, 400, dt, 1)
    raw = P.tridiag_eigs(a, b[:-1], 6, filter=False)
    assert np.sum(np.abs(raw + 5.0) < 1e-6) >= 2          # ghosts present
    eps = 2.0 ** -53 if dt == np.float64 else 2.0 ** -24
    got = P.tridiag_eigs(a, b[:-1], 4, eps_vectors=eps, filter=True)
    tol = 1e-10 if dt == np.float64 else 1e-5
    assert len(got) == 4 and np.allclose(got, lam[:4], rtol=0, atol=tol), got
    # a short run without ghosts: filtering changes nothing
    a2, b2 = _plain_lanczos(A, 40, np.float64, 3)
    assert np.array_equal(P.tridiag_eigs(a2, b2[:-1], 3, filter=True), P.tridiag_eigs(a2, b2[:-1], 3, filter=False))


def _lower_band(A, bw):
    n = A.shape[0]
    L = np.zeros((n, bw + 1), complex)
    for i in range(n):
        for q in range(min(bw, i) + 1):
            L[i, q] = A[i, i - q]
    return L


@pytest.mark.parametrize("bw", [1, 3, 15])
def test_band_eigs_against_lapack(P, bw):
    """ed_band_eigs (the host solver of block Lanczos) on random complex Hermitian band
    matrices: eigenvalues equal LAPACK's (numpy.linalg.eigvalsh) to 1e-12 of |T|, and each
    eigenvector has a residual below 1e-10 |T| and is orthonormal to the others."""
    rng = np.random.default_rng(bw)
    n = 90
    A = np.zeros((n, n), complex)
    for i in range(n):
        for j in range(max(0, i - bw), i):
            A[i, j] = rng.normal() + 1j * rng.normal()
        A[i, i] = rng.normal()
    A = np.tril(A, -1) + np.tril(A, -1).conj().T + np.diag(np.diag(A).real)
    ref = np.linalg.eigvalsh(A)
    k = 6
    ev, Z = P.band_eigs(_lower_band(A, bw), k)
    scale = np.abs(A).sum(axis=1).max()
    assert len(ev) == k and np.allclose(ev, ref[:k], rtol=0, atol=1e-12 * scale), (ev, ref[:k])
    for e in range(k):
        assert np.linalg.norm(A @ Z[e] - ev[e] * Z[e]) <= 1e-10 * scale
    assert np.allclose(Z.conj() @ Z.T, np.eye(k), atol=1e-10)


def test_band_eigs_degenerate_levels(P):
    """Two identical uncoupled blocks: every eigenvalue is doubly degenerate (the copies a
    block Lanczos run holds); the solver returns each value twice with orthonormal vectors
    spanning the level."""
    rng = np.random.default_rng(7)
    m, bw = 30, 3
    B = np.zeros((m, m))
    for i in range(m):
        for j in range(max(0, i - bw), i):
            B[i, j] = B[j, i] = rng.normal()
        B[i, i] = rng.normal()
    A = np.zeros((2 * m, 2 * m), complex)
    A[:m, :m] = B
    A[m:, m:] = B
    ref = np.linalg.eigvalsh(B)
    ev, Z = P.band_eigs(_lower_band(A, bw), 4)
    assert np.allclose(ev, [ref[0], ref[0], ref[1], ref[1]], rtol=0, atol=1e-12 * np.abs(B).sum(axis=1).max())
    assert np.allclose(Z.conj() @ Z.T, np.eye(4), atol=1e-10)
    for e in range(4):
        assert np.linalg.norm(A @ Z[e] - ev[e] * Z[e]) <= 1e-9
    assert len(P.band_eigs(_lower_band(A, bw), 200, vectors=False)[0]) == 2 * m   # at most n values
