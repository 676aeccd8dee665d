"""Kagome J1-J2-J3-J_chi model (Eq. chiralhamiltonian): third neighbours only
across the hexagons, on the same H.x path.

CPU: the J3 bond set of kagome tori has N bonds, two per site, each of length
twice the nearest-neighbour distance with a hexagon centre (no site) at its
midpoint, and every element of the space group (with mirrors when J_chi = 0)
maps it onto itself; every eigenvalue of a symmetric sector is an eigenvalue
of the unsymmetrised fixed-Sz matrix (oracle), so the J3 terms respect the
sector's symmetry.

GPU: kagome12 with J3 and J_chi (complex E1 sector): the full H.x against the
oracle's matrix (C128, C64) and the Lanczos ground energy against the dense
spectrum; the 36-site torus at J2 = J3 = 0.4 with J_chi = 0.2 (T12 x C6 x Z2):
the basis by the counting argument and sampled rows of H.x against the
matrix-free oracle.
"""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.lattice import Cluster, kagome_lattice

EPS64 = np.finfo(np.float64).eps


def _k12(**kw):
    return C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, J3=0.45, irrep="E1", **kw)


@pytest.mark.parametrize("P_", [[[2, 0], [0, 2]], [[3, 0], [0, 3]], [[2, 2], [-2, 4]]])
def test_j3_bond_set(P_):
    cl = Cluster(kagome_lattice(), P_)
    b = np.array(cl.bonds_across_hexagons())
    assert len(b) == cl.N
    assert set(np.bincount(b.ravel(), minlength=cl.N).tolist()) == {2}
    d1 = cl.neighbour_shells(1)[0][0]
    for i, j in b:
        # some image of j at distance 2 d1 from i, whose midpoint is not a site
        ok = False
        for a in range(-2, 3):
            for c in range(-2, 3):
                rj = cl.pos[j] + np.array([a, c]) @ cl.cart_periods()
                if abs(np.linalg.norm(rj - cl.pos[i]) - 2 * d1) < 1e-9 and cl.locate((cl.pos[i] + rj) / 2) is None:
                    ok = True
        assert ok


@pytest.mark.parametrize("point,Jchi", [("rot", 0.3), ("full", 0.0)])
def test_j3_bonds_invariant(point, Jchi):
    p = C.kagome([[2, 2], [-2, 4]], 1.0, 0.4, Jchi, J3=0.4, point=point, irrep="A" if point == "rot" else "A1")
    perm = np.asarray(p.sector.perm)
    key = {(min(i, j), max(i, j), J) for (i, j), J in zip(p.terms.bonds.tolist(), p.terms.J.tolist())}
    for g in perm:
        img = {(min(g[i], g[j]), max(g[i], g[j]), J) for (i, j), J in zip(p.terms.bonds.tolist(), p.terms.J.tolist())}
        assert img == key


def test_j3_sector_spectrum_in_full_spectrum():
    p = _k12()
    reps, stab = oracle.basis(p.sector)
    Hs = oracle.csr(p, reps, stab).toarray()
    es = np.linalg.eigvalsh(Hs)
    Hd, _ = oracle.dense_sz(p)
    ed = np.linalg.eigvalsh(Hd)
    for e in es:
        assert np.min(np.abs(ed - e)) < 1e-10


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


@pytest.mark.gpu
def test_gpu_kagome12_j3_full_parity(P):
    import torch
    from edinputs.vectors import state_vector
    p = _k12()
    reps, stab = oracle.basis(p.sector)
    H = oracle.csr(p, reps, stab)
    b = P.Basis(p.sector)
    greps, gstab = b.export()
    assert np.array_equal(greps, reps)
    h = P.Hamiltonian(b, p.terms)
    assert not h.is_real
    X = state_vector(17, reps, complex_=True)
    ref = H @ X
    bound = 64 * EPS64 * (abs(H) @ np.abs(X)) + 1e-300
    for dt, scale in ((torch.complex128, 1.0), (torch.complex64, float(np.finfo(np.float32).eps / EPS64) * 4)):
        x = torch.tensor(X, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        h.apply(x, y)
        torch.cuda.synchronize()
        assert np.all(np.abs(y.cpu().numpy() - ref) <= scale * bound)
    e_ref = np.linalg.eigvalsh(H.toarray())[0]
    vals, rep = h.lanczos(n_eig=1, tol=1e-12, max_iter=300, dtype=P.ED_C128)
    assert vals[0] == pytest.approx(e_ref, abs=1e-10 * abs(e_ref))


@pytest.mark.gpu
def test_gpu_kagome36_j3_sampled_rows(P):
    import torch
    from test_gpu_workloads import _check_basis, _check_hx
    p = C.kagome([[2, 2], [-2, 4]], 1.0, 0.4, 0.2, J3=0.4, irrep="A", spinflip=1)
    assert p.sector.n_sym == 144 and len(p.terms.bonds) == 36 * 2 + 36 * 2 + 36
    b, reps, drawn, pos = _check_basis(P, p, 600, 11)
    _check_hx(P, p, b, reps, drawn, pos, torch.complex64)
    _check_hx(P, p, b, reps, drawn, pos, torch.complex128)
