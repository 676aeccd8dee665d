"""Batches of sectors: the batched H.x equals per-sector H.x, and block Lanczos
on all sectors at once reproduces each sector's oracle spectrum (with
multiplicities up to the block size)."""
import numpy as np
import pytest

import oracle
from edinputs import configs as C
from edinputs.vectors import state_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def tri12():
    """All (k, rho_k) sectors of the 4x4 square torus with the rotation group C4
    (abelian little groups, so 1-D irreps cover the space), J1=1, J2=0.3, Sz=0."""
    return C.all_sectors("square", [[4, 0], [0, 4]], 1.0, 0.3, n_sublat=2, point="rot")


def _concat(P, probs, nvec, seed, cplx):
    blocks = []
    for p in probs:
        reps, _ = oracle.basis(p.sector)
        blocks.append(np.concatenate([state_vector(seed + v, reps, complex_=cplx) for v in range(nvec)]))
    return np.concatenate(blocks)


def test_sector_dimensions_partition(tri12):
    assert sum(oracle.sector_dim_formula(p.sector) for p in tri12) == oracle.binom(16, 8)


@pytest.mark.parametrize("nvec", [1, 3])
def test_batched_apply_equals_per_sector(P, tri12, nvec):
    import torch
    bases = [P.Basis(p.sector) for p in tri12]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12)]
    batch = P.Batch(hs)
    X = _concat(P, tri12, nvec, 3, True)
    x = torch.tensor(X, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    batch.apply(x, y, nvec=nvec)
    torch.cuda.synchronize()
    Y = y.cpu().numpy()
    off = batch.row_off
    for s, h in enumerate(hs):
        D = int(off[s + 1] - off[s])
        xs = x[nvec * int(off[s]):nvec * int(off[s + 1])].reshape(nvec, D).contiguous()
        ys = torch.empty_like(xs)
        h.apply(xs, ys)
        torch.cuda.synchronize()
        assert np.array_equal(ys.cpu().numpy().ravel(), Y[nvec * int(off[s]):nvec * int(off[s + 1])])
    w = batch.autotune(x, y, nvec=nvec)
    assert w in (1, 2, 4, 8, 16)


@pytest.mark.parametrize("use_graph", [True, False])
def test_block_lanczos_all_sectors(P, tri12, use_graph):
    bases = [P.Basis(p.sector) for p in tri12]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12)]
    batch = P.Batch(hs)
    n_eig = 3
    ev, rep = batch.lanczos(block=4, n_eig=n_eig, tol=1e-12, max_iter=40, seed=5, use_graph=use_graph)
    assert rep.converged_sectors == len(tri12) and rep.used_graph == int(use_graph)
    for s, p in enumerate(tri12):
        ref = np.linalg.eigvalsh(oracle.csr(p).toarray())[:n_eig]
        assert np.allclose(ev[s, :len(ref)], ref, rtol=0, atol=1e-10 * max(1.0, abs(ref[0]))), (s, ev[s], ref)


def test_block_lanczos_plain_recursion_needs_block_one(P, tri12):
    """Without reorthogonalisation the batched solver takes one vector per sector only."""
    bases = [P.Basis(p.sector) for p in tri12[:3]]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12[:3])]
    batch = P.Batch(hs)
    with pytest.raises(P.EdError) as e:
        batch.lanczos(block=4, n_eig=2, tol=1e-10, max_iter=40, reorth=False)
    assert e.value.name == "ED_ERR_ARG"


@pytest.mark.parametrize("reorth", [True, False])
def test_batched_single_vector_lanczos(P, tri12, reorth):
    """Block size 1: one Lanczos vector per sector, all sectors advanced by one graph
    launch per step (converged sectors drop out), with full reorthogonalisation or the
    plain recursion (spurious copies filtered); each sector's ground level to 1e-10 (a
    single vector sees each degenerate level once, so only the lowest is compared)."""
    bases = [P.Basis(p.sector) for p in tri12]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12)]
    batch = P.Batch(hs)
    ev, rep = batch.lanczos(block=1, n_eig=1, tol=1e-12, max_iter=300, seed=7, use_graph=True, reorth=reorth)
    assert rep.converged_sectors == len(tri12) and rep.used_graph == 1
    for s, p in enumerate(tri12):
        e0 = np.linalg.eigvalsh(oracle.csr(p).toarray())[0]
        assert abs(ev[s, 0] - e0) <= 1e-10 * max(1.0, abs(e0)), (s, ev[s, 0], e0)


@pytest.mark.parametrize("nvec", [1, 3])
def test_batched_stored_apply(P, tri12, nvec):
    """Every sector's structure stored (ed_hamiltonian_store, one segment): the batched
    H.x runs the stored-structure kernel over all sectors and equals each sector's own
    stored ed_apply (the same sums in the same order; complex products may be contracted
    into FMAs differently by the two kernels, so to 1e-13 of max|y|), and the
    matrix-free batched H.x to the FP64 bound."""
    import torch
    bases = [P.Basis(p.sector) for p in tri12]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12)]
    batch = P.Batch(hs)
    X = _concat(P, tri12, nvec, 3, True)
    x = torch.tensor(X, dtype=torch.complex128, device="cuda")
    y_free = torch.empty_like(x)
    batch.apply(x, y_free, nvec=nvec)
    for h in hs:
        h.store()
    y = torch.empty_like(x)
    batch.apply(x, y, nvec=nvec)
    torch.cuda.synchronize()
    off = batch.row_off
    for s, h in enumerate(hs):
        D = int(off[s + 1] - off[s])
        xs = x[nvec * int(off[s]):nvec * int(off[s + 1])].reshape(nvec, D).contiguous()
        ys = torch.empty_like(xs)
        h.apply(xs, ys)
        torch.cuda.synchronize()
        ref = y[nvec * int(off[s]):nvec * int(off[s + 1])]
        assert (ys.reshape(-1) - ref).abs().max().item() <= 1e-13 * max(1.0, ref.abs().max().item())
    scale = 64 * np.finfo(np.float64).eps * 16 * 0.3 * 8
    assert (y - y_free).abs().max().item() <= scale * x.abs().max().item()


@pytest.mark.parametrize("block,reorth", [(1, False), (1, True), (4, True)])
def test_batched_stored_lanczos(P, tri12, block, reorth):
    """Block Lanczos (CUDA graph) on the stored structures of all sectors: each sector's
    lowest levels against the oracle's dense spectrum."""
    bases = [P.Basis(p.sector) for p in tri12]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12)]
    for h in hs:
        h.store()
    batch = P.Batch(hs)
    n_eig = 1 if block == 1 else 3
    ev, rep = batch.lanczos(block=block, n_eig=n_eig, tol=1e-12, max_iter=300 if block == 1 else 40, seed=5,
                            use_graph=True, reorth=reorth)
    assert rep.converged_sectors == len(tri12)
    for s, p in enumerate(tri12):
        ref = np.linalg.eigvalsh(oracle.csr(p).toarray())[:n_eig]
        assert np.allclose(ev[s, :len(ref)], ref, rtol=0, atol=1e-10 * max(1.0, abs(ref[0]))), (s, ev[s], ref)


@pytest.mark.parametrize("block,stored", [(1, False), (4, False), (8, True), (1, True)])
def test_batched_fp32_block_lanczos(P, tri12, block, stored):
    """FP32 vectors (complex FP32: the batch has complex sectors), block Gram-Schmidt in FP32
    arithmetic, then the FP64 refinement (Ritz vectors, one batched FP64 H.x,
    Rayleigh-Ritz): every sector's lowest levels within 1e-10 of the oracle's dense
    spectrum, with multiplicities up to the block size."""
    bases = [P.Basis(p.sector) for p in tri12]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12)]
    if stored:
        for h in hs:
            h.store()
    batch = P.Batch(hs)
    assert not batch.is_real
    n_eig = 1 if block == 1 else 3
    ev, rep = batch.lanczos(block=block, n_eig=n_eig, tol=1e-10, max_iter=300 if block == 1 else 40, seed=5,
                            use_graph=True, reorth=True, dtype=P.ED_C64)
    assert rep.converged_sectors == len(tri12)
    for s, p in enumerate(tri12):
        ref = np.linalg.eigvalsh(oracle.csr(p).toarray())[:n_eig]
        assert np.allclose(ev[s, :len(ref)], ref, rtol=0, atol=1e-10 * max(1.0, abs(ref[0]))), (s, ev[s], ref)


def test_batched_fp32_real_sectors(P):
    """Real sectors only (the Gamma sectors of the 4x4 square with C4v): FP32 real vectors
    and the real FP64 refinement, against the oracle."""
    probs = [C.square([[4, 0], [0, 4]], 1.0, 0.3, irrep=irr) for irr in ("A1", "A2", "B1", "B2")]
    bases = [P.Basis(p.sector) for p in probs]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, probs)]
    batch = P.Batch(hs)
    assert batch.is_real
    ev, rep = batch.lanczos(block=2, n_eig=2, tol=1e-10, max_iter=60, seed=3, use_graph=True, reorth=True,
                            dtype=P.ED_F32)
    assert rep.converged_sectors == len(probs)
    for s, p in enumerate(probs):
        ref = np.linalg.eigvalsh(oracle.csr(p).toarray())[:2]
        assert np.allclose(ev[s, :len(ref)], ref, rtol=0, atol=1e-10 * max(1.0, abs(ref[0]))), (s, ev[s], ref)


def test_batched_fp32_needs_reorth(P, tri12):
    """FP32 vectors need the stored blocks (full reorthogonalisation) and n_eig <= 8."""
    bases = [P.Basis(p.sector) for p in tri12[:2]]
    hs = [P.Hamiltonian(b, p.terms) for b, p in zip(bases, tri12[:2])]
    batch = P.Batch(hs)
    with pytest.raises(P.EdError) as e:
        batch.lanczos(block=1, n_eig=1, tol=1e-10, max_iter=40, reorth=False, dtype=P.ED_C64)
    assert e.value.name == "ED_ERR_ARG"
    with pytest.raises(P.EdError) as e:
        batch.lanczos(block=2, n_eig=9, tol=1e-10, max_iter=40, reorth=True, dtype=P.ED_C64)
    assert e.value.name == "ED_ERR_ARG"
