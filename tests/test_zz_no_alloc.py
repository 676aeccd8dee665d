"""The no-allocation representative search against the allocating one.

ed_representatives_noalloc serves callers that cannot allocate device memory
themselves (their memory belongs to another runtime's pool, or their loop must
not call cudaMalloc/cudaFree, which can synchronise the device).  It keeps the
lookup-table image in a file-scope device array and writes into the caller's
buffers.  This test calls it through the C ABI twice in a row, on two
different sectors so that the second call must replace the first call's table
image, and checks every output against ed_representatives.  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from edinputs import configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03511_gb300 import build
    build.build()
    import paper_2210_03511_gb300 as pkg
    L = pkg.lib()
    L.ed_representatives_noalloc.argtypes = [ctypes.POINTER(pkg.ed.ed_sector), ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
    L.ed_representatives_noalloc.restype = ctypes.c_int
    return pkg


def _noalloc(P, sector, states_np):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    states = torch.tensor(states_np.view(np.int64), device=dev)
    n = states.numel()
    rep = torch.empty(n, dtype=torch.int64, device=dev)
    g = torch.empty(n, dtype=torch.int32, device=dev)
    ns = torch.empty(n, dtype=torch.int32, device=dev)
    cp = torch.empty(n, dtype=torch.uint8, device=dev)
    sec, keep = P.ed._sector_struct(sector)
    stream = torch.cuda.current_stream(dev)
    st = P.lib().ed_representatives_noalloc(ctypes.byref(sec), states.data_ptr(), n, rep.data_ptr(), g.data_ptr(),
                                            ns.data_ptr(), cp.data_ptr(), stream.cuda_stream)
    P.ed.check(st)
    torch.cuda.synchronize()
    return (rep.cpu().numpy().view(np.uint64), g.cpu().numpy(), ns.cpu().numpy(), cp.cpu().numpy().astype(bool))


def test_noalloc_matches_allocating_entry_point_twice(P):
    # square32 with 8-site blocks: a 53 KB table image (16-site blocks need 1.7 MB)
    cases = [C.square32(n_sublat=4).sector, C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1").sector]
    rng = np.random.default_rng(11)
    for sector in cases:
        N = sector.n_sites
        states = rng.integers(0, 1 << N, size=5000, dtype=np.uint64)
        ref = P.representatives(sector, states)
        got = _noalloc(P, sector, states)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


def test_noalloc_global_read_tables_vs_oracle(P):
    """A table image between the 200 KB whole-staging limit and the 224 KB array (the
    36-site kagome cluster with its full D6 point group and spin flip: 213.5 KB), so
    the kernel reads the array through global memory instead of staging it: every
    output equals ed_representatives, and a sample equals the oracle's brute force
    (orbit minimum, |Stab|, non-zero projector, an element mapping the state onto it)."""
    sector = C.kagome([[2, 2], [-2, 4]], 1.0, 0.2, 0.0, point="full", spinflip=1, irrep="A1").sector
    rng = np.random.default_rng(13)
    states = np.zeros(4000, dtype=np.uint64)
    for i in range(len(states)):  # states of the sector's S^z = 0 (spin flip needs it)
        bits = np.zeros(36, dtype=np.int64)
        bits[rng.choice(36, 18, replace=False)] = 1
        states[i] = int("".join(map(str, bits)), 2)
    for _ in range(2):  # twice in a row: the second call reuses the array's image
        ref = P.representatives(sector, states)
        got = _noalloc(P, sector, states)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
    rep, g, ns, cp = got
    for i in range(0, len(states), 8):
        r0, g0, n0, ssum = oracle.rep(sector, int(states[i]))
        assert int(rep[i]) == r0 and int(ns[i]) == n0 and bool(cp[i]) == (abs(ssum) > 1e-9)
        assert oracle.apply(sector, int(g[i]), int(states[i])) == r0


def test_noalloc_rejects_oversized_tables(P):
    # the 4x4 square group as one block of 16 sites: its Rep/Sym/SymmetryAction
    # tables exceed the 224 KB array
    from edinputs.lattice import Sector
    base = C.square([[4, 0], [0, 4]], 1.0, 0.5, irrep="A1").sector
    s = Sector(16, 8, base.perm, base.spinflip, base.chi, 1)
    with pytest.raises(P.EdError) as e:
        _noalloc(P, s, np.array([3], dtype=np.uint64))
    assert e.value.name == "ED_ERR_TABLE_TOO_LARGE"


def test_noalloc_refuses_stream_capture(P):
    """Called while its stream is being captured, the entry point returns ED_ERR_ARG
    before touching the device (its table upload reads a host buffer that lives only
    for the call); the capture itself stays valid."""
    import torch
    sector = C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1").sector
    dev = torch.device("cuda", torch.cuda.current_device())
    states = torch.zeros(4, dtype=torch.int64, device=dev)
    out = [torch.empty(4, dtype=t, device=dev) for t in (torch.int64, torch.int32, torch.int32, torch.uint8)]
    sec, keep = P.ed._sector_struct(sector)
    s = torch.cuda.Stream(device=dev)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        graph.capture_begin()
        try:
            st = P.lib().ed_representatives_noalloc(ctypes.byref(sec), states.data_ptr(), 4, out[0].data_ptr(),
                                                    out[1].data_ptr(), out[2].data_ptr(), out[3].data_ptr(),
                                                    s.cuda_stream)
            states.add_(1)  # something to capture
        finally:
            graph.capture_end()
    torch.cuda.synchronize()
    assert st == 1  # ED_ERR_ARG
    assert "captured" in P.lib().ed_last_error().decode()
    graph.replay()
    torch.cuda.synchronize()
    assert int(states[0].item()) == 1  # the captured add ran once, on replay
