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


def test_noalloc_rejects_oversized_tables(P):
    # the 4x4 square group as one block of 16 sites: its Rep/Sym/SymmetryAction
    # tables exceed the 224 KB array
    from edinputs.lattice import Sector
    base = C.square([[4, 0], [0, 4]], 1.0, 0.5, irrep="A1").sector
    s = Sector(16, 8, base.perm, base.spinflip, base.chi, 1)
    with pytest.raises(P.EdError) as e:
        _noalloc(P, s, np.array([3], dtype=np.uint64))
    assert e.value.name == "ED_ERR_TABLE_TOO_LARGE"
