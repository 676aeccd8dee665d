"""The library's representative search run on the CPU (CPU only, no GPU).

The search functions the kernels call (find_rep, the block-count-specialised
find_rep_ns and is_rep) are __host__ __device__; tests/host_rep/harness.cu
compiles them for the host over the library's own table image (its table
builder, linked from libed.so).  Against the oracle's brute force (apply every
element): the representative, |Stab|, compatibility, that the returned element
maps the state onto its representative (any minimising element is valid), and
is_rep agrees with both.  Sectors: 2 blocks of 16 sites (chunked maps), 4
blocks of 8, 8 blocks of 8 with 64-bit words and the sign bit in use, complex
characters, spin flip, and the 9-block kagome36 (generic search only).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from edinputs import configs as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_2210_03511_gb300 import build
    lib_path = build.build()
    libdir = os.path.dirname(lib_path)
    out = str(tmp_path_factory.mktemp("host_rep") / "harness.so")
    cmd = [build.nvcc()] + build.ARCH + ["-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                                         "-I", os.path.join(ROOT, "include"), "-I", build.CSRC,
                                         os.path.join(ROOT, "tests", "host_rep", "harness.cu"), "-o", out,
                                         "-L", libdir, "-led", "-Xlinker", "-rpath", "-Xlinker", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    L = ctypes.CDLL(out)
    f = L.harness_representatives
    f.restype = ctypes.c_int
    return f


def _call(f, sector, states, variant):
    from paper_2210_03511_gb300.ed import _sector_struct
    sec, keep = _sector_struct(sector)
    n = len(states)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    rep = np.zeros(n, np.uint64)
    g = np.zeros(n, np.int32)
    ns = np.zeros(n, np.int32)
    cp = np.zeros(n, np.uint8)
    own = np.zeros(n, np.uint8)
    P = ctypes.POINTER
    rc = f(ctypes.byref(sec), st.ctypes.data_as(P(ctypes.c_uint64)), ctypes.c_int64(n), variant,
           rep.ctypes.data_as(P(ctypes.c_uint64)), g.ctypes.data_as(P(ctypes.c_int32)),
           ns.ctypes.data_as(P(ctypes.c_int32)), cp.ctypes.data_as(P(ctypes.c_uint8)),
           own.ctypes.data_as(P(ctypes.c_uint8)))
    return rc, rep, g, ns, cp.astype(bool), own.astype(bool)


def _states(sector, n, seed):
    rng = np.random.default_rng(seed)
    N, n_up = sector.n_sites, sector.n_up
    out = []
    for t in range(n):
        sites = rng.choice(N, n_up, replace=False)
        if t % 2 == 0 and 0 not in sites and n_up:
            sites[0] = 0          # site 0 is the most significant bit
        out.append(sum(1 << (N - 1 - int(s)) for s in sites))
    reps, _ = oracle.basis(sector) if N <= 16 else (np.zeros(0, np.uint64), None)
    return np.array(out + [int(r) for r in reps[:50]], dtype=np.uint64)


SECTORS = {
    "square32_2x16": lambda: C.square32(),
    "square32_4x8": lambda: C.square32(n_sublat=4),
    "chain64_8x8": lambda: C.chain(64, 1.0, 0.3, translations=True, k=5, n_up=3),
    "kagome12_E1": lambda: C.kagome([[2, 0], [0, 2]], 1.0, 0.2, 0.3, irrep="E1"),
    "chain12_flip": lambda: C.chain(12, 1.0, 0.3, translations=True, spinflip=-1),
    "triangular24_M": lambda: C.triangular24_sectors()[7],
    "kagome36": lambda: C.kagome36(),
}


@pytest.mark.parametrize("name", sorted(SECTORS))
def test_host_search_matches_oracle(harness, name):
    p = SECTORS[name]()
    s = p.sector
    states = _states(s, 400, 5)
    ref = [oracle.rep(s, int(x)) for x in states]
    ran = 0
    for variant in (0, 1):
        rc, rep, g, ns, cp, own = _call(harness, s, states, variant)
        if variant == 1 and rc in (-1, -2):
            continue          # the specialised search covers 2..4 blocks with packed entries
        assert rc == 0, rc
        ran += 1
        for i, (r0, g0, n0, ssum) in enumerate(ref):
            assert int(rep[i]) == r0 and ns[i] == n0 and cp[i] == (abs(ssum) > 1e-9), (i, variant)
            assert oracle.apply(s, int(g[i]), int(states[i])) == r0
            assert own[i] == (r0 == int(states[i]))
    assert ran >= 1
    if s.n_sublat in (2, 3, 4):
        assert ran == 2
