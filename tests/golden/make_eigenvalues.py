#!/usr/bin/env python
"""Write tests/golden/eigenvalues.json: the oracle's lowest eigenvalues of the
workload sectors that are too large for the test suite to rebuild on the fly.

Only the CPU oracle (`oracle/`) and the seeded input generator (`edinputs/`)
are used: the basis by brute-force enumeration, the sparse matrix in that
basis from local operators (`oracle.csr_chunked`, the column-wise assembly of
`oracle.csr` on several threads), and ARPACK (`oracle.lowest_eigs`, tol 1e-13)
as a library step.  Nothing here touches the CUDA library.

    python tests/golden/make_eigenvalues.py [square32_A1] [square32_E1] [triangular24]

With no arguments every set is computed.  Existing entries of the JSON file
for sets not named are kept.  Runtime on 8 host cores: one to two hours for
each 32-site sector (the brute-force representatives apply all 256 or 128
group elements to every one of the C(32,16) = 6.0e8 states; the matrix takes
about twenty minutes more), a few minutes for the 36 triangular sectors.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from edinputs import configs as C  # noqa: E402

OUT = os.path.join(HERE, "eigenvalues.json")
TOL = 1e-13


def square32_complex():
    """Gamma, irrep E1 of T32 x C4 (C4 character +i): the complex sector that carries
    C4v's two-dimensional irrep E at Gamma."""
    return C.square([[4, 4], [4, -4]], 1.0, 0.5, k=(0.0, 0.0), irrep="E1", point="rot", n_sublat=2,
                    max_table_bytes=4 << 20)


def solve(problem, k):
    t0 = time.time()
    reps, stab = oracle.basis(problem.sector)
    t1 = time.time()
    real = bool(problem.sector.is_real and problem.terms.is_real)
    H = oracle.csr_chunked(problem, reps, stab, real=real)
    t2 = time.time()
    ev = oracle.lowest_eigs(H, k, tol=TOL)
    t3 = time.time()
    return {"dim": int(len(reps)), "nnz": int(H.nnz), "real": real, "k": k,
            "eigenvalues": [float(v) for v in ev],
            "seconds": {"basis": round(t1 - t0, 1), "matrix": round(t2 - t1, 1), "arpack": round(t3 - t2, 1)}}


def square32_A1():
    return {"square32 Gamma.A1": dict(solve(C.square32(), 3),
                                      workload="square32 J1=1 J2=0.5, a1=(4,4) a2=(4,-4), T32 x C4v, Gamma.A1, Sz=0")}


def square32_E1():
    return {"square32 Gamma.E1 (T32xC4)": dict(solve(square32_complex(), 3),
                                               workload="square32 J1=1 J2=0.5, a1=(4,4) a2=(4,-4), T32 x C4, "
                                                        "Gamma, C4 character +i, Sz=0")}


def triangular24():
    out = {}
    for p in C.triangular24_sectors():
        name = f"triangular24 {p.meta['sector']}"
        out[name] = dict(solve(p, 2), workload="triangular24 J1=1 J2=0.125, a1=(5,1) a2=(4,-4), T24 x C2v "
                                               f"sector {p.meta['sector']}, Sz=0")
        print(name, out[name]["dim"], out[name]["eigenvalues"], flush=True)
    return out


SETS = {"square32_A1": square32_A1, "square32_E1": square32_E1, "triangular24": triangular24}


def main(argv):
    names = argv or list(SETS)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data.setdefault("_about", "lowest eigenvalues from the CPU oracle: brute-force basis, sparse matrix from "
                              "local operators, ARPACK (scipy eigsh, which='SA', tol=1e-13); written by "
                              "tests/golden/make_eigenvalues.py")
    for n in names:
        oracle.build()
        res = SETS[n]()
        data.update(res)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(n, "done", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
