#!/usr/bin/env python
"""Benchmark of the matrix-free H.x hot path (and Lanczos time-to-E0).

Default workload: the 40-site square cluster (a1=(6,2), a2=(-2,6)), J1=1,
J2=0.55, Sz=0, symmetry group T40 x C4 x Z2 (320 elements), sector
Gamma.A.even (D = 430,909,650), FP64 vectors -- the largest workload that fits
one GPU.  One "step" is one y = H x through the C ABI (ed_apply) on a seeded
synthetic x resident in HBM, on H's stored structure (ed_hamiltonian_store,
built once per Hamiltonian before the timed region; its build time is
reported and added to the time-to-E0); the matrix-free kernel is timed beside
it.  L2 is flushed (256 MB write) between timed steps.  `e2e` repeats the
measurement with x and y in pinned host memory (host->device copy, ed_apply,
device->host copy inside the timed region).  Further objects: the 32-site
square and 36-site chiral kagome workloads, FP64-vs-mixed Lanczos
time-to-E0, batched sectors, and the CPU oracle's rate.

--impl reference times the CPU oracle (brute-force representatives, FP64) on
bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "square32": ("square32 J1=1 J2=0.5 tilted (4,4)x(4,-4), T32xC4v, Gamma.A1, Sz=0, 2 blocks of 16 sites",
                 lambda: __import__("edinputs.configs", fromlist=["x"]).square32("A1", "Gamma")),
    "chain16": ("chain16 J1=1 periodic, no spatial symmetry, Sz=0",
                lambda: __import__("edinputs.configs", fromlist=["x"]).chain16()),
    "kagome36": ("kagome36 J1=1 J2=0.2 Jchi=0.3, T12xC6xZ2, Gamma.A.even, Sz=0",
                 lambda: __import__("edinputs.configs", fromlist=["x"]).kagome36()),
    "square40": ("square40 J1=1 J2=0.55 (6,2)x(-2,6), T40xC4xZ2, Gamma.A.even, Sz=0",
                 lambda: __import__("edinputs.configs", fromlist=["x"]).square40()),
}
METRIC = "H.x Gstate-bonds/s"
UNIT = "Gstate-bonds/s"
FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("ed_apply.cu", "ed_apply_impl.cuh", "ed_device.cuh", "ed_internal.h", "ed_cache.cu", "ed_cache.cuh",
              "ed_cache_lanes.cu"):
        h.update(open(os.path.join(ROOT, "paper_2210_03511_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, dtype: str, kernel: str):
    """DRAM bytes per H.x of `kernel` and ncu context counters from the committed
    summary, if it was taken on these kernel sources; else (None, {})."""
    p = os.path.join(ROOT, "profiles", "hx_traffic.txt")
    if not os.path.exists(p):
        return None, {}
    for line in open(p):
        f = line.split()
        if not f or f[0].startswith("#") or f[0] != f"{workload}:{dtype}:{kernel}":
            continue
        kv = dict(x.split("=", 1) for x in f[1:] if "=" in x)
        if kv.get("kernel_hash") != kernel_hash():
            return None, {}
        extra = {k: float(v) for k, v in kv.items() if k not in ("kernel_hash", "dram_bytes_per_launch")}
        return float(kv["dram_bytes_per_launch"]), extra
    return None, {}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_aggregate(t_dev: float, t_e2e: float, work_local: float, device=None):
    """Across ranks (independent replicas): the slowest rank's times and the summed work.

    Each rank runs the whole workload on its own GPU (the path is replicated,
    not sharded), so the job's throughput is the total work over the slowest
    rank's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_dev, t_e2e, work_local
    tt = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ww = torch.tensor([work_local], dtype=torch.float64, device=device)
    dist.all_reduce(ww, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(tt[1]), float(ww[0])


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ CPU oracle timing
def oracle_sample_states(problem, n: int, seed: int = 0) -> np.ndarray:
    """Random compatible representatives drawn by the oracle (no GPU data)."""
    import oracle
    rng = np.random.default_rng(seed)
    N, n_up = problem.sector.n_sites, problem.sector.n_up
    out = []
    while len(out) < n:
        bits = np.zeros(N, dtype=np.uint8)
        bits[rng.choice(N, n_up, replace=False)] = 1
        s = int("".join(map(str, bits)), 2)
        r, g, ns, ssum = oracle.rep(problem.sector, s)
        if abs(ssum) > 1e-9:
            out.append(r)
    return np.array(out, dtype=np.uint64)


def oracle_rate(problem, budget_s: float, cplx: bool):
    """Time oracle.rows on a bounded sample sized to ~budget_s; returns (Gstate-bonds/s, rows, seconds)."""
    import oracle
    n_terms = len(problem.terms.bonds) + len(problem.terms.tris)
    probe = oracle_sample_states(problem, 64, seed=1)
    t0 = time.perf_counter()
    oracle.rows(problem, probe, 7, cplx)
    per = max((time.perf_counter() - t0) / len(probe), 1e-7)
    n = int(max(16, min(200000, budget_s / per)))
    states = oracle_sample_states(problem, n, seed=2)
    t0 = time.perf_counter()
    oracle.rows(problem, states, 7, cplx)
    dt = time.perf_counter() - t0
    return n * n_terms / dt / 1e9, n, dt


def oracle_baseline(problem, budget_s: float, cplx: bool, D: int, n_apply=None) -> dict:
    """The cpu_baseline object: the oracle's matrix-free rows on all host cores
    (value), on one core (a quarter of the budget), and the full H.x and the
    FP64 Lanczos time-to-E0 extrapolated from the all-core rate (D rows per
    H.x, n_apply H.x per Lanczos run; the vector algebra is left out)."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    r, n, dt = oracle_rate(problem, budget_s, cplx)
    out = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} random representatives, oracle matrix-free rows, {dt:.1f} s"}
    try:
        oracle.set_num_threads(1)
        r1, n1, dt1 = oracle_rate(problem, budget_s / 4, cplx)
    finally:
        oracle.set_num_threads(cores)
    hx_s = D * dt / n
    out["single_core"] = {"value": r1, "sample": f"{n1} representatives, {dt1:.1f} s"}
    out["hx_seconds_extrapolated"] = hx_s
    if n_apply:
        out["time_to_E0_seconds_extrapolated"] = hx_s * n_apply
        out["extrapolation"] = f"D={D} rows per H.x from the all-core rate; {n_apply} H.x of the FP64 Lanczos run"
    return out


# ------------------------------------------------------------------ main
KINDS = {"f64": (8, "float64", 0), "f32": (4, "float32", 1), "c128": (16, "complex128", 3), "c64": (8, "complex64", 2)}


def _edt(pkg, dtype):
    return {"f64": pkg.ED_F64, "f32": pkg.ED_F32, "c128": pkg.ED_C128, "c64": pkg.ED_C64}[dtype]


def hx_timing(H, edt, x, y, steps, warmup, flush, stream, torch):
    """Per-launch times (ms) of `steps` ed_apply calls on device-resident x, y (CUDA
    events on the launching stream, L2 flushed between steps)."""
    for _ in range(warmup):
        H.apply_ptr(edt, x.data_ptr(), y.data_ptr(), 1, stream)
        flush.fill_(1.0)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        H.apply_ptr(edt, x.data_ptr(), y.data_ptr(), 1, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def stored_bytes(D, G, s_x):
    """Algorithmic bytes of one stored-structure H.x: per row |Stab| (2), the Ising
    part (8), x_i and y_i; per element its 4-byte entry and the gathered x_j."""
    return D * (2 + 8 + 2 * s_x) + G * (4 + s_x)


def matrix_free_bytes(D, G, s_x, s_st):
    """Algorithmic bytes of one matrix-free H.x: per row the state word, |Stab|, x_i
    and y_i; per gather x_j (lookup tables and Limits reads excluded)."""
    return D * (s_st + 2 + 2 * s_x) + G * s_x


def workload_config(problem, desc, dim):
    """The `config` object both arms print: the workload's identity (cluster,
    couplings, sector, its dimension) and the timing rule."""
    return {"workload": desc, "dim": int(dim),
            "n_terms": len(problem.terms.bonds) + len(problem.terms.tris), "n_sym": int(problem.sector.n_sym),
            "n_sublat": int(problem.sector.n_sublat),
            "l2": "GPU arm: L2 flushed (256 MB write) between timed steps; the inputs exceed L2 as well"}


def lanczos_pair(pkg, torch, H, real, D, stream, store_for, hx_fp64_s=None):
    """Time-to-E0 (1e-10) of the FP64 run and of the mixed run (FP32 vectors, FP64
    refinement), each on H's stored structure as store_for(dtype) prepares it
    (returning the seconds its build took, added to the run's time).  The FP64
    run is the thesis's plain three-term recursion (the ground energy needs no
    stored vectors); the mixed run needs its Ritz vector for the FP64 Rayleigh
    quotient and keeps its Lanczos vectors in host memory (NVLink-C2C) instead of
    running a second pass, or on the device where they fit.  With hx_fp64_s (the stored FP64 H.x time measured
    beside it) the FP64 run's time outside H.x is reported per step against the
    HBM roofline of the plain recursion's vector algebra: per step, dot_step
    reads v_n and w, axpy_norm_step reads w, v_n, v_(n-1) and writes w, scale_by
    reads w and writes v_(n+1): 8 D s_x bytes."""
    lz = {}
    for name, dt, refine in (("fp64", pkg.ED_F64 if real else pkg.ED_C128, False),
                             ("mixed", pkg.ED_F32 if real else pkg.ED_C64, True)):
        store_s = store_for(dt)
        # the mixed run's plain-recursion vectors (up to 301 of them) stay on the
        # device when they fit 70 % of the free memory, else they go to host memory
        free, _ = torch.cuda.mem_get_info()
        keep = 0 if not refine else (2 if 301 * D * (4 if real else 8) <= 0.7 * free else 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, rep = H.lanczos(n_eig=1, tol=1e-10, max_iter=300, dtype=dt, reorth=False, refine=refine,
                            raise_on_nonconv=False, stream=stream, host_vectors=keep)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        lz[name] = {"seconds": t + store_s, "lanczos_seconds": t, "store_seconds": store_s, "E0": float(ev[0]),
                    "iters": rep.iters, "reorth": False,
                    "lanczos_vectors": {0: "second pass or none", 1: "host memory", 2: "device memory"}[keep],
                    "max_iter": 300,
                    "converged": bool(rep.converged), "ritz": rep.ritz[0], "n_apply": rep.n_apply}
    if hx_fp64_s:
        f = lz["fp64"]
        s_x = 8 if real else 16
        rest = max(f["lanczos_seconds"] - f["n_apply"] * hx_fp64_s, 1e-9) / max(f["iters"], 1)
        b = 8 * D * s_x
        peak, kind = peaks()
        lz["fp64"]["vector_algebra"] = {
            "seconds_per_step": rest, "bytes_per_step": b, "achieved_gbs": b / rest / 1e9,
            "frac": b / rest / 1e9 / peak, "peak_source": f"{kind} hbm_gbs",
            "hx_share": f["n_apply"] * hx_fp64_s / f["lanczos_seconds"],
            "how": "(Lanczos wall time - n_apply x stored H.x time) / iterations; includes host work"}
    lz["mixed_minus_fp64"] = lz["mixed"]["E0"] - lz["fp64"]["E0"]
    lz["raw_fp32_minus_fp64"] = lz["mixed"]["ritz"] - lz["fp64"]["E0"]
    lz["mixed_speedup"] = lz["fp64"]["seconds"] / lz["mixed"]["seconds"]
    return lz


def workload_summary(pkg, torch, name, dtypes, stream, flush, steps=10, warmup=3):
    """Sub-object for a further workload: per dtype the H.x time on the stored
    structure and matrix-free, their fractions of the HBM roofline, and the
    FP64-vs-mixed time-to-E0."""
    from edinputs.vectors import state_vector
    desc, make = WORKLOADS[name]
    problem = make()
    n_terms = len(problem.terms.bonds) + len(problem.terms.tris)
    real = problem.sector.is_real and problem.terms.is_real
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    basis = pkg.Basis(problem.sector, stream=stream)
    t_basis = time.perf_counter() - t0
    H = pkg.Hamiltonian(basis, problem.terms)
    D = basis.dim
    reps, _ = basis.export()
    X = state_vector(7, reps, complex_=not real)
    peak, _ = peaks()
    s_st = 4 if problem.sector.n_sites <= 32 else 8
    out = {"workload": desc, "dim": D, "basis_build_s": round(t_basis, 3)}
    for dtype in dtypes:
        s_x, tname, _ = KINDS[dtype]
        edt = _edt(pkg, dtype)
        x = torch.tensor(X, device=dev).to(getattr(torch, tname))
        y = torch.empty_like(x)
        ms_free = hx_timing(H, edt, x, y, max(2, steps // 2), warmup, flush, stream, torch)
        G, _ = H.counters(stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seg, _ = H.store_autotune(edt, stream=stream)  # segment size chosen by timing
        torch.cuda.synchronize()
        t_store = time.perf_counter() - t0
        info = H.store_info()
        ms = hx_timing(H, edt, x, y, steps, warmup, flush, stream, torch)
        t_s, t_f = statistics.mean(ms) / 1e3, statistics.mean(ms_free) / 1e3
        out[dtype] = {"ms_per_step": t_s * 1e3, "value": D * n_terms / t_s / 1e9, "unit": UNIT,
                      "frac": stored_bytes(D, G, s_x) / t_s / 1e9 / peak,
                      "store": {"autotune_seconds": round(t_store, 3), "seg_log2": seg,
                                "lanes_per_row": H.store_schedule()["lanes_per_row"], "bytes": info["bytes"],
                                "segments": info["segments"], "codes": info["codes"]},
                      "matrix_free": {"ms_per_step": t_f * 1e3, "value": D * n_terms / t_f / 1e9,
                                      "frac": matrix_free_bytes(D, G, s_x, s_st) / t_f / 1e9 / peak}}
        H.store_free()
        del x, y
        torch.cuda.empty_cache()
    seg_of = {_edt(pkg, dt): (out[dt]["store"]["seg_log2"], out[dt]["store"]["lanes_per_row"]) for dt in dtypes}

    def store_for(edt):  # the structure with the schedule tuned for this dtype
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H.store(edt, seg_log2=seg_of[edt][0], stream=stream)
        if seg_of[edt][1] > 1:
            H.store_set_lanes(seg_of[edt][1])
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    fp64_dt = "f64" if real else "c128"
    hx64 = out[fp64_dt]["ms_per_step"] / 1e3 if fp64_dt in out else None
    out["lanczos_time_to_E0"] = lanczos_pair(pkg, torch, H, real, D, stream, store_for, hx64)
    H.close()
    basis.close()
    torch.cuda.empty_cache()
    return out


def sun_summary(pkg, torch, stream, flush, steps=10, warmup=3):
    """SU(3) exchange model on the 21-site triangular torus (T21 x C6, 7 sites of each
    colour, d-ary colours packed in 2 bits a site): basis and stored-structure build,
    H.x (FP64, FP32) and FP64-vs-mixed time-to-E0."""
    from edinputs import configs as EC
    from edinputs.vectors import state_vector
    p = EC.sun_triangular21()
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    b = pkg.BasisSUN(p.sector, stream=stream)
    t_basis = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = pkg.Hamiltonian(b, p.terms, stream=stream)  # builds the stored structure
    torch.cuda.synchronize()
    t_store = time.perf_counter() - t0
    reps, _ = b.export()
    X = state_vector(7, reps)
    n_terms = len(p.terms.bonds)
    out = {"workload": "SU(3) exchange model, triangular 21 sites (4,1)x(-1,5), T21xC6, Gamma.A, 7 sites per colour",
           "dim": b.dim, "basis_build_s": round(t_basis, 3), "store_s": round(t_store, 3),
           "store_bytes": H.store_info()["bytes"]}
    G = H.store_info()["entries"]
    peak, _ = peaks()
    for dtype in ("f64", "f32"):
        s_x, tname, _ = KINDS[dtype]
        x = torch.tensor(X, device=dev).to(getattr(torch, tname))
        y = torch.empty_like(x)
        ms = hx_timing(H, _edt(pkg, dtype), x, y, steps, warmup, flush, stream, torch)
        t = statistics.mean(ms) / 1e3
        out[dtype] = {"ms_per_step": t * 1e3, "value": b.dim * n_terms / t / 1e9, "unit": UNIT,
                      "frac": stored_bytes(b.dim, G, s_x) / t / 1e9 / peak}
    out["lanczos_time_to_E0"] = lanczos_pair(pkg, torch, H, True, b.dim, stream, lambda edt: t_store,
                                             out["f64"]["ms_per_step"] / 1e3)
    H.close()
    b.close()
    torch.cuda.empty_cache()
    return out


def batching_measurement(pkg, torch, stream):
    """Ground energy of every (k, rho_k) sector of the 24-site triangular torus
    (36 sectors, J1=1, J2=0.125, Sz=0): one Lanczos run per sector in sequence
    against one batched Lanczos run over all sectors (every step one persistent
    H.x launch for all sectors, the step replayed as a CUDA graph), with one
    vector per sector (plain recursion or full reorthogonalisation) and with a
    block of 8 seeded Gaussian vectors; FP64 vectors, and FP32 vectors (FP32
    block Gram-Schmidt, FP64 refinement: keys ending in _fp32)."""
    from edinputs import configs as EC
    probs = EC.triangular24_sectors()
    bases = [pkg.Basis(p.sector, stream=stream) for p in probs]
    hs = [pkg.Hamiltonian(b, p.terms) for b, p in zip(bases, probs)]
    # every sector's structure stored once (the sequential runs and the batch use it)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in hs:
        h.store(stream=stream)
    torch.cuda.synchronize()
    t_store = time.perf_counter() - t0
    t0 = time.perf_counter()
    seq = []
    for h in hs:
        dt = pkg.ED_F64 if h.is_real else pkg.ED_C128
        ev, _ = h.lanczos(n_eig=1, tol=1e-10, max_iter=300, dtype=dt, reorth=True, refine=False,
                          raise_on_nonconv=False, stream=stream)
        seq.append(float(ev[0]))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    batch = pkg.Batch(hs)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"workload": "triangular 24 sites, all 36 (k, rho_k) sectors, J2=0.125, Sz=0",
           "total_dim": int(batch.total), "store_s": t_store, "hx_path": "stored structure of every sector",
           "sequential_s": t_seq, "E0_min": min(seq)}
    for blk, reorth, fp32 in ((1, False, False), (1, True, False), (8, True, False), (1, True, True),
                              (8, True, True)):
        tdt, edt = (torch.complex64, pkg.ED_C64) if fp32 else (torch.complex128, pkg.ED_C128)
        x = torch.zeros(blk * batch.total, dtype=tdt, device=dev)
        waves = batch.autotune(x, torch.empty_like(x), nvec=blk)
        del x
        max_it = 300 if blk == 1 else 80
        # blocks: the host's band eigensolve (all sectors) takes longer than a GPU step,
        # so the values are checked every 4 steps (at most 3 steps past convergence)
        every = 1 if blk == 1 else 4
        if blk == 1:  # warm-up run (the block-8 run is long enough to carry its own set-up)
            batch.lanczos(block=blk, n_eig=1, tol=1e-10, max_iter=max_it, seed=3, use_graph=True,
                          raise_on_nonconv=False, reorth=reorth, dtype=edt, check_every=every)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, rep = batch.lanczos(block=blk, n_eig=1, tol=1e-10, max_iter=max_it, seed=3, use_graph=True,
                                raise_on_nonconv=False, reorth=reorth, dtype=edt, check_every=every)
        torch.cuda.synchronize()
        t_bat = time.perf_counter() - t0
        diff = max(abs(float(ev[s, 0]) - seq[s]) for s in range(len(hs)))
        key = f"block{blk}_{'reorth' if reorth else 'plain'}" + ("_fp32" if fp32 else "")
        out[key] = {
            "batched_graph_s": t_bat, "speedup_vs_sequential": t_seq / t_bat, "iters": rep.iters,
            "check_every": every,
            "step_seconds": rep.step_seconds, "converged_sectors": rep.converged_sectors,
            "max_abs_E0_diff": diff, "autotuned_waves": waves}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="square40", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "c128", "c64"])
    ap.add_argument("--no-lanczos", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads' sub-objects and batching")
    ap.add_argument("--matrix-free", action="store_true", help="time the matrix-free kernel only (no stored structure)")
    ap.add_argument("--seg-log2", type=int, default=0,
                    help="log2 column-segment size of the stored structure (0: the library's default)")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per row of the stored pass (1, 2, 4, 8)")
    ap.add_argument("--autotune", action="store_true",
                    help="segment size and lanes per row chosen by ed_hamiltonian_store_autotune (square40: the "
                         "library default, found in about 30 s)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    desc, make = WORKLOADS[args.workload]
    problem = make()
    n_terms = len(problem.terms.bonds) + len(problem.terms.tris)
    real = problem.sector.is_real and problem.terms.is_real
    dtype = args.dtype
    if not real and dtype in ("f64", "f32"):
        dtype = "c128" if dtype == "f64" else "c64"

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        budget = max(0.05, 60.0 / (args.steps + args.warmup))
        rates = []
        tot_rows = 0
        for i in range(args.warmup + args.steps):
            r, n, dt = oracle_rate(problem, budget, not real)
            if i >= args.warmup:
                rates.append(r)
                tot_rows += n
        v = statistics.median(rates)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(problem, desc, oracle.sector_dim_formula(problem.sector)),
                "run": {"rows_per_step_sample": tot_rows // max(1, args.steps), "host": "CPU oracle"},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": f"oracle matrix-free rows on ~{budget:.2f} s random representative samples per step"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2210_03511_gb300 import build as libbuild
    libbuild.build()
    import paper_2210_03511_gb300 as pkg
    from edinputs.vectors import state_vector

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    basis = pkg.Basis(problem.sector, stream=stream)
    t_basis = time.perf_counter() - t0
    H = pkg.Hamiltonian(basis, problem.terms)
    D = basis.dim
    reps, _ = basis.export()
    s_x, tname, _ = KINDS[dtype]
    edt = _edt(pkg, dtype)
    X = state_vector(7, reps, complex_=not real)
    x = torch.tensor(X, device=dev).to(getattr(torch, tname))
    y = torch.empty_like(x)
    del X
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    s_st = 4 if problem.sector.n_sites <= 32 else 8
    peak, peak_kind = peaks()
    # the matrix-free kernel first (its gather counter sizes the algorithmic bytes)
    ms_free = hx_timing(H, edt, x, y, max(3, args.steps // 4), args.warmup, flush, stream, torch)
    gathers, skipped = H.counters(stream)
    y_free = y.clone() if not args.matrix_free else None
    store = None
    if not args.matrix_free:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        autotune = args.autotune
        if autotune:  # segment size and lanes per row chosen by timing (outside the timed region)
            H.store_autotune(edt, stream=stream)
        else:
            H.store(edt, seg_log2=args.seg_log2, stream=stream)
            if args.lanes > 1:
                H.store_set_lanes(args.lanes)
        torch.cuda.synchronize()
        t_store = time.perf_counter() - t0
        info = H.store_info()
        sch = H.store_schedule()
        store = {"seconds": round(t_store, 3), "bytes": info["bytes"], "segments": info["segments"],
                 "codes": info["codes"], "entries": info["entries"],
                 "seg_log2": sch["seg_log2"], "lanes_per_row": sch["lanes_per_row"],
                 "schedule": "autotuned (ed_hamiltonian_store_autotune)" if autotune else
                             ("given" if args.seg_log2 or args.lanes else "library default")}
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd and cvd.replace(",", "").isdigit():
        gpu_index = int(cvd.split(",")[local])
    clk = ClockSampler(gpu_index)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    ms = hx_timing(H, edt, x, y, args.steps, args.warmup, flush, stream, torch)
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    t_dev = sum(ms) / 1e3
    stored_diff = None
    if y_free is not None:
        # the stored structure gives the matrix-free H x up to the summation order across segments
        stored_diff = (y - y_free).abs().max().item() / max(y_free.abs().max().item(), 1e-300)
        del y_free
    # e2e: pinned host x -> device, ed_apply, device -> host, every step
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        e_s[i].record(stream)
        x.copy_(xh, non_blocking=True)
        H.apply_ptr(edt, x.data_ptr(), y.data_ptr(), 1, stream)
        yh.copy_(y, non_blocking=True)
        e_e[i].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_e2e = sum(s.elapsed_time(e) for s, e in zip(e_s, e_e)) / 1e3
    assert torch.equal(yh, y.cpu()), "e2e result differs from device-resident result"
    h2d, d2h = int(x.numel() * x.element_size()), int(y.numel() * y.element_size())
    del xh, yh
    t_dev, t_e2e, work = replica_aggregate(t_dev, t_e2e, float(D * n_terms * args.steps), device=dev)
    value = work / t_dev / 1e9
    e2e = work / t_e2e / 1e9
    t_launch = sum(ms) / 1e3 / args.steps
    t_free = statistics.mean(ms_free) / 1e3
    b_free = matrix_free_bytes(D, gathers, s_x, s_st)
    if args.matrix_free:
        b_alg, kernel = b_free, "hx_kernel"
    else:
        b_alg = stored_bytes(D, gathers, s_x)
        kernel = "cache_pass_lanes" if store["lanes_per_row"] > 1 else "cache_pass_kernel"
    achieved = b_alg / t_launch / 1e9
    traffic, ncu_ctx = profiled_traffic(args.workload, dtype, kernel)
    launches_per_step = 1 if args.matrix_free else store["segments"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": workload_config(problem, desc, D),
            "run": {"hx_path": "matrix-free" if args.matrix_free else
                    "stored structure (built once per Hamiltonian with the schedule in `store`, outside the "
                    "timed region)",
                    "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                    "basis_build_s": round(t_basis, 3)},
            "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "ncu_context": ncu_ctx,
                         "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": b_alg,
                         "gathers_per_launch": gathers, "incompatible_images_per_launch": skipped,
                         "launches_per_step": launches_per_step,
                         "dram_achieved": (traffic / t_launch / 1e9) if traffic else None,
                         "dram_frac": (traffic / t_launch / 1e9 / peak) if traffic else None},
            "matrix_free": {"ms_per_step": t_free * 1e3, "value": D * n_terms / t_free / 1e9,
                            "achieved": b_free / t_free / 1e9, "frac": b_free / t_free / 1e9 / peak},
            "store": store,
            "stored_vs_matrix_free_max_rel_diff": stored_diff,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clocks,
            "wall_s_timed_region": wall}
    del x, y, flush
    torch.cuda.empty_cache()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # the further measurements must not hide the headline: a failure is recorded, not raised
    if not args.no_lanczos and rank == 0:
        if args.matrix_free:
            t_store = 0.0
        try:
            # one structure serves both runs (FP64 and FP32 segments are the same size here)
            hx64 = t_launch if dtype in ("f64", "c128") and not args.matrix_free else None
            line["lanczos_time_to_E0"] = lanczos_pair(pkg, torch, H, real, D, stream, lambda edt: t_store, hx64)
        except Exception as e:
            line["lanczos_time_to_E0"] = {"error": repr(e)}
    H.close()
    basis.close()
    torch.cuda.empty_cache()
    if not args.no_extra and rank == 0:
        extra = {}
        for name, dts in (("square32", ["f64", "f32"]), ("kagome36", ["c64", "c128"])):
            if name != args.workload:
                try:
                    extra[name] = workload_summary(pkg, torch, name, dts, stream, flush)
                except Exception as e:
                    extra[name] = {"error": repr(e)}
                torch.cuda.empty_cache()
        try:
            extra["su3_triangular21"] = sun_summary(pkg, torch, stream, flush)
        except Exception as e:
            extra["su3_triangular21"] = {"error": repr(e)}
        line["other_workloads"] = extra
        if not args.no_lanczos:
            try:
                line["batching_time_to_E0"] = batching_measurement(pkg, torch, stream)
            except Exception as e:
                line["batching_time_to_E0"] = {"error": repr(e)}
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            n_apply = line.get("lanczos_time_to_E0", {}).get("fp64", {}).get("n_apply")
            line["cpu_baseline"] = oracle_baseline(problem, args.cpu_budget, not real, D, n_apply)
        except Exception as e:  # the CPU baseline must not hide the GPU number
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"failed: {e}"}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
