#!/usr/bin/env python
"""Benchmark of the matrix-free H.x hot path (and Lanczos time-to-E0).

Default workload: the 32-site tilted square cluster (a1=(4,4), a2=(4,-4)),
J1=1, J2=0.5, Sz=0, symmetry group T32 x C4v (256 elements), sector Gamma.A1,
FP64 vectors.  One "step" is one y = H x through the C ABI (ed_apply) on a
seeded synthetic x resident in HBM; L2 is flushed (256 MB write) between
timed steps.  `e2e` repeats the measurement with x and y in pinned host memory
(host->device copy, ed_apply, device->host copy inside the timed region).

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
    for f in ("ed_apply.cu", "ed_apply_impl.cuh", "ed_device.cuh", "ed_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2210_03511_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, dtype: str):
    """DRAM bytes per launch of the H.x kernel and ncu context counters from the
    committed summary, if it was taken on these kernel sources; else (None, {})."""
    p = os.path.join(ROOT, "profiles", "hx_traffic.txt")
    if not os.path.exists(p):
        return None, {}
    for line in open(p):
        f = line.split()
        if not f or f[0].startswith("#") or f[0] != f"{workload}:{dtype}":
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
def batching_measurement(pkg, torch, stream):
    """Ground energy of every (k, rho_k) sector of the 24-site triangular torus
    (36 sectors, J1=1, J2=0.125, Sz=0): one Lanczos run per sector in sequence
    against one batched Lanczos run over all sectors (every step one persistent
    H.x launch for all sectors, the step replayed as a CUDA graph), with one
    vector per sector (plain recursion or full reorthogonalisation) and with a
    block of 8 seeded Gaussian vectors."""
    from edinputs import configs as EC
    probs = EC.triangular24_sectors()
    bases = [pkg.Basis(p.sector, stream=stream) for p in probs]
    hs = [pkg.Hamiltonian(b, p.terms) for b, p in zip(bases, probs)]
    torch.cuda.synchronize()
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
           "total_dim": int(batch.total), "sequential_s": t_seq, "E0_min": min(seq)}
    for blk, reorth in ((1, False), (1, True), (8, True)):
        x = torch.zeros(blk * batch.total, dtype=torch.complex128, device=dev)
        waves = batch.autotune(x, torch.empty_like(x), nvec=blk)
        del x
        max_it = 300 if blk == 1 else 80
        if blk == 1:  # warm-up run (the block-8 run is long enough to carry its own set-up)
            batch.lanczos(block=blk, n_eig=1, tol=1e-10, max_iter=max_it, seed=3, use_graph=True,
                          raise_on_nonconv=False, reorth=reorth)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, rep = batch.lanczos(block=blk, n_eig=1, tol=1e-10, max_iter=max_it, seed=3, use_graph=True,
                                raise_on_nonconv=False, reorth=reorth)
        torch.cuda.synchronize()
        t_bat = time.perf_counter() - t0
        diff = max(abs(float(ev[s, 0]) - seq[s]) for s in range(len(hs)))
        out[f"block{blk}_{'reorth' if reorth else 'plain'}"] = {
            "batched_graph_s": t_bat, "speedup_vs_sequential": t_seq / t_bat, "iters": rep.iters,
            "step_seconds": rep.step_seconds, "converged_sectors": rep.converged_sectors,
            "max_abs_E0_diff": diff, "autotuned_waves": waves}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="square32", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "c128", "c64"])
    ap.add_argument("--no-lanczos", action="store_true")
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
                "config": {"workload": desc, "rows_per_step_sample": tot_rows // max(1, args.steps)},
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
    tdt = {"f64": torch.float64, "f32": torch.float32, "c128": torch.complex128, "c64": torch.complex64}[dtype]
    edt = {"f64": pkg.ED_F64, "f32": pkg.ED_F32, "c128": pkg.ED_C128, "c64": pkg.ED_C64}[dtype]
    X = state_vector(7, reps, complex_=not real)
    x = torch.tensor(X, device=dev).to(tdt)
    y = torch.empty_like(x)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        H.apply_ptr(edt, x.data_ptr(), y.data_ptr(), 1, stream)
        flush.fill_(1.0)
    torch.cuda.synchronize()
    gathers, skipped = H.counters(stream)
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd and cvd.replace(",", "").isdigit():
        gpu_index = int(cvd.split(",")[local])
    clk = ClockSampler(gpu_index)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        H.apply_ptr(edt, x.data_ptr(), y.data_ptr(), 1, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_dev = sum(ms) / 1e3
    # e2e: pinned host x -> device, ed_apply, device -> host, every step
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    yd = torch.empty_like(x)
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        e_s[i].record(stream)
        xd.copy_(xh, non_blocking=True)
        H.apply_ptr(edt, xd.data_ptr(), yd.data_ptr(), 1, stream)
        yh.copy_(yd, non_blocking=True)
        e_e[i].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_e2e = sum(s.elapsed_time(e) for s, e in zip(e_s, e_e)) / 1e3
    assert torch.equal(yh, y.cpu()), "e2e result differs from device-resident result"
    # aggregate over ranks (replicas)
    t_dev, t_e2e, work = replica_aggregate(t_dev, t_e2e, float(D * n_terms * args.steps), device=dev)
    value = work / t_dev / 1e9
    e2e = work / t_e2e / 1e9
    # roofline of the H.x kernel: algorithmic bytes per launch
    s_x = {"f64": 8, "f32": 4, "c128": 16, "c64": 8}[dtype]
    s_st = 4 if problem.sector.n_sites <= 32 else 8
    b_alg = D * (s_st + 2 + 2 * s_x) + gathers * s_x
    per_launch = t_dev / args.steps / ws * ws  # seconds per launch on one GPU
    achieved = b_alg / (sum(ms) / 1e3 / args.steps) / 1e9
    peak, peak_kind = peaks()
    traffic, ncu_ctx = profiled_traffic(args.workload, dtype)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": desc, "dim": D, "n_terms": n_terms, "n_sym": int(problem.sector.n_sym),
                       "n_sublat": int(problem.sector.n_sublat), "l2": "flushed: 256 MB write between timed steps",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "basis_build_s": round(t_basis, 4)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "ncu_context": ncu_ctx,
                         "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": b_alg,
                         "gathers_per_launch": gathers, "incompatible_images_per_launch": skipped,
                         # the DRAM bytes the launch really moves (ncu, same kernel sources) over the
                         # same launch time: each gather costs whole random sectors, not s_x bytes
                         "dram_achieved": (traffic / (sum(ms) / 1e3 / args.steps) / 1e9) if traffic else None,
                         "dram_frac": (traffic / (sum(ms) / 1e3 / args.steps) / 1e9 / peak) if traffic else None},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(x.numel() * x.element_size()),
                    "d2h_bytes_per_step": int(y.numel() * y.element_size())},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "wall_s_timed_region": wall}
    if not args.no_lanczos and rank == 0:
        lz = {}
        # full reorthogonalisation while the stored vectors of the run's own dtype take
        # under 180 GB of HBM, else the plain recursion (ghost-filtered, Ritz vectors
        # from a second pass): FP32 vectors halve that memory, one of the gains of
        # the mixed-precision run
        for name, dt, refine in (("fp64", pkg.ED_F64 if real else pkg.ED_C128, False),
                                 ("mixed", pkg.ED_F32 if real else pkg.ED_C64, True)):
            s_vec = {pkg.ED_F64: 8, pkg.ED_F32: 4, pkg.ED_C128: 16, pkg.ED_C64: 8}[dt]
            # stored vectors are allocated for max_iter steps up front: 300 if they fit;
            # FP32 vectors (reorthogonalised in FP32 arithmetic, cheap) also 100 (the runs
            # here converge in under 80 steps); else no storage (FP64 Gram-Schmidt on the
            # large sectors costs more than the plain recursion saves)
            sizes = (300, 100) if refine else (300,)
            reorth, max_it = next(((True, m) for m in sizes if m * D * s_vec < 180e9), (False, 300))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, rep = H.lanczos(n_eig=1, tol=1e-10, max_iter=max_it, dtype=dt, reorth=reorth,
                                refine=refine, raise_on_nonconv=False, stream=stream)
            torch.cuda.synchronize()
            lz[name] = {"seconds": time.perf_counter() - t0, "E0": float(ev[0]), "iters": rep.iters, "reorth": reorth, "max_iter": max_it,
                        "converged": bool(rep.converged), "ritz": rep.ritz[0], "n_apply": rep.n_apply}
        lz["mixed_minus_fp64"] = lz["mixed"]["E0"] - lz["fp64"]["E0"]
        lz["raw_fp32_minus_fp64"] = lz["mixed"]["ritz"] - lz["fp64"]["E0"]
        line["lanczos_time_to_E0"] = lz
    if not args.no_lanczos and rank == 0:
        line["batching_time_to_E0"] = batching_measurement(pkg, torch, stream)
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
