#!/usr/bin/env python
"""Benchmark of the batched shared-LHS banded solve on GB300.

Workload: pentadiagonal A = I + 0.1 D4 ([1, -4, 6, -4, 1] stencil, first and
last two rows clamped), N = 512 rows, M = 65536 systems per GPU, interleaved
(B[i*M + j]), RHS ~ N(0, 1), FP64.  One step is one pass of every row of the
hot path over that batch:
  1. the plain FP64 solve (forward + backward sweep, FP64 arithmetic),
  2. the mixed-precision solve: B stored in FP32, FP32 sweeps, one step of
     iterative refinement with an FP64-accurate residual, FP64 result,
  3. the adjoint solve A^{-T} G and the band-gradient reduction over the batch.
The FP64 and adjoint solves work in place on the previous step's result
(implicit time stepping: X <- A^{-1} X), so no copy is needed between steps;
every FP64 operand (256 MiB) is larger than L2 and the FP32 input (128 MiB)
is re-read only after >= 1 GiB of other traffic, so L2 is not flushed.

``value`` is unknowns solved per second over the whole job: 3 * N * M per GPU
per step, summed over GPUs, divided by the slowest rank's time.

``--impl reference`` times the plain CPU FP64 oracle on the same kind of step
(a bounded column sample) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ROWS, M_SYS, S_HYPER = 512, 65536, 0.1
METRIC = "unknowns/s & HBM GB/s vs 8 TB/s at stated rel err; serving p50/p99 latency"
WORKLOAD = ("penta A=I+0.1*D4 clamped, N=512, M=65536 RHS ~ N(0,1) per GPU, interleaved; "
            "step = FP64 solve + FP32-stored solve with one FP64-accurate refinement step + "
            "FP64 adjoint solve + band-gradient reduction, in that order on one stream")
NOMINAL_HBM_GBS = 8000.0


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# step's kernels from one ncu capture of this workload, valid only while the
# kernel sources (for the sweeps also the launch policy in solve_api.cu, which
# sets their grid) hash to the value they had at capture time.
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch of the kernel
    # inside this benchmark's step (launch list of the timed steps), keyed by
    # the hash of its sources
    "band_grad_f64": {"bytes": 546271744 + 125184, "sha": "7ad65a6ac4c1fb1b"},
    "f64_solve": {"bytes": 470340608 + 431424768, "sha": "9c678e6d1456bd9a"},
    "adjoint_f64": {"bytes": 463214848 + 427328768, "sha": "9c678e6d1456bd9a"},
    "refine_solve": {"bytes": 347321600 + 428031232, "sha": "85b7f7b0d60a8d88"},
}
KERNEL_SOURCES = {
    "f64_solve": ["sweep_df.cu", "df_sweep.cuh", "df_math.cuh", "sweep_kernels.cuh", "internal.h", "solve_api.cu"],
    "adjoint_f64": ["sweep_df.cu", "df_sweep.cuh", "df_math.cuh", "sweep_kernels.cuh", "internal.h",
                    "solve_api.cu"],
    "refine_solve": ["refine.cu", "refine_math.cuh", "sweep_kernels.cuh", "internal.h"],
    "band_grad_f64": ["band_grad.cu", "df_math.cuh", "refine_math.cuh", "sweep_kernels.cuh", "internal.h"],
}


def sources_sha(path_name: str) -> str:
    import hashlib

    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[path_name]:
        with open(os.path.join(ROOT, "paper_1909_04539_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(path_name: str):
    t = NCU_TRAFFIC.get(path_name)
    if t and t["sha"] == sources_sha(path_name):
        return t["bytes"]
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "MEASURED_PEAKS.json (measured copy bandwidth of this GPU model)"
    except OSError:
        return {"hbm_gbs": 6800.0}, "profiling-recipe fallback 6.8 TB/s"


# ------------------------------------------------------------------ clocks

REASON_COLS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed
    region."""

    def __init__(self, device_index: int):
        self.proc = None
        self.lines = []
        exe = shutil.which("nvidia-smi")
        if exe is None:
            return
        import torch
        p = torch.cuda.get_device_properties(device_index)
        ident = str(device_index)
        try:
            ident = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        except AttributeError:
            pass
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.cmd = [exe, f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50", "-i", ident]

    def __enter__(self):
        if getattr(self, "cmd", None):
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            time.sleep(0.15)
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=2)

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(REASON_COLS, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks


def rank_seeds(rank: int):
    """Per-rank seeds of the RHS and of the upstream gradient (weak scaling:
    every rank solves its own systems)."""
    return rank, 1000 + rank


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (all ranks get it)."""
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms_step: float) -> float:
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return units_per_rank * world / (ms_step * 1e-3)


# ------------------------------------------------------------------ ours


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1909_04539_gb300 import build as libbuild
    if rank == 0 or world == 1:
        libbuild.build()
    if world > 1:
        dist.barrier()
    import paper_1909_04539_gb300 as bs
    import synth

    N, M = N_ROWS, M_SYS
    bands = synth.clamped_hyperdiffusion_bands(N, S_HYPER)
    f = bs.Factor(bands)
    seed_b, seed_g = rank_seeds(rank)
    X64 = synth.normal_rhs(N, M, seed_b, "cuda")
    B0 = X64.clone()
    B32 = X64.float()
    XR = torch.empty((N, M), dtype=torch.float64, device="cuda")
    G = synth.uniform_rhs(N, M, seed_g, "cuda")
    db = torch.empty((5, N), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

    # accuracy: the first solve of this rank's batch, kept on sampled columns
    # for the oracle comparison in the CPU-baseline leg, and checked on every
    # system through the FP64 residual |B - A X| / |B| (torch ops)
    Xchk = B0.clone()
    bs.solve(f, Xchk)
    X32chk = B0.float()
    bs.solve(f, X32chk)
    XRchk = bs.solve_refine(f, B32)
    torch.cuda.synchronize()
    cols = np.random.default_rng(7).choice(M, 1024, replace=False)
    B32d = B32.double()
    sample = {"cols": cols, "B": B0[:, cols].cpu().numpy(), "B_all": B0.cpu().numpy(),
              "X64": Xchk[:, cols].cpu().numpy(),
              "X32": X32chk[:, cols].double().cpu().numpy(), "B32": B32d[:, cols].cpu().numpy(),
              "XR": XRchk[:, cols].cpu().numpy()}
    resid = {"f64_solve": rel_residual(bands, B0, Xchk), "f32_solve": rel_residual(bands, B0, X32chk.double()),
             "refine_solve": rel_residual(bands, B32d, XRchk)}
    del Xchk, X32chk, XRchk, B32d

    names = ["f64_solve", "refine_solve", "adjoint_f64", "band_grad_f64"]
    # per step and path: a start and an end event on the path's own stream
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in names]
          for _ in range(args.steps)]
    # The four kernels run in order on one stream.  (The mixed-precision
    # solve is independent of the others; run beside them on a second,
    # low-priority stream it saved nothing -- each kernel fills the GPU's
    # issue slots or its FP64 pipe on its own, 0.889 ms per step either way
    # -- and its sharing of the SMs stretched the other kernels' in-step
    # durations.)
    s_chain = torch.cuda.Stream()
    s_ref = s_chain
    fork = [torch.cuda.Event() for _ in range(2)]

    def timed(e, q, stream, fn):
        if e: e[q][0].record(stream)
        fn()
        if e: e[q][1].record(stream)

    def step(k=None):
        e = ev[k] if k is not None else None
        fk = fork[(k or 0) % 2]
        fk.record(st)
        s_chain.wait_event(fk)
        timed(e, 0, s_chain, lambda: bs.solve(f, X64, stream=s_chain))
        timed(e, 1, s_chain, lambda: bs.solve_refine(f, B32, XR, stream=s_chain))
        timed(e, 2, s_chain, lambda: bs.solve_adjoint(f, G, stream=s_chain))
        timed(e, 3, s_chain, lambda: bs.band_grad(f, G, X64, dbands=db, stream=s_chain))
        st.wait_stream(s_chain)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(st)
        for k in range(args.steps):
            step(k)
        t1.record(st)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    if world > 1:
        ms = max_over_ranks(ms, dist, "cuda")
    per = {n: 0.0 for n in names}
    for k in range(args.steps):
        for q, n in enumerate(names):
            per[n] += ev[k][q][0].elapsed_time(ev[k][q][1]) / args.steps
    ms_step = ms / args.steps
    units_step = 3 * N * M  # three solves of N*M unknowns each: FP64, mixed precision, adjoint
    value = job_value(units_step, world, ms_step)

    # Each kernel of the step also timed alone, back to back, right after the
    # timed region (same data and stream)
    alone = {
        "f64_solve": time_alone(lambda: bs.solve(f, X64, stream=s_chain), s_chain, reps=20),
        "refine_solve": time_alone(lambda: bs.solve_refine(f, B32, XR, stream=s_ref), s_ref, reps=20),
        "adjoint_f64": time_alone(lambda: bs.solve_adjoint(f, G, stream=s_chain), s_chain, reps=20),
        "band_grad_f64": time_alone(lambda: bs.band_grad(f, G, X64, dbands=db, stream=s_chain), s_chain, reps=20),
    }

    peaks, peak_src = _peaks()
    hbm = float(peaks["hbm_gbs"])
    # FP64 FMA ceiling from unit counts and clocks: 2 FP64 FMA per clock per
    # SM (1.25 TFLOP/s nominal at the 2.07 GHz maximum SM clock of 152 SMs);
    # the device's rate measured by bs_measure_fp64_rate is reported beside it
    dev = torch.cuda.get_device_properties(0)
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_fma_derived = 2.0 * dev.multi_processor_count * sm_max_mhz * 1e6
    fp64_fma_live = [bs.measure_fp64_rate() for _ in range(5)]
    fp64_fma_live = statistics.median(fp64_fma_live)
    nm = N * M
    # algorithmic bytes and FP64 work per launch (pentadiagonal); "arith" is
    # what each path computes in
    paths = {
        "f64_solve": {"bytes": 16 * nm, "arith": "fp32 pairs (FP64 data in and out)"},
        "refine_solve": {"bytes": 12 * nm, "arith": "fp32 sweeps + error-free fp32 residuals, fp64 sum"},
        "adjoint_f64": {"bytes": 16 * nm, "arith": "fp32 pairs (FP64 data in and out)"},
        "band_grad_f64": {"bytes": 16 * nm, "arith": "fp64 FMAs for 3 of the 5 products per unknown (those "
                          "with the lower X rows of a thread's window), FP32 pairs for the other two", "dp_fma": 3 * nm},
    }
    for n, p in paths.items():
        p["ncu_dram_bytes"] = ncu_traffic(n)
        t_alone = alone[n] * 1e-3
        t_step = per[n] * 1e-3
        p["ms"] = round(alone[n], 5)
        p["in_step_ms"] = round(per[n], 5)
        p["unknowns_per_s"] = nm / t_alone
        p["hbm_gbs"] = p["bytes"] / t_alone / 1e9
        p["hbm_frac_of_measured"] = p["hbm_gbs"] / hbm
        p["hbm_frac_of_8tbs"] = p["hbm_gbs"] / NOMINAL_HBM_GBS
        p["in_step_hbm_frac_of_measured"] = p["bytes"] / t_step / 1e9 / hbm
        if "dp_fma" in p:
            p["fp64_fma_per_s"] = p["dp_fma"] / t_alone
            p["fp64_frac_of_derived_peak"] = p["fp64_fma_per_s"] / fp64_fma_derived
            p["fp64_frac_of_live_rate"] = p["fp64_fma_per_s"] / fp64_fma_live
    # the dominant kernel: the longest share of the step
    dom = max(names, key=lambda n: per[n])
    dp = paths[dom]
    t_dom = per[dom] * 1e-3
    ach = dp["bytes"] / t_dom / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": ncu_traffic(dom), "algorithmic_bytes": dp["bytes"],
            "timing": "algorithmic bytes / mean in-step duration (CUDA events on the kernel's stream over the "
                      "timed region)",
            "peak_source": peak_src,
            "alone": {"ms": dp["ms"], "frac": dp["hbm_frac_of_measured"]},
            "arith": dp["arith"]}
    if "dp_fma" in dp:
        roof["fp64_pipe"] = {
            "bound_by": "FP64 FMA pipe (3 FMA per unknown)",
            "achieved_fma_per_s": dp["dp_fma"] / t_dom,
            "peak_fma_per_s": fp64_fma_derived,
            "peak_source": "derived: 2 FP64 FMA / clock / SM x SMs x max SM clock (1.25 TFLOP/s nominal)",
            "frac": dp["dp_fma"] / t_dom / fp64_fma_derived,
            "live_rate_fma_per_s": fp64_fma_live,
            "live_rate_source": "self-measured: bs_measure_fp64_rate, median of 5 launches, clocks in 'clocks'",
            "frac_of_live_rate": dp["dp_fma"] / t_dom / fp64_fma_live}

    # the plain FP32 solve (not part of the step): timed alone, error reported
    X32 = B0.float()
    f32_alone = time_alone(lambda: bs.solve(f, X32), st, reps=50)
    f32_alone = {"ms": f32_alone, "unknowns_per_s": nm / (f32_alone * 1e-3),
                 "hbm_gbs": 8 * nm / (f32_alone * 1e-3) / 1e9}
    f32_alone["hbm_frac_of_measured"] = f32_alone["hbm_gbs"] / hbm
    del X32
    # BF16-stored B, FP32 arithmetic, FP32 X (not part of the step): 6 B per unknown
    B16 = B0.to(torch.bfloat16)
    Xb = torch.empty((N, M), dtype=torch.float32, device="cuda")
    t16 = time_alone(lambda: bs.solve_bf16(f, B16, Xb), st, reps=50)
    bf16_alone = {"ms": t16, "unknowns_per_s": nm / (t16 * 1e-3), "hbm_gbs": 6 * nm / (t16 * 1e-3) / 1e9}
    bf16_alone["hbm_frac_of_measured"] = bf16_alone["hbm_gbs"] / hbm
    del B16, Xb

    # the three-pass refinement on the system residual (not part of the step)
    XS = torch.empty_like(XR)
    ms_sys = time_alone(lambda: bs.solve_refine(f, B32, XS, mode=bs.REFINE_SYSTEM), st, reps=30)
    refine_system_alone = {"ms": ms_sys, "unknowns_per_s": nm / (ms_sys * 1e-3),
                           "hbm_gbs": 12 * nm / (ms_sys * 1e-3) / 1e9,
                           "rel_residual": rel_residual(bands, B32.double(), XS)}
    del XS

    # end to end through the public API with host buffers
    e2e = run_e2e(bs, f, N, M, st, args, world)
    serving = None if args.no_serving else run_serving(bs)
    others, other_samples = run_other_configs(bs, st, hbm)

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-pair/f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "M_per_gpu": M, "width": 5, "layout": "interleaved",
                   "arithmetic": "FP64 data; the FP64 solve and adjoint in FP32 pairs (48 significant bits, "
                                 "error-free transformations), the band gradient in FP64 FMAs for 3 of its 5 "
                                 "products per unknown and FP32 pairs for the other two, the mixed-precision "
                                 "solve in FP32 with "
                                 "error-free residuals",
                   "l2": "no flush: FP64 operands (256 MiB) exceed L2; the FP32 input is re-read after >1 GiB of other traffic",
                   "parallelism": f"replicas x{world} (systems partitioned, no collective)"},
        "rel_residual": resid,
        "f32_solve_alone": f32_alone,
        "bf16_solve_alone": bf16_alone,
        "refine_system_alone": refine_system_alone,
        "hbm_gbs_step": (sum(p["bytes"] for p in paths.values())) / (ms_step * 1e-3) / 1e9,
        "paths": {n: {k: (round(v, 6) if isinstance(v, float) else v) for k, v in p.items()}
                  for n, p in paths.items()},
        "roofline": roof,
        "e2e": e2e,
        "serving": serving,
        "other_workloads": others,
        "gpu_launches": 5 * args.steps,  # f64 solve, refine solve, adjoint, band gradient (two kernels)
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, errs = cpu_baseline(args, bands, sample, other_samples)
        line["cpu_baseline"] = cb
        line["rel_err_vs_oracle"] = errs
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_serving(bs, n_lhs=256, n_burst=192, n_poisson=10000, load=0.7, sweep=(0.1, 0.3, 0.5, 0.9, 1.1),
                n_sweep=1000, budget=24 << 30, seed=0):
    """Serving workload: 256 resident LHS (tri/penta 50/50, N log-uniform in
    [64, 4096], diagonally dominant), requests with M log-uniform in
    [1, 65536], FP64 or FP32-stored + refinement 50/50, RHS ~ U(-1,1) in pinned
    host memory, results copied back to host memory.  First a closed burst
    (all requests queued at once) gives the saturation rate, then a Poisson
    stream at `load` times that rate gives p50/p99 latency (submission to
    host-observed completion) at sustained load over `n_poisson` requests;
    shorter streams at the `sweep` loads give the latency-throughput curve."""
    import torch
    import synth
    from paper_1909_04539_gb300 import serve as sv

    specs = [synth.serving_lhs(i) for i in range(n_lhs)]
    facs = [bs.Factor(sp.bands) for sp in specs]
    n_total = n_burst + n_poisson + n_sweep * len(sweep)
    reqs = synth.serving_requests(n_total, rate_hz=1.0, n_lhs=n_lhs, seed=seed)
    max_nm = max(specs[r.lhs_id].N * r.M for r in reqs)
    g = torch.Generator().manual_seed(seed)
    pool = (torch.rand(max_nm + 4096, dtype=torch.float64, generator=g) * 2 - 1).pin_memory()
    pool32 = pool.float().pin_memory()
    out = torch.empty(max_nm, dtype=torch.float64).pin_memory()
    rng = np.random.default_rng(seed + 1)

    def views(r):
        sp = specs[r.lhs_id]
        nm = sp.N * r.M
        o = int(rng.integers(0, 4096))
        src = pool32 if r.refine else pool
        return src[o:o + nm].view(sp.N, r.M), out[:nm].view(sp.N, r.M)

    srv = sv.Server(budget, n_streams=4)
    # warm-up
    for r in reqs[:8]:
        B, X = views(r)
        srv.wait(srv.submit(facs[r.lhs_id], B, X, sv.F32_REFINE if r.refine else sv.F64), 120)
    # saturation: closed burst
    burst = reqs[:n_burst]
    t0 = time.perf_counter()
    ids = []
    for r in burst:
        B, X = views(r)
        ids.append(srv.submit(facs[r.lhs_id], B, X, sv.F32_REFINE if r.refine else sv.F64))
    for i in ids:
        srv.wait(i, 600)
    t_burst = time.perf_counter() - t0
    unk_burst = sum(specs[r.lhs_id].N * r.M for r in burst)
    bytes_burst = sum(specs[r.lhs_id].N * r.M * (12 if r.refine else 16) for r in burst)
    sat_rps = n_burst / t_burst
    for i in ids:
        srv.release(i)

    def poisson(stream, ld, gap_seed):
        """Poisson arrivals at ld * saturation; latency percentiles."""
        rate = ld * sat_rps
        gaps = np.random.default_rng(gap_seed).exponential(1.0 / rate, len(stream))
        ids = []
        t0 = time.perf_counter()
        t_next = t0
        for r, gap in zip(stream, gaps):
            t_next += gap
            while True:
                d = t_next - time.perf_counter()
                if d <= 0:
                    break
                time.sleep(min(d, 0.0005))
            B, X = views(r)
            ids.append(srv.submit(facs[r.lhs_id], B, X, sv.F32_REFINE if r.refine else sv.F64))
        lat = []
        for i in ids:
            srv.wait(i, 600)
            lat.append(srv.poll(i)[1])
        t_stream = time.perf_counter() - t0
        for i in ids:
            srv.release(i)
        lat_ms = np.array(lat) * 1e3
        unk = sum(specs[r.lhs_id].N * r.M for r in stream)
        # size classes of the server (device bytes up to 16 MiB: "small")
        nbytes = np.array([specs[r.lhs_id].N * r.M * (12 if r.refine else 8) for r in stream])
        classes = {}
        for cname, sel in (("small", nbytes <= (16 << 20)), ("large", nbytes > (16 << 20))):
            if sel.any():
                classes[cname] = {"requests": int(sel.sum()), "p50_ms": float(np.percentile(lat_ms[sel], 50)),
                                  "p99_ms": float(np.percentile(lat_ms[sel], 99))}
        return {"offered_requests_per_s": rate, "load_of_saturation": ld, "requests": len(stream),
                "achieved_requests_per_s": len(stream) / t_stream, "unknowns_per_s": unk / t_stream,
                "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "mean_ms": float(lat_ms.mean()), "by_size": classes}

    # sustained: Poisson at load * saturation
    pos = n_burst
    sustained = poisson(reqs[pos:pos + n_poisson], load, seed + 2)
    pos += n_poisson
    curve = []
    for q, ld in enumerate(sweep):
        curve.append(poisson(reqs[pos:pos + n_sweep], ld, seed + 3 + q))
        pos += n_sweep
    st = srv.stats()
    srv.close()
    return {
        "workload": "256 resident LHS (tri/penta, N log-uniform [64,4096]); M log-uniform [1,65536]; "
                    "FP64 or FP32+refine 50/50; host (pinned) RHS in, host results out; Poisson arrivals",
        "saturation": {"requests_per_s": sat_rps, "unknowns_per_s": unk_burst / t_burst,
                       "host_device_gbs": bytes_burst / t_burst / 1e9, "requests": n_burst},
        "sustained": sustained,
        "load_sweep": curve,
        "server": {"hbm_budget_bytes": budget, "streams": 4, "batches": st["batches"],
                   "max_batch_requests": st["max_batch_requests"],
                   "max_concurrent_batches": st["max_concurrent_batches"]},
    }


def run_other_configs(bs, st, hbm):
    """The other workloads, each timed alone (median of CUDA-event timings;
    operands larger than L2 except the small random case): sampled results
    are kept for the oracle comparison of the CPU-baseline leg."""
    import torch
    import synth

    out, samples = {}, {}
    # one-off factorisation (host FP64 elimination, reversed elimination,
    # row partitions, uploads): host wall time, median of 5, kept out of
    # every throughput figure
    fac = {}
    for name, bands, per in (("penta_clamped_N512", synth.clamped_hyperdiffusion_bands(512, 0.1), False),
                             ("tri_spline_N1024", synth.spline_bands(1024), False),
                             ("tri_adi_N4096", synth.adi_bands(4096, 0.5), False),
                             ("periodic_tri_N1024", synth.periodic_toeplitz_bands(1024, (-0.5, 2.0, -0.5)), True)):
        ts = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ff = bs.Factor(bands, periodic=per)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
            ff.close()
        fac[f"{name}_ms"] = statistics.median(ts)
    out["factor"] = fac
    # random tridiagonal, N=64, M=1024, FP64 (L2-resident; the default path is
    # the two-ended sweep).  Device time per solve from a CUDA graph of 100
    # (copy + solve) minus 100 copies; a plain launch loop is bound by the
    # host's launch rate instead, reported beside it
    bands, Bh = synth.random_tri_case(64, 1024, 0)
    f = bs.Factor(bands)
    B0 = torch.tensor(Bh, device="cuda")
    X = B0.clone()
    tcopy = time_graph(lambda: X.copy_(B0))
    us = (time_graph(lambda: (X.copy_(B0), bs.solve(f, X))) - tcopy) * 1e3
    bs.set_option(bs.OPT_TWISTED, 1)
    us1 = (time_graph(lambda: (X.copy_(B0), bs.solve(f, X))) - tcopy) * 1e3
    bs.set_option(bs.OPT_TWISTED, 0)
    loop = time_alone(lambda: (X.copy_(B0), bs.solve(f, X)), st, reps=200) - \
        time_alone(lambda: X.copy_(B0), st, reps=200)
    X.copy_(B0)
    bs.solve(f, X)
    out["random_tri_N64_M1024_f64"] = {"us_per_solve": us, "unknowns_per_s": 64 * 1024 / (us * 1e-6),
                                       "one_thread_per_system_us": us1,
                                       "us_per_call_launch_loop": loop * 1e3}
    samples["random_tri"] = (bands, Bh, X.cpu().numpy(), None)
    # spline [1,4,1]/6, N=1024, M=2^20: FP64 plain vs FP32-stored + refinement
    N, M = 1024, 1 << 20
    bands = synth.spline_bands(N)
    f = bs.Factor(bands)
    B32 = synth.spline_rhs(N, M, 0, "cuda")
    B64 = B32.double()
    X64 = B64.clone()
    XR = torch.empty_like(B64)
    t64 = time_alone(lambda: bs.solve(f, X64), st, reps=10)
    tr = time_alone(lambda: bs.solve_refine(f, B32, XR), st, reps=10)
    X32 = B32.clone()
    t32 = time_alone(lambda: bs.solve(f, X32), st, reps=10)
    del X32
    X64.copy_(B64)
    bs.solve(f, X64)
    bs.solve_refine(f, B32, XR)
    cols = np.random.default_rng(11).choice(M, 256, replace=False)
    samples["spline"] = (bands, B64[:, cols].cpu().numpy(), X64[:, cols].cpu().numpy(), XR[:, cols].cpu().numpy())
    # the same right-hand sides with the periodic spline matrix (cyclic
    # [1,4,1]/6, Sherman-Morrison fused into the sweeps), FP64 and FP32
    pbands = synth.periodic_toeplitz_bands(N, (1 / 6, 4 / 6, 1 / 6))
    fp = bs.Factor(pbands, periodic=True)
    XP = B64.clone()
    tp = time_alone(lambda: bs.solve(fp, XP), st, reps=10)
    XP32 = B32.clone()
    tp32 = time_alone(lambda: bs.solve(fp, XP32), st, reps=10)
    XP.copy_(B64)
    bs.solve(fp, XP)
    samples["periodic_spline"] = (pbands, B64[:, cols].cpu().numpy(), XP[:, cols].cpu().numpy(), None)
    del XP, XP32
    nm = N * M
    out["spline_N1024_M1048576"] = {
        "f64_solve": {"ms": t64, "unknowns_per_s": nm / (t64 * 1e-3), "hbm_gbs": 16 * nm / (t64 * 1e-3) / 1e9},
        "refine_solve": {"ms": tr, "unknowns_per_s": nm / (tr * 1e-3), "hbm_gbs": 12 * nm / (tr * 1e-3) / 1e9,
                         "hbm_frac_of_measured": 12 * nm / (tr * 1e-3) / 1e9 / hbm},
        "refine_over_f64_speedup": t64 / tr,
        "f32_solve": {"ms": t32, "unknowns_per_s": nm / (t32 * 1e-3), "hbm_gbs": 8 * nm / (t32 * 1e-3) / 1e9,
                      "hbm_frac_of_measured": 8 * nm / (t32 * 1e-3) / 1e9 / hbm},
        "periodic_f64_solve": {"ms": tp, "unknowns_per_s": nm / (tp * 1e-3), "hbm_gbs": 16 * nm / (tp * 1e-3) / 1e9,
                               "over_plain_f64": tp / t64},
        "periodic_f32_solve": {"ms": tp32, "unknowns_per_s": nm / (tp32 * 1e-3),
                               "hbm_gbs": 8 * nm / (tp32 * 1e-3) / 1e9}}
    del B32, B64, X64, XR
    torch.cuda.empty_cache()
    # ADI 4096^2, r = 0.5: half-steps on both axes, forward and adjoint, FP64 and FP32
    n, r = 4096, 0.5
    f = bs.Factor(synth.adi_bands(n, r))
    adi = {}
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        u = synth.adi_field(n, 0, "cuda", dt)
        o = torch.empty_like(u)
        for axis in (0, 1):
            for adj in (False, True):
                t = time_alone(lambda: bs.adi_halfstep(f, u, r, axis, out=o, adjoint=adj), st, reps=10)
                es = 8 if dt == torch.float64 else 4
                adi[f"{name}_axis{axis}{'_adjoint' if adj else ''}"] = {
                    "ms": t, "unknowns_per_s": n * n / (t * 1e-3), "hbm_gbs": 2 * es * n * n / (t * 1e-3) / 1e9}
        if dt == torch.float64:
            half = bs.adi_halfstep(f, u, r, 0)
            full = bs.adi_halfstep(f, half, r, 1)
            rows = np.random.default_rng(12).choice(n, 8, replace=False)
            samples["adi"] = (r, u.cpu().numpy(), full.cpu().numpy(), rows)
    out["adi_4096x4096"] = adi
    # a small batch of long tridiagonal systems (N = 4096, M = 4096, FP64):
    # row-partitioned (the default below 256 systems per SM) against one
    # thread per system
    N4, M4 = 4096, 4096
    rng4 = np.random.default_rng(21)
    b4 = synth.random_tri_bands(N4, rng4)
    f4 = bs.Factor(b4)
    B4 = synth.uniform_rhs(N4, M4, 21, "cuda")
    X4 = B4.clone()
    tc4 = time_alone(lambda: X4.copy_(B4), st, reps=20)
    tp = time_alone(lambda: (X4.copy_(B4), bs.solve(f4, X4)), st, reps=20) - tc4
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 2)
    tt = time_alone(lambda: (X4.copy_(B4), bs.solve(f4, X4)), st, reps=20) - tc4
    bs.set_option(bs.OPT_TWISTED, 1)
    tu = time_alone(lambda: (X4.copy_(B4), bs.solve(f4, X4)), st, reps=20) - tc4
    bs.set_option(bs.OPT_PARTITION, 0)
    bs.set_option(bs.OPT_TWISTED, 0)
    out["tri_N4096_M4096_f64"] = {"partitioned_ms": tp, "two_ended_ms": tt, "one_thread_per_system_ms": tu,
                                  "unknowns_per_s": N4 * M4 / (tp * 1e-3), "speedup": tu / tp}
    X4.copy_(B4)
    bs.solve(f4, X4)
    cols4 = np.random.default_rng(22).choice(M4, 16, replace=False)
    samples["tri_N4096"] = (b4, B4[:, cols4].cpu().numpy(), X4[:, cols4].cpu().numpy(), None)
    del B4, X4, f4

    # uniform pentadiagonal matrix (the outermost sub-diagonal one scalar,
    # Sec. 4.1 cuPentUniformBatch): hyperdiffusion (s, -4s, 1 + 6s, -4s, s),
    # N = 512, M = 65536; the FP32-arithmetic sweeps with the scalar (on
    # request) against the general ones (FP64 solves always take the general
    # sweeps)
    uni = {}
    Nu, Mu = 512, 65536
    bu = synth.toeplitz_bands(Nu, (0.1, -0.4, 1.6, -0.4, 0.1))
    fu = bs.Factor(bu)
    B32 = synth.normal_rhs(Nu, Mu, 4, "cuda", torch.float32)
    X32 = B32.clone()
    B16 = B32.bfloat16()
    tcopy = time_alone(lambda: X32.copy_(B32), st, reps=20)
    for dname, fn, tc in (("f32", lambda: (X32.copy_(B32), bs.solve(fu, X32)), tcopy),
                          ("bf16_storage", lambda: bs.solve_bf16(fu, B16, X32), 0.0)):
        row = {}
        for opt, key in ((2, "uniform_ms"), (1, "general_ms")):
            bs.set_option(bs.OPT_UNIFORM, opt)
            row[key] = time_alone(fn, st, reps=20) - tc
        bs.set_option(bs.OPT_UNIFORM, 0)
        row["unknowns_per_s"] = Nu * Mu / (row["uniform_ms"] * 1e-3)
        uni[dname] = row
    X32.copy_(B32)
    bs.solve(fu, X32)
    colsu = np.random.default_rng(23).choice(Mu, 64, replace=False)
    Bs = B32[:, colsu].double().cpu().numpy()
    samples["uniform_penta_f32"] = (bu, Bs, X32[:, colsu].double().cpu().numpy(), None)
    out["uniform_penta_N512_M65536"] = uni
    del B32, X32, B16, fu

    # mixed-precision solve by number of refinement steps and storage type:
    # the clamped penta batch (N = 512, M = 65536) in FP32 and BF16 storage,
    # and stiff hyperdiffusion I + 4000 D4 (N = 512, M = 4096, condition
    # number ~6e4), timed per call; sampled systems for the oracle comparison
    rk = {}
    Nr, Mr = 512, 65536
    br = synth.clamped_hyperdiffusion_bands(Nr, 0.1)
    fr = bs.Factor(br)
    Bn = synth.normal_rhs(Nr, Mr, 9, "cuda")
    colsr = np.random.default_rng(14).choice(Mr, 256, replace=False)
    for sname, Bs in (("f32", Bn.float()), ("bf16", Bn.bfloat16())):
        XR = torch.empty((Nr, Mr), dtype=torch.float64, device="cuda")
        outs = {}
        for k in (0, 1, 2, 3):
            rk[f"penta_clamped_{sname}_k{k}_ms"] = time_alone(lambda: bs.solve_refine(fr, Bs, XR, refine_steps=k), st,
                                                              reps=10)
            bs.solve_refine(fr, Bs, XR, refine_steps=k)
            torch.cuda.synchronize()
            outs[k] = XR[:, colsr].cpu().numpy()
        samples[f"refine_steps_{sname}"] = (br, Bs[:, colsr].double().cpu().numpy(), outs)
        del XR
    del Bn
    ss = 4000.0
    bstiff = synth.toeplitz_bands(512, (ss, -4 * ss, 1 + 6 * ss, -4 * ss, ss))
    fs = bs.Factor(bstiff)
    Bst = synth.uniform_rhs(512, 4096, 15, "cuda").float()
    outs = {}
    for k in (0, 1, 2, 3):
        outs[k] = bs.solve_refine(fs, Bst, refine_steps=k, mode=bs.REFINE_FACTOR).cpu().numpy()
    samples["refine_steps_stiff_f32"] = (bstiff, Bst.double().cpu().numpy(), outs)
    out["refine_steps"] = rk
    del fr, fs

    # the paper's benchmark problems as Crank-Nicolson time stepping (explicit
    # side fused into the sweep): periodic diffusion (-s, 1 + 2s, -s), N = 1024,
    # and hyperdiffusion (s, -4s, 1 + 6s, -4s, s), N = 512; M = 65536, 10 steps
    cn = {}
    for name, N, bands, per in (
            ("periodic_diffusion_N1024", 1024, synth.periodic_toeplitz_bands(1024, (-0.5, 2.0, -0.5)), True),
            ("hyperdiffusion_N512", 512, synth.toeplitz_bands(512, (0.1, -0.4, 1.6, -0.4, 0.1)), False)):
        f = bs.Factor(bands, periodic=per)
        M, K = 65536, 10
        for dt, dname, es in ((torch.float64, "f64", 8), (torch.float32, "f32", 4)):
            C = synth.uniform_rhs(N, M, 3, "cuda", dt)
            if dt == torch.float64:
                cols = np.random.default_rng(13).choice(M, 64, replace=False)
                C0 = C[:, cols].cpu().numpy()
                bs.cn_steps(f, C, 2)
                samples[f"cn_{name}"] = (bands, per, C0, C[:, cols].cpu().numpy())
            t = time_alone(lambda: bs.cn_steps(f, C, K), st, reps=5) / K
            cn[f"{name}_{dname}"] = {"ms_per_step": t, "unknowns_per_s": N * M / (t * 1e-3),
                                     "hbm_gbs": 2 * es * N * M / (t * 1e-3) / 1e9}
            del C
    out["cn_steps_M65536"] = cn
    return out, samples


def time_graph(fn, reps=100) -> float:
    """Per-call milliseconds of fn replayed from a CUDA graph of `reps` calls
    (the best of three replays): device time without the host's launch
    cost."""
    import torch

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for _ in range(reps):
                fn()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()  # the replay runs on the current stream
        g.replay()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / reps)
    return best


def time_alone(fn, st, reps=50, warm=3) -> float:
    """Median per-call milliseconds of fn on stream st (CUDA events)."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:
        a.record(st)
        fn()
        b.record(st)
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in evs]))


def run_e2e(bs, f, N, M, st, args, world):
    """Same three solves through the public API with pinned host buffers:
    each step copies its inputs host->device and its results back.  Steps
    are pipelined the way a user streaming batches would run them: two sets
    of device input buffers and two of output buffers, the host->device
    copies of step k+1 and the device->host copies of step k-1 on their own
    streams while step k computes (ordered by events).  A step first copies
    its in-place operands (B, G) from its input set to its output set on the
    device, so the next step's inputs may arrive while this step's results
    are still being read back.  The same steps run one after another on one
    stream are reported beside it."""
    import torch

    steps = max(1, min(args.steps, 50))
    hB = torch.empty((N, M), dtype=torch.float64, pin_memory=True).normal_()
    hB32 = hB.float().pin_memory()
    hG = torch.empty((N, M), dtype=torch.float64, pin_memory=True).uniform_(-1, 1)

    class Inputs:
        def __init__(self):
            self.dB = torch.empty((N, M), dtype=torch.float64, device="cuda")
            self.dB32 = torch.empty((N, M), dtype=torch.float32, device="cuda")
            self.dG = torch.empty((N, M), dtype=torch.float64, device="cuda")
            self.h2d = torch.cuda.Event()
            self.used = torch.cuda.Event()   # the step's compute has read them

    class Outputs:
        def __init__(self):
            self.dX = torch.empty((N, M), dtype=torch.float64, device="cuda")
            self.dXR = torch.empty((N, M), dtype=torch.float64, device="cuda")
            self.dGB = torch.empty((N, M), dtype=torch.float64, device="cuda")
            self.db = torch.empty((5, N), dtype=torch.float64, device="cuda")
            self.oX = torch.empty((N, M), dtype=torch.float64, pin_memory=True)
            self.oXR = torch.empty((N, M), dtype=torch.float64, pin_memory=True)
            self.oG = torch.empty((N, M), dtype=torch.float64, pin_memory=True)
            self.odb = torch.empty((5, N), dtype=torch.float64, pin_memory=True)
            self.comp = torch.cuda.Event()
            self.d2h = torch.cuda.Event()

    ins, outs = [Inputs(), Inputs()], [Outputs(), Outputs()]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def h2d(I, stream):
        with torch.cuda.stream(stream):
            I.dB.copy_(hB, non_blocking=True)
            I.dB32.copy_(hB32, non_blocking=True)
            I.dG.copy_(hG, non_blocking=True)

    def compute(I, O, stream):
        with torch.cuda.stream(stream):
            O.dX.copy_(I.dB)
            O.dGB.copy_(I.dG)
        bs.solve_refine(f, I.dB32, O.dXR, stream=stream)
        I.used.record(stream)
        bs.solve(f, O.dX, stream=stream)
        bs.solve_adjoint(f, O.dGB, X=O.dX, dbands=O.db, stream=stream)

    def d2h(O, stream):
        with torch.cuda.stream(stream):
            O.oX.copy_(O.dX, non_blocking=True)
            O.oXR.copy_(O.dXR, non_blocking=True)
            O.oG.copy_(O.dGB, non_blocking=True)
            O.odb.copy_(O.db, non_blocking=True)

    def serial_step():
        h2d(ins[0], st)
        compute(ins[0], outs[0], st)
        d2h(outs[0], st)

    def pipelined(n):
        for k in range(n):
            I, O = ins[k % 2], outs[k % 2]
            s_in.wait_event(I.used)    # step k-2 has read this input set
            h2d(I, s_in)
            I.h2d.record(s_in)
            st.wait_event(I.h2d)
            st.wait_event(O.d2h)       # step k-2's results have left this output set
            compute(I, O, st)
            O.comp.record(st)
            s_out.wait_event(O.comp)
            d2h(O, s_out)
            O.d2h.record(s_out)

    serial_step()
    pipelined(2)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # serial
    t0.record(st)
    for _ in range(steps):
        serial_step()
    t1.record(st)
    torch.cuda.synchronize()
    ms_serial = t0.elapsed_time(t1) / steps
    # pipelined: from the first input copy to the last result copy
    t0.record(s_in)
    pipelined(steps)
    t1.record(s_out)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    h2d_b = N * M * (8 + 4 + 8)
    d2h_b = N * M * (8 + 8 + 8) + 5 * N * 8
    return {"value": 3 * N * M * world / (ms * 1e-3), "unit": "unknowns/s", "h2d_bytes_per_step": h2d_b,
            "d2h_bytes_per_step": d2h_b, "ms_per_step": ms, "steps": steps,
            "pipelining": "two input and two output buffer sets; copies in, compute and copies out on three "
                          "streams",
            "serial_ms_per_step": ms_serial,
            "h2d_gbs": h2d_b / (ms * 1e-3) / 1e9, "d2h_gbs": d2h_b / (ms * 1e-3) / 1e9}


# ------------------------------------------------------------------ CPU oracle


def _oracle_step(oracle, bands, B, G):
    X = oracle.solve(bands, B)            # FP64 solve
    oracle.solve(bands, B)                # the FP32-stored solve has the same FP64 reference
    GB = oracle.solve_adjoint(bands, G)   # adjoint
    oracle.band_grad(5, GB, X)            # band gradient
    return X


def cpu_baseline(args, bands, sample, other_samples=None, target_s: float = 12.0):
    """The oracle, as it stands, timed on a bounded column sample of the
    workload (the very columns the GPU solved first), which also gives the
    GPU's error against it."""
    import oracle

    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    N = N_ROWS
    B, cols = sample["B"], sample["cols"]
    m0 = B.shape[1]
    X = oracle.solve(bands, B)
    XR = oracle.solve(bands, sample["B32"])
    X32ref = oracle.solve(bands, sample["B32"])
    errs = {"f64_solve": float(np.linalg.norm(sample["X64"] - X) / np.linalg.norm(X)),
            "f32_solve": float(np.linalg.norm(sample["X32"] - X32ref) / np.linalg.norm(X32ref)),
            "refine_solve": float(np.linalg.norm(sample["XR"] - XR) / np.linalg.norm(XR)),
            "f64_solve_max_system": max_system_err(sample["X64"], X),
            "f32_solve_max_system": max_system_err(sample["X32"], X32ref),
            "refine_solve_max_system": max_system_err(sample["XR"], XR),
            "f32_solve_vs_fp64_input": float(np.linalg.norm(sample["X32"] - X) / np.linalg.norm(X)),
            "tolerance": {"f64_solve": 1e-12, "refine_solve": 1e-12, "f32_solve": fp32_tolerance(bands),
                          "f32_rule": "width * kappa_inf(A) * 2^-24"},
            "metric": "relative L2 over the sampled systems, and the largest relative max-norm error of one "
                      "system (_max_system); the FP32 solve against the oracle's solve of the FP32-rounded input",
            "systems_checked": int(m0)}
    for name, smp in (other_samples or {}).items():
        if name == "adi":
            r, u, full, rows = smp
            ref = oracle.adi_halfstep(oracle.adi_halfstep(u, r, 0), r, 1)
            errs["adi_4096_full_step_f64"] = float(np.linalg.norm(full - ref) / np.linalg.norm(ref))
        elif name.startswith("refine_steps_"):
            b, Bs, outs = smp
            ref = oracle.solve(b, Bs)
            for k, Xk in outs.items():
                errs[f"{name}_k{k}_max_system"] = max_system_err(Xk, ref)
                errs[f"{name}_k{k}"] = float(np.linalg.norm(Xk - ref) / np.linalg.norm(ref))
        elif name.startswith("cn_"):
            b, per, C0, C2 = smp
            ref = oracle.cn_steps(b, C0, 2, periodic=per)
            errs[f"{name}_2_steps_f64"] = float(np.linalg.norm(C2 - ref) / np.linalg.norm(ref))
        else:
            b, Bs, X64s, XRs = smp
            ref = oracle.periodic_tri_solve_bands(b, Bs) if name.startswith("periodic") else oracle.solve(b, Bs)
            key = f"{name}_solve" if name.endswith("_f32") else f"{name}_f64_solve"
            errs[key] = float(np.linalg.norm(X64s - ref) / np.linalg.norm(ref))
            errs[key + "_max_system"] = max_system_err(X64s, ref)
            if XRs is not None:
                errs[f"{name}_refine_solve"] = float(np.linalg.norm(XRs - ref) / np.linalg.norm(ref))
                errs[f"{name}_refine_solve_max_system"] = max_system_err(XRs, ref)
    # timing: the oracle step on a column block of the same batch, grown
    # until one step takes at least a quarter of target_s, then repeated to ~target_s
    Ball = sample["B_all"]
    rng = np.random.default_rng(1)
    m = 2048
    while True:
        Bs = np.ascontiguousarray(Ball[:, :m])
        G = rng.uniform(-1, 1, Bs.shape)
        t = time.perf_counter()
        _oracle_step(oracle, bands, Bs, G)
        dt = time.perf_counter() - t
        if dt > target_s / 4 or m >= Ball.shape[1]:
            break
        m = min(Ball.shape[1], int(m * min(8.0, max(2.0, target_s / 4 / max(dt, 1e-3)))))
    reps = max(1, int(round(target_s / max(dt, 1e-3))))
    t = time.perf_counter()
    for _ in range(reps):
        _oracle_step(oracle, bands, Bs, G)
    dt = (time.perf_counter() - t) / reps
    m0 = m
    cores_used = oracle.num_threads()
    # the same step on one core, on a block sized for about 3 s
    oracle.set_threads(1)
    m1 = int(min(m0, max(256, m0 * 3.0 / max(dt * cores_used, 1e-6))))
    B1, G1 = np.ascontiguousarray(Bs[:, :m1]), np.ascontiguousarray(G[:, :m1])
    t = time.perf_counter()
    _oracle_step(oracle, bands, B1, G1)
    dt1 = time.perf_counter() - t
    oracle.set_threads(cores)
    cb = {"value": 3 * N * m0 / dt, "unit": "unknowns/s", "cores": cores_used, "kind": "oracle",
          "sample": f"{reps} repetitions of one step (FP64 solve, FP64 solve, adjoint + band gradient) on "
                    f"the first {m0} of the {M_SYS} systems, {dt * reps:.1f} s in total",
          "value_1_core": 3 * N * m1 / dt1,
          "sample_1_core": f"one step on the first {m1} systems, one thread, {dt1:.1f} s"}
    return cb, errs


def max_system_err(x, ref) -> float:
    """Largest relative max-norm error of one system (columns of an (N, m)
    block): max_j ||x_j - ref_j||_inf / ||ref_j||_inf."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(x - ref), axis=0) / den))


def fp32_tolerance(bands) -> float:
    """width * kappa_inf(A) * 2^-24: the bound of a solve in FP32 arithmetic
    (each row of a banded LU sweep combines `width` terms; the relative
    forward error is at most kappa_inf times the backward error)."""
    w, n = bands.shape
    h = w // 2
    A = np.zeros((n, n))
    for k in range(w):
        for i in range(n):
            if 0 <= i + k - h < n:
                A[i, i + k - h] = bands[k, i]
    kappa = np.abs(A).sum(axis=1).max() * np.abs(np.linalg.inv(A)).sum(axis=1).max()
    return float(w * kappa * 2.0 ** -24)


def rel_residual(bands, B, X) -> float:
    """|B - A X|_F / |B|_F over every system, in FP64 on the device."""
    import torch

    b = torch.tensor(bands, device=X.device)
    w = b.shape[0]
    h = w // 2
    N = X.shape[0]
    R = B.clone()
    for k in range(w):
        off = k - h
        lo, hi = max(0, -off), N - max(0, off)
        R[lo:hi] -= b[k, lo:hi, None] * X[lo + off:hi + off]
    return float((torch.linalg.norm(R) / torch.linalg.norm(B)).item())


def run_reference(args):
    """--impl reference: the oracle on the host cores, same metric and units."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth

    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    N = N_ROWS
    bands = synth.clamped_hyperdiffusion_bands(N, S_HYPER)
    rng = np.random.default_rng(0)
    m = 2048
    B = rng.standard_normal((N, m))
    G = rng.uniform(-1, 1, (N, m))
    t = time.perf_counter()
    _oracle_step(oracle, bands, B, G)
    dt = time.perf_counter() - t
    # each step a bounded sample: the whole run (warm-up + timed) in about a minute
    per_step = 60.0 / max(1, args.steps + args.warmup)
    m = int(min(M_SYS, max(256, m * per_step / max(dt, 1e-6))))
    B = rng.standard_normal((N, m))
    G = rng.uniform(-1, 1, (N, m))
    for _ in range(args.warmup):
        _oracle_step(oracle, bands, B, G)
    t = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(oracle, bands, B, G)
    dt = (time.perf_counter() - t) / args.steps
    value = 3 * N * m / dt
    sample = f"each step on {m} of the {M_SYS} systems (FP64 solve, FP64 solve, adjoint + band gradient)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "M_per_gpu": M_SYS, "width": 5, "layout": "interleaved",
                   "sample_M": m},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-latency leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
