#!/usr/bin/env python
"""Benchmark of the RSAI(tol) build on GB300: M-columns/s at matched ||AM-I||_F.

Workload: 3-D 7-point upwind convection-diffusion on 64^3 (n = 262144,
nnz = 1,810,432), cell Peclet 5, c = 3 dominant rows per loop, l_max = 10,
eps = 0.3, fixed drop tol = 1e-3 (on A/||A||_1).  A step is one whole build of
M (||A||_1, every column's RSAI(tol) loop in the size bins, M to CSC and CSR)
replayed as one CUDA graph on inputs already resident in HBM; L2 is flushed
(256 MB write) between timed steps.

`value` is the FP32-QR + FP64-refinement build; the plain FP64 build is timed
beside it at the same ||AM-I||_F.  `e2e` times the public C-ABI call with
pinned host buffers (copy in, validate, build, copy M out).  `--impl
reference` times the FP64 CPU oracle on the host cores instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 (torchrun) every rank builds its own replica (weak scaling; the
columns need no exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PARAMS = dict(c=3, l_max=10, eps=0.3, tol=1e-3, drop="fixed")
METRIC = "RSAI M-columns/sec at matched ||AM-I||_F, FP32+refine vs FP64; bwd/fwd ratio"
WORKLOAD = "convdiff3d_7pt_upwind_64^3_Pe5"
# norm1, tau, 4 bins (W, W2, C, G), 3 kernels ordering the global bin's queue, 2 column-stats kernels,
# 2 x 3 scan kernels, pool->CSC, CSC->rows, row sort
KERNELS_PER_BUILD = 20
# GB300's published FP64 rate (a side field; the roofline divides by the measured FMA-chain rate)
PEAK_FP64_PUBLISHED = 1.25e12
# copy bandwidth measured on this GPU type, used only when MEASURED_PEAKS.json is absent
HBM_FALLBACK_GBS = 6800.0


def measured_hbm_gbs():
    """(GB/s, source) of the HBM roofline: MEASURED_PEAKS.json's copy bandwidth, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def fp32_units_peak(sms: int, sm_mhz: float) -> float:
    """FP32 FMA rate from the unit counts: SMs x 128 lanes x 2 flop x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_barrier(pg) -> None:
    """Barrier over the replicas (no-op for one process)."""
    if pg is not None:
        pg.barrier()


def rank_max(pg, x: float, device: str) -> float:
    """The maximum of x over the replicas: the whole job's time is the slowest rank's."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each doing `units_per_rank` in the slowest rank's time."""
    return world * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi samples (200 ms) while running; summary of the samples under load."""

    def __init__(self, uuid: str | None):
        self.proc = None
        # the raw samples go to a temporary file; the line printed carries their summary
        self.path = os.path.join(os.environ.get("RSAI_CLOCKS_DIR", tempfile.gettempdir()), f"rsai_clocks_{os.getpid()}.csv")
        self.uuid = uuid

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                try:
                    rows.append(dict(sm=float(p[1]), smmax=float(p[2]), util=float(p[4]), hw=p[6], hwt=p[7],
                                     swt=p[8], swp=p[9]))
                except ValueError:
                    continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smmax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


# the sources the bin kernels (k_bin_warp, k_bin_block) are compiled from
BIN_KERNEL_SOURCES = ("build_kernels.cu", "column.cuh", "common.cuh", "warp_small.cuh")


def strip_comments(src: str) -> str:
    """C++ source without its comments, trailing blanks and empty lines (string
    and character literals kept): what the compiler sees, up to line breaks."""
    out, i, n = [], 0, len(src)
    while i < n:
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            end = n if j < 0 else j + 2
            out.append("\n" * src.count("\n", i, end))
            i = end
        elif src[i] in "\"'":
            j = i + 1
            while j < n and src[j] != src[i]:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(src[i])
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).split("\n") if ln.strip())


def kernel_source_hash() -> str:
    """Hash of the bin kernels' sources without their comments: a committed ncu
    traffic figure is used only while the code it was taken on is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1503_04500_gb300", "csrc")
    for name in BIN_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode())
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel: str, precision: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernels have not changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
    except Exception:
        return None
    ent = data.get(f"{kernel}:{precision}")
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def run_oracle_sample(A, threads: int, stride: int):
    import numpy as np

    import oracle

    cols = np.arange(0, A.n, stride, dtype=np.int64)
    t0 = time.perf_counter()
    M = oracle.build(A, cols=cols, threads=threads, **PARAMS)
    dt = time.perf_counter() - t0
    return len(cols), dt, M


SPAI_KEYS = ("select", "l_max", "drop", "spar", "frob", "n_c", "build_ms", "first_build_s", "bicgstab_iters",
             "bicgstab_s", "qr_flops", "select_flops")


def powerlaw_1e6_extra(torch, np, rsai, inputs):
    """The n = 1e6 power law (c = 5, l_max = 8, eps = 0.4, FIXED tol = 1e-3),
    FP32+refine: the first build (allocation, checks and build, wall clock),
    one graph-replayed rebuild (CUDA events), the bins' split, and ||r_k|| of
    256 random columns against the FP64 oracle.  There is no FP64 GPU build of
    this workload here: its ~3e14 FP64 flops need more than 280 s at the GPU's
    FP64 rate."""
    import oracle

    kw = dict(c=5, l_max=8, eps=0.4, tol=1e-3, drop="fixed")
    P = inputs.powerlaw(1000000, seed=1503)
    dP = rsai.DeviceMatrix.from_host(P)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = rsai.build(dP, precision="fp32_refine", **kw)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    h.rebuild()
    e1.record(st)
    torch.cuda.synchronize()
    rebuild_ms = e0.elapsed_time(e1)
    s = h.stats()
    rho = h.columns()[0].cpu().numpy()
    ph = h.phase_times()
    h.free()
    cols = np.sort(np.random.default_rng(1503).choice(P.n, 256, replace=False))
    t1 = time.perf_counter()
    ref = oracle.build(P, cols=cols, **kw)
    osec = time.perf_counter() - t1
    rel = np.abs(rho[cols] - ref.rho) / np.maximum(ref.rho, 1e-300)
    return {"workload": "powerlaw_n1e6_seed1503", "n": P.n, "nnz": P.nnz, **kw, "precision": "fp32_refine",
            "first_build_s": first_s, "first_build_columns_per_s": P.n / first_s, "rebuild_ms": rebuild_ms,
            "rebuild_columns_per_s": P.n / (rebuild_ms / 1e3), "phases_ms": ph, "cols_bin": s["cols_bin"],
            "frob": s["frob"], "nnz_M": s["nnz_M"], "n_c": s["n_c"], "n_failed": s["n_failed"],
            "qr_flops": s["qr_flops"], "p_max": s["p_max"], "q_max": s["q_max"],
            "oracle_sample": {"columns": len(cols), "max_rel_rho_diff": float(rel.max()),
                              "within_1e-5": int((rel <= 1e-5).sum()), "oracle_s": osec},
            "fp64_gpu_build": "omitted: ~3e14 FP64 flops, over 280 s at the GPU's FP64 rate"}


def batch_extra(members):
    """`members` of the 512-member batch (half convection-diffusion, half power
    law, n uniform in [1000, 50000]) in one graph-replayed build, FP32+refine,
    with the backward on the frozen pattern and each member's ||A_b M_b - I||_F
    against the FP64 build of the same batch."""
    from paper_1503_04500_gb300 import sweep

    r = sweep.run_batch(count=members, nmax=50000, precision="fp32_refine", rebuilds=1)
    r["members_of_512"] = members
    return r


def reference_arm(args):
    """The FP64 CPU oracle as it stands, on the host cores (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1503_04500_gb300 import inputs

    A = inputs.convdiff3d(64)
    threads = os.cpu_count() or 1
    stride = 2  # each step: every 2nd column (131072 columns)
    for _ in range(args.warmup):
        run_oracle_sample(A, threads, stride * 4)
    times = []
    ncols = 0
    for _ in range(args.steps):
        ncols, dt, _ = run_oracle_sample(A, threads, stride)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = ncols / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "columns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, **PARAMS},
        "cpu_baseline": {"value": value, "unit": "columns/s", "cores": threads, "kind": "oracle",
                         "sample": f"1 column in {stride} ({ncols} of {A.n}) per step"},
        "e2e": {"value": value, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip every measurement besides the 64^3 workload")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the n = 1e6 power law, the batch and the SPAI comparison (a few minutes)")
    ap.add_argument("--batch-members", type=int, default=8,
                    help="members of the 512-member batch configuration built in the batch measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
        return

    import numpy as np
    import torch

    from paper_1503_04500_gb300 import inputs, rsai

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        rank_barrier(pg)
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return rank_max(pg, x, "cuda")

    rsai.load()
    A = inputs.convdiff3d(64)
    dA = rsai.DeviceMatrix.from_host(A)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def timed(handle, steps):
        st = torch.cuda.current_stream()
        ms = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            handle.rebuild()
            e1.record(st)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ms]

    from paper_1503_04500_gb300 import autotune
    from paper_1503_04500_gb300.autograd import Pattern, preconditioned_solve_loss

    h32 = rsai.build(dA, precision="fp32_refine", **PARAMS)
    h64 = rsai.build(dA, precision="fp64", **PARAMS)
    tuned32 = autotune.tune(h32, A.nnz, "fp32_refine", steps=3)
    tuned64 = autotune.tune(h64, A.nnz, "fp64", steps=2)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        h32.rebuild()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    barrier()
    with ClockSampler(uuid) as clk:
        barrier()
        t_wall0 = time.perf_counter()
        ms32 = timed(h32, args.steps)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    clocks = clk.summary()
    dev_ms = max_over_ranks(sum(ms32)) / args.steps
    s32 = h32.stats()
    # FP64 path at the same parameters (the comparison of the metric)
    k64 = max(3, args.steps // 5)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        h64.rebuild()
    barrier()
    ms64 = timed(h64, k64)
    barrier()
    dev_ms64 = max_over_ranks(sum(ms64)) / k64
    s64 = h64.stats()

    # adjoint on the frozen pattern (loss ||AM - I||_F^2: dL/dM = 0, dL/drho_k^2 = 1)
    def bwd_ms(handle, steps):
        nnz = handle.stats()["nnz_M"]
        gM = torch.zeros(nnz, dtype=torch.float64, device="cuda")
        gr = torch.ones(A.n, dtype=torch.float64, device="cuda")
        for _ in range(2):
            handle.backward(dA.val, gM, gr)
        st = torch.cuda.current_stream()
        out = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            handle.backward(dA.val, gM, gr)
            e1.record(st)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return max_over_ranks(statistics.median(out))

    kb = max(3, args.steps // 10)
    bwd32 = bwd_ms(h32, kb)
    bwd64 = bwd_ms(h64, kb)

    # roofline of the dominant kernel (the warp bin): live per-phase CUDA events
    phases32, phases64 = [], []
    for _ in range(5):
        flush.fill_(1.0)
        phases32.append(h32.phase_times())
        flush.fill_(1.0)
        phases64.append(h64.phase_times())
    ph32 = {k: statistics.median(p[k] for p in phases32) for k in phases32[0]}
    ph64 = {k: statistics.median(p[k] for p in phases64) for k in phases64[0]}
    f32_meas = rsai.peak_fma(False)
    f64_meas = rsai.peak_fma(True)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    hbm_gbs, hbm_src = measured_hbm_gbs()
    sm_max_mhz = clocks.get("sm_max_mhz") or 2070.0

    def roofline(stats, ph, precision):
        # the warp-bin phase runs bin H (half a warp per column) and then bins W, W2 (a warp per column)
        t = ph["bin_warp"] / 1e3
        all_in_h = stats.get("cols_bin_half", 0) == stats["n"]
        all_in_w = stats["cols_bin"][0] == stats["n"]
        kname = "k_bin_half" if all_in_h else "k_bin_warp"
        if precision == "fp32_refine":
            F32 = stats["qr_flops"] + stats["refine_flops"]
            F64 = stats["res_flops"] + stats["refine_flops_f64"]
        else:
            F32 = 0.0
            F64 = stats["qr_flops"] + stats["res_flops"]
        t32, t64 = F32 / f32_meas, F64 / f64_meas
        pipe = "fp32" if t32 >= t64 else "fp64"
        F, P = (F32, f32_meas) if pipe == "fp32" else (F64, f64_meas)
        P_units = fp32_units_peak(sms, sm_max_mhz) if pipe == "fp32" else PEAK_FP64_PUBLISHED
        return {
            "bound": "alu", "pipe": pipe, "kernel": f"{kname}<{'float' if precision != 'fp64' else 'double'}>",
            "achieved": F / t / 1e12, "peak": P / 1e12, "unit": "TFLOP/s", "frac": (F / t) / P,
            "traffic": traffic_from_profiles(kname, precision),
            "peak_source": f"measured on this GPU: FMA-chain kernel (rsai_peak_fma), {pipe.upper()}",
            "peak_units": P_units / 1e12, "frac_of_units_peak": (F / t) / P_units,
            "peak_units_source": (f"{sms} SMs x 128 lanes x 2 flop x {sm_max_mhz:.0f} MHz" if pipe == "fp32"
                                  else "published GB300 FP64 rate"),
            "launch_ms": ph["bin_warp"], "flops_fp32": F32, "flops_fp64": F64,
            "t_roof_ms": 1e3 * max(t32, t64, stats["bytes"] / (hbm_gbs * 1e9)),
            "all_columns_in_kernel": all_in_h or (kname == "k_bin_warp" and all_in_w),
            "columns_half_bin": stats.get("cols_bin_half", 0),
            "algorithmic_bytes": stats["bytes"], "hbm_gbs": hbm_gbs, "hbm_source": hbm_src, "sms": sms,
        }

    roof32 = roofline(s32, ph32, "fp32_refine")
    roof64 = roofline(s64, ph64, "fp64")

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).pin_memory()  # noqa: E731
        hA = rsai.DeviceMatrix(A.n, A.nnz, pin(A.row_ptr, np.int64), pin(A.col_idx, np.int32),
                               pin(A.val, np.float64), pin(A.col_ptr, np.int64), pin(A.row_idx, np.int32),
                               pin(A.cval, np.float64))
        cap = s32["nnz_M"] + 1
        out = (torch.empty(A.n + 1, dtype=torch.int64).pin_memory(), torch.empty(cap, dtype=torch.int32).pin_memory(),
               torch.empty(cap, dtype=torch.float64).pin_memory())
        h2d = 2 * (8 * (A.n + 1) + 12 * A.nnz)
        e2e_t = []
        d2h = 0
        for i in range(args.e2e_steps + 1):
            barrier()
            t0 = time.perf_counter()
            h = rsai.build(hA, precision="fp32_refine", **PARAMS)
            st = h.stats()
            h.M_host(st["nnz_M"], out=out)
            h.free()
            t1 = time.perf_counter()
            if i > 0:
                e2e_t.append(t1 - t0)
            d2h = 8 * (A.n + 1) + 12 * st["nnz_M"] + 200
        e2e_s = max_over_ranks(sum(e2e_t) / len(e2e_t))
        e2e = {"value": job_throughput(world, A.n, e2e_s), "unit": "columns/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s}

    # parametric 2-D problem (256^2, A(theta) = L/h^2 + theta1 Cx + theta2 Cy): forward and adjoint
    c4 = None
    if args.extras:
        P4 = inputs.parametric2d(256, (30.0, 10.0))
        d4 = rsai.DeviceMatrix.from_host(P4.base)
        c4 = {"workload": "parametric2d_256^2_theta(30,10)", "n": P4.base.n}
        for prec in ("fp32_refine", "fp64"):
            h4 = rsai.build(d4, precision=prec, **PARAMS)
            autotune.tune(h4, P4.base.nnz, prec, steps=2)
            f_ms = statistics.median(timed(h4, 5))
            nnz4 = h4.stats()["nnz_M"]
            gM = torch.zeros(nnz4, dtype=torch.float64, device="cuda")
            gr = torch.ones(P4.base.n, dtype=torch.float64, device="cuda")
            h4.backward(d4.val, gM, gr)
            st4 = torch.cuda.current_stream()
            bt = []
            for _ in range(5):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st4)
                h4.backward(d4.val, gM, gr)
                e1.record(st4)
                torch.cuda.synchronize()
                bt.append(e0.elapsed_time(e1))
            b_ms = statistics.median(bt)
            c4[prec] = {"fwd_ms": f_ms, "bwd_ms": b_ms, "bwd_fwd_ratio": b_ms / f_ms,
                        "columns_per_s": P4.base.n / (f_ms / 1e3), "frob": h4.stats()["frob"]}
            # loss_2 = ||b - A M y_20||^2 (20 BiCGStab iterations) and its gradient in the values of A
            patA, patM = Pattern.of_matrix(P4.base), Pattern.of_M(h4)
            b4 = torch.as_tensor(inputs.ones_rhs(P4.base), device="cuda")
            lt = {"fwd": [], "fwd_bwd": []}
            for rep in range(4):
                for kind in ("fwd", "fwd_bwd"):
                    av = d4.val.clone().requires_grad_(kind == "fwd_bwd")
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st4)
                    L2 = preconditioned_solve_loss(av, h4, patA, patM, b4, 20)
                    if kind == "fwd_bwd":
                        L2.backward()
                    e1.record(st4)
                    torch.cuda.synchronize()
                    if rep > 0:
                        lt[kind].append(e0.elapsed_time(e1))
            c4[prec]["loss2_y20"] = {"value": L2.item(), "fwd_ms": statistics.median(lt["fwd"]),
                                     "fwd_bwd_ms": statistics.median(lt["fwd_bwd"])}
            h4.free()

    # the uneven-size configurations: the n = 1e6 power law and a batch of the 512-member set
    c3 = c5 = spai_cmp = None
    if args.extras and args.large:
        c3 = powerlaw_1e6_extra(torch, np, rsai, inputs)
        c5 = batch_extra(args.batch_members)
        from paper_1503_04500_gb300 import sweep

        spai_cmp = {}
        for wl, size in (("convdiff3d", 32), ("powerlaw", 20000)):
            r = sweep.compare_spai(wl, size, precision="fp64", rebuilds=1)
            spai_cmp[f"{wl}_{size}"] = {"rsai": {k: r["rsai"][k] for k in SPAI_KEYS},
                                        "spai": {k: r["spai"][k] for k in SPAI_KEYS}, **r["ratio"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        ncols, dt, Mo = run_oracle_sample(A, threads, 1)
        cpu = {"value": ncols / dt, "unit": "columns/s", "cores": threads, "kind": "oracle",
               "sample": f"all {ncols} columns of the workload, FP64, {threads} threads", "seconds": dt,
               "frob_oracle": Mo.frob()}
        # the same oracle on one thread, on every 16th column (columns are independent)
        n1, dt1, _ = run_oracle_sample(A, 1, 16)
        cpu["single_thread"] = {"value": n1 / dt1, "unit": "columns/s", "cores": 1,
                                "sample": f"every 16th column ({n1} of {A.n}), FP64, 1 thread", "seconds": dt1}

    value = job_throughput(world, A.n, dev_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "columns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64refine", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, **PARAMS, "precision": "fp32_refine",
                   "l2": "flushed (256 MB write) between timed steps", "replicas": world},
        "frob": s32["frob"], "nnz_M": s32["nnz_M"], "n_c": s32["n_c"],
        "fp64": {"value": job_throughput(world, A.n, dev_ms64 / 1e3), "ms_per_step": dev_ms64, "frob": s64["frob"],
                 "nnz_M": s64["nnz_M"], "roofline": roof64, "phases_ms": ph64},
        "frob_rel_diff_fp32r_vs_fp64": abs(s32["frob"] - s64["frob"]) / s64["frob"],
        "speedup_fp32r_vs_fp64": dev_ms64 / dev_ms,
        "bwd_fwd_ratio": bwd32 / dev_ms,
        "bwd_ms": bwd32, "bwd_fwd_ratio_fp64": bwd64 / dev_ms64,
        "roofline": roof32, "phases_ms": ph32,
        "tuning": {"fp32_refine": tuned32["tuning"], "fp64": tuned64["tuning"]},
        "parametric2d_256": c4, "powerlaw_1e6": c3, "batch": c5, "rsai_vs_spai": spai_cmp,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        # the half-warp bin adds one launch when the tuned shape uses it
        # (+1: the FP32 copy of A's values that an FP32+refine build makes)
        "gpu_launches": (KERNELS_PER_BUILD + 1 + int(tuned32["tuning"].get("half_bin", 0))) * args.steps,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h32.free()
    h64.free()
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
