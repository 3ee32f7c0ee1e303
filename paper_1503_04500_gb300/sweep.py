"""Parameter sweeps of RSAI(tol) on the synthetic workloads (the analogue of
the paper's tables of ε, c and l_max against sparsity, iterations and time,
Section 5), for the right preconditioner (A M ≈ I) or the left one (M A ≈ I,
built on Aᵀ by the same kernels).

    python -m paper_1503_04500_gb300.sweep --workload convdiff3d --size 32 \
        --eps 0.2,0.3,0.4 --c 3,5 --lmax 5,10 --precision fp32_refine
    python -m paper_1503_04500_gb300.sweep --batch 64 --size 5000 --precision fp32_refine
    python -m paper_1503_04500_gb300.sweep --compare-spai --workload powerlaw --size 20000

One JSON line per setting: spar = nnz(M)/nnz(A), ||AM - I||_F (or ||MA - I||_F),
n_c (columns with ||r_k|| > ε), the build time (median of graph-replayed
rebuilds, CUDA events), and right-preconditioned BiCGStab on A M y = b,
b = A·1, rtol 1e-8 (iterations and time; right variant only).
"""
from __future__ import annotations

import argparse
import itertools
import json
import statistics
import time

from . import inputs, rsai


def _workload(name: str, size: int, seed: int):
    if name == "convdiff2d":
        return inputs.convdiff2d(size, (20.0, 20.0))
    if name == "convdiff3d":
        return inputs.convdiff3d(size)
    if name == "powerlaw":
        return inputs.powerlaw(size, seed=seed)
    if name == "parametric2d":
        return inputs.parametric2d(size).base
    raise ValueError(f"unknown workload {name}")


def _floats(s: str):
    return [float(x) for x in s.split(",") if x]


def _ints(s: str):
    return [int(x) for x in s.split(",") if x]


def run(workload="convdiff2d", size=20, seed=1503, eps=(0.3,), c=(3,), lmax=(10,), drop="fixed", tol=1e-3,
        precision="fp64", side="right", rebuilds=5, solve=True, init="identity", select="rsai", A=None,
        global_ctas=0):
    """Yield one result dict per (eps, c, l_max) setting.  `global_ctas` > 0:
    the rebuilds run the global bin on that many CTAs (and workspace slabs)."""
    import torch

    A = A if A is not None else _workload(workload, size, seed)
    dA = rsai.DeviceMatrix.from_host(A)
    b = torch.as_tensor(inputs.ones_rhs(A), device="cuda")
    st = torch.cuda.current_stream()
    for e, cc, lm in itertools.product(eps, c, lmax):
        kw = dict(c=cc, l_max=lm, eps=e, drop=drop, tol=tol, precision=precision, init=init, select=select)
        t0 = time.perf_counter()
        h = rsai.build_left(dA, **kw) if side == "left" else rsai.build(dA, **kw)
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        right = h.right if side == "left" else h
        if global_ctas > 0:
            right.set_tuning(global_bin_ctas=global_ctas)
        times = []
        for _ in range(rebuilds):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            right.rebuild()
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        s = h.stats()
        out = {"workload": workload, "n": A.n, "nnz_A": A.nnz, "side": side, "init": init, "precision": precision,
               "select": select, "eps": e,
               "c": cc, "l_max": lm, "drop": drop, "tol": tol, "spar": s["nnz_M"] / A.nnz, "frob": s["frob"],
               "n_c": s["n_c"], "p_max": s["p_max"], "q_max": s["q_max"], "cols_bin": s["cols_bin"],
               "qr_flops": s["qr_flops"], "select_flops": s["select_flops"], "loops": s["loops"],
               "build_ms": statistics.median(times) if times else None, "first_build_s": first_s,
               "phases_ms": right.phase_times()}
        if solve and side == "right":
            t1 = time.perf_counter()
            _, iters, relres, status = rsai.bicgstab(dA, h, b)
            torch.cuda.synchronize()
            out.update({"bicgstab_iters": iters, "bicgstab_relres": relres, "bicgstab_status": status,
                        "bicgstab_s": time.perf_counter() - t1})
        h.free()
        yield out


def compare_spai(workload="powerlaw", size=20000, seed=1503, precision="fp64", rebuilds=5, A=None):
    """RSAI(tol) against SPAI on one synthetic matrix, with Section 5.2's
    settings (the analogue of its table): RSAI(tol) with eps = 0.3, c = 3,
    l_max = 10 and the drop of Eq. 4.3 (FIXED tol = 1e-3 on A/||A||_1); SPAI
    with the same eps, three most profitable indices per loop, no dropping and
    l_max = floor(10 nnz(A) / (3 n)) (which keeps nnz(M)/nnz(A) <= 5).  Returns
    both rows (spar, build time, n_c, BiCGStab iterations and time) and the
    ratios SPAI / RSAI(tol) of build time and iterations."""
    import math

    A = A if A is not None else _workload(workload, size, seed)
    lm_spai = int(math.floor(10 * A.nnz / (3 * A.n)))
    r = next(run(workload, size, seed, (0.3,), (3,), (10,), "fixed", 1e-3, precision, "right", rebuilds, True,
                 "identity", "rsai", A))
    sp = next(run(workload, size, seed, (0.3,), (3,), (lm_spai,), "none", 1e-3, precision, "right", rebuilds, True,
                  "identity", "spai", A))
    ratio = {"build_time_spai_over_rsai": sp["build_ms"] / r["build_ms"] if r["build_ms"] else None,
             "iters_spai_over_rsai": (sp["bicgstab_iters"] / r["bicgstab_iters"]) if r.get("bicgstab_iters") else None,
             "n_c_rsai": r["n_c"], "n_c_spai": sp["n_c"], "spar_rsai": r["spar"], "spar_spai": sp["spar"]}
    return {"rsai": r, "spai": sp, "ratio": ratio}


def run_batch(count=64, nmax=5000, precision="fp32_refine", c=3, l_max=10, eps=0.3, drop="fixed", tol=1e-3,
              rebuilds=5):
    """The batch configuration at a chosen size: `count` members (half
    convection-diffusion, half power law, n uniform in [1000, nmax]) built as one
    block-diagonal problem in one graph.  Returns the aggregate columns/s of the
    graph-replayed build, the backward time on the frozen pattern, and, for an
    FP32+refine batch, the largest relative ||A_b M_b - I||_F difference per
    member from the FP64 build of the same batch."""
    import numpy as np
    import torch

    members = [inputs.random_batch_member(i, nmax=nmax) for i in range(count)]
    ntot = sum(A.n for A in members)
    kw = dict(c=c, l_max=l_max, eps=eps, drop=drop, tol=tol)
    h = rsai.build_batch(members, precision=precision, **kw)
    st = torch.cuda.current_stream()
    times = []
    for _ in range(rebuilds):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h.rebuild()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    fwd_ms = statistics.median(times)
    frob, nc, nz = h.block_stats(count)
    # backward on the frozen pattern (the members' values side by side)
    vals = torch.as_tensor(np.concatenate([A.val for A in members]), device="cuda")
    nnzM = h.stats()["nnz_M"]
    gM = torch.ones(nnzM, dtype=torch.float64, device="cuda")
    h.backward(vals, gM)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    h.backward(vals, gM)
    e1.record(st)
    torch.cuda.synchronize()
    bwd_ms = e0.elapsed_time(e1)
    s = h.stats()
    h.free()
    rel = None
    if precision != "fp64":
        h64 = rsai.build_batch(members, precision="fp64", **kw)
        frob64, _, _ = h64.block_stats(count)
        h64.free()
        rel = float(np.max(np.abs(frob - frob64) / frob64))
    return {"workload": f"batch of {count} (n in [1000, {nmax}])", "members": count, "n_total": ntot,
            "nnz_A": int(sum(A.nnz for A in members)), "precision": precision, "cols_bin": s["cols_bin"],
            "build_ms": fwd_ms, "columns_per_s": ntot / (fwd_ms / 1e3), "bwd_ms": bwd_ms,
            "bwd_fwd_ratio": bwd_ms / fwd_ms, "max_member_frob_rel_diff_vs_fp64": rel}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="convdiff2d",
                    choices=["convdiff2d", "convdiff3d", "powerlaw", "parametric2d"])
    ap.add_argument("--size", type=int, default=20, help="grid side N (stencils) or n (power law)")
    ap.add_argument("--seed", type=int, default=1503)
    ap.add_argument("--eps", default="0.3")
    ap.add_argument("--c", default="3")
    ap.add_argument("--lmax", default="10")
    ap.add_argument("--drop", default="fixed", choices=["none", "adaptive", "fixed"])
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_refine"])
    ap.add_argument("--side", default="right", choices=["right", "left"])
    ap.add_argument("--rebuilds", type=int, default=5)
    ap.add_argument("--no-solve", dest="solve", action="store_false")
    ap.add_argument("--init", default="identity", choices=["identity", "A"],
                    help="initial pattern J_k^(0): {k} or the rows of column k of A")
    ap.add_argument("--select", default="rsai", choices=["rsai", "spai"],
                    help="new indices: dominant rows (Algorithm 1) or SPAI's most profitable (Eqs. 2.5-2.7)")
    ap.add_argument("--compare-spai", action="store_true",
                    help="instead of a sweep: RSAI(tol) against SPAI with Section 5.2's settings")
    ap.add_argument("--global-ctas", type=int, default=0,
                    help="CTAs (and workspace slabs) of the global bin in the rebuilds, 0 = one per SM")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of a sweep: a batch of this many random members (n up to --size) in one build")
    a = ap.parse_args(argv)
    if a.compare_spai:
        print(json.dumps(compare_spai(a.workload, a.size, a.seed, a.precision, max(a.rebuilds, 1))), flush=True)
        return
    if a.batch > 0:
        print(json.dumps(run_batch(a.batch, a.size, a.precision, _ints(a.c)[0], _ints(a.lmax)[0], _floats(a.eps)[0],
                                   a.drop, a.tol, max(a.rebuilds, 1))), flush=True)
        return
    for row in run(a.workload, a.size, a.seed, _floats(a.eps), _ints(a.c), _ints(a.lmax), a.drop, a.tol,
                   a.precision, a.side, a.rebuilds, a.solve, a.init, a.select, None, a.global_ctas):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
