"""Benchmark of the fast IMQ product A v (arXiv 2205.04194) on one GB300 per rank.

Default workload: the N = 1,000,000 clustered point set (8 Gaussians of
87,500 points, sigma 0.03, clamped to [0,1]^2, plus 300,000 uniform points),
shape c = 0.01, adaptive quadtree with leaf 64, expansion order p = 12.

A step is one fast product b = A v through the C ABI (gather, P2M, M2M, M2L,
P2L, L2L, L2P+M2P, P2P, scatter) on device-resident FP32 input.  The tree
and operators (imq_plan) are built once before the timed region and timed
separately.  Between timed steps a 512 MiB buffer is written to flush the
129 MB L2 (untimed); each step is bracketed by CUDA events on the launching
stream, and the per-phase kernel times come from the library's own events on
that stream.

One JSON line on rank 0.  With torchrun (N > 1) every rank runs an
independent replica of the same problem ("replicas only": the single-problem
product is not sharded); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IMQ A·v time & CG solve s at 1e-6 rel err, fast vs dense GPU matvec, N=1M"
MUFU_PER_CLK_SM = 16        # rsqrt (MUFU) results per clock per SM
FP32_FMA_PER_CLK_SM = 128   # FP32 lanes per SM
N_SM = 152
FP16_PER_BF16 = 1.0         # nominal dense tensor rates per GPU: fp16 and bf16 are equal


# DRAM traffic per launch of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum),
# from one single-kernel ncu capture on the quarter-size clustered workload, scaled to the 1M launch
# by the units it processes; keyed by the SHA-256 of the kernel sources at capture time: once a
# source changes the figure is stale and the bench reports null.
TRAFFIC = {
    # k_m2l_umma<3>: 22.574848 MB read, 0 written per launch at N = 250,000 (267,324 V pairs), scaled by
    # the V pairs (x 1,121,136 / 267,324) to the 1M launch
    "m2l": {"bytes": 22.574848e6 * 1121136 / 267324, "sources": {
        "paper_2205_04194_gb300/csrc/m2l_umma.cu": "2382ca23c6659b5973089438a6f5dd5615f3786aaa39f452af1da025d4a7d0f4",
        "paper_2205_04194_gb300/csrc/umma.cuh": "389ed8c09540f0a3e24b70570e9738f6acff25805ba38fc440f7a8f9f2b6336e",
        "paper_2205_04194_gb300/csrc/ptx.cuh": "9f11aae585d997f977cfb9515e1a6d3900bf168e91c1a75824dfdb29176bb76c"}},
}


def _traffic(kernel: str):
    import hashlib
    rec = TRAFFIC.get(kernel)
    if rec is None:
        return None
    for rel, digest in rec["sources"].items():
        if digest is None:
            continue
        with open(os.path.join(ROOT, rel), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != digest:
                return None
    return rec["bytes"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"imq_bench_clocks_{os.getpid()}_rank{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over the ranks of the default process group (x itself
    without one): the step time of a replicated run is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_rows(points, c, v, seconds: float, min_rows: int = 8):
    """Time the FP64 dense oracle (O1) on a sample of rows sized to ~`seconds`."""
    from oracle import dense
    n = points.shape[0]
    rng = np.random.default_rng(123)
    rows = rng.choice(n, min_rows, replace=False)
    t0 = time.perf_counter()
    dense.matvec_rows(points, c, v, rows)
    t1 = time.perf_counter() - t0
    nrows = int(max(min_rows, min(n, min_rows * seconds / max(t1, 1e-3))))
    rows = rng.choice(n, nrows, replace=False)
    t0 = time.perf_counter()
    vals = dense.matvec_rows(points, c, v, rows)
    dt = time.perf_counter() - t0
    return dt, nrows, rows, vals, dense.num_threads()


def run_reference(args, wl):
    """The oracle as it stands, on the host cores: FP64 dense rows, scaled to one A v."""
    from oracle import dense
    n = wl.n
    rows_per_step = args.ref_rows
    rng = np.random.default_rng(7)
    times = []
    for k in range(args.warmup + args.steps):
        rows = rng.choice(n, rows_per_step, replace=False)
        t0 = time.perf_counter()
        dense.matvec_rows(wl.points, wl.c, wl.v, rows)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt / rows_per_step * n)
    ms = 1e3 * statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": n, "c": wl.c, "p": wl.p, "leaf": wl.leaf},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": dense.num_threads(), "kind": "oracle",
                             "sample": f"{rows_per_step} rows of the FP64 dense product per step, "
                                       f"scaled by N/rows to one full A v"},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, imq, dev):
    """256 independent problems (N log-uniform in [1e3, 5e4], c uniform in [0.01, 0.2], 4 right-hand
    sides) in one batched plan: plan build, the 4-RHS product, its error on 16 whole problems against
    the dense FP64 product, and a capped CG solve."""
    import torch
    from paper_2205_04194_gb300 import workloads as W
    probs = W.batched_256()
    pts = [torch.from_numpy(x).to(dev) for x, _, _ in probs]
    cs = [c for _, c, _ in probs]
    f = torch.from_numpy(np.concatenate([r for _, _, r in probs], axis=1)).to(dev)   # [4, N_total]
    # leaf size, p and translations by the autotuner: 1e-6 on 32 sampled rows of every problem, tested
    # on the workload's own 4 right-hand sides (the trig sums cancel in the far field)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tune = imq.autotune(pts, cs, 1e-6, p_candidates=(8, 10, 12, 14, 16), leaf_candidates=(32, 64, 128), nrhs=4,
                        domain=(0.0, 0.0, 1.0), v=f.float().contiguous())
    tune_s = time.perf_counter() - t0
    P_b, leaf_b = tune["p"], tune["leaf"]
    tiles = imq.tiles_of(tune)
    n_tot = None
    f32 = f.float().contiguous()
    offs = None
    out = {"n_problems": len(probs), "nrhs": 4, "p": P_b, "leaf": leaf_b,
           "autotune": {"seconds": tune_s, "met": tune["met"], "rel_err": tune["rel_err"],
                        "sampled_rows": tune["sampled_rows"], "choice": tiles,
                        "tried": [(t["p"], t["leaf"], t["translations"], t["p2p_warps"], t["p2p_chunk"],
                                   t["m2l_stages"], t["rel_err"], t["matvec_ms"]) for t in tune["tried"]]}}
    # the tuned configuration, and the same (p, leaf) with the other translation precision: the tuner
    # measures its error on its own random vectors, while the workload's trig-sum right-hand sides
    # cancel in the far field, so FP64 translations can be what meets 1e-6 on the actual data
    variants = [("tuned", tiles)]
    for tr in ("fp32", "mixed", "fp64"):
        if tiles["translations"] != tr:
            variants.append((tr + "_translations", dict(tiles, translations=tr)))
    for name, kw in variants:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bp = imq.BatchedPlan(pts, cs, P_b, leaf_b, domain=(0.0, 0.0, 1.0), **kw)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        n_tot, offs = bp.n, bp.offsets
        for _ in range(3):
            bp.matvec(f32)
        reps = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            b32 = bp.matvec(f32)
        e1.record()
        torch.cuda.synchronize()
        mv_ms = e0.elapsed_time(e1) / reps
        # accuracy on 16 problems, every right-hand side, against the FP64 dense product on the GPU
        errs = []
        for b in np.linspace(0, len(probs) - 1, 16).astype(int):
            sl = slice(int(offs[b]), int(offs[b + 1]))
            ref = imq.dense_matvec(pts[b], cs[b], f[:, sl].contiguous())
            got = b32[:, sl].double()
            errs.append([float(((got[r] - ref[r]).norm() / ref[r].norm()).item()) for r in range(4)])
        errs = np.array(errs)
        out[name] = {"plan": kw, "plan_build_s": build_s, "matvec_f32_ms": mv_ms,
                     "ns_per_point_rhs": mv_ms * 1e6 / (4 * bp.n),
                     "matvec_points_per_s": 4 * bp.n / (mv_ms * 1e-3),
                     "sampled_rel2_err_max": float(errs.max()), "meets_1e-6": bool(errs.max() <= 1e-6),
                     "sampled_rel2_err_max_per_rhs": errs.max(axis=0).tolist(), "sampled_problems": 16}
        if kw.get("translations", "fp32") == "fp32" and "cg" not in out:   # solves on the FP32-translation plan
            for key, kk in (("cg", dict(krylov="cg")), ("gmres", dict(krylov="gmres", gmres_m=40)),
                            ("gmres_two_level", dict(krylov="gmres", gmres_m=40, precond="schwarz2",
                                                     coarse_points=1024))):
                kk = dict(dict(precond="schwarz"), **kk)
                coef, info = bp.solve(f, rtol=1e-6, maxit=args.batched_cg_maxit, schwarz_shift=1e-4, **kk)
                rel = info["problem_rel_residual"]
                out[key] = {"rtol": 1e-6, "maxit_per_rhs": args.batched_cg_maxit,
                            "krylov": "PCG" if kk["krylov"] == "cg" else "GMRES(40), per-problem scalars",
                            "precond": kk["precond"] + " (224-point patches, shift 1e-4/c"
                                       + (", coarse boxes <= 1024 points per problem)" if "coarse_points" in kk else ")"),
                            "status": info["status"], "iterations_max": info["iterations"],
                            "solve_s": info["seconds"], "converged_fraction": float((rel <= 1e-6).mean()),
                            "rel_residual_median": float(np.median(rel)), "rel_residual_max": float(rel.max()),
                            "residual_product": "fast FP64 of the batched plan",
                            "note": "1024 systems (256 problems x 4 right-hand sides); c/h up to ~45"}
        bp.close()
    out["n_total"] = n_tot
    return out


def run_solves(args, imq, wl, d_pts, plan, dev):
    """CG solves (metric config and the 100k config), the paper's Table 1 workload and the
    200k gradient config.  Each is bounded so the default run stays within minutes."""
    import torch
    from paper_2205_04194_gb300 import workloads as W
    out = {}
    # the solve at the metric configuration: f = Franke, 1e-6.  CG with the one- and two-level
    # Schwarz preconditioners loses the sign of p.Ap / r.z at this conditioning (c/h up to ~40) and
    # stalls; restarted GMRES on the same two-level preconditioner converges.  Each solve's true
    # residual is the plan's FP64 fast product (p = 12); the metric solve is also certified with the
    # FP64 fast product at p = 16 and with the dense FP64 product on the GPU.
    f = torch.from_numpy(wl.f).to(dev)
    solves = (("cg_one_level", dict(precond="schwarz", schwarz_shift=1e-5)),
              ("cg_two_level", dict(precond="schwarz2", coarse_points=1024, schwarz_shift=1e-5)),
              ("cg", dict(precond="schwarz2", coarse_points=1024, schwarz_shift=1e-4, krylov="gmres", gmres_m=40)))
    for key, kw in solves:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        coef, info = plan.solve(f, rtol=1e-6, maxit=args.cg_maxit, **kw)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        krylov = kw.get("krylov", "cg")
        out[key] = {"workload": wl.name, "rtol": 1e-6, "maxit": args.cg_maxit,
                    "krylov": "restarted GMRES(40), right-preconditioned" if krylov == "gmres" else "PCG",
                    "precond": kw["precond"] + " (224-point patches, shift %g/c" % kw["schwarz_shift"]
                               + (", coarse boxes <= 1024 points)" if "coarse_points" in kw else ")"),
                    "operator": "fast_f32", "status": info["status"], "iterations": info["iterations"],
                    "outer_steps": info["outer_steps"], "solve_s": info["seconds"],
                    "wall_s_incl_setup": wall, "s_per_iter": info["seconds"] / max(1, info["iterations"]),
                    "true_rel_residual": info["max_rel_residual"], "residual_product": "fast FP64, same tree (p = 12)"}
        if key == "cg":
            # independent certificates of the returned coefficients
            p16 = imq.Plan(d_pts, wl.c, 16, wl.leaf, domain=wl.domain)
            r16 = float((f - p16.matvec(coef)).norm() / f.norm())
            p16.close()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rd = float((f - imq.dense_matvec(d_pts, wl.c, coef)).norm() / f.norm())
            torch.cuda.synchronize()
            out[key].update({"true_rel_residual_fast_f64_p16": r16, "true_rel_residual_dense_f64": rd,
                             "dense_f64_residual_s": time.perf_counter() - t1,
                             "coef_norm_over_f_norm": float(coef.norm() / f.norm()),
                             "note": "solve_s: after preconditioner set-up (patch factors, coarse Gram matrix); "
                                     "wall_s_incl_setup includes it"})
    # 100k uniform, c = 2 x mean NN spacing, FP32 inner / FP64 refinement to 1e-8
    u = W.uniform_100k()
    pl = imq.Plan(torch.from_numpy(u.points).to(dev), u.c, u.p, u.leaf, domain=u.domain)
    coef, info = pl.solve(torch.from_numpy(u.f).to(dev), rtol=1e-8, maxit=3000, precond="schwarz",
                          refine_steps=8, inner_rtol=1e-5, residual="dense")
    out["cg_uniform_100k"] = {"n": u.n, "c": u.c, "p": u.p, "leaf": u.leaf, "rtol": 1e-8,
                              "status": info["status"], "iterations": info["iterations"],
                              "outer_steps": info["outer_steps"], "solve_s": info["seconds"],
                              "true_rel_residual": info["max_rel_residual"], "residual_product": "dense FP64"}
    pl.close()
    # the paper's Table 1 workload: Halton points, c = 1, p = 10, random vector in [-1, 1]
    rows = []
    for n in (20000, 40000, 60000, 80000, 100000):
        t = W.table1_halton(n)
        dp = torch.from_numpy(t.points).to(dev)
        dv = torch.from_numpy(t.v).to(dev)
        pt = imq.Plan(dp, t.c, 10, 64, domain=t.domain)
        ref = imq.dense_matvec(dp, t.c, dv)                        # FP64 dense on the GPU
        b64 = pt.matvec(dv)
        for _ in range(2):
            pt.matvec(dv.float())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b32 = pt.matvec(dv.float())
        e1.record()
        torch.cuda.synchronize()
        fast_ms = e0.elapsed_time(e1)
        e0.record()
        imq.dense_matvec(dp, t.c, dv.float())
        e1.record()
        torch.cuda.synchronize()
        dense_ms = e0.elapsed_time(e1)
        rinf = lambda a: float((a.double() - ref).abs().max() / ref.abs().max())
        row = {"n": n, "fast_f32_ms": fast_ms, "dense_f32_ms": dense_ms, "einf_fast_f32": rinf(b32),
               "einf_fast_f64": rinf(b64)}
        pt.close()
        # the paper's own method (Algorithm 1, uniform levels L in {1, 2, 3}, the best reported
        # as in Table 1), FP64 as in the paper and FP32
        best = None
        for lv in (1, 2, 3):
            tc = imq.Plan(dp, t.c, 10, 0, domain=t.domain, algorithm="treecode", levels=lv)
            for dt_, vv in (("f64", dv), ("f32", dv.float())):
                tc.matvec(vv)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(3):
                    bt = tc.matvec(vv)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 3
                key = "treecode_" + dt_
                if best is None or key not in best or ms < best[key]["ms"]:
                    best = best or {}
                    best[key] = {"L": lv, "ms": ms, "einf": rinf(bt)}
            tc.close()
        row.update(best)
        rows.append(row)
    out["table1"] = {"c": 1.0, "p": 10, "leaf": 64, "rows": rows,
                     "note": "fast = adaptive FMM (leaf 64); treecode = the paper's Algorithm 1 on uniform levels, "
                             "best L of {1, 2, 3}.  Paper Table 1 (Xeon E5-2620 v3, FP64): dense 1.62..128 s, "
                             "translation 1.58..23.3 s, E 2.67e-9..1.06e-8"}
    out["batched_256"] = run_batched(args, imq, dev)
    # gradient of the validation loss at N = 200k, 20k validation points, c = 0.05 (the configuration:
    # c/h ~ 45, the solves are capped and their status and residual are reported beside the gradient)
    from paper_2205_04194_gb300 import autograd as AG
    g = W.grad_200k()
    d_tr, d_va = torch.from_numpy(g["train"]).to(dev), torch.from_numpy(g["val"]).to(dev)
    d_y = torch.from_numpy(g["y_val"]).to(dev)
    ct = torch.tensor(g["c"], dtype=torch.float64, requires_grad=True)
    ft = torch.from_numpy(g["f"]).to(dev).requires_grad_(True)
    cg = dict(rtol=1e-6, maxit=args.grad_maxit, precond="schwarz2", coarse_points=1024, schwarz_shift=1e-4,
              krylov="gmres", gmres_m=40)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = AG.InterpLoss.apply(ct, ft, d_tr, d_va, d_y, 12, 64, (0.0, 0.0, 1.0), torch.float32, cg, True)
    L.backward()
    torch.cuda.synchronize()
    li = AG.InterpLoss.last_info
    out["grad"] = {"n_train": 200000, "n_val": 20000, "c": g["c"], "p": 12, "loss": float(L.item()),
                   "dloss_dc": float(ct.grad.item()), "dloss_df_norm": float(ft.grad.norm().item()),
                   "wall_s": time.perf_counter() - t0, "cg_maxit_per_solve": args.grad_maxit,
                   "solve_status": li["status"], "solve_max_rel_residual": li["max_rel_residual"],
                   "solver": "GMRES(40), two-level Schwarz, rtol 1e-6 per solve",
                   "note": "forward + adjoint; at c/h ~ 45 a finite difference of the loss in c needs solves "
                           "far below 1e-6, so the gradient is checked against central differences at the "
                           "well-conditioned shape (grad_wellcond_200k)"}
    # the same loss at a well-conditioned shape, c = 2 x mean NN spacing: gradient through the FP32 fast
    # operator (solves to 1e-10 with FP64 refinement) against central differences of the loss
    c2 = 2.0 * W.mean_nn_spacing(g["train"])
    cg = dict(rtol=1e-10, maxit=6000, precond="schwarz", refine_steps=10, inner_rtol=1e-4)
    ct = torch.tensor(c2, dtype=torch.float64, requires_grad=True)
    ft = torch.from_numpy(g["f"]).to(dev).requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = AG.InterpLoss.apply(ct, ft, d_tr, d_va, d_y, 12, 64, (0.0, 0.0, 1.0), torch.float32, cg)
    L.backward()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    li = AG.InterpLoss.last_info
    hh = 1e-3 * c2

    def loss_at(cv):
        return AG.InterpLoss.apply(torch.tensor(cv, dtype=torch.float64), ft.detach(), d_tr, d_va, d_y, 12, 64,
                                   (0.0, 0.0, 1.0), torch.float64, cg).item()
    fd = (loss_at(c2 + hh) - loss_at(c2 - hh)) / (2 * hh)
    out["grad_wellcond_200k"] = {"n_train": 200000, "n_val": 20000, "c": c2, "p": 12, "loss": float(L.item()),
                                 "dloss_dc": float(ct.grad.item()), "dloss_dc_central_diff": fd,
                                 "rel_diff": abs(float(ct.grad.item()) - fd) / abs(fd), "fd_step": hh,
                                 "wall_s": wall, "solve_status": li["status"],
                                 "solve_max_rel_residual": li["max_rel_residual"],
                                 "note": "gradient: FP32 evaluation and derivative products, FP32 inner CG with "
                                         "FP64 refinement; central differences: the loss with FP64 evaluation"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=None,
                    help="expansion order; default: the autotuner's smallest p in {8, 12, 16} that meets 1e-6")
    ap.add_argument("--phase-steps", type=int, default=20, help="products timed phase by phase (after the timed region)")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the clustered workload (tests)")
    ap.add_argument("--dense-reps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-rows", type=int, default=96)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip CG, Table 1 and gradient sections")
    ap.add_argument("--cg-maxit", type=int, default=200)
    ap.add_argument("--grad-maxit", type=int, default=100)
    ap.add_argument("--batched-cg-maxit", type=int, default=120, help="iteration cap per right-hand side (batched solves)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2205_04194_gb300 import workloads as W
    wl = W.clustered_1m(p=args.p or 12, scale=args.scale)

    if args.impl == "reference":
        if rank == 0:
            from oracle import dense
            dense.build()
            run_reference(args, wl)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2205_04194_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2205_04194_gb300 import imq

    stream = torch.cuda.current_stream()
    d_pts = torch.from_numpy(wl.points).to(dev)
    d_v = torch.from_numpy(wl.v).float().to(dev)
    d_out = torch.empty_like(d_v)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    tune = None
    if args.p is None:
        # the configuration's p in {8, 12, 16}: the smallest whose product meets 1e-6 on sampled rows
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tune = imq.autotune(d_pts, wl.c, 1e-6, p_candidates=(8, 12, 16), leaf_candidates=(wl.leaf,),
                            domain=wl.domain)
        tune["seconds"] = time.perf_counter() - t0
        wl.p = tune["p"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = imq.Plan(d_pts, wl.c, wl.p, wl.leaf, domain=wl.domain)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    info = plan.info()

    for _ in range(args.warmup):
        plan.matvec(d_v, d_out)
    torch.cuda.synchronize()

    # launches of one product (counted by the library), for gpu_launches
    _, _, per_product = plan.matvec_timed(d_v, d_out)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                 # untimed L2 flush
            ev[k][0].record(stream)
            plan.matvec(d_v, d_out)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = per_product * args.steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(step_ms), dev)
    # phase breakdown (library events around each phase's kernels), outside the timed region
    phase_tot = {k: 0.0 for k in imq.Plan.PHASES}
    for k in range(args.phase_steps):
        flush.fill_(float(k))
        _, ph, _ = plan.matvec_timed(d_v, d_out)
        for key, val in ph.items():
            phase_tot[key] += val
    phase_ms = {k: v / max(1, args.phase_steps) for k, v in phase_tot.items()}

    # dense GPU product (the plain form) on the same input
    dense_ms = None
    d_dense = torch.empty_like(d_v)
    if rank == 0 or world > 1:
        imq.dense_matvec(d_pts, wl.c, d_v, d_dense)
        torch.cuda.synchronize()
        dts = []
        for _ in range(args.dense_reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(1.0)
            a.record(stream)
            imq.dense_matvec(d_pts, wl.c, d_v, d_dense)
            b.record(stream)
            torch.cuda.synchronize()
            dts.append(a.elapsed_time(b))
        dense_ms = statistics.mean(dts)

    # the configuration's three orders p in {8, 12, 16}: time per product (L2 flushed) and, below,
    # the sampled error against the FP64 oracle; and the all-FP64 product at the tuned p
    per_p, outs_p = {}, {}
    if rank == 0:
        for pp in (8, 12, 16):
            pl = plan if pp == wl.p else imq.Plan(d_pts, wl.c, pp, wl.leaf, domain=wl.domain)
            o = torch.empty_like(d_v)
            for _ in range(3):
                pl.matvec(d_v, o)
            ts = []
            for k in range(10):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pl.matvec(d_v, o)
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            per_p[pp] = {"fast_f32_ms": statistics.mean(ts), "k_real": pl.info()["k_real"]}
            outs_p[pp] = o
            if pl is not plan:
                pl.close()
        d_v64 = d_v.double()
        o64 = torch.empty_like(d_v64)
        plan.matvec(d_v64, o64)
        ts = []
        for k in range(3):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.matvec(d_v64, o64)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        f64_ms = statistics.mean(ts)

    # end to end through the public API with pinned host buffers
    h_v = torch.from_numpy(wl.v).float().pin_memory()
    h_out = torch.empty_like(h_v).pin_memory()
    e2e = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.matvec(h_v, h_out)                  # H2D of v, product, D2H of b inside the call
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e.append(1e3 * dt)
    e2e_ms = max_over_ranks(statistics.mean(e2e), dev)

    if rank != 0:
        dist.destroy_process_group()
        return

    extras = {}
    if not args.no_solve:
        extras = run_solves(args, imq, wl, d_pts, plan, dev)

    # accuracy on sampled rows against the FP64 oracle, and the CPU baseline
    b_fast = d_out.double().cpu().numpy()
    b_dense = d_dense.double().cpu().numpy()
    cpu = None
    err = {}
    if not args.no_cpu:
        from oracle import dense as O
        O.build()
        dt, nrows, rows, ref, cores = cpu_oracle_rows(wl.points, wl.c, wl.v, args.cpu_seconds)
        cpu = {"value": 1e3 * dt / nrows * wl.n, "unit": "ms", "cores": cores, "cpu_model": cpu_model(),
               "kind": "oracle",
               "sample": f"{nrows} random rows of the FP64 dense product (oracle O1) on the "
                         f"{wl.n}-point workload, scaled by N/rows to one full A v"}
        rel = lambda a: float(np.linalg.norm(a[rows] - ref) / np.linalg.norm(ref))
        err = {"fast_rel2_sampled": rel(b_fast), "dense_gpu_rel2_sampled": rel(b_dense),
               "fast_f64_rel2_sampled": rel(o64.cpu().numpy()), "rows": int(nrows)}
        for pp, o in outs_p.items():
            per_p[pp]["rel2_sampled"] = rel(o.double().cpu().numpy())

    peaks, src = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    clocks = clk.summary()
    p2p_gps = info["p2p_pairs"] / (phase_ms["p2p"] * 1e-3) / 1e9
    p2p_peak = N_SM * MUFU_PER_CLK_SM * mhz * 1e6 / 1e9
    K = info["k_real"]
    m2l_tf = info["m2l_pairs"] * 2.0 * K * K / (phase_ms["m2l"] * 1e-3) / 1e12
    # tensor-core M2L: 3 fp16 MMAs per product (hi*hi, hi*lo, lo*hi) on K padded to 32 and Kout to 16
    kp, kn = -(-K // 32) * 32, -(-K // 16) * 16
    m2l_exec_tf = 3 * info["m2l_pairs"] * 2.0 * kp * kn / (phase_ms["m2l"] * 1e-3) / 1e12
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    f16_peak = bf16 * FP16_PER_BF16
    dominant = "p2p" if phase_ms["p2p"] >= phase_ms["m2l"] else "m2l"
    if dominant == "p2p":
        roof = {"kernel": "k_p2p<float>", "bound": "alu", "achieved": p2p_gps, "peak": p2p_peak,
                "unit": "Gpair/s", "frac": p2p_gps / p2p_peak, "traffic": None,
                "peak_source": f"derived: {N_SM} SMs x {MUFU_PER_CLK_SM} MUFU rsqrt/clk x {mhz:.0f} MHz "
                               f"({src} sm_max_mhz)"}
    else:
        roof = {"kernel": "k_m2l_umma (tcgen05 kind::f16, fp16 hi/lo split)", "bound": "tensor",
                "achieved": m2l_tf, "peak": f16_peak, "unit": "TFLOP/s", "frac": m2l_tf / f16_peak,
                "traffic": _traffic("m2l") if (wl.n == 1_000_000 and wl.p == 12) else None,
                "achieved_executed": m2l_exec_tf, "frac_executed": m2l_exec_tf / f16_peak,
                "peak_source": f"{src} bf16 burst {bf16:.1f} TFLOP/s (dense fp16 runs at the bf16 rate)",
                "note": "achieved counts the algorithmic 2 K^2 flops per V pair (K = %d); executed counts "
                        "the 3 split MMAs on the padded %d x %d operator" % (K, kn, kp)}
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "c": wl.c, "p": wl.p, "leaf": wl.leaf,
                   "l2": "flushed between steps (512 MiB write, untimed)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 4 * wl.n, "d2h_bytes_per_step": 4 * wl.n},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "dense_gpu_ms": dense_ms,
        "speedup_vs_dense_gpu": (dense_ms / ms) if dense_ms else None,
        "plan_ms": plan_ms,
        "autotune": tune,
        "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms),
        "phase_ms": phase_ms,
        "p2p_gpair_s": p2p_gps, "m2l_tflop_s": m2l_tf,
        "errors": err,
        "tree": {k: info[k] for k in ("n_boxes", "n_leaves", "max_level", "k_real", "n_u", "n_v", "n_w",
                                      "n_x", "p2p_pairs", "m2l_pairs")},
        "per_p": {str(k): v for k, v in per_p.items()},
        "fast_f64_ms": f64_ms,
        "cg": extras.get("cg"),
        "cg_one_level": extras.get("cg_one_level"),
        "cg_two_level": extras.get("cg_two_level"),
        "cg_uniform_100k": extras.get("cg_uniform_100k"),
        "table1_halton": extras.get("table1"),
        "grad_200k": extras.get("grad"),
        "grad_wellcond_200k": extras.get("grad_wellcond_200k"),
        "batched_256": extras.get("batched_256"),
    }
    print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
