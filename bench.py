#!/usr/bin/env python
"""Benchmark: factor + solve of a FEM stiffness system on one B300.

Default workload: 2D heterogeneous diffusion on 512 x 512 cubic (Q3) Lagrange
elements (2,362,369 dofs), k_e = 10^U(-2,2) per element, manufactured load,
elimination tree by recursive bisection to single elements.  One step =
factor (all Foata classes) + solve refined in FP64 to a normwise backward
error <= 1e-12.  The headline path factors in FP32 fronts (precision
``--precision``, default f32); the plain FP64 GPU path is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own replica (the workload has no
exchange step); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fem_inputs as F  # noqa: E402

METRIC = "factor+solve ms and TFLOP/s vs plain FP64 GPU path at rel. residual <=1e-12"
TOL = 1e-12


def _batched_sizes():
    return F.batched_poisson_sizes()


# name: (problems builder, meshes-only builder (for flop counts), kind, default precision, description)
#   kind "solve":   step = factor + FP64-refined solve of every right-hand side
#   kind "adjoint": step = factor + solve + adjoint solve (lambda = A^-T (x - u_target)) + element gradient
WORKLOADS = {
    "diffusion2d_q3_512": (lambda: [F.diffusion_2d(512, 3, seed=F.SEED_BASE + 2)],
                           lambda: [F.structured_mesh((512, 512), 3)], "solve", "f32",
                           "2D heterogeneous diffusion, 512x512 Q3, k=10^U(-2,2), 2,362,369 dofs"),
    "diffusion2d_q3_128": (lambda: [F.diffusion_2d(128, 3, seed=F.SEED_BASE + 2)],
                           lambda: [F.structured_mesh((128, 128), 3)], "solve", "f32",
                           "2D heterogeneous diffusion, 128x128 Q3, k=10^U(-2,2), 148,225 dofs"),
    "batched_q1_256meshes": (lambda: F.batched_poisson(_batched_sizes(), nrhs=4),
                             lambda: [F.structured_mesh((int(n), int(n)), 1) for n in _batched_sizes()], "solve",
                             "f32", "256 independent 2D Q1 Poisson meshes, n ~ U{32..256} (seeded), 4 RHS each, "
                                    "one batched analysis"),
    "diffusion3d_q1_64": (lambda: [F.diffusion_3d_q1(64, seed=F.SEED_BASE + 4)],
                          lambda: [F.structured_mesh((64, 64, 64), 1)], "solve", "f32",
                          "3D diffusion, 64^3 Q1, k=10^U(-1,1), 274,625 dofs"),
    "diffusion3d_q1_32": (lambda: [F.diffusion_3d_q1(32, seed=F.SEED_BASE + 4)],
                          lambda: [F.structured_mesh((32, 32, 32), 1)], "solve", "f32",
                          "3D diffusion, 32^3 Q1, k=10^U(-1,1), 35,937 dofs (small case of the 64^3 recipe)"),
    "adjoint2d_q1_1024": (lambda: [F.adjoint_problem(1024)], lambda: [F.structured_mesh((1024, 1024), 1)],
                          "adjoint", "f32",
                          "adjoint: 2D Q1 diffusion 1024x1024, theta = log k ~ N(0,1), J = 1/2|u - u_target|^2, "
                          "factor + refined solve + refined adjoint solve (FP64 refinement to eta <= 1e-12) "
                          "+ dJ/dtheta"),
    "poisson2d_q1_16": (lambda: [F.poisson_2d_q1(16)], lambda: [F.structured_mesh((16, 16), 1)], "solve", "f64",
                        "2D Poisson, 16x16 Q1, 289 dofs"),
}
# the paper's own model problem (Sec. 2.1): L2 projection (mass matrix, no boundary condition) for
# p = 1, 2, 3 at about 3e5 dofs, the largest size the paper measures (Sec. 4)
for _p, _n in F.L2_SIZES.items():
    WORKLOADS[f"l2proj_q{_p}_{_n}"] = (
        (lambda p=_p, n=_n: [F.l2_projection(n, p)]), (lambda p=_p, n=_n: [F.structured_mesh((n, n), p)]),
        "solve", "f32", f"L2 projection (mass matrix) of a smooth field, {_n}x{_n} Q{_p}, "
                        f"{(_p * _n + 1) ** 2:,} dofs")
# CPU oracle arm per workload: (sample name, builder or None = the full workload itself).  One
# oracle step of each full 2D workload takes roughly 10-40 s on the host cores, so those are timed
# as they are; the 3D workload (about 1e12 flops, mostly in a handful of dense fronts the oracle
# factors one at a time) is timed on the 32^3 case of the same recipe and scaled by flops.
CPU_SAMPLE = {
    "diffusion2d_q3_512": ("diffusion2d_q3_512", None),
    "diffusion2d_q3_128": ("diffusion2d_q3_128", None),
    "batched_q1_256meshes": ("batched_q1_256meshes", None),
    "diffusion3d_q1_64": ("diffusion3d_q1_32", lambda: [F.diffusion_3d_q1(32, seed=F.SEED_BASE + 4)]),
    "diffusion3d_q1_32": ("diffusion3d_q1_32", None),
    "adjoint2d_q1_1024": ("adjoint2d_q1_1024", None),
    "poisson2d_q1_16": ("poisson2d_q1_16", None),
}
for _p, _n in F.L2_SIZES.items():
    CPU_SAMPLE[f"l2proj_q{_p}_{_n}"] = (f"l2proj_q{_p}_{_n}", None)
# warm-up steps of the oracle arm run on this small case of the default recipe (the oracle keeps no
# state between steps; the warm-up only starts the thread pool and pages the code in)
CPU_WARMUP = ("diffusion2d_q3_32", lambda: [F.diffusion_2d(32, 3, seed=F.SEED_BASE + 2)])
REF_TIME_BUDGET_S = 150.0  # the oracle arm stops starting new timed steps after this much time
FP32_SIMT_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock
# DRAM bytes (read + write) over algorithmic bytes of a kernel kind, measured with ncu on three launches of a
# small case of the same recipe (128^2 Q3 for the SIMT and pivot-block kernels, 32^3 Q1 for the tensor-core
# ones; dram__bytes_read.sum + dram__bytes_write.sum against the launches' algorithmic bytes from
# `bench.py --trace-once`).  The roofline's `traffic` is this ratio times the algorithmic bytes per launch of
# the timed workload, i.e. the capture scaled by the units a launch processes.  Valid while the kernel is
# unchanged.
MEASURED_TRAFFIC_RATIO = {"gemm": 0.748, "panel_diag": 0.615, "fused_grp": 0.658, "gemm_tc": 1.202, "tc_pack": 0.308}
FP64_DFMA_TFLOPS = 1.201  # measured DFMA throughput of this B300 (register-resident FMA loop, all SMs)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "src": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_arm_step(probs, kind):
    """One oracle pass over the bounded sample (factor + refined solve, or factor + solve + adjoint
    solve + element gradient); returns (seconds, flops, threads, info)."""
    import oracle as O
    nt = O.max_threads()
    dt, fl, steps, ndof = 0.0, 0.0, 0, 0
    for pr in probs:
        pm = pr.mesh
        s = O.OracleSolver(pm.n_nodes, pm.elem_nodes, O.tree_bisection(pm.nel))
        t0 = time.perf_counter()
        s.factor(F.to_colmajor(pr.Ke), nthreads=nt)
        if kind == "adjoint":
            x = s.solve(pr.b[:, 0])
            lam = s.solve(x - pr.extra["u_target"], adjoint=True)
            O.element_grad(pm.elem_nodes, F.to_colmajor(pr.extra["dK"]), lam, x)
            it = 1  # two substitutions
        else:
            x, it = s.solve_refined(pr.b, maxit=10)
        dt += time.perf_counter() - t0
        fl += s.flops + 2.0 * s.nnz_lu * (it + 1) * pr.nrhs
        steps = max(steps, it)
        ndof += pm.n_nodes
    return dt, fl, nt, {"refine_steps": steps, "n_dof": ndof}


def cpu_model():
    """CPU model name of the host (lscpu / /proc/cpuinfo), for the baseline's description."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_arm_problems(name, probs_full=None):
    """(sample name, problems, same_config): the problems one oracle step runs for workload `name`."""
    sname, sb = CPU_SAMPLE[name]
    if sb is None:
        return sname, (probs_full if probs_full is not None else WORKLOADS[name][0]()), True
    return sname, sb(), False


def full_flops(name, nrhs_of_problem):
    """Algorithmic factor flops and nnz(L+U) of the full workload (oracle's symbolic count)."""
    import oracle as O
    ff, fnnz = 0.0, 0.0
    for pm in WORKLOADS[name][1]():
        s = O.OracleSolver(pm.n_nodes, pm.elem_nodes, O.tree_bisection(pm.nel))
        ff += float(s.flops)
        fnnz += float(s.nnz_lu) * nrhs_of_problem
    return ff, fnnz


def run_reference(args, rank):
    """The oracle arm: the FP64 CPU oracle as it stands, on the host cores.  Warm-up steps run on a
    small case of the same recipe; timed steps run the full workload (the 3D one: its 32^3 case,
    scaled by flops) until `--steps` are done or REF_TIME_BUDGET_S has passed, at least one."""
    if rank != 0:
        return
    name = args.workload
    kind = WORKLOADS[name][2]
    wprobs = CPU_WARMUP[1]()
    for _ in range(args.warmup):
        oracle_arm_step(wprobs, "solve")
    del wprobs
    sname, probs, same = cpu_arm_problems(name)
    times, fls = [], []
    t_start = time.perf_counter()
    while len(times) < args.steps and (not times or time.perf_counter() - t_start < REF_TIME_BUDGET_S):
        dt, fl, nt, info = oracle_arm_step(probs, kind)
        times.append(dt)
        fls.append(fl)
    sample_ms = float(np.mean(times)) * 1e3
    tflops = float(np.mean(fls)) / (sample_ms * 1e-3) / 1e12
    if same:
        ms = sample_ms
        how = "timed on the full workload"
    else:
        ff, fnnz = full_flops(name, probs[0].nrhs)
        full = ff + 2.0 * fnnz * (info["refine_steps"] + 1)
        ms = sample_ms * full / float(np.mean(fls))
        how = (f"timed on {sname} (same recipe, {info['n_dof']} dofs: {sample_ms / 1e3:.1f} s per step) and "
               f"scaled to the full workload by algorithmic flops (a full step is ~{ms / 6e4:.0f} min)")
    what = "factor+solve+adjoint solve+gradient" if kind == "adjoint" else "factor+refined solve"
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus, "steps": len(times),
            "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": name, "desc": WORKLOADS[name][4], "cpu_sample": sname, "same_config": same,
                       "warmup_case": CPU_WARMUP[0]},
            "tflops": tflops, "timed_region_s": float(np.sum(times)),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": nt, "kind": "oracle", "cpu": cpu_model(),
                             "same_config": same,
                             "sample": f"oracle {what} per step, {how}; {len(times)} step(s) timed "
                                       f"(warm-up: {args.warmup} steps of {CPU_WARMUP[0]})"},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def path_roofline(trace, steps, fp64, peaks, info, elem_bytes, nsolve, nrhs, ms_step):
    """Whole-step roofline: every launch record of the traced steps costs at least the slower of its
    algorithmic flops at the peak of its arithmetic (tensor cores for the 3xTF32 products, FP64 DFMA or
    FP32 FFMA otherwise) and its algorithmic bytes at the measured HBM rate; T_roof is their sum per
    step and frac = T_roof / measured step time.  Beside it the step's must-move bytes B_min (element
    matrices once per residual and for the factorization, factors written once and read once per
    solve, the solution vectors) and B_sched = B_min + the contribution blocks written and read once
    (the class-per-launch round trip)."""
    bw = peaks["hbm_gbs"] * 1e9
    p_tc = peaks["bf16_tflops"] / 2 / 3 * 1e12
    p_alu = (FP64_DFMA_TFLOPS if fp64 else FP32_SIMT_PEAK_TFLOPS) * 1e12
    t = 0.0
    for rec in trace:
        p = p_tc if rec["kind"] in ("gemm_tc", "gemm_tcd") else p_alu
        t += max(rec["flops"] / p, rec["bytes"] / bw)
    t_roof_ms = 1e3 * t / max(steps, 1)
    s_f = 8.0 if fp64 else 4.0
    n = float(info["n_dof"]) * nrhs
    b_min = (elem_bytes * (1.0 + nsolve) + s_f * info["nnz_lu"] * (1.0 + nsolve)
             + 8.0 * n * (2.0 + 4.0 * nsolve))
    b_sched = b_min + 2.0 * s_f * info["sum_cb"]
    return {"t_roof_ms": t_roof_ms, "t_measured_ms": ms_step, "frac": t_roof_ms / ms_step if ms_step > 0 else None,
            "b_min_GB": b_min / 1e9, "b_sched_GB": b_sched / 1e9, "t_hbm_floor_ms": 1e3 * b_min / bw,
            "peaks": {"hbm_GBps": peaks["hbm_gbs"], "tensor_3xtf32_TFLOPs": p_tc / 1e12, "alu_TFLOPs": p_alu / 1e12,
                      "src": peaks["src"]}}


def max_over_ranks(value, dist=None, device="cpu"):
    """The slowest rank's time: every rank solves its own replica, the job ends with the last."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rank_info():
    """(world, rank, local rank) of this process, from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def plan_summary(o, tinfo):
    d = o.as_dict()
    keep = {k: d[k] for k in ("precision", "small_front_max", "subtree_levels", "subtree_solve_levels", "tc_min_cb",
                              "super_panel", "fused_threads", "symmetric")}
    keep["tuned"] = None if tinfo is None else {"from_cache": bool(tinfo["from_cache"]),
                                                  "ms_best": tinfo["ms_best"], "ms_default": tinfo["ms_default"],
                                                  "candidates": tinfo["candidates"]}
    return keep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diffusion2d_q3_512", choices=list(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["f32", "tf32", "f64"],
                    help="front arithmetic; default: the workload's (FP32 fronts + FP64 refinement, or FP64)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="direct launches instead of CUDA-graph replay")
    ap.add_argument("--stationary", action="store_true",
                    help="stationary FP64 refinement instead of preconditioned conjugate gradients (the default for "
                         "these symmetric positive definite workloads)")
    ap.add_argument("--refine-trial", action="store_true",
                    help="also measure the tuned plan with the other refinement method (stationary vs. CG)")
    ap.add_argument("--trace-once", action="store_true",
                    help="one untimed factorization with the launch trace on, printed one JSON record per launch "
                         "(kind, class, tasks, algorithmic bytes and flops) in issue order, for matching ncu "
                         "captures to their algorithmic work; no timed steps")
    ap.add_argument("--general", action="store_true",
                    help="factor as a general matrix (LU with both triangles) instead of using its symmetry; every "
                         "workload here is symmetric positive definite")
    ap.add_argument("--bf16-trial", action="store_true",
                    help="also measure the tuned plan with BF16 Schur products on the largest fronts (MF_TF32_BF16, "
                         "one and three BF16 passes): refinement contraction, corrections and step time")
    ap.add_argument("--root-f64-trial", type=int, default=0,
                    help="also measure the tuned plan with the pivot blocks of the top N classes in FP64")
    ap.add_argument("--tcpack-trial", action="store_true",
                    help="also measure the tuned plan with the other 3xTF32 operand path (separate pack pass vs. a "
                         "tensor-core kernel that splits its own operands)")
    ap.add_argument("--panel-trial", action="store_true",
                    help="also measure the tuned plan with the other panel method of the large-front partial LU "
                         "(triangular solves vs. products with explicit pivot-block inverses)")
    ap.add_argument("--sym-trial", action="store_true",
                    help="also measure the tuned plan in symmetric mode (L only beyond the pivot blocks, lower-half "
                         "Schur updates, x = L^-T D L^-1 b)")
    ap.add_argument("--foata-trial", type=int, default=0,
                    help="also measure the tuned plan with the bottom N classes on the scalar-task Foata executor "
                         "(and, for comparison, the tuned plan without subtree fusion)")
    ap.add_argument("--tune", default="cache", choices=["off", "cache", "run"],
                    help="plan autotuner (untimed, before warm-up): off = default plan; cache = tuned plan from "
                         "the package's plan cache, tuning and recording it when missing; run = tune afresh")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local = replica_rank_info()

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_2306_08994_b300 as M
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    builder, _, kind, prec_default, desc = WORKLOADS[args.workload]
    precision = args.precision or prec_default
    probs = builder()
    nrhs = probs[0].nrhs
    Kcm = np.concatenate([F.to_colmajor(p.Ke) for p in probs]) if len(probs) > 1 else F.to_colmajor(probs[0].Ke)
    vals = torch.tensor(Kcm, device="cuda")
    bh = np.concatenate([p.b for p in probs], axis=0)  # (N, nrhs)
    b = torch.tensor(np.ascontiguousarray(bh.T), device="cuda")
    b = b.reshape(-1) if nrhs == 1 else b
    x = torch.empty_like(b)
    meshes = [M.Mesh(p.mesh.elem_nodes, p.mesh.n_nodes, p.mesh.dim, grid_dims=p.mesh.nel) for p in probs]
    use_graph = 0 if args.no_graph else 1
    sym = 0 if args.general else 1
    cg = 0 if (args.general or args.stationary) else 1
    an = M.Analysis(meshes if len(meshes) > 1 else meshes[0],
                    M.default_options(precision=precision, max_nrhs=max(4, nrhs), use_graph=use_graph, symmetric=sym,
                                      refine_cg=cg))
    info = an.info
    # a non-default stream: CUDA graphs cannot capture the legacy default stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if kind == "adjoint":
        dKcm = F.to_colmajor(probs[0].extra["dK"])
        dK = torch.tensor(dKcm, device="cuda")
        ut = torch.tensor(probs[0].extra["u_target"], device="cuda")
        lam = torch.empty_like(b)
        gvec = torch.empty_like(b)  # right-hand side of the adjoint solve, x - u_target
        grad = torch.empty(info["n_elem"], dtype=torch.float64, device="cuda")

    from paper_2306_08994_b300 import autotune as AT
    b1 = b.reshape(nrhs, -1)[0].contiguous()

    def plan_for(analysis):
        if args.tune == "off":
            return analysis.options, None
        return AT.tune(analysis, vals, b1, cache_path=AT.DEFAULT_CACHE if args.tune == "cache" else None,
                       stream=stream)

    opts, tinfo = plan_for(an)
    fac = M.Factors(an, opts)
    if args.trace_once:
        # launches are issued directly (no graph replay) while the trace is on, so the records come
        # in the order the GPU receives the kernels; within a record, one kernel per plan entry
        fac.profile(True)
        fac.profile_read()
        fac.factor(vals)
        if rank == 0:
            for i, rec in enumerate(fac.trace()):
                print(json.dumps(dict(rec, index=i)), flush=True)
        fac.profile_read()
        fac.profile(False)
        return

    def step(f, v, bb, xx, kv=None, kut=None, tol=TOL, maxit=60):
        f.factor(v)
        if kind == "adjoint":
            # forward solve, adjoint solve with the loss gradient x - u_target, dJ/dtheta_e; FP64 fronts
            # solve once each, FP32-family fronts refine both solves in FP64 to the same tolerance
            if f.precision == "f64":
                xx.copy_(bb)
                f.solve(xx)
                torch.sub(xx, ut if kut is None else kut, out=lam)
                f.solve(lam, adjoint=True)
                f.element_grad(dK if kv is None else kv, lam, xx, grad)
                return {"iterations": 0, "backward_error": None, "rel_residual": None}
            r1 = f.refine_solve(v, bb, xx, tol=tol, maxit=maxit)
            torch.sub(xx, ut if kut is None else kut, out=gvec)
            r2 = f.refine_solve(v, gvec, lam, tol=tol, maxit=maxit, adjoint=True)
            f.element_grad(dK if kv is None else kv, lam, xx, grad)
            return {"iterations": r1["iterations"] + r2["iterations"],
                    "backward_error": max(r1["backward_error"], r2["backward_error"]),
                    "rel_residual": max(r1["rel_residual"], r2["rel_residual"])}
        return f.refine_solve(v, bb, xx, tol=tol, maxit=maxit)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        r = step(fac, vals, b, x)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    fac.profile_read()  # reset launch/work accounting
    iters = []
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for i in range(args.steps):
            r = step(fac, vals, b, x)
            iters.append(r["iterations"])
            ev[i + 1].record(stream)
        barrier()
    acct = fac.profile_read()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms = float(np.sum(per)) / args.steps
    ms = max_over_ranks(ms, dist, "cuda")
    st = fac.status()
    launches = int(sum(v["launches"] for v in acct.values()))
    nsolve = (2.0 if kind == "adjoint" else 1.0) + float(np.mean(iters))
    flops = info["factor_flops"] + info["solve_flops"] * nsolve * nrhs
    if kind == "adjoint" and fac.precision == "f64":
        # backward error of the plain FP64 solve: mf_refine_solve with no correction step
        chk = fac.refine_solve(vals, b, torch.empty_like(b), tol=TOL, maxit=0)
        r = {"iterations": 0, "backward_error": chk["backward_error"], "rel_residual": chk["rel_residual"]}
    eta = r["backward_error"]

    # plain FP64 GPU path, same metric
    fp64 = None
    if precision != "f64" and args.fp64_steps > 0:
        an64 = M.Analysis(meshes if len(meshes) > 1 else meshes[0],
                          M.default_options(precision="f64", max_nrhs=max(4, nrhs), use_graph=use_graph,
                                            symmetric=sym, refine_cg=cg))
        opts64, tinfo64 = plan_for(an64)
        f64 = M.Factors(an64, opts64)
        x64 = torch.empty_like(b)
        step(f64, vals, b, x64)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            r64 = step(f64, vals, b, x64)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        nsolve64 = r64["iterations"] + 1
        fp64 = {"ms": ms64, "tflops": (info["factor_flops"] + info["solve_flops"] * nsolve64 * nrhs) / ms64 / 1e9,
                "plan": plan_summary(opts64, tinfo64),
                "backward_error": r64["backward_error"], "rel_residual": r64["rel_residual"],
                "refine_iterations": r64["iterations"],
                "rel_diff_vs_headline": float(torch.linalg.norm(x64 - x) / torch.linalg.norm(x64))}
        x64_keep = x64.clone()
        del f64, an64, x64
        torch.cuda.empty_cache()

    # the refined path timed to the FP64 path's own accuracy: the FP64 path's backward error (within a
    # factor 2), reached with the fewest corrections that reach it (or, if refinement stalls above it,
    # with the corrections that give the smallest backward error)
    matched = None
    if fp64 is not None and kind == "solve" and fp64["backward_error"]:
        target = 2.0 * fp64["backward_error"]
        etas = []
        for c in range(16):
            pr_ = fac.refine_solve(vals, b, x, tol=0.0, maxit=c, check=False)
            etas.append(pr_["backward_error"])
            if etas[-1] <= target:
                break
        reach = [c for c, e in enumerate(etas) if e <= target]
        c_m = reach[0] if reach else int(np.argmin(etas))
        tol_m = target if reach else 0.0
        step(fac, vals, b, x, tol=tol_m, maxit=c_m)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            rm = step(fac, vals, b, x, tol=tol_m, maxit=c_m)
        e1.record(stream)
        barrier()
        ms_m = e0.elapsed_time(e1) / args.steps
        matched = {"ms": ms_m, "target_backward_error": target, "reached": bool(reach),
                   "backward_error": rm["backward_error"], "rel_residual": rm["rel_residual"],
                   "refine_iterations": rm["iterations"], "speedup_vs_fp64": fp64["ms"] / ms_m,
                   "rel_diff_vs_fp64": float(torch.linalg.norm(x64_keep - x) / torch.linalg.norm(x64_keep)),
                   "what": "refined path timed to the FP64 GPU path's own normwise backward error (x2)"}
        del x64_keep
        step(fac, vals, b, x)  # leave x as the headline's solution

    def contraction_probe(f, maxc=12):
        """Backward error after c = 0, 1, ... corrections (each probe restarts the refinement), and
        the median ratio of consecutive values while they fall (the refinement's contraction)."""
        etas = []
        for c in range(maxc + 1):
            pr_ = f.refine_solve(vals, b, x, tol=0.0, maxit=c, check=False)
            etas.append(pr_["backward_error"])
            if etas[-1] <= 1e-16 or not np.isfinite(etas[-1]):
                break
        ratios = [etas[i + 1] / etas[i] for i in range(len(etas) - 1) if etas[i] > 4e-16 and etas[i + 1] > 0]
        return etas, (float(np.median(ratios)) if ratios else None)

    def time_variant(opts_v):
        """Factor time and factor + refined solve (eta <= 1e-12) time of a plan variant, K steps each."""
        fv = M.Factors(an, opts_v)
        fv.factor(vals)
        etas, rho = contraction_probe(fv)
        conv = min(etas) <= TOL
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            fv.factor(vals)
        e1.record(stream)
        rv = None
        if conv:
            for _ in range(args.steps):
                rv = step(fv, vals, b, x)
        e2.record(stream)
        barrier()
        out = {"factor_ms": e0.elapsed_time(e1) / args.steps, "etas": etas, "contraction": rho, "converges": conv,
               "step_ms": e1.elapsed_time(e2) / args.steps if conv else None,
               "refine_iterations": rv["iterations"] if rv else None, "status": fv.status()["rc"]}
        del fv
        torch.cuda.empty_cache()
        return out

    trials = {}
    if kind == "solve" and (args.bf16_trial or args.root_f64_trial or args.foata_trial or args.sym_trial or
                            args.refine_trial or args.panel_trial or args.tcpack_trial):
        import copy
        trials["tuned"] = time_variant(opts)
        if args.bf16_trial:
            for passes in (1, 3):
                o2 = copy.copy(opts)
                o2.precision = M.MF_TF32_BF16
                o2.bf16_passes = passes
                if o2.tc_min_cb == 0:
                    o2.tc_min_cb = 256
                trials[f"bf16_{passes}pass"] = time_variant(o2)
        if args.root_f64_trial:
            o2 = copy.copy(opts)
            o2.root_f64 = args.root_f64_trial
            trials[f"root_f64_{args.root_f64_trial}"] = time_variant(o2)
        if args.tcpack_trial:
            o2 = copy.copy(opts)
            o2.tc_direct = 1 - opts.tc_direct
            trials["tc_direct" if o2.tc_direct else "tc_pack"] = time_variant(o2)
        if args.panel_trial:
            o2 = copy.copy(opts)
            o2.panel_trsm = 1 - opts.panel_trsm
            trials["panel_trsm" if o2.panel_trsm else "panel_inverse"] = time_variant(o2)
        if args.refine_trial and opts.symmetric:
            o2 = copy.copy(opts)
            o2.refine_cg = 1 - opts.refine_cg
            trials["refine_cg" if o2.refine_cg else "refine_stationary"] = time_variant(o2)
        if args.sym_trial:
            o2 = copy.copy(opts)
            o2.symmetric = 1 - opts.symmetric
            trials["symmetric" if o2.symmetric else "general"] = time_variant(o2)
        if args.foata_trial:
            o2 = copy.copy(opts)
            o2.subtree_levels = -1
            trials["tuned_no_subtree"] = time_variant(o2)
            o2.foata_classes = args.foata_trial
            trials[f"foata_{args.foata_trial}"] = time_variant(o2)
        step(fac, vals, b, x)

    # roofline: per-launch event timing (launch trace) over the same K steps; the dominant
    # kernel is the trace kind with the most device time
    fac.profile(True)
    fac.profile_read()
    for _ in range(args.steps):
        step(fac, vals, b, x)
    trace = fac.trace()
    prof = fac.profile_read()
    fac.profile(False)
    peaks = load_peaks()
    kinds = {}
    for rec in trace:
        kd = kinds.setdefault(rec["kind"], {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0})
        kd["ms"] += rec["ms"]
        kd["launches"] += 1
        kd["bytes"] += rec["bytes"]
        kd["flops"] += rec["flops"]
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    bound = {"gemm": "alu", "panel_diag": "alu", "inv_diag": "alu", "panel_trsm": "alu", "gemm_tc": "tensor",
             "gemm_tcd": "tensor"}.get(dom, "hbm")
    if bound == "alu":
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "unit": "TFLOP/s",
                "peak": FP32_SIMT_PEAK_TFLOPS if precision != "f64" else FP64_DFMA_TFLOPS,
                "peak_src": ("derived: 148 SM x 128 FP32 lanes x 2 x 2032 MHz" if precision != "f64" else
                             "measured: DFMA loop on this B300 (1.201 TFLOP/s)")}
    elif bound == "tensor":
        # three TF32 products per FP32-accurate product: the FP32-accurate peak is a third of TF32's
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "unit": "TFLOP/s",
                "peak": peaks["bf16_tflops"] / 2 / 3,
                "peak_src": f"{peaks['src']} bf16 GEMM x 1/2 (TF32 nominal ratio) x 1/3 (three TF32 products)"}
    else:
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_src": peaks["src"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM traffic per launch of the dominant kernel: the small-case capture's traffic / algorithmic ratio
    # scaled to this workload's launches; null for kernels not captured
    ratio = MEASURED_TRAFFIC_RATIO.get(dom)
    roof["traffic"] = None if ratio is None else ratio * d["bytes"] / max(d["launches"], 1)
    roof["traffic_src"] = (None if ratio is None else
                           f"ncu dram bytes / algorithmic bytes = {ratio} on three launches of a small case of the "
                           f"same recipe, times this workload's algorithmic bytes per launch")
    roof["kernel"] = dom
    roof["launches_per_step"] = d["launches"] / args.steps
    roof["per_launch_ms"] = per_launch_ms
    path_roof = path_roofline(trace, args.steps, precision == "f64", peaks, info, float(Kcm.nbytes), nsolve, nrhs, ms)
    families = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                    "GBps": v["bytes"] / max(v["ms"], 1e-9) / 1e6, "TFLOPps": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                for k, v in prof.items() if v["launches"]}
    kernels = {k: {"ms_per_step": v["ms"] / args.steps, "records_per_step": v["launches"] / args.steps,
                   "GBps": v["bytes"] / max(v["ms"], 1e-9) / 1e6, "TFLOPps": v["flops"] / max(v["ms"], 1e-9) / 1e9}
               for k, v in sorted(kinds.items(), key=lambda t: -t[1]["ms"])}

    # end to end through the public API with host buffers: inputs H2D, result D2H every step
    hv = torch.from_numpy(Kcm).pin_memory()
    hb = b.cpu().pin_memory()
    dv = torch.empty_like(vals)
    db = torch.empty_like(b)
    dx = torch.empty_like(b)
    h2d = Kcm.nbytes + b.numel() * 8
    if kind == "adjoint":
        hk = torch.from_numpy(dKcm).pin_memory()
        hu = ut.cpu().pin_memory()
        dk = torch.empty_like(dK)
        du = torch.empty_like(ut)
        hx = torch.empty(grad.shape, dtype=grad.dtype).pin_memory()
        h2d += dKcm.nbytes + ut.numel() * 8
    else:
        hx = torch.empty_like(hb).pin_memory()

    def e2e_step():
        dv.copy_(hv, non_blocking=True)
        db.copy_(hb, non_blocking=True)
        if kind == "adjoint":
            dk.copy_(hk, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            step(fac, dv, db, dx, dk, du)
            hx.copy_(grad, non_blocking=True)
        else:
            step(fac, dv, db, dx)
            hx.copy_(dx, non_blocking=True)

    e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sname, cprobs, same = cpu_arm_problems(args.workload, probs)
        dt, fl, nt, cinfo = oracle_arm_step(cprobs, kind)
        what = "factor+solve+adjoint solve+gradient" if kind == "adjoint" else "factor+refined solve"
        if same:
            val = dt * 1e3
            how = f"one oracle {what} of the full workload ({cinfo['n_dof']} dofs), measured"
        else:
            ff, fnnz = full_flops(args.workload, nrhs)
            full = ff + 2.0 * fnnz * (cinfo["refine_steps"] + 1)
            val = dt * 1e3 * full / fl
            how = (f"one oracle {what} of {sname} (same recipe, {cinfo['n_dof']} dofs) took {dt:.2f} s; "
                   f"scaled to the full workload by algorithmic flops")
        cpu = {"value": val, "unit": "ms", "cores": nt, "kind": "oracle", "cpu": cpu_model(), "same_config": same,
               "sample": how}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if precision == "f64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "n_dof": info["n_dof"], "n_front": info["n_front"],
                       "classes": info["n_classes"], "max_front": info["max_m"], "nrhs": nrhs,
                       "meshes": info["n_meshes"], "precision": precision,
                       "refine": (f"FP64 residual, tol {TOL} normwise backward error" if kind == "solve" else
                                  "none (FP64 path; backward error of the plain solve reported)"),
                       "l2": "inputs larger than L2 (element matrices %.0f MB)" % (Kcm.nbytes / 1e6),
                       "parallelism": "replicas" if world > 1 else "single",
                       "launch": "CUDA graph replay" if use_graph else "direct launches",
                       "plan": plan_summary(opts, tinfo)},
            "tflops": flops / ms / 1e9,
            "backward_error": eta, "rel_residual": r["rel_residual"], "refine_iterations": float(np.mean(iters)),
            "pivots_perturbed": st["n_perturbed"],
            "fp64_path": fp64,
            "speedup_vs_fp64": (fp64["ms"] / ms) if fp64 else None,
            "matched_accuracy": matched,
            "trials": trials or None,
            "refinement": ("preconditioned conjugate gradients in FP64 (M^-1 = L^-T D L^-1 from the FP32 factors)"
                           if opts.refine_cg and opts.symmetric else "stationary FP64 refinement"),
            "accuracy_note": ("value: refined path stopped at normwise backward error <= 1e-12; matched_accuracy: "
                              "the same path stopped at the FP64 path's own backward error; rel_residual = "
                              "||b - A x||_2 / ||b||_2 of the final iterate on both paths"),
            "roofline": roof, "path_roofline": path_roof,
            "families": families,
            "kernels": kernels,
            "gpu_launches": launches,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(hx.numel() * 8)},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
