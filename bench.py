#!/usr/bin/env python
"""Benchmark of the Benchmark Streaming hot path on GB300.

One step = the seven BS operations of Table 1 at the largest configuration
of the streaming sweep: copy, AXPY, norm, inner product and the fused CG
update on FP64 vectors of 2^28 entries (2 GiB each, far larger than L2), then
scatter and gather on the degree-7, 48^3 structured hex mesh with permuted
elements (110592 elements, 56.6M local and 38.3M global nodes).  `value` is
the algorithmic bytes of the step (what each operation must move: copy 16n, AXPY 24n,
norm 8n, dot 16n, CG update 48n, scatter 12 N_L + 8 N_G, gather
12 N_L + 12 N_G + 4) divided by the device time, i.e. the effective HBM GB/s
of the whole step.  Per-operation GB/s and fractions of the measured HBM peak
are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the path has no exchange step at these sizes, so N > 1 runs N
independent replicas (weak scaling); value sums the bytes of all ranks over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "per-op HBM GB/s (% of GB300 peak); time-to-1e-8 CG solve, plain vs batched/learned"
OPS = ["copy", "axpy", "norm", "dot", "cg_update", "scatter", "gather"]
KERNEL_OF = {"copy": "k_copy", "axpy": "k_axpy", "norm": "k_dot", "dot": "k_dot",
             "cg_update": "k_cg_update", "scatter": "k_scatter2", "gather": "k_gather"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=28, help="vector length 2^k for BS1-BS5")
    ap.add_argument("--mesh", default="7,48", help="N,K of the BS6/BS7 mesh")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cg", action="store_true", help="skip the CG time-to-tolerance runs")
    ap.add_argument("--workload", default="stream",
                    choices=["stream", "cg", "batched", "learned"],
                    help="stream: the BS step (default); cg: only the CG solves on --cg-mesh; "
                         "batched: 256 uneven solves, batched vs one at a time; "
                         "learned: learned-preconditioner FPCG vs Jacobi-PCG and plain CG")
    ap.add_argument("--learned-mesh", default="5,64", help="N,K of the learned workload")
    ap.add_argument("--no-plain", action="store_true",
                    help="learned workload: skip the (long) unpreconditioned CG solve")
    ap.add_argument("--no-learned", action="store_true",
                    help="default run: skip the compact learned-preconditioner section")
    ap.add_argument("--no-batched", action="store_true",
                    help="default run: skip the compact batched section")
    ap.add_argument("--nsolves", type=int, default=256, help="solves in the batched workload")
    ap.add_argument("--cg-mesh", default="7,48", help="N,K of the CG time-to-tolerance mesh")
    ap.add_argument("--no-cg-small", action="store_true", help="skip the N=3, 8^3 CG runs")
    return ap.parse_args()


def alg_bytes(n, NL, NG):
    return {"copy": 16 * n, "axpy": 24 * n, "norm": 8 * n, "dot": 16 * n, "cg_update": 48 * n,
            "scatter": 4 * NL + 8 * NG + 8 * NL, "gather": 8 * NL + 4 * NL + 4 * (NG + 1) + 8 * NG}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def config(args, n, N, K, NL, NG):
    return {"workload": f"BS1-BS5 FP64 n=2^{args.log2n}; BS6/BS7 N={N} on {K}^3 hex mesh "
                        f"(N_L={NL}, N_G={NG}), permuted elements",
            "n": n, "degree": N, "mesh_K": K, "N_L": NL, "N_G": NG, "alpha": 0.5, "beta": 1.0,
            "l2": "inputs larger than L2 (2 GiB vectors); no flush needed",
            "parallelism": f"replicas x{args.gpus}"}


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- multi-rank

def max_over_ranks(ms, world, device="cuda"):
    """The slowest rank's time: an all-reduce MAX over the job (identity for
    one rank).  device: where the scalar lives for the backend (cuda for
    NCCL, cpu for gloo)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_step, steps, world, ms):
    """Whole-job GB/s: every rank moves bytes_per_step per step (replicas),
    over the slowest rank's time."""
    return world * bytes_per_step * steps / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------- inputs

def make_inputs(args):
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor

    from paper_2009_10917_gb300 import synth
    n = 1 << args.log2n
    N, K = (int(v) for v in args.mesh.split(","))
    with ThreadPoolExecutor(8) as ex:
        fut = {name: ex.submit(synth.uniform, n, 1, s)
               for s, name in enumerate(["x", "p", "Ap", "xc", "r"])}
        mesh = synth.Mesh(K, N, seed=1)
        fut["qG"] = ex.submit(synth.uniform, mesh.NG, 2, 0)
        host = {k: f.result() for k, f in fut.items()}
    return n, mesh, host


# ---------------------------------------------------------------- ours

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2009_10917_gb300 import bs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    n, mesh, host = make_inputs(args)
    NL, NG = mesh.NL, mesh.NG
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    Z = bs.Map(mesh.E, mesh.N, NG, mesh.ids)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    qL = torch.empty(NL, dtype=torch.float64, device="cuda")
    qG2 = torch.empty(NG, dtype=torch.float64, device="cuda")
    red = torch.zeros(4, dtype=torch.float64, device="cuda")
    ws = bs.workspace()
    stream = torch.cuda.current_stream()

    def step(d, ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        bs.copy(d["x"], y)
        mark(1)
        bs.axpy(0.5, d["x"], 1.0, y)
        mark(2)
        bs.norm(d["x"], red[0:2], ws)
        mark(3)
        bs.dot(d["x"], y, red[2:3], ws)
        mark(4)
        bs.cg_update(0.5, d["p"], d["Ap"], d["xc"], d["r"], red[3:4], ws)
        mark(5)
        Z.scatter(d["qG"], qL)
        mark(6)
        Z.gather(qL, qG2)
        mark(7)

    for _ in range(args.warmup):
        step(dev)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(args.steps)]
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0e.record(stream)
        for k in range(args.steps):
            step(dev, evs[k])
        t1e.record(stream)
        torch.cuda.synchronize()
        barrier()
    total_ms = t0e.elapsed_time(t1e)
    per_op_ms = {op: sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps
                 for i, op in enumerate(OPS)}
    total_ms = max_over_ranks(total_ms, world)
    B = alg_bytes(n, NL, NG)
    step_bytes = sum(B.values())
    value = job_throughput(step_bytes, args.steps, world, total_ms)
    peak, peak_kind = peaks()
    per_op = {op: {"gbs": round(B[op] / (per_op_ms[op] * 1e-3) / 1e9, 1),
                   "ms": round(per_op_ms[op], 4),
                   "frac": round(B[op] / (per_op_ms[op] * 1e-3) / 1e9 / peak, 4),
                   "frac_of_8000": round(B[op] / (per_op_ms[op] * 1e-3) / 1e9 / 8000.0, 4)}
              for op in OPS}
    dom = max(OPS, key=lambda op: per_op_ms[op])
    achieved = B[dom] / (per_op_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": KERNEL_OF[dom], "op": dom,
                "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic_for(KERNEL_OF[dom], dom)}

    # end to end: pinned host inputs copied in and results read back every step
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        out_h = torch.empty(4, dtype=torch.float64).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())

        def e2e_step():
            for k_, v in pinned.items():
                dev[k_].copy_(v, non_blocking=True)
            step(dev)
            out_h.copy_(red, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ksteps = max(3, args.steps // 4)
        a.record(stream)
        for _ in range(ksteps):
            e2e_step()
        b_.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(a.elapsed_time(b_), world)
        e2e = {"value": round(job_throughput(step_bytes, ksteps, world, ems), 1), "unit": "GB/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 32, "steps": ksteps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args)
    cg = learned = batched = None
    if not (args.no_cg and args.no_learned and args.no_batched):
        del dev, y, qL, qG2
        torch.cuda.empty_cache()
    if not args.no_cg:
        cg = cg_section(args)
        torch.cuda.empty_cache()
    if not args.no_learned and rank == 0:
        learned = learned_section(args, compact=True)
        torch.cuda.empty_cache()
    if not args.no_batched and rank == 0:
        batched = batched_section(args, compact=True)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config(args, n, mesh.N, mesh.K, NL, NG),
                "per_op": per_op, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 7 * args.steps, "clocks": clk.summary(), "cg": cg,
                "learned": learned, "batched": batched}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def operator_times(P, p, reps=20):
    """Device time of one A p (ms, CUDA events over reps calls after three
    warm-up calls) in each operator mode: the FP64 element kernel in the
    even-odd form (the default) and direct, each unfused (element kernel,
    gather of every row) and fused (single-copy nodes written by the element
    kernel, gather of the shared rows); the float-float kernel (always
    direct) unfused and fused."""
    import torch

    from paper_2009_10917_gb300 import bs
    out = {}
    Ap = torch.empty_like(p)
    prev = bs.operator_mode(-1)
    cases = [("fp64_evenodd", 0, P.apply_A), ("fp64_direct", bs.BS_OP_DIRECT, P.apply_A),
             ("fp64_evenodd_fused", bs.BS_OP_FUSED, P.apply_A),
             ("fp64_direct_fused", bs.BS_OP_FUSED | bs.BS_OP_DIRECT, P.apply_A),
             ("ff", 0, P.apply_A_ff), ("ff_fused", bs.BS_OP_FUSED, P.apply_A_ff)]
    try:
        for name, mode, fn in cases:
            bs.operator_mode(mode)
            for _ in range(3):
                fn(p, Ap)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                fn(p, Ap)
            e1.record()
            torch.cuda.synchronize()
            out[name] = round(e0.elapsed_time(e1) / reps, 4)
    finally:
        bs.operator_mode(prev)
    return out


def geo_section(Z, m, b, N, K, delta=0.2):
    """The same solve on general hexahedra: every interior vertex of the mesh
    moved by up to delta h (seeded), the operator built from the
    non-affine geometric factors (bs_problem_create_geo).  FP64 CG to 1e-8,
    with the FP64 and with the float-float element kernel, each after a
    16-iteration warm-up, the true residual with the FP64 operator, and the
    device time of one A p (both kernels) against the affine even-odd one."""
    import time

    import torch

    from paper_2009_10917_gb300 import bs, synth
    t0 = time.perf_counter()
    mg = synth.Mesh(K, N, seed=1, perturb=delta)
    Pg = bs.Problem(Z, mg.h, 1.0, verts=mg.verts())
    setup = time.perf_counter() - t0
    out = {"perturb": delta, "setup_seconds": round(setup, 3)}
    for name, fl in (("fp64_cg", 0), ("fp64_cg_ff_operator", bs.BS_CG_FF_OPERATOR)):
        Pg.cg(b, tol=1e-8, maxit=16, flags=bs.BS_CG_GRAPH | bs.BS_CG_FIXED_ITERS | fl)
        x, info = Pg.cg(b, tol=1e-8, maxit=100000, flags=bs.BS_CG_GRAPH | fl)
        r = Pg.apply_A(x)
        bs.axpy(1.0, b, -1.0, r)
        out[name] = {"seconds": round(info["seconds"], 4), "iterations": info["iterations"],
                     "rel_residual_true_fp64": torch.linalg.norm(r).item() /
                     torch.linalg.norm(b).item()}
    out["speedup_ff_vs_fp64_cg"] = round(out["fp64_cg"]["seconds"] /
                                         out["fp64_cg_ff_operator"]["seconds"], 3)
    Ap = torch.empty_like(b)
    Pa = bs.Problem(Z, m.h, 1.0)
    for name, fn in (("geo", Pg.apply_A), ("geo_ff", Pg.apply_A_ff),
                     ("affine_evenodd", Pa.apply_A)):
        for _ in range(3):
            fn(b, Ap)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            fn(b, Ap)
        e1.record()
        torch.cuda.synchronize()
        out.setdefault("operator_ms", {})[name] = round(e0.elapsed_time(e1) / 10, 4)
    # FP64 operations per local node of the element kernel: gradient and its
    # transpose 6 (N+1) multiply-adds, flux 9, mass and coefficient 3
    flops = 2 * (6 * (N + 1) + 12) * m.NL
    out["geo_fp64_gflops_per_apply"] = round(flops / (out["operator_ms"]["geo"] * 1e-3) / 1e9, 1)
    del Pg, Pa, x, r, Ap
    return out


def cg_section(args):
    """Time to tolerance of Algorithm 1 on the GLL Helmholtz operator
    (lambda = 1, b uniform[-1, 1)): plain FP64 CG to 1e-8, the same with the
    float-float element operator, FP32-storage CG inside FP64 iterative
    refinement to 1e-8 (FP64 true residual), and the FP64 and float-float
    solves with the vectors in scattered storage (Sec. 3), each after one
    untimed warm-up solve; plus the small configuration's 50 fixed FP64
    iterations and the algorithmic bytes per iteration of both storages.  Wall
    time measured by the library around each solve (host clock, stream
    synchronised); every result's true residual is recomputed with the FP64
    operator."""
    import torch

    from paper_2009_10917_gb300 import bs, synth
    out = {}
    N, K = (int(v) for v in args.cg_mesh.split(","))
    cases = [] if args.no_cg_small else [("small_N3_K8", (3, 8))]
    for label, (n_, k_) in cases + [(f"N{N}_K{K}", (N, K))]:
        m = synth.Mesh(k_, n_, seed=1)
        Z = bs.Map(m.E, n_, m.NG, m.ids)
        P = bs.Problem(Z, m.h, 1.0)
        b = torch.from_numpy(synth.uniform(m.NG, 1, stream=7)).cuda()
        res = {"N_G": m.NG, "N_L": m.NL}
        if label.startswith("small"):
            P.cg(b, tol=0.0, maxit=50, flags=bs.BS_CG_FIXED_ITERS | bs.BS_CG_GRAPH)
            _, i50 = P.cg(b, tol=0.0, maxit=50, flags=bs.BS_CG_FIXED_ITERS | bs.BS_CG_GRAPH)
            res["fp64_50_iterations_s"] = i50["seconds"]
        runs = [("fp64_cg", lambda: P.cg(b, tol=1e-8, maxit=100000, flags=bs.BS_CG_GRAPH)),
                ("fp64_cg_ff_operator",
                 lambda: P.cg(b, tol=1e-8, maxit=100000,
                              flags=bs.BS_CG_GRAPH | bs.BS_CG_FF_OPERATOR)),
                ("fp32_ir_1e-8", lambda: P.cg_refined_f32(b, tol=1e-8, flags=bs.BS_CG_GRAPH)),
                ("fp64_cg_scattered",
                 lambda: P.cg(b, tol=1e-8, maxit=100000,
                              flags=bs.BS_CG_GRAPH | bs.BS_CG_SCATTERED)),
                ("fp64_cg_ff_operator_scattered",
                 lambda: P.cg(b, tol=1e-8, maxit=100000,
                              flags=bs.BS_CG_GRAPH | bs.BS_CG_FF_OPERATOR | bs.BS_CG_SCATTERED))]
        bn = torch.linalg.norm(b).item()
        for name, fn in runs:
            fn()
            x, info = fn()
            r = P.apply_A(x)  # FP64 operator
            bs.axpy(1.0, b, -1.0, r)
            res[name] = {"seconds": round(info["seconds"], 4), "iterations": info["iterations"],
                         "outer": info["outer"], "rel_residual": info["rel_residual"],
                         "rel_residual_true_fp64": torch.linalg.norm(r).item() / bn}
            del x, r
        if not label.startswith("small"):
            # the same FF solve with the fused operator (single-copy nodes written
            # by the element kernel, gather of the shared rows)
            prev = bs.operator_fusion(1)
            try:
                runs[1][1]()
                x, info = runs[1][1]()
            finally:
                bs.operator_fusion(prev)
            res["fp64_cg_ff_operator_fused"] = {"seconds": round(info["seconds"], 4),
                                                "iterations": info["iterations"]}
            res["speedup_fused_vs_unfused_ff_cg"] = round(
                res["fp64_cg_ff_operator"]["seconds"] / info["seconds"], 3)
            res["operator_ms"] = operator_times(P, b)
            del x
            res["perturbed_hexahedra"] = geo_section(Z, m, b, n_, k_)
        for k in ("fp64_cg_ff_operator", "fp32_ir_1e-8"):
            res[f"speedup_{k}_vs_fp64_at_1e-8"] = round(
                res["fp64_cg"]["seconds"] / res[k]["seconds"], 3)
        # scattered (N_L) against global (N_G) storage of the CG vectors
        res["bytes_per_iteration"] = {"global": 24 * m.NL + 100 * m.NG,
                                      "scattered": 122 * m.NL + 20 * m.NG}
        for k, g in (("fp64_cg_scattered", "fp64_cg"),
                     ("fp64_cg_ff_operator_scattered", "fp64_cg_ff_operator")):
            res[f"time_ratio_{k}_vs_global"] = round(res[k]["seconds"] / res[g]["seconds"], 3)
        out[label] = res
        del P, Z, b
        torch.cuda.empty_cache()
    return out


def batched_section(args, compact=False):
    """The batched configuration: nsolves independent solves, degree N uniform
    in {2..8}, K uniform in {4..24} (seed 7), lambda = 1, b uniform[-1, 1),
    tol 1e-8.  Runs the autotuner for each form (FP64, FP64 with the
    float-float operator, FP32-refined), then times the batched solver with
    the default and the tuned configuration (CUDA graph), and the same solves
    one at a time; every run after a short untimed warm-up."""
    import time

    import torch

    from paper_2009_10917_gb300 import bs, synth
    specs = synth.batched_specs(args.nsolves, 7)
    probs, bs_ = [], []
    keep = []
    for i, (N, K) in enumerate(specs):
        m = synth.Mesh(K, N, seed=1000 + i)
        Z = bs.Map(m.E, N, m.NG, m.ids)
        P = bs.Problem(Z, m.h, 1.0)
        keep.append(Z)
        probs.append(P)
        bs_.append(torch.from_numpy(synth.uniform(m.NG, 1000 + i, stream=3)).cuda())
    xs = [torch.zeros_like(b) for b in bs_]
    out = {"nsolves": len(specs), "sum_N_G": int(sum((k * n + 1) ** 3 for n, k in specs))}

    def timed(fn):
        fn(16)  # warm-up: kernels paged in, graphs built
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn(1000000)
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    FF, F32 = bs.BS_CG_FF_OPERATOR, bs.BS_CG_REFINED_F32
    tuned = {}
    forms = (("fp64_ff_operator", FF), ("fp32_ir", F32)) if compact else (
        ("fp64", 0), ("fp64_ff_operator", FF), ("fp32_ir", F32))
    for name, fl in forms:
        t0 = time.perf_counter()
        cfg, ms = bs.autotune_batched(probs, bs_, flags=fl, iters=4)
        tuned[name] = cfg
        out[f"autotune_{name}"] = {"config": cfg.as_dict(), "ms_per_iteration": round(ms, 3),
                                   "tuning_seconds": round(time.perf_counter() - t0, 2)}
    runs = [("batched_fp64_ff_operator_tuned", FF, tuned["fp64_ff_operator"]),
            ("batched_fp32_ir_tuned", F32, tuned["fp32_ir"])]
    if not compact:
        runs = [("batched_fp64", 0, None), ("batched_fp64_tuned", 0, tuned["fp64"])] + runs + [
            ("batched_fp32_ir", F32, None)]
    for name, fl, cfg in runs:
        dt, (rc, infos) = timed(lambda it: bs.solve_batched(
            probs, bs_, xs, tol=1e-8, maxit=it, flags=bs.BS_CG_GRAPH | fl, check=False,
            config=cfg))
        out[name] = {"seconds": round(dt, 3), "rc": rc,
                     "max_rel_residual": max(i["rel_residual"] for i in infos),
                     "iterations_sum": sum(i["iterations"] for i in infos)}

    def one_by_one(refined, ff, maxit):
        worst = 0.0
        for P, b in zip(probs, bs_):
            if refined:
                _, info = P.cg_refined_f32(b, tol=1e-8, maxit=maxit, flags=bs.BS_CG_GRAPH,
                                           check=False)
            else:
                _, info = P.cg(b, tol=1e-8, maxit=min(maxit, 100000),
                               flags=bs.BS_CG_GRAPH | (FF if ff else 0), check=False)
            worst = max(worst, info["rel_residual"])
        return worst

    seq = (("sequential_fp64", False, False),) if compact else (
        ("sequential_fp64", False, False), ("sequential_fp64_ff_operator", False, True),
        ("sequential_fp32_ir", True, False))
    for name, refined, ff in seq:
        dt, worst = timed(lambda it: one_by_one(refined, ff, it))
        out[name] = {"seconds": round(dt, 3), "max_rel_residual": worst}
    best = min(("batched_fp64_ff_operator_tuned", "batched_fp32_ir_tuned"),
               key=lambda k: out[k]["seconds"])
    out["fastest_batched"] = best
    out["speedup_fastest_batched_vs_sequential_fp64"] = round(
        out["sequential_fp64"]["seconds"] / out[best]["seconds"], 3)
    return out


def learned_section(args, compact=False):
    """The learned-preconditioner configuration: degree N=5 on a 64^3 mesh
    (E = 262144, N_G = 321^3), lambda = 1e-2, per-element coefficient
    lognormal(sigma = 1), b uniform[-1, 1), tol 1e-8.  Times plain FP64 CG,
    Jacobi-PCG and flexible PCG with the network trained on the GPU (20000
    pairs from Jacobi-PCG residuals, 40000 Adam steps), each solve after one
    untimed warm-up solve; the one-off pair and training times are reported
    beside them.  Residuals are the FP64 true residuals ||b - A x|| / ||b||."""
    import torch

    from paper_2009_10917_gb300 import bs, learned, synth
    N, K = (int(v) for v in args.learned_mesh.split(","))
    lam = 1e-2
    m = synth.Mesh(K, N, seed=1)
    coef = synth.lognormal(m.E, 2)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef)
    b = torch.from_numpy(synth.uniform(m.NG, 4242)).cuda()
    bn = torch.linalg.norm(b).item()

    def true_rel(x):
        r = P.apply_A(x)
        bs.axpy(1.0, b, -1.0, r)
        return torch.linalg.norm(r).item() / bn

    def timed(fn):
        fn(60)  # warm-up: a short solve builds the graph and pages the kernels in
        torch.cuda.synchronize()
        t = time.perf_counter()
        x, info = fn(200000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        return {"seconds": round(dt, 3), "iterations": info["iterations"],
                "ms_per_iteration": round(1000 * dt / max(1, info["iterations"]), 4),
                "rel_residual_true": true_rel(x), "rc": info["rc"],
                "jacobi_switch_at": info.get("outer", 0), "fallbacks": info.get("fallbacks", 0)}

    out = {"mesh": f"N={N} {K}^3", "E": m.E, "N_G": m.NG, "lambda": lam,
           "coef": "lognormal(sigma=1) per element", "tol": 1e-8}
    if not args.no_plain and not compact:
        out["plain_fp64_cg"] = timed(lambda it: P.cg(b, tol=1e-8, maxit=it,
                                                     flags=bs.BS_CG_GRAPH, check=False))
    out["jacobi_pcg"] = timed(lambda it: P.cg(b, tol=1e-8, maxit=it,
                                              flags=bs.BS_CG_GRAPH | bs.BS_CG_JACOBI, check=False))
    FF = bs.BS_CG_FF_OPERATOR
    out["jacobi_pcg_ff_operator"] = timed(lambda it: P.cg(
        b, tol=1e-8, maxit=it, flags=bs.BS_CG_GRAPH | bs.BS_CG_JACOBI | FF, check=False))
    net, meta = learned.build_preconditioner(P, m.E, m.NG, npairs=20000, steps=40000)
    out["training"] = meta
    res = timed(lambda it: bs.fpcg_learned(P, net, b, tol=1e-8, maxit=it,
                                           flags=bs.BS_CG_GRAPH | bs.BS_FPCG_ODD, check=False))
    out["learned_fpcg_odd"] = res
    out["learned_fpcg_odd_ff_operator"] = timed(lambda it: bs.fpcg_learned(
        P, net, b, tol=1e-8, maxit=it, flags=bs.BS_CG_GRAPH | bs.BS_FPCG_ODD | FF, check=False))
    if not compact:
        out["learned_fpcg_full_network"] = timed(lambda it: bs.fpcg_learned(
            P, net, b, tol=1e-8, maxit=it, flags=bs.BS_CG_GRAPH, check=False))
    for k in [k for k in ("plain_fp64_cg", "jacobi_pcg") if k in out]:
        out[f"speedup_learned_vs_{k}"] = round(out[k]["seconds"] / res["seconds"], 3)
        out[f"iteration_ratio_{k}_over_learned"] = round(
            out[k]["iterations"] / max(1, res["iterations"]), 3)
    out["speedup_learned_vs_jacobi_pcg_both_ff_operator"] = round(
        out["jacobi_pcg_ff_operator"]["seconds"] / out["learned_fpcg_odd_ff_operator"]["seconds"], 3)
    if "plain_fp64_cg" in out:
        out["speedup_learned_ff_vs_plain_fp64_cg"] = round(
            out["plain_fp64_cg"]["seconds"] / out["learned_fpcg_odd_ff_operator"]["seconds"], 3)
    return out


def run_cg_only(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    print(json.dumps({"metric": "time-to-1e-8 CG solve, plain vs FP32-refined", "unit": "s",
                      "higher_is_better": False, "cg": cg_section(args)}), flush=True)


def traffic_for(kernel, op):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source has not changed since it was taken; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d["ops"][op]
        from paper_2009_10917_gb300 import build
        if ent.get("source_sha") != build.source_digest(build.OP_SOURCES[op]):
            return None
        return ent["dram_bytes_per_launch_full"]
    except Exception:
        return None


# ---------------------------------------------------------------- oracle on the host

def oracle_sample(seconds=10.0):
    """Time the oracle on a bounded sample of the same workload: BS1-BS5 at
    n = 2^22, BS6/BS7 on the degree-7, 16^3 mesh.  Returns (GB/s, detail)."""
    import oracle
    from paper_2009_10917_gb300 import synth
    n = 1 << 22
    x, p, Ap, xc, r = (synth.uniform(n, 1, s) for s in range(5))
    mesh = synth.Mesh(16, 7, seed=1)
    qG = synth.uniform(mesh.NG, 2)
    B = alg_bytes(n, mesh.NL, mesh.NG)
    oracle.lib()
    reps, t = 0, 0.0
    while t < seconds or reps < 1:
        t0 = time.perf_counter()
        y = oracle.copy(x)
        y = oracle.axpy(0.5, x, 1.0, y)
        oracle.norm(x)
        oracle.dot(x, y)
        xc, r, _ = oracle.cg_update(0.5, p, Ap, xc, r)
        qL = oracle.scatter(mesh.ids, qG, __import__("numpy").zeros(mesh.NL))
        oracle.gather(mesh.ids, qL, mesh.NG)
        t += time.perf_counter() - t0
        reps += 1
    gbs = sum(B.values()) * reps / t / 1e9
    return gbs, {"reps": reps, "seconds": round(t, 2),
                 "sample": f"BS1-BS5 at n=2^22, BS6/BS7 on N=7 16^3 mesh, {reps} passes"}


def cpu_baseline(args):
    gbs, d = oracle_sample()
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": d["sample"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 1 << args.log2n
    N, K = (int(v) for v in args.mesh.split(","))
    NL, NG = K ** 3 * (N + 1) ** 3, (K * N + 1) ** 3
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(1.0)
    vals, t_all = [], 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        gbs, d = oracle_sample(2.0)
        t_all += time.perf_counter() - t0
        vals.append(gbs)
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * t_all / max(1, args.steps), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config(args, n, N, K, NL, NG),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1,
                             "kind": "oracle", "sample": d["sample"]},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "cg":
        run_cg_only(a)
    elif a.workload == "batched":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"metric": "time-to-1e-8 CG solve, batched vs one at a time",
                          "unit": "s", "higher_is_better": False,
                          "batched": batched_section(a)}), flush=True)
    elif a.workload == "learned":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"metric": "time-to-1e-8 CG solve, learned FPCG vs Jacobi-PCG",
                          "unit": "s", "higher_is_better": False,
                          "learned": learned_section(a)}), flush=True)
    else:
        run_ours(a)
