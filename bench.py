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
KERNEL_OF = {"copy": "k_copy", "axpy": "k_axpy", "norm": "k_norm_split", "dot": "k_dot",
             "cg_update": "k_cg_update", "scatter": "k_scatter2", "gather": "k_gather_async"}


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
                    choices=["stream", "cg", "batched", "learned", "sweep", "op"],
                    help="stream: the BS step (default); cg: only the CG solves on --cg-mesh; "
                         "batched: 256 uneven solves, batched vs one at a time; "
                         "learned: learned-preconditioner FPCG vs Jacobi-PCG and plain CG; "
                         "sweep: BS1-BS7 over sizes and the T0/Wmax fit of Sec. 4")
    ap.add_argument("--sweep-per-octave", type=int, default=4,
                    help="sweep: log-spaced vector lengths per factor of two")
    ap.add_argument("--sweep-runs", type=int, default=20,
                    help="sweep: back-to-back runs per size")
    ap.add_argument("--sweep-out", default=None, help="sweep: also write the JSON here")
    ap.add_argument("--op", default="gather", choices=OPS,
                    help="op: the one operation to run --reps times (for a profiler)")
    ap.add_argument("--reps", type=int, default=3, help="op: calls of the operation")
    ap.add_argument("--learned-mesh", default="5,64", help="N,K of the learned workload")
    ap.add_argument("--no-plain", action="store_true",
                    help="learned workload: skip the (long) unpreconditioned CG solve")
    ap.add_argument("--no-learned", action="store_true",
                    help="default run: skip the compact learned-preconditioner section")
    ap.add_argument("--no-batched", action="store_true",
                    help="default run: skip the compact batched section")
    ap.add_argument("--nsolves", type=int, default=256, help="solves in the batched workload")
    ap.add_argument("--nsolves-small", type=int, default=1024,
                    help="solves in the batched workload's small-solve mix (0: skip it)")
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
            "l2": (f"inputs larger than L2 ({8 * n / 2 ** 20:.0f} MiB vectors); no flush needed"
                   if 8 * n > 256 * 2 ** 20 else
                   f"{8 * n / 2 ** 20:.1f} MiB vectors: partly L2-resident between steps"),
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

    def step(d, ev=None, wait=None):
        """One pass of BS1-BS7.  wait: events (x; p, Ap, xc, r; q_G) that the
        operations needing those inputs wait for (the end-to-end copies)."""
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        if wait is not None:
            stream.wait_event(wait[0])
        mark(0)
        bs.copy(d["x"], y)
        mark(1)
        bs.axpy(0.5, d["x"], 1.0, y)
        mark(2)
        bs.norm(d["x"], red[0:2], ws)
        mark(3)
        bs.dot(d["x"], y, red[2:3], ws)
        if wait is not None:
            stream.wait_event(wait[1])
        mark(4)
        bs.cg_update(0.5, d["p"], d["Ap"], d["xc"], d["r"], red[3:4], ws)
        if wait is not None:
            stream.wait_event(wait[2])
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

        # the copies run on a side stream in the order the step consumes them
        # (the host link moves about 210 GB/s whatever the number of streams
        # or a kernel reading the pinned buffers), and each group of
        # operations starts as soon as its inputs have arrived
        cstream = torch.cuda.Stream()
        groups = (("x",), ("p", "Ap", "xc", "r"), ("qG",))
        assert sorted(k_ for g_ in groups for k_ in g_) == sorted(pinned), "e2e copies every input"
        ready = [torch.cuda.Event() for _ in groups]

        def e2e_step():
            cstream.wait_stream(stream)  # the previous step has read these buffers
            with torch.cuda.stream(cstream):
                for names, ev in zip(groups, ready):
                    for k_ in names:
                        dev[k_].copy_(pinned[k_], non_blocking=True)
                    ev.record(cstream)
            step(dev, wait=ready)
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
        cpu = cpu_baseline(args, host, mesh)
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
                ("fp32_ir_1e-10", lambda: P.cg_refined_f32(b, tol=1e-10, flags=bs.BS_CG_GRAPH)),
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
        for k in ("fp64_cg_ff_operator", "fp32_ir_1e-8", "fp32_ir_1e-10"):
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
    out["error_vs_fp64_oracle"] = accuracy_section(args)
    return out


def accuracy_section(args, N=7, K=6):
    """Error of each GPU solve against the FP64 oracle on a mesh the oracle
    solves in seconds (degree 7 on 6^3, lambda = 1, the same b recipe): the
    reference solution is the oracle's Algorithm 1 to 1e-13; every GPU
    solution is compared with it in the 2-norm, relative, with its FP64 true
    residual beside it."""
    import numpy as np
    import torch

    import oracle
    from paper_2009_10917_gb300 import bs, synth
    m = synth.Mesh(K, N, seed=1)
    bh = synth.uniform(m.NG, 1, stream=7)
    xo, it_o, *_ = oracle.cg(m.E, N, m.h, 1.0, m.ids, m.NG, bh, tol=1e-13, maxit=100000)
    ro = bh - oracle.apply_A(m.E, N, m.h, 1.0, m.ids, m.NG, xo)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    b = torch.from_numpy(bh).cuda()
    out = {"mesh": f"N={N} {K}^3", "N_G": m.NG, "reference": "oracle FP64 CG to 1e-13",
           "reference_iterations": it_o,
           "reference_rel_residual": float(np.linalg.norm(ro) / np.linalg.norm(bh))}
    runs = [("fp64_cg_1e-8", lambda: P.cg(b, tol=1e-8, maxit=100000)),
            ("fp64_cg_ff_operator_1e-8",
             lambda: P.cg(b, tol=1e-8, maxit=100000, flags=bs.BS_CG_FF_OPERATOR)),
            ("fp32_ir_1e-8", lambda: P.cg_refined_f32(b, tol=1e-8)),
            ("fp32_ir_1e-10", lambda: P.cg_refined_f32(b, tol=1e-10))]
    xn = np.linalg.norm(xo)
    for name, fn in runs:
        x, info = fn()
        xh = x.cpu().numpy()
        r = bh - oracle.apply_A(m.E, N, m.h, 1.0, m.ids, m.NG, xh)
        out[name] = {"rel_error_vs_oracle": float(np.linalg.norm(xh - xo) / xn),
                     "rel_residual_true_fp64": float(np.linalg.norm(r) / np.linalg.norm(bh)),
                     "iterations": info["iterations"], "outer": info["outer"]}
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


def batched_small_section(args):
    """The launch-bound regime of batching: nsolves_small solves on small
    meshes (N uniform in {2..8}, K uniform in {2..5}, seed 11; 125 to 68921
    unknowns each), lambda = 1, tol 1e-8, FP64 arithmetic on both sides, so
    that the batched solver's only advantage is one cooperative launch per
    iteration for all solves instead of a graph replay per solve.  Times the
    batched solver (default and tuned configuration) against the same solves
    one at a time (CUDA graphs), after an untimed warm-up of each."""
    import time

    import torch

    from paper_2009_10917_gb300 import bs, synth
    specs = synth.batched_specs(args.nsolves_small, 11, kmin=2, kmax=5)
    probs, bs_, keep = [], [], []
    for i, (N, K) in enumerate(specs):
        m = synth.Mesh(K, N, seed=5000 + i)
        Z = bs.Map(m.E, N, m.NG, m.ids)
        keep.append(Z)
        probs.append(bs.Problem(Z, m.h, 1.0))
        bs_.append(torch.from_numpy(synth.uniform(m.NG, 5000 + i, stream=3)).cuda())
    xs = [torch.zeros_like(b) for b in bs_]
    out = {"nsolves": len(specs), "sum_N_G": int(sum((k * n + 1) ** 3 for n, k in specs)),
           "max_N_G": int(max((k * n + 1) ** 3 for n, k in specs))}

    def timed(fn):
        fn(16)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn(1000000)
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    t0 = time.perf_counter()
    cfg, ms = bs.autotune_batched(probs, bs_, flags=0, iters=8)
    out["autotune_fp64"] = {"config": cfg.as_dict(), "ms_per_iteration": round(ms, 3),
                            "tuning_seconds": round(time.perf_counter() - t0, 2)}
    for name, c in (("batched_fp64", None), ("batched_fp64_tuned", cfg)):
        dt, (rc, infos) = timed(lambda it: bs.solve_batched(
            probs, bs_, xs, tol=1e-8, maxit=it, flags=bs.BS_CG_GRAPH, check=False, config=c))
        out[name] = {"seconds": round(dt, 3), "rc": rc,
                     "max_rel_residual": max(i["rel_residual"] for i in infos),
                     "iterations_sum": sum(i["iterations"] for i in infos),
                     "iterations_max": max(i["iterations"] for i in infos)}

    def one_by_one(maxit):
        worst, its = 0.0, 0
        for P, b in zip(probs, bs_):
            _, info = P.cg(b, tol=1e-8, maxit=min(maxit, 100000), flags=bs.BS_CG_GRAPH,
                           check=False)
            worst = max(worst, info["rel_residual"])
            its += info["iterations"]
        return worst, its

    dt, (worst, its) = timed(one_by_one)
    out["sequential_fp64"] = {"seconds": round(dt, 3), "max_rel_residual": worst,
                              "iterations_sum": its}
    best = min(("batched_fp64", "batched_fp64_tuned"), key=lambda k: out[k]["seconds"])
    out["speedup_batched_fp64_vs_sequential_fp64"] = round(
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
    # the exact element-interior block Jacobi: the map the network imitates
    BJ = bs.BS_CG_BLOCK_JACOBI
    out["block_jacobi_pcg"] = timed(lambda it: P.cg(b, tol=1e-8, maxit=it,
                                                    flags=bs.BS_CG_GRAPH | BJ, check=False))
    out["block_jacobi_pcg_ff_operator"] = timed(lambda it: P.cg(
        b, tol=1e-8, maxit=it, flags=bs.BS_CG_GRAPH | BJ | FF, check=False))
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
    out["speedup_block_jacobi_vs_jacobi_pcg_both_ff_operator"] = round(
        out["jacobi_pcg_ff_operator"]["seconds"] / out["block_jacobi_pcg_ff_operator"]["seconds"], 3)
    out["iteration_ratio_learned_over_block_jacobi"] = round(
        res["iterations"] / max(1, out["block_jacobi_pcg"]["iterations"]), 3)
    if "plain_fp64_cg" in out:
        out["speedup_learned_ff_vs_plain_fp64_cg"] = round(
            out["plain_fp64_cg"]["seconds"] / out["learned_fpcg_odd_ff_operator"]["seconds"], 3)
    return out


def _sweep_time(calls, runs, flush):
    """Device time (s) per run of `runs` back-to-back calls, captured in one
    CUDA graph (launch cost on the device only) and replayed after an L2
    flush; calls(k) issues run k."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        calls(0)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in range(runs):
            calls(k)
    best = None
    for _ in range(3):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3 / runs
        best = t if best is None else min(best, t)
    del g
    return best


def sweep_section(args):
    """The streaming sweep of Sec. 6.2 on this GPU.  BS1-BS5 on FP64 vectors
    of n = 2^10 .. 2^28 entries (log-spaced, --sweep-per-octave sizes per
    factor of two, the powers of two among them), each timed as --sweep-runs
    back-to-back calls through the C ABI captured in a CUDA graph, best of
    three replays, after an L2 flush: once on the SAME buffers every run (what
    a solver does; small vectors then live in L2) and once ROTATING through
    distinct buffers (each run reads memory no earlier run touched, so every
    size comes from HBM).  Each op's (bytes, seconds) pairs are fitted by least
    squares to T(B) = T0 + B / Wmax (eq. time_model), with the Fischer-Brown
    point B_0.8 = 4 T0 Wmax.  BS6/BS7: degree N = 1..15 on K^3 meshes of about
    8e7 local nodes (K = round(cbrt(8e7) / (N + 1))), and the degree-7 K-sweep
    that Table 2's BS6/BS7 fits use."""
    import numpy as np
    import torch

    from paper_2009_10917_gb300 import bs, perfmodel, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    runs = args.sweep_runs
    peak, peak_kind = peaks()
    flush = torch.empty(256 << 20, dtype=torch.float32, device="cuda")  # 1 GiB > L2
    ppo = max(1, args.sweep_per_octave)
    ns = sorted({int(round(2.0 ** (10 + i / ppo))) for i in range(18 * ppo + 1)})
    nmax = 1 << 28
    pool_n = max(nmax, runs * (1 << 23))
    host = synth.uniform(pool_n, 1, 0)
    pools = [torch.from_numpy(host).cuda()]
    del host
    for k in range(1, 4):  # the other roles: shifted copies of the same values
        pools.append(torch.roll(pools[0], 7919 * k))
    red = torch.zeros(4, dtype=torch.float64, device="cuda")
    ws = bs.workspace()
    B_of = {"copy": 16, "axpy": 24, "norm": 8, "dot": 16, "cg_update": 48}

    def views(n, k, rotate):
        """The four role vectors of run k: distinct slices when rotating and
        the whole set still fits the pools, else the first slice."""
        off = k * n if rotate and (k + 1) * n <= pool_n else 0
        return [p[off:off + n] for p in pools]

    def op_call(op, n, rotate):
        def calls(k):
            a, b, c, d = views(n, k, rotate)
            if op == "copy":
                bs.copy(a, b)
            elif op == "axpy":
                bs.axpy(0.5, a, 1.0, b)
            elif op == "norm":
                bs.norm(a, red[0:2], ws)
            elif op == "dot":
                bs.dot(a, b, red[2:3], ws)
            else:
                bs.cg_update(1e-3, a, b, c, d, red[3:4], ws)
        return calls

    streaming = {}
    for op in ("copy", "axpy", "norm", "dot", "cg_update"):
        res = {"same_buffers": [], "rotating": []}
        for n in ns:
            for mode, rot in (("same_buffers", False), ("rotating", True)):
                t = _sweep_time(op_call(op, n, rot), runs, flush)
                res[mode].append([n, B_of[op] * n, t])
        for mode in ("same_buffers", "rotating"):
            B = np.array([r[1] for r in res[mode]], dtype=np.float64)
            T = np.array([r[2] for r in res[mode]], dtype=np.float64)
            t0, w = perfmodel.fit(B, T)
            res[mode + "_fit"] = {"T0_us": round(t0 * 1e6, 3), "Wmax_GBs": round(w / 1e9, 1),
                                  "Wmax_frac": round(w / 1e9 / peak, 4),
                                  "B08_MiB": round(perfmodel.fischer_brown(t0, w) / 2 ** 20, 2)}
            big = B >= 64 * 2 ** 20
            res[mode + "_min_frac_at_64MB_plus"] = round(float((B[big] / T[big]).min()) / 1e9 / peak, 4)
            res[mode + "_max_GBs"] = round(float((B / T).max()) / 1e9, 1)
        streaming[op] = res
    del pools
    torch.cuda.empty_cache()

    def mesh_case(N, K, rotate):
        m = synth.Mesh(K, N, seed=1)
        Z = bs.Map(m.E, N, m.NG, m.ids)
        b_sc = 12 * m.NL + 8 * m.NG
        b_ga = 12 * m.NL + 12 * m.NG + 4
        reps = 1
        if rotate:
            reps = max(1, min(runs, -(-(512 << 20) // (8 * (m.NL + m.NG)))))
        qGs = [torch.from_numpy(synth.uniform(m.NG, 2, 0)).cuda() for _ in range(1)]
        qGs += [qGs[0].clone() for _ in range(reps - 1)]
        qLs = [torch.empty(m.NL, dtype=torch.float64, device="cuda") for _ in range(reps)]
        Z.scatter(qGs[0], qLs[0])
        for q in qLs[1:]:
            q.copy_(qLs[0])
        outs = [torch.empty(m.NG, dtype=torch.float64, device="cuda") for _ in range(reps)]
        t_sc = _sweep_time(lambda k: Z.scatter(qGs[k % reps], qLs[k % reps]), runs, flush)
        t_ga = _sweep_time(lambda k: Z.gather(qLs[k % reps], outs[k % reps]), runs, flush)
        out = {"N": N, "K": K, "N_L": m.NL, "N_G": m.NG, "scatter_bytes": b_sc,
               "gather_bytes": b_ga, "scatter_s": t_sc, "gather_s": t_ga,
               "scatter_GBs": round(b_sc / t_sc / 1e9, 1), "gather_GBs": round(b_ga / t_ga / 1e9, 1),
               "scatter_frac": round(b_sc / t_sc / 1e9 / peak, 4),
               "gather_frac": round(b_ga / t_ga / 1e9 / peak, 4)}
        del Z, qGs, qLs, outs
        torch.cuda.empty_cache()
        return out

    degree = [mesh_case(N, max(1, int(round((8e7) ** (1 / 3) / (N + 1)))), False)
              for N in range(1, 16)]
    ksweep = [mesh_case(7, K, True) for K in (2, 3, 4, 6, 8, 11, 16, 22, 30, 40, 48, 54)]
    fits = {}
    for op in ("scatter", "gather"):
        B = np.array([c[op + "_bytes"] for c in ksweep], dtype=np.float64)
        T = np.array([c[op + "_s"] for c in ksweep], dtype=np.float64)
        t0, w = perfmodel.fit(B, T)
        fits[op] = {"T0_us": round(t0 * 1e6, 3), "Wmax_GBs": round(w / 1e9, 1),
                    "Wmax_frac": round(w / 1e9 / peak, 4),
                    "B08_MiB": round(perfmodel.fischer_brown(t0, w) / 2 ** 20, 2)}
    return {"peak_GBs": peak, "peak_kind": peak_kind, "runs_per_size": runs,
            "timing": "CUDA graph of back-to-back C-ABI calls, best of 3 replays, L2 flushed "
                      "before each replay",
            "sizes": len(ns), "streaming": streaming,
            "gather_scatter_by_degree_8e7_local_nodes": degree,
            "gather_scatter_N7_K_sweep": ksweep, "gather_scatter_N7_fit": fits}


def run_one_op(args):
    """One BS operation, --reps calls on the --log2n vectors or the --mesh
    mesh, nothing else: a short, fixed launch sequence for a profiler."""
    import torch

    from paper_2009_10917_gb300 import bs, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    op, n = args.op, 1 << args.log2n
    if op in ("scatter", "gather"):
        N, K = (int(v) for v in args.mesh.split(","))
        m = synth.Mesh(K, N, seed=1)
        Z = bs.Map(m.E, N, m.NG, m.ids)
        qG = torch.from_numpy(synth.uniform(m.NG, 2)).cuda()
        qL = torch.from_numpy(synth.uniform(m.NL, 3)).cuda()
        for _ in range(args.reps):
            Z.scatter(qG, qL) if op == "scatter" else Z.gather(qL, qG)
    else:
        x, y, z, w = (torch.from_numpy(synth.uniform(n, 1, s)).cuda() for s in range(4))
        for _ in range(args.reps):
            if op == "copy":
                bs.copy(x, y)
            elif op == "axpy":
                bs.axpy(0.5, x, 1.0, y)
            elif op == "norm":
                bs.norm(x)
            elif op == "dot":
                bs.dot(x, y)
            else:
                bs.cg_update(1e-3, x, y, z, w)
    torch.cuda.synchronize()
    print(json.dumps({"op": op, "reps": args.reps, "done": True}), flush=True)


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

def oracle_ops(host, mesh, omp=None):
    """The seven operations of the step as oracle calls on the host inputs
    at the benchmark's own sizes, in the step's order: [(op, call, bytes)].
    omp: an oracle.Omp (the plain loops over all host cores) instead of the
    single-threaded oracle."""
    import numpy as np

    import oracle
    n = host["x"].size
    B = alg_bytes(n, mesh.NL, mesh.NG)
    st = {"y": np.empty(n), "qL": np.zeros(mesh.NL), "qG2": np.empty(mesh.NG)}
    xc, r = host["xc"].copy(), host["r"].copy()
    if omp is None:
        calls = {
            "copy": lambda: st.__setitem__("y", oracle.copy(host["x"])),
            "axpy": lambda: st.__setitem__("y", oracle.axpy(0.5, host["x"], 1.0, st["y"])),
            "norm": lambda: oracle.norm(host["x"]),
            "dot": lambda: oracle.dot(host["x"], st["y"]),
            "cg_update": lambda: oracle.cg_update(0.5, host["p"], host["Ap"], xc, r),
            "scatter": lambda: st.__setitem__("qL", oracle.scatter(mesh.ids, host["qG"], st["qL"])),
            "gather": lambda: oracle.gather(mesh.ids, st["qL"], mesh.NG)}
    else:
        rs, ci = oracle.csr(mesh.ids, mesh.NG)  # set-up of the CSR gather, not timed
        calls = {
            "copy": lambda: omp.copy(host["x"], st["y"]),
            "axpy": lambda: omp.axpy(0.5, host["x"], 1.0, st["y"]),
            "norm": lambda: omp.norm(host["x"]),
            "dot": lambda: omp.dot(host["x"], st["y"]),
            "cg_update": lambda: omp.cg_update(0.5, host["p"], host["Ap"], xc, r),
            "scatter": lambda: omp.scatter(mesh.ids, host["qG"], st["qL"]),
            "gather": lambda: omp.gather(rs, ci, st["qL"], st["qG2"])}
    return [(op, calls[op], B[op]) for op in OPS]


def time_oracle_pass(ops):
    """One pass over the ops: (GB/s, seconds, per-op seconds)."""
    per, tot, byt = {}, 0.0, 0
    for op, call, b in ops:
        t0 = time.perf_counter()
        call()
        per[op] = time.perf_counter() - t0
        tot += per[op]
        byt += b
    return byt / tot / 1e9, tot, per


def cpu_baseline(args, host, mesh):
    """The oracle on the host cores at the benchmark's own sizes (one full
    pass of the step, inputs already in memory): single-threaded as it
    stands, and the OpenMP build of its plain loops on every core."""
    import oracle
    oracle.lib()
    gbs, secs, per = time_oracle_pass(oracle_ops(host, mesh))
    sample = (f"one pass of BS1-BS7 at the benchmark's sizes (n=2^{args.log2n}; N={mesh.N} "
              f"on {mesh.K}^3), inputs in host memory")
    out = {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": sample, "seconds": round(secs, 2),
           "per_op_seconds": {k: round(v, 3) for k, v in per.items()}}
    try:
        om = oracle.Omp()
        time_oracle_pass(oracle_ops(host, mesh, om))  # first touch of the work arrays
        g2, s2, per2 = time_oracle_pass(oracle_ops(host, mesh, om))
        out["omp"] = {"value": round(g2, 3), "unit": "GB/s", "cores": om.threads,
                      "nproc": os.cpu_count(), "kind": "oracle loops, OpenMP",
                      "sample": sample, "seconds": round(s2, 2),
                      "per_op_seconds": {k: round(v, 3) for k, v in per2.items()}}
    except Exception as exc:  # no OpenMP runtime on this host
        out["omp"] = {"unavailable": str(exc)[:200]}
    return out


def run_reference(args):
    """The reference arm: the oracle (the paper's definitions as written),
    single-threaded on the host, at the benchmark's own sizes.  Each step is
    one operation of the step at full size, in the step's order, so K steps
    cover K/7 passes; value = algorithmic bytes of the timed steps over their
    time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.lib()
    n, mesh, host = make_inputs(args)
    ops = oracle_ops(host, mesh)
    for k in range(args.warmup):
        ops[k % len(ops)][1]()
    t_all, byt = 0.0, 0
    for k in range(args.steps):
        op, call, b = ops[(args.warmup + k) % len(ops)]
        t0 = time.perf_counter()
        call()
        t_all += time.perf_counter() - t0
        byt += b
    value = byt / max(t_all, 1e-12) / 1e9
    sample = (f"{args.steps} steps, one operation of the step each, at the benchmark's "
              f"sizes (n=2^{args.log2n}; N={mesh.N} on {mesh.K}^3)")
    line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * t_all / max(1, args.steps), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config(args, n, mesh.N, mesh.K, mesh.NL, mesh.NG),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "cg":
        run_cg_only(a)
    elif a.workload == "op":
        run_one_op(a)
    elif a.workload == "sweep":
        res = sweep_section(a)
        line = {"metric": "per-op HBM GB/s over sizes; T0/Wmax fit (Sec. 4, Table 2)",
                "unit": "GB/s", "higher_is_better": True, "sweep": res}
        if a.sweep_out:
            with open(a.sweep_out, "w") as f:
                json.dump(line, f, indent=1)
        print(json.dumps(line), flush=True)
    elif a.workload == "batched":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        res = {"metric": "time-to-1e-8 CG solve, batched vs one at a time",
               "unit": "s", "higher_is_better": False, "batched": batched_section(a)}
        if a.nsolves_small > 0:
            res["batched_small"] = batched_small_section(a)
        print(json.dumps(res), flush=True)
    elif a.workload == "learned":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"metric": "time-to-1e-8 CG solve, learned FPCG vs Jacobi-PCG",
                          "unit": "s", "higher_is_better": False,
                          "learned": learned_section(a)}), flush=True)
    else:
        run_ours(a)
