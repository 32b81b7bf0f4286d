"""Benchmark of the stochastic conservative field transfer on one GB300.

A step is one pass of the whole path on one synthetic workload: build the
source location grid and the target mass matrix, compute the control values,
run the fused Monte Carlo assembly, solve M u = b in FP64 and evaluate the
conservation error, i.e. sft_source_create + sft_target_create +
sft_transfer + sft_conservation_error (+ destroy), with the meshes already
resident in device memory when the timed region starts.

Default workload ("tri4m"): 3,998,792-triangle jittered source mesh with the
Gaussian + jump field in FP32, 2,000,000-triangle Delaunay target, N = 64
samples per element, FP32 sampling with compensated partials, FP64 CG to 1e-10.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torchrun; every rank runs an independent replica of the
workload (the single transfer is not sharded), and rank 0 reports the sum of
the ranks' queries over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "source queries/s and transfer ms at fixed L2 + conservation error, vs roofline"
WORKLOADS = {
    "tri4m": "2D: 3,998,792-triangle jittered source (f = exp(-|x-c|^2/0.01) + 0.5 sign(x-0.5), FP32 "
             "coords) -> 2,000,000-triangle Delaunay target, N = 64, FP32 sampling + compensated partials, "
             "FP64 load vector and CG to 1e-10",
    "tet5m": "3D: 4,983,504-tet jittered Kuhn source (8 Gaussians + jump at z = 0.4, FP32) -> 2,958,234-tet "
             "target, N = 32, FP32 sampling + compensated partials, FP64 CG to 1e-10",
    "sur3d": "surrogate source: the tri4m source field (3,998,792 triangles, Gaussian + jump, FP32) extruded "
             "along z, learned by the 3-256-256-256-256-1 SiLU network (BF16 weights/activations, FP32 "
             "accumulation) from 2,000,000 seeded exact queries, transferred onto the tet5m target "
             "(2,958,234 tets) with N = 64; per-element exact fallback on the first 4 samples at "
             "tau = 1e-2 max|f|; FP64 load vector and CG to 1e-10",
    "tri4m_online": "online transfers of the tri4m meshes (initialization once: node and sample locations "
                    "recorded; each step new source values, control from the recorded node locations, assembly "
                    "gathering at the recorded sample locations, FP64 CG to 1e-10)",
    "tet5m_online": "online transfers of the tet5m meshes (as tri4m_online, 3D, N = 32)",
    "batch256": "256 batched requests, 2D/3D 50/50, 1e4..5e5 target elements (log-uniform, seeded), 1..8 fields, "
                "N in {8,16,32,64,128}; 2D sources: 2,048- and 3,998,792-triangle meshes, 3D source: "
                "4,983,504 tets, 8 fields each; one graph-replayed plan per step (control, persistent "
                "assembly, one batched solve to 1e-10: FP64 residuals, FP32 CG on the scaled matrices)",
    "roundtrip": "round trips (the paper's iterative analysis): f2 on a 2,000,000-triangle Delaunay mesh "
                 "(1,002,001 nodes) -> 199,712-triangle jittered mesh -> back, N = 20, FP32 sampling, FP64 "
                 "values and CG to 1e-10; two plans built once, a step is one round trip (two online "
                 "transfers, each leg's solution the next leg's source values)",
}
# algorithmic HBM bytes of the assembly kernel (minimum a black-box P1 query
# and a target element must move): per query cell range 8 B + one candidate
# id 4 B + the containing element record (2D 36 B, 3D 64 B); per target
# element conn + coords + g + b read-modify-write (2D 72 B, 3D 112 B)
BYTES_PER_QUERY = {2: 48, 3: 76}
BYTES_PER_ELEM = {2: 72, 3: 112}
# the same minimum with FP64 records, values, coordinates and control values
# (the all-FP64 path): per query 8 + 4 + 2 x (2D 36, 3D 64); per element
# conn 4k + coords 8kd + g 8k + b read-modify-write 16k
BYTES_PER_QUERY_FP64 = {2: 84, 3: 140}
BYTES_PER_ELEM_FP64 = {2: 132, 3: 208}
KERNEL_FILES = ["paper_2603_00538_gb300/csrc/assemble.cu", "paper_2603_00538_gb300/csrc/common.cuh",
                "paper_2603_00538_gb300/csrc/accum.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "assemble_traffic.txt")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes per launch of the assembly kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    for line in open(TRAFFIC_FILE):
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if parts.get("workload") == workload and parts.get("kernel_hash") == kernel_hash():
            try:
                return float(parts["dram_bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 100 ms) while the timed region runs. The
    sampler process is started, and its first sample awaited, before the
    region begins, so that nvidia-smi's own start-up does not land inside a
    timed step; the summary uses the samples taken inside the region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._proc = None
        self.t0 = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            deadline = time.time() + 5.0
            while not self.rows and time.time() < deadline and self._proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self._proc = None
        self.t0 = time.time()
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append([time.time()] + parts)

    def __exit__(self, *a):
        if self._proc:
            time.sleep(0.25)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        inside = [r[1:] for r in self.rows if self.t0 is not None and r[0] >= self.t0]
        rows = inside or [r[1:] for r in self.rows]   # a region shorter than one sample period
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    return rank, world, local


def aggregate(total_ms: float, units: float, world: int, dev=None):
    """Whole-job timing over ranks (every rank calls it): the slowest rank's
    elapsed time and the sum of the units all ranks processed."""
    if world <= 1:
        return float(total_ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def make_workload(name: str, scale: float = 1.0):
    src, tgt, p = W.config_meshes(name.replace("_online", ""), scale)
    return src, tgt, p


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_2603_00538_gb300 as sft

    rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    src, tgt, p = make_workload(args.workload, args.scale)
    N, tol = p["samples_per_elem"], p["cg_tol"]
    dim = src.dim
    if args.adaptive:
        args.adapt_ref = _mean_measure(tgt)
    prec = sft.SFT_PREC_FP64 if args.precision == "fp64" else sft.SFT_PREC_FP32
    stream = torch.cuda.current_stream()
    sc, sk, sv = (torch.as_tensor(np.ascontiguousarray(a)).to(dev) for a in (src.coords, src.conn, src.values))
    tc, tk = (torch.as_tensor(np.ascontiguousarray(a)).to(dev) for a in (tgt.coords, tgt.conn))
    u = torch.zeros((src.nfields, tgt.nnodes), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    stats_last = {}
    cons_last = [None]

    def step():
        s = sft.sft_source_create(sc, sk, sv, args.grid_scale)
        t = sft.sft_target_create(tc, tk)
        _, st, _ = sft.sft_transfer(s, t, N, prec, seed=0, cg_tol=tol, u_out=u, **_xfer(args))
        cons_last[0] = sft.sft_conservation_error(s, t, u[0])
        stats_last.update(st)
        s.close()
        t.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    asm_ms, solve_ms, setup_ms = [], [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))          # evict L2 between steps (untimed)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            asm_ms.append(stats_last["ms_assembly"])
            solve_ms.append(stats_last["ms_solve"])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    queries = int(stats_last["queries"])
    total_ms, all_queries = aggregate(float(sum(step_ms)), queries * args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    value = all_queries / (total_ms / 1e3)

    # kernels launched per step (profiled once, outside the timed region)
    launches_per_step = count_launches(step)

    # end to end through the public API with host (pinned) buffers
    e2e = run_e2e(args, src, tgt, N, tol, prec) if rank == 0 else None

    # errors at which the throughput is measured
    e_mass = cons_last[0][0]
    e_l2, e_l2_se = estimate_l2(src, tgt, u[0].cpu().numpy(), dev) if rank == 0 else (None, None)
    # the FP32 path against an all-FP64 run of the same workload (untimed)
    prec_cmp = precision_comparison(args, sc, sk, sv, tc, tk, N, tol) if rank == 0 else None
    # exact judge and comparison method (2D): mesh intersection (untimed)
    mi = mesh_intersection_leg(args, sc, sk, sv, tc, tk, u[0], N, tol) if rank == 0 and dim == 2 else None

    if rank == 0:
        hbm, which = peaks()
        mean_asm = float(np.mean(asm_ms))
        bq, be = (BYTES_PER_QUERY_FP64, BYTES_PER_ELEM_FP64) if args.precision == "fp64" else \
            (BYTES_PER_QUERY, BYTES_PER_ELEM)
        n_samples = queries - tgt.nnodes          # samples drawn (N per element unless --adaptive)
        alg_bytes = bq[dim] * n_samples + be[dim] * tgt.nelems
        achieved = alg_bytes / (mean_asm / 1e3) / 1e9
        traffic = measured_traffic(args.workload) if args.precision == "fp32" else None
        cpu = cpu_baseline(args, src, tgt, p, args.cpu_frac_baseline) if not args.skip_cpu else None
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}"
                                   + ("" if args.scale == 1.0 else f" (element counts x{args.scale})")
                                   + (" [all-FP64 run: FP64 sampling, location and evaluation]"
                                      if args.precision == "fp64" else ""),
                       "queries_per_step": queries, "target_elements": tgt.nelems, "samples_per_elem": N,
                       "source_elements": src.nelems, "grid_scale_L": args.grid_scale, "sampling": args.sampling,
                       "adaptive_counts": (f"N_t = min(8N, max(1, ceil(N |T| / {args.adapt_ref:.6g})))"
                                           if args.adaptive else "off"),
                       "precision": args.precision,
                       "l2": "flushed between steps (256 MB write)",
                       "accumulation": "FP64 load vector, CG and reductions",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "breakdown_ms": {"assembly_kernel": mean_asm, "solve": float(np.mean(solve_ms)),
                             "step_min": min(step_ms), "step_max": max(step_ms),
                             "transfer_call": stats_last["ms_total"], "control": stats_last["ms_control"]},
            "assembly_queries_per_s": n_samples / (mean_asm / 1e3),
            "accuracy": {"E_mass": e_mass, "E_L2_estimate": e_l2, "E_L2_stderr": e_l2_se,
                         "cg_iters": stats_last["cg_iters"], "cg_rel_resid": stats_last["cg_rel_resid"],
                         "fallback_queries": stats_last["fallback_queries"],
                         "fp32_vs_fp64": prec_cmp,
                         "E_L2_exact": mi["E_L2"] if mi else None},
            "mesh_intersection": mi,
            "roofline": {"kernel": "sft::k_assemble", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                         "peak_source": which, "algorithmic_bytes": alg_bytes},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": launches_per_step * args.steps if launches_per_step else None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """Batched workload: a step is one sft_batch_run over all requests (meshes
    resident, the plan built and autotuned beforehand); compared with the
    same requests run one by one through sft_transfer."""
    import torch
    import paper_2603_00538_gb300 as sft

    rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    srcm, reqs = W.batch_workload(scale=args.scale)
    srcs = [sft.mesh_source(m, device=dev) for m in srcm]
    tgts = [sft.mesh_target(q["target"], device=dev) for q in reqs]
    opts = [dict(samples_per_elem=q["samples_per_elem"], field_count=q["nfields"], seed=r, stream_id=r,
                 cg_tol=1e-10, cg_max_iter=1000) for r, q in enumerate(reqs)]
    rsrc = [srcs[q["source"]] for q in reqs]
    t0 = time.perf_counter()
    plan = sft.sft_batch_create(rsrc, tgts, opts, autotune=True)
    plan_s = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sft.sft_batch_run(plan)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times, stats = [], None
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, stats = sft.sft_batch_run(plan)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    queries = int(stats["queries"])
    total_ms, all_queries = aggregate(float(sum(times)), queries * args.steps, world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = all_queries / (total_ms / 1e3)
    launches = count_launches(lambda: sft.sft_batch_run(plan))
    # sequential plain launches of the same requests
    seq_ms = []
    u_bufs = [torch.zeros((q["nfields"], q["target"].nnodes), dtype=torch.float64, device=dev) for q in reqs]
    for r, q in enumerate(reqs):      # warm
        sft.sft_transfer(rsrc[r], tgts[r], q["samples_per_elem"], sft.SFT_PREC_FP32, seed=r, stream_id=r,
                         cg_tol=1e-10, u_out=u_bufs[r], field_count=q["nfields"])
    torch.cuda.synchronize()
    t_seq = time.perf_counter()
    for r, q in enumerate(reqs):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sft.sft_transfer(rsrc[r], tgts[r], q["samples_per_elem"], sft.SFT_PREC_FP32, seed=r, stream_id=r,
                         cg_tol=1e-10, u_out=u_bufs[r], field_count=q["nfields"])
        b.record(stream)
        b.synchronize()
        seq_ms.append(a.elapsed_time(b))
    seq_wall = (time.perf_counter() - t_seq) * 1e3
    # end to end: new field values for every source (H2D from pinned memory),
    # the batched run, every solution back to pinned host memory
    pinned_vals = [torch.as_tensor(m.values).pin_memory() for m in srcm]
    host_u = [torch.zeros(u.shape, dtype=torch.float64).pin_memory() for u in u_bufs]
    h2d = sum(v.numel() * v.element_size() for v in pinned_vals)
    d2h = sum(u.numel() * u.element_size() for u in host_u)

    def e2e_step():
        for s_, v in zip(srcs, pinned_vals):
            sft.sft_source_set_values(s_, v)
        sft.sft_batch_run(plan)
        for r in range(len(reqs)):
            sft.sft_batch_result(plan, r, u_out=host_u[r])

    e2e_step()
    torch.cuda.synchronize()
    k_e2e = max(1, min(args.steps, 3))
    t1 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t1) * 1e3 / k_e2e
    if rank == 0:
        hbm, which = peaks()
        alg = 0
        for q in reqs:
            d = q["dim"]
            alg += BYTES_PER_QUERY[d] * q["elems"] * q["samples_per_elem"] + BYTES_PER_ELEM[d] * q["elems"]
        achieved = alg / (stats["ms_assembly"] / 1e3) / 1e9
        cpu = None
        if not args.skip_cpu:
            import oracle
            sm = srcm[0]
            q0 = [q for q in reqs if q["source"] == 0][:4]
            t2 = time.perf_counter()
            nq = 0
            for q in q0:
                src_nf = W.Mesh(sm.coords, sm.conn, sm.values[:q["nfields"]])
                oracle.transfer(src_nf, q["target"], 1, q["samples_per_elem"], cg_tol=1e-10)
                nq += q["elems"] * q["samples_per_elem"] + q["target"].nnodes
            dt = time.perf_counter() - t2
            cpu = {"value": nq / dt, "unit": "queries/s", "cores": 1, "kind": "oracle", "seconds": dt,
                   "sample": f"the first {len(q0)} requests on the 2,048-triangle source, full oracle transfers"}
        seq_sorted = sorted(seq_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch256: {WORKLOADS['batch256']}" + ("" if args.scale == 1.0 else f" (element counts x{args.scale})"), "requests": len(reqs),
                       "queries_per_step": queries, "target_elements": int(sum(q["elems"] for q in reqs)),
                       "l2": "flushed between steps (256 MB write)", "plan_build_s": plan_s,
                       "graph": stats["graph"], "tiles": stats["tile"],
                       "autotuned_groups": sft.sft_batch_groups(plan),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "breakdown_ms": {"control": stats["ms_control"], "assembly": stats["ms_assembly"],
                             "solve": stats["ms_solve"], "cg_max_iters": stats["max_cg_iters"]},
            "sequential": {"total_ms_device": float(sum(seq_ms)), "wall_ms": seq_wall,
                           "p50_ms": seq_sorted[len(seq_sorted) // 2],
                           "p99_ms": seq_sorted[min(len(seq_sorted) - 1, int(0.99 * len(seq_sorted)))],
                           "speedup_batched": float(sum(seq_ms)) / ms_per_step},
            "batched_latency_ms": {"p50": float(np.median(times)), "p99": float(np.percentile(times, 99))},
            "roofline": {"kernel": "sft::k_batch_assemble (all groups)", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "peak_source": which, "algorithmic_bytes": alg},
            "cpu_baseline": cpu,
            "e2e": {"value": queries / (e2e_ms / 1e3), "unit": "queries/s", "ms_per_step": e2e_ms, "steps": k_e2e,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "timing": "host wall clock: new source values H2D, batched run, every solution D2H"},
            "clocks": clk.summary(),
            "gpu_launches": launches * args.steps if launches else None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# algorithmic HBM bytes of the online (recorded-location) assembly: per query
# the recorded element id and mu_1..d (2D 12 B, 3D 16 B) + the element's
# nodal values (one 16-byte load); per target element as for the full query
ONLINE_BYTES_PER_QUERY = {2: 28, 3: 32}


def run_online(args):
    """Online workload: the plan (initialization) is built once outside the
    timed region; a step is new source values (two device-resident value sets
    alternate) + sft_plan_transfer + the conservation error."""
    import torch
    import paper_2603_00538_gb300 as sft

    rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    src, tgt, p = make_workload(args.workload, args.scale)
    N, tol = p["samples_per_elem"], p["cg_tol"]
    dim = src.dim
    stream = torch.cuda.current_stream()
    S = sft.mesh_source(src, device=dev)
    T = sft.mesh_target(tgt, device=dev)
    vals = [torch.as_tensor(np.ascontiguousarray(src.values)).to(dev),
            torch.as_tensor(np.ascontiguousarray(src.values * np.float32(0.5) + np.float32(0.25))).to(dev)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = sft.sft_plan_create(S, T, N, sft.SFT_PREC_FP32, seed=0, cg_tol=tol, out_device=True,
                               sampling=_sampling(args))
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    u = torch.zeros((src.nfields, tgt.nnodes), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    last = {}

    def step(k):
        sft.sft_source_set_values(S, vals[k % 2])
        _, st, _ = sft.sft_plan_transfer(plan, u_out=u)
        last["cons"] = sft.sft_conservation_error(S, T, u[0])
        last.update(st)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    asm_ms, solve_ms = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step(k)
            ev[k][1].record(stream)
            asm_ms.append(last["ms_assembly"])
            solve_ms.append(last["ms_solve"])
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    queries = int(last["queries"])
    total_ms, all_queries = aggregate(float(sum(step_ms)), queries * args.steps, world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = all_queries / (total_ms / 1e3)
    launches = count_launches(lambda: step(0))
    # end to end: new values from pinned host memory, u back to pinned memory
    pin_vals = torch.as_tensor(np.ascontiguousarray(src.values)).pin_memory()
    u_h = torch.zeros((src.nfields, tgt.nnodes), dtype=torch.float64).pin_memory()
    plan_h = sft.sft_plan_create(S, T, N, sft.SFT_PREC_FP32, seed=0, cg_tol=tol, out_device=False,
                                 sampling=_sampling(args))

    def e2e_step():
        sft.sft_source_set_values(S, pin_vals)
        sft.sft_plan_transfer(plan_h, u_out=u_h)
        sft.sft_conservation_error(S, T, u_h[0])

    e2e_step()
    torch.cuda.synchronize()
    k_e2e = max(1, min(args.steps, 5))
    t1 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t1) * 1e3 / k_e2e
    if rank == 0:
        hbm, which = peaks()
        mean_asm = float(np.mean(asm_ms))
        alg_bytes = ONLINE_BYTES_PER_QUERY[dim] * tgt.nelems * N + BYTES_PER_ELEM[dim] * tgt.nelems
        achieved = alg_bytes / (mean_asm / 1e3) / 1e9
        cpu = None
        if not args.skip_cpu:
            cpu = cpu_baseline(args, src, tgt, p, args.cpu_frac_baseline)
            cpu["sample"] += "; the oracle has no plan, so this is its full transfer"
        base = args.workload.replace("_online", "")
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}; meshes: {WORKLOADS[base]}",
                       "queries_per_step": queries, "target_elements": tgt.nelems, "samples_per_elem": N,
                       "plan_create_s": plan_s, "plan_bytes": sft.sft_plan_bytes(plan),
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "breakdown_ms": {"assembly_kernel": mean_asm, "solve": float(np.mean(solve_ms)),
                             "control": last["ms_control"], "transfer_call": last["ms_total"],
                             "step_min": min(step_ms), "step_max": max(step_ms)},
            "assembly_queries_per_s": tgt.nelems * N / (mean_asm / 1e3),
            "accuracy": {"E_mass": last["cons"][0], "cg_iters": last["cg_iters"],
                         "cg_rel_resid": last["cg_rel_resid"]},
            "roofline": {"kernel": "sft::k_assemble (recorded locations)", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "peak_source": which, "algorithmic_bytes": alg_bytes},
            "cpu_baseline": cpu,
            "e2e": {"value": queries / (e2e_ms / 1e3), "unit": "queries/s", "ms_per_step": e2e_ms, "steps": k_e2e,
                    "h2d_bytes_per_step": int(pin_vals.numel() * pin_vals.element_size()),
                    "d2h_bytes_per_step": int(u_h.numel() * u_h.element_size()),
                    "timing": "host wall clock: new source values H2D, online transfer, u D2H, conservation error "
                              "(the timed step's calls)"},
            "clocks": clk.summary(),
            "gpu_launches": launches * args.steps if launches else None,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    plan_h.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# FLOPs of one network query: 2 * (3*256 + 3*256^2 + 256) multiply-adds
NET_FLOP_PER_QUERY = 2 * (3 * 256 + 3 * 256 * 256 + 256)
SUR_KERNEL_FILES = ["paper_2603_00538_gb300/csrc/surrogate.cu", "paper_2603_00538_gb300/csrc/mlp.cuh",
                    "paper_2603_00538_gb300/csrc/tc.cuh"]


def run_roundtrip(args):
    """Round-trip workload: plans mesh 1 -> mesh 2 and mesh 2 -> mesh 1 built
    once; the field starts at the reference f2 after the warm-up; a step is
    one round trip. Reports the discrete l2 and conservation errors on mesh 1
    after the timed round trips and, from an untimed run, after each of the
    first ten."""
    import torch
    import paper_2603_00538_gb300 as sft

    rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m1, m2, p = W.config_meshes("roundtrip", args.scale)
    N, tol = p["samples_per_elem"], p["cg_tol"]
    stream = torch.cuda.current_stream()
    s1, t1 = sft.mesh_source(m1, device=dev), sft.mesh_target(m1, device=dev)
    s2, t2 = sft.mesh_source(m2, device=dev), sft.mesh_target(m2, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rt = sft.RoundTrip(s1, t1, s2, t2, N, seeds=(0, 1), cg_tol=tol, sampling=_sampling(args),
                       warm_start=not args.cold_start)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    ref = torch.as_tensor(np.ascontiguousarray(m1.values)).to(dev)
    f = ref.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lump = torch.as_tensor(sft.sft_target_mass(t1)[3]).to(dev)

    def errors(x):
        e_l2 = float(torch.linalg.norm(x[0] - ref[0]) / torch.linalg.norm(ref[0]))
        i_ref = float(lump @ ref[0])
        return e_l2, abs(float(lump @ x[0]) - i_ref) / abs(i_ref)

    curve = []
    for _ in range(10):
        rt.run(f, 1)
        curve.append(errors(f))
    for _ in range(args.warmup):
        rt.run(f, 1)
    f.copy_(ref)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            rt.run(f, 1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    final = errors(f)
    queries = int(rt.queries)
    total_ms, all_queries = aggregate(float(sum(step_ms)), queries * args.steps, world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = all_queries / (total_ms / 1e3)
    launches = count_launches(lambda: rt.run(f, 1))
    # end to end: the field from pinned host memory, the round trip, the field back
    f_h = torch.as_tensor(np.ascontiguousarray(m1.values)).pin_memory()
    k_e2e = max(1, min(args.steps, 5))

    def e2e_step():
        f.copy_(f_h, non_blocking=True)
        rt.run(f, 1)
        f_h.copy_(f, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    t1w = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    e2e_ms = (time.perf_counter() - t1w) * 1e3 / k_e2e
    if rank == 0:
        hbm, which = peaks()
        cpu = None
        if not args.skip_cpu:
            import oracle
            ms1, ms2, _ = W.config_meshes("roundtrip", 0.1)
            t0c = time.perf_counter()
            oracle.roundtrip(ms1, ms2, ms1.values[0], 1, 1, N, cg_tol=tol, sampling=_sampling(args))
            dt = time.perf_counter() - t0c
            qc = (ms2.nnodes + ms2.nelems * N) + (ms1.nnodes + ms1.nelems * N)
            cpu = {"value": qc / dt, "unit": "queries/s", "cores": 1, "kind": "oracle", "seconds": dt,
                   "sample": f"one oracle round trip on the same generators at 1/10 of the element counts "
                             f"({ms1.nelems} and {ms2.nelems} triangles, grid builds included)"}
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"roundtrip: {WORKLOADS['roundtrip']}" + ("" if args.scale == 1.0 else f" (element counts x{args.scale})"), "queries_per_step": queries,
                       "mesh1_elements": m1.nelems, "mesh2_elements": m2.nelems, "samples_per_elem": N,
                       "sampling": args.sampling, "plan_create_s": plan_s,
                       "solve_start": "zero" if args.cold_start else "each leg's previous result (warm start)",
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "breakdown_ms": {"round_trip_min": min(step_ms), "round_trip_max": max(step_ms)},
            "accuracy": {"after_timed_round_trips": {"round_trips": args.steps, "E_l2": final[0],
                                                     "E_mass": final[1]},
                         "per_round_trip_first_10": [{"E_l2": a, "E_mass": b} for a, b in curve]},
            "roofline": None,
            "cpu_baseline": cpu,
            "e2e": {"value": queries / (e2e_ms / 1e3), "unit": "queries/s", "ms_per_step": e2e_ms, "steps": k_e2e,
                    "h2d_bytes_per_step": int(f_h.numel() * f_h.element_size()),
                    "d2h_bytes_per_step": int(f_h.numel() * f_h.element_size()),
                    "timing": "host wall clock: field H2D, one round trip, field D2H"},
            "clocks": clk.summary(),
            "gpu_launches": launches * args.steps if launches else None,
        }
        print(json.dumps(line), flush=True)
    rt.close()


def run_surrogate(args):
    """Surrogate workload: the network is trained once (timed separately); a
    step is one sft_transfer_surrogate (control at the target nodes from the
    network, fused sampling / network / fallback / scatter kernel, FP64 CG)
    plus the conservation error. Compared with the exact-only transfer of the
    same source on the same samples (every query a mesh location)."""
    import torch
    import paper_2603_00538_gb300 as sft

    rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    src, tgt, p = make_workload("sur3d", args.scale)
    N, tol = p["samples_per_elem"], p["cg_tol"]
    S = sft.mesh_source(src, device=dev)
    T = sft.mesh_target(tgt, device=dev)
    stream = torch.cuda.current_stream()
    # training set and training (outside the timed region)
    t0 = time.perf_counter()
    pts, f, fmax = sft.sft_surrogate_dataset(S, p["train_points"], seed=1, stream_id=0)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    net = sft.sft_mlp_create(W.mlp_init(0).astype(np.float32))
    t0 = time.perf_counter()
    hist = sft.sft_mlp_train(net, pts, f, epochs=args.sur_epochs, batch=16384, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    tau = p["tau_rel"] * fmax
    u = torch.zeros(tgt.nnodes, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    last = {}

    def step():
        _, st, _ = sft.sft_transfer_surrogate(net, S, T, N, seed=0, cg_tol=tol, subsample=p["subsample"], tau=tau,
                                              u_out=u)
        last["cons"] = sft.sft_conservation_error(S, T, u)
        last.update(st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    asm_ms = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            asm_ms.append(last["ms_assembly"])
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    queries = int(last["net_queries"])
    total_ms, all_queries = aggregate(float(sum(step_ms)), queries * args.steps, world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = all_queries / (total_ms / 1e3)
    launches = count_launches(step)
    stats_sur = dict(last)
    u_sur = u.clone()

    # the same transfer with every query exact (no network)
    ue = torch.zeros_like(u)
    ex = {}
    for _ in range(2):
        _, ex, _ = sft.sft_transfer_surrogate(None, S, T, N, seed=0, cg_tol=tol, u_out=ue)
    ex_ms = []
    for k in range(max(3, min(args.steps, 10))):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, ex, _ = sft.sft_transfer_surrogate(None, S, T, N, seed=0, cg_tol=tol, u_out=ue)
        b.record(stream)
        torch.cuda.synchronize()
        ex_ms.append(a.elapsed_time(b))
    cons_ex = sft.sft_conservation_error(S, T, ue)
    m = torch.as_tensor(_lumped_mass(tgt)).to(dev)
    rel_diff = float(torch.sqrt((m * (u_sur - ue) ** 2).sum() / (m * ue ** 2).sum()).item())

    # end to end: target mesh from pinned host memory, u back to pinned memory
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    tc_h, tk_h = pin(tgt.coords), pin(tgt.conn)
    u_h = torch.zeros(tgt.nnodes, dtype=torch.float64).pin_memory()

    def e2e_step():
        t_ = sft.sft_target_create(tc_h, tk_h)
        sft.sft_transfer_surrogate(net, S, t_, N, seed=0, cg_tol=tol, subsample=p["subsample"], tau=tau, u_out=u_h)
        t_.close()

    e2e_step()
    torch.cuda.synchronize()
    k_e2e = max(1, min(args.steps, 3))
    t1 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t1) * 1e3 / k_e2e

    if rank == 0:
        mean_asm = float(np.mean(asm_ms))
        # network work actually done: every sample of the elements that keep
        # the network, plus the decision subsample of every element
        net_queries = (tgt.nelems - int(stats_sur["fallback_elems"])) * N + tgt.nelems * int(p["subsample"])
        flops = NET_FLOP_PER_QUERY * net_queries
        achieved = flops / (mean_asm / 1e3) / 1e12
        peak, which = tensor_peak()
        cpu = None if args.skip_cpu else sur_cpu_baseline(src, tgt, p, net, tau)
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "sur3d: " + WORKLOADS["sur3d"]
                                   + ("" if args.scale == 1.0 else f" (element counts x{args.scale})"),
                       "queries_per_step": queries, "target_elements": tgt.nelems, "samples_per_elem": N,
                       "source_elements": src.nelems, "train_points": p["train_points"],
                       "train_epochs": args.sur_epochs, "train_s": train_s, "dataset_s": data_s,
                       "train_loss_first_last": [float(hist[0]), float(hist[-1])], "tau": tau,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "breakdown_ms": {"assembly_kernel": mean_asm, "control": stats_sur["ms_control"],
                             "solve": stats_sur["ms_solve"], "transfer_call": stats_sur["ms_total"],
                             "step_min": min(step_ms), "step_max": max(step_ms)},
            "fallback": {"elements": int(stats_sur["fallback_elems"]),
                         "fraction": stats_sur["fallback_elems"] / tgt.nelems,
                         "exact_queries": int(stats_sur["exact_queries"])},
            "accuracy": {"E_mass": last["cons"][0], "E_mass_exact_path": cons_ex[0],
                         "rel_diff_u_vs_exact_path": rel_diff, "cg_iters": stats_sur["cg_iters"]},
            "exact_path": {"ms_per_step": float(np.mean(ex_ms)), "assembly_ms": ex["ms_assembly"],
                           "queries_per_s": (tgt.nelems * N + tgt.nnodes) / (float(np.mean(ex_ms)) / 1e3),
                           "surrogate_over_exact_time": ms_per_step / float(np.mean(ex_ms))},
            "roofline": {"kernel": "sft::k_surrogate_net (with the decision and exact passes)", "bound": "tensor", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": which, "algorithmic_flops": flops, "network_queries": net_queries,
                         "flop_model": "0.395 MFLOP per network query: N per element that keeps the network "
                                       "+ the s-sample decision subsample of every element; time = the whole "
                                       "assembly (decision, network pass, exact pass of the fallbacks)"},
            "cpu_baseline": cpu,
            "e2e": {"value": queries / (e2e_ms / 1e3), "unit": "queries/s", "ms_per_step": e2e_ms, "steps": k_e2e,
                    "h2d_bytes_per_step": int(tc_h.numel() * tc_h.element_size() + tk_h.numel() * tk_h.element_size()),
                    "d2h_bytes_per_step": int(u_h.numel() * u_h.element_size()),
                    "timing": "host wall clock: target mesh H2D + target setup, surrogate transfer, u D2H"},
            "clocks": clk.summary(),
            "gpu_launches": launches * args.steps if launches else None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def tensor_peak():
    """Dense BF16 tensor peak: the sustained (seconds-long) measurement, the
    kernel runs inside a long step."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured (sustained)"
    return 1700.0, "fallback (sustained)"


def _lumped_mass(mesh):
    x = mesh.coords.astype(np.float64)[mesh.conn]
    if mesh.conn.shape[1] == 3:
        e1, e2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
        vol = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    else:
        vol = np.linalg.det(x[:, 1:] - x[:, :1]) / 6.0
    m = np.zeros(mesh.coords.shape[0])
    np.add.at(m, mesh.conn.ravel(), np.repeat(vol / mesh.conn.shape[1], mesh.conn.shape[1]))
    return m


def sur_cpu_baseline(src, tgt, p, net, tau, nelem=256):
    """The oracle's surrogate transfer (FP64 network, FP32 sampler and
    location) on the first `nelem` target elements (Morton order) with the
    trained weights and the full exact source."""
    import paper_2603_00538_gb300 as sft
    from oracle import surrogate as OS
    params = sft.sft_mlp_params(net).astype(np.float64)
    tgt_s = _sample_target(tgt, nelem / tgt.nelems)
    t0 = time.perf_counter()
    OS.surrogate_transfer(params, tgt_s.coords, tgt_s.conn, p["samples_per_elem"],
                          exact=(src.coords, src.conn, src.values[0]), tau=tau, s=p["subsample"])
    dt = time.perf_counter() - t0
    q = tgt_s.nelems * p["samples_per_elem"] + tgt_s.nnodes
    return {"value": q / dt, "unit": "queries/s", "cores": 1, "kind": "oracle", "seconds": dt,
            "sample": f"the first {tgt_s.nelems} target elements (Morton order) with the trained network and "
                      f"the full exact source (grid build included), one oracle surrogate transfer"}


def count_launches(step):
    """Kernels libsft launches in one step (its own launch counter)."""
    import torch
    import paper_2603_00538_gb300 as sft
    n0 = sft.sft_kernel_launches()
    step()
    torch.cuda.synchronize()
    return sft.sft_kernel_launches() - n0


def mesh_intersection_leg(args, sc, sk, sv, tc, tk, u, N, tol):
    """The exact judge at full size (2D): the supermesh L2 error of the
    benchmark's solution u, and the mesh-intersection load vector (the
    paper's comparison method) timed with CUDA events against the Monte
    Carlo assembly of the same source and target; the Monte Carlo load
    vector's distance from the exact one."""
    import torch
    import paper_2603_00538_gb300 as sft
    s = sft.sft_source_create(sc, sk, sv, args.grid_scale)
    t = sft.sft_target_create(tc, tk)
    stream = torch.cuda.current_stream()
    b = torch.zeros(tc.shape[0], dtype=torch.float64, device=sc.device)
    sft.sft_mi_load_vector(s, t, 0, b_out=b)            # builds the FP64 location structure once
    ms = []
    for _ in range(3):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sft.sft_mi_load_vector(s, t, 0, b_out=b)
        z.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(z))
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    e, n = sft.sft_mi_l2_error(s, t, u, 0)
    z.record(stream)
    torch.cuda.synchronize()
    bmc = torch.zeros((sv.shape[0], tc.shape[0]), dtype=torch.float64, device=sc.device)
    umc = torch.zeros_like(bmc)
    _, st, _ = sft.sft_transfer(s, t, N, sft.SFT_PREC_FP32, seed=0, cg_tol=tol, u_out=umc, b_out=bmc,
                                **_xfer(args))
    bx = b.cpu().numpy()
    bm = bmc[0].cpu().numpy()
    s.close()
    t.close()
    return {"E_L2": e / n, "load_vector_ms": float(np.median(ms)), "l2_error_ms": a.elapsed_time(z),
            "mc_assembly_ms": st["ms_assembly"],
            "b_mc_vs_exact_rel_l2": float(np.linalg.norm(bm - bx) / np.linalg.norm(bx)),
            "method": "2D clipping of every overlapping (target, source) triangle pair, FP64, edge-midpoint rule"}


def precision_comparison(args, sc, sk, sv, tc, tk, N, tol):
    """One FP32-path transfer and one all-FP64 transfer of the same workload
    (same Philox streams: the FP32 uniforms are the FP64 ones rounded to 24
    bits), outside the timed region: the FP32 path's load vector and solution
    against the FP64 run (2-norm ratio and largest entry against the largest
    entry), each run's conservation error and assembly time."""
    import torch
    import paper_2603_00538_gb300 as sft
    out, res = {}, {}
    s = sft.sft_source_create(sc, sk, sv, args.grid_scale)
    t = sft.sft_target_create(tc, tk)
    for name, prec in (("fp32", sft.SFT_PREC_FP32), ("fp64", sft.SFT_PREC_FP64)):
        u = torch.zeros((sv.shape[0], tc.shape[0]), dtype=torch.float64, device=sc.device)
        b = torch.zeros_like(u)
        sft.sft_transfer(s, t, N, prec, seed=0, cg_tol=tol, u_out=u, b_out=b, **_xfer(args))
        _, st, _ = sft.sft_transfer(s, t, N, prec, seed=0, cg_tol=tol, u_out=u, b_out=b, **_xfer(args))
        e = sft.sft_conservation_error(s, t, u[0])[0]
        res[name] = (b[0].cpu().numpy(), u[0].cpu().numpy())
        out[f"E_mass_{name}"] = e
        out[f"assembly_ms_{name}"] = st["ms_assembly"]
    s.close()
    t.close()
    for k, i in (("b", 0), ("u", 1)):
        a, r = res["fp32"][i], res["fp64"][i]
        out[f"{k}_rel_l2"] = float(np.linalg.norm(a - r) / np.linalg.norm(r))
        out[f"{k}_rel_max"] = float(np.max(np.abs(a - r)) / np.max(np.abs(r)))
    return out


def run_e2e(args, src, tgt, N, tol, prec):
    import torch
    import paper_2603_00538_gb300 as sft
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    sc, sk, sv, tc, tk = (pin(a) for a in (src.coords, src.conn, src.values, tgt.coords, tgt.conn))
    u = torch.zeros((src.nfields, tgt.nnodes), dtype=torch.float64).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in (sc, sk, sv, tc, tk))
    d2h = u.numel() * u.element_size() + 8

    def step():
        s = sft.sft_source_create(sc, sk, sv, args.grid_scale)
        t = sft.sft_target_create(tc, tk)
        _, st, _ = sft.sft_transfer(s, t, N, prec, seed=0, cg_tol=tol, u_out=u, **_xfer(args))
        e = sft.sft_conservation_error(s, t, u[0])
        s.close()
        t.close()
        return st["queries"], e

    for _ in range(max(1, min(args.warmup, 3))):
        step()
    torch.cuda.synchronize()
    k = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    q = 0
    for _ in range(k):
        q, _ = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    return {"value": q / dt, "unit": "queries/s", "ms_per_step": dt * 1e3, "steps": k,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "timing": "host wall clock around sft_* calls with pinned host buffers"}


def estimate_l2(src, tgt, u, dev, npts=1 << 22):
    """E_L2 estimate (not exact): both meshes queried at the same uniform
    random points of the unit domain through sft_locate."""
    import torch
    import paper_2603_00538_gb300 as sft
    rng = np.random.default_rng(12345)
    pts = torch.as_tensor(rng.random((npts, src.dim))).to(dev)
    s = sft.mesh_source(src, device=dev)
    tsrc = sft.sft_source_create(torch.as_tensor(tgt.coords.astype(np.float64)).to(dev),
                                 torch.as_tensor(tgt.conn).to(dev), torch.as_tensor(u[None, :]).to(dev))
    fs = torch.zeros((1, npts), dtype=torch.float64, device=dev)
    ft = torch.zeros_like(fs)
    es = torch.zeros(npts, dtype=torch.int32, device=dev)
    et = torch.zeros_like(es)
    sft.sft_locate(s, pts, sft.SFT_PREC_FP64, elem_out=es, val_out=fs)
    sft.sft_locate(tsrc, pts, sft.SFT_PREC_FP64, elem_out=et, val_out=ft)
    d2 = ((fs - ft) ** 2).cpu().numpy()[0]
    f2 = (fs ** 2).cpu().numpy()[0]
    e = math.sqrt(d2.mean() / f2.mean())
    se = 0.5 * e * math.sqrt(d2.var() / npts) / max(d2.mean(), 1e-300)
    s.close()
    tsrc.close()
    return e, se


# ---------------------------------------------------------------------------
# the oracle: CPU baseline and the reference arm
# ---------------------------------------------------------------------------
def _sample_target(tgt, frac):
    """The first `frac` of the target elements (Morton order: a compact patch),
    nodes renumbered."""
    ne = max(1, int(tgt.nelems * frac))
    conn = tgt.conn[:ne]
    used = np.unique(conn)
    remap = -np.ones(tgt.nnodes, np.int64)
    remap[used] = np.arange(used.size)
    return W.Mesh(tgt.coords[used], remap[conn].astype(np.int32))


def oracle_step(src, tgt_s, p, sampling=0, adapt_ref_measure=0.0):
    import oracle
    t0 = time.perf_counter()
    r = oracle.transfer(src, tgt_s, 1, p["samples_per_elem"], seed=0, cg_tol=p["cg_tol"], cg_max_iter=1000,
                        sampling=sampling, adapt_ref_measure=adapt_ref_measure)
    dt = time.perf_counter() - t0
    return (int(r["samples"]) + tgt_s.nnodes) / dt, dt, r


def _sampling(args) -> int:
    """sft_sampling value of --sampling (0 uniform, 1 stratified, 2 importance)."""
    return {"uniform": 0, "stratified": 1, "importance": 2}[getattr(args, "sampling", "uniform")]


def _xfer(args) -> dict:
    """Sampling options of one sft_transfer / oracle.transfer call: the scheme
    and, with --adaptive, per-element sample counts against the mean target
    element measure (adapt_ref_measure; 0 = N everywhere)."""
    return {"sampling": _sampling(args), "adapt_ref_measure": float(getattr(args, "adapt_ref", 0.0))}


def _mean_measure(mesh) -> float:
    """Mean element measure of a simplicial mesh (FP64, host)."""
    x = mesh.coords.astype(np.float64)[mesh.conn.astype(np.int64)]     # [E, d+1, d]
    J = x[:, 1:, :] - x[:, :1, :]
    d = J.shape[1]
    return float(np.abs(np.linalg.det(J)).mean() / (2.0 if d == 2 else 6.0))


def cpu_baseline(args, src, tgt, p, frac):
    tgt_s = _sample_target(tgt, frac)
    v, dt, _ = oracle_step(src, tgt_s, p, **_xfer(args))
    return {"value": v, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "seconds": dt,
            "sample": f"full source mesh (grid build included) and the first {tgt_s.nelems} target "
                      f"elements in Morton order ({frac:.3g} of the workload), one full oracle transfer"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "batch256":
        import oracle
        srcm, reqs = W.batch_workload(scale=args.scale)
        q0 = [q for q in reqs if q["source"] == 0][:4]

        def one():
            t0 = time.perf_counter()
            for q in q0:
                oracle.transfer(W.Mesh(srcm[0].coords, srcm[0].conn, srcm[0].values[:q["nfields"]]),
                                q["target"], 1, q["samples_per_elem"], cg_tol=1e-10)
            return time.perf_counter() - t0
        q = sum(q["elems"] * q["samples_per_elem"] + q["target"].nnodes for q in q0)
        sample = f"the first {len(q0)} requests on the 2,048-triangle source per step, full oracle transfers"
    elif args.workload == "sur3d":
        from oracle import surrogate as OS
        src, tgt, p = make_workload(args.workload, args.scale)
        tgt_s = _sample_target(tgt, min(1.0, 64 / tgt.nelems))
        params = W.mlp_init(0).astype(np.float32).astype(np.float64)
        tau = p["tau_rel"] * float(np.abs(src.values[0]).max())

        def one():
            t0 = time.perf_counter()
            OS.surrogate_transfer(params, tgt_s.coords, tgt_s.conn, p["samples_per_elem"],
                                  exact=(src.coords, src.conn, src.values[0]), tau=tau, s=p["subsample"])
            return time.perf_counter() - t0
        q = tgt_s.nelems * p["samples_per_elem"] + tgt_s.nnodes
        sample = (f"the first {tgt_s.nelems} target elements (Morton order) per step, the initial network "
                  f"weights, the full exact source (grid build included)")
    elif args.workload == "roundtrip":
        import oracle
        ms1, ms2, p = W.config_meshes("roundtrip", 0.01 * args.scale)

        def one():
            t0 = time.perf_counter()
            oracle.roundtrip(ms1, ms2, ms1.values[0], 1, 1, p["samples_per_elem"], cg_tol=p["cg_tol"],
                             sampling=_sampling(args))
            return time.perf_counter() - t0
        q = (ms2.nnodes + ms2.nelems * p["samples_per_elem"]) + (ms1.nnodes + ms1.nelems * p["samples_per_elem"])
        sample = (f"one oracle round trip per step on the same generators at 1/100 of the element counts "
                  f"({ms1.nelems} and {ms2.nelems} triangles)")
    else:
        src, tgt, p = make_workload(args.workload, args.scale)
        tgt_s = _sample_target(tgt, args.cpu_frac)

        if args.adaptive:
            args.adapt_ref = _mean_measure(tgt)
        seen = {}

        def one():
            _, dt, r = oracle_step(src, tgt_s, p, **_xfer(args))
            seen["q"] = int(r["samples"]) + tgt_s.nnodes   # queries of the step (adaptive counts included)
            return dt
        q = None
        sample = (f"full source mesh and the first {tgt_s.nelems} target elements (Morton order, "
                  f"{args.cpu_frac:.3g} of the workload) per step")
    for _ in range(args.warmup):
        one()
    times = [one() for _ in range(args.steps)]
    if q is None:
        q = seen["q"]
    ms = 1e3 * float(np.mean(times))
    value = q / (ms / 1e3)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}"
                               + ("" if args.scale == 1.0 else f" (element counts x{args.scale})"), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="tri4m")
    ap.add_argument("--cpu-frac", type=float, default=0.05,
                    help="fraction of the target elements per reference-arm step")
    ap.add_argument("--cpu-frac-baseline", type=float, default=0.4,
                    help="fraction of the target elements in the cpu_baseline sample")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--sur-epochs", type=int, default=40, help="training epochs of the surrogate (sur3d)")
    ap.add_argument("--grid-scale", type=float, default=1.0,
                    help="source grid cells per axis = int(L * nelems^(1/d)) (tri4m / tet5m)")
    ap.add_argument("--sampling", choices=["uniform", "stratified", "importance"], default="uniform",
                    help="sample scheme of the mesh-source workloads (tri4m, tet5m and their online forms; "
                         "importance: tri4m / tet5m only)")
    ap.add_argument("--adaptive", action="store_true",
                    help="tri4m / tet5m: per-element sample counts proportional to the element measure "
                         "(reference measure = the mean target element measure)")
    ap.add_argument("--cold-start", action="store_true",
                    help="roundtrip: start every solve from 0 instead of the leg's previous result")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="tri4m / tet5m: arithmetic of sampling, location and evaluation (fp32: compensated "
                         "FP32 partials, FP64 load vector / CG / reductions; fp64: all FP64)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="element-count scale of the workload (1 = the named workload)")
    args = ap.parse_args()
    args.adapt_ref = 0.0
    if (args.sampling == "importance" or args.adaptive) and args.workload not in ("tri4m", "tet5m"):
        ap.error("--sampling importance and --adaptive apply to tri4m and tet5m only")
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "sur3d":
        run_surrogate(args)
    elif args.workload == "roundtrip":
        run_roundtrip(args)
    elif args.workload.endswith("_online"):
        run_online(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
