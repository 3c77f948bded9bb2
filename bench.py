"""Benchmark: walk-on-boundary path vertices per second on one GB300.

Workload (the second configuration of the method's benchmark set): a
non-convex star-shaped mesh (icosphere level 6, 81,920 triangles, radius
1 + 0.3 * seeded real spherical harmonics up to degree 6), Dirichlet data
g = 1 / |x - (3, 0, 0)|, double-layer formulation, query points on a
256 x 256 z = 0 slice of [-1.3, 1.3]^2 clipped to the interior, 1,024 walks
per point, up to 16 boundary vertices per walk, Philox seed 0.  A step is one
wob_solve over all queries (walk kernel + per-query FP64 reduction); a path
vertex is one line query.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream, with a 512 MB buffer written between steps to flush L2;
max over ranks.  Under torchrun every rank solves its own replica (problem
index = rank, independent random streams): weak scaling, no collective on
the data path.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WoB path vertices/sec on 1 GB300"
UNIT = "path vertices/s"
WALKS, MAX_LEN, SEED = 1024, 16, 0
X0 = (3.0, 0.0, 0.0)

# Algorithmic per-event costs: lane operations of the FP32/INT32 pipes counted
# from the traversal source (per 8-wide node: header decode and eight 3-slab
# tests on dequantised child boxes; per triangle: the sheared edge functions,
# flags and hit test; per hit: one Philox block and the key comparison; per
# line: axis, setup, float-float refinement (about 365 FP32 operations),
# data term and accumulation), and the bytes fetched per node and triangle.
OPS_NODE, OPS_TRI, OPS_HIT, OPS_LINE = 320, 41, 100, 585
BYTES_NODE, BYTES_TRI = 96, 48
# DRAM bytes (read + write) of one full-size k_dl_walks launch of this
# workload (queries, leaf size, bytes) from ncu dram__bytes_read.sum +
# dram__bytes_write.sum (profiles/k_dl_walks_star6_wide.md); None while the
# kernel has changed since the last capture.
TRAFFIC_FULL = (29497, 1, 27.07e6 + 135.12e6)
# The walk kernel's issue-slot use from the same profile: fraction of cycles
# with an instruction issued, and active threads per warp instruction; None
# while the kernel has changed since the last capture.
ISSUE_PROFILE = (0.722, 10.77)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _workload(kind: str = "star"):
    """The headline star (coefficients N(0,1)/(l+1)^2, seed 0: a near-convex
    shape, 1.06 hits per line) or, for `--workload spiky`, the same generator
    with coefficients N(0,1)/(l+1)^0.5 and seed 3, a genuinely non-convex
    star whose lines meet the surface up to 7 times (the pick-one-of-m of
    Sec. 4.4.1 with m > 2); queries on its z = 0 slice."""
    from paper_2305_04403_gb300 import inputs as I
    if kind == "spiky":
        v, f, shape = I.star_mesh(6, 0.3, 6, 3, 0.5)
    else:
        v, f, shape = I.star_mesh(6)
    q = I.star_slice_queries(shape, 256)
    return v, f, q


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self) -> dict:
        mhz, maxmhz, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1].split()[0]))
                maxmhz = float(parts[2].split()[0])
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": maxmhz,
                "reasons": sorted(reasons), "samples": len(mhz)}


def _l2_probe(mb: int = 96, passes: int = 20, reps: int = 5) -> float:
    """L2 read bandwidth (GB/s): the library's streaming-read probe (16-byte
    loads that bypass L1, every SM) over a buffer that fits in the 129 MB
    L2, `passes` reads per call, CUDA events, median of `reps` calls after a
    warm-up call."""
    import torch
    import paper_2305_04403_gb300 as wob
    buf = torch.ones(mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    wob.probe_l2_read(buf, passes, out)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wob.probe_l2_read(buf, passes, out)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b) / passes)
    return buf.numel() * 4 / (float(np.median(ms)) / 1e3) / 1e9


def _over_ranks(dist, x: float, op: str, device) -> float:
    """Max or sum of a per-rank number over the ranks (x itself without a
    process group): the timed region is the slowest rank's, the work is
    every rank's."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _star_config(Q: int, leaf: int, ws: int, kind: str = "star") -> dict:
    """The headline workload's `config` (both arms of the benchmark)."""
    shape = ("spiky star-shaped icosphere L6 (81,920 tris; SH coefficients N(0,1)/(l+1)^0.5, "
             "seed 3)" if kind == "spiky" else "star-shaped icosphere L6 (81,920 tris)")
    return {"workload": f"{shape}, z=0 slice Q={Q}, "
                        f"{WALKS} walks, M={MAX_LEN}, Dirichlet double layer, g=1/|x-(3,0,0)|",
            "queries": Q, "walks": WALKS, "max_len": MAX_LEN, "leaf_size": leaf,
            "l2": "flushed (512 MB write) between timed steps",
            "parallelism": f"{ws} independent replica(s)"}


def run_ours(args):
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    v, f, q = _workload(args.workload)
    if args.queries:
        q = q[:: max(1, len(q) // args.queries)][:args.queries].copy()
    Q = q.shape[0]
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    prob = wob.Problem(bvh, kind=wob.DIRICHLET_DL, side=1, data_mode=wob.DATA_POINT, x0=X0,
                       problem=rank)
    qd = torch.from_numpy(q).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # algorithmic work of one step (deterministic walks: exact counts)
    _, _, st = wob.solve_counted(prob, qd, WALKS, MAX_LEN, seed=SEED)
    lines = st["lines"]

    for _ in range(args.warmup):
        wob.solve(prob, qd, WALKS, MAX_LEN, seed=SEED)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            est, var = wob.solve(prob, qd, WALKS, MAX_LEN, seed=SEED)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = _over_ranks(dist, sum(step_ms), "max", "cuda")
    lines_all = _over_ranks(dist, float(lines), "sum", "cuda")  # every replica's line queries
    if dist:
        dist.barrier()
    clocks = clk.summary()

    # end to end through the host-buffer entry point (pinned host memory)
    qh = torch.from_numpy(q).pin_memory()
    est_h = torch.empty(Q, dtype=torch.float64).pin_memory()
    var_h = torch.empty(Q, dtype=torch.float64).pin_memory()
    lib = wob.load_library()
    import ctypes
    pc = prob._c()

    def host_step():
        rc = lib.wob_solve_host(ctypes.byref(pc), ctypes.c_void_p(qh.data_ptr()), None, Q, WALKS,
                                MAX_LEN, SEED, ctypes.c_void_p(est_h.data_ptr()),
                                ctypes.c_void_p(var_h.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(lib.wob_last_error().decode())

    host_step()
    e2e_steps = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    e2e_s = _over_ranks(dist, time.perf_counter() - t0, "max", "cuda")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    peaks, which = _peaks()
    l2_gbs = _l2_probe()
    per_launch_s = total_ms / 1e3 / args.steps
    ops = (st["node_visits"] * OPS_NODE + st["tri_tests"] * OPS_TRI + st["hits"] * OPS_HIT
           + st["lines"] * OPS_LINE)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * sm_max * 1e6 / 1e12  # T lane-ops/s
    achieved_ops = ops / per_launch_s / 1e12
    # algorithmic bytes of the traversal: every 8-wide node and leaf triangle
    # the lines fetch (served from L1/L2: the BVH is L2-resident)
    bytes_step = st["node_visits"] * BYTES_NODE + st["tri_tests"] * BYTES_TRI
    achieved_gbs = bytes_step / per_launch_s / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    value = lines_all * args.steps / (total_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 geometry / f64 accumulation",
        "data": "synthetic (seeded star mesh, slice queries)",
        "config": _star_config(Q, args.leaf, ws, args.workload),
        "clocks": clocks,
        "e2e": {"value": lines_all * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": Q * 12, "d2h_bytes_per_step": Q * 16},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "l1l2-bytes", "achieved": achieved_gbs, "peak": hbm,
                     "unit": "GB/s", "frac": achieved_gbs / hbm,
                     "traffic": (TRAFFIC_FULL[2] if TRAFFIC_FULL and
                                 (Q, args.leaf) == TRAFFIC_FULL[:2] else None),
                     "kernel": "k_dl_walks",
                     "algorithmic_bytes_per_launch": bytes_step,
                     "bytes_per_unit": {"wide_node": BYTES_NODE, "triangle": BYTES_TRI},
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({which})",
                     "l2_probe_gbs": l2_gbs, "frac_of_l2_probe": achieved_gbs / l2_gbs,
                     "l2_probe": "wob_probe_l2_read: 20 streaming reads (16-byte loads, L1 "
                                 "bypassed) of a 96 MB buffer, L2-resident after a warm-up "
                                 "call; median of 5 calls",
                     "issue_active": ISSUE_PROFILE[0] if ISSUE_PROFILE else None,
                     "lanes_per_inst": ISSUE_PROFILE[1] if ISSUE_PROFILE else None,
                     "alu": {"achieved": achieved_ops, "peak": alu_peak, "unit": "T lane-ops/s",
                             "frac": achieved_ops / alu_peak,
                             "peak_source": f"152 SMs x 128 FP32/INT32 lanes x {sm_max:.0f} MHz "
                                            f"({which} sm_max_mhz)"}},
        "per_line": {"nodes": st["node_visits"] / lines, "tris": st["tri_tests"] / lines,
                     "hits": st["hits"] / lines, "flagged": st["flagged"] / lines},
    }
    if ws == 1 and not args.no_cpu_baseline:  # the oracle's host timing: N = 1 only
        line["cpu_baseline"] = cpu_baseline(v, f, q, args.cpu_queries)
    if dist:
        dist.destroy_process_group()
    if ws == 1 and not args.no_rmse and args.workload == "star":
        line["time_to_rmse"] = _time_to_rmse_summary(args)
    return line


def _time_to_rmse_summary(args) -> dict:
    """The second half of the metric, measured in the default run: the
    learned control variate's time to RMSE 1e-3 on the fifth configuration
    (icosphere L3, g = x^2 - y^2 + 0.5 z, 65,536 queries), beside plain WoB
    at its best path length (projected from measured seconds per walk,
    per-walk variance and truncation bias, with a bounded direct run to
    check the model).  The full record is `--workload cv`."""
    import copy
    a = copy.copy(args)
    a.warmup, a.plain_cap, a.cv_mc = 1, args.rmse_plain_cap, 0
    r = run_cv(a)
    return {"metric": r["metric"], "unit": "s", "higher_is_better": False,
            "workload": r["config"]["workload"],
            "cv": {"time_to_rmse_s": r["cv"]["solve_s"], "measured": True,
                   "train_s": r["cv"]["train_s"], "walks": r["cv"]["walks"],
                   "rmse": r["cv"]["rmse"], "residual_len": r["config"]["cv_len"]},
            "plain_best": {"M": r["best_plain"]["M"],
                           "time_to_rmse_s": r["best_plain"]["time_to_rmse_s"],
                           "projected": True, "direct_check": r["best_plain"]["direct_check"]},
            "speedup_solve": r["speedup_solve"],
            "speedup_incl_training": r["speedup_incl_training"],
            "clocks": r["clocks"], "gpu_launches": r["gpu_launches"]}


def run_batched(args):
    """Secondary workload: 512 independent Dirichlet problems (seeded stars
    and tori of 500-50,000 triangles, 64-16,384 queries each, 256 walks,
    path length 8-24) as one graph-captured launch with an autotuned
    schedule.  A step is one graph replay."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    from paper_2305_04403_gb300 import inputs as I
    torch.cuda.set_device(0)
    items = I.batch_workload(args.problems)
    keep, probs = [], []
    for i, it in enumerate(items):
        mesh = wob.build_mesh(it.verts, it.tris)
        bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
        keep.append((mesh, bvh))
        probs.append(wob.Problem(bvh, kind=wob.DIRICHLET_DL, side=1, data_mode=wob.DATA_POINT,
                                 x0=X0, problem=i))
    t0 = time.perf_counter()
    b = wob.Batch(probs, [it.queries for it in items], 256, [it.max_len for it in items])
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    info = b.info()
    for _ in range(args.warmup):
        b.run(seed=SEED)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            b.run(seed=SEED)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    lines = info["max_lines"]
    T = sum(len(it.tris) for it in items)
    return {
        "metric": METRIC, "value": lines * args.steps / (total_ms / 1e3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 geometry / f64 accumulation",
        "data": "synthetic (seeded stars and tori)",
        "config": {"workload": f"{len(items)} independent Dirichlet problems in one "
                               f"graph-captured launch, {T} triangles, {info['queries']} "
                               f"queries, 256 walks, M 8-24",
                   "walks": info["walks"], "path_vertices": lines,
                   "schedule": {"tile_rounds": info["tile_rounds"], "order": info["order"],
                                "from_cache": info["from_cache"],
                                "tune_ms": info["tune_ms"]},
                   "create_s": create_s, "l2": "flushed (512 MB write) between timed steps"},
        "clocks": clk.summary(), "gpu_launches": 3 * args.steps,
    }


def run_sl(args):
    """Third configuration: single-layer walks with area sampling (Sec. 4.3,
    Table 1) on a seeded displaced torus (R = 1, tube 0.35, 500 x 200 quads =
    200,000 triangles): an interior Neumann problem with data dh/dn of
    h = 1/|x - (0, 0, 5)| and an exterior Robin problem (alpha = 2) with
    h = 1/|x - (1, 0, 0.05)| (x0 inside the solid torus, so h is harmonic
    outside it); 131,072 queries each, half on the boundary (area-uniform,
    with their triangles) and half off it (inside resp. outside the torus),
    512 walks, M = 24.  A step is both solves; a path vertex is one area
    sample (Q x N x M per solve: a walk stops early only on an exact
    coincidence of two points)."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    from paper_2305_04403_gb300 import inputs as I
    torch.cuda.set_device(0)
    v, f, shape = I.displaced_torus()
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    Q, N, M = args.sl_queries, 512, 24
    half = Q // 2
    probs, qs, prs = [], [], []
    for k, (kind, side, alpha, x0, inside) in enumerate(
            [(wob.NEUMANN_SL, 1, 0.0, (0.0, 0.0, 5.0), True),
             (wob.ROBIN_SL, -1, 2.0, (1.0, 0.0, 0.05), False)]):
        pb, prim = I.boundary_points(v, f, half, seed=10 + k)
        off = I.torus_queries(shape, Q - half, inside, seed=20 + k)
        q = np.concatenate([pb, off]).astype(np.float32)
        pr = np.concatenate([prim, np.full(Q - half, -1, np.int32)])
        probs.append(wob.Problem(bvh, kind=kind, side=side, alpha=alpha,
                                 data_mode=wob.DATA_POINT, x0=x0, problem=k, ris=args.sl_ris))
        qs.append(torch.from_numpy(q).cuda())
        prs.append(torch.from_numpy(pr).cuda())
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        for prob, q, pr in zip(probs, qs, prs):
            wob.solve(prob, q, N, M, seed=SEED, query_prim=pr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    verts = 2 * Q * N * M
    return {
        "metric": METRIC, "value": verts * args.steps / (total_ms / 1e3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32 + compensated f32 (float-float) / f64 accumulation" if args.sl_ris <= 1
                  else "f32 geometry / f64 walk arithmetic"),
        "data": "synthetic (seeded displaced torus, seeded queries)",
        "config": {"workload": f"displaced torus ({len(f)} tris), single layer, "
                               f"{'area sampling' if args.sl_ris <= 1 else f'RIS ({args.sl_ris} candidates)'}: "
                               f"interior Neumann + exterior Robin (alpha 2), {Q} queries each "
                               f"(half on the boundary), {N} walks, M = {M}",
                   "path_vertices_per_step": verts,
                   "l2": "flushed (512 MB write) between timed steps"},
        "clocks": clk.summary(), "gpu_launches": 4 * args.steps,
    }


def run_nd(args):
    """Neumann problem through the paper's direct boundary integral equation
    (Sec. 4.2) on the third configuration's torus: interior, data dh/dn of
    h = 1/|x - (0, 0, 5)|, 131,072 queries (half on the boundary, half
    inside), 512 walks, M = 24.  Every vertex takes one line query (all
    hits, 8-wide BVH) and one area sample for the G q source; from inside a
    closed surface every line hits, so a walk has exactly M line queries.
    A step is one solve; a path vertex is one line query."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    from paper_2305_04403_gb300 import inputs as I
    torch.cuda.set_device(0)
    v, f, shape = I.displaced_torus()
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    Q, N, M = args.sl_queries, 512, 24
    half = Q // 2
    pb, prim = I.boundary_points(v, f, half, seed=10)
    off = I.torus_queries(shape, Q - half, True, seed=20)
    q = torch.from_numpy(np.concatenate([pb, off]).astype(np.float32)).cuda()
    pr = torch.from_numpy(np.concatenate([prim, np.full(Q - half, -1, np.int32)])).cuda()
    prob = wob.Problem(bvh, kind=wob.NEUMANN_DIRECT, side=1, data_mode=wob.DATA_POINT,
                       x0=(0.0, 0.0, 5.0))
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        wob.solve(prob, q, N, M, seed=SEED, query_prim=pr)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            wob.solve(prob, q, N, M, seed=SEED, query_prim=pr)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    lines = (Q - half) * N * M + half * N * (M - 1)
    return {
        "metric": METRIC, "value": lines * args.steps / (total_ms / 1e3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 geometry / f64 walk arithmetic",
        "data": "synthetic (seeded displaced torus, seeded queries)",
        "config": {"workload": f"displaced torus ({len(f)} tris), interior Neumann through the "
                               f"direct boundary integral equation, {Q} queries (half on the "
                               f"boundary), {N} walks, M = {M}",
                   "line_queries_per_step": lines, "area_samples_per_step": Q * N * M + (Q - half) * N,
                   "l2": "flushed (512 MB write) between timed steps"},
        "clocks": clk.summary(), "gpu_launches": 2 * args.steps,
    }


def run_grad(args):
    """The default workload (star L6 slice, 1,024 walks, M = 16) through
    wob_solve_grad: value and gradient from the same walks (Sec. 4.1.3).  A
    step is one solve; a path vertex is one line query (the same count as
    the default workload, from the counting walks)."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    torch.cuda.set_device(0)
    v, f, q = _workload()
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    prob = wob.Problem(bvh, kind=wob.DIRICHLET_DL, side=1, data_mode=wob.DATA_POINT, x0=X0)
    qd = torch.from_numpy(q).cuda()
    _, _, st = wob.solve_counted(prob, qd, WALKS, MAX_LEN, seed=SEED)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        wob.solve_grad(prob, qd, WALKS, MAX_LEN, seed=SEED)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            wob.solve_grad(prob, qd, WALKS, MAX_LEN, seed=SEED)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    return {
        "metric": METRIC, "value": st["lines"] * args.steps / (total_ms / 1e3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 geometry / f64 accumulation",
        "data": "synthetic (seeded star mesh, slice queries)",
        "config": {"workload": f"star-shaped icosphere L6, z=0 slice Q={len(q)}, {WALKS} walks, "
                               f"M={MAX_LEN}: value + gradient from the same walks",
                   "l2": "flushed (512 MB write) between timed steps"},
        "clocks": clk.summary(), "gpu_launches": 5 * args.steps,
    }


def run_mixed(args):
    """Mixed boundary conditions (Sec. 4.3) with the paper's settings: every
    triangle of the 200,000-triangle displaced torus takes a Dirichlet,
    Neumann or Robin (alpha = 1) condition at random (seed 0), k = 4,
    p_k = 2/3, next points by resampled importance sampling from 16 uniform
    candidates, M = 4; data from h = 1/|x - (0, 0, 5)|; 131,072 queries inside
    the torus, 512 walks.  A path vertex is one vertex of a walk (a picked
    point or a stay)."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    from paper_2305_04403_gb300 import inputs as I
    torch.cuda.set_device(0)
    v, f, shape = I.displaced_torus()
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    Q, N, M = args.sl_queries, 512, 4
    q = torch.from_numpy(I.torus_queries(shape, Q, True, seed=20)).cuda()
    bc = torch.from_numpy(np.random.default_rng(0).integers(0, 3, len(f)).astype(np.uint8)).cuda()
    prob = wob.Problem(bvh, kind=wob.MIXED_SL, side=1, alpha=1.0, data_mode=wob.DATA_POINT,
                       x0=(0.0, 0.0, 5.0), bc_type=bc, k_mix=4.0, p_k=2.0 / 3.0, ris=16)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        wob.solve(prob, q, N, M, seed=SEED)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            wob.solve(prob, q, N, M, seed=SEED)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    verts = Q * N * M
    return {
        "metric": METRIC, "value": verts * args.steps / (total_ms / 1e3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 geometry / f64 walk arithmetic",
        "data": "synthetic (seeded displaced torus, seeded conditions and queries)",
        "config": {"workload": f"displaced torus ({len(f)} tris), mixed Dirichlet / Neumann / "
                               f"Robin conditions at random, k = 4, p_k = 2/3, RIS with 16 "
                               f"candidates, {Q} interior queries, {N} walks, M = {M}",
                   "path_vertices_per_step": verts, "area_samples_per_step": 16 * verts,
                   "l2": "flushed (512 MB write) between timed steps"},
        "clocks": clk.summary(), "gpu_launches": 2 * args.steps,
    }


def run_fwd(args):
    """Forward (adjoint) single-layer estimator for an interior Neumann
    problem with sparse data (Sec. 4.4.3 and the Neumann example of Sec. 5):
    the 200,000-triangle displaced torus, P1 data zero except for six signed
    Gaussian bumps (width 0.05, integrating to zero), 131,072 queries inside
    the torus, 65,536 paths of M = 24 vertices that start where |q| is large
    (boundary-value-weighted, beta = 0.1), every vertex connected to every
    query.  A step is one wob_solve_forward call; the unit is one
    (path vertex, query) connection.  Beside it, untimed: the same call with
    area-uniform starts and the backward single-layer walks (512 per query),
    compared by variance x time."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    from paper_2305_04403_gb300 import inputs as I
    torch.cuda.set_device(0)
    v, f, shape = I.displaced_torus()
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    Q, P, M, N = args.sl_queries, args.fwd_paths, 24, 512
    q = torch.from_numpy(I.torus_queries(shape, Q, True, seed=20)).cuda()
    vd = torch.from_numpy(I.bump_data(v, f)).cuda()
    prob = wob.Problem(bvh, kind=wob.NEUMANN_SL, side=1, data_mode=wob.DATA_VERTEX_P1,
                       vertex_data=vd)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    no_q = torch.empty((0, 3), dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        out, ms = None, []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return out, float(np.median(ms))

    fwd = lambda mode, qq=q: wob.solve_forward(prob, qq, P, M, seed=SEED, start_mode=mode, beta=0.1)
    for _ in range(args.warmup):
        fwd(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            out_w = fwd(1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(c) for a, c in ev)
    t_w = total_ms / args.steps
    _, t_paths = timed(lambda: fwd(1, no_q), 3)
    out_u, t_u = timed(lambda: fwd(0), 2)
    (est_b, var_b), t_b = timed(lambda: wob.solve(prob, q, N, M, seed=SEED), 2)
    ew, vw = out_w["est"].cpu().numpy(), out_w["var"].cpu().numpy() / P
    eu, vu = out_u["est"].cpu().numpy(), out_u["var"].cpu().numpy() / P
    eb, vb = est_b.cpu().numpy(), var_b.cpu().numpy() / N
    z = np.abs(ew - eb) / np.sqrt(vw + vb)
    pairs = P * M * Q
    t_conn = max(t_w - t_paths, 1e-6)
    sm = clk.summary()
    sm_max = sm.get("sm_max_mhz") or 2070.0
    peak = 152 * 16 * sm_max * 1e6 / 1e9          # G pairs/s: one MUFU rsqrt per pair
    achieved = pairs / (t_conn / 1e3) / 1e9
    return {
        "metric": METRIC + " (forward estimator: vertex-query connections)",
        "value": pairs * args.steps / (total_ms / 1e3), "unit": "connections/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_w,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 geometry and connections / f64 path weights and sums",
        "data": "synthetic (seeded displaced torus, six seeded bumps, seeded queries)",
        "config": {"workload": f"displaced torus ({len(f)} tris), interior Neumann, sparse data "
                               f"(6 bumps), forward single-layer paths with boundary-value-weighted "
                               f"starts: {P} paths x M = {M} connected to {Q} interior queries",
                   "path_vertices_per_step": P * M, "connections_per_step": pairs,
                   "paths_only_ms": t_paths,
                   "l2": "flushed (512 MB write) between timed steps"},
        "compare": {
            "ms": {"forward_weighted": t_w, "forward_uniform": t_u, f"backward_{N}_walks": t_b},
            "median_var_of_estimate": {"forward_weighted": float(np.median(vw)),
                                       "forward_uniform": float(np.median(vu)),
                                       f"backward_{N}_walks": float(np.median(vb))},
            "median_var_x_time_gain_vs_backward": {
                "forward_weighted": float(np.median(vb * t_b / (vw * t_w))),
                "forward_uniform": float(np.median(vb * t_b / (vu * t_u)))},
            "agreement_forward_vs_backward": {"frac_within_4_sigma": float((z <= 4).mean()),
                                              "median_z": float(np.median(z))}},
        "clocks": sm, "gpu_launches": (4 + 2) * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G pairs/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_fwd_connect",
                     "peak_source": f"152 SMs x 16 MUFU rsqrt/clk x {sm_max:.0f} MHz; connection "
                                    f"time = step - the same call with no queries"},
    }


def run_cv(args):
    """Learned control variate vs plain WoB: time to RMSE 1e-3 against the
    exact solution on the icosphere-L3 mesh (1,280 triangles) with
    g = x^2 - y^2 + 0.5 z evaluated at the hits (the polyhedral problem's
    exact solution is then the polynomial itself), 65,536 queries uniform in
    the ball of radius 0.9 (seed 1).

    CV: the network is initialised on the device (seed 2) and trained by
    wob_cv_train on 1M area-uniform boundary points (seed 3) with targets
    from 64 density walks of length 4; then residual walks of length
    --cv-len are added in batches of --cv-batch walks until the RMSE of
    D nu_t + mean(residual walks) is <= 1e-3 (measured, CUDA events; the
    RMSE check after each batch is inside the timed region).  Training
    time is reported separately.

    Plain WoB, M in {4, 5, 6, 8}: reaching 1e-3 takes 10^6-10^7 walks per
    query (minutes to an hour), so the time is projected from measured
    quantities: walks per second and mean per-walk variance sigma^2 on all
    queries (512 walks), and the squared truncation bias b^2 estimated on
    the first 256 queries with --bias-walks walks (mean squared error minus
    the noise term).  RMSE(N)^2 = b^2 + sigma^2 / N gives the walks needed.
    The best M is then run directly for --plain-cap seconds and its RMSE
    compared with the projection."""
    import torch
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    from paper_2305_04403_gb300 import inputs as I
    torch.cuda.set_device(0)
    target = 1e-3
    v, f = I.icosphere(3)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=args.leaf)
    prob = wob.Problem(bvh, kind=wob.DIRICHLET_DL, side=1, data_mode=wob.DATA_POLY,
                       poly=I.POLY_CONFIG1, problem=0)
    Q = args.cv_queries
    qh = I.ball_queries(Q, 0.9, 1)
    q = torch.from_numpy(qh).cuda()
    exact = torch.from_numpy(I.poly_eval(I.POLY_CONFIG1, qh.astype(np.float64))).cuda()
    stream = torch.cuda.current_stream()

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def rmse(est):
        return float(torch.sqrt(torch.mean((est - exact) ** 2)).item())

    def lap(start):
        e = ev()
        e.synchronize()
        return start.elapsed_time(e) / 1e3

    cvo = wob.ControlVariate(mesh, level=2, near=2.0)
    launches = 0
    # warm-up at the timed sizes: kernels loaded, memory pools grown
    for _ in range(args.warmup):
        p = wob.mlp_init(2)
        m, vv = torch.zeros_like(p), torch.zeros_like(p)
        cvo.train(prob, p, m, vv, points=1 << 20, walks=64, max_len=4, epochs=1)
        s_ = torch.zeros(Q, dtype=torch.float64, device="cuda")
        d_ = torch.empty(Q, dtype=torch.float32, device="cuda")
        cvo.solve_range(prob, p, q, 0, args.cv_batch, args.cv_len, s_, torch.zeros_like(s_),
                        dnt=d_)
        rmse(d_.double() + s_ / args.cv_batch)
        if args.cv_mc:
            wob.cv_solve_mc(prob, p, q, 0, args.cv_batch, args.cv_len, args.cv_mc, s_,
                            torch.zeros_like(s_))
        wob.solve_range(prob, q, 0, 512, 4, s_, torch.zeros_like(s_))
        rmse(s_ / 512)
        lap(ev())
    torch.cuda.synchronize()

    with Clocks(0) as clk:
        # ---- CV: train, then progressive residual walks
        p = wob.mlp_init(2)
        m, vv = torch.zeros_like(p), torch.zeros_like(p)
        steps_per_epoch = -(-(1 << 20) // 4096)
        t0 = ev()
        loss = cvo.train(prob, p, m, vv, points=1 << 20, walks=64, max_len=4, point_seed=3,
                         walk_seed=0, epochs=args.cv_epochs, batch=4096, lr=1e-3,
                         lr_end=1e-4, tail_epochs=args.cv_tail)
        t1 = ev()
        torch.cuda.synchronize()
        train_s = t0.elapsed_time(t1) / 1e3
        launches += 6 + args.cv_epochs * steps_per_epoch * 3 + 2
        s_ = torch.zeros(Q, dtype=torch.float64, device="cuda")
        ss = torch.zeros_like(s_)
        dnt = torch.empty(Q, dtype=torch.float32, device="cuda")
        curve, n_cv = [], 0
        t0 = ev()
        while True:
            if args.cv_mc:   # Monte Carlo integrals: D nu_t is inside the walk values
                wob.cv_solve_mc(prob, p, q, n_cv, args.cv_batch, args.cv_len, args.cv_mc, s_, ss,
                                seed=SEED)
                launches += 5 + 4 * args.cv_len
                n_cv += args.cv_batch
                e = rmse(s_ / n_cv)
            else:
                cvo.solve_range(prob, p, q, n_cv, args.cv_batch, args.cv_len, s_, ss, seed=SEED,
                                dnt=dnt if n_cv == 0 else None)
                launches += 2 + 3 * args.cv_len + (1 if n_cv == 0 else 0)
                n_cv += args.cv_batch
                e = rmse(dnt.double() + s_ / n_cv)
            curve.append([lap(t0), n_cv, e])
            if e <= target or n_cv >= args.cv_max_walks:
                break
        cv_s = curve[-1][0]
        cv_var = float(((ss - s_ * s_ / n_cv) / (n_cv - 1)).mean().item())
        cv_projection = None
        if curve[-1][2] > target:  # cap reached: project as for plain WoB
            b2 = max(curve[-1][2] ** 2 - cv_var / n_cv, 0.0)
            need = cv_var / (target ** 2 - b2) if b2 < target ** 2 else None
            cv_projection = {"bias2_estimate": b2, "walks_needed": need,
                             "time_to_rmse_s": cv_s * need / n_cv if need else None}

        # ---- plain WoB: rate and variance on all queries, bias on a subset
        plain = {}
        nb = 256
        for M in (4, 5, 6, 8):
            s_.zero_()
            ss.zero_()
            a = ev()
            wob.solve_range(prob, q, 0, 512, M, s_, ss, seed=SEED)
            b = ev()
            torch.cuda.synchronize()
            t_walk = a.elapsed_time(b) / 1e3 / 512          # seconds per walk of every query
            var = float(((ss - s_ * s_ / 512) / 511).mean().item())
            sb = torch.zeros(nb, dtype=torch.float64, device="cuda")
            sbb = torch.zeros_like(sb)
            chunk = 1 << 18
            for k in range(args.bias_walks // chunk):
                wob.solve_range(prob, q[:nb], k * chunk, chunk, M, sb, sbb, seed=SEED + 1)
            nbw = (args.bias_walks // chunk) * chunk
            mse = float(torch.mean((sb / nbw - exact[:nb]) ** 2).item())
            vb = float(((sbb - sb * sb / nbw) / (nbw - 1)).mean().item())
            bias2 = mse - vb / nbw
            launches += 2 + 2 * (args.bias_walks // chunk)
            need = var / (target ** 2 - bias2) if bias2 < target ** 2 else None
            plain[str(M)] = {"seconds_per_walk": t_walk, "per_walk_var": var,
                             "bias_rms": float(np.sqrt(max(bias2, 0.0))),
                             "bias2_estimate": bias2, "bias_walks": nbw,
                             "walks_needed": need,
                             "time_to_rmse_s": need * t_walk if need else None}
        ok = {k: r for k, r in plain.items() if r["time_to_rmse_s"]}
        best = min(ok, key=lambda k: ok[k]["time_to_rmse_s"])
        # direct run of the best M for a bounded time: RMSE vs the model
        Mb = int(best)
        s_.zero_()
        ss.zero_()
        n_pl, chunk = 0, 2048
        t0 = ev()
        while True:
            wob.solve_range(prob, q, n_pl, chunk, Mb, s_, ss, seed=SEED + 2)
            n_pl += chunk
            launches += 2
            el = lap(t0)
            if el >= args.plain_cap:
                break
        e_pl = rmse(s_ / n_pl)
        pred = float(np.sqrt(max(plain[best]["bias2_estimate"], 0.0)
                             + plain[best]["per_walk_var"] / n_pl))
        torch.cuda.synchronize()

    best_t = plain[best]["time_to_rmse_s"]
    return {
        "metric": "time-to-RMSE 1e-3, learned control variate vs plain WoB",
        "value": cv_s, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * cv_s, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 network / f32 quadrature / f64 accumulation",
        "data": "synthetic (icosphere, seeded ball queries)",
        "config": {"workload": "icosphere L3 (1,280 tris), g = x^2 - y^2 + 0.5 z at the hits, "
                               f"Q = {Q} in the r <= 0.9 ball; CV trained on 1M boundary "
                               "densities (64 walks, M = 4)",
                   "cv_len": args.cv_len, "cv_batch": args.cv_batch,
                   "cv_epochs": args.cv_epochs, "cv_lr": f"1e-3, last {args.cv_tail} epochs 1e-4",
                   "quadrature": ("none: D nu_t and H nu_t from %d extra all-hits lines per "
                                  "point (Monte Carlo)" % args.cv_mc) if args.cv_mc else
                                 "Radon 7-point, level-2 near field within 2 edge lengths"},
        "cv": {"train_s": train_s, "solve_s": cv_s, "walks": n_cv, "rmse": curve[-1][2],
               "per_walk_var": cv_var, "final_train_loss": float(loss[-1].mean().item()),
               "curve": curve, "projection_if_capped": cv_projection},
        "plain": plain,
        "best_plain": {"M": Mb, "time_to_rmse_s": best_t, "projected": True,
                       "direct_check": {"walks": n_pl, "seconds": el, "rmse": e_pl,
                                        "model_rmse": pred}},
        "speedup_solve": best_t / cv_s, "speedup_incl_training": best_t / (cv_s + train_s),
        "clocks": clk.summary(), "gpu_launches": launches,
    }


def cpu_baseline(v, f, q, nq: int) -> dict:
    """The oracle as it stands, on the host cores, on a bounded sample."""
    import oracle as O
    sel = q[:: max(1, len(q) // nq)][:nq]
    t0 = time.perf_counter()
    r = O.dl_walks(v, f, sel, WALKS, MAX_LEN, seed=SEED, mode=O.DATA_POINT, x0=X0,
                   want_lines=True)
    dt = time.perf_counter() - t0
    lines = int((r["line_m"] >= 0).sum())
    return {"value": lines / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{len(sel)} queries x {WALKS} walks x up to {MAX_LEN} vertices "
                      f"({lines} line queries, brute force over 81,920 triangles), {dt:.1f} s"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return None
    import oracle as O
    v, f, q = _workload()
    sel = q[:: max(1, len(q) // args.cpu_queries)][:args.cpu_queries]
    for _ in range(args.warmup):
        O.dl_walks(v, f, sel[:1], 64, MAX_LEN, seed=SEED, mode=O.DATA_POINT, x0=X0)
    t_total, lines_total = 0.0, 0
    for i in range(args.steps):
        t0 = time.perf_counter()
        r = O.dl_walks(v, f, sel, WALKS // 8, MAX_LEN, seed=SEED, mode=O.DATA_POINT, x0=X0,
                       walk_begin=i * (WALKS // 8), want_lines=True)
        t_total += time.perf_counter() - t0
        lines_total += int((r["line_m"] >= 0).sum())
    value = lines_total / t_total
    sample = (f"{len(sel)} of the {len(q)} queries x {WALKS // 8} walks x up to {MAX_LEN} "
              f"vertices per step (step i takes walks {WALKS // 8} i and on), brute force over "
              f"81,920 triangles")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded star mesh, slice queries)",
            "config": _star_config(len(q), args.leaf, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--leaf", type=int, default=1)
    ap.add_argument("--cpu-queries", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--queries", type=int, default=0,
                    help="evenly subsample this many queries (profiling runs; 0 = all)")
    ap.add_argument("--workload", default="star",
                    choices=["star", "spiky", "batched", "cv", "sl", "nd", "grad", "mixed", "fwd"])
    ap.add_argument("--sl-ris", type=int, default=0,
                    help="sl workload: resampling candidates (0 = area sampling)")
    ap.add_argument("--sl-queries", type=int, default=131072)
    ap.add_argument("--fwd-paths", type=int, default=1 << 16, help="fwd workload: paths")
    ap.add_argument("--cv-len", type=int, default=2, help="residual walk length (cv workload)")
    ap.add_argument("--cv-queries", type=int, default=65536,
                    help="queries of the cv workload (the metric is defined at 65,536)")
    ap.add_argument("--cv-batch", type=int, default=64)
    ap.add_argument("--cv-mc", type=int, default=0,
                    help="cv workload: Monte Carlo integrals with this many extra lines per "
                         "point instead of quadrature (0 = quadrature)")
    ap.add_argument("--cv-epochs", type=int, default=23)
    ap.add_argument("--cv-tail", type=int, default=3, help="final epochs at lr 1e-4")
    ap.add_argument("--cv-max-walks", type=int, default=1 << 16)
    ap.add_argument("--bias-walks", type=int, default=1 << 22)
    ap.add_argument("--plain-cap", type=float, default=20.0)
    ap.add_argument("--no-rmse", action="store_true",
                    help="default workload: skip the control variate's time to RMSE 1e-3")
    ap.add_argument("--rmse-plain-cap", type=float, default=8.0,
                    help="default workload: seconds of the direct plain-WoB check run")
    ap.add_argument("--problems", type=int, default=512)
    args = ap.parse_args()
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "batched":
        line = run_batched(args)
    elif args.workload == "cv":
        line = run_cv(args)
    elif args.workload == "sl":
        line = run_sl(args)
    elif args.workload == "nd":
        line = run_nd(args)
    elif args.workload == "grad":
        line = run_grad(args)
    elif args.workload == "mixed":
        line = run_mixed(args)
    elif args.workload == "fwd":
        line = run_fwd(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
