#!/usr/bin/env python3
"""Benchmark of the LBVH hot path: one step = one full build plus one full
range query of the same size, on synthetic inputs already resident in HBM.

Workload (default): 2^25 points uniform in [0,1)^3 (FP32), 63-bit Morton codes;
a build (bounds, Morton codes, the radix sort of the codes' top bits beside the
index in 4 or 5 passes plus the runs of equal top bits, Algorithm 4 construct) and
2^25 sphere queries centred at the points with the radius that holds 16
expected neighbours (Algorithm 1, CSR output with sorted hit lists).

Prints ONE JSON line (rank 0). ``value`` is primitives per second through the
whole step (build + query), whole job, device-timed with CUDA events on the
stream the kernels run on. ``e2e`` is the same metric through the C-ABI calls
from host buffers: each step copies the points and queries from pinned host
memory, builds, and queries with lbvh_query_into_host, which leaves the CSR
result in pinned host memory (chunk copies overlapped with the next chunk's
walk; --e2e-staged: query into device arrays, then copy). ``roofline`` reports the
dominant kernel's algorithmic bytes over its event-timed duration against the
measured HBM copy bandwidth. ``cpu_baseline`` times the CPU oracle on a
bounded sample of the same workload (rank 0, N=1 only).

``--impl reference`` times the CPU oracle itself, as the reference arm.

Multi-GPU: every rank builds and queries its own independent instance (no
data-path collective; replicas only); ``value`` = all ranks' primitives over
the slowest rank's time.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_00665_gb300 import inputs  # noqa: E402

METRIC = "build+query Mprims/s (one LBVH build and n radius queries per step)"
REFIT_METRIC = "refit Mprims/s (new boxes for moved primitives on a kept topology)"
UNIT = "Mprims/s"

# Algorithmic bytes per primitive (or per query) of each stage: the data the
# method itself must move, independent of how a kernel moves it.
#   bounds      read the points                              12
#   encode      read the points, write the 64-bit codes      12 + 8
#   sort pass   read one 8-byte word (key bits above the index), write one 8 + 8
#               (the last pass of a 30-bit sort writes the 4-byte index alone)
#   sort runs   read the sorted words, write the permutation 8 + 4 (codes
#               wider than 30 bits: the runs of equal top bits put in order)
#   construct   key 8 + perm 4 + point 12 read, leaf 16 and internal node 32
#               written (the store words and sibling boxes of the nodes inside
#               a CTA's leaves stay in shared memory)
#   query walk  query 12 read, count 4 written, 4 per hit kept, tree read once (48 B/leaf)
#   query copy  count 4 and offset 8 read per query, 4 per hit read and 4 written
def alg_bytes(stage: str, n: int, nq: int, hits: int, boxes: bool = False, box_queries: bool = False,
              long_lists: tuple = (0, 0), order_passes: int = 4):
    """Algorithmic bytes of one launch of a stage (the data the method must
    move): pb = bytes of a primitive, lb = of a leaf record, qb = of a query;
    long_lists = (queries with more hits than the walk keeps, their hits);
    order_passes = sort passes of the query order (4 for 30-bit order codes,
    3 for 24-bit ones, the tuner's choice)."""
    knn = box_queries == "knn"
    qb = 32 if box_queries == "ray" else (24 if box_queries and not knn else 12)
    pb, lb = (24, 32) if boxes else (12, 16)
    table = {
        "bounds": pb * n,
        "encode": (pb + 8) * n,
        **{f"sort_pass{k}": 16 * n for k in range(8)},
        "sort_runs": 12 * n,
        # codes, perm, primitive read; leaf + internal node write
        "construct": (8 + 4 + pb + lb + 32) * n,
        # query + count per query, each kept hit, the tree once
        # (kNN: the query, index and squared distance of each neighbour, the tree once)
        "query_walk": (qb * nq + 8 * hits if knn else (qb + 4) * nq + 4 * hits) + (32 + lb) * n,
        "query_order": (qb + 4 + order_passes * 16) * nq,  # order codes packed with the index
        "query_scan": 4 * nq + 8 * (nq + 1),
        "query_copy": 12 * nq + 8 * hits,
        # the second walk of the long lists: query + offsets, hits written, then sorted in place
        "query_overflow": (qb + 16) * long_lists[0] + 12 * long_lists[1],
    }
    return table.get(stage)

def model_build_bytes(n: int, bits: int, boxes: bool = False) -> int:
    """Algorithmic bytes of a whole build in the reference model of the path:
    bounds read the primitives; encode reads them and writes 8-byte codes;
    the sort reads 8 B for the global histogram and moves 12 B in and 12 B
    out per pass (8-bit digits); the construct reads code, permutation and
    primitive, writes the leaf's skip and box and the internal node, touches
    one 8-byte store word and re-reads a sibling box (24 B). Points: 144 + 24
    per pass = 336 B/prim at 63 bits (8 passes); boxes read and write 24-byte
    primitives and 32-byte leaves instead."""
    passes = (bits + 7) // 8
    per = (200 if boxes else 144) + 24 * passes
    return per * n


def moved_build_bytes(n: int, bits: int, boxes: bool = False, passes: int | None = None) -> int:
    """Bytes this implementation's build kernels read and write, counted
    from their layouts (each element once): bounds and encode stream the
    primitives, the encoder writes one 8-byte word; codes of at most 30 bits
    are sorted as code << 32 | index words (the last pass writes the 4-byte
    permutation alone); wider codes as top bits << ib | index words, ib =
    ceil(log2 n), over bytes ib // 8 .. 7 (or one byte fewer, the tuner's
    choice: `passes` is the number of passes that ran), then one pass reads
    the sorted words and writes the permutation (the runs of equal sorted
    bits gather their primitives again: not counted); the construct reads
    the permutation and gathers each primitive, writes the sorted code, the
    leaf and the internal node."""
    pb, lb = (24, 32) if boxes else (12, 16)
    if bits <= 30:
        passes = (bits + 7) // 8
        sort = 16 * (passes - 1) + 12
    else:
        ib = max(1, (n - 1).bit_length())
        sort = 16 * (passes if passes is not None else 8 - ib // 8) + 12
    return (pb + (pb + 8) + sort + (4 + pb + 8 + lb + 32)) * n


BATCH_WORKLOADS = {
    # name: (description, clouds, min size, max size, seed, Morton bits)
    "batched_4096_clouds": ("4,096 independent FP32 point clouds, sizes floor(exp(U(ln 256, ln 262144))) "
                            "(seed 1), uniform in [0,1)^3; each built (30-bit codes) and queried with its own "
                            "points at the radius for 16 expected neighbours of its size; all in one CUDA-graph "
                            "launch vs a loop of single builds", 4096, 256, 262144, 1, 30),
    "batched_256_clouds": ("256 clouds, sizes log-uniform in [256, 262144] (seed 1), as batched_4096_clouds "
                           "(short case)", 256, 256, 262144, 1, 30),
}

SERVED_WORKLOADS = {
    # name: (description, requests, rate per s, min size, max size, seed, Morton bits, budget bytes)
    "served_poisson_2000": ("Poisson stream at 2,000 requests/s; each request builds a tree of its own "
                            "FP32 point cloud (sizes log-uniform in [1,024, 4,194,304]; uniform or "
                            "64-component Gaussian mixture, alternating at random) with 63-bit codes and "
                            "answers one ~16-neighbour sphere query per point; trees stay resident under a "
                            "60 GB HBM budget with LRU eviction; served with continuous batching vs "
                            "one-at-a-time processing of the same arrivals", 400, 2000.0, 1024, 4194304, 2, 63,
                            60 << 30),
    "served_saturated_400": ("the 400 requests of served_poisson_2000 offered all at once (every arrival at "
                             "t = 0): the load exceeds capacity, so both arms run at their highest sustained "
                             "throughput", 400, float("inf"), 1024, 4194304, 2, 63, 60 << 30),
    "served_poisson_short": ("as served_poisson_2000 with 60 requests (short case)", 60, 2000.0, 1024, 4194304,
                             2, 63, 60 << 30),
    "served_poisson_2000_budget4gb": ("as served_poisson_2000 under a 4 GB HBM budget: the resident trees do not "
                                      "all fit, so admission evicts the least recently used ones while requests "
                                      "arrive", 400, 2000.0, 1024, 4194304, 2, 63, 4 << 30),
}

WORKLOADS = {
    # name: (description, n, bits, kind, generator)
    "uniform_2^25_63bit": ("2^25 FP32 points uniform in [0,1)^3, 63-bit Morton codes; build + 2^25 sphere "
                           "queries at the points, radius for 16 expected neighbours", 1 << 25, 63),
    "uniform_2^24_63bit": ("2^24 FP32 points uniform in [0,1)^3, 63-bit Morton codes; build + 2^24 sphere "
                           "queries at the points, radius for 16 expected neighbours (profiling case)", 1 << 24, 63),
    "uniform_16384_30bit": ("16,384 FP32 points uniform in [0,1)^3 (seed 0), 30-bit codes; build + 16,384 "
                            "sphere queries at the points, radius for 16 expected neighbours", 16384, 30),
    "refit_uniform_2^25_63bit": ("refit of a 2^25-point tree (63-bit codes, built once from uniform points in "
                                 "[0,1)^3) to moved points: every step gives the tree new coordinates (the points "
                                 "plus N(0, 0.001) jitter, two alternating sets) and recomputes all boxes on the "
                                 "kept topology", 1 << 25, 63, "refit"),
    "construction_rates": ("construction rate vs n of the three hierarchy algorithms the paper compares "
                           "(Algorithm 4, Karras, Algorithm 3 + a skip pass) on its two synthetic clouds: filled "
                           "cube (uniform in [-a,a]^3) and hollow cube (uniform on the six faces in turn), "
                           "a = n^(1/3), 63-bit codes, n = 2^12 .. 2^25; median device time of 10 builds each",
                           1 << 25, 63, "curves"),
    "rays_mixture_boxes_2^25_63bit": ("2^25 FP32 boxes from the 64-component Gaussian mixture of "
                                      "mixture_boxes_2^25_63bit (63-bit codes); build + 2^22 ray-segment queries "
                                      "(origins uniform in [0,1)^3, directions uniform on the sphere, t in "
                                      "[0, 0.05]), walked in input order", 1 << 25, 63, "rays"),
    "mixture_boxes_2^25_63bit": ("2^25 FP32 boxes, centres from a 64-component Gaussian mixture (sigma 0.005, "
                                 "component centres uniform in [0,1)^3), half-extents lognormal(ln 1e-4, 0.5); "
                                 "63-bit codes; build + 2^24 box-overlap queries from the same mixture",
                                 1 << 25, 63, "mixture_boxes"),
    "mixture_boxes_2^25_30bit": ("as mixture_boxes_2^25_63bit with 30-bit codes: most centres of a component "
                                 "share a code, so the index tie-break decides much of the tree",
                                 1 << 25, 30, "mixture_boxes"),
    "knn_uniform_2^25_63bit": ("2^25 FP32 points uniform in [0,1)^3, 63-bit Morton codes; build + the 16 "
                               "nearest neighbours of every point (lbvh_knn: Algorithm 1 with a shrinking ball)",
                               1 << 25, 63, "knn"),
    "knn_uniform_2^24_63bit": ("as knn_uniform_2^25_63bit with 2^24 points (profiling case)", 1 << 24, 63, "knn"),
    "mixture_boxes_2^23_63bit": ("as mixture_boxes_2^25_63bit with 2^23 boxes and 2^22 queries (profiling case)",
                                 1 << 23, 63, "mixture_boxes"),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lbvh", "reference"], default="lbvh")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(SERVED_WORKLOADS),
                    default="uniform_2^25_63bit")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-staged", action="store_true",
                    help="e2e results into device arrays, then copied to host (instead of lbvh_query_into_host)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--server-slots", type=int, default=2,
                    help="worker slots of the request server (served workloads): batches in flight at once")
    ap.add_argument("--tuning", default=None, metavar="SORT,WALK",
                    help="fix the sort and walk variants instead of running the autotuner (profiling runs: "
                         "no trial launches before the measured ones)")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed


def dist_setup(use_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid and len({r[0] for r in rows} | {parts[0]}) > 1:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- workload


def workload_family(workload: str) -> str:
    w = WORKLOADS[workload]
    return w[3] if len(w) > 3 else "uniform"


def make_inputs(workload: str, seed: int):
    """(description, n, bits, prims, queries or None (= the prims), boxes?, box queries?, radius)."""
    desc, n, bits = WORKLOADS[workload][:3]
    if workload_family(workload) == "rays":
        prims = inputs.gaussian_mixture_boxes(n, seed=seed)
        return desc, n, bits, prims, inputs.random_rays(n // 8, seed=seed + 1, tmax=0.05), True, "ray", 0.0
    if workload_family(workload) == "mixture_boxes":
        prims = inputs.gaussian_mixture_boxes(n, seed=seed)
        queries = inputs.gaussian_mixture_boxes(n // 2, seed=seed + 1, component_seed=seed)
        return desc, n, bits, prims, queries, True, True, 0.0
    pts = inputs.uniform_points(n, seed=seed)
    if workload_family(workload) == "knn":
        return desc, n, bits, pts, None, False, "knn", 0.0
    r = inputs.radius_for_neighbours(n)
    return desc, n, bits, pts, None, False, False, r


def measured_hbm_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_for(stage: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since the capture; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        table = json.load(f)
    e = table.get(stage)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2402_00665_gb300", "csrc", e["source"])
    if not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if sha != e.get("source_sha"):
        return None
    return e.get("bytes_per_launch_full")


# ---------------------------------------------------------------- oracle timing


# One bounded sample of the workload for the CPU oracle, the same for the
# reference arm (one sample per step) and the cpu_baseline leg (the median of
# CPU_BASELINE_SAMPLES samples): a full build of 2^22 primitives and 2^17 of
# its queries (about 2-3 s of one core), or the whole workload when it is
# smaller.
ORACLE_N, ORACLE_Q = 1 << 22, 1 << 17
CPU_BASELINE_SAMPLES = 5


def oracle_sample(seed: int, n_sample: int = ORACLE_N, q_sample: int = ORACLE_Q, bits: int = 63,
                  family: str = "uniform"):
    """The CPU oracle on a bounded sample of the same workload: a full build of
    n_sample primitives and q_sample of its queries (uniform points with radius
    queries for 16 neighbours at that size, or mixture boxes with box queries
    from the same mixture). Returns (prims/s, description)."""
    import oracle
    if family == "rays":
        prims = inputs.gaussian_mixture_boxes(n_sample, seed=seed + 101)
        q = inputs.random_rays(q_sample, seed=seed + 102, tmax=0.05)
        kind, qkind, r, what = oracle.BOXES, oracle.RAY, 0.0, "Gaussian-mixture boxes"
        qwhat = "ray-segment queries (t in [0, 0.05])"
    elif family == "mixture_boxes":
        prims = inputs.gaussian_mixture_boxes(n_sample, seed=seed + 101)
        q = inputs.gaussian_mixture_boxes(q_sample, seed=seed + 102, component_seed=seed + 101)
        kind, qkind, r, what = oracle.BOXES, oracle.BOX, 0.0, "Gaussian-mixture boxes", 
        qwhat = "box-overlap queries from the same mixture"
    elif family == "knn":
        prims = inputs.uniform_points(n_sample, seed=seed + 101)
        q_sample = min(q_sample, 64)  # brute force: every primitive per query
        q = prims[:q_sample]
        kind, qkind, r, what = oracle.POINTS, None, 0.0, "uniform points"
        qwhat = "16-nearest-neighbour queries at its points (brute force)"
    else:
        prims = inputs.uniform_points(n_sample, seed=seed + 101)
        q = prims[:q_sample]
        kind, qkind, r, what = oracle.POINTS, oracle.SPHERE, inputs.radius_for_neighbours(n_sample), "uniform points"
        qwhat = "16-neighbour sphere queries at its points"
    t0 = time.perf_counter()
    tree = oracle.build(prims, kind, bits)
    t1 = time.perf_counter()
    if qkind is None:
        oracle.knn(prims, kind, q, 16)
    else:
        oracle.query(tree, q, qkind, radius=r)
    t2 = time.perf_counter()
    per_prim = (t1 - t0) / n_sample + (t2 - t1) / q_sample
    desc = (f"oracle (C, 1 thread) build of {n_sample} {what} at {bits} bits "
            f"({t1 - t0:.2f} s) + {q_sample} {qwhat} ({t2 - t1:.2f} s); "
            f"throughput = 1 / (build s/prim + query s/query)")
    return 1.0 / per_prim, desc, t2 - t0


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload in BATCH_WORKLOADS:
        d = BATCH_WORKLOADS[args.workload]
        desc, n, bits = d[0], int(inputs.cloud_sizes(d[1], d[2], d[3], d[4]).sum()), d[5]
    elif args.workload in SERVED_WORKLOADS:
        d = SERVED_WORKLOADS[args.workload]
        desc, n, bits = d[0], int(inputs.poisson_requests(d[1], d[2], d[3], d[4], d[5])[1].sum()), d[6]
    else:
        desc, n, bits = WORKLOADS[args.workload][:3]
    family = workload_family(args.workload) if args.workload in WORKLOADS else "uniform"
    metric = METRIC
    samples = []
    step_s = []  # oracle seconds of each timed (sampled) step
    if family == "curves":
        import oracle
        metric = "construction rate Mprims/s (Algorithm 4, filled cube, largest n)"
        m = 1 << 19
        pts = inputs.filled_cube(m, seed=args.seed)
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.build(pts, oracle.POINTS, bits)
            dt = time.perf_counter() - t0
            if step >= args.warmup:
                samples.append(m / dt)
                step_s.append(dt)
        sdesc = f"oracle build (C, 1 thread) of a {m}-point filled cube, per step"
    elif family == "refit":
        import oracle
        metric = REFIT_METRIC
        m = 1 << 20
        pts = inputs.uniform_points(m, seed=args.seed)
        ot = oracle.build(pts, oracle.POINTS, bits)
        rng = np.random.default_rng(args.seed + 1)
        for step in range(args.warmup + args.steps):
            mv = (pts + rng.normal(0.0, 0.001, size=pts.shape)).astype(np.float32)
            t0 = time.perf_counter()
            oracle.refit(ot, mv)
            dt = time.perf_counter() - t0
            if step >= args.warmup:
                samples.append(m / dt)
                step_s.append(dt)
        sdesc = f"oracle refit (C boxes in post-order, 1 thread) of a {m}-point tree, per step"
    else:
        for step in range(args.warmup + args.steps):
            v, sdesc, dt = oracle_sample(args.seed + step, n_sample=min(ORACLE_N, n), q_sample=min(ORACLE_Q, n),
                                         bits=bits, family=family)
            if step >= args.warmup:
                samples.append(v)
                step_s.append(dt)
    value = statistics.median(samples) / 1e6
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        # a step is one bounded sample of the workload (see cpu_baseline.sample); the
        # whole workload at this rate would take config.n / value
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(step_s) * 1e3,
        "full_workload_s_at_this_rate": n / (value * 1e6),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": n, "morton_bits": bits},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sdesc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm


def run_gpu(args, world, rank, local):
    import torch
    from paper_2402_00665_gb300 import lbvh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, n, bits, prims_host, queries_host, boxes, box_queries, radius = make_inputs(args.workload,
                                                                                       args.seed + rank)
    kind = lbvh.BOXES if boxes else lbvh.POINTS
    knn = box_queries == "knn"
    qkind = lbvh.RAY if box_queries == "ray" else (lbvh.BOX if box_queries and not knn else lbvh.SPHERE)
    pts = torch.from_numpy(prims_host).to(dev)
    # queries in their own buffer (the points themselves for the uniform
    # workloads): the general query path (query centres Morton-encoded and
    # sorted) runs, not the shortcut for a tree queried with its own primitives
    if queries_host is None:
        queries_host = prims_host
    qpts = torch.from_numpy(queries_host).to(dev)
    nq = qpts.shape[0]
    stream = torch.cuda.current_stream(dev)

    tree = lbvh.Tree()
    if args.tuning:
        tune_sort, tune_walk = (int(x) for x in args.tuning.split(","))
        tree.set_tuning(tune_sort, tune_walk)
        tune_how = "fixed by --tuning"
    else:
        # the autotuner picks the sort and walk variants on these very inputs
        # (device-timed, two runs of each candidate) before anything is timed
        tune_sort, tune_walk = tree.autotune(pts, kind, bits, queries=None if knn else qpts, qkind=qkind,
                                             radius=float(radius))
        tune_how = "lbvh_tree_autotune on these inputs before the warm-up"
    tune_how += (" (sort choice: tile shape = choice % half the choices; the second half sorts one top byte "
                 "fewer for codes wider than 30 bits; walk choice: kind = choice % half, the second half orders "
                 "the queries by 24-bit instead of 30-bit Morton codes)")
    tree.set_profiling(True)
    offsets = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    # size the hit buffer once (a production caller does the same)
    tree.build(pts, kind, bits)
    hits = None
    if not knn:
        st, total = tree.query_into(qpts, qkind, offsets, None, radius=float(radius))
        assert st in (lbvh.OK, lbvh.ERR_CAPACITY), st
        hits = torch.empty(max(int(total * 1.05) + 1024, 1), dtype=torch.int32, device=dev)
    K = 16

    def step():
        tree.build(pts, kind, bits)
        if knn:
            tree.knn(qpts, K)
            return nq * K
        s, tot = tree.query_into(qpts, qkind, offsets, hits, radius=float(radius))
        if s != lbvh.OK:
            raise lbvh.LbvhError(s, "lbvh_query_into")
        return tot

    for _ in range(args.warmup):
        step()
    tree.check()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    uuid = None
    try:
        uuid = "GPU-" + str(props.uuid) if not str(props.uuid).startswith("GPU-") else str(props.uuid)
    except Exception:
        pass

    stage_sum: dict[str, float] = {}
    stage_cnt: dict[str, int] = {}
    launches0 = lbvh.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        total_hits = 0
        for _ in range(args.steps):
            total_hits = step()
            for k, v in tree.stage_times().items():
                stage_sum[k] = stage_sum.get(k, 0.0) + v
                stage_cnt[k] = stage_cnt.get(k, 0) + 1
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = lbvh.kernel_launches() - launches0
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = n * world / (ms_step * 1e-3) / 1e6
    clock = clocks.summary()

    stage_ms = {k: stage_sum[k] / stage_cnt[k] for k in stage_sum}
    build_ms = sum(v for k, v in stage_ms.items() if not k.startswith("query"))
    query_ms = sum(v for k, v in stage_ms.items() if k.startswith("query"))
    dominant = max(stage_ms, key=lambda k: stage_ms[k])
    peak, peak_kind = measured_hbm_gbs()
    long_lists = (0, 0)
    if not knn:
        lens = offsets[1:] - offsets[:-1]
        long_mask = lens > 64  # the walk keeps 64 hits per query; longer lists walk again
        long_lists = (int(long_mask.sum().item()), int(lens[long_mask].sum().item()))
    order_passes = 3 if tune_walk >= lbvh.walk_variant_count() // 2 else 4
    alg = {k: alg_bytes(k, n, nq, total_hits, boxes, box_queries, long_lists, order_passes) for k in stage_ms
           if alg_bytes(k, n, nq, total_hits) is not None}
    achieved = alg[dominant] / (stage_ms[dominant] * 1e-3) / 1e9
    build_model = model_build_bytes(n, bits, boxes)
    build_moved = moved_build_bytes(n, bits, boxes, sum(1 for k in stage_ms if k.startswith("sort_pass")))

    # ---- the walk's own roofline: node visits against the same walk on a
    # tree small enough that every node load hits L1 (the ceiling of its
    # dependent-load loop on this GPU)
    walk = None
    if qkind != lbvh.RAY and not knn and dominant == "query_walk":
        lv, iv = tree.walk_visits(qpts, qkind, radius=float(radius))
        visits_s = (lv + iv) / (stage_ms["query_walk"] * 1e-3)
        small_n = 2048
        sp = torch.from_numpy(inputs.uniform_points(small_n, seed=77)).to(dev)
        sq = torch.from_numpy(inputs.uniform_points(1 << 24, seed=78)).to(dev)
        st_ = lbvh.Tree()
        st_.set_profiling(True)
        st_.build(sp, lbvh.POINTS, bits)
        soff = torch.empty((1 << 24) + 1, dtype=torch.int64, device=dev)
        sr = float(inputs.radius_for_neighbours(small_n))
        ms_small = []
        for _ in range(4):
            st_.query_into(sq, lbvh.SPHERE, soff, None, radius=sr)
            ms_small.append(st_.stage_times()["query_walk"])
        slv, siv = st_.walk_visits(sq, lbvh.SPHERE, radius=sr)
        st_.close()
        small_visits_s = (slv + siv) / (min(ms_small[1:]) * 1e-3)
        walk = {"visits_per_query": (lv + iv) / nq, "leaf_visits_per_query": lv / nq,
                "internal_visits_per_query": iv / nq, "visits_per_s": visits_s,
                "node_bytes_per_s": (16 * lv + 32 * iv) / (stage_ms["query_walk"] * 1e-3),
                "l1_resident_visits_per_s": small_visits_s, "l1_frac": visits_s / small_visits_s,
                "l1_ceiling": f"the same walk (2^24 sphere queries, ~16 hits) on a {small_n}-point tree whose "
                              "nodes all stay in L1"}

    # ---- end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e and not knn:
        host_pts = torch.from_numpy(prims_host).pin_memory()
        host_q = torch.from_numpy(queries_host).pin_memory()
        # two steps in flight: step k runs on lane k & 1 (its own tree,
        # stream, device inputs and page-locked result arrays), so the copy of
        # step k's last result chunk to the host overlaps step k + 1's build;
        # step k's inputs go up on a side stream while step k - 1 queries.
        # Every step still copies its own inputs up and its own CSR down
        # inside the timed region; the region ends when both lanes are done.
        trees = [tree, lbvh.Tree()]
        trees[1].set_tuning(tune_sort, tune_walk)
        for t_ in trees:
            t_.set_profiling(False)
            # one chunk: the CSR's copy to the host overlaps the other lane's
            # build and walk instead of this query's own later chunks
            t_.set_host_chunks(1)
        host_off = [torch.empty(nq + 1, dtype=torch.int64).pin_memory() for _ in range(2)]
        host_hits = [torch.empty(hits.numel(), dtype=torch.int32).pin_memory() for _ in range(2)]
        dpts = [torch.empty_like(pts), torch.empty_like(pts)]
        dq = [torch.empty_like(qpts), torch.empty_like(qpts)]
        # --e2e-staged: each lane's device CSR
        dev_off = [offsets, torch.empty_like(offsets) if args.e2e_staged else None]
        dev_hits = [hits, torch.empty_like(hits) if args.e2e_staged else None]
        lanes = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        side = torch.cuda.Stream(dev)
        uploaded = [torch.cuda.Event(), torch.cuda.Event()]
        consumed = [torch.cuda.Event(), torch.cuda.Event()]  # a lane's last read of its device inputs

        def upload(slot):
            with torch.cuda.stream(side):
                side.wait_event(consumed[slot])  # the lane's previous step has read them
                dpts[slot].copy_(host_pts, non_blocking=True)
                dq[slot].copy_(host_q, non_blocking=True)
                uploaded[slot].record(side)

        def e2e_run(steps):
            # results through lbvh_query_into_host, which stages the CSR on
            # the device chunk by chunk and copies each chunk to the
            # page-locked host arrays while the next one runs, or with
            # --e2e-staged into device arrays and then copied
            tot = 0
            upload(0)
            for k in range(steps):
                slot = k & 1
                lane = lanes[slot]
                # the lane's previous step (k - 2) must be done before its
                # tree, staging and host arrays are reused
                lane.synchronize()
                lane.wait_event(uploaded[slot])
                trees[slot].build(dpts[slot], kind, bits, stream=lane)
                if k + 1 < steps:
                    upload(slot ^ 1)
                if args.e2e_staged:
                    s, tot = trees[slot].query_into(dq[slot], qkind, dev_off[slot], dev_hits[slot],
                                                    radius=float(radius), stream=lane)
                    if s != lbvh.OK:
                        raise lbvh.LbvhError(s, "lbvh_query_into")
                    with torch.cuda.stream(lane):
                        host_off[slot].copy_(dev_off[slot], non_blocking=True)
                        host_hits[slot][:tot].copy_(dev_hits[slot][:tot], non_blocking=True)
                else:
                    s, tot = trees[slot].query_into_host(dq[slot], qkind, host_off[slot], host_hits[slot],
                                                         radius=float(radius), stream=lane)
                    if s != lbvh.OK:
                        raise lbvh.LbvhError(s, "lbvh_query_into_host")
                consumed[slot].record(lane)
            for lane in lanes:
                lane.synchronize()
            return tot

        e2e_run(2)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tot = e2e_run(args.steps)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev) / args.steps
        assert int(host_off[(args.steps - 1) & 1][-1]) == tot  # the last step's CSR reached the host
        trees[1].close()
        e2e = {"value": n * world / dt / 1e6, "unit": UNIT, "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": int((pts.numel() + qpts.numel()) * 4),
               "d2h_bytes_per_step": int((nq + 1) * 8 + tot * 4),
               "note": "pinned host primitives and queries -> device (each step's inputs copied on a side "
                       "stream while the previous step queries), build, query, CSR offsets + hits "
                       + ("-> device, then copied to pinned host" if args.e2e_staged
                          else "-> pinned host by lbvh_query_into_host (the CSR staged on the device in one "
                               "chunk, lbvh_tree_set_host_chunks(1), then copied)")
                       + "; two steps in flight on two trees and streams, so one step's result copy overlaps "
                         "the next step's build and walk"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the reference arm's sample (same sizes and seeds), median of a few
        got = [oracle_sample(args.seed + s, n_sample=min(ORACLE_N, n), q_sample=min(ORACLE_Q, n), bits=bits,
                             family=workload_family(args.workload))
               for s in range(CPU_BASELINE_SAMPLES)]
        v = statistics.median(g[0] for g in got)
        cpu = {"value": v / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"median of {CPU_BASELINE_SAMPLES} samples, each: " + got[0][1]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": n, "nq": nq,
                       "morton_bits": bits, "radius": float(radius), "mean_hits": total_hits / nq,
                       "l2": f"inputs larger than L2 (primitives {pts.numel() * 4 / 1e6:.0f} MB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "long_lists": {"queries": long_lists[0], "hits": long_lists[1]},
            "us_per_step": ms_step * 1e3,
            "launches_per_step": launches / args.steps,
            "tuning": {"sort_variant": tune_sort, "walk_variant": tune_walk,
                       "sort_passes": sum(1 for k in stage_ms if k.startswith("sort_pass")),
                       "query_order_bits": 24 if order_passes == 3 else 30,
                       "how": tune_how},
            "build_mprims_s": n / (build_ms * 1e-3) / 1e6,
            "query_mqueries_s": nq / (query_ms * 1e-3) / 1e6,
            "build_ms": build_ms,
            "build_hbm_frac": build_model / (build_ms * 1e-3) / 1e9 / peak,
            "build_bytes_per_prim_model": build_model / n,
            "build_hbm_frac_moved": build_moved / (build_ms * 1e-3) / 1e9 / peak,
            "build_bytes_per_prim_moved": build_moved / n,
            "walk": walk,
            "stage_ms": {k: round(v, 4) for k, v in sorted(stage_ms.items(), key=lambda kv: -kv[1])},
            "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                         "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic_for(dominant),
                         "algorithmic_bytes": alg[dominant],
                         **({"limiter": "L1: dependent node loads of the walk (see walk.l1_frac)",
                             "l1_frac": walk["l1_frac"]} if walk else {})},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clock,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    tree.close()


def run_refit(args, world, rank, local):
    """Refit configuration: a tree built once, then refitted every step."""
    import torch
    from paper_2402_00665_gb300 import lbvh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, n, bits = WORKLOADS[args.workload][:3]
    base = inputs.uniform_points(n, seed=args.seed + rank)
    rng = np.random.default_rng(args.seed + rank + 1)
    moved_host = [(base + rng.normal(0.0, 0.001, size=base.shape)).astype(np.float32) for _ in range(2)]
    moved = [torch.from_numpy(m).to(dev) for m in moved_host]
    stream = torch.cuda.current_stream(dev)
    tree = lbvh.Tree()
    tree.set_profiling(True)
    tree.build(torch.from_numpy(base).to(dev), lbvh.POINTS, bits)
    for k in range(args.warmup):
        tree.refit(moved[k % 2])
    tree.check()
    torch.cuda.synchronize()
    stage_sum: dict[str, float] = {}
    launches0 = lbvh.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(None) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for k in range(args.steps):
            tree.refit(moved[k % 2])
            for name, v in tree.stage_times().items():
                stage_sum[name] = stage_sum.get(name, 0.0) + v
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    tree.check()
    launches = lbvh.kernel_launches() - launches0
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps
    value = n * world / (ms_step * 1e-3) / 1e6
    stage_ms = {k: v / args.steps for k, v in stage_sum.items()}
    peak, peak_kind = measured_hbm_gbs()
    alg = {k: alg_bytes(k, n, 0, 0) for k in stage_ms if alg_bytes(k, n, 0, 0) is not None}
    achieved = alg["construct"] / (stage_ms["construct"] * 1e-3) / 1e9
    refit_frac = sum(alg.values()) / (sum(stage_ms.values()) * 1e-3) / 1e9 / peak

    e2e = None
    if not args.no_e2e:
        host = [torch.from_numpy(m).pin_memory() for m in moved_host]
        dpts = torch.empty_like(moved[0])
        for k in range(2):
            dpts.copy_(host[k], non_blocking=True)
            tree.refit(dpts)
            tree.check()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            dpts.copy_(host[k % 2], non_blocking=True)
            tree.refit(dpts)
            tree.check()  # reads the control block back: the step's result status
        dt = max_over_ranks(time.perf_counter() - t0, world, dev) / args.steps
        e2e = {"value": n * world / dt / 1e6, "unit": UNIT, "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": int(dpts.numel() * 4), "d2h_bytes_per_step": 128,
               "note": "pinned host points -> device, refit, control block (status) -> host"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        m = 1 << 22
        pts = inputs.uniform_points(m, seed=args.seed + 7)
        ot = oracle.build(pts, oracle.POINTS, bits)
        mv = (pts + np.random.default_rng(8).normal(0.0, 0.001, size=pts.shape)).astype(np.float32)
        t0 = time.perf_counter()
        oracle.refit(ot, mv)
        dt = time.perf_counter() - t0
        cpu = {"value": m / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle refit (C boxes in post-order, 1 thread) of a {m}-point tree: {dt:.2f} s"}
    if rank == 0:
        line = {
            "metric": REFIT_METRIC, "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": n, "morton_bits": bits,
                       "l2": f"inputs larger than L2 (points {n * 12 / 1e6:.0f} MB, two alternating sets)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "refit_hbm_frac": refit_frac,
            "stage_ms": {k: round(v, 4) for k, v in sorted(stage_ms.items(), key=lambda kv: -kv[1])},
            "roofline": {"bound": "hbm", "kernel": "construct", "achieved": achieved, "peak": peak,
                         "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic_for("construct"), "algorithmic_bytes": alg["construct"]},
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks.summary(), "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    tree.close()


CURVE_SIZES = [1 << k for k in range(12, 26)]
ALGORITHM_NAMES = {0: "modified_apetrei_alg4", 1: "karras", 2: "apetrei_alg3"}


def run_curves(args, world, rank, local):
    """Build rate vs n for the three algorithms on the filled and hollow cubes."""
    import torch
    from paper_2402_00665_gb300 import lbvh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, _, bits = WORKLOADS[args.workload][:3]
    stream = torch.cuda.current_stream(dev)
    reps = max(args.steps, 1)
    table: dict = {}
    launches0 = lbvh.kernel_launches()
    with ClockSampler(None) as clocks:
        for geometry, gen in (("filled_cube", inputs.filled_cube), ("hollow_cube", inputs.hollow_cube)):
            table[geometry] = {}
            for n in CURVE_SIZES:
                pts = torch.from_numpy(gen(n, seed=args.seed + rank)).to(dev)
                row = {}
                for alg, name in ALGORITHM_NAMES.items():
                    tree = lbvh.Tree()
                    tree.set_profiling(True)
                    for _ in range(max(args.warmup, 1)):
                        tree.build(pts, lbvh.POINTS, bits, algorithm=alg)
                    tree.check()
                    times, hier, second = [], [], []
                    for _ in range(reps):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        tree.build(pts, lbvh.POINTS, bits, algorithm=alg)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        times.append(e0.elapsed_time(e1))
                        st = tree.stage_times()
                        hier.append(st.get("construct", 0.0))
                        second.append(st.get("build_second_pass", 0.0))
                    tree.check()
                    tree.close()
                    ms = statistics.median(times)
                    row[name] = {"build_ms": round(ms, 4), "mprims_s": round(n / (ms * 1e-3) / 1e6, 1),
                                 "hierarchy_ms": round(statistics.median(hier), 4),
                                 "second_pass_ms": round(statistics.median(second), 4)}
                table[geometry][str(n)] = row
                del pts
    launches = lbvh.kernel_launches() - launches0
    top = table["filled_cube"][str(CURVE_SIZES[-1])]
    if rank == 0:
        line = {
            "metric": "construction rate Mprims/s (Algorithm 4, filled cube, largest n)",
            "value": top[ALGORITHM_NAMES[0]]["mprims_s"], "unit": UNIT, "n_gpus": world, "steps": reps,
            "warmup": max(args.warmup, 1), "ms_per_step": top[ALGORITHM_NAMES[0]]["build_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "morton_bits": bits,
                       "sizes": CURVE_SIZES, "timing": "CUDA events around each whole build (bounds, codes, "
                       "sort, hierarchy, second pass), median of the steps; hierarchy_ms / second_pass_ms "
                       "from the library's stage events",
                       "parallelism": "replicas" if world > 1 else "single"},
            "rates": table, "gpu_launches": launches, "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)


def run_batch(args, world, rank, local):
    """Batched configuration: all clouds in one graph launch per step, and the
    same work as a loop of one lbvh_build + lbvh_query_into per cloud."""
    import torch
    from paper_2402_00665_gb300 import lbvh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, count, lo, hi, seed, bits = BATCH_WORKLOADS[args.workload]
    sizes, pts_host = inputs.batched_clouds(count, lo, hi, seed + rank)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    radii_inst = np.array([inputs.radius_for_neighbours(int(k)) for k in sizes], np.float32)
    radii = torch.from_numpy(np.repeat(radii_inst, sizes).astype(np.float32)).to(dev)
    pts = torch.from_numpy(pts_host).to(dev)
    stream = torch.cuda.current_stream(dev)

    batch = lbvh.Batch()
    cap = int(20 * n)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    hits = torch.empty(cap, dtype=torch.int32, device=dev)

    def batch_step():
        _, _, tot, st = batch.build_query(pts, off, lbvh.POINTS, bits, radii=radii, offsets=offsets, hits=hits)
        if st != lbvh.OK:
            raise lbvh.LbvhError(st, "lbvh_batch_build_query")
        return tot

    for _ in range(args.warmup):
        total = batch_step()
    torch.cuda.synchronize()
    launches0 = lbvh.kernel_launches()
    barrier(world)
    with ClockSampler(None) as clocks:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            total = batch_step()
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = lbvh.kernel_launches() - launches0
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    value = n * world / (ms_step * 1e-3) / 1e6

    # the loop of single builds: same clouds, same queries, one call pair each
    tree = lbvh.Tree()
    loff = torch.empty(int(sizes.max()) + 1, dtype=torch.int64, device=dev)
    lhits = torch.empty(int(40 * sizes.max()) + 1024, dtype=torch.int32, device=dev)

    def loop_pass():
        tot = 0
        for k in range(count):
            a, e = int(off[k]), int(off[k + 1])
            tree.build(pts[a:e], lbvh.POINTS, bits)
            st, t = tree.query_into(pts[a:e], lbvh.SPHERE, loff[:e - a + 1], lhits, radius=float(radii_inst[k]))
            if st != lbvh.OK:
                raise lbvh.LbvhError(st, "lbvh_query_into")
            tot += t
        return tot

    loop_pass()
    torch.cuda.synchronize()
    ev0.record(stream)
    loop_total = loop_pass()
    ev1.record(stream)
    torch.cuda.synchronize()
    loop_ms = ev0.elapsed_time(ev1)
    assert loop_total == total, (loop_total, total)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "clouds": count, "n": n,
                       "morton_bits": bits, "mean_hits": total / n,
                       "l2": "inputs larger than L2 (points 1.9 GB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "loop_of_single_builds": {"value": n / (loop_ms * 1e-3) / 1e6, "unit": UNIT, "ms": loop_ms},
            "speedup_vs_loop": loop_ms / ms_step,
            "sort_variant": batch.sort_variant(),
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    batch.close()
    tree.close()


def mixture_radius(n: int, k: float = 16.0, components: int = 64, sigma: float = 0.005) -> float:
    """Radius holding ~k neighbours of a point of an equal-weight Gaussian
    mixture: the expected density at a sample of one component is
    (n / components) / ((4 pi)^(3/2) sigma^3)."""
    density = (n / components) / ((4.0 * math.pi) ** 1.5 * sigma ** 3)
    return float(np.float32((3.0 * k / (4.0 * math.pi * density)) ** (1.0 / 3.0)))


def span_overlap(spans):
    """(busy s, overlap s) of device spans (rows slot, begin, end): the time
    at least one job ran, and the time two or more ran at once."""
    events = sorted([(float(b), 1) for _, b, _ in spans] + [(float(e), -1) for _, _, e in spans])
    busy = overlap = 0.0
    depth, last = 0, None
    for t, d in events:
        if last is not None:
            if depth >= 1:
                busy += t - last
            if depth >= 2:
                overlap += t - last
        depth += d
        last = t
    return busy, overlap


# Batches of up to 256 requests; the number of worker slots (batches in
# flight at once) is --server-slots, 2 by default.
SERVER_MAX_BATCH = 256


def run_served(args, world, rank, local):
    """Served configuration: requests arrive on a Poisson schedule; the request
    server batches them continuously; the same arrivals are then processed one
    at a time (lbvh_build + lbvh_query_into per request, in arrival order)."""
    import threading

    import torch
    from paper_2402_00665_gb300 import lbvh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, count, rate, lo, hi, seed, bits, budget = SERVED_WORKLOADS[args.workload]
    saturated = math.isinf(rate)
    # the saturated workload offers the nominal mix's requests all at once
    arrivals, sizes, kinds = inputs.poisson_requests(count, 2000.0 if saturated else rate, lo, hi, seed + rank)
    if saturated:
        arrivals = np.zeros_like(arrivals)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    host = np.empty((int(off[-1]), 3), np.float32)
    radii = np.empty(count, np.float32)
    for k in range(count):
        n = int(sizes[k])
        if kinds[k] == 0:
            host[off[k]:off[k + 1]] = inputs.uniform_points(n, seed=1000 + k)
            radii[k] = inputs.radius_for_neighbours(n)
        else:
            host[off[k]:off[k + 1]] = inputs.gaussian_mixture_points(n, seed=1000 + k)
            radii[k] = mixture_radius(n)
    pts = torch.from_numpy(host).to(dev)
    views = [pts[off[k]:off[k + 1]] for k in range(count)]
    caps = [int(40 * sizes[k]) + 1024 for k in range(count)]
    torch.cuda.synchronize()

    def percentiles(lat):
        lat = np.sort(np.asarray(lat))
        return float(np.percentile(lat, 50) * 1e3), float(np.percentile(lat, 99) * 1e3)

    # ---- served: a submitter follows the arrival schedule
    slots = args.server_slots
    srv = lbvh.Server(budget, slots=slots, max_batch=SERVER_MAX_BATCH)

    def replay(keep: bool):
        """Submit the requests on their arrival schedule (a submitter thread)
        and wait for each in turn; returns (wall s, latencies, batch sizes, hits)."""
        tickets = [None] * count
        t0 = time.perf_counter()

        def submitter():
            for k in range(count):
                delay = t0 + arrivals[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets[k] = srv.submit(views[k], lbvh.POINTS, bits, radius=float(radii[k]), capacity=caps[k],
                                        key=k + 1 if keep else 0)

        th = threading.Thread(target=submitter)
        th.start()
        lat, sizes_seen, hits = [], [], 0
        for k in range(count):
            while tickets[k] is None:
                time.sleep(0.0001)
            _, _, info = srv.wait(tickets[k])
            if info["status"] != lbvh.OK:
                raise lbvh.LbvhError(info["status"], "served request")
            lat.append(info["latency_s"])
            sizes_seen.append(info["batch_size"])
            hits += info["total"]
        wall = time.perf_counter() - t0
        th.join()
        return wall, lat, sizes_seen, hits

    # warm-up: one untimed replay of the same schedule whose trees are not
    # kept, so the server's buffers have the sizes of steady serving
    replay(keep=False)
    torch.cuda.synchronize()
    spans0 = len(srv.device_spans())
    phases0 = srv.phase_seconds()
    batches0 = srv.stats()["batches"]
    launches0 = lbvh.kernel_launches()
    with ClockSampler(None) as clocks:
        served_s, lat, batch_sizes, totals = replay(keep=True)
    launches = lbvh.kernel_launches() - launches0
    stats = srv.stats()
    phases = {k: v - phases0[k] for k, v in srv.phase_seconds().items()}
    spans = srv.device_spans()[spans0:]
    busy_s, overlap_s = span_overlap(spans)
    server_latency = srv.latency()  # the server's own record (includes the warm-up replay)
    srv.close()
    served_p50, served_p99 = percentiles(lat)

    # ---- one at a time, same arrivals
    tree = lbvh.Tree()
    fo = torch.empty(int(sizes.max()) + 1, dtype=torch.int64, device=dev)
    fh = torch.empty(max(caps), dtype=torch.int32, device=dev)

    def fifo_replay():
        lat, hits = [], 0
        t0 = time.perf_counter()
        for k in range(count):
            wait = t0 + arrivals[k] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            tree.build(views[k], lbvh.POINTS, bits)
            st, tot = tree.query_into(views[k], lbvh.SPHERE, fo[:int(sizes[k]) + 1], fh, radius=float(radii[k]))
            if st != lbvh.OK:
                raise lbvh.LbvhError(st, "lbvh_query_into")
            hits += tot
            lat.append(time.perf_counter() - (t0 + arrivals[k]))
        return time.perf_counter() - t0, lat, hits

    fifo_replay()  # warm-up, untimed
    torch.cuda.synchronize()
    fifo_s, flat, ftotal = fifo_replay()
    tree.close()
    assert ftotal == totals, (ftotal, totals)
    fifo_p50, fifo_p99 = percentiles(flat)
    n = int(off[-1])
    value = n * world / served_s / 1e6
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": served_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "requests": count, "rate_per_s": rate,
                       "n_total": n, "morton_bits": bits, "budget_bytes": budget,
                       "offered_mprims_s": None if saturated else n / float(arrivals[-1]) / 1e6,
                       "arrivals": "all at t = 0" if saturated else f"Poisson, {rate:g} per s",
                       "mean_hits": totals / n, "parallelism": "replicas" if world > 1 else "single"},
            "served": {"throughput_mprims_s": value, "p50_ms": served_p50, "p99_ms": served_p99,
                       "wall_s": served_s, "mean_batch": float(np.mean(batch_sizes)),
                       "batches": stats["batches"] - batches0, "slots": slots,
                       "device": {"jobs": int(len(spans)), "busy_s": busy_s, "overlap_s": overlap_s,
                                  "overlap_frac": overlap_s / busy_s if busy_s > 0 else 0.0,
                                  "jobs_per_slot": [int((spans[:, 0] == s).sum()) for s in range(slots)],
                                  "how": "CUDA events around each batch on its slot's stream, against one "
                                         "reference event; overlap = device time with two or more batches "
                                         "in flight"},
                       "max_batch": SERVER_MAX_BATCH, "resident_trees": stats["resident_trees"],
                       "resident_bytes": stats["resident_bytes"], "evictions": stats["evictions"],
                       "worker_phase_s": phases,
                       "server_reported_latency_all_requests": server_latency},
            "one_at_a_time": {"throughput_mprims_s": n / fifo_s / 1e6, "p50_ms": fifo_p50, "p99_ms": fifo_p99,
                              "wall_s": fifo_s},
            "speedup_vs_one_at_a_time": fifo_s / served_s,
            "timing": "wall clock from the first arrival to the last completion; latency = arrival to results; "
                      "server warmed by one untimed replay of the same schedule (trees not kept)",
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload in SERVED_WORKLOADS and args.impl == "lbvh":
        import torch
        if not torch.cuda.is_available():
            raise SystemExit("bench.py needs a CUDA GPU for the lbvh arm")
        world, rank, local = dist_setup(True)
        run_served(args, world, rank, local)
        return
    if args.workload in BATCH_WORKLOADS and args.impl == "lbvh":
        import torch
        if not torch.cuda.is_available():
            raise SystemExit("bench.py needs a CUDA GPU for the lbvh arm")
        world, rank, local = dist_setup(True)
        run_batch(args, world, rank, local)
        return
    if args.impl == "reference":
        world, rank, _ = dist_setup(False)
        run_reference(args, world, rank)
        return
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for the lbvh arm")
    world, rank, local = dist_setup(True)
    if workload_family(args.workload) == "refit":
        run_refit(args, world, rank, local)
    elif workload_family(args.workload) == "curves":
        run_curves(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
