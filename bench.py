#!/usr/bin/env python
"""Benchmark: certified h(A, B) queries per second on one GB300.

Workload (one pair per step and per rank): A = torus R=1, r=0.3 on a 400 x 250 grid
(200,000 triangles, vertex normal noise sigma 1e-3), B = the same torus re-triangulated
on a 224 x 112 grid with 0.3-cell jitter (50,176 triangles), tol = 1e-5 x bbox diagonal of
A; float32 vertices, seeded synthetic data.  A step is the whole hot path: BVH build of B,
round 0 (vertex queries, lower bound, bounds of every face) and every frontier round to
convergence.  Inputs are resident in HBM; L2 is flushed (256 MiB write) between timed
steps; steps are timed with CUDA events on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank runs its own replica of the pair (independent units, no
collective on the data path); the value is all ranks' pairs / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import meshgen as mg  # noqa: E402

METRIC = "certified h(A,B) queries/s"
UNIT = "pairs/s"
WORKLOAD = 2
# CPU-baseline sample: the oracle on 1/16 of A's faces (a band of the torus) against all of B
SLICES = 16
# the reference arm's step: 1/64 of A's faces, so that the default 205 steps take about a
# minute on 16 host cores
REF_SLICES = 64
# flops per unit, counted from the kernel source (see the design notes): one point-triangle
# closest-point evaluation (Voronoi-region method, face-region path) and one child-box test
FLOPS_PER_LEAF_TEST = 80
FLOPS_PER_BOX_TEST = 17
FLOPS_PER_ITEM_BOUND = 100
BYTES_PER_NODE = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true")
    return ap.parse_args()


def workload_desc(p):
    return (f"{p.name}: torus pair, A {len(p.FA):,} triangles (400x250 grid, normal noise 1e-3), "
            f"B {len(p.FB):,} triangles (224x112 grid, 0.3-cell jitter), tol 1e-5 x bbox diagonal of A")


# ----------------------------------------------------------------------------- CPU oracle


def oracle_sample(p, k: int, eps_abs: float, slices: int = SLICES):
    """Oracle on slice k of A's faces (1/slices of them) against all of B; returns seconds."""
    import oracle

    n = len(p.FA)
    a, b = k * n // slices, (k + 1) * n // slices
    t = time.perf_counter()
    r = oracle.hausdorff(p.VA, p.FA[a:b], p.VB, p.FB, eps_abs, 0)
    dt = time.perf_counter() - t
    return dt, r


def cpu_baseline(p, eps_abs, slices=(0, SLICES // 2)):
    import oracle

    oracle.build()
    t = 0.0
    for k in slices:
        dt, _ = oracle_sample(p, k, eps_abs)
        t += dt
    frac = len(slices) / SLICES
    return dict(value=frac / t, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=f"FP64 oracle (brute-force distances, best-first queue) on {len(slices)} slices of 1/{SLICES} "
                       f"of A's faces each against all of B at the same absolute eps; {t:.2f} s for "
                       f"{frac:.4f} of the pair, scaled to pairs/s")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    p = mg.workload(WORKLOAD)
    VA = p.VA.astype(np.float64)
    eps_abs = p.tol * float(np.linalg.norm(VA.max(0) - VA.min(0)))
    for w in range(args.warmup):
        oracle_sample(p, w % REF_SLICES, eps_abs, REF_SLICES)
    ts = []
    for k in range(args.steps):
        dt, _ = oracle_sample(p, k % REF_SLICES, eps_abs, REF_SLICES)
        ts.append(dt)
    total = sum(ts)
    value = args.steps / REF_SLICES / total
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * total / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=workload_desc(p), sample=f"each step: 1/{REF_SLICES} of A's faces (rotating bands)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                                  sample=f"each step is 1/{REF_SLICES} of A's faces against all of B; value scaled to "
                                         "whole pairs per second"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows, self.proc = [], None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=[], samples=0)
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx) if mx else None, reasons=reasons,
                    samples=len(sm))


# ----------------------------------------------------------------------------- GPU arm


def source_digest() -> str:
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2406_10357_gb300", "csrc")
    for f in sorted(os.listdir(src)):
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kind: str, precision: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_digest") != source_digest() or kv.get(f"{kind}.{precision}.bytes_per_launch") is None:
        return None
    return float(kv[f"{kind}.{precision}.bytes_per_launch"])


def kernel_launches(nB: int, stats: dict, mixed: bool, leaf_size: int = 1) -> int:
    """Kernels one hd_build_B + hd_hausdorff call launches.  hd_hausdorff counts its own
    (stats["kernel_launches"]); the build's sequence is fixed by n_B: centroids, Morton
    codes, per sort pass a digit count and a scatter (plus a scan when B needs more than 64
    sort tiles), the gather, then the radix tree, the aligned-block boxes (one launch per 8
    levels), the node boxes and the node emission (one root kernel instead when B fits in
    one leaf), and B's eta and validity."""
    bits = 10
    while bits < 16 and (1 << (3 * (bits - 4))) < nB:
        bits += 1
    passes = -(-3 * bits // 8)
    tile = 256 * (4 if nB <= 64 * 256 * 4 else 16)
    fused = -(-nB // tile) <= 64
    levels = max(1, (nB - 1).bit_length())  # aligned-block levels, 8 per launch
    build = 2 + passes * (2 if fused else 3) + 1 + ((3 + -(-levels // 8)) if nB > leaf_size else 1) + 1
    return build + int(stats["kernel_launches"])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def run_ours(args):
    import torch

    import paper_2406_10357_gb300 as hd
    from paper_2406_10357_gb300 import build as hb
    from paper_2406_10357_gb300 import multi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not hb.up_to_date():
        hb.build()
    if dist:
        dist.barrier()

    p = mg.workload(WORKLOAD)
    VA = torch.from_numpy(p.VA).to(dev)
    FA = torch.from_numpy(p.FA).to(dev)
    VB = torch.from_numpy(p.VB).to(dev)
    FB = torch.from_numpy(p.FB).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    prec = hd.HD_MIXED if args.precision == "mixed" else hd.HD_FP64
    # the build is queued without a host wait (B's validity is checked by hd_hausdorff's
    # first read-back), so the run's set-up overlaps it
    opt = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec, flags=hd.HD_FLAG_ASYNC_BUILD)

    def step(o):
        bvh = hd.hd_build_B(VB, FB, o)
        r = hd.hd_hausdorff(bvh, VA, FA, p.tol, o)
        if r["status"] != hd.HD_OK:
            raise RuntimeError(f"step failed: {r}")
        return r

    def timed(o, k):
        ts, rs = [], []
        for _ in range(k):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs.append(step(o))
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, rs

    for _ in range(args.warmup):
        step(opt)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ts, rs = timed(opt, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()

    total_ms = sum(ts)
    total_ms = multi.max_over_ranks(total_ms, device=dev)  # the slowest rank's time
    value = world * args.steps / (total_ms / 1e3)

    # the per-kernel-kind durations for the roofline: the same K steps again with the
    # library's CUDA events around each kind.  An event between two kernels stops the second
    # from being scheduled while the first runs (the chained launches), so these events are
    # kept out of the timed steps above; value_traced is the throughput with them.
    hd.hd_trace_read(reset=True)
    hd.hd_trace_enable(True)
    if dist:
        dist.barrier()
    ts_tr, rs_tr = timed(opt, args.steps)
    torch.cuda.synchronize()
    hd.hd_trace_enable(False)
    trace = hd.hd_trace_read(reset=True)
    value_traced = world * args.steps / (multi.max_over_ranks(sum(ts_tr), device=dev) / 1e3)

    # mixed vs FP64 at the same tol (same workload, fewer steps)
    fp64 = None
    if not args.no_fp64_arm and prec == hd.HD_MIXED:
        o64 = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_FP64, flags=hd.HD_FLAG_ASYNC_BUILD)
        step(o64)
        k64 = max(3, args.steps // 4)
        t64, r64 = timed(o64, k64)
        fp64 = dict(value=k64 / (sum(t64) / 1e3), ms_per_step=sum(t64) / k64, lower=r64[-1]["lower"],
                    upper=r64[-1]["upper"])

    # the branch and bound alone (B's BVH built once, outside the timed region), as the paper's
    # timings can be read both with and without the build
    bvh_once = hd.hd_build_B(VB, FB, opt)
    bnb_ts = []
    for _ in range(max(3, args.steps // 4)):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hd.hd_hausdorff(bvh_once, VA, FA, p.tol, opt)
        e1.record(stream)
        torch.cuda.synchronize()
        bnb_ts.append(e0.elapsed_time(e1))
    del bvh_once
    bnb_ms = multi.max_over_ranks(sum(bnb_ts), device=dev) / len(bnb_ts)
    bnb_only = dict(value=world * 1e3 / bnb_ms, unit=UNIT, ms_per_step=bnb_ms,
                    note="hd_hausdorff only; B's BVH built once before the timed region")

    # end to end through the C ABI with host buffers in pinned memory (their copies to the
    # device inside the timed region)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    VAh, FAh, VBh, FBh = pin(p.VA), pin(p.FA), pin(p.VB), pin(p.FB)
    e2e_ts, e2e_r = [], None
    for _ in range(max(3, args.steps // 4)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bvh = hd.hd_build_B(VBh, FBh, opt)
        e2e_r = hd.hd_hausdorff(bvh, VAh, FAh, p.tol, opt)
        lo, up = e2e_r["lower"], e2e_r["upper"]  # result already on the host
        e2e_ts.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_ts)
    e2e_total = multi.max_over_ranks(e2e_total, device=dev)
    h2d = p.VA.nbytes + p.FA.nbytes + p.VB.nbytes + p.FB.nbytes
    d2h = int(e2e_r["stats"]["d2h_bytes"])  # the run-state snapshots the call read back

    # roofline of the dominant kernel kind, from the traced steps
    stats = [r["stats"] for r in rs_tr]
    leaf = sum(s["leaf_tests"] for s in stats)
    boxes = sum(s["box_tests"] for s in stats)
    evals = sum(s["pointtri_evals"] for s in stats)
    dom = max(("query", "bound", "select", "build", "prep", "small_rounds"), key=lambda k: trace[k]["ms"])
    q = trace["query"]
    peaks, src = measured_peaks()
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if prec == hd.HD_MIXED:
        peak_tf = 152 * 128 * 2 * clock_mhz * 1e6 / 1e12  # FP32 lanes x FMA x max SM clock
        peak_note = f"FP32: 152 SMs x 128 lanes x 2 flops x {clock_mhz:.0f} MHz (derived, {src} clock)"
    else:
        peak_tf = 1.25  # FP64 nominal for GB300 (the pool's profiling recipe)
        peak_note = "FP64 nominal 1.25 TFLOP/s"
    share = {k: round(trace[k]["ms"] / max(1e-9, sum(v["ms"] for v in trace.values())), 4) for k in trace}
    # traversal: 80 flops per leaf test + 17 per child box; cascade: 80 per point-triangle
    # evaluation of u3 + 100 per bounded sub-triangle (exact case, u1, u2); bounded
    # sub-triangles per step = faces of A + 4 per split
    items = sum(len(p.FA) + 4 * s["splits"] for s in stats)
    kinds = {
        "query": dict(kernel="k_query (nearest-triangle traversal)",
                      flops=FLOPS_PER_LEAF_TEST * leaf + FLOPS_PER_BOX_TEST * boxes,
                      algorithmic=f"{FLOPS_PER_LEAF_TEST} flops x leaf tests + {FLOPS_PER_BOX_TEST} flops x box tests",
                      l2_bytes=BYTES_PER_NODE * boxes / 2 + 48 * leaf),
        "bound": dict(kernel="k_bound_faces/k_bound_children (UpperBound cascade)",
                      flops=FLOPS_PER_LEAF_TEST * (evals - leaf) + FLOPS_PER_ITEM_BOUND * items,
                      algorithmic=f"{FLOPS_PER_LEAF_TEST} flops x u3 point-triangle evaluations + "
                                  f"{FLOPS_PER_ITEM_BOUND} flops x bounded sub-triangles",
                      l2_bytes=3 * 64 * items + 48 * (evals - leaf)),
    }

    def roofline_of(kind):
        t, k = trace[kind], kinds[kind]
        achieved = k["flops"] / (t["ms"] / 1e3) / 1e12 if t["ms"] > 0 else 0.0
        return dict(kernel=k["kernel"], bound="alu", achieved=achieved, peak=peak_tf, unit="TFLOP/s",
                    frac=achieved / peak_tf, traffic=profiled_traffic(kind, args.precision), peak_note=peak_note,
                    algorithmic=k["algorithmic"], launches=t["launches"],
                    ms_per_launch=t["ms"] / max(1, t["launches"]),
                    l2_bytes_per_launch=k["l2_bytes"] / max(1, t["launches"]))

    main_kind = "bound" if trace["bound"]["ms"] > trace["query"]["ms"] else "query"
    roof = roofline_of(main_kind)
    roof.update(dominant_kind=dom, share=share,
                timing="CUDA events around each kernel kind, on the launching stream, over a second pass of "
                       "the K steps (value_traced)")
    roof_other = roofline_of("query" if main_kind == "bound" else "bound")

    launches = sum(kernel_launches(len(p.FB), r["stats"], prec == hd.HD_MIXED) for r in rs)  # the timed steps

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32" if prec == hd.HD_MIXED else "f64", data="synthetic",
                config=dict(workload=workload_desc(p), precision=args.precision, l2="flushed between steps (256 MiB write)",
                            parallelism="replicas" if world > 1 else "single",
                            build="queued without a host wait (HD_FLAG_ASYNC_BUILD)"),
                value_traced=value_traced,
                pointtri_evals_per_s=world * evals / (total_ms / 1e3),
                result=dict(lower=rs[-1]["lower"], upper=rs[-1]["upper"], eps_abs=rs[-1]["stats"]["eps_abs"],
                            rounds=rs[-1]["stats"]["rounds"], splits=rs[-1]["stats"]["splits"]),
                roofline=roof, roofline_other_kernel=roof_other, e2e=dict(value=world * len(e2e_ts) / e2e_total, unit=UNIT, h2d_bytes_per_step=h2d,
                                        d2h_bytes_per_step=d2h),
                gpu_launches=launches, clocks=clk, fp64_arm=fp64, bnb_only=bnb_only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        VAd = p.VA.astype(np.float64)
        line["cpu_baseline"] = cpu_baseline(p, p.tol * float(np.linalg.norm(VAd.max(0) - VAd.min(0))))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
