#!/usr/bin/env python
"""Benchmark: certified h(A, B) queries per second on one GB300.

Headline workload (one pair per step and per rank): the large soup.  A = a 975 x 975
superquadric (exponents 0.8 / 1.2) plus 100,000 random triangles near its surface, up to 0.1
off it (2,001,350 triangles); B = an independently triangulated, jittered 1000 x 1000 copy of
the superquadric (2,000,000 triangles); tol = 1e-6 x bbox diagonal of A; float32 vertices,
seeded synthetic data.  A step is the whole hot path: BVH build of B, round 0 (vertex
queries, lower bound, bounds of every face) and every frontier round to convergence, in the
certified FP32 arithmetic (MIXED).  Inputs are resident in HBM and larger than L2; L2 is also
flushed (256 MiB write) between timed steps; steps are timed with CUDA events on the launching
stream.

Beside the headline the same run reports: the same step in FP64, the branch and bound alone
(B's BVH built once), the end-to-end call from pinned host buffers, the torus benchmark pair
(200,000 vs 50,176 triangles, tol 1e-5 dA) in MIXED and FP64, and the batched workload (1024
pairs of 1K-200K triangles a side, tol 1e-4 dA) as one batched MIXED call against sequential
per-pair FP64 calls.

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
HEADLINE = 5  # the large soup, 2M x 2M triangles
TORUS = 2     # the near-identical torus pair
BATCH_PAIRS = 1024
# CPU-baseline sample: the oracle on a few samples of 1/SLICES of A's faces each against all
# of B.  A sample takes band k of the surface's faces and band k of the random triangles, in
# their proportion (95 / 5): the random triangles hold the largest distances, so l starts
# near h as in the whole pair and the surface faces are discarded by their round-0 bounds
# (the whole pair needs no split at its tolerance); the cost is then the brute-force vertex
# queries, about 2M point-triangle tests each.
SLICES = 4096
CPU_SLICES = (512, 1536, 2560, 3584)
N_RANDOM = 100_000  # random triangles at the end of A's faces in the large soup
# the reference arm's step: one sample of 1/REF_SLICES of A's faces, so that the default 25
# steps take about a minute on 16 host cores
REF_SLICES = 8192
# algorithmic bytes of the traversal, per unit (see the design notes): a 4-wide node fetched
# (128 B), a leaf triangle tested (48 B as float4 x 3 in MIXED, 72 B as 9 doubles in FP64),
# and the query's pool vertex read and written back (64 + 64 B)
BYTES_PER_NODE = 128
BYTES_PER_QUERY = 128
# flops per unit, counted from the kernel source: one point-triangle closest-point evaluation
# (Voronoi-region method, face-region path) and one bounded sub-triangle (exact case, u1, u2)
FLOPS_PER_PT_EVAL = 80
FLOPS_PER_ITEM_BOUND = 100


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="only the headline workload (for profiling)")
    ap.add_argument("--batch-pairs", type=int, default=BATCH_PAIRS)
    return ap.parse_args()


def workload_desc(p):
    return (f"{p.name}: large soup, A {len(p.FA):,} triangles (975x975 superquadric 0.8/1.2 + 100,000 random "
            f"triangles up to 0.1 off it), B {len(p.FB):,} triangles (1000x1000 jittered superquadric), "
            f"tol 1e-6 x bbox diagonal of A")


def eps_of(p):
    R = np.asarray(p.VA, np.float64)[np.unique(p.FA.ravel())]
    return p.tol * float(np.linalg.norm(R.max(0) - R.min(0)))


# ----------------------------------------------------------------------------- CPU oracle


def oracle_band(p, k: int, slices: int, eps_abs: float):
    """Oracle on sample k of A's faces (band k of 1/slices of the surface faces and of the
    random triangles) against all of B; returns seconds."""
    import oracle

    ns = len(p.FA) - N_RANDOM
    rows = np.concatenate([p.FA[k * ns // slices:(k + 1) * ns // slices],
                           p.FA[ns + k * N_RANDOM // slices:ns + (k + 1) * N_RANDOM // slices]])
    t = time.perf_counter()
    r = oracle.hausdorff(p.VA, rows, p.VB, p.FB, eps_abs, 0)
    return time.perf_counter() - t, r


def cpu_baseline(p, eps_abs):
    import oracle

    oracle.build()
    t = sum(oracle_band(p, k, SLICES, eps_abs)[0] for k in CPU_SLICES)
    frac = len(CPU_SLICES) / SLICES
    return dict(value=frac / t, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=f"FP64 oracle (brute-force distances, best-first queue) on {len(CPU_SLICES)} samples of "
                       f"1/{SLICES} of A's faces each (a band of the surface faces and one of the random "
                       f"triangles), against all of B at the same absolute eps; {t:.2f} s for {frac:.5f} of the "
                       f"pair, scaled to pairs/s")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    p = mg.workload(HEADLINE)
    eps_abs = eps_of(p)
    stride = 2897  # bands visited in a fixed scattered order
    for w in range(args.warmup):
        oracle_band(p, (w * stride) % REF_SLICES, REF_SLICES, eps_abs)
    ts = []
    for k in range(args.steps):
        dt, _ = oracle_band(p, ((args.warmup + k) * stride) % REF_SLICES, REF_SLICES, eps_abs)
        ts.append(dt)
    total = sum(ts)
    value = args.steps / REF_SLICES / total
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * total / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=workload_desc(p),
                            sample=f"each step: 1/{REF_SLICES} of A's faces (a band of the surface and one of the "
                                   "random triangles)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                                  sample=f"each step is 1/{REF_SLICES} of A's faces (a band of the surface and one "
                                         "of the random triangles) against all of B; value scaled to whole pairs "
                                         "per second"),
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


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    key = f"{workload}.{kernel}.bytes_per_launch"
    if kv.get("source_digest") != source_digest() or key not in kv:
        return None
    return float(kv[key])


def build_launches(nB: int, leaf_size: int = 1) -> int:
    """Kernels one hd_build_B launches; the sequence is fixed by n_B: centroids, Morton codes,
    per sort pass (8 code bits each, the code's last 1 or 2 bits dropped) a digit count and a scatter (plus a scan when B needs more than 64 sort
    tiles), the hint grid (cleared, then filled), the gather, then the radix tree, the aligned-block boxes (one launch per 8
    levels), the node boxes and the node emission (one root kernel instead when B fits in one
    leaf), and B's eta and validity."""
    bits = 10
    while bits < 16 and (1 << (3 * (bits - 4))) < nB:
        bits += 1
    drop = (3 * bits) % 8 if (3 * bits) % 8 <= 2 else 0  # low code bits that would take a pass alone
    passes = -(-(3 * bits - drop) // 8)
    tile = 256 * (4 if nB <= 64 * 256 * 4 else 8)
    fused = -(-nB // tile) <= 64
    levels = max(1, (nB - 1).bit_length())  # aligned-block levels, 8 per launch
    return 2 + passes * (2 if fused else 3) + 2 + 1 + ((3 + -(-levels // 8)) if nB > leaf_size else 1) + 1


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def l2_copy_peak(torch, dev, mb: int = 32, reps: int = 400):
    """Bandwidth of a device copy whose source and destination (mb MiB each) stay in L2:
    read + write bytes over CUDA-event time, best of 5 runs of `reps` copies."""
    a = torch.empty(mb << 20, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    a.fill_(1)
    for _ in range(20):
        b.copy_(a)
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * (mb << 20) * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


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
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    prec = hd.HD_MIXED if args.precision == "mixed" else hd.HD_FP64

    def on_device(p):
        return tuple(torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (p.VA, p.FA, p.VB, p.FB))

    def options(precision):
        # the build is queued without a host wait (B's validity is checked by hd_hausdorff's
        # first read-back), so the run's set-up overlaps it
        return hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=precision, flags=hd.HD_FLAG_ASYNC_BUILD)

    def step(p, d, o):
        VA, FA, VB, FB = d
        bvh = hd.hd_build_B(VB, FB, o)
        r = hd.hd_hausdorff(bvh, VA, FA, p.tol, o)
        if r["status"] != hd.HD_OK:
            raise RuntimeError(f"step failed: {r}")
        return r

    def timed(p, d, o, k):
        ts, rs = [], []
        for _ in range(k):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs.append(step(p, d, o))
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, rs

    p = mg.workload(HEADLINE)
    d = on_device(p)
    opt = options(prec)
    for _ in range(args.warmup):
        step(p, d, opt)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ts, rs = timed(p, d, opt, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = multi.max_over_ranks(sum(ts), device=dev)  # the slowest rank's time
    value = world * args.steps / (total_ms / 1e3)

    # the per-kernel-kind durations for the roofline: the same K steps again with the
    # library's CUDA events around each kind.  An event between two kernels stops the second
    # from being scheduled while the first runs (the chained launches), so these events are
    # kept out of the timed steps above; value_traced is the throughput with them.
    hd.hd_trace_read(reset=True)
    hd.hd_trace_enable(True)
    ts_tr, rs_tr = timed(p, d, opt, args.steps)
    torch.cuda.synchronize()
    hd.hd_trace_enable(False)
    trace = hd.hd_trace_read(reset=True)
    value_traced = world * args.steps / (multi.max_over_ranks(sum(ts_tr), device=dev) / 1e3)

    extras = {}
    if not args.no_extras:
        # MIXED against FP64 at the same tolerance (same workload, fewer steps)
        if not args.no_fp64_arm and prec == hd.HD_MIXED:
            o64 = options(hd.HD_FP64)
            step(p, d, o64)
            k64 = max(3, args.steps // 4)
            t64, r64 = timed(p, d, o64, k64)
            extras["fp64_arm"] = dict(value=world * k64 / (multi.max_over_ranks(sum(t64), device=dev) / 1e3),
                                      unit=UNIT, ms_per_step=sum(t64) / k64, lower=r64[-1]["lower"],
                                      upper=r64[-1]["upper"])
        # the branch and bound alone (B's BVH built once, outside the timed region), as the
        # paper's timings can be read both with and without the build
        bvh_once = hd.hd_build_B(d[2], d[3], opt)
        bnb_ts = []
        for _ in range(max(3, args.steps // 4)):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hd.hd_hausdorff(bvh_once, d[0], d[1], p.tol, opt)
            e1.record(stream)
            torch.cuda.synchronize()
            bnb_ts.append(e0.elapsed_time(e1))
        del bvh_once
        bnb_ms = multi.max_over_ranks(sum(bnb_ts), device=dev) / len(bnb_ts)
        extras["bnb_only"] = dict(value=world * 1e3 / bnb_ms, unit=UNIT, ms_per_step=bnb_ms,
                                  note="hd_hausdorff only; B's BVH built once before the timed region")

    # end to end through the C ABI with host buffers in pinned memory (their copies to the
    # device inside the timed region, the bracket read back)
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
        del bvh
    e2e_total = multi.max_over_ranks(sum(e2e_ts), device=dev)
    h2d = p.VA.nbytes + p.FA.nbytes + p.VB.nbytes + p.FB.nbytes
    d2h = int(e2e_r["stats"]["d2h_bytes"])  # the run-state snapshots the call read back

    if not args.no_extras:
        extras["torus_pair"] = torus_pair(args, torch, hd, multi, dev, on_device, options, timed, step, world)
        extras["batched"] = batched_pairs(args, torch, hd, dev, prec)

    # roofline of the dominant kernel kind, from the traced steps
    peaks, src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    l2 = l2_copy_peak(torch, dev)
    stats = [r["stats"] for r in rs_tr]
    tri_bytes = 48 if prec == hd.HD_MIXED else 72
    sumk = lambda k: sum(s[k] for s in stats)
    nodes_long, leaf_long = sumk("long_node_visits"), sumk("long_leaf_tests")
    nodes_lane, leaf_lane = sumk("node_visits") - nodes_long, sumk("leaf_tests") - leaf_long
    q_long = sumk("long_queries")
    q_lane = sumk("queries")  # every query starts in the lane traversal
    items = sum(len(p.FA) + 4 * s["splits"] for s in stats)
    u3_evals = sumk("pointtri_evals") - sumk("leaf_tests")
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_tf = sms * 128 * 2 * clock_mhz * 1e6 / 1e12
    kinds = {
        "query": dict(kernel="k_query (lane traversal, a1/a3/a4)", bound="hbm",
                      bytes=BYTES_PER_NODE * nodes_lane + tri_bytes * leaf_lane + BYTES_PER_QUERY * q_lane,
                      algorithmic=f"{BYTES_PER_NODE} B x nodes fetched + {tri_bytes} B x leaf triangles tested + "
                                  f"{BYTES_PER_QUERY} B x queries (pool vertex read and written)"),
        "query_long": dict(kernel="k_query_long (warp-cooperative traversal of long queries, a3)", bound="hbm",
                           bytes=BYTES_PER_NODE * nodes_long + tri_bytes * leaf_long + BYTES_PER_QUERY * q_long,
                           algorithmic=f"{BYTES_PER_NODE} B x nodes fetched + {tri_bytes} B x leaf triangles tested + "
                                       f"{BYTES_PER_QUERY} B x long queries"),
        "bound": dict(kernel="k_bound_faces/k_bound_children/k_bound_u4 (UpperBound cascade, a5)", bound="alu",
                      flops=FLOPS_PER_PT_EVAL * u3_evals + FLOPS_PER_ITEM_BOUND * items,
                      algorithmic=f"{FLOPS_PER_PT_EVAL} flops x u3 point-triangle evaluations + "
                                  f"{FLOPS_PER_ITEM_BOUND} flops x bounded sub-triangles"),
    }

    def roofline_of(kind):
        t, k = trace[kind], kinds[kind]
        n = max(1, t["launches"])
        sec = t["ms"] / 1e3 / n  # average launch duration
        if k["bound"] == "hbm":
            per = k["bytes"] / n
            achieved = per / sec / 1e9 if sec > 0 else 0.0
            out = dict(kernel=k["kernel"], bound="hbm", achieved=achieved, peak=hbm, unit="GB/s",
                       frac=achieved / hbm, traffic=profiled_traffic(kind, "large_soup"),
                       peak_note=f"HBM copy bandwidth ({src}, MEASURED_PEAKS.json)",
                       l2_peak=l2, frac_of_l2=achieved / l2 if l2 else None,
                       l2_peak_note="device copy of a 32 MiB buffer held in L2, CUDA events, measured in this run",
                       algorithmic=k["algorithmic"], bytes_per_launch=per)
        else:
            per = k["flops"] / n
            achieved = per / sec / 1e12 if sec > 0 else 0.0
            out = dict(kernel=k["kernel"], bound="alu", achieved=achieved, peak=fp32_tf, unit="TFLOP/s",
                       frac=achieved / fp32_tf, traffic=profiled_traffic(kind, "large_soup"),
                       peak_note=f"FP32: {sms} SMs x 128 lanes x 2 flops x {clock_mhz:.0f} MHz ({src} max clock)",
                       algorithmic=k["algorithmic"], flops_per_launch=per)
        out.update(launches=t["launches"], ms_per_launch=t["ms"] / n)
        return out

    share = {k: round(trace[k]["ms"] / max(1e-9, sum(v["ms"] for v in trace.values())), 4) for k in trace}
    main_kind = max(kinds, key=lambda k: trace[k]["ms"])
    roof = roofline_of(main_kind)
    roof.update(dominant_kind=max(trace, key=lambda k: trace[k]["ms"]), share=share,
                timing="CUDA events around each kernel kind, on the launching stream, over a second pass of "
                       "the K steps (value_traced)",
                choice="the traversal or bound kind with the largest traced time (the build, several kernels, "
                       "has no single roofline); the query_long kind also times its list reordering "
                       "(k_long_hist, k_long_scan, k_long_scatter: about 15% of the kind in the launch list)")
    roof_other = {k: roofline_of(k) for k in kinds if k != main_kind}

    launches = sum(build_launches(len(p.FB)) + int(r["stats"]["kernel_launches"]) for r in rs)  # the timed steps

    s0 = rs[-1]["stats"]
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32" if prec == hd.HD_MIXED else "f64", data="synthetic",
                config=dict(workload=workload_desc(p), precision=args.precision,
                            l2="inputs larger than L2, and L2 flushed between steps (256 MiB write)",
                            parallelism="replicas" if world > 1 else "single",
                            build="included in every step, queued without a host wait (HD_FLAG_ASYNC_BUILD)"),
                value_traced=value_traced,
                pointtri_evals_per_s=world * sum(r["stats"]["pointtri_evals"] for r in rs) / (total_ms / 1e3),
                result=dict(lower=rs[-1]["lower"], upper=rs[-1]["upper"], eps_abs=s0["eps_abs"], rounds=s0["rounds"],
                            splits=s0["splits"], queries=s0["queries"], long_queries=s0["long_queries"],
                            promoted=s0["promoted"], fp64_escalations=s0["fp64_escalations"]),
                roofline=roof, roofline_other_kernels=roof_other,
                e2e=dict(value=world * len(e2e_ts) / e2e_total, unit=UNIT, h2d_bytes_per_step=h2d,
                         d2h_bytes_per_step=d2h),
                gpu_launches=launches, clocks=clk, **extras)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, eps_of(p))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def torus_pair(args, torch, hd, multi, dev, on_device, options, timed, step, world):
    """The torus benchmark pair (200,000 vs 50,176 triangles, tol 1e-5 dA), build included."""
    p = mg.workload(TORUS)
    d = on_device(p)
    out = dict(workload=f"{p.name}: torus 400x250 (normal noise 1e-3) vs re-triangulated 224x112 (0.3-cell jitter), "
                        "tol 1e-5 x bbox diagonal of A")
    for name, pr, k in (("mixed", hd.HD_MIXED, args.steps), ("fp64", hd.HD_FP64, max(3, args.steps // 4))):
        o = options(pr)
        for _ in range(3):
            step(p, d, o)
        ts, rs = timed(p, d, o, k)
        out[name] = dict(value=world * k / (multi.max_over_ranks(sum(ts), device=dev) / 1e3), unit=UNIT,
                         ms_per_step=sum(ts) / k, lower=rs[-1]["lower"], upper=rs[-1]["upper"])
    return out


def batched_pairs(args, torch, hd, dev, prec):
    """The batched workload: `n` pairs (1K-200K triangles a side, tol 1e-4 dA) in one batched
    call, against the same pairs run one after another in FP64; device-resident inputs, times
    from CUDA events on the current stream (BVH builds timed apart)."""
    n = args.batch_pairs
    pairs = mg.batch_workload(n)
    dev_pairs = [tuple(torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (q.VA, q.FA, q.VB, q.FB))
                 for q in pairs]
    tol = pairs[0].tol

    def ev_time(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    ob = hd.hd_options_default()
    t_build, bvhs = ev_time(lambda: [hd.hd_build_B(VB, FB, ob) for (_, _, VB, FB) in dev_pairs])
    As = [(VA, FA) for (VA, FA, _, _) in dev_pairs]
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec)
    hd.hd_hausdorff_batched(bvhs, As, tol, o)  # warm-up
    best, rs = None, None
    for _ in range(2):
        t, rr = ev_time(lambda: hd.hd_hausdorff_batched(bvhs, As, tol, o))
        if best is None or t < best:
            best, rs = t, rr
    ok = sum(r["status"] == hd.HD_OK for r in rs)
    statuses = {}
    for r in rs:
        statuses[r["status_str"]] = statuses.get(r["status_str"], 0) + 1
    # the same pairs as single runs on host threads with a stream each (HD_FLAG_BATCH_STREAMS)
    ost = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec, flags=hd.HD_FLAG_BATCH_STREAMS)
    t_st, r_st = ev_time(lambda: hd.hd_hausdorff_batched(bvhs, As, tol, ost))
    o64 = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_FP64)
    t64, r64 = ev_time(lambda: [hd.hd_hausdorff(b, VA, FA, tol, o64) for b, (VA, FA) in zip(bvhs, As)])
    ok64 = sum(r["status"] == hd.HD_OK for r in r64)
    nf = sum(len(q.FA) + len(q.FB) for q in pairs)
    return dict(workload=f"{n} pairs of the batched workload (triangles per side log-uniform in [1K, 200K], "
                         f"{nf:,} in total), tol 1e-4 x bbox diagonal of each A",
                batched_mixed=dict(value=n / best, unit=UNIT, seconds=best, ok=ok, statuses=statuses,
                                   rounds=max(r["stats"]["rounds"] for r in rs),
                                   splits=sum(r["stats"]["splits"] for r in rs),
                                   kernel_launches=rs[0]["stats"]["kernel_launches"]),
                streams_mixed=dict(value=n / t_st, unit=UNIT, seconds=t_st,
                                   ok=sum(r["status"] == hd.HD_OK for r in r_st),
                                   splits=sum(r["stats"]["splits"] for r in r_st),
                                   peak_frontier_sum=sum(r["stats"]["peak_frontier"] for r in r_st),
                                   rounds_max=max(r["stats"]["rounds"] for r in r_st),
                                   note="single runs on host threads, one stream each (HD_FLAG_BATCH_STREAMS)"),
                batched_mixed_with_builds=dict(value=n / (best + t_build), unit=UNIT, build_seconds=t_build),
                sequential_fp64=dict(value=n / t64, unit=UNIT, seconds=t64, ok=ok64),
                speedup_vs_sequential_fp64=t64 / best)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
