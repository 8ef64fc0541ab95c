"""Timed sweeps over the method's parameters, on one GPU.

orders -- every cascade order of every non-empty subset of {u1, u2, u3, u4} (64 orders; the
          paper compares cascades in Section 5), timed on a batch of workload-4 pairs.
tol    -- runtime against the tolerance, from 1e-1 to 1e-8 relative (the paper's runtime
          versus epsilon study, Section 5), on workloads 2 and 5.
batch  -- workload 4: the batched call untuned and autotuned (MIXED), the host-thread stream
          path, the batched call in FP64, and sequential per-pair calls in FP64, all at the
          same tolerance.
run    -- one workload at its own tolerance: a warm-up call, then timed calls (the command the
          kernel profiles of a workload are taken with).

    python -m paper_2406_10357_gb300.sweep orders [--pairs 64] [--precision mixed]
    python -m paper_2406_10357_gb300.sweep tol [--workloads 2 5] [--scale 1.0]
    python -m paper_2406_10357_gb300.sweep batch [--pairs 1024] [--tune-pairs 32]
    python -m paper_2406_10357_gb300.sweep run --workloads 3 [--scale 0.05] [--reps 1]

Each line printed is one JSON record; the inputs are the seeded synthetic workloads of
``meshgen``.
"""
from __future__ import annotations

import argparse
import itertools
import json
import time


def all_orders():
    """The 64 cascade orders: every permutation of every non-empty subset of the four bounds."""
    return [o for k in range(1, 5) for o in itertools.permutations((1, 2, 3, 4), k)]


def _timed(fn, reps: int):
    import torch

    fn()  # warm-up
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    ts.sort()
    return ts[len(ts) // 2], out


def sweep_orders(n_pairs: int, precision: int, reps: int = 3):
    import torch

    import meshgen as mg
    import paper_2406_10357_gb300 as hd

    pairs = mg.batch_workload(n_pairs=n_pairs)
    dev = [(torch.from_numpy(p.VA).cuda(), torch.from_numpy(p.FA).cuda()) for p in pairs]
    bvhs = [hd.hd_build_B(torch.from_numpy(p.VB).cuda(), torch.from_numpy(p.FB).cuda()) for p in pairs]
    for order in all_orders():
        o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=precision, bound_order=order)
        t, rs = _timed(lambda: hd.hd_hausdorff_batched(bvhs, dev, pairs[0].tol, o), reps)
        st = [r["stats"] for r in rs]
        yield dict(sweep="orders", order=list(order), pairs=n_pairs, seconds=t, pairs_per_s=n_pairs / t,
                   ok=sum(r["status"] == hd.HD_OK for r in rs), splits=sum(s["splits"] for s in st),
                   pointtri_evals=sum(s["pointtri_evals"] for s in st),
                   discards={k: sum(s["discards"][k] for s in st) for k in st[0]["discards"]})


def sweep_tol(workloads, scale: float, precision: int, reps: int = 3):
    import torch

    import meshgen as mg
    import paper_2406_10357_gb300 as hd

    for k in workloads:
        p = mg.workload(k, scale)
        VA, FA = torch.from_numpy(p.VA).cuda(), torch.from_numpy(p.FA).cuda()
        bvh = hd.hd_build_B(torch.from_numpy(p.VB).cuda(), torch.from_numpy(p.FB).cuda())
        for e in range(1, 9):
            tol = 10.0 ** -e
            o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=precision)
            t, r = _timed(lambda: hd.hd_hausdorff(bvh, VA, FA, tol, o), reps)
            yield dict(sweep="tol", workload=k, scale=scale, faces_A=len(p.FA), faces_B=len(p.FB), tol=tol,
                       seconds=t, lower=r["lower"], upper=r["upper"], status=r["status_str"],
                       rounds=r["stats"]["rounds"], splits=r["stats"]["splits"],
                       pointtri_evals=r["stats"]["pointtri_evals"])


def sweep_batch(n_pairs: int, tune_pairs: int, reps: int = 2):
    """Workload 4: the batched call untuned and autotuned (MIXED), against sequential per-pair
    calls in FP64, all at the same tolerance."""
    import torch

    import meshgen as mg
    import paper_2406_10357_gb300 as hd
    from paper_2406_10357_gb300 import autotune as at

    pairs = mg.batch_workload(n_pairs=n_pairs)
    dev = [tuple(torch.from_numpy(x).cuda() for x in (p.VA, p.FA, p.VB, p.FB)) for p in pairs]
    tol = pairs[0].tol
    t0 = time.perf_counter()
    opt_t, table = at.autotune(dev[:tune_pairs], tol, hd.HD_MIXED, tune_order=False)
    t_tune = time.perf_counter() - t0
    best = min(table, key=lambda r: r["seconds"])
    yield dict(sweep="batch", what="autotune", tune_pairs=tune_pairs, seconds=t_tune, candidates=len(table),
               best={k: best[k] for k in ("block_size", "leaf_size", "frontier_chunk", "bound_order")})

    def run(opt, leaf, batched):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bvhs = [hd.hd_build_B(VB, FB, hd.hd_options_default(leaf_size=leaf)) for (_, _, VB, FB) in dev]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if batched:
            rs = hd.hd_hausdorff_batched(bvhs, [(VA, FA) for (VA, FA, _, _) in dev], tol, opt)
        else:
            rs = [hd.hd_hausdorff(b, VA, FA, tol, opt) for b, (VA, FA, _, _) in zip(bvhs, dev)]
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, sum(r["status"] == hd.HD_OK for r in rs)

    arms = [("batched MIXED, untuned", hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_MIXED), 1, True),
            ("batched MIXED, autotuned", opt_t, best["leaf_size"], True),
            ("MIXED single runs on host-thread streams",
             hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_MIXED, flags=hd.HD_FLAG_BATCH_STREAMS), 1,
             True),
            ("batched FP64", hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_FP64), 1, True),
            ("sequential per-pair FP64", hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_FP64), 1, False)]
    for name, opt, leaf, batched in arms:
        res = [run(opt, leaf, batched) for _ in range(reps)]
        tb, tr, ok = min(res, key=lambda x: x[1])
        yield dict(sweep="batch", what=name, pairs=n_pairs, build_seconds=tb, run_seconds=tr, pairs_per_s=n_pairs / tr,
                   pairs_per_s_with_build=n_pairs / (tb + tr), ok=ok)


def run_workloads(workloads, scale: float, precision: int, reps: int, frontier_bytes: int):
    import torch

    import meshgen as mg
    import paper_2406_10357_gb300 as hd

    for k in workloads:
        p = mg.workload(k, scale)
        VA, FA = torch.from_numpy(p.VA).cuda(), torch.from_numpy(p.FA).cuda()
        bvh = hd.hd_build_B(torch.from_numpy(p.VB).cuda(), torch.from_numpy(p.FB).cuda())
        o = hd.hd_options_default(tol_mode=p.tol_mode, precision=precision, max_frontier_bytes=frontier_bytes)
        t, r = _timed(lambda: hd.hd_hausdorff(bvh, VA, FA, p.tol, o), reps)
        yield dict(sweep="run", workload=k, scale=scale, faces_A=len(p.FA), faces_B=len(p.FB), tol=p.tol,
                   seconds=t, lower=r["lower"], upper=r["upper"], status=r["status_str"], stats=r["stats"])


def main(argv=None):
    import paper_2406_10357_gb300 as hd

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("what", choices=["orders", "tol", "batch", "run"])
    ap.add_argument("--tune-pairs", type=int, default=32)
    ap.add_argument("--pairs", type=int, default=64)
    ap.add_argument("--workloads", type=int, nargs="+", default=[2, 5])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--frontier-bytes", type=int, default=0, help="run: max_frontier_bytes (0: the default)")
    a = ap.parse_args(argv)
    prec = hd.HD_MIXED if a.precision == "mixed" else hd.HD_FP64
    if a.what == "orders":
        rows = sweep_orders(a.pairs, prec, a.reps)
    elif a.what == "tol":
        rows = sweep_tol(a.workloads, a.scale, prec, a.reps)
    elif a.what == "run":
        rows = run_workloads(a.workloads, a.scale, prec, a.reps, a.frontier_bytes)
    else:
        rows = sweep_batch(a.pairs, a.tune_pairs, a.reps)
    for row in rows:
        row["precision"] = a.precision
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
