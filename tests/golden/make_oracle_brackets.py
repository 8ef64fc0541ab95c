"""Oracle brackets of the large parity cases, computed once on the CPU and stored.

The FP64 oracle (``oracle/``, brute-force distances) needs from seconds to minutes for the
full-size benchmark pair, the large soup at 1/16 of its face count and the first 32 pairs of
the batched workload.  This script runs it on those inputs and writes
``oracle_brackets.json`` beside it; the GPU parity tests read a stored bracket only when the
input they regenerate has the same SHA-256 digest as the one the bracket was computed on,
and run the oracle themselves otherwise (another machine's libm may round a generated
coordinate differently).  Nothing here touches the CUDA library.

Each entry records the oracle's bracket [lower, upper], its status, the tolerance it ran at
and how long it took.  A batched pair whose oracle run at the workload's own tolerance
(1e-4 of A's bbox diagonal) does not finish within the wall budget is run again with the
paper's face cap m (Section 4: at most m n_A sub-triangles) set so that the run fits the
budget: the oracle then stops with CAPACITY and a bracket wider than eps, which still
contains h, so the GPU bracket must still meet it.  The entry records the cap
(``max_face_factor``); every split costs three brute-force queries against all of B, which
is what makes the oracle slow on a coarse A against a fine B.

    python tests/golden/make_oracle_brackets.py [--only KEY ...] [--budget SECONDS]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_brackets.json")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BATCH_PAIRS = 32
BUDGET_S = 240.0
EVALS_PER_S = 1e7  # brute-force point-triangle tests per second of one split's three queries


def digest(p) -> str:
    """SHA-256 of the pair's four arrays as the parity tests pass them."""
    h = hashlib.sha256()
    for a in (p.VA, p.FA, p.VB, p.FB):
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


def cases():
    """(key, builder) of every stored case; the builder regenerates the seeded input."""
    import meshgen as mg

    out = [("w2_full", lambda: mg.workload(2)),
           ("w5_1_16", lambda: mg.workload(5, 1 / 16)),
           ("w3_0.05", lambda: mg.workload(3, 0.05))]
    for i in range(BATCH_PAIRS):
        out.append((f"w4_pair{i}", (lambda i=i: mg.batch_workload(i + 1)[i])))
    return out


def _run(args):
    key, tol, m, q = args
    import oracle

    p = dict(cases())[key]()
    t = time.perf_counter()
    r = oracle.hausdorff(p.VA, p.FA, p.VB, p.FB, tol, p.tol_mode, max_face_factor=m)
    q.put(dict(lower=r["lower"], upper=r["upper"], status=r["status"], seconds=time.perf_counter() - t,
               splits=int(r["stats"]["splits"])))


def run_one(key, tol, budget, m=1e7):
    """The oracle on case `key` at `tol` (face cap m) in a child process, killed after
    `budget` seconds."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_run, args=((key, tol, m, q),))
    proc.start()
    proc.join(budget)
    if proc.is_alive():
        proc.kill()
        proc.join()
        return None
    return q.get() if not q.empty() else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*")
    ap.add_argument("--budget", type=float, default=BUDGET_S)
    a = ap.parse_args()
    import oracle

    oracle.build()
    table = json.load(open(OUT)) if os.path.exists(OUT) else {"about": __doc__.split("\n\n")[0], "cases": {}}
    for key, make in cases():
        if a.only and key not in a.only:
            continue
        p = make()
        entry = None
        # the uncapped run, then caps that allow about (budget / 2) x EVALS_PER_S / (3 n_B)
        # splits, then a quarter of that
        splits = 0.5 * a.budget * EVALS_PER_S / (3 * len(p.FB))
        for m in (1e7, 1 + 4 * splits / len(p.FA), 1 + splits / len(p.FA)):
            r = run_one(key, p.tol, a.budget, m)
            if r is not None:
                entry = dict(r, tol=p.tol, tol_mode=p.tol_mode, max_face_factor=m, name=p.name,
                             sizes=list(p.sizes), digest=digest(p), threads=oracle.num_threads(),
                             budget_s=a.budget)
                break
        if entry is None:
            print(f"{key}: no oracle bracket within {a.budget} s even with the face cap", flush=True)
            continue
        print(key, json.dumps(entry), flush=True)
        # merge into the file as it is now (another run of this script may have added entries)
        table = json.load(open(OUT)) if os.path.exists(OUT) else table
        table["cases"][key] = entry
        tmp = OUT + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, OUT)


def stored(key: str, p):
    """The stored oracle entry for case `key` if `p` is the input it was computed on, else None."""
    if not os.path.exists(OUT):
        return None
    e = json.load(open(OUT))["cases"].get(key)
    if e is None or e["digest"] != digest(p):
        return None
    return e


if __name__ == "__main__":
    main()
