"""The autotuner on a 4-pair sample of the batched workload (reduced sizes): it times every
candidate option set on the GPU and returns the fastest; the options it chooses must give
brackets within eps that meet the oracle's for every pair of the sample."""
import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _dA(V, F):
    R = np.asarray(V, float)[np.unique(np.asarray(F).ravel())]
    return float(np.linalg.norm(R.max(0) - R.min(0)))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_choice_gives_oracle_brackets(orc, precision):
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd
    from paper_2406_10357_gb300.autotune import autotune, candidates

    pairs = mg.batch_workload(n_pairs=4, lo=300, hi=3000)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    sample = [(t(p.VA), t(p.FA), t(p.VB), t(p.FB)) for p in pairs]
    prec = hd.HD_MIXED if precision == "mixed" else hd.HD_FP64
    opt, table = autotune(sample, pairs[0].tol, prec, reps=1)
    assert len(table) == len(candidates()) and all(r["seconds"] > 0 for r in table)
    best = min((r for r in table if r["all_ok"]), key=lambda r: r["seconds"])
    assert (opt.block_size, opt.leaf_size, opt.frontier_chunk) == (best["block_size"], best["leaf_size"],
                                                                   best["frontier_chunk"])
    bvhs = [hd.hd_build_B(p.VB, p.FB, hd.hd_options_default(leaf_size=opt.leaf_size)) for p in pairs]
    rs = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], pairs[0].tol, opt)
    for p, r in zip(pairs, rs):
        eps = p.tol * _dA(p.VA, p.FA)
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
        assert r["status"] == hd.HD_OK, (p.name, r)
        assert r["upper"] - r["lower"] <= eps * (1 + 1e-12)
        assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + 1e-12 * eps, p.name
