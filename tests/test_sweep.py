"""Host logic of the parameter sweeps (no GPU work)."""
from paper_2406_10357_gb300 import sweep


def test_all_orders_are_the_64_ordered_subsets():
    orders = sweep.all_orders()
    assert len(orders) == 64 and len(set(orders)) == 64
    assert all(1 <= len(o) <= 4 and len(set(o)) == len(o) and set(o) <= {1, 2, 3, 4} for o in orders)
    assert (1, 2, 3, 4) in orders and (4,) in orders and (3, 1) in orders


def test_autotune_candidates_cover_the_grid():
    from paper_2406_10357_gb300 import autotune as at

    c = at.candidates()
    assert len(c) == len(at.BLOCK_SIZES) * len(at.LEAF_SIZES) * len(at.CHUNKS)
    assert all(x["bound_order"] == (1, 2, 3, 4) for x in c)  # the paper's order unless asked
    assert len(at.candidates(tune_order=True)) == len(c) * len(at.ORDERS)
    assert {x["block_size"] for x in c} == set(at.BLOCK_SIZES) and {x["leaf_size"] for x in c} == set(at.LEAF_SIZES)
