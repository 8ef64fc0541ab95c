"""Host logic of the parameter sweeps (no GPU work)."""
from paper_2406_10357_gb300 import sweep


def test_all_orders_are_the_64_ordered_subsets():
    orders = sweep.all_orders()
    assert len(orders) == 64 and len(set(orders)) == 64
    assert all(1 <= len(o) <= 4 and len(set(o)) == len(o) and set(o) <= {1, 2, 3, 4} for o in orders)
    assert (1, 2, 3, 4) in orders and (4,) in orders and (3, 1) in orders
