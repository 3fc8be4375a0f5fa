"""Host-side scheduling logic of the serving loop (no GPU): admission and tick
planning (shortest remaining work first, budgeted by multiply-adds)."""
from paper_1805_04463_gb300.serve import Request, admit_ok, item_cost, plan_tick


def _req(rid, n, total, nxt=0):
    r = Request(rid, 0, n, rid, 0.0)
    r.total_items, r.next_item = total, nxt
    r.bitset_bytes, r.operand_bytes = n * n // 8, 2 * n * n
    return r


def test_admission_budgets_and_slots():
    r = _req(0, 65536, 100)
    assert admit_ok(r, 0, 0, 0, 60e9, 150e9, 4)
    assert not admit_ok(r, 60e9 - r.bitset_bytes + 1, 0, 0, 60e9, 150e9, 4)     # bitset budget
    assert not admit_ok(r, 0, 150e9 - r.operand_bytes + 1, 0, 60e9, 150e9, 4)   # operand budget
    assert not admit_ok(r, 0, 0, 4, 60e9, 150e9, 4)                             # slots
    assert admit_ok(r, 60e9 - r.bitset_bytes, 150e9 - r.operand_bytes, 3, 60e9, 150e9, 4)


def test_plan_tick_shortest_remaining_first_and_budget():
    small, big = _req(1, 1024, 10), _req(2, 65536, 1000)
    c_small, c_big = item_cost(1024, 10), item_cost(65536, 1000)
    grants = plan_tick([big, small], budget_macs=c_small * 10 + c_big * 5)
    assert [g[0].rid for g in grants] == [1, 2]               # small one first
    assert grants[0][1:] == (0, 10)                            # whole small request
    assert grants[1][1:] == (0, 5)                             # the rest of the budget to the big one


def test_plan_tick_always_progresses_and_respects_cursor():
    big = _req(2, 65536, 1000, nxt=998)
    grants = plan_tick([big], budget_macs=1.0)                 # budget smaller than one item
    assert grants == [(big, 998, 999)]
    done = _req(3, 2048, 5, nxt=5)
    assert plan_tick([done], budget_macs=1e15) == []
