"""Host-side serving logic (no device): which requests a turn advances.

serve.select_turn implements the shortest-remaining-work-first turns of the
continuous-batching server: every admitted request when no work target is
set; otherwise requests in increasing remaining work until the turn holds the
target number of point-updates, plus any request not advanced for longer
than the aging limit.
"""
from paper_2502_09537_b300.serve import select_turn


def test_no_target_advances_everything():
    items = [(3, 100, 50, 0.0), (0, 10, 5, 0.0), (7, 1000, 1, 0.0)]
    assert select_turn(items, 10, 0.0, 5.0, 1.0) == [3, 0, 7]


def test_shortest_remaining_work_first_up_to_the_target():
    # remaining work: inst 1: 10*5=50, inst 2: 100*2=200, inst 3: 1000*1=1000, inst 4: 100*50=5000
    items = [(4, 100, 50, 0.0), (3, 1000, 1, 0.0), (2, 100, 2, 0.0), (1, 10, 5, 0.0)]
    # quantum 10: turn work of 1 = 10*5 = 50, of 2 = 100*2 = 200 -> 250 >= 220 stops there
    assert select_turn(items, 10, 220.0, 5.0, 1.0) == [1, 2]
    assert select_turn(items, 10, 1e9, 5.0, 1.0) == [1, 2, 3, 4]
    assert select_turn(items, 10, 1.0, 5.0, 1.0) == [1]


def test_aging_limit_lets_waiting_requests_in():
    items = [(1, 10, 5, 9.0), (2, 100, 2, 9.0), (4, 100, 50, 2.0)]
    # instance 4 last advanced at t = 2; at t = 9 it has waited 7 > 5 s
    assert select_turn(items, 10, 1.0, 5.0, 9.0) == [1, 4]


def test_ties_are_broken_by_instance():
    items = [(5, 10, 10, 0.0), (2, 10, 10, 0.0), (9, 10, 10, 0.0)]
    assert select_turn(items, 10, 100.0, 5.0, 0.0) == [2]
    assert select_turn(items, 10, 150.0, 5.0, 0.0) == [2, 5]
