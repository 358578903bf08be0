"""Host logic of the serving loop (admission by slots and memory budget,
FCFS with backfill, arrival times, error propagation), with a fake executor:
no GPU involved."""
import threading
import time

import pytest

from paper_2604_23979_gb300.serve import Scheduler


class Tracker:
    def __init__(self, costs, hold):
        self.costs = costs
        self.hold = hold
        self.lock = threading.Lock()
        self.running = 0
        self.used = 0
        self.max_running = 0
        self.max_used = 0
        self.slots_seen = set()
        self.order = []

    def __call__(self, i, slot):
        with self.lock:
            self.running += 1
            self.used += self.costs[i]
            self.max_running = max(self.max_running, self.running)
            self.max_used = max(self.max_used, self.used)
            self.slots_seen.add(slot)
            self.order.append(i)
        time.sleep(self.hold[i] if isinstance(self.hold, list) else self.hold)
        with self.lock:
            self.running -= 1
            self.used -= self.costs[i]


def test_slots_bound_concurrency():
    costs = [1] * 6
    tr = Tracker(costs, 0.05)
    admit, done, maxc = Scheduler(2, 100).run([0.0] * 6, costs, tr)
    assert tr.max_running <= 2 and maxc <= 2
    assert tr.slots_seen <= {0, 1}
    assert all(d > a for a, d in zip(admit, done))
    assert sorted(tr.order) == list(range(6))


def test_memory_budget_bounds_concurrency():
    costs = [60, 60, 30, 30, 60]
    tr = Tracker(costs, 0.05)
    Scheduler(4, 100).run([0.0] * 5, costs, tr)
    assert tr.max_used <= 100
    assert sorted(tr.order) == list(range(5))


def test_backfill_passes_a_blocked_head():
    # 0 (cost 90) runs; 1 (cost 50) cannot fit; 2 (cost 10) arrives later but fits
    costs = [90, 50, 10]
    tr = Tracker(costs, [0.3, 0.05, 0.05])
    admit, done, _ = Scheduler(4, 100).run([0.0, 0.01, 0.02], costs, tr)
    assert admit[2] < admit[1]
    assert admit[1] >= done[0] - 1e-3


def test_arrivals_are_honoured_and_fcfs_when_unconstrained():
    arrivals = [0.0, 0.05, 0.10, 0.15]
    costs = [1] * 4
    tr = Tracker(costs, 0.01)
    admit, done, _ = Scheduler(1, 10).run(arrivals, costs, tr)
    assert all(a >= t - 1e-3 for a, t in zip(admit, arrivals))
    assert tr.order == [0, 1, 2, 3]


def test_worker_error_is_raised():
    def boom(i, slot):
        if i == 1:
            raise RuntimeError("device step failed")
        time.sleep(0.01)

    with pytest.raises(RuntimeError, match="device step failed"):
        Scheduler(2, 10).run([0.0, 0.0, 0.0], [1, 1, 1], boom)


def test_request_larger_than_budget_is_rejected():
    with pytest.raises(ValueError):
        Scheduler(2, 10).run([0.0], [11], lambda i, s: None)


def test_measured_charge_frees_budget_for_the_queue():
    """A request admitted on an upper-bound estimate that recharges itself
    with its measured footprint lets a waiting request start while it runs;
    without the recharge the second request waits for the first to end."""
    def run(recharge):
        sched = Scheduler(4, 100)
        started = {}

        def execute(i, slot):
            started[i] = time.perf_counter()
            if i == 0:
                if recharge:
                    sched.recharge(0, 30)
                time.sleep(0.4)
            else:
                time.sleep(0.05)

        t0 = time.perf_counter()
        admit, done, maxc = sched.run([0.0, 0.02], [90, 60], execute)
        return admit, done, maxc

    admit, done, maxc = run(True)
    assert maxc == 2 and admit[1] < done[0]
    admit, done, maxc = run(False)
    assert maxc == 1 and admit[1] >= done[0]


def test_recharge_above_the_estimate_holds_back_the_queue():
    """A measured footprint larger than the estimate is charged in full."""
    sched = Scheduler(4, 100)

    def execute(i, slot):
        if i == 0:
            sched.recharge(0, 95)
            time.sleep(0.3)
        else:
            time.sleep(0.02)

    admit, done, maxc = sched.run([0.0, 0.05], [40, 40], execute)
    assert maxc == 1 and admit[1] >= done[0]
