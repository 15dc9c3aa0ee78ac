"""Host logic of the continuous-batching server, on CPU with a fake device
backend and a simulated clock: arrival-order admission within capacity and
budget, retirement at tolerance or step cap, latency accounting."""
import dataclasses

import pytest

from paper_1503_03337_gb300 import inputs
from paper_1503_03337_gb300.serving import Busy, Server, summarize


class FakeStats:
    def __init__(self, step, prev, res):
        self.step, self.prev_step = step, prev
        self.sum_abs_u = (1.0, 0.0, 0.0)
        self.sum_abs_du = (res, 0.0, 0.0)
        self.sum_u = (0.0, 0.0, 0.0)
        self.sum_P = 0.0
        self.max_abs_u = 0.0
        self.nonfinite = 0


class FakeBackend:
    """Residual of a domain = 10^(-steps / decay); the clock advances by the
    cell updates done (1 update per ns)."""

    def __init__(self, capacity, budget_cells, clock):
        self.capacity, self.budget, self.clock = capacity, budget_cells, clock
        self.slots = {}
        self.max_active = 0
        self.admitted = []

    def add(self, case):
        used = sum(c.cells for c, _ in self.slots.values())
        if len(self.slots) >= self.capacity or used + case.cells > self.budget:
            raise Busy()
        slot = min(set(range(self.capacity)) - set(self.slots))
        self.slots[slot] = (case, 0)
        self.max_active = max(self.max_active, len(self.slots))
        self.admitted.append(case.name)
        return slot

    def remove(self, slot):
        del self.slots[slot]

    def step(self, n, chunk):
        for s, (c, k) in self.slots.items():
            self.slots[s] = (c, k + n)
        self.clock.t += n * sum(c.cells for c, _ in self.slots.values()) * 1e-9

    def reductions(self):
        out = {}
        for s, (c, k) in self.slots.items():
            decay = float(c.name.split(":")[1])
            out[s] = FakeStats(k, k - 100 if k > 100 else -1, 10 ** (-k / decay))
        self.last = out
        return out

    def residual(self, slot):
        st = self.last[slot]
        return st.sum_abs_du[0] / st.sum_abs_u[0]


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


def make_trace(n, rate=50.0, seed=1):
    tr = inputs.request_trace(n, rate=rate, seed=seed, lmin=16, lmax=48, max_steps=3000)
    return tr


def case_of(r):
    c = inputs.cavity(r.Q, r.L, 400.0)
    # encode a per-request convergence speed in the name (steps per decade)
    c.name = "req%d:%d" % (r.rid, 150 + 40 * (r.rid % 7))
    return c


@pytest.mark.parametrize("capacity", (1, 3, 8))
def test_server_admits_in_order_and_completes(capacity):
    clock = Clock()
    be = FakeBackend(capacity, budget_cells=10 ** 9, clock=clock)
    trace = make_trace(30)
    srv = Server(be, check_every=100, tol=1e-8, case_of=case_of, clock=clock, sleep=clock.sleep)
    out = srv.run(trace)
    assert len(out) == 30 and be.max_active <= capacity
    order = [int(n.split(":")[0][3:]) for n in be.admitted]
    arrivals = {r.rid: r.arrival for r in trace}
    assert [arrivals[i] for i in order] == sorted(arrivals[i] for i in order)
    for r in trace:
        o = out[r.rid]
        assert r.arrival <= o.admitted <= o.done
        assert o.steps % 100 == 0 and 0 < o.steps <= r.max_steps
        decay = 150 + 40 * (r.rid % 7)
        # retires at the first check whose residual is <= 1e-8, or at the cap
        first = next((k for k in range(200, r.max_steps + 1, 100) if 10 ** (-k / decay) <= 1e-8),
                     r.max_steps)
        assert o.steps == first
    s = summarize(out, clock.t)
    assert s["p99_s"] >= s["p50_s"] > 0


def test_budget_limits_concurrency():
    clock = Clock()
    trace = make_trace(12, rate=1e6)  # all arrive at once
    cells = [case_of(r).cells for r in trace]
    budget = int(2.5 * max(cells))
    be = FakeBackend(64, budget_cells=budget, clock=clock)
    Server(be, case_of=case_of, clock=clock, sleep=clock.sleep).run(trace)
    assert be.max_active >= 2
    assert be.max_active < 12


def test_saturation_budget_limits_admission():
    clock = Clock()
    trace = make_trace(16, rate=1e6)
    be = FakeBackend(64, 10 ** 9, clock)
    cells = [case_of(r).cells for r in trace]
    cap = int(1.5 * max(cells))
    srv = Server(be, case_of=case_of, clock=clock, sleep=clock.sleep, max_active_cells=cap)
    out = srv.run(trace)
    assert len(out) == 16
    # never more cells active than the cap, except a single oversized domain
    assert be.max_active >= 1
