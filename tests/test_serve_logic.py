"""Host-side scheduling logic of the continuous-batching server, on a fake batch
(no GPU): admission by footprint, FIFO with backfill, joining at block boundaries,
retirement when the step count is reached, latency accounting."""
import numpy as np
import pytest

from paper_2502_10640_gb300 import capi, serve


class FakeBatch:
    """Records the calls the server makes; footprint = 100 bytes per particle."""

    def __init__(self, budget, graph_block=None):
        self.budget = budget
        self.slots = {}
        self.log = []
        self.clock = None

    def info(self):
        return {"active": len(self.slots), "bytes_used": sum(100 * n for n, _ in self.slots.values()),
                "budget": self.budget}

    def add(self, pos, w, dt, eps, vel=None):
        slot = next(i for i in range(1000) if i not in self.slots)
        self.slots[slot] = (pos.shape[0], 0)
        self.log.append(("add", slot, pos.shape[0]))
        return slot

    def step(self, k):
        self.log.append(("step", k, sorted(self.slots)))
        self.slots = {s: (n, st + k) for s, (n, st) in self.slots.items()}
        self.clock.t += 0.01 * k

    def state(self, slot, n):
        st = self.slots[slot][1]
        return np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)), st

    def diagnostics(self, slot):
        return {"step": self.slots[slot][1]}

    def remove(self, slot):
        self.log.append(("remove", slot))
        del self.slots[slot]

    def close(self):
        pass


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


@pytest.fixture
def fake(monkeypatch):
    clock = FakeClock()
    made = []

    def make_batch(budget, graph_block=None):
        b = FakeBatch(budget, graph_block)
        b.clock = clock
        made.append(b)
        return b
    monkeypatch.setattr(capi, "Batch", make_batch)
    monkeypatch.setattr(capi, "pp_batch_footprint", lambda n: 100 * n)
    return clock, made


def req(rid, arrival, n, steps):
    return serve.ServeRequest(rid, arrival, n, 1.0, 1e-15, 0.0, steps, np.zeros((n, 3)))


def test_fifo_admission_backfill_and_block_boundaries(fake):
    clock, made = fake
    srv = serve.Server(budget_bytes=100 * 100, block_steps=8, clock=clock, sleep=clock.sleep)
    trace = [req(0, 0.0, 60, 20), req(1, 0.0, 60, 5), req(2, 0.0, 30, 3), req(3, 0.5, 10, 1)]
    rep = srv.run(trace)
    b = made[0]
    # 0 fits (60); 1 does not (120 > 100) and waits; 2 backfills (90)
    assert b.log[0] == ("add", 0, 60) and b.log[1] == ("add", 1, 30)
    # first block is cut at the shortest remaining count (3 steps)
    assert b.log[2] == ("step", 3, [0, 1])
    assert rep["completed"] == 4 and rep["rejected"] == 0
    done = {r.rid: r for r in srv.results}
    assert all(done[i].steps == trace[i].steps for i in range(4))
    assert done[1].admitted >= done[2].completed          # 1 joined after 2 left
    assert rep["p50_latency_s"] <= rep["p99_latency_s"] <= rep["max_latency_s"]
    assert rep["pairs"] == sum(r.n ** 2 * r.steps for r in trace)


def test_without_backfill_the_queue_is_strict_fifo(fake):
    clock, made = fake
    srv = serve.Server(budget_bytes=100 * 100, block_steps=8, backfill=False, clock=clock,
                       sleep=clock.sleep)
    srv.run([req(0, 0.0, 60, 4), req(1, 0.0, 60, 4), req(2, 0.0, 30, 4)])
    adds = [e for e in made[0].log if e[0] == "add"]
    assert [a[2] for a in adds] == [60, 60, 30]             # 2 waited behind 1


def test_request_larger_than_the_budget_is_rejected(fake):
    clock, made = fake
    srv = serve.Server(budget_bytes=100 * 50, clock=clock, sleep=clock.sleep)
    rep = srv.run([req(0, 0.0, 60, 4), req(1, 0.0, 20, 4)])
    assert rep["rejected"] == 1 and rep["completed"] == 1 and srv.rejected == [0]


def test_idle_server_waits_for_the_next_arrival(fake):
    clock, made = fake
    srv = serve.Server(budget_bytes=10 ** 6, clock=clock, sleep=clock.sleep)
    rep = srv.run([req(0, 2.0, 10, 2)])
    assert rep["completed"] == 1
    assert srv.results[0].admitted >= 2.0


def test_percentile_nearest_rank():
    assert serve.percentile([3, 1, 2], 50) == 2
    assert serve.percentile(list(range(1, 101)), 99) == 99
    assert serve.percentile([5.0], 99) == 5.0


def test_cancel_waiting_and_running_requests(fake):
    clock, made = fake
    srv = serve.Server(budget_bytes=100 * 100, block_steps=4, clock=clock, sleep=clock.sleep)
    trace = [req(0, 0.0, 60, 40), req(1, 0.0, 60, 4), req(2, 0.0, 10, 8), req(3, 5.0, 10, 4)]

    def after_block(s):
        if s.blocks == 1:
            s.cancel(0)          # running: removed at this boundary, its memory freed
            s.cancel(1)          # waiting for memory: dropped
            s.cancel(3)          # not arrived yet: dropped on arrival
    rep = srv.run(trace, on_block=after_block)
    b = made[0]
    assert sorted(srv.cancelled) == [0, 1, 3]
    assert rep["cancelled"] == 3 and rep["completed"] == 1
    assert [r.rid for r in srv.results] == [2]
    assert ("remove", 0) in b.log
    assert all(e[2] != 60 or e[1] == 0 for e in b.log if e[0] == "add")   # 1 never admitted
