"""Scheduling logic of the continuous-batching server, with a fake executor (no GPU)."""
import pytest

from paper_2606_29129_gb300.serve import Request, Server

CAL = {c: {"k": 0, "cublas": 1e-13, "N": {12: 1e-9, 14: 1e-12, 16: 1e-14, 18: 1e-16}}
       for c in range(9)}


class FakeExecutor:
    """Slots whose batches finish after a fixed number of polls."""

    def __init__(self, slots=2, slot_workspace=10_000, latency=3):
        self._slots = slots
        self.slot_workspace = slot_workspace
        self.latency = latency
        self.batches = []
        self.live = set()

    def slots(self):
        return range(self._slots)

    def workspace_bytes(self, reqs):
        return sum(r.num_moduli * (r.m + r.n) for r in reqs)

    def admit(self, r):
        self.live.add(r.rid)

    def launch(self, slot, reqs):
        assert self.workspace_bytes(reqs) <= self.slot_workspace
        token = {"left": self.latency, "slot": slot, "reqs": [r.rid for r in reqs]}
        self.batches.append(token)
        return token

    def poll(self, token):
        token["left"] -= 1
        return token["left"] <= 0

    def finish(self, token, reqs):
        for r in reqs:
            r.C = ("result", r.rid)

    def release(self, r):
        self.live.discard(r.rid)


def make(rid, m=10, n=10, k=10, target=None):
    return Request(rid=rid, m=m, n=n, k=k, target=target, arrival=float(rid) + 1.0)


def test_all_requests_finish_within_budget():
    ex = FakeExecutor()
    srv = Server(ex, io_budget_bytes=8 * 3 * 100 * 4, calibration=CAL, clock=lambda: 0.0)
    for i in range(20):
        srv.submit(make(i))
    steps = 0
    while not srv.idle():
        srv.step()
        steps += 1
        assert srv.io_used <= srv.io_budget
        assert steps < 1000
    assert len(srv.finished) == 20
    assert all(r.C == ("result", r.rid) for r in srv.finished)
    assert srv.peak_io <= srv.io_budget
    assert not ex.live


def test_admission_is_fifo_and_n_follows_target():
    ex = FakeExecutor(slots=1, latency=1)
    srv = Server(ex, io_budget_bytes=10**9, calibration=CAL, clock=lambda: 0.0)
    for i, t in enumerate([1e-8, 1e-11, 1e-13, 1e-15, None]):
        srv.submit(make(i, target=t))
    assert [r.num_moduli for r in srv.waiting] == [12, 14, 16, 18, 16]
    srv.run_until_idle()
    order = [rid for b in ex.batches for rid in b["reqs"]]
    assert order == sorted(order)


def test_batches_respect_slot_workspace():
    ex = FakeExecutor(slots=2, slot_workspace=16 * 40)
    srv = Server(ex, io_budget_bytes=10**9, max_batch=100, calibration=CAL, clock=lambda: 0.0)
    for i in range(30):
        srv.submit(make(i))
    srv.run_until_idle()
    assert len(srv.finished) == 30
    assert all(len(b["reqs"]) <= 2 for b in ex.batches)


def test_oversized_request_is_rejected():
    ex = FakeExecutor(slot_workspace=100)
    srv = Server(ex, io_budget_bytes=10**9, calibration=CAL, clock=lambda: 0.0)
    srv.submit(make(0, m=1000, n=1000, k=10))
    assert srv.idle() and srv.finished[0].error


def test_late_arrivals_start_while_a_batch_runs():
    """Continuous batching: a request that arrives while one batch is on the device starts on the
    other slot before that batch finishes."""
    ex = FakeExecutor(slots=2, latency=5)
    srv = Server(ex, io_budget_bytes=10**9, calibration=CAL, clock=lambda: 0.0)
    srv.submit(make(0))
    srv.step()
    assert 0 in [rid for b in ex.batches for rid in b["reqs"]]
    srv.submit(make(1))
    srv.step()
    assert len(srv.running) == 2            # both slots busy at once
    assert ex.batches[0]["left"] > 0         # the first batch has not finished yet
    srv.run_until_idle()
    assert len(srv.finished) == 2
