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


# ---------------------------------------------------------------- residue cache (host logic)
from paper_2606_29129_gb300.serve import ResidueCache  # noqa: E402


def test_cache_hits_and_lru_eviction_under_capacity():
    c = ResidueCache(100)
    a = c.put("a", 40)
    b = c.put("b", 40)
    assert c.used == 80 and a.refs == b.refs == 1
    assert c.put("c", 40) is None              # a and b are referenced: no room
    c.release(a)
    c.release(b)
    assert c.get("a") is a and a.refs == 1     # a is now the most recently used
    c.release(a)
    d = c.put("d", 40)                         # evicts b, the least recently used
    assert d is not None and "b" not in c.entries and "a" in c.entries
    assert c.used == 80 and c.evictions == 1 and c.peak <= c.capacity
    assert c.get("b") is None and c.misses == 1 and c.hits == 1


def test_cache_never_evicts_referenced_and_drops_private():
    c = ResidueCache(100)
    p = c.put(("private", 1, "A"), 60, private=True)
    assert not c.fits(50)
    c.release(p)                               # private entries go with their last reference
    assert c.used == 0 and not c.entries
    x = c.put("x", 100)
    assert c.put("y", 1) is None
    c.discard(x)
    assert c.used == 0


class CachingFakeExecutor(FakeExecutor):
    """A fake executor whose admissions take cache entries for A and B, like the GPU one."""

    def __init__(self, capacity, **kw):
        super().__init__(**kw)
        self.cache = ResidueCache(capacity)
        self.encoded = 0

    def too_large(self, r):
        return 2 * r.m * r.k > self.cache.capacity

    def admit(self, r):
        got = []
        for side, key in (("A", r.a_key), ("B", r.b_key)):
            ck = None if key is None else (side, key, r.num_moduli)
            e = self.cache.get(ck) if ck is not None else None
            if e is None:
                e = self.cache.put(ck or ("private", r.rid, side), r.m * r.k, ck is None)
                if e is None:
                    for g in got:
                        self.cache.release(g)
                    return False
                self.encoded += 1
            got.append(e)
        r.dev["enc"] = got
        self.live.add(r.rid)
        return True

    def release(self, r):
        for e in r.dev.pop("enc", []):
            self.cache.release(e)
        self.live.discard(r.rid)


def test_server_with_cache_reuses_operands_and_respects_capacity():
    ex = CachingFakeExecutor(capacity=1000, slots=2, latency=2)
    srv = Server(ex, io_budget_bytes=10**9, calibration=CAL, clock=lambda: 0.0)
    # 40 requests over 4 operand pairs (10 x 10 x 10: 100 bytes per operand in this fake)
    for i in range(40):
        r = make(i)
        r.a_key, r.b_key = ("A", i % 4), ("B", i % 4)
        srv.submit(r)
    steps = 0
    while not srv.idle():
        srv.step()
        steps += 1
        assert ex.cache.used <= ex.cache.capacity
        assert steps < 1000
    assert len(srv.finished) == 40 and all(r.error is None for r in srv.finished)
    assert ex.encoded == 8                      # every operand encoded once
    assert ex.cache.hits == 72 and not ex.live


def test_server_admission_waits_for_cache_room():
    """Operands without keys take private entries; when the cache is full of entries in use the
    next request waits and is admitted after a batch retires."""
    ex = CachingFakeExecutor(capacity=400, slots=1, latency=2)
    srv = Server(ex, io_budget_bytes=10**9, max_batch=1, calibration=CAL, clock=lambda: 0.0)
    for i in range(6):
        srv.submit(make(i))
    srv.step()
    assert len(srv.waiting) == 4                # two requests hold the 400 bytes
    srv.run_until_idle()
    assert len(srv.finished) == 6 and ex.cache.used == 0


def test_batch_work_cap():
    ex = FakeExecutor(slots=1, latency=1)
    srv = Server(ex, io_budget_bytes=10**9, calibration=CAL, clock=lambda: 0.0,
                 max_batch_flops=2.0 * 10 * 10 * 10 * 3)
    for i in range(7):
        srv.submit(make(i))
    srv.run_until_idle()
    assert [len(b["reqs"]) for b in ex.batches] == [3, 3, 1]


def test_result_pool_reuses_buffers_by_bucket():
    from paper_2606_29129_gb300.serve import ResultPool

    made = []
    pool = ResultPool(lambda n: made.append(n) or ("buf", len(made), n))
    a = pool.take(1000)              # bucket 1024
    assert a[2] == 1024 and pool.allocated == 1
    pool.give(a, 1000)
    assert pool.take(900) is a       # same bucket: reused, nothing allocated
    assert pool.take(1025)[2] == 2048 and pool.allocated == 2
    pool.prewarm(64, 3)
    assert len(pool.free[64]) == 3 and pool.allocated == 5
