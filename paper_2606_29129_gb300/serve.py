"""Continuous-batching server for emulated DGEMM requests.

Requests (FP64 A, B on the host, with a relative-error target) arrive at any time.  The server
keeps a FIFO of waiting requests and a set of execution slots (CUDA streams, each with a handle
and a fixed device workspace).  Each scheduling step

  1. retires finished batches: their results are on the host, their device memory is released;
  2. admits waiting requests, in order, while their device inputs fit the HBM budget (the
     residue planes live in the slot workspaces and the residue cache, which have their own
     shares of the budget); admission uploads the inputs, or finds them already encoded;
  3. starts a batch on every idle slot: the admitted requests that fit the slot's workspace (and
     the batch's work cap) go out as one grouped call, whose residue matrices stay in device
     memory for the life of the batch; the CRT writes each result straight into a page-locked
     host buffer (the device writes host memory faster than a device-to-host copy runs).

Residue cache.  Under the proposed scaling (Section 4, eq. (proposed-mu)/(proposed-nu)) the
shift of a row of op(A) depends on that row alone and the shift of a column of op(B) on that
column alone, so the shifts and bf16 residue planes of an operand (Step 2) are a function of the
operand and N.  With a cache, every operand is encoded once on the device
(ozaki2_encode_operands) into a buffer of the cache, keyed by the request's operand identity
(`a_key`, `b_key`) and N; later requests with the same operand skip its upload, scaling and
conversion, and every batch runs only the residue GEMMs and the reconstruction
(ozaki2_dgemm_grouped_encoded).  Entries are evicted least recently used when room is needed,
never while a queued or running batch uses them.  Operands without a key are encoded into
private entries that are dropped after their request.

Requests that arrive while others run are admitted as memory frees up and start on the next
idle slot, so their work overlaps the batches already on the device.  Each request's N comes
from its accuracy target through the calibration table of `autotune`.  Every result is the
same bits the request would get alone (the grouped call computes each problem exactly as
ozaki2_dgemm does).

The executor is separate from the scheduling logic, so the admission, batching and cache rules
can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

from . import autotune


@dataclasses.dataclass
class Request:
    rid: int
    m: int
    n: int
    k: int
    target: float | None          # max relative error wanted; None = as accurate as cuBLAS
    A: object = None              # host column-major storage (k, m) float64
    B: object = None              # host column-major storage (n, k) float64
    a_key: object = None          # identity of A for the residue cache (None: not reused)
    b_key: object = None          # identity of B
    out: object = None            # caller's page-locked host buffer (n, m) float64 for the
                                  # result, or None (the executor takes one from its pool)
    buffer: object = None         # the page-locked buffer C lives in
    arrival: float = 0.0
    num_moduli: int = 0
    admitted: float | None = None
    started: float | None = None
    done: float | None = None
    C: object = None              # host result, column-major storage (n, m)
    error: str | None = None
    dev: dict = dataclasses.field(default_factory=dict)

    @property
    def io_bytes(self) -> int:
        """Device bytes of the request's FP64 inputs while they are uploaded (the result is
        written to host memory)."""
        return 8 * (self.m * self.k + self.k * self.n)

    @property
    def flops(self) -> float:
        return 2.0 * self.m * self.n * self.k

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class Server:
    """Scheduling logic: admission by memory budget, batching onto idle slots, retirement."""

    def __init__(self, executor, io_budget_bytes: int, max_batch: int = 64,
                 calibration=None, default_n: int = 16, clock=time.perf_counter,
                 max_batch_flops: float | None = None):
        self.ex = executor
        self.io_budget = io_budget_bytes
        self.io_used = 0
        self.max_batch = max_batch
        # work cap of one batch (sum of 2mnk): a batch takes requests while it stays under the
        # cap (always at least one), so small requests are not held behind a long batch
        self.max_batch_flops = max_batch_flops
        self.step_seconds = 0.0        # host time spent in step() (scheduling and launches)
        self.calibration = calibration or {}
        self.default_n = default_n
        self.clock = clock
        self.waiting = collections.deque()
        self.admitted = collections.deque()
        self.running = {}              # slot -> (token, [requests])
        self.finished = []
        self.peak_io = 0

    # ---------------------------------------------------------------- requests
    def submit(self, req: Request):
        if not req.arrival:
            req.arrival = self.clock()
        req.num_moduli = autotune.choose_n(self.calibration, req.k, req.target, self.default_n)
        need = self.ex.workspace_bytes([req])
        req.dev["ws_bytes"] = need
        too_large = getattr(self.ex, "too_large", None)
        if req.io_bytes > self.io_budget or need > self.ex.slot_workspace or \
                (too_large is not None and too_large(req)):
            req.error = "request larger than the server's memory budget"
            req.done = self.clock()
            self.finished.append(req)
            return
        self.waiting.append(req)

    def idle(self) -> bool:
        return not (self.waiting or self.admitted or self.running)

    # ---------------------------------------------------------------- one step
    def step(self) -> int:
        """Retire, admit, launch.  Returns the number of requests started."""
        t0 = time.perf_counter()
        try:
            return self._step()
        finally:
            self.step_seconds += time.perf_counter() - t0

    def _step(self) -> int:
        for slot in list(self.running):
            token, reqs = self.running[slot]
            if self.ex.poll(token):
                self.ex.finish(token, reqs)
                now = self.clock()
                for r in reqs:
                    r.done = now
                    self.io_used -= r.io_bytes
                    self.ex.release(r)
                    self.finished.append(r)
                del self.running[slot]
        while self.waiting and self.io_used + self.waiting[0].io_bytes <= self.io_budget:
            r = self.waiting[0]
            if self.ex.admit(r) is False:   # no room in the executor yet (its cache is full)
                break
            self.waiting.popleft()
            self.io_used += r.io_bytes
            self.peak_io = max(self.peak_io, self.io_used)
            r.admitted = self.clock()
            self.admitted.append(r)
        started = 0
        for slot in self.ex.slots():
            if slot in self.running or not self.admitted:
                continue
            batch = []
            work = 0.0
            ws = 0   # the sum of the requests' own workspaces bounds the batch's from above
            while self.admitted and len(batch) < self.max_batch:
                nxt = self.admitted[0]
                need = nxt.dev.get("ws_bytes") or self.ex.workspace_bytes([nxt])
                if ws + need > self.ex.slot_workspace:
                    break
                if batch and self.max_batch_flops and work + nxt.flops > self.max_batch_flops:
                    break
                ws += need
                work += nxt.flops
                batch.append(self.admitted.popleft())
            if not batch:
                continue
            now = self.clock()
            for r in batch:
                r.started = now
            self.running[slot] = (self.ex.launch(slot, batch), batch)
            started += len(batch)
        return started

    def run_until_idle(self, poll_sleep: float = 0.0):
        while not self.idle():
            if not self.step() and poll_sleep:
                time.sleep(poll_sleep)


class ResultPool:
    """Reusable page-locked host buffers for results, in power-of-two buckets of float64
    elements.  Page-locking host memory costs more than the emulated product of a mid-size
    request, so a server hands each result buffer back to the pool once the client has consumed
    the result (GpuExecutor.recycle)."""

    def __init__(self, alloc=None):
        self.free = collections.defaultdict(list)
        self.allocated = 0
        self._alloc = alloc

    @staticmethod
    def bucket(numel: int) -> int:
        return 1 << max(0, (max(numel, 1) - 1).bit_length())

    def take(self, numel: int):
        b = self.bucket(numel)
        if self.free[b]:
            return self.free[b].pop()
        self.allocated += 1
        return self._alloc(b)

    def give(self, buf, numel: int):
        self.free[self.bucket(numel)].append(buf)

    def prewarm(self, numel: int, count: int):
        b = self.bucket(numel)
        while len(self.free[b]) < count:
            self.allocated += 1
            self.free[b].append(self._alloc(b))


class CacheEntry:
    __slots__ = ("key", "nbytes", "refs", "private", "buf", "op", "ready")

    def __init__(self, key, nbytes, private):
        self.key, self.nbytes, self.refs, self.private = key, nbytes, 1, private
        self.buf = self.op = self.ready = None


class ResidueCache:
    """Encoded operands kept in device memory, least recently used first out, within a byte
    capacity.  Host logic only: the executor attaches the device buffer to each entry.  An entry
    is referenced while a request that uses it waits or runs; referenced entries are never
    evicted.  Private entries (operands without a key) are dropped when their last reference
    goes."""

    def __init__(self, capacity_bytes: int):
        self.capacity = capacity_bytes
        self.used = 0
        self.peak = 0
        self.entries = collections.OrderedDict()    # key -> entry, least recently used first
        self.hits = self.misses = self.evictions = 0

    def get(self, key):
        """The entry of `key` with one more reference, or None (a miss)."""
        e = self.entries.get(key)
        if e is None:
            self.misses += 1
            return None
        self.hits += 1
        e.refs += 1
        self.entries.move_to_end(key)
        return e

    def fits(self, nbytes: int) -> bool:
        """Whether nbytes could be made room for by evicting unreferenced entries."""
        free = self.capacity - self.used
        free += sum(e.nbytes for e in self.entries.values() if e.refs == 0)
        return nbytes <= free

    def put(self, key, nbytes: int, private: bool = False):
        """A new entry with one reference, after evicting unreferenced entries (least recently
        used first) until it fits; None when it cannot fit now."""
        if not self.fits(nbytes):
            return None
        for k in [k for k, e in self.entries.items() if e.refs == 0]:
            if self.used + nbytes <= self.capacity:
                break
            self._drop(k)
            self.evictions += 1
        e = CacheEntry(key, nbytes, private)
        self.entries[key] = e
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        return e

    def release(self, e: CacheEntry):
        e.refs -= 1
        if e.refs == 0 and e.private and e.key in self.entries:
            self._drop(e.key)

    def discard(self, e: CacheEntry):
        """Remove an entry that was never filled (its admission was undone)."""
        if self.entries.get(e.key) is e:
            self._drop(e.key)

    def _drop(self, key):
        e = self.entries.pop(key)
        self.used -= e.nbytes
        e.buf = e.op = e.ready = None


class GpuExecutor:
    """Execution slots on one GPU: a stream, an ozaki2 handle and a fixed workspace per slot.

    cache_bytes > 0 turns on the residue cache: operands are encoded once (on the upload stream)
    into entries of at most cache_bytes in total, and batches run ozaki2_dgemm_grouped_encoded.
    With cache_bytes = 0 the inputs are uploaded per request and batches run
    ozaki2_dgemm_grouped."""

    def __init__(self, slots: int = 2, slot_workspace_bytes: int = 8 << 30, device: int = 0,
                 cache_bytes: int = 0, result_pool: ResultPool | None = None):
        import torch

        from . import ozaki2 as oz

        self.oz = oz
        self.torch = torch
        self.results = result_pool or ResultPool(
            lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True))
        self.device = torch.device("cuda", device)
        self.slot_workspace = slot_workspace_bytes
        self._slots = []
        for _ in range(slots):
            stream = torch.cuda.Stream(device=self.device)
            h = oz.Handle()
            ws = torch.empty(slot_workspace_bytes, dtype=torch.uint8, device=self.device)
            h.set_workspace(ws, slot_workspace_bytes)
            self._slots.append({"stream": stream, "handle": h, "ws": ws})
        self.upload = torch.cuda.Stream(device=self.device)
        self.cache = ResidueCache(cache_bytes) if cache_bytes > 0 else None
        self.encoder = oz.Handle() if self.cache else None
        # makespan breakdown: bytes over the link, device time of the encodings and of the
        # batches (CUDA events, read when each batch retires)
        self.stats = {"upload_bytes": 0, "result_bytes": 0, "encoded_operands": 0,
                      "encode_ms": 0.0, "batch_ms": 0.0, "batches": 0}
        self._encode_events = []

    def slots(self):
        return range(len(self._slots))

    def _operand_bytes(self, side, r):
        lines = r.m if side == "A" else r.n
        return self.oz.ozaki2_operand_bytes(side, lines, r.k, r.num_moduli)

    def too_large(self, r: Request) -> bool:
        if not self.cache:
            return False
        return self._operand_bytes("A", r) + self._operand_bytes("B", r) > self.cache.capacity

    def workspace_bytes(self, reqs) -> int:
        if not reqs:
            return 0
        probs = self.oz.problems_array([dict(m=r.m, n=r.n, k=r.k, A=1, lda=max(1, r.m), B=1,
                                             ldb=max(1, r.k), C=1, ldc=max(1, r.m),
                                             num_moduli=r.num_moduli) for r in reqs])
        if not self.cache:
            return self.oz.ozaki2_grouped_workspace_size(len(reqs), probs)
        # every side encoded: the workspace holds the product residues and the tables
        ops = (self.oz.Operand * (2 * len(reqs)))()
        for i, r in enumerate(reqs):
            ops[2 * i] = self.oz.Operand(b"A", b"N", r.m, r.k, 1, max(1, r.m), r.num_moduli,
                                         256, 0)
            ops[2 * i + 1] = self.oz.Operand(b"B", b"N", r.n, r.k, 1, max(1, r.k),
                                             r.num_moduli, 256, 0)
        ra = self.oz.encoded_refs(ops, [2 * i for i in range(len(reqs))])
        rb = self.oz.encoded_refs(ops, [2 * i + 1 for i in range(len(reqs))])
        return self.oz.ozaki2_grouped_encoded_workspace_size(len(reqs), probs, ra, rb)

    @staticmethod
    def _pinned(torch, x):
        t = x if isinstance(x, torch.Tensor) else torch.from_numpy(x)
        return t if t.is_pinned() else t.pin_memory()

    def admit(self, r: Request):
        """Device buffers for the request: its encoded operands (cache hits, or new entries
        encoded from an upload), or the uploaded inputs without a cache.  Returns False, with
        nothing held, when the cache cannot make room now."""
        torch = self.torch
        if self.cache:
            return self._admit_cached(r)
        with torch.cuda.stream(self.upload):
            r.dev["A"] = self._pinned(torch, r.A).to(self.device, non_blocking=True)
            r.dev["B"] = self._pinned(torch, r.B).to(self.device, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.upload)
            r.dev["uploaded"] = ev
        self.stats["upload_bytes"] += 8 * (r.m * r.k + r.k * r.n)
        # the result is written by the CRT kernel straight into page-locked host memory
        r.dev["host_C"] = self._result_buffer(r)
        return True

    def _result_buffer(self, r: Request):
        """The caller's page-locked result buffer, else one from the result pool."""
        torch = self.torch
        if r.out is not None:
            if not (isinstance(r.out, torch.Tensor) and r.out.is_pinned() and
                    r.out.dtype == torch.float64 and r.out.is_contiguous() and
                    r.out.numel() >= r.m * r.n):
                raise ValueError("Request.out must be a contiguous page-locked float64 tensor "
                                 "of at least m * n elements")
            r.buffer = r.out
        else:
            r.buffer = self.results.take(r.m * r.n)
        return r.buffer

    def recycle(self, r: Request):
        """Hands a finished request's pool buffer back (its C is no longer valid after this)."""
        if r.buffer is not None and r.out is None:
            self.results.give(r.buffer, r.m * r.n)
        r.buffer = None
        r.C = None

    def _admit_cached(self, r: Request):
        torch, oz, cache = self.torch, self.oz, self.cache
        entries, fresh = {}, []
        for side, key, X in (("A", r.a_key, r.A), ("B", r.b_key, r.B)):
            lines = r.m if side == "A" else r.n
            ckey = None if key is None else (side, key, lines, r.k, r.num_moduli)
            e = cache.get(ckey) if ckey is not None else None
            if e is None:
                private = ckey is None
                e = cache.put(("private", r.rid, side) if private else ckey,
                              self._operand_bytes(side, r), private)
                if e is None:  # undo: hits lose their reference, new entries go
                    new = {id(f[1]) for f in fresh}
                    for held in entries.values():
                        if id(held) in new:
                            cache.discard(held)
                        else:
                            cache.release(held)
                    return False
                fresh.append((side, e, X, lines))
            entries[side] = e
        if fresh:
            # encode the missing operands on the upload stream; the library copies each
            # page-locked host matrix into device memory with a kernel (the link's full rate)
            # before scaling and converting it
            with torch.cuda.stream(self.upload):
                ops = []
                keep = []
                for side, e, X, lines in fresh:
                    e.buf = torch.empty(e.nbytes, dtype=torch.uint8, device=self.device)
                    hX = self._pinned(torch, X)
                    keep.append(hX)
                    self.stats["upload_bytes"] += 8 * lines * r.k
                    # A as stored: column-major m x k (ld m); B: k x n (ld k)
                    ld = max(1, r.m if side == "A" else r.k)
                    ops.append(dict(side=side, trans="N", lines=lines, k=r.k, X=hX, ld=ld,
                                    num_moduli=r.num_moduli, data=e.buf))
                arr = oz.operands_array(ops)
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(self.upload)
                rc = oz.ozaki2_encode_operands(len(ops), arr, self.encoder)
                if rc:
                    raise oz.Ozaki2Error("ozaki2_encode_operands", rc)
                t1.record(self.upload)
                for i, (_, e, _, _) in enumerate(fresh):
                    e.op = oz.Operand.from_buffer_copy(arr[i])
                    e.ready = t1
                self._encode_events.append((t0, t1))
                self.stats["encoded_operands"] += len(fresh)
                # host matrices that were pinned here must outlive the staging copy
                r.dev["pinned_inputs"] = keep
        r.dev["enc"] = entries
        r.dev["host_C"] = self._result_buffer(r)
        return True

    def launch(self, slot: int, reqs):
        torch, oz = self.torch, self.oz
        s = self._slots[slot]
        with torch.cuda.stream(s["stream"]):
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            if not self.cache:
                for r in reqs:
                    s["stream"].wait_event(r.dev["uploaded"])
                probs = oz.problems_array([dict(m=r.m, n=r.n, k=r.k, A=r.dev["A"],
                                                lda=max(1, r.m), B=r.dev["B"], ldb=max(1, r.k),
                                                C=r.dev["host_C"], ldc=max(1, r.m),
                                                num_moduli=r.num_moduli) for r in reqs])
                start.record(s["stream"])
                rc = oz.ozaki2_dgemm_grouped(len(reqs), probs, s["handle"])
                if rc:
                    raise oz.Ozaki2Error("ozaki2_dgemm_grouped", rc)
            else:
                waited = set()
                for r in reqs:
                    for e in r.dev["enc"].values():
                        if e.ready is not None and id(e.ready) not in waited:
                            s["stream"].wait_event(e.ready)
                            waited.add(id(e.ready))
                ops = (oz.Operand * (2 * len(reqs)))()
                for i, r in enumerate(reqs):
                    ops[2 * i] = r.dev["enc"]["A"].op
                    ops[2 * i + 1] = r.dev["enc"]["B"].op
                # A and B are not read for encoded sides; the encodings' buffers stand in
                probs = oz.problems_array([dict(m=r.m, n=r.n, k=r.k, A=r.dev["enc"]["A"].buf,
                                                lda=max(1, r.m), B=r.dev["enc"]["B"].buf,
                                                ldb=max(1, r.k), C=r.dev["host_C"],
                                                ldc=max(1, r.m), num_moduli=r.num_moduli)
                                           for r in reqs])
                ra = oz.encoded_refs(ops, [2 * i for i in range(len(reqs))])
                rb = oz.encoded_refs(ops, [2 * i + 1 for i in range(len(reqs))])
                start.record(s["stream"])
                rc = oz.ozaki2_dgemm_grouped_encoded(len(reqs), probs, ra, rb, s["handle"])
                if rc:
                    raise oz.Ozaki2Error("ozaki2_dgemm_grouped_encoded", rc)
            end.record(s["stream"])
        return (start, end)

    def poll(self, token) -> bool:
        return token[1].query()

    def finish(self, token, reqs):
        start, end = token
        end.synchronize()
        self.stats["batch_ms"] += start.elapsed_time(end)
        self.stats["batches"] += 1
        for r in reqs:
            r.C = r.dev["host_C"].view(-1)[: r.m * r.n].view(r.n, r.m).numpy()
            self.stats["result_bytes"] += 8 * r.m * r.n

    def release(self, r: Request):
        if self.cache and "enc" in r.dev:
            for e in r.dev["enc"].values():
                self.cache.release(e)
        r.dev.clear()

    def breakdown(self) -> dict:
        """Link bytes, device milliseconds of the encodings and batches, cache counters."""
        self.torch.cuda.synchronize()
        enc = sum(a.elapsed_time(b) for a, b in self._encode_events)
        self._encode_events.clear()
        self.stats["encode_ms"] += enc
        out = dict(self.stats)
        if self.cache:
            out.update(cache_hits=self.cache.hits, cache_misses=self.cache.misses,
                       cache_evictions=self.cache.evictions,
                       cache_peak_gb=self.cache.peak / 2**30)
        return out
