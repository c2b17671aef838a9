"""Continuous-batching server for emulated DGEMM requests.

Requests (FP64 A, B on the host, with a relative-error target) arrive at any time.  The server
keeps a FIFO of waiting requests and a set of execution slots (CUDA streams, each with a handle
and a fixed device workspace).  Each scheduling step

  1. retires finished batches: their results are on the host, their device memory is released;
  2. admits waiting requests, in order, while their device inputs and outputs fit the HBM
     budget (the residue planes live in the slot workspaces, which are part of the budget);
     admission uploads the inputs;
  3. starts a batch on every idle slot: the admitted requests that fit the slot's workspace go
     out as one grouped call (ozaki2_dgemm_grouped), whose residue matrices stay in device memory
     for the life of the batch; the CRT writes each result straight into a page-locked host
     buffer (the device writes host memory faster than a device-to-host copy runs).

Requests that arrive while others run are admitted as memory frees up and start on the next
idle slot, so their work overlaps the batches already on the device.  Each request's N comes
from its accuracy target through the calibration table of `autotune`.  Every result is the
same bits the request would get alone (the grouped call computes each problem exactly as
ozaki2_dgemm does).

The executor is separate from the scheduling logic, so the admission and batching rules can be
exercised without a GPU.
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
        return 8 * (self.m * self.k + self.k * self.n + self.m * self.n)

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class Server:
    """Scheduling logic: admission by memory budget, batching onto idle slots, retirement."""

    def __init__(self, executor, io_budget_bytes: int, max_batch: int = 64,
                 calibration=None, default_n: int = 16, clock=time.perf_counter):
        self.ex = executor
        self.io_budget = io_budget_bytes
        self.io_used = 0
        self.max_batch = max_batch
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
        if req.io_bytes > self.io_budget or need > self.ex.slot_workspace:
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
            r = self.waiting.popleft()
            self.io_used += r.io_bytes
            self.peak_io = max(self.peak_io, self.io_used)
            self.ex.admit(r)
            r.admitted = self.clock()
            self.admitted.append(r)
        started = 0
        for slot in self.ex.slots():
            if slot in self.running or not self.admitted:
                continue
            batch = []
            while self.admitted and len(batch) < self.max_batch and \
                    self.ex.workspace_bytes(batch + [self.admitted[0]]) <= self.ex.slot_workspace:
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


class GpuExecutor:
    """Execution slots on one GPU: a stream, an ozaki2 handle and a fixed workspace per slot."""

    def __init__(self, slots: int = 2, slot_workspace_bytes: int = 8 << 30, device: int = 0):
        import torch

        from . import ozaki2 as oz

        self.oz = oz
        self.torch = torch
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

    def slots(self):
        return range(len(self._slots))

    def workspace_bytes(self, reqs) -> int:
        if not reqs:
            return 0
        probs = self.oz.problems_array([dict(m=r.m, n=r.n, k=r.k, A=1, lda=max(1, r.m), B=1,
                                             ldb=max(1, r.k), C=1, ldc=max(1, r.m),
                                             num_moduli=r.num_moduli) for r in reqs])
        return self.oz.ozaki2_grouped_workspace_size(len(reqs), probs)

    def admit(self, r: Request):
        """Device buffers for the request and the upload of its inputs."""
        torch = self.torch

        def host(x):
            t = x if isinstance(x, torch.Tensor) else torch.from_numpy(x)
            return t if t.is_pinned() else t.pin_memory()

        with torch.cuda.stream(self.upload):
            r.dev["A"] = host(r.A).to(self.device, non_blocking=True)
            r.dev["B"] = host(r.B).to(self.device, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.upload)
            r.dev["uploaded"] = ev
        # the result is written by the CRT kernel straight into page-locked host memory
        r.dev["host_C"] = torch.empty((r.n, r.m), dtype=torch.float64, pin_memory=True)

    def launch(self, slot: int, reqs):
        torch, oz = self.torch, self.oz
        s = self._slots[slot]
        with torch.cuda.stream(s["stream"]):
            for r in reqs:
                s["stream"].wait_event(r.dev["uploaded"])
            probs = oz.problems_array([dict(m=r.m, n=r.n, k=r.k, A=r.dev["A"], lda=max(1, r.m),
                                            B=r.dev["B"], ldb=max(1, r.k), C=r.dev["host_C"],
                                            ldc=max(1, r.m), num_moduli=r.num_moduli)
                                       for r in reqs])
            rc = oz.ozaki2_dgemm_grouped(len(reqs), probs, s["handle"])
            if rc:
                raise oz.Ozaki2Error("ozaki2_dgemm_grouped", rc)
            ev = torch.cuda.Event()
            ev.record(s["stream"])
        return ev

    def poll(self, token) -> bool:
        return token.query()

    def finish(self, token, reqs):
        token.synchronize()
        for r in reqs:
            r.C = r.dev["host_C"].numpy()

    def release(self, r: Request):
        r.dev.clear()
