"""Serving loop for IMF evaluations coming from many concurrent topology-optimisation loops.

Each TO loop (Alg. 2 of arXiv 2002.07627) calls the IMF (Alg. 1) once per iteration with the
same tools and orientations and a new density. The server keeps one resident libimf handle per
design id (its tool spectra stay on the device between iterations), admits requests while the
HBM footprint of the resident designs fits the budget (evicting idle designs, least recently
used first), and runs admitted requests on a pool of CUDA streams. Continuous batching: a
request that arrives while others are on the GPU starts as soon as a stream slot is free and
its design is resident and idle, so work from different loops overlaps on the device.

The scheduler is written against an executor interface; `GpuExecutor` drives libimf through
its C ABI, and the tests drive the same scheduler with a fake executor on the CPU.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


@dataclass
class DesignSpec:
    shape: tuple                  # (nz, ny, nx)
    tools: list                   # synth.Tool list (holder, cutter, origin, quats, sharp)
    fixture: np.ndarray | None = None
    lam: float = 0.01
    tau: float = 0.5
    theta_rel: float = 0.01

    @property
    def units(self) -> int:
        return int(np.prod(self.shape)) * sum(len(t.quats) for t in self.tools)


@dataclass
class _Req:
    design_id: object
    rho: np.ndarray
    t_submit: float
    future: Future
    t_start: float = 0.0


@dataclass
class _Resident:
    state: object
    bytes: int
    busy: bool = False
    last_used: float = 0.0


@dataclass
class ServerStats:
    latencies: list = field(default_factory=list)     # seconds, submit -> result
    queue_waits: list = field(default_factory=list)   # seconds, submit -> launch
    completed: int = 0
    failed: int = 0
    evictions: int = 0
    creations: int = 0
    max_resident_bytes: int = 0
    max_running: int = 0
    units: int = 0

    def percentile(self, q):
        return float(np.percentile(self.latencies, q)) if self.latencies else float("nan")


class ImfServer:
    def __init__(self, executor, hbm_budget: int, slots: int = 4, poll_s: float = 2e-4):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.slots = max(1, int(slots))
        self.poll_s = poll_s
        self.specs = {}
        self.resident = collections.OrderedDict()   # design_id -> _Resident (LRU order)
        self.pending = collections.deque()
        self.running = {}                           # slot -> (req, token)
        self.stats = ServerStats()
        self._lock = threading.Lock()
        self._wake = threading.Condition(self._lock)
        self._stop = False
        self._thread = threading.Thread(target=self._loop, name="imf-server", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------------ API
    def register(self, design_id, spec: DesignSpec):
        with self._lock:
            self.specs[design_id] = spec

    def submit(self, design_id, rho: np.ndarray) -> Future:
        fut = Future()
        with self._lock:
            if design_id not in self.specs:
                fut.set_exception(KeyError(f"unknown design id {design_id!r}"))
                return fut
            self.pending.append(_Req(design_id, rho, time.perf_counter(), fut))
            self._wake.notify()
        return fut

    def close(self, drain: bool = True, timeout: float = 120.0):
        t0 = time.perf_counter()
        if drain:
            while True:
                with self._lock:
                    if not self.pending and not self.running:
                        break
                if time.perf_counter() - t0 > timeout:
                    break
                time.sleep(self.poll_s)
        with self._lock:
            self._stop = True
            self._wake.notify()
        self._thread.join(timeout=10)
        with self._lock:
            for rid, r in list(self.resident.items()):
                self.ex.destroy(r.state)
            self.resident.clear()
            while self.pending:
                self.pending.popleft().future.set_exception(RuntimeError("server closed"))

    # ------------------------------------------------------------------ scheduler
    def _resident_bytes(self):
        return sum(r.bytes for r in self.resident.values())

    def _make_room(self, need: int) -> bool:
        """Evict idle designs (least recently used first) until `need` more bytes fit."""
        if need > self.budget:
            return False
        while self._resident_bytes() + need > self.budget:
            victim = next((k for k, r in self.resident.items() if not r.busy), None)
            if victim is None:
                return False
            r = self.resident.pop(victim)
            self.ex.destroy(r.state)
            self.stats.evictions += 1
        return True

    def _complete(self):
        now = time.perf_counter()
        for slot, (req, token) in list(self.running.items()):
            try:
                if not self.ex.done(token):
                    continue
                out = self.ex.result(token)
                req.future.set_result(out)
                self.stats.completed += 1
                self.stats.latencies.append(now - req.t_submit)
                self.stats.units += self.specs[req.design_id].units
            except Exception as exc:  # a failing request fails alone
                req.future.set_exception(exc)
                self.stats.failed += 1
            del self.running[slot]
            r = self.resident.get(req.design_id)
            if r is not None:
                r.busy = False
                r.last_used = now

    def _admit(self):
        free = [s for s in range(self.slots) if s not in self.running]
        if not free:
            return
        keep = collections.deque()
        while self.pending and free:
            req = self.pending.popleft()
            r = self.resident.get(req.design_id)
            if r is not None and r.busy:
                keep.append(req)          # one request per design at a time (its buffers)
                continue
            if r is None:
                spec = self.specs[req.design_id]
                need = int(self.ex.footprint(spec))
                if need > self.budget:
                    req.future.set_exception(MemoryError(
                        f"design {req.design_id!r} needs {need} bytes, above the HBM budget {self.budget}"))
                    self.stats.failed += 1
                    continue
                if not self._make_room(need):
                    keep.append(req)      # wait for a running design to finish
                    continue
                try:
                    state = self.ex.create(req.design_id, spec)
                except Exception as exc:
                    req.future.set_exception(exc)
                    self.stats.failed += 1
                    continue
                r = _Resident(state, need)
                self.resident[req.design_id] = r
                self.stats.creations += 1
                self.stats.max_resident_bytes = max(self.stats.max_resident_bytes, self._resident_bytes())
            slot = free.pop(0)
            self.resident.move_to_end(req.design_id)
            try:
                req.t_start = time.perf_counter()
                token = self.ex.launch(r.state, req.rho, slot)
            except Exception as exc:
                req.future.set_exception(exc)
                self.stats.failed += 1
                free.insert(0, slot)
                continue
            r.busy = True
            self.stats.queue_waits.append(req.t_start - req.t_submit)
            self.running[slot] = (req, token)
            self.stats.max_running = max(self.stats.max_running, len(self.running))
        # requests that could not start keep their order ahead of later arrivals
        while keep:
            self.pending.appendleft(keep.pop())

    def _loop(self):
        while True:
            with self._lock:
                if self._stop:
                    return
                self._complete()
                self._admit()
                idle = not self.running and not self.pending
                if idle:
                    self._wake.wait(timeout=0.05)
                    continue
            time.sleep(self.poll_s)


class GpuExecutor:
    """Runs requests through libimf on a pool of CUDA streams, one stream per slot."""

    def __init__(self, slots: int, device: int = 0, orient_batch: int = 16):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        # orientations per device batch of every served handle; the admission footprint counts
        # the work buffers of exactly that many slots
        self.orient_batch = int(orient_batch)

    def footprint(self, spec: DesignSpec) -> int:
        """Bytes a served design holds on the device: the library's planned footprint (spectra,
        tables, set-up peak and the work buffers of `orient_batch` slots, imf_footprint) plus the
        request buffers this executor allocates with torch (rho, fixture, f_bar, Gamma)."""
        from .batch import planned_footprint
        from .synth import Design
        fp = planned_footprint(Design(np.zeros(spec.shape, np.float32), spec.fixture, spec.tools),
                               orient_batch=self.orient_batch)
        n = int(np.prod(spec.shape))
        return int(fp.total) + n * (4 + 4 + 1 + (1 if spec.fixture is not None else 0))

    def library_budget(self, spec: DesignSpec) -> int:
        from .batch import planned_footprint
        from .synth import Design
        return int(planned_footprint(Design(np.zeros(spec.shape, np.float32), spec.fixture, spec.tools),
                                     orient_batch=self.orient_batch).total)

    def create(self, design_id, spec: DesignSpec):
        from . import binding
        torch = self.torch
        torch.cuda.set_device(self.dev)
        # the library enforces the admitted footprint (IMF_ERR_BUDGET beyond it)
        imf = binding.Imf(spec.shape, lam=spec.lam, tau=spec.tau, theta_rel=spec.theta_rel,
                          orient_batch=self.orient_batch, hbm_budget_bytes=self.library_budget(spec))
        imf.set_tools(spec.tools)
        st = {"imf": imf,
              "rho": torch.empty(spec.shape, dtype=torch.float32, device=self.dev),
              "fix": None if spec.fixture is None else torch.from_numpy(np.ascontiguousarray(spec.fixture, np.uint8)).to(self.dev),
              "fbar": torch.empty(spec.shape, dtype=torch.float32, device=self.dev),
              "sec": torch.empty(spec.shape, dtype=torch.uint8, device=self.dev),
              "h_rho": torch.empty(spec.shape, dtype=torch.float32).pin_memory(),
              "h_fbar": torch.empty(spec.shape, dtype=torch.float32).pin_memory(),
              "h_sec": torch.empty(spec.shape, dtype=torch.uint8).pin_memory()}
        return st

    def destroy(self, st):
        st["imf"].close()

    def launch(self, st, rho: np.ndarray, slot: int):
        torch = self.torch
        s = self.streams[slot]
        st["h_rho"].numpy()[...] = rho
        with torch.cuda.stream(s):
            st["rho"].copy_(st["h_rho"], non_blocking=True)
            st["imf"].compute(st["rho"], st["fix"], st["fbar"], st["sec"], stream=s)
            st["h_fbar"].copy_(st["fbar"], non_blocking=True)
            st["h_sec"].copy_(st["sec"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, st)

    def done(self, token) -> bool:
        return token[0].query()

    def result(self, token):
        ev, st = token
        ev.synchronize()
        st["imf"].sync()
        return st["h_fbar"].numpy().copy(), st["h_sec"].numpy().copy()
