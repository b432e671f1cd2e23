"""Serving loop for IMF evaluations coming from many concurrent topology-optimisation loops.

Each TO loop (Alg. 2 of arXiv 2002.07627) calls the IMF (Alg. 1) once per iteration with the
same tools and orientations and a new density. The server keeps one resident libimf handle per
design id (its tool spectra stay on the device between iterations), admits requests while the
HBM footprint of the resident designs fits the budget (evicting idle designs, least recently
used first), and runs admitted requests on a pool of CUDA streams. Continuous batching: a
request that arrives while others are on the GPU starts as soon as a stream slot is free and
its design is resident and has an idle context (or room for one more), so work from different
loops, and several requests of one design, overlap on the device.

The scheduler is written against an executor interface; `GpuExecutor` drives libimf through
its C ABI, and the tests drive the same scheduler with a fake executor on the CPU. Up to
`max_inflight` requests of one design run at once, each on a context of its own (a clone of the
design's handle: shared tool spectra, own work buffers), admitted against the same budget.
"""
from __future__ import annotations

import collections
import threading
import time
import warnings
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
    bytes: int                    # the design's footprint with its first context
    ctx_bytes: int = 0            # each further context
    contexts: int = 1
    free: list = field(default_factory=lambda: [0])   # idle context indices
    last_used: float = 0.0

    @property
    def busy(self) -> bool:
        return len(self.free) < self.contexts

    @property
    def total(self) -> int:
        return self.bytes + (self.contexts - 1) * self.ctx_bytes


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
    max_contexts: int = 1
    units: int = 0

    def percentile(self, q):
        return float(np.percentile(self.latencies, q)) if self.latencies else float("nan")


@dataclass
class _Token:
    inner: object
    ctx: int


def token_ctx(tok):
    return tok.ctx


class ImfServer:
    def __init__(self, executor, hbm_budget: int, slots: int = 4, poll_s: float = 2e-4, max_inflight: int = 2):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.slots = max(1, int(slots))
        # requests of one design in flight at once: each runs on a context of its own (shared
        # tool spectra, own work buffers) where the executor can add contexts, else one
        self.max_inflight = max(1, int(max_inflight)) if hasattr(executor, "add_context") else 1
        self.poll_s = poll_s
        self.specs = {}
        self.small_units = 0
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
            # requests at most this size (voxel-orientations) count as small: the median design
            units = sorted(sp.units for sp in self.specs.values())
            self.small_units = units[(len(units) - 1) // 2]

    def _pick_slot(self, free, design_id):
        """A free slot for a request: with an executor that reports stream priorities, small
        requests take a high-priority slot and large ones a low-priority slot when one is free."""
        prio = getattr(self.ex, "slot_priority", None)
        if prio is not None:
            want = 1 if self.specs[design_id].units <= self.small_units else 0
            for i, sl in enumerate(free):
                if prio(sl) == want:
                    return free.pop(i)
        return free.pop(0)

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
        return sum(r.total for r in self.resident.values())

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

    def _grow(self, design_id, r) -> bool:
        """One more context for a resident design, within the budget (idle designs evicted
        first, never this one); False when it does not fit."""
        if self._resident_bytes() + r.ctx_bytes > self.budget:
            pinned = self.resident.pop(design_id)      # keep the growing design out of eviction
            ok = self._make_room(r.ctx_bytes + pinned.total)
            self.resident[design_id] = pinned
            self.resident.move_to_end(design_id)
            if not ok or self._resident_bytes() + r.ctx_bytes > self.budget:
                return False
        try:
            self.ex.add_context(r.state)
        except Exception:
            return False
        r.free.append(r.contexts)
        r.contexts += 1
        self.stats.max_contexts = max(self.stats.max_contexts, r.contexts)
        self.stats.max_resident_bytes = max(self.stats.max_resident_bytes, self._resident_bytes())
        return True

    def _complete(self):
        now = time.perf_counter()
        for slot, (req, token) in list(self.running.items()):
            try:
                if not self.ex.done(token.inner):
                    continue
                out = self.ex.result(token.inner)
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
                r.free.append(token_ctx(token))
                r.last_used = now

    def _admit(self):
        free = [s for s in range(self.slots) if s not in self.running]
        if not free:
            return
        keep = collections.deque()
        while self.pending and free:
            req = self.pending.popleft()
            r = self.resident.get(req.design_id)
            if r is not None and not r.free:
                # every context of the design is busy: add one if allowed and it fits
                if r.contexts >= self.max_inflight or not self._grow(req.design_id, r):
                    keep.append(req)
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
                ctx_need = int(self.ex.context_footprint(spec)) if self.max_inflight > 1 else 0
                r = _Resident(state, need, ctx_need)
                self.resident[req.design_id] = r
                self.stats.creations += 1
                self.stats.max_resident_bytes = max(self.stats.max_resident_bytes, self._resident_bytes())
            slot = self._pick_slot(free, req.design_id)
            self.resident.move_to_end(req.design_id)
            ctx = r.free.pop(0)
            try:
                req.t_start = time.perf_counter()
                token = self.ex.launch(r.state, req.rho, slot) if self.max_inflight == 1 else \
                    self.ex.launch(r.state, req.rho, slot, ctx)
            except Exception as exc:
                req.future.set_exception(exc)
                self.stats.failed += 1
                free.insert(0, slot)
                r.free.insert(0, ctx)
                continue
            token = _Token(token, ctx)
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

    def __init__(self, slots: int, device: int = 0, orient_batch: int = 16, high_priority_slots: int = 0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        # the first `high_priority_slots` streams (-1: half of them; none by default) get the
        # device's highest stream priority, and the server puts small requests there so that their
        # blocks are scheduled ahead of a large request's. It lowers the median latency under
        # light load but starves the large requests: the 99th percentile grows at every rate
        nhi = slots // 2 if high_priority_slots < 0 else min(slots, high_priority_slots)
        self._prio = [1 if i < nhi else 0 for i in range(slots)]
        self.streams = [torch.cuda.Stream(self.dev, priority=-1 if i < nhi else 0) for i in range(slots)]
        # orientations per device batch of every served handle; the admission footprint counts
        # the work buffers of exactly that many slots
        self.orient_batch = int(orient_batch)

    def slot_priority(self, slot: int) -> int:
        """1 for a high-priority stream, 0 otherwise."""
        return self._prio[slot]

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

    def context_footprint(self, spec: DesignSpec) -> int:
        """Device bytes of one more concurrent context of a resident design: the work buffers
        of `orient_batch` slots (the tool spectra are shared) and the request buffers."""
        from .batch import planned_footprint
        from .synth import Design
        fp = planned_footprint(Design(np.zeros(spec.shape, np.float32), spec.fixture, spec.tools),
                               orient_batch=self.orient_batch)
        return int(fp.work) + int(np.prod(spec.shape)) * (4 + 4 + 1)

    def _buffers(self, spec: DesignSpec, imf):
        torch = self.torch
        return {"imf": imf,
                "rho": torch.empty(spec.shape, dtype=torch.float32, device=self.dev),
                "fbar": torch.empty(spec.shape, dtype=torch.float32, device=self.dev),
                "sec": torch.empty(spec.shape, dtype=torch.uint8, device=self.dev),
                "h_rho": torch.empty(spec.shape, dtype=torch.float32).pin_memory(),
                "h_fbar": torch.empty(spec.shape, dtype=torch.float32).pin_memory(),
                "h_sec": torch.empty(spec.shape, dtype=torch.uint8).pin_memory()}

    def create(self, design_id, spec: DesignSpec):
        from . import binding
        torch = self.torch
        torch.cuda.set_device(self.dev)
        # the library enforces the admitted footprint (IMF_ERR_BUDGET beyond it)
        imf = binding.Imf(spec.shape, lam=spec.lam, tau=spec.tau, theta_rel=spec.theta_rel,
                          orient_batch=self.orient_batch, hbm_budget_bytes=self.library_budget(spec))
        imf.set_tools(spec.tools)
        fix = None if spec.fixture is None else torch.from_numpy(np.ascontiguousarray(spec.fixture, np.uint8)).to(self.dev)
        return {"spec": spec, "fix": fix, "ctxs": [self._buffers(spec, imf)]}

    def add_context(self, st):
        """A further context of a resident design: a clone of its handle (shared tool spectra,
        own work buffers) with its own request buffers."""
        self.torch.cuda.set_device(self.dev)
        st["ctxs"].append(self._buffers(st["spec"], st["ctxs"][0]["imf"].clone()))

    def destroy(self, st):
        for c in reversed(st["ctxs"]):
            c["imf"].close()

    def launch(self, st, rho: np.ndarray, slot: int, ctx: int = 0):
        torch = self.torch
        s = self.streams[slot]
        c = st["ctxs"][ctx]
        # host copies through torch (several threads, without the interpreter lock) rather than
        # numpy: at 256^3 a request moves 64 MB in and 80 MB out on the host
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", UserWarning)      # read-only inputs are only read
            c["h_rho"].copy_(torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)))
        with torch.cuda.stream(s):
            c["rho"].copy_(c["h_rho"], non_blocking=True)
            c["imf"].compute(c["rho"], st["fix"], c["fbar"], c["sec"], stream=s)
            c["h_fbar"].copy_(c["fbar"], non_blocking=True)
            c["h_sec"].copy_(c["sec"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, c)

    def done(self, token) -> bool:
        return token[0].query()

    def result(self, token):
        ev, c = token
        ev.synchronize()
        c["imf"].sync()
        return c["h_fbar"].clone().numpy(), c["h_sec"].clone().numpy()
