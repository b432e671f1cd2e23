"""Batched IMF evaluation of many designs of uneven size (the batched form).

Each design keeps a resident libimf handle (tool spectra stay on the device); the library's
autotuner picks, for its grid and tool, the orientation batch, the FFT form (two-pass splits or
radix stages), the launch forms of the FFT passes and the work units of the minimum over sharp
points; and its imf_compute is captured once as a CUDA graph. A run replays every design's graph over a pool of streams, so
small designs overlap on the device and launch gaps disappear. The plain form for comparison
runs the designs one after another on one stream with default options and no graphs.

Everything on the device runs in libimf's kernels; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import binding


def planned_footprint(design, orient_batch: int = 0, slots: int = 0):
    """Device footprint of one design from the library's own plan (imf_footprint on a plan_only
    handle: the tool is resampled and every size planned on the host; nothing is allocated).
    Returns the ImfFootprint (resident spectra and tables, work buffers for `slots` orientation
    slots or the first compute's default, set-up peak, total)."""
    imf = binding.Imf(design.rho.shape, orient_batch=orient_batch, plan_only=True)
    try:
        imf.set_tools(design.tools)
        return imf.footprint(slots)
    finally:
        imf.close()


def handle_budget(design, work_budget: int) -> int:
    """HBM cap of one resident handle: its spectra and tables plus `work_budget` bytes of work
    buffers, and never below what its set-up needs transiently."""
    fp = planned_footprint(design, slots=1)
    return int(max(fp.setup_peak, fp.resident + max(work_budget, fp.work)))


@dataclass
class _Entry:
    design: object
    imf: object
    rho: object
    fix: object
    fbar: object
    sec: object
    units: int
    batch: int = 0
    tuned: dict | None = None


class BatchRunner:
    def __init__(self, designs, n_streams: int = 8, autotune: bool = True, graphs: bool = True, device: int = 0,
                 work_budget: int = 2 << 30):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(max(1, n_streams))]
        self.graphs = graphs
        self.entries = []
        for d in designs:
            # cap each design's device memory at its spectra plus `work_budget` of work buffers
            imf = binding.Imf(d.rho.shape, hbm_budget_bytes=handle_budget(d, work_budget))
            imf.set_tools(d.tools)
            rho = torch.from_numpy(np.ascontiguousarray(d.rho)).to(self.dev)
            fix = None if d.fixture is None else torch.from_numpy(np.ascontiguousarray(d.fixture)).to(self.dev)
            fbar = torch.empty_like(rho)
            sec = torch.empty(rho.shape, dtype=torch.uint8, device=self.dev)
            units = int(np.prod(d.rho.shape)) * sum(len(t.quats) for t in d.tools)
            e = _Entry(d, imf, rho, fix, fbar, sec, units)
            s = self.streams[len(self.entries) % len(self.streams)]
            if autotune:
                e.batch = imf.autotune(rho, fix, stream=s)
                o = imf.options()
                e.tuned = {k: o[k] for k in ("orient_batch", "fft_stages_only", "fft_tma", "fft_wide_pencils",
                                             "fft_tma_x", "erode_groups")}
            if graphs:
                imf.capture_graph(rho, fix, fbar, sec, stream=s)
            self.entries.append(e)
        torch.cuda.synchronize(self.dev)

    @property
    def units(self) -> int:
        return sum(e.units for e in self.entries)

    def launch_all(self):
        # largest designs first so the small ones fill the gaps at the end
        order = sorted(range(len(self.entries)), key=lambda i: -self.entries[i].units)
        for k, i in enumerate(order):
            e = self.entries[i]
            s = self.streams[k % len(self.streams)]
            if self.graphs:
                e.imf.launch_graph(stream=s)
            else:
                e.imf.compute(e.rho, e.fix, e.fbar, e.sec, stream=s)

    def run(self, reps: int = 1) -> float:
        """Wall time (s) of `reps` passes over all designs, device-synchronised."""
        self.torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            self.launch_all()
        self.torch.cuda.synchronize(self.dev)
        return (time.perf_counter() - t0) / reps

    def check(self):
        for e in self.entries:
            e.imf.sync()

    def close(self):
        for e in self.entries:
            e.imf.close()
        self.entries = []


def run_plain(designs, reps: int = 1, device: int = 0, work_budget: int = 2 << 30):
    """The plain form: one design at a time on one stream, default options, no graphs; each
    handle's device memory is capped like the batched form's (spectra + `work_budget` of work
    buffers), since all handles stay resident. Returns (seconds per pass, units per pass)."""
    import torch
    dev = torch.device("cuda", device)
    items = []
    for d in designs:
        imf = binding.Imf(d.rho.shape, hbm_budget_bytes=handle_budget(d, work_budget))
        imf.set_tools(d.tools)
        rho = torch.from_numpy(np.ascontiguousarray(d.rho)).to(dev)
        fix = None if d.fixture is None else torch.from_numpy(np.ascontiguousarray(d.fixture)).to(dev)
        items.append((imf, rho, fix, torch.empty_like(rho), torch.empty(rho.shape, dtype=torch.uint8, device=dev)))
    for imf, rho, fix, fb, sec in items:
        imf.compute(rho, fix, fb, sec)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        for imf, rho, fix, fb, sec in items:
            imf.compute(rho, fix, fb, sec)
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / reps
    units = sum(int(np.prod(d.rho.shape)) * sum(len(t.quats) for t in d.tools) for d in designs)
    for it in items:
        it[0].close()
    return dt, units
