"""Topology optimisation with the accessibility constraint (Alg. 2 of arXiv 2002.07627,
Sec. 2.2) on one GPU: the SIMP steps of include/imf_to.h around the IMF of include/imf.h.

Every field operation runs in the library's kernels (projection, FEA, sensitivity and filter,
IMF, penalty, OC update); this module holds the loop of Alg. 2 and the choice of the
accessibility weight w_acc, which Sec. 2.2 leaves as "a constant or adaptively updated based on
the secluded volume": `constant` keeps w fixed; `adaptive` raises w by `w_step` (up to
`w_max`) after an iteration whose secluded volume exceeds `gamma_tol` of the part's volume
(the paper's ~1 % relaxation of the constraint V_Gamma = 0) and lowers it by `w_step` (down to
`w_min`) otherwise.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import binding


@dataclass
class WSchedule:
    kind: str = "constant"        # "constant" | "adaptive"
    w: float = 0.5
    w_min: float = 0.0
    w_max: float = 0.9
    w_step: float = 0.05
    gamma_tol: float = 0.01

    def next(self, w, secluded_voxels, part_voxels):
        if self.kind == "constant":
            return w
        if secluded_voxels > self.gamma_tol * max(part_voxels, 1.0):
            return min(self.w_max, w + self.w_step)
        return max(self.w_min, w - self.w_step)


@dataclass
class ToResult:
    xi: np.ndarray
    rho: np.ndarray
    history: list = field(default_factory=list)


def run_to2d(nelx=256, nely=128, volfrac=0.5, tools=None, iters=50, delta=1e-3, schedule: WSchedule | None = None,
             beta=2.0, fixture_cols=2, lam=0.01, tau=0.5, theta_rel=0.01, move=0.2, eta=0.5, device=0, xi0=None,
             cg_tol=1e-8, **fea_opts) -> ToResult:
    """Alg. 2 on the 2D cantilever (synth.cantilever2d): tools = None runs the unconstrained
    optimisation (no IMF), a list of synth.Tool the accessibility-constrained one. Stops when
    the mean design change is at most `delta` or after `iters` iterations."""
    import torch
    from . import synth
    dev = torch.device("cuda", device)
    torch.cuda.set_device(dev)
    force, fixed, fixture = synth.cantilever2d(nelx, nely, fixture_cols)
    to = binding.To2d(nelx, nely, beta=beta, cg_tol=cg_tol, **fea_opts)
    f_d = torch.from_numpy(force).to(dev)
    fixed_d = torch.from_numpy(fixed).to(dev)
    fix_d = torch.from_numpy(fixture).to(dev)
    if xi0 is None:
        xi0 = np.where(fixture != 0, 1.0, volfrac).astype(np.float32)
    xi = torch.from_numpy(np.ascontiguousarray(xi0, np.float32)).to(dev)
    xi_new = torch.empty_like(xi)
    rho = torch.empty_like(xi)
    sens = torch.empty_like(xi)
    imf = None
    if tools:
        imf = binding.Imf((1, nely, nelx), lam=lam, tau=tau, theta_rel=theta_rel)
        imf.set_tools(tools)
        fbar = torch.empty((1, nely, nelx), dtype=torch.float32, device=dev)
        sec = torch.empty((1, nely, nelx), dtype=torch.uint8, device=dev)
    sch = schedule or WSchedule()
    w = sch.w
    hist = []
    stream = torch.cuda.current_stream(dev)
    for it in range(iters):
        t0 = time.perf_counter()
        to.project(xi, rho, stream)
        c, cg_it, cg_res = to.analyze(rho, f_d, fixed_d, stream=stream)
        to.sensitivity(xi, rho, sens, stream)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        n_sec = 0
        if imf is not None:
            r3 = rho.view(1, nely, nelx)
            imf.compute(r3, fix_d.view(1, nely, nelx), fbar, sec, stream=stream)
            imf.penalize(sens.view(1, nely, nelx), r3, fbar, sec, fix_d.view(1, nely, nelx), w_acc=w, stream=stream)
            imf.sync()
            n_sec = int(sec.sum().item())
        t2 = time.perf_counter()
        change, vol = to.update(xi, sens, fix_d, volfrac, xi_new, move=move, eta=eta, stream=stream)
        t3 = time.perf_counter()
        part = float((rho > tau).sum().item())
        hist.append({"iter": it, "compliance": c, "cg_iters": cg_it, "cg_residual": cg_res, "secluded": n_sec,
                     "w_acc": w, "change": change, "vol": vol, "fea_s": t1 - t0, "imf_s": t2 - t1, "update_s": t3 - t2})
        xi, xi_new = xi_new, xi
        if imf is not None:
            w = sch.next(w, n_sec, part)
        if change <= delta:
            break
    to.project(xi, rho, stream)
    torch.cuda.synchronize(dev)
    res = ToResult(xi.cpu().numpy(), rho.cpu().numpy(), hist)
    to.close()
    if imf is not None:
        imf.close()
    return res
