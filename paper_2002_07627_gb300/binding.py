"""Thin ctypes binding of libimf (include/imf.h): argument marshalling only.

Every step of the IMF path runs in the library's CUDA kernels. There is no CPU fallback: if
the library has not been built, or no GPU is present, these calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB, HOSTLIB

IMF_OK = 0
STATUS_NAMES = {0: "IMF_OK", 1: "IMF_ERR_INVALID_ARG", 2: "IMF_ERR_OOM", 3: "IMF_ERR_CUDA",
                4: "IMF_ERR_TIMEOUT", 5: "IMF_ERR_NOT_READY", 6: "IMF_ERR_BUDGET", 7: "IMF_ERR_OVERFLOW"}
IMF_AUTO, IMF_FP32_FFT, IMF_BF16_DIRECT = 0, 1, 2
IMF_SHARP_ALL, IMF_SHARP_BOUNDARY, IMF_SHARP_NEAREST = 0, 1, 2

# every symbol include/imf.h declares
EXPORTS = ["imf_default_options", "imf_create", "imf_set_tool", "imf_compute", "imf_compute_host",
           "imf_penalize_sensitivity", "imf_sync_status", "imf_last_error", "imf_destroy",
           "imf_get_tool_info", "imf_get_offsets", "imf_set_debug", "imf_get_last_g", "imf_get_stats",
           "imf_set_profiling", "imf_get_kernel_time", "imf_reset_kernel_times",
           "imf_penalize_sensitivity_noalloc", "imf_capture_graph", "imf_launch_graph", "imf_autotune",
           "imf_set_path", "imf_selftest_mma", "imf_get_last_bits", "imf_footprint",
           "imf_compute_accessible_sets", "imf_process_plan", "imf_get_options", "imf_clone"]
# every symbol include/imf_to.h declares
EXPORTS_TO = ["imf_to2d_default_options", "imf_to2d_create", "imf_to2d_destroy", "imf_to2d_last_error",
              "imf_to2d_project", "imf_to2d_analyze", "imf_to2d_sensitivity", "imf_to2d_update", "imf_to2d_result"]


class ImfOptions(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("voxel", ctypes.c_double), ("lambda_", ctypes.c_double), ("tau", ctypes.c_double),
                ("theta_rel", ctypes.c_double), ("precision", ctypes.c_int), ("recheck", ctypes.c_int),
                ("recheck_band", ctypes.c_double), ("orient_batch", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("erode_groups", ctypes.c_int),
                ("fft_stages_only", ctypes.c_int), ("accessible_by_sweep", ctypes.c_int),
                ("separate_yx_passes", ctypes.c_int), ("plan_only", ctypes.c_int),
                ("sharp_sampling", ctypes.c_int), ("sharp_k", ctypes.c_int), ("fft_wide_pencils", ctypes.c_int),
                ("fft_tma", ctypes.c_int), ("erode_levels", ctypes.c_int),
                ("fft_tma_x", ctypes.c_int), ("sweep_loop", ctypes.c_int),
                ("erode_xt", ctypes.c_int)]


class ImfToolInfo(ctypes.Structure):
    _fields_ = [("n_orient", ctypes.c_int), ("P", ctypes.c_int * 3), ("kmax", ctypes.c_int * 3),
                ("win", ctypes.c_int * 3), ("size_T", ctypes.c_long), ("theta", ctypes.c_double),
                ("band", ctypes.c_double), ("n_rt", ctypes.c_long), ("n_rk", ctypes.c_long),
                ("n_sharp", ctypes.c_long), ("path", ctypes.c_int), ("spectra_bytes", ctypes.c_size_t)]


class ImfStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_long), ("computes", ctypes.c_long), ("flagged", ctypes.c_long),
                ("flagged_total", ctypes.c_long), ("n_kernels", ctypes.c_int), ("owned_bytes", ctypes.c_size_t)]


class To2dOptions(ctypes.Structure):
    _fields_ = [("nelx", ctypes.c_int), ("nely", ctypes.c_int), ("E0", ctypes.c_double), ("Emin", ctypes.c_double),
                ("nu", ctypes.c_double), ("penal", ctypes.c_double), ("beta", ctypes.c_double),
                ("rmin", ctypes.c_double), ("cg_tol", ctypes.c_double), ("cg_max_iter", ctypes.c_int)]


class ImfFootprint(ctypes.Structure):
    _fields_ = [("resident", ctypes.c_size_t), ("work", ctypes.c_size_t), ("setup_peak", ctypes.c_size_t),
                ("total", ctypes.c_size_t), ("slots", ctypes.c_int)]


_lib = None


def load(path: str | None = None):
    """Load libimf.so (built by paper_2002_07627_gb300.build). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libimf is not built ({path} missing): run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    P, I, D, Lg = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
    H = ctypes.c_void_p
    L.imf_default_options.argtypes = [ctypes.POINTER(ImfOptions)]
    L.imf_default_options.restype = None
    L.imf_create.argtypes = [ctypes.POINTER(ImfOptions), ctypes.POINTER(H)]
    L.imf_set_tool.argtypes = [H, I, P, P, P, I, I, I, P, P, I]
    L.imf_compute.argtypes = [H, P, P, P, P, P, P, P]
    L.imf_compute_host.argtypes = [H, P, P, P, P, P, P, P]
    L.imf_penalize_sensitivity.argtypes = [H, P, P, P, P, P, D, P]
    L.imf_sync_status.argtypes = [H]
    L.imf_last_error.argtypes = [H]
    L.imf_last_error.restype = ctypes.c_char_p
    L.imf_destroy.argtypes = [H]
    L.imf_destroy.restype = None
    L.imf_get_tool_info.argtypes = [H, I, ctypes.POINTER(ImfToolInfo)]
    L.imf_get_offsets.argtypes = [H, I, I, I, P, Lg, ctypes.POINTER(Lg)]
    L.imf_set_debug.argtypes = [H, I]
    L.imf_get_last_g.argtypes = [H, I, P, Lg, ctypes.POINTER(I)]
    L.imf_get_last_bits.argtypes = [H, I, P, Lg, ctypes.POINTER(I)]
    L.imf_get_stats.argtypes = [H, ctypes.POINTER(ImfStats)]
    L.imf_footprint.argtypes = [H, I, ctypes.POINTER(ImfFootprint)]
    L.imf_compute_accessible_sets.argtypes = [H, P, P, P, P, P, P]
    L.imf_get_options.argtypes = [H, ctypes.POINTER(ImfOptions)]
    L.imf_clone.argtypes = [H, ctypes.POINTER(H)]
    LL = ctypes.c_longlong
    L.imf_process_plan.argtypes = [H, P, I, P, P, I, P, P, ctypes.POINTER(I), ctypes.POINTER(LL),
                                   ctypes.POINTER(LL), P]
    L.imf_set_profiling.argtypes = [H, I]
    L.imf_get_kernel_time.argtypes = [H, I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(D),
                                      ctypes.POINTER(Lg)]
    L.imf_reset_kernel_times.argtypes = [H]
    L.imf_penalize_sensitivity_noalloc.argtypes = [P, P, P, P, P, Lg, D, D, P]
    L.imf_capture_graph.argtypes = [H, P, P, P, P, P, P, P]
    L.imf_launch_graph.argtypes = [H, P]
    L.imf_autotune.argtypes = [H, P, P, P, P, P, ctypes.POINTER(I)]
    L.imf_set_path.argtypes = [H, I, I]
    L.imf_selftest_mma.argtypes = [I, I, P, P, P]
    L.imf_to2d_default_options.argtypes = [ctypes.POINTER(To2dOptions)]
    L.imf_to2d_default_options.restype = None
    L.imf_to2d_create.argtypes = [ctypes.POINTER(To2dOptions), ctypes.POINTER(H)]
    L.imf_to2d_destroy.argtypes = [H]
    L.imf_to2d_destroy.restype = None
    L.imf_to2d_last_error.argtypes = [H]
    L.imf_to2d_last_error.restype = ctypes.c_char_p
    L.imf_to2d_project.argtypes = [H, P, P, P]
    L.imf_to2d_analyze.argtypes = [H, P, P, P, P, P]
    L.imf_to2d_sensitivity.argtypes = [H, P, P, P, P]
    L.imf_to2d_update.argtypes = [H, P, P, P, D, D, D, P, ctypes.POINTER(D), ctypes.POINTER(D), P]
    L.imf_to2d_result.argtypes = [H, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D)]
    for name in EXPORTS + EXPORTS_TO:
        if name not in ("imf_default_options", "imf_destroy", "imf_last_error", "imf_to2d_default_options",
                        "imf_to2d_destroy", "imf_to2d_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def host_fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Run the kernels' Stockham butterflies on the CPU (host emulation, tests only)."""
    L = ctypes.CDLL(HOSTLIB)
    L.imf_host_fft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    a = np.ascontiguousarray(np.stack([x.real, x.imag], -1).astype(np.float32))
    out = np.zeros_like(a)
    rc = L.imf_host_fft(len(x), sign, a.ctypes.data, out.ctypes.data)
    if rc < 0:
        raise ValueError(f"no plan for length {len(x)}")
    return out[..., 0].astype(np.float64) + 1j * out[..., 1]


def host_fft2(x: np.ndarray, sign: int = -1):
    """Run the kernels' two-pass register transform on the CPU (host emulation, tests only).
    Returns (spectrum, (A, B)) or raises ValueError when the length has no supported split."""
    L = ctypes.CDLL(HOSTLIB)
    L.imf_host_fft2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    a = np.ascontiguousarray(np.stack([x.real, x.imag], -1).astype(np.float32))
    out = np.zeros_like(a)
    rc = L.imf_host_fft2(len(x), sign, a.ctypes.data, out.ctypes.data)
    if rc < 0:
        raise ValueError(f"no two-pass split for length {len(x)}")
    return out[..., 0].astype(np.float64) + 1j * out[..., 1], (rc // 100, rc % 100)


class ImfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


@dataclass
class ToolInfo:
    n_orient: int
    P: tuple
    kmax: tuple
    win: tuple
    size_T: int
    theta: float
    band: float
    n_rt: int
    n_rk: int
    n_sharp: int
    path: int
    spectra_bytes: int


class Imf:
    """One design grid on the current CUDA device; mirrors the C ABI one-to-one."""

    def __init__(self, shape_zyx, lam=0.01, tau=0.5, theta_rel=0.01, precision=IMF_AUTO, recheck=True,
                 recheck_band=0.0, orient_batch=0, hbm_budget_bytes=0, voxel=1.0, erode_groups=0, fft_stages_only=False,
                 accessible_by_sweep=False, separate_yx_passes=False, plan_only=False, sharp_sampling=IMF_SHARP_ALL,
                 sharp_k=1, fft_wide_pencils=-1, fft_tma=-1, erode_levels=False, fft_tma_x=-1,
                 sweep_loop=False, erode_xt=0):
        self.lib = load()
        opt = ImfOptions()
        self.lib.imf_default_options(ctypes.byref(opt))
        nz, ny, nx = shape_zyx
        opt.nx, opt.ny, opt.nz = nx, ny, nz
        opt.voxel, opt.lambda_, opt.tau, opt.theta_rel = voxel, lam, tau, theta_rel
        opt.precision, opt.recheck, opt.recheck_band = precision, int(recheck), recheck_band
        opt.orient_batch, opt.hbm_budget_bytes = orient_batch, hbm_budget_bytes
        opt.erode_groups = erode_groups
        opt.fft_stages_only = int(fft_stages_only)
        opt.accessible_by_sweep = int(accessible_by_sweep)
        opt.separate_yx_passes = int(separate_yx_passes)
        opt.plan_only = int(plan_only)
        opt.sharp_sampling, opt.sharp_k = int(sharp_sampling), int(sharp_k)
        opt.fft_wide_pencils = int(fft_wide_pencils)
        opt.fft_tma = int(fft_tma)
        opt.erode_levels = int(erode_levels)
        opt.fft_tma_x = int(fft_tma_x)
        opt.sweep_loop = int(sweep_loop)
        opt.erode_xt = int(erode_xt)
        self.shape = (nz, ny, nx)
        self.opt = opt
        h = ctypes.c_void_p()
        self._check(self.lib.imf_create(ctypes.byref(opt), ctypes.byref(h)), handle=None)
        self.h = h

    def _check(self, st, handle="self"):
        if st != IMF_OK:
            msg = ""
            if handle is not None and getattr(self, "h", None):
                msg = self.lib.imf_last_error(self.h).decode()
            raise ImfError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.imf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- setup
    def set_tool(self, tool_id, holder, cutter, origin, quats, sharp=None):
        holder = np.ascontiguousarray(holder, np.uint8)
        cutter = np.ascontiguousarray(cutter, np.uint8)
        tz, ty, tx = cutter.shape
        if holder.shape != cutter.shape:
            raise ValueError("holder and cutter shapes differ")
        sh = None if sharp is None else np.ascontiguousarray(sharp, np.uint8)
        o = (ctypes.c_int * 3)(*[int(v) for v in origin])
        q = np.ascontiguousarray(np.asarray(quats, np.float64).reshape(-1, 4))
        self._check(self.lib.imf_set_tool(self.h, tool_id, holder.ctypes.data, cutter.ctypes.data,
                                          None if sh is None else sh.ctypes.data, tx, ty, tz, o,
                                          q.ctypes.data, len(q)))

    def set_tools(self, tools):
        for i, t in enumerate(tools):
            self.set_tool(i, t.holder, t.cutter, t.origin, t.quats, getattr(t, "sharp", None))
        self.n_tools = len(tools)

    # --- compute (torch CUDA tensors)
    def compute(self, rho, fixture=None, fbar=None, secluded=None, raw=None, accessible=None, stream=None):
        import torch
        self._check_tensor(rho, torch.float32)
        if fixture is not None:
            self._check_tensor(fixture, torch.uint8)
        if fbar is None:
            fbar = torch.empty_like(rho)
        if secluded is None:
            secluded = torch.empty(rho.shape, dtype=torch.uint8, device=rho.device)
        s = (stream or torch.cuda.current_stream(rho.device)).cuda_stream
        self._check(self.lib.imf_compute(self.h, _ptr(rho), _ptr(fixture), _ptr(fbar), _ptr(secluded),
                                         _ptr(raw), _ptr(accessible), s))
        return fbar, secluded

    def compute_host(self, rho: np.ndarray, fixture=None, want_raw=True, want_acc=True, stream=None):
        rho = np.ascontiguousarray(rho, np.float32)
        fix = None if fixture is None else np.ascontiguousarray(fixture, np.uint8)
        fbar = np.empty(self.shape, np.float32)
        sec = np.empty(self.shape, np.uint8)
        raw = np.empty(self.shape, np.float32) if want_raw else None
        acc = np.empty(self.shape, np.uint8) if want_acc else None
        s = 0 if stream is None else stream.cuda_stream
        p = lambda a: None if a is None else a.ctypes.data
        self._check(self.lib.imf_compute_host(self.h, p(rho), p(fix), p(fbar), p(sec), p(raw), p(acc), s))
        return fbar, sec, raw, acc

    def penalize(self, sens, rho, fbar, secluded, fixture=None, w_acc=0.5, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream(sens.device)).cuda_stream
        self._check(self.lib.imf_penalize_sensitivity(self.h, _ptr(sens), _ptr(rho), _ptr(fbar), _ptr(secluded),
                                                      _ptr(fixture), float(w_acc), s))
        return sens

    def accessible_sets(self, rho, fixture=None, stream=None):
        """Per-orientation accessible sets (imf_compute_accessible_sets) as a uint32 tensor
        [n_orient_total][nz][ny][(nx + 31) // 32]; also returns f_bar and Gamma."""
        import torch
        nz, ny, nx = self.shape
        n = sum(self.tool_info(i).n_orient for i in range(self.n_tools))
        sets = torch.empty((n, nz, ny, (nx + 31) // 32), dtype=torch.int32, device=rho.device)
        fbar = torch.empty_like(rho)
        sec = torch.empty(rho.shape, dtype=torch.uint8, device=rho.device)
        s = (stream or torch.cuda.current_stream(rho.device)).cuda_stream
        self._check(self.lib.imf_compute_accessible_sets(self.h, _ptr(rho), _ptr(fixture), _ptr(fbar), _ptr(sec),
                                                         _ptr(sets), s))
        return sets, fbar, sec

    def process_plan(self, sets, rho, fixture=None, max_steps=None, stream=None):
        """Greedy process plan (imf_process_plan): list of (set index, voxels removed), |N| and
        the inaccessible rest."""
        import torch
        n_sets = int(sets.shape[0])
        max_steps = n_sets if max_steps is None else int(max_steps)
        order = np.zeros(max(1, max_steps), np.int32)
        removed = np.zeros(max(1, max_steps), np.int64)
        n_steps = ctypes.c_int()
        neg, left = ctypes.c_longlong(), ctypes.c_longlong()
        s = (stream or torch.cuda.current_stream(rho.device)).cuda_stream
        self._check(self.lib.imf_process_plan(self.h, _ptr(sets), n_sets, _ptr(rho), _ptr(fixture), max_steps,
                                              order.ctypes.data, removed.ctypes.data, ctypes.byref(n_steps),
                                              ctypes.byref(neg), ctypes.byref(left), s))
        k = n_steps.value
        return list(zip(order[:k].tolist(), removed[:k].tolist())), neg.value, left.value

    def capture_graph(self, rho, fixture, fbar, secluded, raw=None, accessible=None, stream=None):
        """Record one compute with these exact tensors into a replayable CUDA graph."""
        import torch
        s = (stream or torch.cuda.current_stream(rho.device)).cuda_stream
        self._check(self.lib.imf_capture_graph(self.h, _ptr(rho), _ptr(fixture), _ptr(fbar), _ptr(secluded),
                                               _ptr(raw), _ptr(accessible), s))

    def launch_graph(self, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.imf_launch_graph(self.h, s))

    def autotune(self, rho, fixture=None, stream=None) -> int:
        import torch
        fb = torch.empty_like(rho)
        sec = torch.empty(rho.shape, dtype=torch.uint8, device=rho.device)
        s = (stream or torch.cuda.current_stream(rho.device)).cuda_stream
        best = ctypes.c_int()
        self._check(self.lib.imf_autotune(self.h, _ptr(rho), _ptr(fixture), _ptr(fb), _ptr(sec), s,
                                          ctypes.byref(best)))
        return best.value

    def options(self) -> dict:
        """The handle's current options (imf_get_options; the tuned ones after autotune)."""
        o = ImfOptions()
        self._check(self.lib.imf_get_options(self.h, ctypes.byref(o)))
        return {name: getattr(o, name) for name, _ in ImfOptions._fields_}

    def clone(self) -> "Imf":
        """A second handle sharing this one's tools, with its own work buffers (imf_clone)."""
        h = ctypes.c_void_p()
        self._check(self.lib.imf_clone(self.h, ctypes.byref(h)))
        c = Imf.__new__(Imf)
        c.lib, c.opt, c.shape, c.h = self.lib, self.opt, self.shape, h
        c.n_tools = getattr(self, "n_tools", 1)
        return c

    def set_path(self, tool_id, path):
        self._check(self.lib.imf_set_path(self.h, tool_id, path))

    def sync(self):
        self._check(self.lib.imf_sync_status(self.h))

    # --- introspection
    def tool_info(self, tool_id=0) -> ToolInfo:
        info = ImfToolInfo()
        self._check(self.lib.imf_get_tool_info(self.h, tool_id, ctypes.byref(info)))
        return ToolInfo(info.n_orient, tuple(info.P), tuple(info.kmax), tuple(info.win), info.size_T, info.theta,
                        info.band, info.n_rt, info.n_rk, info.n_sharp, info.path, info.spectra_bytes)

    def offsets(self, tool_id, orient, which) -> np.ndarray:
        n = ctypes.c_long()
        self._check(self.lib.imf_get_offsets(self.h, tool_id, orient, which, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 3), np.int32)
        self._check(self.lib.imf_get_offsets(self.h, tool_id, orient, which, out.ctypes.data, n.value,
                                             ctypes.byref(n)))
        return out[:n.value]

    def last_g(self, slot=0):
        info = self.tool_info(0)
        o = ctypes.c_int()
        self._check(self.lib.imf_get_last_g(self.h, slot, None, 0, ctypes.byref(o)))
        wx, wy, wz = info.win
        gpx = (wx + 3) & ~3
        buf = np.zeros(wz * wy * gpx, np.float32)
        self._check(self.lib.imf_get_last_g(self.h, slot, buf.ctypes.data, buf.size, ctypes.byref(o)))
        return o.value, buf.reshape(wz, wy, gpx)[:, :, :wx]

    def set_debug(self, keep_last_g=True):
        """Keep the last orientation batch's collision field and free bits (tests)."""
        self._check(self.lib.imf_set_debug(self.h, int(keep_last_g)))

    def last_bits(self, slot=0):
        """(caller's orientation index, free flags [wz][wy][wx] as uint8) of a slot of the last
        batch, unpacked from the library's bit words."""
        info = self.tool_info(0)
        o = ctypes.c_int()
        wx, wy, wz = info.win
        wpr = (wx + 31) // 32 + 2
        buf = np.zeros(wz * wy * wpr, np.uint32)
        self._check(self.lib.imf_get_last_bits(self.h, slot, buf.ctypes.data, buf.size, ctypes.byref(o)))
        bits = np.unpackbits(buf.view(np.uint8).reshape(wz, wy, wpr * 4), axis=-1, bitorder="little")
        return o.value, bits[:, :, :wx]

    def stats(self) -> ImfStats:
        s = ImfStats()
        self._check(self.lib.imf_get_stats(self.h, ctypes.byref(s)))
        return s

    def footprint(self, slots=0) -> ImfFootprint:
        """Planned device bytes of this handle (imf_footprint); `slots` orientation slots of work
        buffers, 0 = the first compute's default."""
        f = ImfFootprint()
        self._check(self.lib.imf_footprint(self.h, int(slots), ctypes.byref(f)))
        return f

    def set_profiling(self, on=True):
        self._check(self.lib.imf_set_profiling(self.h, int(on)))

    def kernel_times(self) -> dict:
        out = {}
        st = self.stats()
        for i in range(st.n_kernels):
            name = ctypes.c_char_p()
            ms = ctypes.c_double()
            cnt = ctypes.c_long()
            self._check(self.lib.imf_get_kernel_time(self.h, i, ctypes.byref(name), ctypes.byref(ms),
                                                     ctypes.byref(cnt)))
            if cnt.value:
                out[name.value.decode()] = (ms.value, cnt.value)
        return out

    def reset_kernel_times(self):
        self._check(self.lib.imf_reset_kernel_times(self.h))

    @staticmethod
    def _check_tensor(t, dtype):
        if not t.is_cuda:
            raise ValueError("libimf takes CUDA tensors (device memory); use compute_host for host arrays")
        if t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"expected a contiguous {dtype} tensor")


class To2d:
    """The SIMP steps of the topology-optimisation loop (include/imf_to.h) for a 2D grid of
    nelx x nely unit elements on the current CUDA device; mirrors the C ABI one-to-one."""

    def __init__(self, nelx, nely, **kw):
        self.lib = load()
        o = To2dOptions()
        self.lib.imf_to2d_default_options(ctypes.byref(o))
        o.nelx, o.nely = int(nelx), int(nely)
        for k, v in kw.items():
            setattr(o, k, v)
        self.opt = o
        h = ctypes.c_void_p()
        st = self.lib.imf_to2d_create(ctypes.byref(o), ctypes.byref(h))
        if st != IMF_OK:
            raise ImfError(st, "imf_to2d_create")
        self.h = h

    def _check(self, st):
        if st != IMF_OK:
            raise ImfError(st, self.lib.imf_to2d_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.imf_to2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _s(stream, t):
        import torch
        return (stream or torch.cuda.current_stream(t.device)).cuda_stream

    def project(self, xi, rho, stream=None):
        self._check(self.lib.imf_to2d_project(self.h, _ptr(xi), _ptr(rho), self._s(stream, xi)))
        return rho

    def analyze(self, rho, force, fixed, u=None, stream=None):
        """FEA; returns (compliance, CG iterations, relative residual)."""
        self._check(self.lib.imf_to2d_analyze(self.h, _ptr(rho), _ptr(force), _ptr(fixed), _ptr(u),
                                              self._s(stream, rho)))
        c, it, res = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.imf_to2d_result(self.h, ctypes.byref(c), ctypes.byref(it), ctypes.byref(res)))
        return c.value, it.value, res.value

    def sensitivity(self, xi, rho, sens, stream=None):
        self._check(self.lib.imf_to2d_sensitivity(self.h, _ptr(xi), _ptr(rho), _ptr(sens), self._s(stream, xi)))
        return sens

    def update(self, xi, S, passive, volfrac, xi_new, move=0.2, eta=0.5, stream=None):
        """OC update; returns (mean |xi_new - xi| over free elements, mean projected density)."""
        chg, vol = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.imf_to2d_update(self.h, _ptr(xi), _ptr(S), _ptr(passive), float(volfrac), float(move),
                                             float(eta), _ptr(xi_new), ctypes.byref(chg), ctypes.byref(vol),
                                             self._s(stream, xi)))
        return chg.value, vol.value
