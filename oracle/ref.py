"""Orchestration of the FP64 oracle in the order of Algorithm 1 (arXiv 2002.07627, Sec. 2.1.5).

Test infrastructure only (see the package docstring). The heavy definitions are in
`imf_oracle.c`; this module calls them per tool and per orientation and applies the
normalisation, allowance, secluded-region and sensitivity-penalty definitions in NumPy FP64.

Readings of the paper used here (each is listed with its reason in the design notes):
  * minima start at +inf (Alg. 1 initialises them to 0, which would make every minimum 0);
  * h(x) = g(x - Rk) as in Eq. eq_imf_2 (Alg. 1 writes Translate(g, -Rk));
  * rho_O = min(1, rho_Omega + 1_F) and 1_T = 1_H OR 1_K (the implicit unions of Alg. 1);
  * free translations are g <= theta_i with theta_i = theta_rel * |T_i| (sign() of Eq.
    eq_conv_D thresholds at 0, which is degenerate for densities in (0, 1));
  * everything outside the grid is empty air; Omega_0 is the set of grid cells outside the
    fixture; the maximum M and the outputs f_bar, A and Gamma are taken on Omega_0 only;
  * f_bar = f / M with M = max over Omega_0 of f; M = 0 gives f_bar = 0 and an empty Gamma;
  * sharp points default to every voxel of the resampled cutter [1_RK]; a user subset is
    given as an indicator over the cutter array and resampled by the same rule, so it is
    always a subset of RK;
  * S_phi is normalised by max |S_phi| over Omega_0 (left unchanged when that is 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "imf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, OpenMP, no floating-point contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
           "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I = ctypes.c_int
        Lg = ctypes.c_long
        L.oracle_quat_to_matrix.argtypes = [P, P]
        L.oracle_rotate_box.argtypes = [I, I, I, P, P, P, P]
        L.oracle_rotate.argtypes = [P, I, I, I, P, P, P, P, P]
        L.oracle_rotate.restype = Lg
        L.oracle_collision.argtypes = [P, I, I, I, P, Lg, P, P, P]
        L.oracle_sweep.argtypes = [P, P, P, P, Lg, I, I, I, P, P]
        L.oracle_erode.argtypes = [P, P, P, P, Lg, I, I, I, P]
        L.oracle_erode.restype = I
        L.oracle_point_query.argtypes = [P, I, I, I, I, P, P, P, P, P, P, P, Lg, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i3(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))


# ----------------------------------------------------------------------------------------
# rotation and resampling (Alg. 1 "Rotate"; Sec. 2.1.5)
# ----------------------------------------------------------------------------------------

def quat_to_matrix(q) -> np.ndarray:
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(4))
    R = np.zeros(9, np.float64)
    lib().oracle_quat_to_matrix(_p(q), _p(R))
    return R.reshape(3, 3)


def rotate_indicator(arr: np.ndarray, origin, R: np.ndarray):
    """Resample the binary array arr[tz][ty][tx] under R about `origin` (x, y, z).
    Returns (lo (3,), dense uint8 box [ez][ey][ex]) on the conservative box."""
    arr = np.ascontiguousarray(arr, dtype=np.uint8)
    tz, ty, tx = arr.shape
    o = _i3(origin)
    Rf = np.ascontiguousarray(np.asarray(R, np.float64).reshape(9))
    lo = np.zeros(3, np.int32)
    ext = np.zeros(3, np.int32)
    lib().oracle_rotate_box(tx, ty, tz, _p(o), _p(Rf), _p(lo), _p(ext))
    out = np.zeros((ext[2], ext[1], ext[0]), np.uint8)
    lib().oracle_rotate(_p(arr), tx, ty, tz, _p(o), _p(Rf), _p(lo), _p(ext), _p(out))
    return lo, out


def offsets_of(lo, box: np.ndarray) -> np.ndarray:
    """Offsets (x, y, z) of the ones of a dense box, in [z][y][x] scan order (int32 [n][3])."""
    z, y, x = np.nonzero(box)
    return np.ascontiguousarray(np.stack([x + lo[0], y + lo[1], z + lo[2]], -1).astype(np.int32))


def resample_tool(tool, q) -> dict:
    """Rotated tool assembly RT = R(H OR K), cutter RK = R K and the sharp points for one
    orientation (Alg. 1: Define 1_T = 1_H + 1_K, then Rotate; sharp points = Support(1_RK))."""
    R = quat_to_matrix(q)
    T = ((tool.holder != 0) | (tool.cutter != 0)).astype(np.uint8)
    lo_t, box_t = rotate_indicator(T, tool.origin, R)
    lo_k, box_k = rotate_indicator(tool.cutter, tool.origin, R)
    RT = offsets_of(lo_t, box_t)
    RK = offsets_of(lo_k, box_k)
    if getattr(tool, "sharp", None) is None:
        sharp = RK
    else:
        # sharp points given as an indicator over the cutter array, resampled like the cutter
        mask = ((np.asarray(tool.sharp) != 0) & (tool.cutter != 0)).astype(np.uint8)
        lo_s, box_s = rotate_indicator(mask, tool.origin, R)
        sharp = offsets_of(lo_s, box_s)
    return dict(R=R, RT=RT, RK=RK, sharp=sharp, size_T=int(T.sum()))


# ----------------------------------------------------------------------------------------
# the per-orientation definitions
# ----------------------------------------------------------------------------------------

def sharp_sample(cutter, origin, mode: str, k: int = 1) -> np.ndarray:
    """Sharp-point sample of a cutter array [tz][ty][tx] in the tool frame (Sec. 2.1.5: the
    cutter boundary may be sampled more or less densely; App. B: down to O(1) representative
    points). mode "all": every cutter voxel; "boundary": cutter voxels with at least one of the
    six face neighbours outside the cutter (or outside the array); "nearest": the k boundary
    voxels with the smallest squared distance to the tool origin (x, y, z), ties broken by the
    C-order index. Returns a uint8 mask."""
    K = np.asarray(cutter) != 0
    if mode == "all":
        return K.astype(np.uint8)
    P = np.pad(K, 1, constant_values=False)
    inner = (P[:-2, 1:-1, 1:-1] & P[2:, 1:-1, 1:-1] & P[1:-1, :-2, 1:-1] & P[1:-1, 2:, 1:-1] &
             P[1:-1, 1:-1, :-2] & P[1:-1, 1:-1, 2:])
    B = K & ~inner
    if mode == "boundary":
        return B.astype(np.uint8)
    if mode != "nearest":
        raise ValueError(mode)
    z, y, x = np.nonzero(B)
    d2 = (x - origin[0]) ** 2 + (y - origin[1]) ** 2 + (z - origin[2]) ** 2
    lin = np.ravel_multi_index((z, y, x), K.shape)
    order = np.lexsort((lin, d2))[:k]
    out = np.zeros(K.shape, np.uint8)
    out[z[order], y[order], x[order]] = 1
    return out


def rho_obstacle(rho, fixture) -> np.ndarray:
    """rho_O = min(1, rho_Omega + 1_F) in FP64 (Alg. 1 "implicit union", Eq. eq_imf_4)."""
    r = np.asarray(rho, np.float64)
    if fixture is not None:
        r = np.minimum(1.0, r + (np.asarray(fixture) != 0))
    return np.ascontiguousarray(r)


def collision(rhoO: np.ndarray, RT: np.ndarray, tlo, text) -> np.ndarray:
    """g(t) = sum_{v in RT} rho_O(t + v) on the box (tlo, text) (Eq. eq_ident)."""
    nz, ny, nx = rhoO.shape
    text = _i3(text)
    g = np.zeros((text[2], text[1], text[0]), np.float64)
    RT = np.ascontiguousarray(RT, np.int32)
    lib().oracle_collision(_p(rhoO), nx, ny, nz, _p(RT), len(RT), _p(_i3(tlo)), _p(text), _p(g))
    return g


def sweep(freeb: np.ndarray, tlo, RK: np.ndarray, shape_zyx, count: bool = False):
    """A(x) = [sum_{k in RK} free(x - k) > 0] on the grid (Eq. eq_conv_A)."""
    nz, ny, nx = shape_zyx
    freeb = np.ascontiguousarray(freeb, np.uint8)
    text = _i3(freeb.shape[::-1])
    A = np.zeros(shape_zyx, np.uint8)
    cnt = np.zeros(shape_zyx, np.int32) if count else None
    RK = np.ascontiguousarray(RK, np.int32)
    lib().oracle_sweep(_p(freeb), _p(_i3(tlo)), _p(text), _p(RK), len(RK), nx, ny, nz, _p(A),
                       _p(cnt) if count else None)
    return (A, cnt) if count else A


def erode(g: np.ndarray, tlo, sharp: np.ndarray, shape_zyx) -> np.ndarray:
    """gamma(x) = min_{k in sharp} g(x - k) on the grid (Eq. eq_imf_2)."""
    nz, ny, nx = shape_zyx
    g = np.ascontiguousarray(g, np.float64)
    text = _i3(g.shape[::-1])
    out = np.zeros(shape_zyx, np.float64)
    sharp = np.ascontiguousarray(sharp, np.int32)
    rc = lib().oracle_erode(_p(g), _p(_i3(tlo)), _p(text), _p(sharp), len(sharp), nx, ny, nz, _p(out))
    if rc != 0:
        raise ValueError("erosion query outside the translation box")
    return out


def translation_box(shape_zyx, *offset_lists):
    """Box of translations t = x - k for x on the grid and k in any of the lists."""
    nz, ny, nx = shape_zyx
    n = np.array([nx, ny, nz])
    allk = np.concatenate([k for k in offset_lists if len(k)], 0)
    kmin = allk.min(0)
    kmax = allk.max(0)
    tlo = -kmax
    text = (n - 1 - kmin) - tlo + 1
    return tlo.astype(np.int32), text.astype(np.int32)


# ----------------------------------------------------------------------------------------
# Algorithm 1 and the sensitivity penalty
# ----------------------------------------------------------------------------------------

def finalize(f: np.ndarray, rho, fixture, lam: float, tau: float):
    """Normalisation, allowance and secluded region (Alg. 1, last four steps):
    M = max_{Omega_0} f;  f_bar = f / M;  B = [f_bar > lam];  f_bar <- f_bar * B;
    Gamma = Omega_0 * [rho <= tau] * B. Fixture cells get f_bar = 0 and Gamma = 0."""
    f = np.asarray(f, np.float64)
    omega0 = np.ones(f.shape, bool) if fixture is None else (np.asarray(fixture) == 0)
    M = float(f[omega0].max()) if omega0.any() else 0.0
    if M > 0 and np.isfinite(M):
        fbar = f / M
    else:
        fbar = np.zeros_like(f)
    fbar = np.where(omega0, fbar, 0.0)
    B = fbar > lam
    fbar = fbar * B
    solid = np.asarray(rho, np.float64) > tau
    gamma = omega0 & ~solid & B
    return fbar, gamma.astype(np.uint8), M


def imf(design, lam: float = 0.01, tau: float = 0.5, theta_rel: float = 0.01,
        keep: bool = False) -> dict:
    """Algorithm 1 with the readings listed in the module docstring, for every tool of the
    design (Eq. eq_imf_3 / eq_imf_5: minimum over tools, union of accessible sets)."""
    rho = np.asarray(design.rho)
    shape = rho.shape
    rhoO = rho_obstacle(rho, design.fixture)
    f = np.full(shape, np.inf)
    A = np.zeros(shape, bool)
    per = []
    for tool in design.tools:
        T = (tool.holder != 0) | (tool.cutter != 0)
        theta = theta_rel * float(T.sum())
        for q in tool.quats:
            rs = resample_tool(tool, q)
            if len(rs["RK"]) == 0:
                per.append(None)
                continue
            tlo, text = translation_box(shape, rs["RK"], rs["sharp"])
            g = collision(rhoO, rs["RT"], tlo, text)
            free = (g <= theta).astype(np.uint8)
            A_R = sweep(free, tlo, rs["RK"], shape)
            gam = erode(g, tlo, rs["sharp"], shape) if len(rs["sharp"]) else np.full(shape, np.inf)
            f = np.minimum(f, gam)
            A |= A_R.astype(bool)
            if keep:
                per.append(dict(rs, tlo=tlo, g=g, free=free, A=A_R, gamma=gam, theta=theta))
    fbar, gam_sec, M = finalize(f, rho, design.fixture, lam, tau)
    omega0 = np.ones(shape, bool) if design.fixture is None else (np.asarray(design.fixture) == 0)
    out = dict(f=f, fbar=fbar, secluded=gam_sec, accessible=(A & omega0).astype(np.uint8), M=M)
    if keep:
        out["per_orientation"] = per
    return out


def penalize(sens, rho, fbar, secluded, fixture, w_acc: float, tau: float = 0.5) -> np.ndarray:
    """Filtered sensitivity (Eq. eq_filtered_sens with the filter of Eq. eq_accFilter):
    S = (1 - w) S_phi / max_{Omega_0}|S_phi| + w S_IMF, where S_IMF = f_bar on Omega
    (rho > tau), 1 on Gamma, 0 elsewhere."""
    s = np.asarray(sens, np.float64)
    omega0 = np.ones(s.shape, bool) if fixture is None else (np.asarray(fixture) == 0)
    m = float(np.abs(s[omega0]).max()) if omega0.any() else 0.0
    sbar = s / m if m > 0 else s
    solid = np.asarray(rho, np.float64) > tau
    s_imf = np.where(solid, np.asarray(fbar, np.float64), np.where(np.asarray(secluded) != 0, 1.0, 0.0))
    return (1.0 - w_acc) * sbar + w_acc * s_imf


def point_query(rho, fixture, tools, pts, theta_rel: float = 0.01):
    """f(x) and A(x) (before normalisation) at the given grid points (x, y, z), computed by the
    literal definitions, for grids too large for a full oracle run."""
    rhoO = rho_obstacle(rho, fixture)
    nz, ny, nx = rhoO.shape
    rt, sh, rk, nrt, nsh, nrk, th = [], [], [], [], [], [], []
    for tool in tools:
        T = (tool.holder != 0) | (tool.cutter != 0)
        theta = theta_rel * float(T.sum())
        for q in tool.quats:
            rs = resample_tool(tool, q)
            rt.append(rs["RT"]); sh.append(rs["sharp"]); rk.append(rs["RK"])
            nrt.append(len(rs["RT"])); nsh.append(len(rs["sharp"])); nrk.append(len(rs["RK"]))
            th.append(theta)

    def cat(lst):
        a = [x.reshape(-1, 3) for x in lst if len(x)]
        return np.ascontiguousarray(np.concatenate(a, 0) if a else np.zeros((1, 3)), np.int32)

    RTc, SHc, RKc = cat(rt), cat(sh), cat(rk)
    nrt = np.asarray(nrt, np.int64); nsh = np.asarray(nsh, np.int64); nrk = np.asarray(nrk, np.int64)
    th = np.asarray(th, np.float64)
    pts = np.ascontiguousarray(np.asarray(pts, np.int32).reshape(-1, 3))
    f = np.zeros(len(pts), np.float64)
    A = np.zeros(len(pts), np.uint8)
    lib().oracle_point_query(_p(rhoO), nx, ny, nz, len(nrt), _p(RTc), _p(nrt), _p(SHc), _p(nsh),
                             _p(RKc), _p(nrk), _p(th), len(pts), _p(pts), _p(f), _p(A))
    return f, A


def imf_subblock(design, x0, ext, theta_rel: float = 0.01):
    """f and A (before normalisation) on the sub-block [x0, x0 + ext) of a large grid, by the
    same literal steps as `imf` (direct FP64 collision sums on the translations the block
    needs, brute-force sweep and minimum), with the whole design as obstacle. x0, ext are
    (x, y, z)."""
    rho = np.asarray(design.rho)
    rhoO = rho_obstacle(rho, design.fixture)
    x0 = np.asarray(x0, np.int32)
    ext = np.asarray(ext, np.int32)
    shape = (int(ext[2]), int(ext[1]), int(ext[0]))
    f = np.full(shape, np.inf)
    A = np.zeros(shape, bool)
    for tool in design.tools:
        T = (tool.holder != 0) | (tool.cutter != 0)
        theta = theta_rel * float(T.sum())
        for q in tool.quats:
            rs = resample_tool(tool, q)
            if len(rs["RK"]) == 0:
                continue
            tlo_rel, text = translation_box(shape, rs["RK"], rs["sharp"])
            g = collision(rhoO, rs["RT"], tlo_rel + x0, text)
            free = (g <= theta).astype(np.uint8)
            A |= sweep(free, tlo_rel, rs["RK"], shape).astype(bool)
            if len(rs["sharp"]):
                f = np.minimum(f, erode(g, tlo_rel, rs["sharp"], shape))
    return f, A.astype(np.uint8)


def process_plan(sets, negative, max_steps=None):
    """Greedy machining process plan (Sec. 3.4.1): starting from the whole negative space N
    (a boolean grid), each step takes the oriented tool whose accessible set (one boolean grid
    per orientation, `sets`) covers the most of what is left of N, lowest index on ties, and
    removes that part; it stops when N is empty or no set covers any of the rest. Returns
    ([(set index, voxels removed), ...], |N|, voxels left)."""
    rem = np.asarray(negative, bool).copy()
    total = int(rem.sum())
    steps = []
    limit = len(sets) if max_steps is None else max_steps
    while rem.any() and len(steps) < limit:
        counts = [int(np.count_nonzero(np.asarray(s, bool) & rem)) for s in sets]
        best = int(np.argmax(counts))
        if counts[best] == 0:
            break
        steps.append((best, counts[best]))
        rem &= ~np.asarray(sets[best], bool)
    return steps, total, int(rem.sum())
