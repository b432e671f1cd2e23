"""Seeded synthetic inputs for the IMF path (designs, fixtures, tools, orientation sets).

This module is shared by the CPU oracle, the tests and the benchmark. It builds inputs only and
holds none of the IMF arithmetic (no rotation resampling, correlation, sweep or minimum).

The paper's parts (cantilever, GE bracket, quadcopter, support bracket; Sec. 3) are not
available, so these generators stand in for them with the paper's sizes: a 2D density on a
regular grid (Sec. 3.1 uses 256x128 in 2D), 3D beam-union densities of 1e5-1.7e7 voxels
(Table 3 and Sec. 3.4), a fixture slab at the bottom of the domain, and a cylindrical
cutter with a wider cylindrical holder on top (the tool assembly T = H u K of Sec. 2.1).

Array conventions: C order [nz][ny][nx] with x fastest; a 2D case has nz = 1. A tool is given
as two uint8 arrays (holder, cutter) of shape [tz][ty][tx] plus the index (ox, oy, oz) of the
tool-frame origin voxel. Orientations are unit quaternions (w, x, y, z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Tool:
    holder: np.ndarray            # uint8 [tz][ty][tx]
    cutter: np.ndarray            # uint8 [tz][ty][tx]
    origin: tuple                 # (ox, oy, oz) voxel index of the tool-frame origin
    quats: np.ndarray             # float64 [n_orient][4], (w, x, y, z)
    sharp: np.ndarray | None = None   # optional uint8 [tz][ty][tx] sharp-point subset of the cutter

    @property
    def shape_xyz(self):
        tz, ty, tx = self.cutter.shape
        return tx, ty, tz


@dataclass
class Design:
    rho: np.ndarray               # float32 [nz][ny][nx], density of the part in [0, 1]
    fixture: np.ndarray | None    # uint8 [nz][ny][nx] or None
    tools: list = field(default_factory=list)
    name: str = ""


# ----------------------------------------------------------------------------------------
# orientation sets
# ----------------------------------------------------------------------------------------

def quat_about_z(angle_rad: float) -> np.ndarray:
    """Unit quaternion of a rotation by `angle_rad` about +z (a 2D in-plane rotation)."""
    return np.array([math.cos(angle_rad / 2), 0.0, 0.0, math.sin(angle_rad / 2)])


def planar_angles(n: int, span_deg: float = 180.0) -> np.ndarray:
    """n angles k*span/(n-1), k = 0..n-1, both ends included (0 and 180 deg for n = 8)."""
    if n == 1:
        return np.zeros(1)
    return np.array([k * span_deg / (n - 1) for k in range(n)]) * math.pi / 180.0


def planar_quats(n: int, span_deg: float = 180.0) -> np.ndarray:
    return np.stack([quat_about_z(a) for a in planar_angles(n, span_deg)])


def quat_from_z_to(d) -> np.ndarray:
    """Minimal rotation taking +z to the unit vector d (axis z x d, angle acos(d_z))."""
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    ax = np.array([-d[1], d[0], 0.0])            # z x d
    s = np.linalg.norm(ax)
    if s < 1e-15:
        if d[2] > 0:
            return np.array([1.0, 0.0, 0.0, 0.0])
        return np.array([0.0, 1.0, 0.0, 0.0])    # half turn about x
    ang = math.atan2(s, d[2])
    ax = ax / s
    return np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)])


def fibonacci_hemisphere(n: int) -> np.ndarray:
    """n directions on the upper hemisphere: z_i = 1-(i+0.5)/n, phi_i = i*pi*(3-sqrt 5)."""
    out = []
    ga = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n):
        z = 1.0 - (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        out.append((r * math.cos(i * ga), r * math.sin(i * ga), z))
    return np.array(out)


def fibonacci_quats(n: int) -> np.ndarray:
    return np.stack([quat_from_z_to(d) for d in fibonacci_hemisphere(n)])


# ----------------------------------------------------------------------------------------
# tools
# ----------------------------------------------------------------------------------------

def planar_tool(cut_w=3, cut_h=12, hold_w=9, hold_h=10, n_orient=8) -> Tool:
    """2D tool: a cut_w x cut_h cutter, origin at the centre of its tip row, with a
    hold_w x hold_h holder directly above it (+y is the tool axis, tip to holder)."""
    tx = max(cut_w, hold_w)
    ty = cut_h + hold_h
    holder = np.zeros((1, ty, tx), np.uint8)
    cutter = np.zeros((1, ty, tx), np.uint8)
    c0 = (tx - cut_w) // 2
    h0 = (tx - hold_w) // 2
    cutter[0, 0:cut_h, c0:c0 + cut_w] = 1
    holder[0, cut_h:cut_h + hold_h, h0:h0 + hold_w] = 1
    origin = (c0 + cut_w // 2, 0, 0)
    return Tool(holder, cutter, origin, planar_quats(n_orient))


def cylinder_tool(r_cut=3, l_cut=20, r_hold=8, l_hold=16, quats=None) -> Tool:
    """3D tool: cutter cylinder (radius r_cut, length l_cut) with its tip at the origin and its
    axis along +z, holder cylinder (r_hold, l_hold) stacked on top of it. A voxel (i, j, k)
    with offset u from the origin is in a cylinder of radius r iff u_x^2 + u_y^2 <= r^2."""
    rr = max(r_cut, r_hold)
    tx = ty = 2 * rr + 1
    tz = l_cut + l_hold
    k, j, i = np.meshgrid(np.arange(tz), np.arange(ty), np.arange(tx), indexing="ij")
    ux, uy, uz = i - rr, j - rr, k
    d2 = ux * ux + uy * uy
    cutter = ((uz < l_cut) & (d2 <= r_cut * r_cut)).astype(np.uint8)
    holder = ((uz >= l_cut) & (d2 <= r_hold * r_hold)).astype(np.uint8)
    if quats is None:
        quats = np.array([[1.0, 0, 0, 0]])
    return Tool(holder, cutter, (rr, rr, 0), np.asarray(quats, np.float64))


def box_tool(ext=(3, 3, 3), origin=None, cutter_mask=None, quats=None) -> Tool:
    """An axis-aligned box tool of extents (ex, ey, ez); by default all of it is cutter."""
    ex, ey, ez = ext
    cutter = np.ones((ez, ey, ex), np.uint8) if cutter_mask is None else cutter_mask.astype(np.uint8)
    holder = np.zeros_like(cutter)
    if origin is None:
        origin = (0, 0, 0)
    if quats is None:
        quats = np.array([[1.0, 0, 0, 0]])
    return Tool(holder, cutter, tuple(origin), np.asarray(quats, np.float64))


# ----------------------------------------------------------------------------------------
# densities
# ----------------------------------------------------------------------------------------

def _gauss_blur(a: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma=sigma, mode="reflect")


def planar_density(nx=64, ny=64, seed=0, sigma=3.0, gain=4.0) -> np.ndarray:
    """Seeded 2D density: U(0,1) noise, Gaussian blur (sigma cells, reflecting boundary),
    z-score, then a logistic sigmoid with the given gain. Shape [1][ny][nx], float32."""
    rng = np.random.default_rng(seed)
    a = rng.random((ny, nx))
    a = _gauss_blur(a, sigma)
    a = (a - a.mean()) / (a.std() + 1e-30)
    a = 1.0 / (1.0 + np.exp(-gain * a))
    return a.astype(np.float32)[None]


def beam_density(n=(128, 128, 128), n_beams=40, r_range=(2.0, 5.0), seed=0, sigma=1.0,
                 margin=0.0) -> np.ndarray:
    """Seeded 3D density: union of n_beams capsules (segment endpoints uniform in the box,
    radius uniform in r_range), Gaussian blur (sigma voxels), clipped to [0, 1].
    n = (nx, ny, nz); returns float32 [nz][ny][nx]."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    ind = np.zeros((nz, ny, nx), np.float32)
    lo = np.array([margin, margin, margin])
    hi = np.array([nx - 1 - margin, ny - 1 - margin, nz - 1 - margin], np.float64)
    for _ in range(n_beams):
        p0 = lo + rng.random(3) * (hi - lo)
        p1 = lo + rng.random(3) * (hi - lo)
        r = r_range[0] + rng.random() * (r_range[1] - r_range[0])
        bmin = np.maximum(np.floor(np.minimum(p0, p1) - r - 1), 0).astype(int)
        bmax = np.minimum(np.ceil(np.maximum(p0, p1) + r + 1), [nx - 1, ny - 1, nz - 1]).astype(int)
        zz, yy, xx = np.meshgrid(np.arange(bmin[2], bmax[2] + 1), np.arange(bmin[1], bmax[1] + 1),
                                 np.arange(bmin[0], bmax[0] + 1), indexing="ij")
        pts = np.stack([xx, yy, zz], -1).astype(np.float64)
        d = p1 - p0
        dd = float(d @ d)
        s = np.clip(((pts - p0) @ d) / dd, 0.0, 1.0) if dd > 0 else np.zeros(pts.shape[:-1])
        q = p0 + s[..., None] * d
        inside = ((pts - q) ** 2).sum(-1) <= r * r
        sub = ind[bmin[2]:bmax[2] + 1, bmin[1]:bmax[1] + 1, bmin[0]:bmax[0] + 1]
        sub[inside] = 1.0
    if sigma > 0:
        ind = _gauss_blur(ind, sigma)
    return np.clip(ind, 0.0, 1.0).astype(np.float32)


def slab_fixture(shape_zyx, thickness: int, axis: str = "z") -> np.ndarray:
    """Fixture: the first `thickness` layers along `axis` ('z' in 3D, 'y' in 2D) are solid."""
    f = np.zeros(shape_zyx, np.uint8)
    if axis == "z":
        f[:thickness] = 1
    elif axis == "y":
        f[:, :thickness] = 1
    else:
        raise ValueError(axis)
    return f


# ----------------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------------

def config_planar64(seed=0) -> Design:
    """2D 64x64: smoothed-noise density, fixture = bottom 4 rows, 3x12 cutter with a 9x10
    holder, 8 orientations over 0-180 deg."""
    rho = planar_density(64, 64, seed=seed)
    fix = slab_fixture(rho.shape, 4, axis="y")
    return Design(rho, fix, [planar_tool()], name="planar64")


def config_beams(n=128, n_beams=40, n_orient=64, seed=0, r_cut=3, l_cut=20, r_hold=8, l_hold=16,
                 plate=6) -> Design:
    """3D beams: n^3 grid, n_beams capsules r in [2, 5], plate-thick base fixture, cylinder
    cutter (r_cut, l_cut) plus holder (r_hold, l_hold), n_orient Fibonacci-hemisphere axes."""
    if isinstance(n, int):
        n = (n, n, n)
    rho = beam_density(n, n_beams=n_beams, seed=seed)
    fix = slab_fixture(rho.shape, plate, axis="z")
    tool = cylinder_tool(r_cut, l_cut, r_hold, l_hold, fibonacci_quats(n_orient))
    return Design(rho, fix, [tool], name=f"beams{n[0]}x{n[1]}x{n[2]}_R{n_orient}")


def config_batch(n_designs=64, seed=0, lo=48, hi=192, r_lo=2, r_hi=6, nr_lo=16, nr_hi=128):
    """Uneven batch: cubic grids with log-uniform edge in [lo, hi], n_orient ~ U{nr_lo..nr_hi},
    cutter radius ~ U{r_lo..r_hi} with a holder 2.5x wider; lengths as the 3D beams tool."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n_designs):
        edge = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        nr = int(rng.integers(nr_lo, nr_hi + 1))
        rc = int(rng.integers(r_lo, r_hi + 1))
        rh = int(round(2.5 * rc))
        nb = max(4, int(40 * (edge / 128) ** 2))
        rho = beam_density((edge,) * 3, n_beams=nb, seed=seed * 1000 + d + 1)
        fix = slab_fixture(rho.shape, max(2, edge // 24), axis="z")
        tool = cylinder_tool(rc, 20, rh, 16, fibonacci_quats(nr))
        out.append(Design(rho, fix, [tool], name=f"batch{d}_{edge}_R{nr}_r{rc}"))
    return out


def cantilever2d(nelx=256, nely=128, fixture_cols=2):
    """Load case of the 2D cantilever beam (Sec. 3.1, Fig. of the beam boundary conditions; a
    reading of the figure): nelx x nely unit elements, every node of the left edge clamped, a
    unit downward force at the middle node of the right edge, and the leftmost `fixture_cols`
    element columns the clamping fixture (passive solid in the optimisation, fixture of the
    IMF). Nodes are numbered j (nelx + 1) + i with dofs (2 n, 2 n + 1) = (x, y). Returns
    (force float64 [2 (nelx+1)(nely+1)], clamped-dof mask uint8, fixture uint8 [nely][nelx])."""
    ndof = 2 * (nelx + 1) * (nely + 1)
    force = np.zeros(ndof)
    node = (nely // 2) * (nelx + 1) + nelx
    force[2 * node + 1] = -1.0
    fixed = np.zeros(ndof, np.uint8)
    for j in range(nely + 1):
        n = j * (nelx + 1)
        fixed[2 * n] = fixed[2 * n + 1] = 1
    fixture = np.zeros((nely, nelx), np.uint8)
    fixture[:, :fixture_cols] = 1
    return force, fixed, fixture


def to2d_tools(n_orient=8):
    """Two planar tool assemblies for the 2D optimisation (Sec. 3.1 uses one thin and one thick
    cutter): a 1-voxel-wide and a 3-voxel-wide cutter, 12 tall, with 7- and 9-wide holders; the
    orientations are spread over 0-180 degrees."""
    return [planar_tool(1, 12, 7, 10, n_orient=n_orient), planar_tool(3, 12, 9, 10, n_orient=n_orient)]
