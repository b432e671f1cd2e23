"""Independent set-based brute force for tiny grids (test infrastructure only).

Shares no code with `imf_oracle.c`: tools are rotated only by exact quarter turns (integer
permutations of the offset set, no floating point), collisions are counted by set or dict
lookups, and the accessible set is built as the explicit Minkowski sum of the free
translations with the rotated cutter (Eq. eq_A of Sec. 2.1.1):
    A_R = Omega_0 n ((O + (-RT))^c + RK),
where (O + (-RT))^c is taken inside the box of translations that can touch the grid.
"""
from __future__ import annotations

import itertools

import numpy as np


def tool_offsets(arr: np.ndarray, origin) -> list:
    """Offsets u = index - origin of the ones of arr[tz][ty][tx], as (x, y, z) tuples."""
    z, y, x = np.nonzero(arr)
    ox, oy, oz = origin
    return [(int(a - ox), int(b - oy), int(c - oz)) for a, b, c in zip(x, y, z)]


def quarter_turn(u, axis: str, k: int):
    """Rotate an integer offset by k quarter turns (counter-clockwise, right-hand rule)."""
    x, y, z = u
    for _ in range(k % 4):
        if axis == "z":
            x, y = -y, x
        elif axis == "x":
            y, z = -z, y
        elif axis == "y":
            z, x = -x, z
    return (x, y, z)


def rotate_set(offsets, turns) -> list:
    """Apply a sequence of (axis, k) quarter turns, first element first."""
    out = []
    for u in offsets:
        v = u
        for axis, k in turns:
            v = quarter_turn(v, axis, k)
        out.append(v)
    return sorted(set(out))


def brute_imf(rho: np.ndarray, fixture, orientations, theta: float):
    """f(x) = min_R min_{k in RK} sum_{v in RT} rho_O(x - k + v) and the accessible set
    A = U_R ((free translations) + RK) n Omega_0, by explicit enumeration.
    `orientations` is a list of (RT, RK) offset lists. rho may be binary or a density."""
    nz, ny, nx = rho.shape
    rhoO = rho.astype(np.float64).copy()
    if fixture is not None:
        rhoO = np.minimum(1.0, rhoO + (fixture != 0))
    dens = {}
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if rhoO[z, y, x] != 0:
            dens[(x, y, z)] = rhoO[z, y, x]
    grid = list(itertools.product(range(nx), range(ny), range(nz)))
    f = {p: np.inf for p in grid}
    acc = set()
    for RT, RK in orientations:
        cache = {}

        def g(t):
            if t not in cache:
                cache[t] = sum(dens.get((t[0] + v[0], t[1] + v[1], t[2] + v[2]), 0.0) for v in RT)
            return cache[t]

        # translations that bring some cutter voxel onto the grid
        trans = {(p[0] - k[0], p[1] - k[1], p[2] - k[2]) for p in grid for k in RK}
        free = {t for t in trans if g(t) <= theta}
        # Minkowski sum of the free translations with the cutter, clipped to the grid
        for t in free:
            for k in RK:
                x = (t[0] + k[0], t[1] + k[1], t[2] + k[2])
                if 0 <= x[0] < nx and 0 <= x[1] < ny and 0 <= x[2] < nz:
                    acc.add(x)
        for p in grid:
            m = min(g((p[0] - k[0], p[1] - k[1], p[2] - k[2])) for k in RK)
            if m < f[p]:
                f[p] = m
    F = np.zeros(rho.shape)
    A = np.zeros(rho.shape, np.uint8)
    for (x, y, z), v in f.items():
        F[z, y, x] = v
    for (x, y, z) in acc:
        if fixture is None or fixture[z, y, x] == 0:
            A[z, y, x] = 1
    return F, A
