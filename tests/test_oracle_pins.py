"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics, not by itself.

Closed forms (box over box, single-voxel tool), hand-worked fixtures under tests/golden/,
exact quarter-turn rotations, an independent NumPy FFT correlation, the independent set-based
brute force of oracle/brute.py, and the invariants the paper states (Omega in B, conservative
sharp-point sampling, flat slab, closed cavity, sweep = threshold of the minimum).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.ref import offsets_of, translation_box
from paper_2002_07627_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def axis_quat(axis, deg):
    a = math.radians(deg)
    v = {"x": (1, 0, 0), "y": (0, 1, 0), "z": (0, 0, 1)}[axis]
    return np.array([math.cos(a / 2), *(math.sin(a / 2) * np.array(v, float))])


# ---------------------------------------------------------------- rotation (Alg. 1 Rotate)

def test_quat_matrix_closed_forms():
    assert np.array_equal(oracle.quat_to_matrix([1, 0, 0, 0]), np.eye(3))
    Rz = oracle.quat_to_matrix(axis_quat("z", 90))
    assert np.allclose(Rz, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    Rx = oracle.quat_to_matrix(axis_quat("x", 90))
    assert np.allclose(Rx, [[1, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-15)
    Ry = oracle.quat_to_matrix(axis_quat("y", 90))
    assert np.allclose(Ry, [[0, 0, 1], [0, 1, 0], [-1, 0, 0]], atol=1e-15)
    # a non-unit quaternion gives the same rotation as its normalisation
    assert np.allclose(oracle.quat_to_matrix(3 * axis_quat("y", 33)),
                       oracle.quat_to_matrix(axis_quat("y", 33)), atol=1e-15)


def test_quat_matrix_is_a_homomorphism():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b = rng.normal(size=4), rng.normal(size=4)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        Ra, Rb = oracle.quat_to_matrix(a), oracle.quat_to_matrix(b)
        assert np.allclose(Ra @ Ra.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(Ra) - 1) < 1e-14
        assert np.allclose(oracle.quat_to_matrix(qmul(a, b)), Ra @ Rb, atol=1e-14)


def _tool_set(arr, origin, q):
    R = oracle.quat_to_matrix(q)
    lo, box = oracle.rotate_indicator(arr, origin, R)
    return sorted(map(tuple, offsets_of(lo, box).tolist()))


def test_rotate_identity_returns_input():
    rng = np.random.default_rng(1)
    arr = (rng.random((5, 4, 6)) < 0.4).astype(np.uint8)
    origin = (2, 1, 3)
    got = _tool_set(arr, origin, [1, 0, 0, 0])
    assert got == sorted(brute.tool_offsets(arr, origin))


@pytest.mark.parametrize("axis", ["x", "y", "z"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_rotate_quarter_turns_are_permutations(axis, k):
    rng = np.random.default_rng(2 + k)
    arr = (rng.random((5, 7, 6)) < 0.5).astype(np.uint8)
    origin = (2, 3, 1)
    got = _tool_set(arr, origin, axis_quat(axis, 90 * k))
    want = brute.rotate_set(brute.tool_offsets(arr, origin), [(axis, k)])
    assert got == want


def test_rotate_quarter_turn_round_trip():
    tool = synth.cylinder_tool(2, 5, 4, 3)
    T = (tool.holder | tool.cutter)
    for axis in "xyz":
        R1 = oracle.quat_to_matrix(axis_quat(axis, 90))
        lo, box = oracle.rotate_indicator(T, tool.origin, R1)
        # rotate back: the box array with origin at -lo
        back = _tool_set(box, tuple(-lo), axis_quat(axis, -90))
        assert back == sorted(brute.tool_offsets(T, tool.origin))


def test_rotate_45_degree_bar_golden():
    g = _gold("rotate_bar_45deg.json")
    tx, ty, tz = g["tool_xyz"]
    arr = np.ones((tz, ty, tx), np.uint8)
    got = _tool_set(arr, g["origin"], g["quat_wxyz"])
    assert got == sorted(map(tuple, g["expected_offsets"]))


def test_rotate_preserves_volume_roughly():
    tool = synth.cylinder_tool(3, 20, 8, 16, synth.fibonacci_quats(12))
    T = (tool.holder | tool.cutter)
    n = int(T.sum())
    for q in tool.quats:
        m = len(_tool_set(T, tool.origin, q))
        assert abs(m - n) <= 0.06 * n


# ---------------------------------------------------------------- collision (Eq. eq_ident)

def test_collision_box_over_box_closed_form():
    """g(t) = product over axes of the overlap length of [lo_O, hi_O) and [lo_T + t, hi_T + t)."""
    nz, ny, nx = 9, 10, 11
    rho = np.zeros((nz, ny, nx))
    Olo, Ohi = np.array([2, 3, 1]), np.array([7, 8, 6])     # x, y, z (half-open)
    rho[Olo[2]:Ohi[2], Olo[1]:Ohi[1], Olo[0]:Ohi[0]] = 1.0
    ext = np.array([3, 4, 2])
    org = np.array([1, 0, 1])
    RT = np.array([(i - org[0], j - org[1], k - org[2]) for k in range(ext[2]) for j in range(ext[1])
                   for i in range(ext[0])], np.int32)
    tlo = np.array([-6, -6, -5])
    text = np.array([20, 20, 16])
    g = oracle.collision(rho, RT, tlo, text)
    Tlo = -org
    Thi = ext - org
    for k in range(text[2]):
        for j in range(text[1]):
            for i in range(text[0]):
                t = tlo + np.array([i, j, k])
                ov = np.maximum(0, np.minimum(Ohi, Thi + t) - np.maximum(Olo, Tlo + t))
                assert g[k, j, i] == float(np.prod(ov))


def test_collision_single_voxel_tool_is_the_density():
    rng = np.random.default_rng(3)
    rho = rng.random((4, 5, 6))
    g = oracle.collision(rho, np.zeros((1, 3), np.int32), [-1, -1, -1], [8, 7, 6])
    ref = np.zeros((6, 7, 8))
    ref[1:5, 1:6, 1:7] = rho
    assert np.array_equal(g, ref)


def test_collision_matches_numpy_fft_correlation():
    rng = np.random.default_rng(4)
    nz, ny, nx = 7, 9, 8
    rho = rng.random((nz, ny, nx))
    tool = synth.cylinder_tool(2, 3, 3, 2)
    rs = oracle.resample_tool(tool, synth.fibonacci_quats(5)[3])
    RT = rs["RT"]
    vmin, vmax = RT.min(0), RT.max(0)
    tlo = -vmax
    text = np.array([nx, ny, nz]) - 1 - vmin - tlo + 1
    g = oracle.collision(rho, RT, tlo, text)
    # linear correlation by zero-padded FFT: G(t) = sum_x rho(x) tau(x - t)
    P = np.array([nx, ny, nz]) + (vmax - vmin) + 1
    a = np.zeros(P[::-1])
    a[:nz, :ny, :nx] = rho
    tau = np.zeros(P[::-1])
    for v in RT:
        idx = (v - vmin)
        tau[idx[2], idx[1], idx[0]] = 1.0
    c = np.fft.ifftn(np.fft.fftn(a) * np.conj(np.fft.fftn(tau))).real
    # c[s] = sum_x a(x) tau(x - s) = sum_v rho(s + v - vmin) -> g(t) at s = t + vmin (mod P)
    for k in range(text[2]):
        for j in range(text[1]):
            for i in range(text[0]):
                t = tlo + np.array([i, j, k])
                s = (t + vmin) % P
                assert abs(c[s[2], s[1], s[0]] - g[k, j, i]) < 1e-9


# ---------------------------------------------------------------- hand-worked IMF values

def _golden_design(case, gd):
    nx, ny, nz = gd["grid_xyz"]
    rho = np.zeros((nz, ny, nx), np.float32)
    sx, sy, sz = gd["solid"]
    rho[sz, sy, sx] = case["rho"]
    tx, ty, tz = gd["tool_xyz"]
    cut = np.zeros((tz, ty, tx), np.uint8)
    hol = np.zeros((tz, ty, tx), np.uint8)
    for x, y, z in gd["cutter_cells"]:
        cut[z, y, x] = 1
    for x, y, z in gd["holder_cells"]:
        hol[z, y, x] = 1
    tool = synth.Tool(hol, cut, tuple(gd["origin"]), np.array([[1.0, 0, 0, 0]]))
    return synth.Design(rho, None, [tool])


def test_single_obstacle_golden_values():
    gd = _gold("single_obstacle_2d.json")
    for case in gd["cases"]:
        d = _golden_design(case, gd)
        out = oracle.imf(d, theta_rel=gd["theta_rel"])
        for p, fv, av in zip(case["points"], case["f"], case["accessible"]):
            x, y, z = p
            assert abs(out["f"][z, y, x] - fv) < 1e-12, (p, out["f"][z, y, x], fv)
            assert out["accessible"][z, y, x] == av, p
        fq, aq = oracle.point_query(d.rho, None, d.tools, case["points"], theta_rel=gd["theta_rel"])
        assert np.allclose(fq, case["f"], atol=1e-12)
        assert list(aq) == case["accessible"]


# ---------------------------------------------------------------- brute force (eq_A)

def _quarter_design(seed, binary=True):
    rng = np.random.default_rng(seed)
    nz, ny, nx = 6, 7, 8
    if binary:
        rho = (rng.random((nz, ny, nx)) < 0.25).astype(np.float32)
    else:
        rho = rng.random((nz, ny, nx)).astype(np.float32)
    fix = np.zeros((nz, ny, nx), np.uint8)
    fix[0] = 1
    cut = np.zeros((3, 3, 3), np.uint8)
    hol = np.zeros((3, 3, 3), np.uint8)
    cut[0, 1, 1] = cut[1, 1, 1] = 1          # 2-voxel cutter along +z
    hol[2, :, 1] = 1                         # 3-voxel holder bar across y on top
    hol[2, 1, 0] = 1
    turns = [[], [("x", 1)], [("y", 1)], [("x", 2)], [("z", 1), ("x", 1)]]
    quats = []
    for t in turns:
        q = np.array([1.0, 0, 0, 0])
        for axis, k in t:
            q = qmul(axis_quat(axis, 90 * k), q)
        quats.append(q)
    tool = synth.Tool(hol, cut, (1, 1, 0), np.array(quats))
    return synth.Design(rho, fix, [tool]), turns


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("binary", [True, False])
def test_oracle_matches_set_brute_force(seed, binary):
    d, turns = _quarter_design(seed, binary)
    tool = d.tools[0]
    T = tool.holder | tool.cutter
    theta = 0.01 * T.sum()
    orients = []
    for t in turns:
        RT = brute.rotate_set(brute.tool_offsets(T, tool.origin), t)
        RK = brute.rotate_set(brute.tool_offsets(tool.cutter, tool.origin), t)
        orients.append((RT, RK))
    fb, Ab = brute.brute_imf(d.rho, d.fixture, orients, theta)
    out = oracle.imf(d)
    assert np.allclose(out["f"], fb, atol=1e-12)
    assert np.array_equal(out["accessible"], Ab)


# ---------------------------------------------------------------- invariants of Sec. 2.1

def test_flat_slab_is_accessible_from_its_open_side():
    nz, ny, nx = 14, 12, 12
    rho = np.zeros((nz, ny, nx), np.float32)
    rho[:4] = 1.0
    tool = synth.cylinder_tool(1, 3, 2, 3)          # axis +z: comes from above
    d = synth.Design(rho, None, [tool])
    out = oracle.imf(d)
    assert np.all(out["f"][4:] == 0)
    assert np.all(out["accessible"][4:] == 1)
    assert np.all(out["f"][:4] >= 1.0)
    assert np.all(out["accessible"][:4] == 0)


def test_closed_cavity_is_inaccessible_from_every_orientation():
    n = 16
    rho = np.zeros((n, n, n), np.float32)
    rho[3:13, 3:13, 3:13] = 1.0
    rho[7:10, 7:10, 7:10] = 0.0                     # 3^3 cavity, smaller than the tool
    tool = synth.cylinder_tool(1, 3, 2, 4, synth.fibonacci_quats(10))
    d = synth.Design(rho, None, [tool])
    out = oracle.imf(d, theta_rel=0.01)
    cav = np.zeros_like(rho, bool)
    cav[7:10, 7:10, 7:10] = True
    assert np.all(out["f"][cav] > 0)
    assert np.all(out["accessible"][cav] == 0)
    assert np.all(out["secluded"][cav] == 1)


def test_sweep_equals_threshold_of_min_over_sharp_points():
    """With the sharp points = support of RK, A_R(x) = [gamma_R(x) <= theta] for every x."""
    d = synth.config_planar64(seed=3)
    d.rho = d.rho[:, :40, :36].copy()
    d.fixture = d.fixture[:, :40, :36].copy()
    out = oracle.imf(d, keep=True)
    for rec in out["per_orientation"]:
        assert np.array_equal(rec["A"].astype(bool), rec["gamma"] <= rec["theta"])


def test_omega_subset_of_B_for_binary_designs():
    rng = np.random.default_rng(7)
    rho = (rng.random((1, 30, 30)) < 0.3).astype(np.float32)
    tool = synth.planar_tool(3, 6, 7, 5, n_orient=6)
    d = synth.Design(rho, None, [tool])
    out = oracle.imf(d)
    solid = rho > 0.5
    assert np.all(out["f"][solid] >= 1.0)
    assert np.all(out["accessible"][solid] == 0)


def test_more_sharp_points_and_orientations_only_lower_the_imf():
    d = synth.config_planar64(seed=1)
    d.rho = d.rho[:, :36, :40].copy()
    d.fixture = d.fixture[:, :36, :40].copy()
    tool = d.tools[0]
    full = oracle.imf(d)
    # fewer orientations
    d2 = synth.Design(d.rho, d.fixture, [synth.Tool(tool.holder, tool.cutter, tool.origin, tool.quats[::2])])
    few = oracle.imf(d2)
    assert np.all(few["f"] >= full["f"])
    assert np.all(few["accessible"] <= full["accessible"])
    # fewer sharp points: only the tip row of the cutter
    sharp = np.zeros_like(tool.cutter)
    sharp[0, 0] = tool.cutter[0, 0]
    d3 = synth.Design(d.rho, d.fixture, [synth.Tool(tool.holder, tool.cutter, tool.origin, tool.quats, sharp)])
    tipf = oracle.imf(d3)
    assert np.all(tipf["f"] >= full["f"])


def test_shift_equivariance():
    rng = np.random.default_rng(9)
    rho = np.zeros((1, 40, 40), np.float32)
    rho[0, 10:22, 8:20] = rng.random((12, 12)).astype(np.float32)
    tool = synth.planar_tool(1, 3, 3, 3, n_orient=4)
    a = oracle.imf(synth.Design(rho, None, [tool]))["f"]
    rho2 = np.roll(rho, (5, 7), axis=(1, 2))
    b = oracle.imf(synth.Design(rho2, None, [tool]))["f"]
    # away from the grid boundary (where air is added or removed) the field just moves
    assert np.allclose(np.roll(a, (5, 7), axis=(1, 2))[0, 12:30, 12:30], b[0, 12:30, 12:30], atol=1e-12)


def test_sweep_count_is_a_convolution():
    rng = np.random.default_rng(11)
    free = (rng.random((6, 7, 8)) < 0.3).astype(np.uint8)
    tlo = np.array([-3, -2, -1])
    RK = np.array([(0, 0, 0), (1, 0, 0), (0, 2, 1), (-1, 1, 0)], np.int32)
    A, cnt = oracle.sweep(free, tlo, RK, (4, 5, 6), count=True)
    # scipy-free direct check: cnt(x) = sum_k free(x - k)
    ref = np.zeros((4, 5, 6), np.int32)
    for z in range(4):
        for y in range(5):
            for x in range(6):
                for k in RK:
                    t = np.array([x, y, z]) - k - tlo
                    if np.all(t >= 0) and np.all(t < [8, 7, 6]):
                        ref[z, y, x] += free[t[2], t[1], t[0]]
    assert np.array_equal(cnt, ref)
    assert np.array_equal(A, (ref > 0).astype(np.uint8))


# ---------------------------------------------------------------- Alg. 1 tail and Eq. eq_accFilter

def test_finalize_golden():
    g = _gold("finalize_penalize_1d.json")["finalize"]
    f = np.array(g["f"])[None, None]
    rho = np.array(g["rho"])[None, None]
    fix = np.array(g["fixture"], np.uint8)[None, None]
    for c in g["cases"]:
        fbar, sec, M = oracle.finalize(f, rho, fix, c["lambda"], g["tau"])
        assert M == g["M"]
        assert np.allclose(fbar.ravel(), c["fbar"], atol=0)
        assert list(sec.ravel()) == c["secluded"]


def test_finalize_zero_maximum():
    fbar, sec, M = oracle.finalize(np.zeros((1, 2, 3)), np.zeros((1, 2, 3)), None, 0.01, 0.5)
    assert M == 0 and not fbar.any() and not sec.any()


def test_penalize_golden():
    g = _gold("finalize_penalize_1d.json")["penalize"]
    arr = lambda k: np.array(g[k])[None, None]
    s = oracle.penalize(arr("sens"), arr("rho"), arr("fbar"), arr("secluded"), None, g["w_acc"], g["tau"])
    assert np.allclose(s.ravel(), g["expected"], atol=1e-15)


def test_point_query_matches_full_grid():
    d = synth.config_planar64(seed=2)
    out = oracle.imf(d)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, 64, 40), rng.integers(0, 64, 40), np.zeros(40, int)], -1)
    f, A = oracle.point_query(d.rho, d.fixture, d.tools, pts)
    for (x, y, z), fv, av in zip(pts, f, A):
        assert abs(out["f"][z, y, x] - fv) < 1e-9
        if d.fixture[z, y, x] == 0:
            assert out["accessible"][z, y, x] == av


def test_translation_box_covers_every_query():
    RK = np.array([(2, -1, 0), (-3, 4, 1)], np.int32)
    tlo, text = translation_box((5, 6, 7), RK)
    assert list(tlo) == [-2, -4, -1]
    assert list(text) == [7 + 3 + 2 - 1 + 1, 6 + 4 + 1, 5 + 1 + 0]


def test_subblock_equals_slice_of_full_grid():
    d = synth.config_planar64(seed=4)
    full = oracle.imf(d)
    f, A = oracle.imf_subblock(d, (7, 13, 0), (33, 29, 1))
    assert np.array_equal(f, full["f"][:, 13:42, 7:40])
    acc = (full["f"][:, 13:42, 7:40] <= 0.01 * 126)
    assert np.array_equal(A.astype(bool), acc)


# ---------------------------------------------------------------------------------------------
# Sharp-point sampling (Sec. 2.1.5 sampling remark; App. B, O(1) representative points)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ext", [(3, 4, 5), (2, 6, 7), (1, 5, 5), (6, 6, 6)])
def test_sharp_boundary_of_a_box_cutter_closed_form(ext):
    """A solid a x b x c box: the boundary has abc - (a-2)(b-2)(c-2) voxels (every voxel when
    an extent is at most 2), and the interior voxels are exactly the box shrunk by one."""
    a, b, c = ext
    K = np.ones((c, b, a), np.uint8)
    B = oracle.sharp_sample(K, (0, 0, 0), "boundary")
    inner = max(a - 2, 0) * max(b - 2, 0) * max(c - 2, 0)
    assert B.sum() == a * b * c - inner
    if inner:
        assert not B[1:-1, 1:-1, 1:-1].any()
    assert np.array_equal(oracle.sharp_sample(K, (0, 0, 0), "all"), K)


def test_sharp_nearest_points_are_nested_and_start_at_the_origin():
    """On the cylinder cutter (origin at the centre of the tip face, a boundary voxel): k = 1
    gives the origin voxel itself; the k-sets are nested in k and lie in the boundary; k above
    the boundary size gives the whole boundary; a hand-checked k = 5 set is the origin and its
    four face neighbours in the tip face (all at squared distance 1)."""
    from paper_2002_07627_gb300 import synth
    t = synth.cylinder_tool(3, 20, 8, 16, synth.fibonacci_quats(1))
    ox, oy, oz = t.origin
    B = oracle.sharp_sample(t.cutter, t.origin, "boundary")
    assert B[oz, oy, ox] == 1 and t.cutter[oz, oy, ox]
    one = oracle.sharp_sample(t.cutter, t.origin, "nearest", 1)
    assert one.sum() == 1 and one[oz, oy, ox] == 1
    prev = one
    for k in (2, 5, 9, 40, 200):
        cur = oracle.sharp_sample(t.cutter, t.origin, "nearest", k)
        assert cur.sum() == min(k, B.sum())
        assert np.all(cur >= prev) and np.all(B >= cur)
        prev = cur
    five = oracle.sharp_sample(t.cutter, t.origin, "nearest", 5)
    want = np.zeros_like(five)
    for dx, dy, dz in ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)):
        want[oz + dz, oy + dy, ox + dx] = 1
    assert oz == 0 or not t.cutter[oz - 1, oy, ox]          # the origin lies on the tip face
    assert np.array_equal(five, want)
    assert np.array_equal(oracle.sharp_sample(t.cutter, t.origin, "nearest", 10 ** 6), B)


def test_sharp_boundary_of_a_cylinder_excludes_its_core():
    """The interior of the r=3 cylinder cutter (voxels whose six neighbours are all cutter) is
    not sampled; a one-voxel-thick cutter is all boundary."""
    from paper_2002_07627_gb300 import synth
    t = synth.cylinder_tool(3, 20, 8, 16, synth.fibonacci_quats(1))
    K = t.cutter != 0
    B = oracle.sharp_sample(t.cutter, t.origin, "boundary") != 0
    z, y, x = np.nonzero(K & ~B)
    assert len(z) > 0
    for zz, yy, xx in zip(z, y, x):
        assert all(K[zz + dz, yy + dy, xx + dx] for dz, dy, dx in
                   ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)))
    thin = np.zeros((5, 1, 1), np.uint8)
    thin[:, 0, 0] = 1
    assert oracle.sharp_sample(thin, (0, 0, 0), "boundary").sum() == 5


# ---------------------------------------------------------------------------------------------
# Greedy process plan (Sec. 3.4.1)
# ---------------------------------------------------------------------------------------------

def test_process_plan_golden():
    """Hand-worked greedy set cover (tests/golden/process_plan_greedy.json)."""
    g = json.load(open(os.path.join(GOLD, "process_plan_greedy.json")))
    n = g["universe"]
    neg = np.zeros(n, bool)
    neg[g["negative"]] = True
    sets = []
    for s in g["sets"]:
        m = np.zeros(n, bool)
        m[s] = True
        sets.append(m)
    steps, total, left = oracle.process_plan(sets, neg)
    assert [list(s) for s in steps] == g["steps"]
    assert total == len(g["negative"]) and left == g["left"]


def test_process_plan_invariants_on_random_sets():
    """Removed volumes never grow from step to step (greedy on a shrinking remainder); the
    chosen sets cover exactly |N| - left voxels of N; every uncovered voxel of N lies in no set;
    no set is chosen twice; a full set finishes in one step."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(20, 200))
        neg = rng.random(n) < 0.6
        sets = [rng.random(n) < rng.uniform(0.05, 0.5) for _ in range(int(rng.integers(1, 12)))]
        steps, total, left = oracle.process_plan(sets, neg)
        rem = [c for _, c in steps]
        assert rem == sorted(rem, reverse=True)
        assert sum(rem) + left == total == neg.sum()
        chosen = [i for i, _ in steps]
        assert len(set(chosen)) == len(chosen)
        covered = np.zeros(n, bool)
        for i in chosen:
            covered |= sets[i]
        unreached = neg & ~covered
        assert unreached.sum() == left
        assert not any((s & unreached).any() for s in sets)
    full = np.ones(10, bool)
    assert oracle.process_plan([full & False, full], full)[0] == [(1, 10)]
