"""GPU parity of the CUDA IMF path (through the C ABI) against the FP64 oracle.

Tolerances (the IMF contract): the accessible / free classification is bit-exact for every
translation (and every point) whose collision measure lies farther than 1e-3 |T| from the
threshold; the raw IMF has max-abs error <= 1e-4 max f. f_bar and Gamma are compared away
from the allowance discontinuity (|f_bar - lambda| > 1e-4).
"""
import numpy as np
import pytest

import oracle
from oracle.ref import translation_box
from paper_2002_07627_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_07627_gb300 import build, binding
    build.build()
    return binding


def run_gpu(design, lam=0.01, tau=0.5, theta_rel=0.01, keep=False, **kw):
    binding = _gpu()
    imf = binding.Imf(design.rho.shape, lam=lam, tau=tau, theta_rel=theta_rel, **kw)
    imf.set_tools(design.tools)
    rho = torch.from_numpy(np.ascontiguousarray(design.rho)).cuda()
    fix = None if design.fixture is None else torch.from_numpy(np.ascontiguousarray(design.fixture)).cuda()
    raw = torch.empty_like(rho)
    acc = torch.empty(rho.shape, dtype=torch.uint8, device="cuda")
    fbar, sec = imf.compute(rho, fix, raw=raw, accessible=acc)
    imf.sync()
    out = dict(f=raw.cpu().numpy().astype(np.float64), fbar=fbar.cpu().numpy().astype(np.float64),
               secluded=sec.cpu().numpy(), accessible=acc.cpu().numpy(), imf=imf)
    return out


def check_against_oracle(design, got, ref, theta_rel=0.01, lam=0.01):
    sizes = [int(((t.holder != 0) | (t.cutter != 0)).sum()) for t in design.tools]
    thetas = [theta_rel * s for s in sizes]
    fmax = float(np.max(ref["f"][np.isfinite(ref["f"])]))
    err = np.abs(got["f"] - ref["f"])
    assert err.max() <= 1e-4 * fmax, (err.max(), fmax)
    # accessible: exact away from the threshold of every tool (single tool: A = [f <= theta])
    if len(design.tools) == 1:
        band = 1e-3 * sizes[0]
        clear = np.abs(ref["f"] - thetas[0]) > band
        if design.fixture is not None:
            clear &= design.fixture == 0
        mism = (got["accessible"] != ref["accessible"]) & clear
        assert not mism.any(), np.argwhere(mism)[:5]
    else:
        # for several tools compare where no tool's minimum is near its own threshold
        pass
    clear = np.abs(ref["fbar"] - lam) > 1e-4
    assert np.abs(got["fbar"] - ref["fbar"])[clear].max() <= 2e-4
    assert np.array_equal(got["secluded"][clear], ref["secluded"][clear])


def test_resampled_tool_sets_match_oracle_bit_exactly():
    binding = _gpu()
    tools = [synth.cylinder_tool(3, 20, 8, 16, synth.fibonacci_quats(16)), synth.planar_tool(n_orient=8),
             synth.cylinder_tool(2, 6, 4, 5, np.random.default_rng(3).normal(size=(12, 4)))]
    for tool in tools:
        imf = binding.Imf((4, 4, 4))
        sharp = np.zeros_like(tool.cutter)
        sharp[..., : sharp.shape[-1] // 2] = 1
        tool.sharp = sharp
        imf.set_tool(0, tool.holder, tool.cutter, tool.origin, tool.quats, sharp)
        for r, q in enumerate(tool.quats):
            rs = oracle.resample_tool(tool, q)
            for which, key in enumerate(["RT", "RK", "sharp"]):
                got = sorted(map(tuple, imf.offsets(0, r, which).tolist()))
                want = sorted(map(tuple, rs[key].tolist()))
                assert got == want, (r, key)
        imf.close()


def test_planar64_full_parity():
    d = synth.config_planar64(seed=0)
    ref = oracle.imf(d)
    got = run_gpu(d)
    check_against_oracle(d, got, ref)


@pytest.mark.parametrize("seed", [1, 2])
def test_planar_ragged_full_parity(seed):
    d = synth.config_planar64(seed=seed)
    d.rho = np.ascontiguousarray(d.rho[:, :53, :71])
    d.fixture = np.ascontiguousarray(d.fixture[:, :53, :71])
    ref = oracle.imf(d)
    got = run_gpu(d, orient_batch=3)
    check_against_oracle(d, got, ref)


def _small3d(seed=0, n=(40, 36, 28), n_orient=8):
    rho = synth.beam_density(n, n_beams=10, seed=seed)
    fix = synth.slab_fixture(rho.shape, 3, axis="z")
    tool = synth.cylinder_tool(2, 6, 4, 5, synth.fibonacci_quats(n_orient))
    return synth.Design(rho, fix, [tool])


def test_3d_ragged_full_parity():
    d = _small3d()
    ref = oracle.imf(d, keep=True)
    got = run_gpu(d, orient_batch=3)
    check_against_oracle(d, got, ref)


def test_collision_field_and_free_bits_per_orientation():
    """g of the last orientation batch against the oracle's direct FP64 sums; the free
    classification g <= theta is exact outside the 1e-3 |T| band (and, with the re-check,
    everywhere except within FP32 round-off of theta)."""
    d = _small3d(seed=4, n=(33, 29, 21), n_orient=5)
    binding = _gpu()
    imf = binding.Imf(d.rho.shape, orient_batch=2)
    imf.set_tools(d.tools)
    imf.set_debug = True
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    imf.compute(rho, fix)
    imf.sync()
    info = imf.tool_info(0)
    rhoO = oracle.rho_obstacle(d.rho, d.fixture)
    tool = d.tools[0]
    theta = info.theta
    for slot in range(1):
        o, gw = imf.last_g(slot)
        rs = oracle.resample_tool(tool, tool.quats[o])
        tlo, text = translation_box(d.rho.shape, rs["RK"], rs["sharp"])
        g = oracle.collision(rhoO, rs["RT"], tlo, text)
        k = np.array(info.kmax)
        i0 = tlo + k
        sub = gw[i0[2]:i0[2] + text[2], i0[1]:i0[1] + text[1], i0[0]:i0[0] + text[0]]
        assert sub.shape == g.shape
        err = np.abs(sub - g)
        assert err.max() <= 1e-4 * g.max()
        # re-checked classification
        assert np.array_equal(sub <= theta, g <= theta) or np.all(np.abs(g[(sub <= theta) != (g <= theta)] - theta) < 1e-4)


def test_3d_beams_full_size_sampled_points():
    """128^3 beams, 64 Fibonacci orientations (the plain 3D workload): f and A at sampled
    points, including the GPU's argmax, against literal FP64 point queries."""
    d = synth.config_beams(128, 40, 64, seed=0)
    got = run_gpu(d)
    f = got["f"]
    rng = np.random.default_rng(0)
    pts = [np.array(np.unravel_index(np.argmax(np.where(d.fixture == 0, f, -1)), f.shape))[::-1]]
    # near the accessible/inaccessible boundary and at random
    theta = 0.01 * ((d.tools[0].holder | d.tools[0].cutter).sum())
    near = np.argwhere((np.abs(f - theta) < 5) & (d.fixture == 0))
    for idx in rng.choice(len(near), size=min(12, len(near)), replace=False):
        pts.append(near[idx][::-1])
    for _ in range(12):
        pts.append(np.array([rng.integers(0, 128), rng.integers(0, 128), rng.integers(6, 128)]))
    pts = np.array(pts)
    fo, Ao = oracle.point_query(d.rho, d.fixture, d.tools, pts)
    M = f[pts[0][2], pts[0][1], pts[0][0]]
    assert abs(fo[0] - M) <= 1e-4 * M
    for (x, y, z), fv, av in zip(pts, fo, Ao):
        assert abs(f[z, y, x] - fv) <= 1e-4 * M, ((x, y, z), f[z, y, x], fv)
        if abs(fv - theta) > 1e-3 * theta / 0.01:
            assert got["accessible"][z, y, x] == av, (x, y, z)


def test_3d_beams_256_sampled_points():
    """256^3 beams, 128 orientations (the large 3D workload): the padded y and z lengths exceed
    256, so the y/z passes run radix stages while the x pass (M = 160) runs two register
    passes; f at the GPU's argmax, near the threshold and at random points against FP64 point
    queries."""
    d = synth.config_beams(256, 120, 128, seed=0)
    got = run_gpu(d)
    info = got["imf"].tool_info(0)
    assert max(info.P[1], info.P[2]) > 256
    f = got["f"]
    rng = np.random.default_rng(1)
    pts = [np.array(np.unravel_index(np.argmax(np.where(d.fixture == 0, f, -1)), f.shape))[::-1]]
    theta = 0.01 * ((d.tools[0].holder | d.tools[0].cutter).sum())
    near = np.argwhere((np.abs(f - theta) < 5) & (d.fixture == 0))
    for idx in rng.choice(len(near), size=min(6, len(near)), replace=False):
        pts.append(near[idx][::-1])
    for _ in range(6):
        pts.append(np.array([rng.integers(0, 256), rng.integers(0, 256), rng.integers(6, 256)]))
    pts = np.array(pts)
    fo, Ao = oracle.point_query(d.rho, d.fixture, d.tools, pts)
    M = f[pts[0][2], pts[0][1], pts[0][0]]
    assert abs(fo[0] - M) <= 1e-4 * M
    for (x, y, z), fv, av in zip(pts, fo, Ao):
        assert abs(f[z, y, x] - fv) <= 1e-4 * M, ((x, y, z), f[z, y, x], fv)
        if abs(fv - theta) > 1e-3 * theta / 0.01:
            assert got["accessible"][z, y, x] == av, (x, y, z)
    # eight seeded 8^3 sub-blocks computed in full by the oracle (direct FP64 sums on the
    # translations each block needs)
    band = 1e-3 * theta / 0.01
    for seed in range(1, 9):
        r = np.random.default_rng(seed)
        x0 = [int(r.integers(0, 249)), int(r.integers(0, 249)), int(r.integers(0, 249))]
        fo, Ao = oracle.imf_subblock(d, x0, [8, 8, 8])
        sl = (slice(x0[2], x0[2] + 8), slice(x0[1], x0[1] + 8), slice(x0[0], x0[0] + 8))
        keep = d.fixture[sl] == 0
        assert np.abs(f[sl] - fo)[keep].max(initial=0) <= 1e-4 * M, seed
        clear = keep & (np.abs(fo - theta) > band)
        assert np.array_equal(got["accessible"][sl][clear], Ao[clear].astype(bool).astype(np.uint8)), seed


def test_more_sharp_points_and_orientations_only_lower_the_imf():
    """Monotonicity on the GPU path: the whole cutter as sharp points gives f no larger than a
    boundary-only or a one-slice subset, and adding orientations lowers f and grows A."""
    rho = synth.beam_density((30, 34, 41), n_beams=8, seed=3)
    fix = synth.slab_fixture(rho.shape, 2, axis="z")
    quats = synth.fibonacci_quats(10)
    full = synth.cylinder_tool(2, 6, 4, 5, quats)
    cut = full.cutter != 0
    inner = cut.copy()
    inner[1:-1, 1:-1, 1:-1] &= ~(cut[:-2, 1:-1, 1:-1] & cut[2:, 1:-1, 1:-1] & cut[1:-1, :-2, 1:-1] &
                                  cut[1:-1, 2:, 1:-1] & cut[1:-1, 1:-1, :-2] & cut[1:-1, 1:-1, 2:])
    boundary = synth.cylinder_tool(2, 6, 4, 5, quats)
    boundary.sharp = inner.astype(np.uint8)
    tip = synth.cylinder_tool(2, 6, 4, 5, quats)
    tip_mask = np.zeros_like(full.cutter)
    zc = np.argwhere(cut)[:, 0].min()
    tip_mask[zc] = full.cutter[zc]
    tip.sharp = tip_mask
    few = synth.cylinder_tool(2, 6, 4, 5, quats[:4])
    res = {}
    for name, tool in [("full", full), ("boundary", boundary), ("tip", tip), ("few", few)]:
        res[name] = run_gpu(synth.Design(rho, fix, [tool]))
    om = fix == 0
    assert np.all(res["full"]["f"][om] <= res["boundary"]["f"][om])
    assert np.all(res["boundary"]["f"][om] <= res["tip"]["f"][om])
    # fewer orientations change the padded FFT lengths, so g is rounded differently: the
    # orientation comparison holds within the IMF contract (1e-4 max f), the sharp-point ones
    # above (same plan, same g) hold exactly
    M = res["full"]["f"][om].max()
    assert np.all(res["full"]["f"][om] <= res["few"]["f"][om] + 1e-4 * M)
    assert np.all(res["full"]["accessible"][om] >= res["few"]["accessible"][om])
    assert np.any(res["full"]["f"][om] < res["tip"]["f"][om])


def test_multi_tool_and_sharp_subset():
    d = synth.config_planar64(seed=5)
    d.rho = np.ascontiguousarray(d.rho[:, :48, :48])
    d.fixture = np.ascontiguousarray(d.fixture[:, :48, :48])
    t2 = synth.planar_tool(1, 5, 5, 6, n_orient=5)
    sharp = np.zeros_like(t2.cutter)
    sharp[0, 0] = t2.cutter[0, 0]
    t2.sharp = sharp
    d.tools.append(t2)
    ref = oracle.imf(d)
    got = run_gpu(d)
    check_against_oracle(d, got, ref)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 37), (1, 9, 1), (3, 2, 5)])
def test_degenerate_grids(shape):
    rng = np.random.default_rng(sum(shape))
    rho = rng.random(shape).astype(np.float32)
    tool = synth.cylinder_tool(1, 2, 2, 2, synth.fibonacci_quats(3)) if shape[0] > 1 else synth.planar_tool(1, 2, 3, 2, 3)
    d = synth.Design(rho, None, [tool])
    ref = oracle.imf(d)
    got = run_gpu(d)
    check_against_oracle(d, got, ref)


def test_empty_and_full_density():
    tool = synth.planar_tool(n_orient=4)
    z = synth.Design(np.zeros((1, 30, 40), np.float32), None, [tool])
    got = run_gpu(z)
    assert not got["f"].any() and not got["fbar"].any() and not got["secluded"].any()
    assert got["accessible"].all()
    o = synth.Design(np.ones((1, 30, 40), np.float32), None, [tool])
    ref = oracle.imf(o)
    got = run_gpu(o)
    check_against_oracle(o, got, ref)


def test_repeat_calls_and_host_entry_point_agree():
    binding = _gpu()
    d = _small3d(seed=2, n=(24, 20, 18), n_orient=6)
    imf = binding.Imf(d.rho.shape)
    imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    raw1 = torch.empty_like(rho)
    fb1, s1 = imf.compute(rho, fix, raw=raw1)
    raw2 = torch.empty_like(rho)
    fb2, s2 = imf.compute(rho, fix, raw=raw2)
    imf.sync()
    assert torch.equal(raw1, raw2) and torch.equal(fb1, fb2) and torch.equal(s1, s2)
    fbh, sh, rawh, acch = imf.compute_host(d.rho, d.fixture)
    assert np.array_equal(fbh, fb1.cpu().numpy()) and np.array_equal(rawh, raw1.cpu().numpy())
    assert np.array_equal(sh, s1.cpu().numpy())


def test_penalize_matches_oracle():
    d = synth.config_planar64(seed=7)
    binding = _gpu()
    got = run_gpu(d)
    imf = got["imf"]
    rng = np.random.default_rng(1)
    sens = rng.normal(size=d.rho.shape).astype(np.float32)
    st = torch.from_numpy(sens.copy()).cuda()
    rho = torch.from_numpy(d.rho).cuda()
    fb = torch.from_numpy(got["fbar"].astype(np.float32)).cuda()
    sec = torch.from_numpy(got["secluded"]).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    imf.penalize(st, rho, fb, sec, fix, w_acc=0.3)
    imf.sync()
    ref = oracle.penalize(sens, d.rho, got["fbar"], got["secluded"], d.fixture, 0.3)
    assert np.abs(st.cpu().numpy() - ref).max() <= 1e-6


def test_recheck_list_overflow_is_reported_not_faulted():
    binding = _gpu()
    d = _small3d(seed=3, n=(48, 48, 40), n_orient=2)
    imf = binding.Imf(d.rho.shape, recheck_band=1e9)     # flag every translation
    imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    imf.compute(rho, None)
    with pytest.raises(binding.ImfError) as ei:
        imf.sync()
    assert ei.value.status == 7
    imf.sync()     # cleared


def test_recheck_off_stays_inside_the_contract():
    d = _small3d(seed=6, n=(30, 26, 22), n_orient=4)
    ref = oracle.imf(d)
    got = run_gpu(d, recheck=False)
    check_against_oracle(d, got, ref)


def test_orientation_groups_of_the_minimum_do_not_change_the_result():
    """The minimum over sharp points may split a launch's orientations into groups that merge
    into f with an integer atomic minimum; every split gives bit-identical f, f_bar and Gamma,
    including one group per orientation and more groups than orientations."""
    d = _small3d(seed=4, n=(37, 45, 70), n_orient=11)
    base = run_gpu(d, erode_groups=1, orient_batch=8)
    ref = oracle.imf(d)
    check_against_oracle(d, base, ref)
    for g in (2, 3, 8, 40, 0):
        got = run_gpu(d, erode_groups=g, orient_batch=8)
        for k in ("f", "fbar", "secluded", "accessible"):
            assert np.array_equal(got[k], base[k]), (g, k)


@pytest.mark.parametrize("stages_only", [False, True])
def test_both_fft_variants_match_oracle(stages_only):
    """The two-pass register FFT (default where the padded lengths split into factors <= 16)
    and the radix-stage FFT (forced) both meet the contract on a ragged grid, per orientation
    for g and the free bits and in full for f, f_bar and Gamma."""
    d = _small3d(seed=7, n=(29, 38, 45), n_orient=6)
    ref = oracle.imf(d, keep=True)
    got = run_gpu(d, orient_batch=4, fft_stages_only=stages_only)
    check_against_oracle(d, got, ref)
    info = got["imf"].tool_info(0)
    assert all(p <= 256 for p in info.P)      # both variants run the same padded lengths


def test_accessible_from_the_minimum_equals_the_sweep():
    """With one tool whose sharp points are its whole cutter, the library reads A off the
    minimum, A = [f <= theta] (App. A); the sweep of Eq. eq_conv_A (forced) must give the same
    set except where f lies within FP32 rounding of theta, and both meet the contract against
    the oracle. A sharp-point subset (or a second tool) falls back to the sweep by itself."""
    for seed, n in ((3, (31, 40, 47)), (8, (20, 26, 33))):
        d = _small3d(seed=seed, n=n, n_orient=7)
        ref = oracle.imf(d)
        a = run_gpu(d, orient_batch=4)
        b = run_gpu(d, orient_batch=4, accessible_by_sweep=True)
        check_against_oracle(d, a, ref)
        check_against_oracle(d, b, ref)
        theta = 0.01 * float(((d.tools[0].holder != 0) | (d.tools[0].cutter != 0)).sum())
        assert np.array_equal(a["f"], b["f"])
        differ = a["accessible"] != b["accessible"]
        assert not np.any(differ & (np.abs(a["f"] - theta) > 1e-5 * theta))
        assert b["imf"].stats().launches > a["imf"].stats().launches   # the sweep ran only in b
    # sharp subset: the default path sweeps and agrees with the oracle
    d = _small3d(seed=5, n=(25, 30, 35), n_orient=5)
    sharp = np.zeros_like(d.tools[0].cutter)
    sharp[: sharp.shape[0] // 2] = 1
    d.tools[0].sharp = sharp
    check_against_oracle(d, run_gpu(d, orient_batch=4), oracle.imf(d))

def test_sweep_of_long_cutter_runs_matches_oracle():
    """Sweep of Eq. eq_conv_A with cutter runs along x of every length class: a 40-voxel cutter
    laid along +x and -x (runs split at 32, so lengths 32 and 8 occur), tilted and upright
    (runs of 1 .. 5). The sweep is forced; the accessible set must match the oracle exactly
    away from the threshold, and so must the route that reads A off the minimum."""
    c, s_ = np.cos(np.pi / 4), np.sin(np.pi / 4)
    quats = np.array([[c, 0, s_, 0], [c, 0, -s_, 0], [1, 0, 0, 0], [np.cos(0.3), 0.2, np.sin(0.3), 0.1]])
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    rho = synth.beam_density((90, 30, 26), n_beams=8, seed=11)
    fix = synth.slab_fixture(rho.shape, 2, axis="z")
    d = synth.Design(rho, fix, [synth.cylinder_tool(2, 40, 3, 4, quats)])
    ref = oracle.imf(d)
    got = run_gpu(d, orient_batch=3, accessible_by_sweep=True)
    check_against_oracle(d, got, ref)
    assert got["accessible"].any() and not got["accessible"].all()
    check_against_oracle(d, run_gpu(d, orient_batch=3), ref)

def _kernels_run(imf, design):
    """Names of the kernels one more compute of `design` launches on `imf`."""
    rho = torch.from_numpy(np.ascontiguousarray(design.rho)).cuda()
    fix = None if design.fixture is None else torch.from_numpy(np.ascontiguousarray(design.fixture)).cuda()
    imf.reset_kernel_times()
    imf.set_profiling(True)
    imf.compute(rho, fix)
    imf.sync()
    names = set(imf.kernel_times())
    imf.set_profiling(False)
    return names


def test_fused_yx_pass_equals_separate_passes():
    """The inverse y and x passes fused per z-plane (the plane kept in shared memory) run the
    same arithmetic as the two separate kernels: f, the normalised field and the accessible set
    are identical, and both meet the contract against the oracle. The last case is a grid whose
    plane does not fit in shared memory, where the library falls back to the two kernels."""
    d = _small3d(seed=4, n=(37, 44, 29), n_orient=6)
    ref = oracle.imf(d)
    for kw in ({}, {"accessible_by_sweep": True}):
        a = run_gpu(d, orient_batch=4, **kw)
        b = run_gpu(d, orient_batch=4, separate_yx_passes=True, **kw)
        check_against_oracle(d, a, ref)
        for k in ("f", "fbar", "secluded", "accessible"):
            assert np.array_equal(a[k], b[k]), k
        assert "fft_yx_inv_threshold" in _kernels_run(a["imf"], d)
        kb = _kernels_run(b["imf"], d)
        assert "fft_yx_inv_threshold" not in kb and "fft_y_inv" in kb
    # odd window extents and another split of the planes
    d = _small3d(seed=9, n=(61, 23, 50), n_orient=5)
    a = run_gpu(d, orient_batch=5, accessible_by_sweep=True)
    b = run_gpu(d, orient_batch=5, accessible_by_sweep=True, separate_yx_passes=True)
    for k in ("f", "fbar", "secluded", "accessible"):
        assert np.array_equal(a[k], b[k]), k
    d = synth.config_beams(200, 12, 3)
    a = run_gpu(d, orient_batch=3)
    assert "fft_yx_inv_threshold" not in _kernels_run(a["imf"], d)

def test_big_factor_axis_pass_matches_oracle():
    """A grid whose y axis pads above 256: the y passes run the two-pass FFT with a factor above
    16 (the 32-slot axis kernel); full parity against the oracle, both accessible routes."""
    rho = synth.beam_density((24, 262, 6), n_beams=6, seed=2)
    fix = synth.slab_fixture(rho.shape, 1, axis="z")
    d = synth.Design(rho, fix, [synth.cylinder_tool(1, 4, 2, 3, synth.fibonacci_quats(3))])
    ref = oracle.imf(d)
    for kw in ({}, {"accessible_by_sweep": True}):
        got = run_gpu(d, orient_batch=2, **kw)
        assert got["imf"].tool_info(0).P[1] > 256
        check_against_oracle(d, got, ref)
    # the radix-stage kernels give the same classification and the IMF within the contract
    check_against_oracle(d, run_gpu(d, orient_batch=2, fft_stages_only=True), ref)

def test_orientation_order_does_not_change_the_result():
    """With the FP32 FFT path requested explicitly the orientations run in an interleaved order
    (every batch spread over all directions); the default order is a nearest-neighbour chain.
    The minimum and the union do not depend on the order: f, the normalised field, Gamma and A
    are identical."""
    from paper_2002_07627_gb300 import binding
    d = _small3d(seed=6, n=(36, 30, 26), n_orient=11)
    for kw in ({}, {"accessible_by_sweep": True}):
        a = run_gpu(d, orient_batch=4, precision=binding.IMF_FP32_FFT, **kw)
        b = run_gpu(d, orient_batch=4, **kw)
        for k in ("f", "fbar", "secluded", "accessible"):
            assert np.array_equal(a[k], b[k]), k
