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


def accessible_bounds(design, ref, theta_rel=0.01):
    """Accessible sets that the contract fixes, from the oracle's per-orientation collision
    fields (Eq. eq_conv_A per orientation, union over orientations and tools, Eq. eq_A_multi):
    `sure` = the sweep of the translations that are free by more than the band
    (g < theta_i - 1e-3 |T_i|), which every correct result contains; `maybe` = the sweep of the
    translations within the band, where either classification is correct. A point in neither
    set must be inaccessible."""
    shape = design.rho.shape
    sure = np.zeros(shape, bool)
    maybe = np.zeros(shape, bool)
    per = ref["per_orientation"]
    i = 0
    for tool in design.tools:
        size = float(((tool.holder != 0) | (tool.cutter != 0)).sum())
        theta, band = theta_rel * size, 1e-3 * size
        for _ in tool.quats:
            p = per[i]
            i += 1
            if p is None:
                continue
            g = p["g"]
            sure |= oracle.sweep((g < theta - band).astype(np.uint8), p["tlo"], p["RK"], shape).astype(bool)
            maybe |= oracle.sweep((np.abs(g - theta) <= band).astype(np.uint8), p["tlo"], p["RK"], shape).astype(bool)
    assert i == len(per)
    return sure, maybe


def check_against_oracle(design, got, ref, theta_rel=0.01, lam=0.01):
    """The IMF contract against the oracle run `ref` (oracle.imf(design, keep=True)): raw f
    within 1e-4 max f everywhere; the accessible set exact wherever no translation that reaches
    the point lies within 1e-3 |T_i| of its tool's threshold (any number of tools, any sharp
    subset); f_bar and Gamma away from the allowance discontinuity."""
    fmax = float(np.max(ref["f"][np.isfinite(ref["f"])]))
    err = np.abs(got["f"] - ref["f"])
    assert err.max() <= 1e-4 * fmax, (err.max(), fmax)
    sure, maybe = accessible_bounds(design, ref, theta_rel)
    om0 = np.ones(design.rho.shape, bool) if design.fixture is None else design.fixture == 0
    A = got["accessible"] != 0
    assert not (A & ~om0).any(), "fixture cells must be inaccessible"
    missing = sure & om0 & ~A
    assert not missing.any(), ("accessible points missing", np.argwhere(missing)[:5])
    extra = A & ~sure & ~maybe
    assert not extra.any(), ("points accessible only within round-off of nothing", np.argwhere(extra)[:5])
    # the oracle's own accessible set obeys the same bounds (pins the bound computation)
    Ao = ref["accessible"] != 0
    assert not (sure & om0 & ~Ao).any() and not (Ao & ~sure & ~maybe).any()
    # f_bar and Gamma away from the allowance discontinuity, compared on the normalised IMF before
    # the allowance (f / M): after it, a point just below lambda reads 0 and would look clear
    M = float(ref["M"])
    pre = ref["f"] / M if M > 0 else np.zeros_like(ref["f"])
    clear = (np.abs(pre - lam) > 1e-4) | ~om0
    assert np.abs(got["fbar"] - ref["fbar"])[clear].max(initial=0) <= 2e-4
    assert np.array_equal(got["secluded"][clear], ref["secluded"][clear])


def oracle_ref(design, **kw):
    """The oracle's result with the per-orientation fields the accessible-set check needs."""
    return oracle.imf(design, keep=True, **kw)


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
    ref = oracle_ref(d)
    got = run_gpu(d)
    check_against_oracle(d, got, ref)


@pytest.mark.parametrize("seed", [1, 2])
def test_planar_ragged_full_parity(seed):
    d = synth.config_planar64(seed=seed)
    d.rho = np.ascontiguousarray(d.rho[:, :53, :71])
    d.fixture = np.ascontiguousarray(d.fixture[:, :53, :71])
    ref = oracle_ref(d)
    got = run_gpu(d, orient_batch=3)
    check_against_oracle(d, got, ref)


def _small3d(seed=0, n=(40, 36, 28), n_orient=8):
    rho = synth.beam_density(n, n_beams=10, seed=seed)
    fix = synth.slab_fixture(rho.shape, 3, axis="z")
    tool = synth.cylinder_tool(2, 6, 4, 5, synth.fibonacci_quats(n_orient))
    return synth.Design(rho, fix, [tool])


def test_3d_ragged_full_parity():
    d = _small3d()
    ref = oracle_ref(d)
    got = run_gpu(d, orient_batch=3)
    check_against_oracle(d, got, ref)


def test_collision_field_and_free_bits_per_orientation():
    """Every slot of the last orientation batch: the collision field g on the whole translation
    window against the oracle's direct FP64 sums (Eq. eq_ident), and the free bits the kernels
    wrote (threshold epilogue plus near-threshold re-check, Eq. eq_conv_D) against g <= theta of
    the oracle: exact outside the 1e-3 |T| band and, with the re-check, everywhere except within
    FP32 round-off of theta."""
    d = _small3d(seed=4, n=(33, 29, 21), n_orient=6)
    binding = _gpu()
    imf = binding.Imf(d.rho.shape, orient_batch=3)
    imf.set_tools(d.tools)
    imf.set_debug(True)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    imf.compute(rho, fix)
    imf.sync()
    info = imf.tool_info(0)
    rhoO = oracle.rho_obstacle(d.rho, d.fixture)
    tool = d.tools[0]
    theta = info.theta
    band = 1e-3 * info.size_T
    k = np.array(info.kmax)
    seen = set()
    for slot in range(3):
        o, gw = imf.last_g(slot)
        o2, bits = imf.last_bits(slot)
        assert o == o2
        seen.add(o)
        rs = oracle.resample_tool(tool, tool.quats[o])
        g = oracle.collision(rhoO, rs["RT"], -k, info.win)
        assert gw.shape == g.shape == bits.shape
        err = np.abs(gw - g)
        assert err.max() <= 1e-4 * g.max(), (o, err.max())
        free = g <= theta
        clear = np.abs(g - theta) > band
        assert np.array_equal(bits[clear] != 0, free[clear]), o
        diff = (bits != 0) != free
        assert np.all(np.abs(g[diff] - theta) < 1e-4 * theta), o
        # the kernels' bits agree with their own g (the re-check rewrites both), up to the FP32
        # rounding of theta in the epilogue's comparison
        own = (bits != 0) != (gw <= theta)
        assert np.all(np.abs(gw[own] - theta) <= 1e-6 * theta), o
    assert len(seen) == 3


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
    # eight seeded 16^3 sub-blocks computed in full by the oracle (direct FP64 sums on the
    # translations each block needs, the whole design as obstacle)
    band = 1e-3 * theta / 0.01
    for seed in range(1, 9):
        r = np.random.default_rng(seed)
        x0 = [int(r.integers(0, 113)), int(r.integers(0, 113)), int(r.integers(0, 113))]
        fo, Ao = oracle.imf_subblock(d, x0, [16, 16, 16])
        sl = (slice(x0[2], x0[2] + 16), slice(x0[1], x0[1] + 16), slice(x0[0], x0[0] + 16))
        keep = d.fixture[sl] == 0
        assert np.abs(f[sl] - fo)[keep].max(initial=0) <= 1e-4 * M, seed
        clear = keep & (np.abs(fo - theta) > band)
        assert np.array_equal(got["accessible"][sl][clear], Ao[clear].astype(bool).astype(np.uint8)), seed


def test_3d_beams_256_sampled_points():
    """256^3 beams, 128 orientations (the large 3D workload): the padded y and z lengths exceed
    256, so the y and z passes run the two-pass FFT with a factor above 16 (the 32-slot axis
    kernel) and the x pass (M = 160) the 16 x 10 split; f at the GPU's argmax, near the
    threshold and at random points against FP64 point queries, then eight seeded 8^3
    sub-blocks in full."""
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
    ref = oracle_ref(d)
    got = run_gpu(d)
    check_against_oracle(d, got, ref)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 37), (1, 9, 1), (3, 2, 5)])
def test_degenerate_grids(shape):
    rng = np.random.default_rng(sum(shape))
    rho = rng.random(shape).astype(np.float32)
    tool = synth.cylinder_tool(1, 2, 2, 2, synth.fibonacci_quats(3)) if shape[0] > 1 else synth.planar_tool(1, 2, 3, 2, 3)
    d = synth.Design(rho, None, [tool])
    ref = oracle_ref(d)
    got = run_gpu(d)
    check_against_oracle(d, got, ref)


def test_empty_and_full_density():
    tool = synth.planar_tool(n_orient=4)
    z = synth.Design(np.zeros((1, 30, 40), np.float32), None, [tool])
    got = run_gpu(z)
    assert not got["f"].any() and not got["fbar"].any() and not got["secluded"].any()
    assert got["accessible"].all()
    o = synth.Design(np.ones((1, 30, 40), np.float32), None, [tool])
    ref = oracle_ref(o)
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
    ref = oracle_ref(d)
    got = run_gpu(d, recheck=False)
    check_against_oracle(d, got, ref)


def test_orientation_groups_of_the_minimum_do_not_change_the_result():
    """The minimum over sharp points may split a launch's orientations into groups that merge
    into f with an integer atomic minimum; every split gives bit-identical f, f_bar and Gamma,
    including one group per orientation and more groups than orientations."""
    d = _small3d(seed=4, n=(37, 45, 70), n_orient=11)
    base = run_gpu(d, erode_groups=1, orient_batch=8)
    ref = oracle_ref(d)
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
    ref = oracle_ref(d)
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
        ref = oracle_ref(d)
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
    check_against_oracle(d, run_gpu(d, orient_batch=4), oracle_ref(d))

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
    ref = oracle_ref(d)
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
    ref = oracle_ref(d)
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
    ref = oracle_ref(d)
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


@pytest.mark.parametrize("mode,k", [("boundary", 1), ("nearest", 1), ("nearest", 6)])
def test_sharp_sampling_modes_match_oracle(mode, k):
    """The library's sharp-point sampling options (Sec. 2.1.5 sampling remark; App. B, O(1)
    representative points) against the oracle given the oracle's own sample of the cutter: the
    resampled sharp sets are identical for every orientation and the IMF meets the contract."""
    import dataclasses
    from paper_2002_07627_gb300 import binding
    d = _small3d(seed=12, n=(30, 28, 26), n_orient=6)
    tool = d.tools[0]
    mask = oracle.sharp_sample(tool.cutter, tool.origin, mode, k)
    sampled = dataclasses.replace(tool, sharp=mask)
    ref_design = synth.Design(d.rho, d.fixture, [sampled])
    ref = oracle_ref(ref_design)
    mode_id = {"boundary": binding.IMF_SHARP_BOUNDARY, "nearest": binding.IMF_SHARP_NEAREST}[mode]
    got = run_gpu(d, sharp_sampling=mode_id, sharp_k=k, orient_batch=4)
    for r, q in enumerate(tool.quats):
        want = sorted(map(tuple, oracle.resample_tool(sampled, q)["sharp"].tolist()))
        have = sorted(map(tuple, got["imf"].offsets(0, r, 2).tolist()))
        assert have == want, r
    check_against_oracle(ref_design, got, ref)


def test_sharp_sampling_is_conservative_and_monotone():
    """Fewer sharp points can only raise the IMF (Sec. 2.1.5): on one plan (same padded grid,
    same collision fields) f(all) <= f(boundary) <= f(16 nearest) <= f(4 nearest) <= f(1 nearest)
    pointwise and exactly, the secluded set can only shrink along the chain, and the accessible
    set (a sweep by the whole cutter) does not depend on the sampling."""
    from paper_2002_07627_gb300 import binding
    d = _small3d(seed=13, n=(34, 30, 28), n_orient=7)
    chain = [(binding.IMF_SHARP_ALL, 1), (binding.IMF_SHARP_BOUNDARY, 1), (binding.IMF_SHARP_NEAREST, 16),
             (binding.IMF_SHARP_NEAREST, 4), (binding.IMF_SHARP_NEAREST, 1)]
    res = [run_gpu(d, sharp_sampling=m, sharp_k=k, orient_batch=4, accessible_by_sweep=True) for m, k in chain]
    om = d.fixture == 0
    for a, b in zip(res, res[1:]):
        assert a["imf"].tool_info(0).P == b["imf"].tool_info(0).P
        assert np.all(a["f"][om] <= b["f"][om])
        assert np.array_equal(a["accessible"], b["accessible"])
    assert np.any(res[0]["f"][om] < res[-1]["f"][om])
    n_sharp = [r["imf"].tool_info(0).n_sharp for r in res]
    assert n_sharp == sorted(n_sharp, reverse=True) and n_sharp[-1] == 7


def _unpack_sets(sets, shape):
    nz, ny, nx = shape
    w = sets.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(w.view(np.uint8).reshape(w.shape[0], nz, ny, -1), axis=-1, bitorder="little")
    return bits[..., :nx].astype(bool)


def test_accessible_sets_and_greedy_process_plan_match_oracle():
    """Per-orientation accessible sets (Eq. eq_conv_A per orientation) and the greedy machining
    process plan of Sec. 3.4.1 on a binary design: g is an integer there, and theta sits half a
    voxel between integers, so every translation is classified exactly (farther than the
    1e-3 |T| band from theta) and both the sets and the plan must equal the oracle's bit for
    bit and step for step; two tools, so the set index runs over both tools' orientations."""
    binding = _gpu()
    rho = (synth.beam_density((34, 38, 30), n_beams=9, seed=21) > 0.5).astype(np.float32)
    fix = synth.slab_fixture(rho.shape, 2, axis="z")
    t1 = synth.cylinder_tool(2, 6, 4, 5, synth.fibonacci_quats(7))
    t2 = synth.cylinder_tool(1, 4, 3, 3, synth.fibonacci_quats(3))
    d = synth.Design(rho, fix, [t1, t2])
    size = int(((t1.holder != 0) | (t1.cutter != 0)).sum())
    size2 = int(((t2.holder != 0) | (t2.cutter != 0)).sum())
    theta_rel = (np.floor(0.01 * size) + 0.5) / size
    # the second tool's threshold must sit between integers too
    assert abs(theta_rel * size2 - np.round(theta_rel * size2)) > 1e-3 * size2 + 1e-9
    ref = oracle.imf(d, keep=True, theta_rel=theta_rel)
    imf = binding.Imf(rho.shape, theta_rel=theta_rel, orient_batch=3)
    imf.set_tools(d.tools)
    r = torch.from_numpy(rho).cuda()
    f = torch.from_numpy(fix).cuda()
    sets, fbar, sec = imf.accessible_sets(r, f)
    imf.sync()
    got = _unpack_sets(sets, rho.shape)
    per = ref["per_orientation"]
    assert got.shape[0] == len(per) == 10
    want = np.stack([p["A"].astype(bool) for p in per])
    assert np.array_equal(got, want)
    steps, neg, left = imf.process_plan(sets, r, f)
    negative = (fix == 0) & (rho <= 0.5)
    osteps, oneg, oleft = oracle.process_plan(list(want), negative)
    assert steps == osteps and neg == oneg and left == oleft
    assert len(steps) >= 2 and left < neg
    # the union of the sets is the accessible output of imf_compute (on Omega_0)
    acc = torch.empty(rho.shape, dtype=torch.uint8, device="cuda")
    imf.compute(r, f, accessible=acc)
    imf.sync()
    assert np.array_equal(acc.cpu().numpy() != 0, want.any(0) & (fix == 0))


def test_tma_fed_axis_passes_equal_the_one_shot_kernels():
    """The persistent y / z FFT passes fed by tensor copies (block-synchronous or warp-
    specialised, 8 or 16 pencils per item) and the copy-fed x pass run the same arithmetic as
    the one-shot kernels (fft_tma 0, fft_tma_x 0): f, f_bar, Gamma and A are bit-identical with
    every choice (the y and x passes forced into separate kernels), on grids whose
    padded lengths use the 16-slot shape, the 32-slot shape (a y length above 256) and lengths
    below the persistent kernel's minimum (which keep the one-shot kernel); and the result meets
    the contract against the oracle."""
    rho = synth.beam_density((24, 262, 6), n_beams=6, seed=2)
    big = synth.Design(rho, synth.slab_fixture(rho.shape, 1, axis="z"),
                       [synth.cylinder_tool(1, 4, 2, 3, synth.fibonacci_quats(3))])
    cases = [(_small3d(seed=4, n=(70, 66, 64), n_orient=5), {}), (big, {}),
             (_small3d(seed=5, n=(20, 18, 16), n_orient=4), {"accessible_by_sweep": True}),
             (_small3d(seed=6, n=(150, 24, 20), n_orient=4), {"accessible_by_sweep": True})]
    for d, kw in cases:
        b = run_gpu(d, orient_batch=3, fft_tma=0, fft_tma_x=0, **kw)
        for mode in (-1, 5, 10):      # the default, every pass block-synchronous, every pass warp-specialised
            for wide in (-1, 0):
                a = run_gpu(d, orient_batch=3, fft_tma=mode, fft_wide_pencils=wide, separate_yx_passes=True, **kw)
                for k in ("f", "fbar", "secluded", "accessible"):
                    assert np.array_equal(a[k], b[k]), (mode, wide, k)
    d = cases[0][0]
    check_against_oracle(d, run_gpu(d, orient_batch=3), oracle_ref(d))
    assert max(run_gpu(big, orient_batch=2)["imf"].tool_info(0).P) > 256
    # the long x axis pads to M >= 64, where the copy-fed x pass applies; oracle parity too
    d = cases[3][0]
    got = run_gpu(d, orient_batch=3, separate_yx_passes=True)
    assert got["imf"].tool_info(0).P[0] // 2 >= 64
    assert "irfft_x_threshold" in _kernels_run(got["imf"], d)
    check_against_oracle(d, got, oracle_ref(d))



@pytest.mark.parametrize("nx,split", [(120, (10, 7)), (132, (15, 5))])
def test_copy_fed_x_pass_with_odd_rows_per_item(nx, split):
    """The copy-fed x pass takes R = 256 / A rows per item; with A = 10 or 15 (R = 25, 17) the R
    rows of half spectrum are no whole number of 128-byte lines, and each of the two stages must
    still start on a 128-byte boundary (tensor copies require it). With enough items that every
    block reuses its stages, the pass equals the one-shot x pass bit for bit and meets the
    contract against the oracle."""
    d = _small3d(seed=7, n=(nx, 60, 40), n_orient=8)
    got = run_gpu(d, orient_batch=8, separate_yx_passes=True)
    M = got["imf"].tool_info(0).P[0] // 2
    assert M == split[0] * split[1]
    assert "irfft_x_threshold" in _kernels_run(got["imf"], d)
    one = run_gpu(d, orient_batch=8, separate_yx_passes=True, fft_tma_x=0)
    for k in ("f", "fbar", "secluded", "accessible"):
        assert np.array_equal(got[k], one[k]), k
    check_against_oracle(d, got, oracle_ref(d))


@pytest.mark.parametrize("seed,n", [(4, (37, 45, 70)), (9, (61, 23, 50))])
def test_level_minimum_equals_pairwise_minimum(seed, n):
    """The minimum over sharp points with dyadic min levels built in the tile (option) and with
    pairwise minima per run (default) select the same minimum (min is exact): f, f_bar, Gamma and A are
    bit-identical, for every orientation-group split, and the result meets the contract; runs
    longer than 16 (a 40-voxel cutter laid along x) exercise levels 3 and 4."""
    d = _small3d(seed=seed, n=n, n_orient=9)
    base = run_gpu(d, orient_batch=5, erode_levels=False)
    for g in (0, 1, 3):
        got = run_gpu(d, orient_batch=5, erode_groups=g, erode_levels=True)
        for k in ("f", "fbar", "secluded", "accessible"):
            assert np.array_equal(got[k], base[k]), (g, k)
    check_against_oracle(d, base, oracle_ref(d))
    c, s_ = np.cos(np.pi / 4), np.sin(np.pi / 4)
    quats = np.array([[c, 0, s_, 0], [c, 0, -s_, 0], [1, 0, 0, 0]])
    rho = synth.beam_density((90, 30, 26), n_beams=8, seed=11)
    d2 = synth.Design(rho, synth.slab_fixture(rho.shape, 2, axis="z"), [synth.cylinder_tool(2, 40, 3, 4, quats)])
    a = run_gpu(d2, orient_batch=3, erode_levels=True)
    b = run_gpu(d2, orient_batch=3, erode_levels=False)
    for k in ("f", "fbar", "secluded", "accessible"):
        assert np.array_equal(a[k], b[k]), k
    check_against_oracle(d2, a, oracle_ref(d2))



def test_sweep_loop_equals_parallel_sweep():
    """The sweep of Eq. eq_conv_A with the batch's orientations walked inside each thread (early
    exit once a word is fully accessible, option) and with one thread per word and orientation
    (default) give the same accessible set (A only grows), on several batch splits; both meet the contract."""
    d = _small3d(seed=11, n=(45, 38, 33), n_orient=13)
    ref = oracle_ref(d)
    for ob in (4, 13):
        a = run_gpu(d, orient_batch=ob, accessible_by_sweep=True, sweep_loop=True)
        b = run_gpu(d, orient_batch=ob, accessible_by_sweep=True)
        assert np.array_equal(a["accessible"], b["accessible"]), ob
        check_against_oracle(d, a, ref)


@pytest.mark.parametrize("seed,n", [(5, (37, 45, 70)), (12, (90, 30, 26))])
def test_erosion_outputs_per_thread_forms_agree(seed, n):
    """The pairwise minimum over sharp points with 8 and with 16 consecutive x outputs per thread
    (option erode_xt; 8 is the default) takes the minimum of the same candidates, in three-value
    blocks and merged run pairs whose cover only overlaps (min is exact): f, f_bar, Gamma and A
    are bit-identical on grids whose x extent is no multiple of either, for every orientation
    group split, and the 16-wide form meets the contract against the oracle; runs of every length
    up to the cap (a 40-voxel cutter along x) are exercised."""
    d = _small3d(seed=seed, n=n, n_orient=9)
    base = run_gpu(d, orient_batch=5, erode_xt=16)
    for g in (0, 1, 3):
        got = run_gpu(d, orient_batch=5, erode_groups=g, erode_xt=8)
        for k in ("f", "fbar", "secluded", "accessible"):
            assert np.array_equal(got[k], base[k]), (g, k)
    check_against_oracle(d, base, oracle_ref(d))
    c, s_ = np.cos(np.pi / 4), np.sin(np.pi / 4)
    quats = np.array([[c, 0, s_, 0], [c, 0, -s_, 0], [1, 0, 0, 0], [0.9, 0.3, 0.3, 0.1]])
    quats = quats / np.linalg.norm(quats, axis=1, keepdims=True)
    rho = synth.beam_density((90, 30, 26), n_beams=8, seed=seed)
    d2 = synth.Design(rho, synth.slab_fixture(rho.shape, 2, axis="z"), [synth.cylinder_tool(2, 40, 3, 4, quats)])
    a = run_gpu(d2, orient_batch=4, erode_xt=16)
    b = run_gpu(d2, orient_batch=4, erode_xt=8)
    for k in ("f", "fbar", "secluded", "accessible"):
        assert np.array_equal(a[k], b[k]), k
    check_against_oracle(d2, a, oracle_ref(d2))
