"""Host-side checks that need no GPU: the library builds, loads and exports every symbol the
header declares; the kernels' FFT butterflies (run on the CPU through the host-test library)
match numpy.fft for every radix mix the planner produces; argument checks fail on the host."""
import ctypes
import re
import os

import numpy as np
import pytest

from paper_2002_07627_gb300 import binding, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_exactly_the_exported_symbols(lib):
    hdr = open(os.path.join(ROOT, "include", "imf.h")).read()
    declared = set(re.findall(r"\b(imf_[a-z_]+)\s*\(", hdr))
    assert declared == set(binding.EXPORTS)
    hdr_to = open(os.path.join(ROOT, "include", "imf_to.h")).read()
    declared_to = set(re.findall(r"\b(imf_[a-z0-9_]+)\s*\(", hdr_to))
    assert declared_to == set(binding.EXPORTS_TO)
    declared |= declared_to
    out = os.popen(f"nm -D --defined-only {build.LIB}").read()
    exported = set(re.findall(r" T (imf_[a-z0-9_]+)", out))
    assert declared <= exported


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 21, 25, 30, 35, 42, 49, 56, 60, 64, 84,
                               90, 96, 98, 105, 112, 120, 126, 128, 135, 147, 150, 168, 175, 180, 192, 196, 210,
                               224, 240, 250, 252, 256, 294, 300, 343, 384, 392, 420, 512])
def test_host_fft_matches_numpy(lib, L):
    rng = np.random.default_rng(L)
    x = rng.normal(size=L) + 1j * rng.normal(size=L)
    fwd = binding.host_fft(x, -1)
    inv = binding.host_fft(x, +1)
    scale = np.sqrt(L) * np.abs(x).max()
    assert np.max(np.abs(fwd - np.fft.fft(x))) < 2e-6 * scale * max(1.0, np.log2(L))
    assert np.max(np.abs(inv - np.fft.ifft(x) * L)) < 2e-6 * scale * max(1.0, np.log2(L))


_SPLIT_SIZES = (2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24)
_SPLIT_LENGTHS = sorted({a * b for a in _SPLIT_SIZES for b in _SPLIT_SIZES if a >= b})


@pytest.mark.parametrize("L", _SPLIT_LENGTHS)
def test_host_two_pass_fft_matches_numpy(lib, L):
    """The two-pass register transform (every length A B with A, B in the supported set, factors
    above 16 included: the y and z passes use them for lengths above 256) agrees with numpy's
    FFT in both directions, and its split is the balanced one with A >= B."""
    rng = np.random.default_rng(1000 + L)
    x = rng.normal(size=L) + 1j * rng.normal(size=L)
    fwd, (A, B) = binding.host_fft2(x, -1)
    inv, _ = binding.host_fft2(x, +1)
    assert A * B == L and A >= B and A in _SPLIT_SIZES and B in _SPLIT_SIZES
    assert A == min(a for a in _SPLIT_SIZES if L % a == 0 and L // a in _SPLIT_SIZES and a >= L // a)
    scale = np.sqrt(L) * np.abs(x).max()
    assert np.max(np.abs(fwd - np.fft.fft(x))) < 2e-6 * scale * max(1.0, np.log2(L))
    assert np.max(np.abs(inv - np.fft.ifft(x) * L)) < 2e-6 * scale * max(1.0, np.log2(L))


def test_host_two_pass_fft_single_tones(lib):
    """A unit impulse at n0 transforms to exp(-+2 pi i n0 k / L) exactly up to rounding: pins
    the sign convention and the index maps n = n1 + B n2, k = k2 + A k1 separately."""
    for L in (96, 168, 192, 150, 210, 320, 400, 576):
        for n0 in (0, 1, 7, L - 1):
            x = np.zeros(L, complex)
            x[n0] = 1.0
            k = np.arange(L)
            for sign in (-1, 1):
                got, _ = binding.host_fft2(x, sign)
                assert np.max(np.abs(got - np.exp(sign * 2j * np.pi * n0 * k / L))) < 4e-6


def test_host_two_pass_fft_rejects_unsplittable_lengths(lib):
    for L in (11, 13 * 4, 17 * 2, 7 * 7 * 7, 512):
        with pytest.raises(ValueError):
            binding.host_fft2(np.ones(L, complex))


def test_host_fft_rejects_rough_lengths(lib):
    with pytest.raises(ValueError):
        binding.host_fft(np.ones(11, complex))


def test_default_options_and_create_checks(lib):
    opt = binding.ImfOptions()
    lib.imf_default_options(ctypes.byref(opt))
    assert opt.lambda_ == 0.01 and opt.tau == 0.5 and opt.theta_rel == 0.01 and opt.recheck == 1
    h = ctypes.c_void_p()
    assert lib.imf_create(ctypes.byref(opt), ctypes.byref(h)) == 1      # 0x0x0 grid
    opt.nx, opt.ny, opt.nz = 8, 8, 1
    opt.lambda_ = 1.5
    assert lib.imf_create(ctypes.byref(opt), ctypes.byref(h)) == 1      # lambda out of range
    opt.lambda_ = 0.01
    assert opt.erode_xt == 0
    opt.erode_xt = 12
    assert lib.imf_create(ctypes.byref(opt), ctypes.byref(h)) == 1      # 8 or 16 outputs per thread only
    opt.erode_xt = 0
    assert lib.imf_create(ctypes.byref(opt), ctypes.byref(h)) == 0
    # host-side argument errors need no GPU
    assert lib.imf_compute(h, None, None, None, None, None, None, None) == 5   # no tool yet
    assert b"imf_set_tool" in lib.imf_last_error(h)
    cut = np.ones((1, 1, 1), np.uint8)
    org = (ctypes.c_int * 3)(0, 0, 0)
    q = np.array([1.0, 0, 0, 0])
    assert lib.imf_set_tool(h, 3, cut.ctypes.data, cut.ctypes.data, None, 1, 1, 1, org, q.ctypes.data, 1) == 1
    zero = np.zeros((1, 1, 1), np.uint8)
    assert lib.imf_set_tool(h, 0, zero.ctypes.data, zero.ctypes.data, None, 1, 1, 1, org, q.ctypes.data, 1) == 1
    assert b"empty cutter" in lib.imf_last_error(h)
    assert lib.imf_penalize_sensitivity(h, None, None, None, None, None, 0.5, None) == 1
    lib.imf_destroy(h)
    lib.imf_destroy(None)


def test_mma_selftest_rejects_bad_shapes_on_the_host(lib):
    """The tensor-core self-test checks N, K and the operands' shared-memory size before any
    allocation (the arrays below are never read): N outside [16, 256] or not a multiple of 16,
    K below 16 or not a multiple of 16, and (128 + N) K 2 bytes above 200 KB are refused."""
    import ctypes
    f = lib.imf_selftest_mma
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    a = (ctypes.c_uint16 * 16)()
    d = (ctypes.c_float * 16)()
    for n, k in ((0, 16), (8, 16), (24, 16), (272, 16), (16, 0), (16, 8), (16, 24), (16, -16),
                 (256, 512), (16, 720)):
        assert f(n, k, ctypes.addressof(a), ctypes.addressof(a), ctypes.addressof(d)) == 1, (n, k)
    assert f(16, 16, None, ctypes.addressof(a), ctypes.addressof(d)) == 1


def test_noalloc_penalty_rejects_bad_arguments_on_the_host(lib):
    """The allocation-free penalty checks its arguments before any CUDA call: NULL arrays,
    n < 1, n above the scratch limit, w_acc outside [0, 1) and tau outside [0, 1] are refused
    with IMF_ERR_INVALID_ARG. The pointers below are never dereferenced."""
    f = lib.imf_penalize_sensitivity_noalloc
    p = 0x1000
    assert f(None, p, p, p, None, 10, 0.3, 0.5, None) == 1
    assert f(p, None, p, p, None, 10, 0.3, 0.5, None) == 1
    assert f(p, p, None, p, None, 10, 0.3, 0.5, None) == 1
    assert f(p, p, p, None, None, 10, 0.3, 0.5, None) == 1
    assert f(p, p, p, p, None, 0, 0.3, 0.5, None) == 1
    assert f(p, p, p, p, None, -5, 0.3, 0.5, None) == 1
    assert f(p, p, p, p, None, 268435456 + 1, 0.3, 0.5, None) == 1
    assert f(p, p, p, p, None, 10, 1.0, 0.5, None) == 1
    assert f(p, p, p, p, None, 10, -0.1, 0.5, None) == 1
    assert f(p, p, p, p, None, 10, float("nan"), 0.5, None) == 1
    assert f(p, p, p, p, None, 10, 0.3, 1.5, None) == 1
    assert f(p, p, p, p, None, 10, 0.3, -0.5, None) == 1


def test_plan_only_footprint_of_the_128_workload(lib):
    """The planner runs on the host (plan_only handle: the tool is resampled on the CPU with the
    device kernel's arithmetic and nothing touches a device). For the 128^3 x 64 workload's tool
    it picks the padded grid (192, 192, 168) the GPU runs use; the footprint adds the resident
    spectra (n_orient Pz Py Hs complex64) and tables, the work buffers of 64 orientation slots
    and the set-up peak; a plan-only handle refuses to compute."""
    tool = synth.cylinder_tool(3, 20, 8, 16, synth.fibonacci_quats(64))
    imf = binding.Imf((128, 128, 128), plan_only=True)
    imf.set_tools([tool])
    info = imf.tool_info(0)
    assert info.P == (192, 192, 168)
    Hs = (192 // 2 + 1 + 1) & ~1
    assert info.spectra_bytes == 64 * 168 * 192 * Hs * 8
    fp = imf.footprint()
    assert fp.slots == 64
    assert info.spectra_bytes < fp.resident < 1.01 * info.spectra_bytes
    wx, wy, wz = info.win
    gpx, wpr = (wx + 3) & ~3, (wx + 31) // 32 + 2
    per_slot = wz * 192 * Hs * 8 + wz * wy * Hs * 8 + wz * wy * gpx * 4 + wz * wy * wpr * 4 * 5
    assert fp.work > 64 * per_slot and fp.work < 64 * per_slot + 200 * 2 ** 20
    assert fp.total == max(fp.resident + fp.work, fp.setup_peak)
    assert fp.setup_peak > info.spectra_bytes
    fp1 = imf.footprint(1)
    assert fp1.slots == 1 and fp1.work < fp.work
    with pytest.raises(binding.ImfError) as ei:
        imf._check(imf.lib.imf_compute(imf.h, 1, None, 1, 1, None, None, None))
    assert ei.value.status == 5
    imf.close()


def test_stage_reciprocals_are_exact(lib):
    L = ctypes.CDLL(build.HOSTLIB)
    L.imf_host_check_div.restype = ctypes.c_long
    # every stage divisor up to the longest plan, for every butterfly index the kernels use
    assert L.imf_host_check_div(4096, 1 << 20) == 0


def _host_plan(sh, K, maxl=16):
    import ctypes
    from paper_2002_07627_gb300 import build
    L = ctypes.CDLL(build.HOSTLIB)
    sh = np.ascontiguousarray(np.asarray(sh, np.int32).reshape(-1, 3))
    Ka = np.ascontiguousarray(np.asarray(K, np.int32))
    consts = np.zeros(7, np.int64)
    L.imf_host_erode_constants(consts.ctypes.data_as(ctypes.c_void_p))
    chunks = np.zeros((4096, 44), np.int32)
    runs = np.zeros((1 << 16, 2), np.int32)
    smem = ctypes.c_long(0)
    nruns = ctypes.c_int(0)
    L.imf_host_plan_erode.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_long),
                                      ctypes.POINTER(ctypes.c_int)]
    n = L.imf_host_plan_erode(sh.ctypes.data, len(sh), Ka.ctypes.data, maxl, len(chunks), chunks.ctypes.data,
                              len(runs), runs.ctypes.data, ctypes.byref(smem), ctypes.byref(nruns))
    assert n >= 0
    c = dict(zip(["tx", "ty", "tz", "xt", "maxl", "budget", "maxruns"], consts.tolist()))
    c["maxl"] = maxl
    return chunks[:n], runs[:nruns.value], smem.value, c


def _plan_cases():
    from oracle.ref import resample_tool
    cases = []
    big = synth.cylinder_tool(3, 20, 8, 16, synth.fibonacci_quats(64))
    for i in (0, 7, 23, 41, 63):
        cases.append(resample_tool(big, big.quats[i])["sharp"])
    small = synth.cylinder_tool(2, 6, 4, 6, np.random.default_rng(5).normal(size=(3, 4)))
    for q in small.quats:
        cases.append(resample_tool(small, q)["sharp"])
    planar = synth.planar_tool(n_orient=8)
    cases.append(resample_tool(planar, planar.quats[3])["sharp"])
    long_x = synth.box_tool(ext=(37, 3, 2))                 # runs longer than the 16-sample limit
    cases.append(resample_tool(long_x, np.array([1.0, 0, 0, 0]))["sharp"])
    return cases


@pytest.mark.parametrize("maxl", [16, 31])
@pytest.mark.parametrize("case", range(10))
def test_erosion_plan_covers_every_sharp_point_once_within_the_tile(lib, case, maxl):
    """The plan of the tiled minimum over sharp points (Eq. eq_imf_2), decoded with only the
    window origin K and each chunk's tile origin: its runs cover every sharp point exactly once,
    sit in length groups of at most 16 (the pairwise kernel) or 31 (the level kernel), every
    thread position reads inside its chunk's tile, the tile and its run descriptors fit the
    budget together and the 32 lanes of a warp (8 rows x 4 planes) hit 32 banks."""
    sh = np.asarray(_plan_cases()[case], np.int64)
    rng = np.random.default_rng(case)
    K = sh.max(0) + rng.integers(0, 5, size=3)      # any window origin at or beyond the largest offset
    chunks, runs, smem, c = _host_plan(sh, K, maxl)
    covered = []
    nxt = c["tx"] // c["xt"]
    for ch in chunks:
        run0, run1, txh, tyh, tzh, P, Q, ox, oy, oz = ch[:10]
        lend = ch[10:42]
        assert P % 2 == 1 and P >= txh and Q >= tyh * P
        banks = {(tz * Q + ty * P) % 32 for tz in range(4) for ty in range(8)}
        assert len(banks) == 32
        # tile and run descriptors (8 bytes each, 8-byte aligned behind the tile) fit together
        need = 4 * ((tzh * Q + 1) // 2 * 2) + 8 * (run1 - run0)
        assert need <= max(c["budget"], 4 * c["tz"] * Q + 8 * c["maxruns"]) and need <= smem
        assert 0 < run1 - run0 <= c["maxruns"] and lend[0] == 0 and lend[c["maxl"]] == run1 - run0
        for Lr in range(1, c["maxl"] + 1):
            seg = runs[run0 + lend[Lr - 1]: run0 + lend[Lr]]
            assert np.all(seg[:, 1] == Lr)
        for off, Lr in runs[run0:run1]:
            iz, rem = divmod(int(off), int(Q))
            iy, ix = divmod(rem, int(P))
            # the reads of the thread farthest from the block origin stay in the tile
            assert ix + (nxt - 1) * c["xt"] + c["xt"] + Lr - 2 <= txh - 1
            assert iy + c["ty"] - 1 <= tyh - 1 and iz + c["tz"] - 1 <= tzh - 1
            kz, ky, kx_last = K[2] - oz - iz, K[1] - oy - iy, K[0] - ox - ix
            covered += [(kx, ky, kz) for kx in range(kx_last - Lr + 1, kx_last + 1)]
    assert len(covered) == len(sh)
    assert sorted(covered) == sorted(map(tuple, sh.tolist()))


def _sliding_or(row_bits, start, L):
    """32 bits: bit t is the OR of row_bits[start + t .. start + t + L - 1] (0 past the row)."""
    n = len(row_bits)
    out = 0
    for t in range(32):
        lo, hi = start + t, min(n, start + t + L)
        if lo < hi and row_bits[lo:hi].any():
            out |= 1 << t
    return out


def test_sweep_run_from_dilation_levels_equals_the_sliding_or(lib):
    """One cutter run of the sweep (Eq. eq_conv_A) as the kernels compute it: dilation levels
    D_j of the free bits and two windows of length 2^j per run must give the sliding OR of
    length L for every run length 1 .. 32, every bit shift and output word, on sparse, dense
    and structured rows (brute force on the unpacked bits)."""
    L_ = ctypes.CDLL(build.HOSTLIB)
    L_.imf_host_sweep_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p]
    rng = np.random.default_rng(7)
    wpr = 8
    rows = [rng.random(32 * wpr) < p for p in (0.02, 0.3, 0.9)]
    iso = np.zeros(32 * wpr, bool)
    iso[[0, 31, 32, 63, 100, 159, 160, 200]] = True          # isolated bits at word edges
    rows.append(iso)
    out = np.zeros(1, np.uint32)
    for bits in rows:
        words = np.packbits(bits.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).ravel()
        words = np.ascontiguousarray(words)
        for L in range(1, 33):
            for s in list(range(0, 40)) + [63, 64, 95]:
                for q in (0, 1, 2):
                    rc = L_.imf_host_sweep_run(words.ctypes.data, wpr, q, s, L, out.ctypes.data)
                    if q + s // 32 + 2 >= wpr:
                        continue
                    assert rc == 0, (L, s, q)
                    assert int(out[0]) == _sliding_or(bits, 32 * q + s, L), (L, s, q)
    assert L_.imf_host_sweep_run(words.ctypes.data, wpr, 0, 0, 33, out.ctypes.data) == 1   # runs are <= 32
    assert L_.imf_host_sweep_run(words.ctypes.data, wpr, 7, 0, 4, out.ctypes.data) == 1    # past the row


def test_flag_bytes_pack_into_bits(lib):
    """The x pass's packing of 32 free-flag bytes into one word: bit b = low bit of byte b,
    whatever the other bits of the bytes hold (the multiply must not carry between groups)."""
    L_ = ctypes.CDLL(build.HOSTLIB)
    L_.imf_host_pack_flags.argtypes = [ctypes.c_void_p]
    L_.imf_host_pack_flags.restype = ctypes.c_uint32
    rng = np.random.default_rng(3)
    cases = [np.zeros(32, np.uint8), np.ones(32, np.uint8)] + [rng.integers(0, 2, 32).astype(np.uint8) for _ in range(200)]
    cases += [rng.integers(0, 256, 32).astype(np.uint8) for _ in range(200)]
    for b in cases:
        b = np.ascontiguousarray(b)
        want = sum(int(v & 1) << i for i, v in enumerate(b))
        assert L_.imf_host_pack_flags(b.ctypes.data) == want


def _is_smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def test_planner_picks_smooth_two_pass_lengths_close_to_the_minimum(lib):
    """The padded FFT length (the linear correlation needs any length >= the minimum): it is
    2-3-5-7 smooth, at most 1/8 above the smallest smooth length, and a two-pass split is used
    whenever a smooth length in that range has one (the cost model prefers them). Above 256 the
    y and z passes (factors up to 24) find splits the x pass (factors up to 16) cannot."""
    L_ = ctypes.CDLL(build.HOSTLIB)
    L_.imf_host_plan_length.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]
    A, B = ctypes.c_int(), ctypes.c_int()
    sizes = (2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24)
    for maxA in (16, 24):
        ok_sizes = [s for s in sizes if s <= maxA]
        splittable = {a * b for a in ok_sizes for b in ok_sizes if a >= b}
        for n in range(4, 600):
            L = L_.imf_host_plan_length(n, maxA, ctypes.byref(A), ctypes.byref(B))
            n0 = next(m for m in range(n, 10 * n) if _is_smooth(m))
            assert _is_smooth(L) and n <= L <= n0 + n0 // 8, (n, maxA, L)
            if any(m in splittable for m in range(n0, n0 + n0 // 8 + 1) if _is_smooth(m)):
                assert A.value * B.value == L and A.value >= B.value and A.value <= maxA, (n, maxA, L)
    # the 256^3 workload's y axis: 294 needs a factor above 16
    L = L_.imf_host_plan_length(294, 16, ctypes.byref(A), ctypes.byref(B))
    assert A.value == 0
    L = L_.imf_host_plan_length(294, 24, ctypes.byref(A), ctypes.byref(B))
    assert A.value > 16 and A.value * B.value == L


def _rotations(n, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=1)
    return np.ascontiguousarray(R)


def test_orientation_order_chain_and_interleave(lib):
    """The internal orientation order: a greedy nearest-neighbour chain from the first rotation
    (Frobenius distance; brute force here), and on the FFT path its interleave by the radical
    inverse, which is a permutation of the chain whose every prefix of length 2^k takes one
    chain position from each block of n / 2^k consecutive positions."""
    L_ = ctypes.CDLL(build.HOSTLIB)
    L_.imf_host_orient_order.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    for n, seed in ((1, 0), (7, 1), (64, 2), (100, 3)):
        R = _rotations(n, seed)
        chain = np.zeros(n, np.int32)
        spread = np.zeros(n, np.int32)
        L_.imf_host_orient_order(R.ctypes.data, n, 0, chain.ctypes.data)
        L_.imf_host_orient_order(R.ctypes.data, n, 1, spread.ctypes.data)
        # brute-force greedy chain
        used, cur, want = np.zeros(n, bool), 0, []
        for _ in range(n):
            want.append(cur)
            used[cur] = True
            if used.all():
                break
            d = np.where(used, np.inf, ((R - R[cur]) ** 2).sum(1))
            cur = int(np.argmin(d))
        assert chain.tolist() == want
        assert sorted(spread.tolist()) == list(range(n))
        pos = {c: i for i, c in enumerate(chain.tolist())}
        ranks = [pos[c] for c in spread.tolist()]
        if n == 64:
            for k in range(7):
                m = 1 << k
                assert sorted(r // (n // m) for r in ranks[:m]) == list(range(m)), k
