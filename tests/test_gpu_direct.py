"""The direct tensor-core path (tcgen05 implicit GEMM, BF16 hi/lo inputs, FP32 accumulation in
TMEM): the MMA building block against exact and FP64 references, then the whole IMF through
the direct path against the FP64 oracle and against the FFT path."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2002_07627_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_07627_gb300 import binding, build
    build.build()
    return binding


def _bf16_bits(x):
    x = np.asarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)       # round to nearest even
    return r


def _bf16_value(b):
    return (b.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("N,K", [(16, 16), (16, 64), (32, 48), (64, 128), (128, 64), (256, 32)])
def test_tcgen05_mma_selftest(N, K):
    binding = _lib()
    lib = binding.load()
    rng = np.random.default_rng(N * 1000 + K)
    # small integers: every product and partial sum is exact in FP32
    A = rng.integers(-3, 4, size=(128, K)).astype(np.float32)
    B = rng.integers(-2, 3, size=(N, K)).astype(np.float32)
    Ab, Bb = _bf16_bits(A), _bf16_bits(B)
    D = np.zeros((128, N), np.float32)
    st = lib.imf_selftest_mma(N, K, Ab.ctypes.data, Bb.ctypes.data, D.ctypes.data)
    assert st == 0
    assert np.array_equal(D, A @ B.T)
    # random BF16 values against an FP64 reference
    A = rng.normal(size=(128, K)).astype(np.float32)
    B = (rng.random((N, K)) < 0.5).astype(np.float32)
    Ab, Bb = _bf16_bits(A), _bf16_bits(B)      # keep both alive across the call
    st = lib.imf_selftest_mma(N, K, Ab.ctypes.data, Bb.ctypes.data, D.ctypes.data)
    assert st == 0
    ref = _bf16_value(Ab).astype(np.float64) @ B.T.astype(np.float64)
    assert np.abs(D - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max()) * K


def _run(design, precision, **kw):
    binding = _lib()
    imf = binding.Imf(design.rho.shape, precision=precision, **kw)
    imf.set_tools(design.tools)
    rho = torch.from_numpy(np.ascontiguousarray(design.rho)).cuda()
    fix = None if design.fixture is None else torch.from_numpy(np.ascontiguousarray(design.fixture)).cuda()
    raw = torch.empty_like(rho)
    acc = torch.empty(rho.shape, dtype=torch.uint8, device="cuda")
    fbar, sec = imf.compute(rho, fix, raw=raw, accessible=acc)
    imf.sync()
    info = imf.tool_info(0)
    out = dict(f=raw.cpu().numpy().astype(np.float64), fbar=fbar.cpu().numpy().astype(np.float64),
               secluded=sec.cpu().numpy(), accessible=acc.cpu().numpy(), info=info)
    imf.close()
    return out


def _check(design, got, ref):
    size = int(((design.tools[0].holder != 0) | (design.tools[0].cutter != 0)).sum())
    theta = 0.01 * size
    fmax = float(ref["f"].max())
    assert np.abs(got["f"] - ref["f"]).max() <= 1e-4 * fmax
    clear = np.abs(ref["f"] - theta) > 1e-3 * size
    if design.fixture is not None:
        clear &= design.fixture == 0
    assert np.array_equal(got["accessible"][clear], ref["accessible"][clear])
    ok = np.abs(ref["fbar"] - 0.01) > 1e-4
    assert np.abs(got["fbar"] - ref["fbar"])[ok].max() <= 2e-4
    assert np.array_equal(got["secluded"][ok], ref["secluded"][ok])


def test_direct_path_planar64_matches_oracle():
    d = synth.config_planar64(seed=0)
    got = _run(d, precision=2)
    assert got["info"].path == 2
    _check(d, got, oracle.imf(d))


def test_direct_path_3d_ragged_matches_oracle_and_fft():
    rho = synth.beam_density((37, 29, 23), n_beams=8, seed=3)
    fix = synth.slab_fixture(rho.shape, 2, axis="z")
    tool = synth.cylinder_tool(2, 5, 3, 4, synth.fibonacci_quats(20))
    d = synth.Design(rho, fix, [tool])
    got = _run(d, precision=2, orient_batch=16)
    assert got["info"].path == 2
    _check(d, got, oracle.imf(d))
    fft = _run(d, precision=1)
    assert np.abs(got["f"] - fft["f"]).max() <= 1e-4 * fft["f"].max()


def test_auto_precision_autotunes_between_paths():
    binding = _lib()
    d = synth.config_planar64(seed=1)
    imf = binding.Imf(d.rho.shape, precision=0)
    imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    imf.autotune(rho, fix)
    assert imf.tool_info(0).path in (1, 2)
    for path in (1, 2):
        imf.set_path(0, path)
        raw = torch.empty_like(rho)
        imf.compute(rho, fix, raw=raw)
        imf.sync()
        if path == 1:
            f1 = raw.cpu().numpy()
        else:
            f2 = raw.cpu().numpy()
    assert np.abs(f1 - f2).max() <= 1e-4 * f1.max()
    imf.close()


def test_direct_path_tall_tool_in_z_slabs_matches_oracle_and_fft():
    """A tool ~70 voxels tall, tilted at most 20 degrees: one box of its union for a tile (about
    56 x 43 words per plane over ~72 planes, ~700 KB) exceeds shared memory, so the
    direct path loads it in z-slabs (one tensor copy per tile and slab, each slab's taps padded
    to whole chunks, the MMAs accumulating across slabs). The result meets the contract against
    the oracle and agrees with the FFT path."""
    rho = synth.beam_density((40, 36, 28), n_beams=8, seed=5)
    fix = synth.slab_fixture(rho.shape, 2, axis="z")
    ang = np.radians([0.0, 12.0, -12.0, 20.0])           # tilts about x: a narrow, tall union
    quats = np.stack([np.cos(ang / 2), np.sin(ang / 2), 0 * ang, 0 * ang], -1)
    tool = synth.cylinder_tool(3, 20, 8, 50, quats)
    d = synth.Design(rho, fix, [tool])
    from oracle.ref import resample_tool
    union = np.concatenate([resample_tool(tool, q)["RT"] for q in tool.quats])
    ext = union.max(0) - union.min(0) + 1
    assert ext[2] >= 70 and (35 + ext[0]) * (1 + ext[1]) * (1 + ext[2]) * 4 > 227 * 1024
    got = _run(d, precision=2, orient_batch=4)
    assert got["info"].path == 2
    _check(d, got, oracle.imf(d))
    fft = _run(d, precision=1)
    assert np.abs(got["f"] - fft["f"]).max() <= 1e-4 * fft["f"].max()
