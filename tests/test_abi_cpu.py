"""Host-side checks that need no GPU: the library builds, loads and exports every symbol the
header declares; the kernels' FFT butterflies (run on the CPU through the host-test library)
match numpy.fft for every radix mix the planner produces; argument checks fail on the host."""
import ctypes
import re
import os

import numpy as np
import pytest

from paper_2002_07627_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_exactly_the_exported_symbols(lib):
    hdr = open(os.path.join(ROOT, "include", "imf.h")).read()
    declared = set(re.findall(r"\b(imf_[a-z_]+)\s*\(", hdr))
    assert declared == set(binding.EXPORTS)
    out = os.popen(f"nm -D --defined-only {build.LIB}").read()
    exported = set(re.findall(r" T (imf_[a-z_]+)", out))
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


_SPLIT_SIZES = (2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16)
_SPLIT_LENGTHS = sorted({a * b for a in _SPLIT_SIZES for b in _SPLIT_SIZES if a >= b})


@pytest.mark.parametrize("L", _SPLIT_LENGTHS)
def test_host_two_pass_fft_matches_numpy(lib, L):
    """The two-pass register transform (every length A B with A, B in the supported set) agrees
    with numpy's FFT in both directions, and its split is the balanced one with A >= B."""
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
    for L in (96, 168, 192, 150, 210):
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


def test_stage_reciprocals_are_exact(lib):
    L = ctypes.CDLL(build.HOSTLIB)
    L.imf_host_check_div.restype = ctypes.c_long
    # every stage divisor up to the longest plan, for every butterfly index the kernels use
    assert L.imf_host_check_div(4096, 1 << 20) == 0
