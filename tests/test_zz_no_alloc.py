"""The allocation-free sensitivity penalty (imf_penalize_sensitivity_noalloc).

It serves callers that cannot allocate device memory, such as a host framework that owns all
device memory through its own pool or code that must not stall the device. Its output must
equal the regular entry point's, within the tolerance of the penalty tests, on two calls in a
row (the second call reuses the scratch array the first one left behind), and the FP64
oracle's penalty. The cases cover a fixture and none, an all-zero S_phi (the maximum is 0, so
S_phi is left unnormalised) and a grid of more than 16 scratch partials. The file is named to
be collected last. Its host-side argument rejections are checked without a GPU in
test_abi_cpu.py.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("shape,with_fixture,zero_sens", [((19, 37, 45), True, False), ((19, 37, 45), False, False),
                                                          ((11, 23, 29), True, True), ((40, 64, 64), True, False)])
def test_noalloc_penalty_matches_the_regular_entry_point_twice(shape, with_fixture, zero_sens):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_07627_gb300 import binding, build
    build.build()
    lib = binding.load()
    dev = torch.device("cuda", 0)
    n = int(np.prod(shape))
    imf = binding.Imf(shape)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        rng = np.random.default_rng(call + 10 * n)
        s_np = np.zeros(shape, np.float32) if zero_sens else (rng.normal(size=shape) * (3 + call)).astype(np.float32)
        r_np = rng.random(shape).astype(np.float32)
        fb_np = rng.random(shape).astype(np.float32)
        sec_np = (rng.random(shape) < 0.2).astype(np.uint8)
        fix_np = (rng.random(shape) < 0.1).astype(np.uint8) if with_fixture else None
        sens = torch.from_numpy(s_np).to(dev)
        rho = torch.from_numpy(r_np).to(dev)
        fbar = torch.from_numpy(fb_np).to(dev)
        sec = torch.from_numpy(sec_np).to(dev)
        fix = torch.from_numpy(fix_np).to(dev) if with_fixture else None
        a = sens.clone()
        imf.penalize(a, rho, fbar, sec, fix, w_acc=0.3)
        b = sens.clone()
        st = lib.imf_penalize_sensitivity_noalloc(b.data_ptr(), rho.data_ptr(), fbar.data_ptr(), sec.data_ptr(),
                                                  fix.data_ptr() if fix is not None else None, n, 0.3, 0.5,
                                                  stream.cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.max(torch.abs(a - b)).item() <= 1e-6
        ref = oracle.penalize(s_np, r_np, fb_np, sec_np, fix_np, 0.3)
        assert np.abs(b.cpu().numpy() - ref).max() <= 1e-5
    imf.close()
