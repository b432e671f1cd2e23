"""The allocation-free sensitivity penalty (imf_penalize_sensitivity_noalloc).

It serves callers that cannot allocate device memory, such as a host framework that owns all
device memory through its own pool or code that must not stall the device. Its output must
equal the regular entry point's, within the tolerance of the penalty tests, on two calls in a
row (the second call reuses the scratch array the first one left behind). The file is named to
be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_penalty_matches_the_regular_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_07627_gb300 import binding, build
    build.build()
    lib = binding.load()
    dev = torch.device("cuda", 0)
    shape = (19, 37, 45)
    n = int(np.prod(shape))
    imf = binding.Imf(shape)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        rng = np.random.default_rng(call)
        sens = torch.from_numpy((rng.normal(size=shape) * (3 + call)).astype(np.float32)).to(dev)
        rho = torch.from_numpy(rng.random(shape).astype(np.float32)).to(dev)
        fbar = torch.from_numpy(rng.random(shape).astype(np.float32)).to(dev)
        sec = torch.from_numpy((rng.random(shape) < 0.2).astype(np.uint8)).to(dev)
        fix = torch.from_numpy((rng.random(shape) < 0.1).astype(np.uint8)).to(dev)
        a = sens.clone()
        imf.penalize(a, rho, fbar, sec, fix, w_acc=0.3)
        b = sens.clone()
        st = lib.imf_penalize_sensitivity_noalloc(b.data_ptr(), rho.data_ptr(), fbar.data_ptr(), sec.data_ptr(),
                                                  fix.data_ptr(), n, 0.3, 0.5, stream.cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.max(torch.abs(a - b)).item() <= 1e-6
    # sizes above the scratch limit are rejected on the host
    assert lib.imf_penalize_sensitivity_noalloc(b.data_ptr(), rho.data_ptr(), fbar.data_ptr(), sec.data_ptr(),
                                                None, 268435456 + 1, 0.3, 0.5, stream.cuda_stream) == 1
    imf.close()
