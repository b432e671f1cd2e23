"""Batched and served forms on the GPU: CUDA-graph replays and autotuned batches give the same
results as a plain imf_compute, and a served request gives the same result alone and when it
runs mixed with requests of other designs."""
import numpy as np
import pytest

from paper_2002_07627_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_07627_gb300 import build
    build.build()


def _designs():
    out = []
    for i, (n, nr, rc) in enumerate([(40, 12, 2), (33, 7, 3), (48, 16, 2), (24, 5, 2)]):
        rho = synth.beam_density((n, n - 3, n - 5), n_beams=6, seed=10 + i)
        fix = synth.slab_fixture(rho.shape, 2, axis="z")
        tool = synth.cylinder_tool(rc, 6, int(2.5 * rc), 5, synth.fibonacci_quats(nr))
        out.append(synth.Design(rho, fix, [tool]))
    return out


def _plain(d):
    from paper_2002_07627_gb300 import binding
    imf = binding.Imf(d.rho.shape)
    imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    fb, sec = imf.compute(rho, fix)
    imf.sync()
    out = fb.cpu().numpy(), sec.cpu().numpy()
    imf.close()
    return out


def test_batch_runner_graphs_and_autotune_match_plain_compute():
    _need_gpu()
    from paper_2002_07627_gb300.batch import BatchRunner
    ds = _designs()
    ref = [_plain(d) for d in ds]
    br = BatchRunner(ds, n_streams=3, autotune=True, graphs=True)
    for e in br.entries:
        assert e.batch in (4, 8, 16, 32, 64)
    for _ in range(2):
        br.run()
    br.check()
    for e, (fb, sec) in zip(br.entries, ref):
        assert np.array_equal(e.fbar.cpu().numpy(), fb)
        assert np.array_equal(e.sec.cpu().numpy(), sec)
    br.close()


def test_served_result_is_the_same_alone_and_in_the_mix():
    _need_gpu()
    from paper_2002_07627_gb300.serve import DesignSpec, GpuExecutor, ImfServer
    ds = _designs()
    specs = [DesignSpec(d.rho.shape, d.tools, d.fixture) for d in ds]
    # alone
    srv = ImfServer(GpuExecutor(1), hbm_budget=8 << 30, slots=1)
    srv.register("a", specs[0])
    alone = srv.submit("a", ds[0].rho).result(timeout=120)
    srv.close()
    # in the mix: other designs' requests before, around and after it, 3 slots
    srv = ImfServer(GpuExecutor(3), hbm_budget=8 << 30, slots=3)
    for i, s in enumerate(specs):
        srv.register(i, s)
    futs = []
    rng = np.random.default_rng(2)
    for k in range(12):
        i = int(rng.integers(1, len(ds)))
        pert = np.clip(ds[i].rho + 0.01 * k, 0, 1).astype(np.float32)
        futs.append(srv.submit(i, pert))
        if k == 5:
            target = srv.submit(0, ds[0].rho)
    mixed = target.result(timeout=120)
    for f in futs:
        f.result(timeout=120)
    assert srv.stats.max_running >= 2          # the requests did overlap
    srv.close()
    assert np.array_equal(alone[0], mixed[0]) and np.array_equal(alone[1], mixed[1])
    ref = _plain(ds[0])
    assert np.array_equal(alone[0], ref[0]) and np.array_equal(alone[1], ref[1])


def test_autotune_under_a_tight_budget_then_compute():
    """The autotuner probes batch sizes that do not fit the handle's budget; afterwards the
    handle must still compute the same result as an unconstrained one."""
    _need_gpu()
    from paper_2002_07627_gb300 import binding
    from paper_2002_07627_gb300.batch import spectra_bytes_estimate
    d = _designs()[2]
    ref = _plain(d)
    imf = binding.Imf(d.rho.shape, hbm_budget_bytes=int(spectra_bytes_estimate(d)) + (24 << 20))
    imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    best = imf.autotune(rho, fix)
    assert best >= 4
    fb, sec = imf.compute(rho, fix)
    imf.sync()
    assert np.array_equal(fb.cpu().numpy(), ref[0]) and np.array_equal(sec.cpu().numpy(), ref[1])
    imf.close()
