"""Batched and served forms on the GPU: CUDA-graph replays and autotuned batches give the same
results as a plain imf_compute, and a served request gives the same result alone and when it
runs mixed with requests of other designs."""
import numpy as np
import pytest

import oracle
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


def _check_vs_oracle(d, fbar, sec, lam=0.01):
    """f_bar and Gamma of one design against the FP64 oracle, away from the allowance
    discontinuity (the IMF contract of the plain form)."""
    ref = oracle.imf(d)
    # away from the allowance discontinuity, compared on f / M before the allowance
    M = float(ref["M"])
    pre = ref["f"] / M if M > 0 else np.zeros_like(ref["f"])
    clear = np.abs(pre - lam) > 1e-4
    if d.fixture is not None:
        clear |= d.fixture != 0
    assert np.abs(fbar.astype(np.float64) - ref["fbar"])[clear].max(initial=0) <= 2e-4
    assert np.array_equal(sec[clear], ref["secluded"][clear])


def test_batch_runner_graphs_and_autotune_match_plain_compute():
    """The batched form (autotuned orientation batch, FFT form, pass launch forms and erosion
    work units; CUDA graphs; a stream pool) gives results bit-identical to a plain compute with
    default options, and meets the contract against the oracle."""
    _need_gpu()
    from paper_2002_07627_gb300.batch import BatchRunner
    ds = _designs()
    ref = [_plain(d) for d in ds]
    br = BatchRunner(ds, n_streams=3, autotune=True, graphs=True)
    for e in br.entries:
        assert e.batch in (4, 8, 16, 32, 64)
        assert e.tuned["fft_stages_only"] in (0, 1) and e.tuned["fft_tma"] in (-1, 0, 1, 10)
        assert e.tuned["fft_wide_pencils"] in (-1, 0) and e.tuned["erode_groups"] in (0, 2, 4, 8, 16)
    for _ in range(2):
        br.run()
    br.check()
    for e, (fb, sec), d in zip(br.entries, ref, ds):
        assert np.array_equal(e.fbar.cpu().numpy(), fb)
        assert np.array_equal(e.sec.cpu().numpy(), sec)
        _check_vs_oracle(d, e.fbar.cpu().numpy(), e.sec.cpu().numpy())
    br.close()


@pytest.mark.parametrize("high_prio", [0, 2])
def test_served_result_is_the_same_alone_and_in_the_mix(high_prio):
    """high_prio: stream slots at the device's highest priority (small requests go there)."""
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
    srv = ImfServer(GpuExecutor(3, high_priority_slots=high_prio), hbm_budget=8 << 30, slots=3)
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
    _check_vs_oracle(ds[0], alone[0], alone[1])


def test_autotune_under_a_tight_budget_then_compute():
    """The autotuner probes batch sizes that do not fit the handle's budget; afterwards the
    handle must still compute the same result as an unconstrained one."""
    _need_gpu()
    from paper_2002_07627_gb300 import binding
    from paper_2002_07627_gb300.batch import planned_footprint
    d = _designs()[2]
    ref = _plain(d)
    fp = planned_footprint(d, slots=1)
    imf = binding.Imf(d.rho.shape, hbm_budget_bytes=int(max(fp.setup_peak, fp.resident + fp.work)) + (24 << 20))
    imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    best = imf.autotune(rho, fix)
    assert best >= 4
    fb, sec = imf.compute(rho, fix)
    imf.sync()
    assert np.array_equal(fb.cpu().numpy(), ref[0]) and np.array_equal(sec.cpu().numpy(), ref[1])
    _check_vs_oracle(d, fb.cpu().numpy(), sec.cpu().numpy())
    imf.close()


def test_planned_footprint_equals_what_the_handle_allocates():
    """The admission figure comes from the library's plan (plan_only handle, host only): a real
    handle of the same design owns exactly the planned resident bytes after set-up and the
    planned total after its first compute, and plans the same padded grid and window; one and
    two tools, a 2D grid, a budget-free default slot count and an explicit one."""
    _need_gpu()
    from paper_2002_07627_gb300 import binding
    from paper_2002_07627_gb300.batch import planned_footprint
    ds = _designs()[:2]
    two = synth.Design(ds[0].rho, ds[0].fixture, ds[0].tools + [synth.cylinder_tool(1, 4, 3, 3, synth.fibonacci_quats(5))])
    for d, ob in ((ds[0], 0), (ds[1], 3), (two, 4), (synth.config_planar64(seed=1), 0)):
        fp = planned_footprint(d, orient_batch=ob)
        imf = binding.Imf(d.rho.shape, orient_batch=ob)
        imf.set_tools(d.tools)
        assert imf.stats().owned_bytes == fp.resident
        plan = binding.Imf(d.rho.shape, orient_batch=ob, plan_only=True)
        plan.set_tools(d.tools)
        for i in range(len(d.tools)):
            a, b = imf.tool_info(i), plan.tool_info(i)
            assert (a.P, a.win, a.kmax, a.n_rt, a.n_rk, a.n_sharp) == (b.P, b.win, b.kmax, b.n_rt, b.n_rk, b.n_sharp)
        plan.close()
        rho = torch.from_numpy(np.ascontiguousarray(d.rho)).cuda()
        fix = None if d.fixture is None else torch.from_numpy(np.ascontiguousarray(d.fixture)).cuda()
        imf.compute(rho, fix)
        imf.sync()
        assert imf.stats().owned_bytes == fp.resident + fp.work
        assert fp.total >= fp.resident + fp.work
        imf.close()


def test_concurrent_requests_of_one_design_on_clones_match_plain():
    """Several requests of one design in flight at once run on clones of its handle (shared tool
    spectra, own work buffers, imf_clone): every result equals a plain compute of the same
    density, and the server did run more than one context of the design."""
    _need_gpu()
    from paper_2002_07627_gb300 import binding
    from paper_2002_07627_gb300.serve import DesignSpec, GpuExecutor, ImfServer
    d = _designs()[0]
    spec = DesignSpec(d.rho.shape, d.tools, d.fixture)
    srv = ImfServer(GpuExecutor(4), hbm_budget=8 << 30, slots=4, max_inflight=3)
    srv.register(0, spec)
    rhos = [np.clip(d.rho + 0.02 * k, 0, 1).astype(np.float32) for k in range(9)]
    futs = [srv.submit(0, r) for r in rhos]
    outs = [f.result(timeout=120) for f in futs]
    assert srv.stats.max_contexts >= 2
    srv.close()
    imf = binding.Imf(d.rho.shape, orient_batch=16)
    imf.set_tools(d.tools)
    fix = torch.from_numpy(d.fixture).cuda()
    for r, (fb, sec) in zip(rhos, outs):
        a, b = imf.compute(torch.from_numpy(r).cuda(), fix)
        imf.sync()
        assert np.array_equal(fb, a.cpu().numpy()) and np.array_equal(sec, b.cpu().numpy())
    imf.close()


def test_clone_shares_tools_and_outlives_its_parent():
    """A clone computes the same result as its parent; destroying the parent first leaves the
    clone's shared tools intact; set_tool on a handle whose tools are shared is refused."""
    _need_gpu()
    from paper_2002_07627_gb300 import binding
    d = _designs()[1]
    imf = binding.Imf(d.rho.shape)
    imf.set_tools(d.tools)
    c = imf.clone()
    with pytest.raises(binding.ImfError):
        imf.set_tools(d.tools)
    rho = torch.from_numpy(d.rho).cuda()
    fix = torch.from_numpy(d.fixture).cuda()
    a, b = imf.compute(rho, fix)
    imf.sync()
    ref = a.cpu().numpy(), b.cpu().numpy()
    imf.close()
    x, y = c.compute(rho, fix)
    c.sync()
    assert np.array_equal(x.cpu().numpy(), ref[0]) and np.array_equal(y.cpu().numpy(), ref[1])
    c.close()
