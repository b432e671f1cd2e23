"""GPU parity of the topology-optimisation steps around the IMF (include/imf_to.h, Alg. 2)
against the FP64 oracle (oracle/to2d.py), through the C ABI: projection, FEA (conjugate
gradient against the oracle's direct solve), filtered sensitivity, optimality-criteria update,
one accessibility-constrained iteration, and the constraint's effect over a short run."""
import numpy as np
import pytest

from oracle import to2d
from paper_2002_07627_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_07627_gb300 import binding, build
    build.build()
    return binding


def _case(nelx=48, nely=24, seed=0):
    f, fixed, fix = synth.cantilever2d(nelx, nely)
    xi = np.random.default_rng(seed).uniform(0.05, 0.95, (nely, nelx)).astype(np.float32)
    xi[fix != 0] = 1.0
    return f, fixed, fix, xi


def test_projection_fea_and_sensitivity_match_oracle():
    """rho = Heaviside(xi) (Eq. eq_Heaviside), u and the compliance from the conjugate gradient
    (tolerance 1e-10) against the oracle's direct solve, and the filtered sensitivity -dc/dxi."""
    binding = _need()
    f, fixed, fix, xi = _case()
    nely, nelx = xi.shape
    to = binding.To2d(nelx, nely, cg_tol=1e-10)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xi_d, rho_d, s_d = d(xi), torch.empty(xi.shape, device="cuda"), torch.empty(xi.shape, device="cuda")
    u_d = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    to.project(xi_d, rho_d)
    c, it, res = to.analyze(rho_d, d(f), d(fixed), u_d)
    to.sensitivity(xi_d, rho_d, s_d)
    torch.cuda.synchronize()
    rho_o, drho_o = to2d.heaviside(xi.astype(np.float64), 2.0)
    assert np.abs(rho_d.cpu().numpy() - rho_o).max() < 2e-7
    # the oracle solves with the GPU's (FP32) densities so both sides share the same K
    rho_g = rho_d.cpu().numpy().astype(np.float64)
    u_o, c_o, _ = to2d.fea(rho_g, f, fixed.astype(bool))
    assert res <= 1e-10 and it > 0
    assert abs(c - c_o) <= 1e-8 * abs(c_o)
    assert np.abs(u_d.cpu().numpy() - u_o).max() <= 1e-8 * np.abs(u_o).max()
    s_o = to2d.filter_sensitivity(xi.astype(np.float64), -to2d.compliance_sensitivity(rho_g, drho_o, u_o), 1.5)
    assert np.abs(s_d.cpu().numpy() - s_o).max() <= 1e-5 * np.abs(s_o).max()
    to.close()


def test_oc_update_matches_oracle():
    """The optimality-criteria update on the same xi and S: the same bisection, so the same
    multiplier and design (FP32 storage), the target volume reached, passive elements at 1."""
    binding = _need()
    f, fixed, fix, xi = _case(seed=1)
    nely, nelx = xi.shape
    S = np.random.default_rng(2).uniform(0.0, 1.0, xi.shape).astype(np.float32)
    to = binding.To2d(nelx, nely)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty(xi.shape, device="cuda")
    chg, vol = to.update(d(xi), d(S), d(fix), 0.45, out, move=0.2)
    x_o, lam, vol_o = to2d.oc_update(xi.astype(np.float64), S.astype(np.float64), 0.45, 2.0, fix != 0, 0.2)
    x = out.cpu().numpy()
    assert np.abs(x - x_o).max() <= 1e-6
    assert abs(vol - vol_o) <= 1e-7 and abs(vol - 0.45) <= 1e-6
    assert np.all(x[fix != 0] == 1.0)
    assert abs(chg - np.abs(x_o - xi)[fix == 0].mean()) <= 1e-6
    to.close()


def test_one_constrained_iteration_matches_oracle():
    """One iteration of Alg. 2 with the accessibility penalty (two planar tools, w_acc 0.5) from
    the same design: compliance as the oracle's; the new design equals the oracle's except at
    the few elements whose normalised IMF lies within the allowance band (the B / Gamma decision
    of Alg. 1 at lambda, where either side is correct)."""
    _need()
    from paper_2002_07627_gb300 import topopt
    nelx, nely = 64, 32
    f, fixed, fix, _ = _case(nelx, nely)
    xi0 = np.random.default_rng(5).uniform(0.2, 0.8, (nely, nelx)).astype(np.float32)
    xi0[fix != 0] = 1.0
    tools = synth.to2d_tools(4)
    g = topopt.run_to2d(nelx, nely, 0.5, tools, iters=1, delta=-1, xi0=xi0, cg_tol=1e-10)
    o = to2d.to_loop(xi0.astype(np.float64), f, fixed.astype(bool), fix, 0.5, tools, 1)
    assert abs(g.history[0]["compliance"] - o[0]["compliance"]) <= 1e-6 * o[0]["compliance"]
    diff = np.abs(g.xi - o[0]["xi"]) > 1e-4
    assert diff.mean() < 0.01, diff.sum()
    assert abs(g.history[0]["secluded"] - o[0]["secluded"]) <= max(3, 0.01 * o[0]["secluded"])


def test_accessibility_constraint_reduces_the_secluded_volume():
    """Over a short run on the 96 x 48 cantilever the accessibility-constrained optimisation
    (w_acc 0.5) ends with less secluded volume than the unconstrained one measured with the same
    tools (Sec. 3.1: the constraint removes the inaccessible regions at some cost in compliance),
    and both keep the volume fraction."""
    binding = _need()
    from paper_2002_07627_gb300 import topopt
    nelx, nely = 96, 48
    tools = synth.to2d_tools(8)
    con = topopt.run_to2d(nelx, nely, 0.5, tools, iters=30, delta=-1)
    unc = topopt.run_to2d(nelx, nely, 0.5, None, iters=30, delta=-1)
    _, _, fix = synth.cantilever2d(nelx, nely)
    imf = binding.Imf((1, nely, nelx))
    imf.set_tools(tools)
    r = torch.from_numpy(np.ascontiguousarray(unc.rho[None])).cuda()
    _, sec = imf.compute(r, torch.from_numpy(fix[None]).cuda())
    imf.sync()
    v_unc = int(sec.sum().item())
    v_con = con.history[-1]["secluded"]
    assert v_con < v_unc, (v_con, v_unc)
    for res in (con, unc):
        assert abs(res.history[-1]["vol"] - 0.5) < 1e-5
