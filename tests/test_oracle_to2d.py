"""Pins of the topology-optimisation oracle (oracle/to2d.py; Alg. 2, Eq. eq_Heaviside) against
facts fixed by mechanics and calculus, not by the oracle itself: the element matrix's rigid-body
null space and constant-strain energy, a plate under uniform tension reproduced exactly, a
cantilever against Timoshenko beam theory, compliance sensitivities against finite
differences, and the optimality-criteria update's constraints."""
import numpy as np
import pytest

from oracle import to2d
from paper_2002_07627_gb300 import synth


def test_heaviside_closed_form_and_derivative():
    """rho(0) = 0 and rho(1) = 1 for any beta, monotone, and drho/dxi equals a central finite
    difference (Eq. eq_Heaviside)."""
    for beta in (2.0, 8.0):
        r, _ = to2d.heaviside(np.array([0.0, 1.0]), beta)
        assert abs(r[0]) < 1e-15 and abs(r[1] - 1.0) < 1e-15
        x = np.linspace(0.01, 0.99, 50)
        r, d = to2d.heaviside(x, beta)
        assert np.all(np.diff(r) > 0)
        h = 1e-6
        fd = (to2d.heaviside(x + h, beta)[0] - to2d.heaviside(x - h, beta)[0]) / (2 * h)
        assert np.abs(fd - d).max() < 1e-7


def test_element_matrix_rigid_modes_and_constant_strain():
    """The unit-square element matrix is symmetric positive semi-definite with exactly the three
    rigid-body motions (two translations, one rotation) as null space, and a constant strain
    stores exactly 1/2 eps^T D eps (area 1)."""
    nu = 0.3
    k = to2d.element_stiffness(nu)
    assert np.abs(k - k.T).max() < 1e-15
    ev = np.linalg.eigvalsh(k)
    assert np.sum(np.abs(ev) < 1e-12) == 3 and ev.min() > -1e-12
    corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    for mode in ([1, 0], [0, 1], None):
        u = np.zeros(8)
        for a, (x, y) in enumerate(corners):
            u[2 * a:2 * a + 2] = mode if mode is not None else (-(y - 0.5), x - 0.5)
        assert np.abs(k @ u).max() < 1e-14
    D = 1 / (1 - nu * nu) * np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])
    eps = np.array([1e-3, -2e-3, 5e-4])
    u = np.zeros(8)
    for a, (x, y) in enumerate(corners):
        u[2 * a] = eps[0] * x + 0.5 * eps[2] * y
        u[2 * a + 1] = eps[1] * y + 0.5 * eps[2] * x
    assert abs(0.5 * u @ k @ u - 0.5 * eps @ D @ eps) < 1e-18


def test_plate_under_uniform_tension_is_exact():
    """A plate (10 x 4 elements, E = 1) with the left edge on rollers (ux = 0), the bottom-left
    node pinned and a uniform traction 1 on the right edge: plane stress gives ux = x and
    uy = -nu y exactly, which bilinear elements reproduce to round-off; it pins the node
    numbering, the dof order and the assembly."""
    nelx, nely, nu = 10, 4, 0.3
    ndof = 2 * (nelx + 1) * (nely + 1)
    f = np.zeros(ndof)
    fixed = np.zeros(ndof, bool)
    for j in range(nely + 1):
        n0 = j * (nelx + 1)
        fixed[2 * n0] = True
        nr = n0 + nelx
        f[2 * nr] = 0.5 if j in (0, nely) else 1.0
    fixed[1] = True
    rho = np.ones((nely, nelx))
    u, c, K = to2d.fea(rho, f, fixed, nu=nu, penal=3.0, E0=1.0, Emin=1e-3)
    i, j = np.meshgrid(np.arange(nelx + 1), np.arange(nely + 1))
    assert np.abs(u[0::2] - i.ravel()).max() < 1e-9
    assert np.abs(u[1::2] + nu * j.ravel()).max() < 1e-9
    assert abs(c - u @ (K @ u)) < 1e-9 * c


def test_cantilever_against_timoshenko_beam():
    """The solid cantilever (64 x 16, tip load 1 at mid-height): the load-point deflection (the
    compliance) lies within 10 % below Timoshenko's P L^3 / (3 E I) + P L / (kappa G A) (bilinear
    elements are slightly stiff in bending)."""
    nelx, nely, nu = 64, 16, 0.3
    f, fixed, fix = synth.cantilever2d(nelx, nely, fixture_cols=0)
    u, c, _ = to2d.fea(np.ones((nely, nelx)), f, fixed.astype(bool), nu=nu)
    E, L, H = 1.0, float(nelx), float(nely)
    I, A, G, kappa = H ** 3 / 12.0, H, E / (2 * (1 + nu)), 5.0 / 6.0
    delta = L ** 3 / (3 * E * I) + L / (kappa * G * A)
    assert 0.9 * delta < c < delta


def test_compliance_sensitivity_matches_finite_differences():
    """dc/dxi of the oracle (self-adjoint compliance, Heaviside chain rule) equals a central
    finite difference of the compliance in each design variable."""
    rng = np.random.default_rng(3)
    nelx, nely, beta = 8, 5, 2.0
    f, fixed, _ = synth.cantilever2d(nelx, nely, fixture_cols=0)
    fixed = fixed.astype(bool)
    xi = rng.uniform(0.2, 0.9, (nely, nelx))

    def comp(x):
        return to2d.fea(to2d.heaviside(x, beta)[0], f, fixed)[1]

    rho, drho = to2d.heaviside(xi, beta)
    u, c, _ = to2d.fea(rho, f, fixed)
    dc = to2d.compliance_sensitivity(rho, drho, u)
    h = 1e-6
    for (y, x) in [(0, 0), (2, 3), (4, 7), (1, 5)]:
        xp, xm = xi.copy(), xi.copy()
        xp[y, x] += h
        xm[y, x] -= h
        fd = (comp(xp) - comp(xm)) / (2 * h)
        assert abs(fd - dc[y, x]) <= 1e-5 * abs(dc).max(), (y, x, fd, dc[y, x])


def test_filter_keeps_uniform_fields_and_weights_neighbours():
    """The sensitivity filter returns a uniform field unchanged, and a single spike spreads to
    its 3 x 3 neighbours with the hat weights max(0, rmin - distance) (rmin = 1.5)."""
    xi = np.full((6, 7), 0.5)
    s = np.full((6, 7), 2.0)
    assert np.abs(to2d.filter_sensitivity(xi, s, 1.5) - 2.0).max() < 1e-14
    s = np.zeros((6, 7))
    s[3, 3] = 1.0
    out = to2d.filter_sensitivity(np.ones((6, 7)), s, 1.5)
    wsum = 1.5 + 4 * 0.5 + 4 * (1.5 - np.sqrt(2))
    assert abs(out[3, 4] - 0.5 / wsum) < 1e-14 and abs(out[2, 2] - (1.5 - np.sqrt(2)) / wsum) < 1e-14
    assert out[3, 5] == 0.0


def test_oc_update_meets_its_constraints():
    """The update reaches a reachable target mean projected density (bisection tolerance),
    stays within the move limit and [0, 1], keeps passive elements at 1, and with a uniform S
    every free element moves by the same factor."""
    rng = np.random.default_rng(4)
    xi = rng.uniform(0.1, 0.9, (9, 12))
    S = rng.uniform(0.0, 2.0, xi.shape)
    passive = np.zeros(xi.shape, bool)
    passive[:, :2] = True
    x, lam, vol = to2d.oc_update(xi, S, 0.55, 2.0, passive, move=0.2)
    assert abs(vol - 0.55) < 1e-6
    assert np.all(x[passive] == 1.0)
    free = ~passive
    assert np.all(np.abs(x - xi)[free] <= 0.2 + 1e-12) and x.min() >= 0 and x.max() <= 1
    xu = np.full((5, 6), 0.3)
    x, _, vol = to2d.oc_update(xu, np.ones(xu.shape), 0.32, 2.0, None, move=0.5)
    assert np.ptp(x) < 1e-12 and abs(vol - 0.32) < 1e-6
