"""Plain FP64 CPU oracle of the SIMP topology-optimisation loop around the IMF (Alg. 2 of
arXiv 2002.07627, Sec. 2.2) on a 2D grid of unit square elements.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): imported by `tests/` and by the
CPU legs of `bench.py`, never by the product path.

Steps, in the order of Alg. 2, each written from its definition:
  * Heaviside projection (Eq. eq_Heaviside): rho = 1 - exp(-beta xi) + xi exp(-beta);
  * FEA: bilinear four-node plane-stress elements, element stiffness by 2 x 2 Gauss quadrature
    of B^T D B over the unit square, SIMP modulus E(rho) = Emin + rho^p (E0 - Emin), global
    stiffness assembled as a sparse matrix and solved directly with the clamped dofs removed;
  * objective: compliance c = f^T u; its sensitivity with respect to the design variable,
    dc/dxi_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e * drho/dxi_e (the compliance is
    self-adjoint, Sec. 2.2);
  * S_phi = -dc/dxi >= 0, smoothed by a sensitivity filter with linear hat weights
    max(0, rmin - dist) (a "SIMP filtering" step of Alg. 2's Update; the filter weights the
    sensitivity by xi as in the usual mesh-independence filter);
  * optimality-criteria update of xi with a move limit and a bisection on the Lagrange
    multiplier of the volume constraint, evaluated on the projected density.
The load case (forces, clamped dofs, fixture) is an input, made by the seeded generators in
paper_2002_07627_gb300/synth.py (cantilever2d).
Node numbering: node (i, j) with i along x (0..nelx), j along y (0..nely) has index
j * (nelx + 1) + i and dofs (2 n, 2 n + 1) = (ux, uy); element (ex, ey) has corners
(ex, ey), (ex+1, ey), (ex+1, ey+1), (ex, ey+1) in that (counter-clockwise) order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def heaviside(xi, beta):
    """Eq. eq_Heaviside: rho = 1 - exp(-beta xi) + xi exp(-beta), and drho / dxi."""
    xi = np.asarray(xi, np.float64)
    rho = 1.0 - np.exp(-beta * xi) + xi * np.exp(-beta)
    drho = beta * np.exp(-beta * xi) + np.exp(-beta)
    return rho, drho


def element_stiffness(nu, E=1.0):
    """8 x 8 stiffness of a unit square bilinear plane-stress element, dof order (ux, uy) of
    corners (0,0), (1,0), (1,1), (0,1), by 2 x 2 Gauss quadrature of B^T D B."""
    D = E / (1.0 - nu * nu) * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]])
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    g = 0.5 / np.sqrt(3.0)
    k = np.zeros((8, 8))
    for s in (0.5 - g, 0.5 + g):
        for t in (0.5 - g, 0.5 + g):
            # bilinear shape functions N_a(s, t) = (1 +- ...) on [0, 1]^2 and their gradients
            dN = np.zeros((4, 2))
            for a, (xa, ya) in enumerate(corners):
                fx = s if xa == 1.0 else 1.0 - s
                fy = t if ya == 1.0 else 1.0 - t
                dfx = 1.0 if xa == 1.0 else -1.0
                dfy = 1.0 if ya == 1.0 else -1.0
                dN[a] = (dfx * fy, fx * dfy)
            B = np.zeros((3, 8))
            for a in range(4):
                B[0, 2 * a] = dN[a, 0]
                B[1, 2 * a + 1] = dN[a, 1]
                B[2, 2 * a] = dN[a, 1]
                B[2, 2 * a + 1] = dN[a, 0]
            k += 0.25 * B.T @ D @ B        # weight 1/4 per point on the unit square
    return k


def element_dofs(nelx, nely):
    """[nely][nelx][8] global dof indices of every element (corner order as in the module doc)."""
    ex, ey = np.meshgrid(np.arange(nelx), np.arange(nely))
    n = lambda i, j: j * (nelx + 1) + i
    nodes = np.stack([n(ex, ey), n(ex + 1, ey), n(ex + 1, ey + 1), n(ex, ey + 1)], -1)
    return np.stack([2 * nodes, 2 * nodes + 1], -1).reshape(nely, nelx, 8)


def fea(rho, force, fixed, nu=0.3, penal=3.0, E0=1.0, Emin=1e-3):
    """Displacements u ([2 (nelx+1)(nely+1)]) and compliance c = f^T u for element densities
    rho [nely][nelx]; `fixed` is a boolean dof mask (clamped dofs, u = 0)."""
    rho = np.asarray(rho, np.float64)
    nely, nelx = rho.shape
    ndof = 2 * (nelx + 1) * (nely + 1)
    k0 = element_stiffness(nu)
    Ee = Emin + rho ** penal * (E0 - Emin)
    edof = element_dofs(nelx, nely).reshape(-1, 8)
    rows = np.repeat(edof, 8, axis=1).ravel()
    cols = np.tile(edof, (1, 8)).ravel()
    vals = (Ee.ravel()[:, None, None] * k0[None]).reshape(-1)
    K = sp.coo_matrix((vals, (rows, cols)), shape=(ndof, ndof)).tocsc()
    free = ~np.asarray(fixed, bool)
    f = np.asarray(force, np.float64)
    u = np.zeros(ndof)
    u[free] = spla.spsolve(K[free][:, free], f[free])
    return u, float(f @ u), K


def compliance_sensitivity(rho, drho, u, nu=0.3, penal=3.0, E0=1.0, Emin=1e-3):
    """dc/dxi per element: -p rho^(p-1) (E0 - Emin) u_e^T k0 u_e times drho/dxi."""
    rho = np.asarray(rho, np.float64)
    nely, nelx = rho.shape
    k0 = element_stiffness(nu)
    ue = u[element_dofs(nelx, nely)]                      # [nely][nelx][8]
    ce = np.einsum("yxa,ab,yxb->yx", ue, k0, ue)
    return -penal * rho ** (penal - 1.0) * (E0 - Emin) * ce * drho


def filter_sensitivity(xi, s, rmin):
    """Mesh-independence filter of the sensitivity s with hat weights H_ef = max(0, rmin - |e - f|)
    over element centres: s_e <- sum_f H_ef xi_f s_f / (max(1e-3, xi_e) sum_f H_ef)."""
    xi = np.asarray(xi, np.float64)
    nely, nelx = xi.shape
    r = int(np.ceil(rmin)) - 1
    num = np.zeros_like(xi)
    den = np.zeros_like(xi)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            w = max(0.0, rmin - np.hypot(dx, dy))
            if w == 0.0:
                continue
            # neighbour f = e + (dx, dy), inside the grid
            ys = slice(max(0, -dy), nely - max(0, dy))
            xs = slice(max(0, -dx), nelx - max(0, dx))
            yn = slice(max(0, dy), nely - max(0, -dy))
            xn = slice(max(0, dx), nelx - max(0, -dx))
            num[ys, xs] += w * xi[yn, xn] * s[yn, xn]
            den[ys, xs] += w
    return num / (np.maximum(1e-3, xi) * den)


def oc_update(xi, S, volfrac, beta, passive=None, move=0.2, eta=0.5, tol=1e-9):
    """Optimality-criteria update: xi_new = clamp(xi * (S / lam)^eta) within the move limit
    and [0, 1], with lam found by bisection so that the mean projected density (Eq.
    eq_Heaviside) of the free elements equals volfrac. S >= 0 is the (penalised) sensitivity;
    passive elements (fixture) keep xi = 1. Returns (xi_new, lam, mean projected density)."""
    xi = np.asarray(xi, np.float64)
    S = np.maximum(np.asarray(S, np.float64), 0.0)
    free = np.ones(xi.shape, bool) if passive is None else ~np.asarray(passive, bool)

    def new_xi(lam):
        x = xi * (S / lam) ** eta
        x = np.clip(x, np.maximum(0.0, xi - move), np.minimum(1.0, xi + move))
        return np.where(free, x, 1.0)

    lo, hi = 1e-12, 1e12
    while hi / lo > 1.0 + tol:
        mid = np.sqrt(lo * hi)
        vol = heaviside(new_xi(mid), beta)[0][free].mean()
        if vol > volfrac:
            lo = mid
        else:
            hi = mid
    lam = np.sqrt(lo * hi)
    x = new_xi(lam)
    return x, lam, float(heaviside(x, beta)[0][free].mean())


def to_loop(xi0, force, fixed, fixture, volfrac, tools, iters, w_acc=0.5, beta=2.0, nu=0.3, penal=3.0, Emin=1e-3,
            rmin=1.5, move=0.2, eta=0.5, lam=0.01, tau=0.5, theta_rel=0.01):
    """Alg. 2 with the oracle's IMF (oracle.imf) and penalty (oracle.penalize): returns the list
    of per-iteration records (compliance, secluded voxels, change, xi after the update)."""
    from . import ref
    from paper_2002_07627_gb300.synth import Design
    xi = np.asarray(xi0, np.float64).copy()
    out = []
    for _ in range(iters):
        rho, drho = heaviside(xi, beta)
        u, c, _ = fea(rho, force, fixed, nu, penal, 1.0, Emin)
        s = -compliance_sensitivity(rho, drho, u, nu, penal, 1.0, Emin)
        s = filter_sensitivity(xi, s, rmin)
        sec_n = 0
        if tools:
            r = ref.imf(Design(rho[None].astype(np.float32), fixture[None], tools), lam, tau, theta_rel)
            s = ref.penalize(s[None], rho[None], r["fbar"], r["secluded"], fixture[None], w_acc, tau)[0]
            sec_n = int(r["secluded"].sum())
        xi_new, _, vol = oc_update(xi, s, volfrac, beta, fixture != 0, move, eta)
        free = fixture == 0
        out.append({"compliance": c, "secluded": sec_n, "change": float(np.abs(xi_new - xi)[free].mean()), "vol": vol,
                    "xi": xi_new.copy()})
        xi = xi_new
    return out
