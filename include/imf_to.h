/*
 * libimf, topology-optimisation loop around the IMF (Alg. 2 of arXiv 2002.07627, Sec. 2.2):
 * the density-based (SIMP) steps a caller needs between two IMF evaluations, on one GPU, for a
 * 2D grid of unit square elements (the IMF grid with nz = 1, element (ex, ey) at index
 * ey * nelx + ex).
 *
 *   Heaviside projection (Eq. eq_Heaviside): rho = 1 - exp(-beta xi) + xi exp(-beta);
 *   FEA: bilinear four-node plane-stress elements, SIMP modulus E(rho) = Emin + rho^p (E0 - Emin),
 *        K(rho) u = f solved by a matrix-free Jacobi-preconditioned conjugate gradient in FP64;
 *   compliance c = f^T u and its sensitivity to xi (self-adjoint, Sec. 2.2), smoothed by a
 *        mesh-independence filter (hat weights max(0, rmin - distance));
 *   optimality-criteria update of xi with a move limit and the volume constraint on the
 *        projected density (Alg. 2's Update), driven by the penalised sensitivity S of
 *        Eq. eq_filtered_sens (imf_penalize_sensitivity computes S from S_phi).
 *
 * Nodes: node (i, j), i = 0..nelx, j = 0..nely, has index j (nelx + 1) + i and dofs 2 n (x) and
 * 2 n + 1 (y); element (ex, ey) has corners (ex, ey), (ex+1, ey), (ex+1, ey+1), (ex, ey+1).
 * The caller owns every array (device memory unless stated); the handle owns its solver
 * vectors. Calls marked synchronous wait for the stream; the others are asynchronous.
 */
#ifndef IMF_TO_H
#define IMF_TO_H

#include <stddef.h>
#include <stdint.h>

#include "imf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct imf_to2d_s *imf_to2d;

typedef struct {
    int nelx, nely;          /* elements along x and y                                        */
    double E0, Emin;         /* Young's modulus of solid and void (Emin > 0 keeps K regular)  */
    double nu;               /* Poisson ratio (0.3 in Sec. 3.1)                               */
    double penal;            /* SIMP exponent p                                               */
    double beta;             /* Heaviside sharpness (2 in 2D, 8 in 3D, Sec. 2.2)              */
    double rmin;             /* sensitivity filter radius in elements (> 1)                   */
    double cg_tol;           /* stop when |r| <= cg_tol |f| (free dofs)                        */
    int cg_max_iter;         /* iteration cap of the conjugate gradient                      */
} imf_to2d_options;

/* Defaults: E0 = 1, Emin = 1e-3, nu = 0.3, penal = 3, beta = 2, rmin = 1.5, cg_tol = 1e-8,
 * cg_max_iter = 20000 (grid 0 x 0, which imf_to2d_create rejects). */
void imf_to2d_default_options(imf_to2d_options *opt);

/* Allocates the solver vectors. Errors: IMF_ERR_INVALID_ARG, IMF_ERR_OOM. */
imf_status imf_to2d_create(const imf_to2d_options *opt, imf_to2d *out);
void imf_to2d_destroy(imf_to2d h);
const char *imf_to2d_last_error(imf_to2d h);

/* Eq. eq_Heaviside on DEVICE float [nely][nelx] arrays (rho may alias xi). Asynchronous. */
imf_status imf_to2d_project(imf_to2d h, const float *xi, float *rho, void *cuda_stream);

/* FEA of the design rho (DEVICE float [nely][nelx]) under the DEVICE FP64 load `force`
 * [2 (nelx+1)(nely+1)] with the DEVICE uint8 dof mask `fixed` (nonzero = clamped, u = 0).
 * Keeps u in the handle (for imf_to2d_sensitivity) and copies it to `u_out` (DEVICE FP64, or
 * NULL). Synchronous: the host checks the residual every few iterations. Compliance, iteration
 * count and relative residual via imf_to2d_result. Errors: IMF_ERR_INVALID_ARG,
 * IMF_ERR_CUDA; IMF_ERR_TIMEOUT when cg_max_iter is reached before cg_tol (u is the last
 * iterate). */
imf_status imf_to2d_analyze(imf_to2d h, const float *rho, const double *force, const uint8_t *fixed, double *u_out,
                            void *cuda_stream);

/* Compliance sensitivity of the last analysis with respect to xi, as the non-negative field
 * S_phi = -dc/dxi (-dc/drho times the Heaviside derivative at xi), filtered; DEVICE float
 * [nely][nelx] out. Asynchronous. */
imf_status imf_to2d_sensitivity(imf_to2d h, const float *xi, const float *rho, float *sens, void *cuda_stream);

/* Optimality-criteria update xi_new = clamp(xi (S / lam)^eta) within [xi - move, xi + move] and
 * [0, 1], lam by bisection so that the mean projected density of the non-passive elements is
 * volfrac; passive elements (DEVICE uint8, or NULL) keep xi = 1. S: DEVICE float, >= 0.
 * change_out (HOST, or NULL) receives the mean |xi_new - xi| over the non-passive elements
 * (Alg. 2's volume difference), vol_out (HOST, or NULL) the mean projected density reached.
 * Synchronous (bisection on the host, one volume reduction per step).
 * Errors: IMF_ERR_INVALID_ARG (NULL, volfrac outside (0, 1), move <= 0), IMF_ERR_CUDA. */
imf_status imf_to2d_update(imf_to2d h, const float *xi, const float *S, const uint8_t *passive, double volfrac,
                           double move, double eta, float *xi_new, double *change_out, double *vol_out,
                           void *cuda_stream);

/* Results of the last imf_to2d_analyze (HOST outputs, any may be NULL). */
imf_status imf_to2d_result(imf_to2d h, double *compliance, int *cg_iters, double *cg_rel_residual);

#ifdef __cplusplus
}
#endif

#endif /* IMF_TO_H */
