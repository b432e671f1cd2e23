// The SIMP steps of the topology-optimisation loop around the IMF (Alg. 2; include/imf_to.h):
// Heaviside projection, matrix-free FEA with a Jacobi-preconditioned conjugate gradient (FP64),
// compliance sensitivity with its filter, and the optimality-criteria update.
//
// The stiffness operator is applied node by node: a node gathers the contributions of its (up
// to four) elements, E_e times the rows of the element matrix k0 that belong to its corner, so
// no atomics are needed. The conjugate gradient keeps its scalars on the device (rotating slots,
// so that a kernel never reads a slot another block of the same launch is resetting); the host
// only reads the residual every few iterations to decide when to stop.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "imf_to.h"

namespace {

constexpr int kT = 256;
constexpr int kCheckEvery = 16;      // CG iterations between residual checks on the host

// scalar slots: rz[3], pq[2], rr[3], ff, vol, cnt, change
enum { S_RZ = 0, S_PQ = 3, S_RR = 5, S_FF = 8, S_VOL = 9, S_CNT = 10, S_CHG = 11, S_N = 16 };

inline int blocks(long n, int cap = 152 * 8)
{
    long b = (n + kT - 1) / kT;
    return (int)(b < 1 ? 1 : b > cap ? cap : b);
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[kT / 32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kT / 32; ++i) t += red[i];
    __syncthreads();
    return t;   // valid in thread 0
}

struct Grid {
    int nelx, nely;
    __device__ __forceinline__ int nx1() const { return nelx + 1; }
};

// ---------------------------------------------------------------------------------------
// Eq. eq_Heaviside
// ---------------------------------------------------------------------------------------
__global__ void heaviside_kernel(const float *xi, float *rho, long n, double beta)
{
    const double eb = exp(-beta);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double x = xi[i];
        rho[i] = (float)(1.0 - exp(-beta * x) + x * eb);
    }
}

// E_e = Emin + rho^p (E0 - Emin)
__global__ void moduli_kernel(const float *rho, double *E, long n, double E0, double Emin, double p)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        E[i] = Emin + pow((double)rho[i], p) * (E0 - Emin);
}

// the element matrix row of corner a, component d, applied to the element's displacements
__device__ __forceinline__ double krow(const double *k0, int a, int d, const double *ue)
{
    const double *row = k0 + (2 * a + d) * 8;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 8; ++b) s += row[b] * ue[b];
    return s;
}

// gather of element (ex, ey)'s corner displacements from v
__device__ __forceinline__ void gather(const double *v, int nx1, int ex, int ey, double *ue)
{
    const int n0 = ey * nx1 + ex, n1 = n0 + 1, n2 = n0 + nx1 + 1, n3 = n0 + nx1;
    ue[0] = v[2 * n0]; ue[1] = v[2 * n0 + 1];
    ue[2] = v[2 * n1]; ue[3] = v[2 * n1 + 1];
    ue[4] = v[2 * n2]; ue[5] = v[2 * n2 + 1];
    ue[6] = v[2 * n3]; ue[7] = v[2 * n3 + 1];
}

// (K v) at node (i, j), both components; the node is corner 2 of element (i-1, j-1), 3 of
// (i, j-1), 1 of (i-1, j) and 0 of (i, j)
__device__ __forceinline__ void apply_node(const Grid g, const double *k0, const double *E, const double *v, int i, int j,
                                           double &qx, double &qy)
{
    qx = qy = 0.0;
    const int ex[4] = {i - 1, i, i - 1, i}, ey[4] = {j - 1, j - 1, j, j}, corner[4] = {2, 3, 1, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (ex[k] < 0 || ey[k] < 0 || ex[k] >= g.nelx || ey[k] >= g.nely) continue;
        double ue[8];
        gather(v, g.nx1(), ex[k], ey[k], ue);
        const double Ee = E[(long)ey[k] * g.nelx + ex[k]];
        qx += Ee * krow(k0, corner[k], 0, ue);
        qy += Ee * krow(k0, corner[k], 1, ue);
    }
}

__global__ void diag_kernel(const Grid g, const double *k0, const double *E, const uint8_t *fixed, double *diag)
{
    const long nn = (long)(g.nelx + 1) * (g.nely + 1);
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < nn; n += (long)gridDim.x * blockDim.x) {
        const int i = (int)(n % (g.nelx + 1)), j = (int)(n / (g.nelx + 1));
        const int ex[4] = {i - 1, i, i - 1, i}, ey[4] = {j - 1, j - 1, j, j}, corner[4] = {2, 3, 1, 0};
        double dx = 0.0, dy = 0.0;
        for (int k = 0; k < 4; ++k) {
            if (ex[k] < 0 || ey[k] < 0 || ex[k] >= g.nelx || ey[k] >= g.nely) continue;
            const double Ee = E[(long)ey[k] * g.nelx + ex[k]];
            dx += Ee * k0[(2 * corner[k]) * 8 + 2 * corner[k]];
            dy += Ee * k0[(2 * corner[k] + 1) * 8 + 2 * corner[k] + 1];
        }
        diag[2 * n] = fixed[2 * n] ? 1.0 : dx;
        diag[2 * n + 1] = fixed[2 * n + 1] ? 1.0 : dy;
    }
}

// x = 0, r = f (free dofs), z = r / diag, p = z; rz -> slot 0, rr -> slot 0, ff
__global__ void cg_init_kernel(long ndof, const double *f, const uint8_t *fixed, const double *diag, double *x, double *r,
                               double *z, double *p, double *sc)
{
    double rz = 0.0, rr = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ndof; i += (long)gridDim.x * blockDim.x) {
        const double ri = fixed[i] ? 0.0 : f[i];
        const double zi = ri / diag[i];
        x[i] = 0.0;
        r[i] = ri;
        z[i] = zi;
        p[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    rz = block_sum(rz);
    rr = block_sum(rr);
    if (threadIdx.x == 0) {
        atomicAdd(sc + S_RZ, rz);
        atomicAdd(sc + S_RR, rr);
        atomicAdd(sc + S_FF, rr);
    }
}

// q = K p on the free dofs (0 on clamped ones), p . q -> pq slot
__global__ void cg_matvec_kernel(const Grid g, const double *k0, const double *E, const uint8_t *fixed, const double *p,
                                 double *q, double *pq)
{
    const long nn = (long)(g.nelx + 1) * (g.nely + 1);
    double s = 0.0;
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < nn; n += (long)gridDim.x * blockDim.x) {
        const int i = (int)(n % (g.nelx + 1)), j = (int)(n / (g.nelx + 1));
        double qx, qy;
        apply_node(g, k0, E, p, i, j, qx, qy);
        if (fixed[2 * n]) qx = 0.0;
        if (fixed[2 * n + 1]) qy = 0.0;
        q[2 * n] = qx;
        q[2 * n + 1] = qy;
        s += p[2 * n] * qx + p[2 * n + 1] * qy;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(pq, s);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = r / diag; r . z and r . r -> next slots
__global__ void cg_update_xr_kernel(long ndof, const double *diag, const double *p, const double *q, double *x, double *r,
                                    double *z, const double *rz_cur, const double *pq, double *rz_next, double *rr_next)
{
    const double alpha = *rz_cur / *pq;
    double rz = 0.0, rr = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ndof; i += (long)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        const double zi = ri / diag[i];
        r[i] = ri;
        z[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    rz = block_sum(rz);
    rr = block_sum(rr);
    if (threadIdx.x == 0) {
        atomicAdd(rz_next, rz);
        atomicAdd(rr_next, rr);
    }
}

// beta = rz_next / rz_cur; p = z + beta p; block 0 clears the slots the next iteration fills
__global__ void cg_update_p_kernel(long ndof, const double *z, double *p, const double *rz_cur, const double *rz_next,
                                   double *clear_pq, double *clear_rz, double *clear_rr)
{
    const double beta = *rz_next / *rz_cur;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ndof; i += (long)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *clear_pq = 0.0;
        *clear_rz = 0.0;
        *clear_rr = 0.0;
    }
}

// S_phi = p rho^(p-1) (E0 - Emin) u_e^T k0 u_e * drho/dxi  (= -dc/dxi)
__global__ void sens_kernel(const Grid g, const double *k0, const double *u, const float *xi, const float *rho, double p,
                            double dE, double beta, double *s)
{
    const long ne = (long)g.nelx * g.nely;
    const double eb = exp(-beta);
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ne; e += (long)gridDim.x * blockDim.x) {
        const int ex = (int)(e % g.nelx), ey = (int)(e / g.nelx);
        double ue[8];
        gather(u, g.nx1(), ex, ey, ue);
        double ce = 0.0;
        for (int a = 0; a < 8; ++a) {
            double ka = 0.0;
            for (int b = 0; b < 8; ++b) ka += k0[a * 8 + b] * ue[b];
            ce += ue[a] * ka;
        }
        const double x = xi[e];
        const double drho = beta * exp(-beta * x) + eb;
        s[e] = p * pow((double)rho[e], p - 1.0) * dE * ce * drho;
    }
}

// s_e <- sum_f H_ef xi_f s_f / (max(1e-3, xi_e) sum_f H_ef), H_ef = max(0, rmin - |e - f|)
__global__ void filter_kernel(const Grid g, const float *xi, const double *s, double rmin, float *out)
{
    const long ne = (long)g.nelx * g.nely;
    const int r = (int)ceil(rmin) - 1;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ne; e += (long)gridDim.x * blockDim.x) {
        const int ex = (int)(e % g.nelx), ey = (int)(e / g.nelx);
        double num = 0.0, den = 0.0;
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                const double w = rmin - sqrt((double)(dx * dx + dy * dy));
                const int fx = ex + dx, fy = ey + dy;
                if (w <= 0.0 || fx < 0 || fy < 0 || fx >= g.nelx || fy >= g.nely) continue;
                const long f = (long)fy * g.nelx + fx;
                num += w * (double)xi[f] * s[f];
                den += w;
            }
        out[e] = (float)(num / (fmax(1e-3, (double)xi[e]) * den));
    }
}

__device__ __forceinline__ double oc_new(double x, double S, double lam, double move, double eta)
{
    double v = x * pow(fmax(S, 0.0) / lam, eta);
    v = fmin(v, fmin(1.0, x + move));
    v = fmax(v, fmax(0.0, x - move));
    return v;
}

// sum over the free elements of the projected density of the candidate update at lam (and
// their count); with `out`, also writes xi_new and sums |xi_new - xi|
__global__ void oc_kernel(long n, const float *xi, const float *S, const uint8_t *passive, double lam, double move,
                          double eta, double beta, double *sc, float *out)
{
    const double eb = exp(-beta);
    double vol = 0.0, cnt = 0.0, chg = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const bool pas = passive && passive[i];
        const double x = xi[i];
        const double v = pas ? 1.0 : oc_new(x, S[i], lam, move, eta);
        if (out) out[i] = (float)v;
        if (pas) continue;
        vol += 1.0 - exp(-beta * v) + v * eb;
        cnt += 1.0;
        chg += fabs(v - x);
    }
    vol = block_sum(vol);
    cnt = block_sum(cnt);
    chg = block_sum(chg);
    if (threadIdx.x == 0) {
        atomicAdd(sc + S_VOL, vol);
        atomicAdd(sc + S_CNT, cnt);
        if (out) atomicAdd(sc + S_CHG, chg);
    }
}

// 8 x 8 unit-square plane-stress element matrix by 2 x 2 Gauss quadrature of B^T D B (corner
// order (0,0), (1,0), (1,1), (0,1); dofs (ux, uy) per corner), E = 1
void element_matrix(double nu, double *k)
{
    const double c = 1.0 / (1.0 - nu * nu);
    const double D[3][3] = {{c, c * nu, 0.0}, {c * nu, c, 0.0}, {0.0, 0.0, c * (1.0 - nu) / 2.0}};
    const int cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
    const double g = 0.5 / std::sqrt(3.0), pts[2] = {0.5 - g, 0.5 + g};
    for (int i = 0; i < 64; ++i) k[i] = 0.0;
    for (double s : pts)
        for (double t : pts) {
            double B[3][8] = {{0}};
            for (int a = 0; a < 4; ++a) {
                const double fx = cx[a] ? s : 1.0 - s, fy = cy[a] ? t : 1.0 - t;
                const double dfx = cx[a] ? 1.0 : -1.0, dfy = cy[a] ? 1.0 : -1.0;
                const double nxd = dfx * fy, nyd = fx * dfy;
                B[0][2 * a] = nxd;
                B[1][2 * a + 1] = nyd;
                B[2][2 * a] = nyd;
                B[2][2 * a + 1] = nxd;
            }
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) {
                    double v = 0.0;
                    for (int m = 0; m < 3; ++m)
                        for (int q = 0; q < 3; ++q) v += B[m][i] * D[m][q] * B[q][j];
                    k[i * 8 + j] += 0.25 * v;
                }
        }
}

} // namespace

struct imf_to2d_s {
    imf_to2d_options opt{};
    std::string err;
    long ne = 0, ndof = 0;
    double *k0 = nullptr, *E = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
           *diag = nullptr, *sc = nullptr, *s = nullptr;
    double compliance = 0.0, rel_res = 0.0;
    int iters = 0;
    bool have_u = false;
};

namespace {

imf_status fail(imf_to2d h, imf_status st, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

#define TO_CU(call)                                                                                                \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return fail(h, IMF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));               \
    } while (0)

} // namespace

extern "C" {

void imf_to2d_default_options(imf_to2d_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->E0 = 1.0;
    o->Emin = 1e-3;
    o->nu = 0.3;
    o->penal = 3.0;
    o->beta = 2.0;
    o->rmin = 1.5;
    o->cg_tol = 1e-8;
    o->cg_max_iter = 20000;
}

imf_status imf_to2d_create(const imf_to2d_options *o, imf_to2d *out)
{
    if (!o || !out) return IMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (o->nelx < 1 || o->nely < 1 || (long)o->nelx * o->nely > (1L << 28) || !(o->E0 > 0) || !(o->Emin > 0) ||
        !(o->Emin < o->E0) || !(o->nu > -1.0 && o->nu < 0.5) || !(o->penal >= 1.0) || !(o->beta > 0) ||
        !(o->rmin > 1.0) || !(o->cg_tol > 0) || o->cg_max_iter < 1)
        return IMF_ERR_INVALID_ARG;
    imf_to2d h = new (std::nothrow) imf_to2d_s();
    if (!h) return IMF_ERR_OOM;
    h->opt = *o;
    h->ne = (long)o->nelx * o->nely;
    h->ndof = 2L * (o->nelx + 1) * (o->nely + 1);
    double k[64];
    element_matrix(o->nu, k);
    bool ok = cudaMalloc(&h->k0, 64 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&h->E, h->ne * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&h->s, h->ne * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&h->sc, S_N * sizeof(double)) == cudaSuccess;
    for (double **v : {&h->x, &h->r, &h->z, &h->p, &h->q, &h->diag})
        ok = ok && cudaMalloc(v, h->ndof * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemcpy(h->k0, k, sizeof k, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        imf_to2d_destroy(h);
        return IMF_ERR_OOM;
    }
    *out = h;
    return IMF_OK;
}

void imf_to2d_destroy(imf_to2d h)
{
    if (!h) return;
    for (double *v : {h->k0, h->E, h->x, h->r, h->z, h->p, h->q, h->diag, h->sc, h->s}) cudaFree(v);
    delete h;
}

const char *imf_to2d_last_error(imf_to2d h) { return h ? h->err.c_str() : "null handle"; }

imf_status imf_to2d_project(imf_to2d h, const float *xi, float *rho, void *stream)
{
    if (!h || !xi || !rho) return fail(h, IMF_ERR_INVALID_ARG, "NULL argument");
    heaviside_kernel<<<blocks(h->ne), kT, 0, (cudaStream_t)stream>>>(xi, rho, h->ne, h->opt.beta);
    TO_CU(cudaGetLastError());
    return IMF_OK;
}

imf_status imf_to2d_analyze(imf_to2d h, const float *rho, const double *force, const uint8_t *fixed, double *u_out,
                            void *stream)
{
    if (!h || !rho || !force || !fixed) return fail(h, IMF_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const imf_to2d_options &o = h->opt;
    const Grid g{o.nelx, o.nely};
    const long nn = (long)(o.nelx + 1) * (o.nely + 1);
    moduli_kernel<<<blocks(h->ne), kT, 0, s>>>(rho, h->E, h->ne, o.E0, o.Emin, o.penal);
    diag_kernel<<<blocks(nn), kT, 0, s>>>(g, h->k0, h->E, fixed, h->diag);
    TO_CU(cudaMemsetAsync(h->sc, 0, S_N * sizeof(double), s));
    cg_init_kernel<<<blocks(h->ndof), kT, 0, s>>>(h->ndof, force, fixed, h->diag, h->x, h->r, h->z, h->p, h->sc);
    double ff = 0.0, rr = 0.0;
    TO_CU(cudaMemcpyAsync(&ff, h->sc + S_FF, sizeof ff, cudaMemcpyDeviceToHost, s));
    TO_CU(cudaStreamSynchronize(s));
    const double stop2 = o.cg_tol * o.cg_tol * ff;
    int it = 0;
    bool done = ff == 0.0;
    while (!done && it < o.cg_max_iter) {
        double *sc = h->sc;
        cg_matvec_kernel<<<blocks(nn), kT, 0, s>>>(g, h->k0, h->E, fixed, h->p, h->q, sc + S_PQ + it % 2);
        cg_update_xr_kernel<<<blocks(h->ndof), kT, 0, s>>>(h->ndof, h->diag, h->p, h->q, h->x, h->r, h->z,
                                                           sc + S_RZ + it % 3, sc + S_PQ + it % 2,
                                                           sc + S_RZ + (it + 1) % 3, sc + S_RR + (it + 1) % 3);
        cg_update_p_kernel<<<blocks(h->ndof), kT, 0, s>>>(h->ndof, h->z, h->p, sc + S_RZ + it % 3,
                                                          sc + S_RZ + (it + 1) % 3, sc + S_PQ + (it + 1) % 2,
                                                          sc + S_RZ + (it + 2) % 3, sc + S_RR + (it + 2) % 3);
        ++it;
        if (it % kCheckEvery == 0 || it == o.cg_max_iter) {
            TO_CU(cudaMemcpyAsync(&rr, sc + S_RR + it % 3, sizeof rr, cudaMemcpyDeviceToHost, s));
            TO_CU(cudaStreamSynchronize(s));
            done = rr <= stop2;
        }
    }
    TO_CU(cudaGetLastError());
    if (u_out) TO_CU(cudaMemcpyAsync(u_out, h->x, h->ndof * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // compliance c = f^T u on the host from one copy (a small vector)
    std::vector<double> u(h->ndof), f(h->ndof);
    TO_CU(cudaMemcpyAsync(u.data(), h->x, h->ndof * sizeof(double), cudaMemcpyDeviceToHost, s));
    TO_CU(cudaMemcpyAsync(f.data(), force, h->ndof * sizeof(double), cudaMemcpyDeviceToHost, s));
    TO_CU(cudaStreamSynchronize(s));
    double c = 0.0;
    for (long i = 0; i < h->ndof; ++i) c += f[i] * u[i];
    h->compliance = c;
    h->iters = it;
    h->rel_res = ff > 0 ? std::sqrt(rr / ff) : 0.0;
    h->have_u = true;
    if (!done) return fail(h, IMF_ERR_TIMEOUT, "conjugate gradient: %d iterations, relative residual %g", it, h->rel_res);
    return IMF_OK;
}

imf_status imf_to2d_sensitivity(imf_to2d h, const float *xi, const float *rho, float *sens, void *stream)
{
    if (!h || !xi || !rho || !sens) return fail(h, IMF_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_u) return fail(h, IMF_ERR_NOT_READY, "imf_to2d_sensitivity before imf_to2d_analyze");
    cudaStream_t s = (cudaStream_t)stream;
    const imf_to2d_options &o = h->opt;
    const Grid g{o.nelx, o.nely};
    sens_kernel<<<blocks(h->ne), kT, 0, s>>>(g, h->k0, h->x, xi, rho, o.penal, o.E0 - o.Emin, o.beta, h->s);
    filter_kernel<<<blocks(h->ne), kT, 0, s>>>(g, xi, h->s, o.rmin, sens);
    TO_CU(cudaGetLastError());
    return IMF_OK;
}

imf_status imf_to2d_update(imf_to2d h, const float *xi, const float *S, const uint8_t *passive, double volfrac,
                           double move, double eta, float *xi_new, double *change_out, double *vol_out, void *stream)
{
    if (!h || !xi || !S || !xi_new) return fail(h, IMF_ERR_INVALID_ARG, "NULL argument");
    if (!(volfrac > 0.0 && volfrac < 1.0) || !(move > 0.0) || !(eta > 0.0))
        return fail(h, IMF_ERR_INVALID_ARG, "volfrac %g / move %g / eta %g out of range", volfrac, move, eta);
    cudaStream_t s = (cudaStream_t)stream;
    const double beta = h->opt.beta;
    double res[3] = {0, 0, 0};
    auto volume = [&](double lam, float *out) -> imf_status {
        TO_CU(cudaMemsetAsync(h->sc + S_VOL, 0, 3 * sizeof(double), s));
        oc_kernel<<<blocks(h->ne), kT, 0, s>>>(h->ne, xi, S, passive, lam, move, eta, beta, h->sc, out);
        TO_CU(cudaMemcpyAsync(res, h->sc + S_VOL, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        TO_CU(cudaStreamSynchronize(s));
        return IMF_OK;
    };
    // bisection on the multiplier in log space (the oracle's loop, step for step)
    double lo = 1e-12, hi = 1e12;
    while (hi / lo > 1.0 + 1e-9) {
        const double mid = std::sqrt(lo * hi);
        imf_status st = volume(mid, nullptr);
        if (st != IMF_OK) return st;
        const double vol = res[1] > 0 ? res[0] / res[1] : 0.0;
        if (vol > volfrac) lo = mid;
        else hi = mid;
    }
    imf_status st = volume(std::sqrt(lo * hi), xi_new);
    if (st != IMF_OK) return st;
    if (change_out) *change_out = res[1] > 0 ? res[2] / res[1] : 0.0;
    if (vol_out) *vol_out = res[1] > 0 ? res[0] / res[1] : 0.0;
    return IMF_OK;
}

imf_status imf_to2d_result(imf_to2d h, double *compliance, int *cg_iters, double *cg_rel_residual)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (compliance) *compliance = h->compliance;
    if (cg_iters) *cg_iters = h->iters;
    if (cg_rel_residual) *cg_rel_residual = h->rel_res;
    return IMF_OK;
}

} // extern "C"
