/*
 * Plain FP64 CPU oracle of the inaccessibility measure field (IMF).
 *
 * TEST INFRASTRUCTURE ONLY. This file is called by the tests, by the entry point's smoke check
 * and by the CPU-baseline leg of the benchmark. It shares no code, header or table with the
 * CUDA library: every definition below is written directly from the paper
 * (Mirzendehdel, Behandish, Nelaturi, "Topology Optimization with Accessibility Constraint
 * for Multi-Axis Machining", arXiv 2002.07627), in the most literal form available:
 * direct sums, brute-force sweeps and brute-force minima, with no FFT, blocking or fusion.
 *
 * Conventions: grids are C order [nz][ny][nx] (x fastest). Offsets are int32 triples
 * (x, y, z). A "box" is lo[3] (inclusive) and ext[3] (extents), indexed like a grid.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (floating-point contraction must be
 * off so that the rotation arithmetic below is the exact sequence of IEEE operations written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX3(x, y, z, ex, ey) ((((long)(z)) * (ey) + (y)) * (long)(ex) + (x))

/*
 * Unit quaternion (w, x, y, z) to the 3x3 rotation matrix R (row major, v = R u).
 * Sec. 2.1 leaves the parameterisation of SO(3) open; Alg. 1 gives orientations as unit
 * quaternions. The quaternion is first normalised by its Euclidean norm.
 */
void oracle_quat_to_matrix(const double q[4], double R[9])
{
    double n = sqrt(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/*
 * Conservative box of offsets v that the rotated tool can occupy (Alg. 1, "Rotate").
 * A tool voxel u (offset from the origin voxel o) covers the cube u + [-1/2, 1/2]^3; the
 * rotated array occupies R applied to the union of those cubes, whose bounding box is the
 * bounding box of the 8 rotated corners of the array's voxel-edge box. One voxel of margin
 * is added on every side.
 */
void oracle_rotate_box(int tx, int ty, int tz, const int o[3], const double R[9], int lo[3], int ext[3])
{
    double cmin[3] = {1e300, 1e300, 1e300}, cmax[3] = {-1e300, -1e300, -1e300};
    const double a[3][2] = {{-o[0] - 0.5, tx - o[0] - 0.5},
                            {-o[1] - 0.5, ty - o[1] - 0.5},
                            {-o[2] - 0.5, tz - o[2] - 0.5}};
    for (int c = 0; c < 8; ++c) {
        double u[3] = {a[0][c & 1], a[1][(c >> 1) & 1], a[2][(c >> 2) & 1]};
        for (int i = 0; i < 3; ++i) {
            double v = R[3 * i + 0] * u[0] + R[3 * i + 1] * u[1] + R[3 * i + 2] * u[2];
            if (v < cmin[i]) cmin[i] = v;
            if (v > cmax[i]) cmax[i] = v;
        }
    }
    for (int i = 0; i < 3; ++i) {
        lo[i] = (int)floor(cmin[i]) - 1;
        ext[i] = ((int)ceil(cmax[i]) + 1) - lo[i] + 1;
    }
}

/*
 * Rotation and re-sampling of a binary tool array on the uniform grid (Alg. 1, "Rotate"),
 * read as nearest-neighbour inverse mapping about the origin voxel: for an integer offset v,
 *   p = R^T v,   u = floor(p + 1/2) per component,   out(v) = arr(o + u)  (0 outside arr).
 * R^T v is evaluated per component j as (R_0j v_0 + R_1j v_1) + R_2j v_2.
 * Writes out[] over the box (lo, ext). Returns the number of ones written.
 */
long oracle_rotate(const uint8_t *arr, int tx, int ty, int tz, const int o[3], const double R[9],
                   const int lo[3], const int ext[3], uint8_t *out)
{
    long count = 0;
    for (int k = 0; k < ext[2]; ++k)
        for (int j = 0; j < ext[1]; ++j)
            for (int i = 0; i < ext[0]; ++i) {
                double v0 = lo[0] + i, v1 = lo[1] + j, v2 = lo[2] + k;
                int ui[3];
                for (int c = 0; c < 3; ++c) {
                    double p = (R[0 * 3 + c] * v0 + R[1 * 3 + c] * v1) + R[2 * 3 + c] * v2;
                    ui[c] = (int)floor(p + 0.5);
                }
                int ax = o[0] + ui[0], ay = o[1] + ui[1], az = o[2] + ui[2];
                uint8_t b = 0;
                if (ax >= 0 && ax < tx && ay >= 0 && ay < ty && az >= 0 && az < tz)
                    b = arr[IDX3(ax, ay, az, tx, ty)] ? 1 : 0;
                out[IDX3(i, j, k, ext[0], ext[1])] = b;
                count += b;
            }
    return count;
}

/* density of the obstacle at an integer point; empty air outside the grid */
static inline double rho_at(const double *rho, int nx, int ny, int nz, long x, long y, long z)
{
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0.0;
    return rho[IDX3(x, y, z, nx, ny)];
}

/*
 * Collision measure of the oriented tool at translation t (Eq. eq_ident, Eq. eq_conv_1 with
 * the reflection folded into the index):  g(t) = sum_{v in RT} rho_O(t + v),
 * summed in FP64 in the order of the offset list, for every t in the box (tlo, text).
 */
void oracle_collision(const double *rho, int nx, int ny, int nz, const int32_t *off, long n_off,
                      const int tlo[3], const int text[3], double *g)
{
    long nrow = (long)text[1] * text[2];
#pragma omp parallel for schedule(dynamic, 4)
    for (long r = 0; r < nrow; ++r) {
        int j = (int)(r % text[1]), k = (int)(r / text[1]);
        for (int i = 0; i < text[0]; ++i) {
            long t0 = tlo[0] + i, t1 = tlo[1] + j, t2 = tlo[2] + k;
            double s = 0.0;
            for (long m = 0; m < n_off; ++m)
                s += rho_at(rho, nx, ny, nz, t0 + off[3 * m], t1 + off[3 * m + 1], t2 + off[3 * m + 2]);
            g[IDX3(i, j, k, text[0], text[1])] = s;
        }
    }
}

static inline int in_box(const int lo[3], const int ext[3], long a, long b, long c)
{
    return a >= lo[0] && b >= lo[1] && c >= lo[2] && a < lo[0] + ext[0] && b < lo[1] + ext[1] &&
           c < lo[2] + ext[2];
}

/*
 * Sweep of the cutter over the collision-free translations (Eq. eq_conv_A / eq_conv_2):
 *   cnt(x) = sum_{k in RK} free(x - k),   A(x) = sign(cnt(x)) = [cnt(x) > 0],
 * for every grid point x; free is given on the box (tlo, text) and is 0 outside it.
 * Either output may be NULL.
 */
void oracle_sweep(const uint8_t *freeb, const int tlo[3], const int text[3], const int32_t *off,
                  long n_off, int nx, int ny, int nz, uint8_t *A, int32_t *cnt)
{
    long nrow = (long)ny * nz;
#pragma omp parallel for schedule(dynamic, 4)
    for (long r = 0; r < nrow; ++r) {
        int y = (int)(r % ny), z = (int)(r / ny);
        for (int x = 0; x < nx; ++x) {
            int32_t c = 0;
            for (long m = 0; m < n_off; ++m) {
                long a = (long)x - off[3 * m], b = (long)y - off[3 * m + 1], d = (long)z - off[3 * m + 2];
                if (in_box(tlo, text, a, b, d))
                    c += freeb[IDX3(a - tlo[0], b - tlo[1], d - tlo[2], text[0], text[1])] ? 1 : 0;
            }
            if (A) A[IDX3(x, y, z, nx, ny)] = c > 0;
            if (cnt) cnt[IDX3(x, y, z, nx, ny)] = c;
        }
    }
}

/*
 * Minimum over sharp points of the shifted collision measure (Eq. eq_imf_2 / eq_imf_4):
 *   gamma(x) = min_{k in sharp} g(x - k)
 * for every grid point x. g is given on the box (tlo, text); a query outside the box is an
 * error (returns -1). With no sharp points gamma = +inf (Alg. 1 starts its minima at +inf).
 */
int oracle_erode(const double *g, const int tlo[3], const int text[3], const int32_t *off, long n_off,
                 int nx, int ny, int nz, double *gamma)
{
    int bad = 0;
    long nrow = (long)ny * nz;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (long r = 0; r < nrow; ++r) {
        int y = (int)(r % ny), z = (int)(r / ny);
        for (int x = 0; x < nx; ++x) {
            double m = INFINITY;
            for (long s = 0; s < n_off; ++s) {
                long a = (long)x - off[3 * s], b = (long)y - off[3 * s + 1], d = (long)z - off[3 * s + 2];
                if (!in_box(tlo, text, a, b, d)) { bad = 1; continue; }
                double v = g[IDX3(a - tlo[0], b - tlo[1], d - tlo[2], text[0], text[1])];
                if (v < m) m = v;
            }
            gamma[IDX3(x, y, z, nx, ny)] = m;
        }
    }
    return bad ? -1 : 0;
}

/*
 * Point queries for large grids: for each query point x and each orientation r,
 *   gamma_r(x) = min_{k in sharp_r} g_r(x - k),   g_r(t) = sum_{v in RT_r} rho_O(t + v),
 *   A_r(x)     = OR_{k in RK_r} [g_r(x - k) <= theta_r],
 * and f(x) = min_r gamma_r(x), A(x) = OR_r A_r(x). Orientation lists are concatenated, with
 * per-orientation counts. This is Eq. eq_imf_4 evaluated literally at single points.
 */
void oracle_point_query(const double *rho, int nx, int ny, int nz, int n_orient,
                        const int32_t *rt, const long *n_rt, const int32_t *sharp, const long *n_sharp,
                        const int32_t *rk, const long *n_rk, const double *theta, long n_pts,
                        const int32_t *pts, double *f_out, uint8_t *A_out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (long p = 0; p < n_pts; ++p) {
        long x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
        double f = INFINITY;
        int acc = 0;
        long o_rt = 0, o_sh = 0, o_rk = 0;
        for (int r = 0; r < n_orient; ++r) {
            const int32_t *RT = rt + 3 * o_rt, *SH = sharp + 3 * o_sh, *RK = rk + 3 * o_rk;
            for (long s = 0; s < n_sharp[r]; ++s) {
                long t0 = x - SH[3 * s], t1 = y - SH[3 * s + 1], t2 = z - SH[3 * s + 2];
                double g = 0.0;
                for (long m = 0; m < n_rt[r]; ++m)
                    g += rho_at(rho, nx, ny, nz, t0 + RT[3 * m], t1 + RT[3 * m + 1], t2 + RT[3 * m + 2]);
                if (g < f) f = g;
            }
            if (!acc) {
                for (long s = 0; s < n_rk[r]; ++s) {
                    long t0 = x - RK[3 * s], t1 = y - RK[3 * s + 1], t2 = z - RK[3 * s + 2];
                    double g = 0.0;
                    for (long m = 0; m < n_rt[r]; ++m)
                        g += rho_at(rho, nx, ny, nz, t0 + RT[3 * m], t1 + RT[3 * m + 1], t2 + RT[3 * m + 2]);
                    if (g <= theta[r]) { acc = 1; break; }
                }
            }
            o_rt += n_rt[r];
            o_sh += n_sharp[r];
            o_rk += n_rk[r];
        }
        f_out[p] = f;
        A_out[p] = (uint8_t)acc;
    }
}
