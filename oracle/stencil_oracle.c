/* Plain CPU oracle for iterated first-order Jacobi stencils with clamped boundaries.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use this file; the engine shares no code with it and never calls it.
 *
 * What it computes (arXiv 1802.00438):
 *   - Sec. 2.1: Jacobi iteration, one buffer read and the other written, then swapped.
 *   - Table 2: the four update equations (Diffusion 2D/3D, Hotspot 2D/3D), evaluated in the
 *     printed order with every operation rounded separately (built with -ffp-contract=off).
 *   - Sec. 5.1: out-of-bound neighbours fall back on the boundary cell itself.
 *   - Eqs. 1-2 with rad > 1 (the paper's named extension): star diffusion of radius R, the
 *     first-order diffusion order extended outwards one distance at a time.
 *   - Table 2 row 1 with every coefficient an array (Sec. 5.1 lets a kernel variable be a
 *     scalar argument or an array): diffusion 2D whose cells carry their own five weights.
 * The spatial and temporal blocking of Sec. 3 reorganise this computation without changing
 * a single cell's arithmetic, so the blocked engine must reproduce these values exactly
 * when it evaluates the same operations in the same order.
 *
 * Precisions: float (the paper's single precision, Sec. 5.1) for parity, double as the
 * error reference.  OpenMP splits each step over rows or planes; every cell of a step is
 * independent, so the result does not depend on the thread count.
 *
 * Parity pins live in the test suite (hand-computed steps, impulse response, invariants,
 * dense-matrix brute force, the DCT closed form).  The adjoint below is pinned by the
 * dot-product test against a dense matrix and by central finite differences.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REAL float
#define SFX f32
#include "stencil_oracle_body.h"
#undef REAL
#undef SFX

#define REAL double
#define SFX f64
#include "stencil_oracle_body.h"
#undef REAL
#undef SFX

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------
 * Adjoint of a 2D run (double precision), for the differentiation pattern.
 *
 * Forward map of one step: u_{t+1} = F(u_t; theta, p), F the Table 2 update with the clamped
 * boundary.  Loss L = sum_i w_i u_N[i].  Reverse mode:
 *   lambda_N = w,   lambda_t = J_t^T lambda_{t+1}   (J_t = dF/du at u_t; F is affine in u),
 *   dL/du_0 = lambda_0,
 *   dL/dtheta = sum_{t<N} sum_i lambda_{t+1}[i] * dF_i/dtheta (u_t),
 *   dL/dp_i   = sum_{t<N} lambda_{t+1}[i] * dF_i/dp_i.
 * The transpose is applied as the plain scatter it is by definition: every output cell i adds
 * lambda[i] times its weight on each neighbour into that neighbour's (clamped) slot.  That
 * is why this part runs on one thread.
 *
 * Forward states are kept every `ckpt` steps and each segment is recomputed before its
 * reverse sweep; ckpt <= 0 keeps every state.
 * --------------------------------------------------------------------------------------- */

/* dF_i/dtheta for one cell, given its neighbourhood; writes ncoef partials into g. */
static void dfdtheta(int kind, const double *k, double c, double w, double e, double n, double s,
                     double p, double *g)
{
    if (kind == 0) {                       /* [cc,cw,ce,cs,cn] */
        g[0] = c; g[1] = w; g[2] = e; g[3] = s; g[4] = n;
    } else {                               /* [k_dt,Rx,Ry,Rz,amb] */
        double t1 = (n + s) - 2.0 * c, t2 = (e + w) - 2.0 * c, t3 = k[4] - c;
        double q = p + t1 * k[2] + t2 * k[1] + t3 * k[3];
        g[0] = q;
        g[1] = k[0] * t2;
        g[2] = k[0] * t1;
        g[3] = k[0] * t3;
        g[4] = k[0] * k[3];
    }
}

/* lam_out = J^T lam_in for one step (J independent of u: the update is affine in u). */
static void transpose_step(int kind, const double *k, const double *lin, double *lout, long nx,
                           long ny)
{
    /* weights of F_i on (c, w, e, s, n) */
    double wc, ww, we, ws, wn;
    if (kind == 0) {
        wc = k[0]; ww = k[1]; we = k[2]; ws = k[3]; wn = k[4];
    } else {
        wc = 1.0 - k[0] * (2.0 * k[2] + 2.0 * k[1] + k[3]);
        ww = we = k[0] * k[1];
        wn = ws = k[0] * k[2];
    }
    memset(lout, 0, (size_t)nx * ny * sizeof(double));
    for (long y = 0; y < ny; y++) {
        long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
        for (long x = 0; x < nx; x++) {
            long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
            double l = lin[y * nx + x];
            lout[y * nx + x] += wc * l;
            lout[y * nx + xw] += ww * l;
            lout[y * nx + xe] += we * l;
            lout[ys * nx + x] += ws * l;
            lout[yn * nx + x] += wn * l;
        }
    }
}

int orc_adjoint2d_f64(int kind, const double *u0, const double *power, const double *coef,
                      long nx, long ny, int steps, int ckpt, const double *wgt, double *grad_u0,
                      double *grad_coef, double *grad_power)
{
    if (!u0 || !coef || !wgt || !grad_u0 || !grad_coef || nx < 1 || ny < 1 || steps < 0)
        return -1;
    if (kind != 0 && kind != 1) return -1;
    if (kind == 1 && (!power || !grad_power)) return -1;
    size_t n = (size_t)nx * ny;
    if (ckpt <= 0 || ckpt > steps) ckpt = steps > 0 ? steps : 1;
    int nseg = (steps + ckpt - 1) / ckpt;
    double *cks = (double *)malloc((size_t)(nseg > 0 ? nseg : 1) * n * sizeof(double));
    double *seg = (double *)malloc((size_t)(ckpt + 1) * n * sizeof(double));
    double *la = (double *)malloc(n * sizeof(double));
    double *lb = (double *)malloc(n * sizeof(double));
    if (!cks || !seg || !la || !lb) {
        free(cks); free(seg); free(la); free(lb);
        return -1;
    }
    /* forward, keeping u at steps 0, ckpt, 2 ckpt, ... */
    memcpy(seg, u0, n * sizeof(double));
    for (int s = 0; s < steps; s++) {
        if (s % ckpt == 0) memcpy(cks + (size_t)(s / ckpt) * n, seg, n * sizeof(double));
        double *nx_ = seg + n;
        if (kind == 0) diff2d_step_f64(seg, nx_, nx, ny, coef);
        else thermal2d_step_f64(seg, nx_, power, nx, ny, coef);
        memcpy(seg, nx_, n * sizeof(double));
    }
    int ncoef = 5;
    for (int j = 0; j < ncoef; j++) grad_coef[j] = 0.0;
    if (kind == 1) memset(grad_power, 0, n * sizeof(double));
    memcpy(la, wgt, n * sizeof(double));                 /* lambda_N */
    for (int sg = nseg - 1; sg >= 0; sg--) {
        int t0 = sg * ckpt, t1 = t0 + ckpt < steps ? t0 + ckpt : steps;
        memcpy(seg, cks + (size_t)sg * n, n * sizeof(double));
        for (int t = t0; t < t1 - 1; t++) {               /* states t0 .. t1-1 */
            double *a = seg + (size_t)(t - t0) * n, *b = a + n;
            if (kind == 0) diff2d_step_f64(a, b, nx, ny, coef);
            else thermal2d_step_f64(a, b, power, nx, ny, coef);
        }
        for (int t = t1 - 1; t >= t0; t--) {
            const double *u = seg + (size_t)(t - t0) * n;  /* u_t; la holds lambda_{t+1} */
            for (long y = 0; y < ny; y++) {
                long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
                for (long x = 0; x < nx; x++) {
                    long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
                    double g[5];
                    double p = kind == 1 ? power[y * nx + x] : 0.0;
                    dfdtheta(kind, coef, u[y * nx + x], u[y * nx + xw], u[y * nx + xe],
                             u[yn * nx + x], u[ys * nx + x], p, g);
                    double l = la[y * nx + x];
                    for (int j = 0; j < ncoef; j++) grad_coef[j] += l * g[j];
                    if (kind == 1) grad_power[y * nx + x] += l * coef[0];
                }
            }
            transpose_step(kind, coef, la, lb, nx, ny);  /* lambda_t */
            double *tmp = la; la = lb; lb = tmp;
        }
    }
    memcpy(grad_u0, la, n * sizeof(double));
    free(cks); free(seg); free(la); free(lb);
    return 0;
}
