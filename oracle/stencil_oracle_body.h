/* Body of the plain CPU oracle, included once per precision by stencil_oracle.c with
 * REAL (float | double) and SFX (f32 | f64) defined.  TEST INFRASTRUCTURE ONLY.
 *
 * Every function is plain Jacobi iteration (Sec. 2.1): read one buffer, write the other,
 * swap, no blocking of any kind.  Each cell applies the Table 2 update in the order it is
 * printed, left to right, every product and sum rounded on its own (the file is compiled
 * with -ffp-contract=off so that no multiply-add is fused).  Out-of-range neighbours fall
 * back on the boundary cell itself (Sec. 5.1), evaluated per axis at every step.
 *
 * Neighbour orientation (the paper names the directions but the figure that fixes them is
 * lost): x is the fastest axis, w = x-1, e = x+1, n = y-1, s = y+1, b = z-1, a = z+1.
 */

#define CAT2(a, b) a##_##b
#define CAT(a, b) CAT2(a, b)

/* Diffusion 2D, Table 2 row 1: cc*c + cw*w + ce*e + cs*s + cn*n.  k = [cc,cw,ce,cs,cn]. */
static void CAT(diff2d_step, SFX)(const REAL *in, REAL *out, long nx, long ny, const REAL *k)
{
#pragma omp parallel for schedule(static)
    for (long y = 0; y < ny; y++) {
        long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
        for (long x = 0; x < nx; x++) {
            long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
            REAL c = in[y * nx + x];
            REAL w = in[y * nx + xw], e = in[y * nx + xe];
            REAL n = in[yn * nx + x], s = in[ys * nx + x];
            REAL r = k[0] * c;
            r = r + k[1] * w;
            r = r + k[2] * e;
            r = r + k[3] * s;
            r = r + k[4] * n;
            out[y * nx + x] = r;
        }
    }
}

/* Diffusion 3D, Table 2 row 2: ... + cb*b + ca*a.  k = [cc,cw,ce,cs,cn,cb,ca]. */
static void CAT(diff3d_step, SFX)(const REAL *in, REAL *out, long nx, long ny, long nz,
                                  const REAL *k)
{
    long pl = nx * ny;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; z++) {
        long zb = z > 0 ? z - 1 : 0, za = z < nz - 1 ? z + 1 : nz - 1;
        for (long y = 0; y < ny; y++) {
            long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
            for (long x = 0; x < nx; x++) {
                long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
                long i = z * pl + y * nx + x;
                REAL c = in[i];
                REAL w = in[z * pl + y * nx + xw], e = in[z * pl + y * nx + xe];
                REAL n = in[z * pl + yn * nx + x], s = in[z * pl + ys * nx + x];
                REAL b = in[zb * pl + y * nx + x], a = in[za * pl + y * nx + x];
                REAL r = k[0] * c;
                r = r + k[1] * w;
                r = r + k[2] * e;
                r = r + k[3] * s;
                r = r + k[4] * n;
                r = r + k[5] * b;
                r = r + k[6] * a;
                out[i] = r;
            }
        }
    }
}

/* Hotspot 2D, Table 2 row 3:
 *   c + sdc*(p + (n + s - 2c)*Ry + (e + w - 2c)*Rx + (amb - c)*Rz)
 * k = [sdc(k_dt), Rx, Ry, Rz, amb].  Fifteen operations, as the table counts them. */
static void CAT(thermal2d_step, SFX)(const REAL *in, REAL *out, const REAL *pw, long nx,
                                     long ny, const REAL *k)
{
    REAL sdc = k[0], rx = k[1], ry = k[2], rz = k[3], amb = k[4];
    REAL two = (REAL)2;
#pragma omp parallel for schedule(static)
    for (long y = 0; y < ny; y++) {
        long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
        for (long x = 0; x < nx; x++) {
            long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
            REAL c = in[y * nx + x];
            REAL w = in[y * nx + xw], e = in[y * nx + xe];
            REAL n = in[yn * nx + x], s = in[ys * nx + x];
            REAL p = pw[y * nx + x];
            REAL t1 = (n + s) - two * c;
            REAL t2 = (e + w) - two * c;
            REAL t3 = amb - c;
            REAL q = p + t1 * ry;
            q = q + t2 * rx;
            q = q + t3 * rz;
            out[y * nx + x] = c + sdc * q;
        }
    }
}

/* Hotspot 3D, Table 2 row 4:
 *   c*cc + n*cn + s*cs + e*ce + w*cw + a*ca + b*cb + sdc*p + ca*amb
 * k = [cc,cw,ce,cs,cn,cb,ca,sdc,amb]. */
static void CAT(thermal3d_step, SFX)(const REAL *in, REAL *out, const REAL *pw, long nx,
                                     long ny, long nz, const REAL *k)
{
    REAL cc = k[0], cw = k[1], ce = k[2], cs = k[3], cn = k[4], cb = k[5], ca = k[6];
    REAL sdc = k[7], amb = k[8];
    long pl = nx * ny;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; z++) {
        long zb = z > 0 ? z - 1 : 0, za = z < nz - 1 ? z + 1 : nz - 1;
        for (long y = 0; y < ny; y++) {
            long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
            for (long x = 0; x < nx; x++) {
                long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
                long i = z * pl + y * nx + x;
                REAL c = in[i];
                REAL w = in[z * pl + y * nx + xw], e = in[z * pl + y * nx + xe];
                REAL n = in[z * pl + yn * nx + x], s = in[z * pl + ys * nx + x];
                REAL b = in[zb * pl + y * nx + x], a = in[za * pl + y * nx + x];
                REAL r = c * cc;
                r = r + n * cn;
                r = r + s * cs;
                r = r + e * ce;
                r = r + w * cw;
                r = r + a * ca;
                r = r + b * cb;
                r = r + sdc * pw[i];
                r = r + ca * amb;
                out[i] = r;
            }
        }
    }
}

/* Star diffusion of radius R (the rad of Eqs. 1-2 above 1, the paper's named extension to
 * higher-order stencils), 2D: 4R+1 points, 3D: 6R+1 points.  k = [cc, then for d = 1..R:
 * cw_d, ce_d, cs_d, cn_d (2D) or cw_d, ce_d, cs_d, cn_d, cb_d, ca_d (3D)], where the d-suffixed
 * neighbour lies d cells away in that direction.  Evaluated as Table 2 evaluates the first-order
 * diffusion, extended outwards: r = cc*c, then distance 1 in the order w, e, s, n (b, a), then
 * distance 2 in the same order, and so on, every product and sum rounded on its own.  Each
 * neighbour index is clamped to the grid on its own axis (Sec. 5.1's fallback on the boundary
 * cell, applied at every distance).  For R = 1 this is exactly the Table 2 update. */
static void CAT(star_step, SFX)(const REAL *in, REAL *out, int ndim, int R, long nx, long ny,
                                long nz, const REAL *k)
{
    long pl = nx * ny;
    long planes = ndim == 3 ? nz : 1;
    int per = ndim == 3 ? 6 : 4;
#pragma omp parallel for schedule(static)
    for (long zy = 0; zy < planes * ny; zy++) {
        long z = zy / ny, y = zy % ny;
        for (long x = 0; x < nx; x++) {
            long i = z * pl + y * nx + x;
            REAL r = k[0] * in[i];
            for (int d = 1; d <= R; d++) {
                long xw = x - d >= 0 ? x - d : 0, xe = x + d <= nx - 1 ? x + d : nx - 1;
                long ys = y + d <= ny - 1 ? y + d : ny - 1, yn = y - d >= 0 ? y - d : 0;
                const REAL *kd = k + 1 + (long)per * (d - 1);
                r = r + kd[0] * in[z * pl + y * nx + xw];
                r = r + kd[1] * in[z * pl + y * nx + xe];
                r = r + kd[2] * in[z * pl + ys * nx + x];
                r = r + kd[3] * in[z * pl + yn * nx + x];
                if (ndim == 3) {
                    long zb = z - d >= 0 ? z - d : 0, za = z + d <= nz - 1 ? z + d : nz - 1;
                    r = r + kd[4] * in[zb * pl + y * nx + x];
                    r = r + kd[5] * in[za * pl + y * nx + x];
                }
            }
            out[i] = r;
        }
    }
}

/* Diffusion 2D with per-cell coefficients: Table 2 row 1 with every coefficient an array
 * (Sec. 5.1 lets a kernel variable be a scalar argument or an array), evaluated in the same order:
 * cc_i*c + cw_i*w + ce_i*e + cs_i*s + cn_i*n, the coefficients those of the cell being updated.
 * k holds five planar grids [cc | cw | ce | cs | cn], each nx*ny, row-major. */
static void CAT(vdiff2d_step, SFX)(const REAL *in, REAL *out, long nx, long ny, const REAL *k)
{
    long pl = nx * ny;
#pragma omp parallel for schedule(static)
    for (long y = 0; y < ny; y++) {
        long yn = y > 0 ? y - 1 : 0, ys = y < ny - 1 ? y + 1 : ny - 1;
        for (long x = 0; x < nx; x++) {
            long xw = x > 0 ? x - 1 : 0, xe = x < nx - 1 ? x + 1 : nx - 1;
            long i = y * nx + x;
            REAL r = k[i] * in[i];
            r = r + k[pl + i] * in[y * nx + xw];
            r = r + k[2 * pl + i] * in[y * nx + xe];
            r = r + k[3 * pl + i] * in[ys * nx + x];
            r = r + k[4 * pl + i] * in[yn * nx + x];
            out[i] = r;
        }
    }
}

/* `steps` Jacobi iterations of the per-cell-coefficient diffusion 2D. */
int CAT(orc_run_vdiff2d, SFX)(const REAL *u0, REAL *out, const REAL *k, long nx, long ny,
                              int steps)
{
    if (!u0 || !out || !k || nx < 1 || ny < 1 || steps < 0) return -1;
    size_t n = (size_t)nx * ny;
    REAL *a = (REAL *)malloc(n * sizeof(REAL));
    REAL *b = (REAL *)malloc(n * sizeof(REAL));
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, u0, n * sizeof(REAL));
    for (int s = 0; s < steps; s++) {
        CAT(vdiff2d_step, SFX)(a, b, nx, ny, k);
        REAL *t = a; a = b; b = t;
    }
    memcpy(out, a, n * sizeof(REAL));
    free(a);
    free(b);
    return 0;
}

/* `steps` Jacobi iterations of the radius-R star diffusion (ndim 2 or 3, R >= 1). */
int CAT(orc_run_star, SFX)(int ndim, int R, const REAL *u0, REAL *out, const REAL *coef,
                           long nx, long ny, long nz, int steps)
{
    if (!u0 || !out || !coef || nx < 1 || ny < 1 || nz < 1 || steps < 0 || R < 1) return -1;
    if (ndim == 2) nz = 1;
    else if (ndim != 3) return -1;
    size_t n = (size_t)nx * ny * nz;
    REAL *a = (REAL *)malloc(n * sizeof(REAL));
    REAL *b = (REAL *)malloc(n * sizeof(REAL));
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, u0, n * sizeof(REAL));
    for (int s = 0; s < steps; s++) {
        CAT(star_step, SFX)(a, b, ndim, R, nx, ny, nz, coef);
        REAL *t = a; a = b; b = t;
    }
    memcpy(out, a, n * sizeof(REAL));
    free(a);
    free(b);
    return 0;
}

/* `steps` Jacobi iterations of stencil (kind, ndim) from u0 into out (Sec. 2.1: read one
 * buffer, write the other, swap).  steps == 0 copies.  Returns 0, or -1 on a bad argument or
 * a failed allocation. */
int CAT(orc_run, SFX)(int kind, int ndim, const REAL *u0, REAL *out, const REAL *power,
                      const REAL *coef, long nx, long ny, long nz, int steps)
{
    if (!u0 || !out || !coef || nx < 1 || ny < 1 || nz < 1 || steps < 0) return -1;
    if (ndim == 2) nz = 1;
    else if (ndim != 3) return -1;
    if (kind == 1 && !power) return -1;
    if (kind != 0 && kind != 1) return -1;
    size_t n = (size_t)nx * ny * nz;
    REAL *a = (REAL *)malloc(n * sizeof(REAL));
    REAL *b = (REAL *)malloc(n * sizeof(REAL));
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, u0, n * sizeof(REAL));
    for (int s = 0; s < steps; s++) {
        if (kind == 0 && ndim == 2) CAT(diff2d_step, SFX)(a, b, nx, ny, coef);
        else if (kind == 0) CAT(diff3d_step, SFX)(a, b, nx, ny, nz, coef);
        else if (ndim == 2) CAT(thermal2d_step, SFX)(a, b, power, nx, ny, coef);
        else CAT(thermal3d_step, SFX)(a, b, power, nx, ny, nz, coef);
        REAL *t = a; a = b; b = t;
    }
    memcpy(out, a, n * sizeof(REAL));
    free(a);
    free(b);
    return 0;
}

#undef CAT
#undef CAT2
