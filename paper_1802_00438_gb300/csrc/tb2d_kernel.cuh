// 2D temporally-blocked Jacobi sweep: one pass advances the grid by `tsteps` (<= T) steps.
//
// Method (arXiv 1802.00438): spatial blocking in x with overlapped tiles (Sec. 3.1, Fig. 4)
// and streaming along y without blocking (Sec. 3.1); temporal blocking by a chain of T
// stages, stage t computing time step t a fixed number of rows behind stage t-1 (Sec. 3.2);
// halos of width >= rad*T (Eq. 2) computed redundantly, only the compute block written back
// (Sec. 3.2); when the pass fuses fewer than T steps the trailing stages forward their input
// (Sec. 3.2).  Clamped boundary (Sec. 5.1) applied at every stage.
//
// GPU mapping.
//   Block  = W warps side by side along x; a tile is BX = 32*V*W cells wide incl. halos of
//            H = roundup(T, 4) cells per side, so tile origins are 16-byte aligned.
//   Thread = V consecutive cells of a row.
//   Stream = a block walks down y over one or more (tile column, row range) segments; a
//            segment [s0, s1) loads rows s0-tsteps .. s1-1+tsteps (clamped to the grid).
//   Stage 0 reads its three rows (r-1, r, r+1 of time 0) directly from a shared-memory ring
//            that cp.async fills PF rows ahead; stages 1..T-1 hold their three-row window of
//            the previous time level in registers.  The window rotates through three register
//            sets, so the loop body is unrolled three times (one per phase) and no register
//            is copied when the window slides.
//   x-neighbours of a thread's edge cells come from the adjacent lanes by shuffle; across
//            warps, lane 0 / lane 31 of every warp publish their edge cell in shared memory
//            and the neighbour warp reads it one row later (one barrier per row).  Lanes with
//            nothing to publish store to a spare slot, so the store is branch-free.
//   Power rows (Hotspot) stay in a ring of >= T+PF+1 rows so every stage reads the power of
//            the row it is computing; per-cell diffusion coefficients (kind KVDIFF: five
//            planar arrays cc, cw, ce, cs, cn) travel the same way, one ring per plane.
//   Three variants of the row body: PLAIN (interior warps), EDGE (a warp holding x = 0 or
//            x = nx-1 clamps its neighbours) and SPECIAL (rows at the top or bottom of the grid,
//            or a pass that forwards trailing stages); interior rows of interior warps carry
//            no boundary test at all.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace stn {

constexpr int pow2_at_least(int v)
{
    int p = 1;
    while (p < v) p *= 2;
    return p;
}

template <int KIND, bool EXACT, int T, int V, int W>
struct TB2 {
    static constexpr int NT = 32 * W;
    static constexpr int BX = 32 * V * W;
    static constexpr int H = (T + 3) / 4 * 4;
    static constexpr int CX = BX - 2 * H;
    static constexpr int PF = 3;                              // rows requested ahead
    static constexpr int NBF = pow2_at_least(PF + 3);         // field ring: r-1 .. r+1, PF ahead
    static constexpr int NBP = (KIND != KDIFF) ? pow2_at_least(T + PF + 1) : 0;
    static constexpr int NPL = (KIND == KVDIFF) ? 5 : 1;     // planes of per-cell input
    static constexpr int NS = T > 1 ? T - 1 : 1;              // register-window stages 1..T-1
    static constexpr int NX = (W > 1 && T > 1) ? (T - 1) : 0; // exchanged stage outputs
    static constexpr int XB = (W + 3) * 2;                    // floats per (parity, stage) block
    static constexpr size_t SMEM =
        sizeof(float) * ((size_t)(NBF + NPL * NBP) * BX + (size_t)2 * (NX > 0 ? NX : 1) * XB);
    static_assert(V % 4 == 0, "V must be a multiple of 4");
    static_assert(CX > 0, "tile narrower than its halos");
};

enum { MODE_PLAIN = 0, MODE_EDGE = 1, MODE_SPECIAL = 2 };

struct Ctx2 {
    const float *__restrict__ in;
    float *__restrict__ out;
    const float *__restrict__ pw;   // power map, or the first of the coefficient planes
    long long ld_in, ld_out, ld_pw;
    long long pw_plane;   // floats from one coefficient plane to the next (KVDIFF)
    float *ringF, *ringP, *xch;   // ringP: NPL rings of NBP rows each
    int nx, ny, tsteps;
    int x0, xt;           // tile origin, my first cell
    int y_start, last_row, s0, s1;
    unsigned lmask, rmask;   // bit j: my cell j is x = 0 / x = nx-1 (a mask rather than an
                             // index: a per-cell index compare can be rewritten into an indexed
                             // store, which would push the row to local memory)
    int st_lo, st_hi;     // my cells [st_lo, st_hi) are stored
    bool st_full;         // all V cells stored with vector stores
    int xr_off, xw_off;   // exchange read / write offsets of this lane
    bool edge;            // this warp holds x = 0 or x = nx-1
    bool is0, is31;       // lane 0 / lane 31
    int vec_in, vec_out, vec_pw;
    int tid, lane, wid;
    float k0, k1, k2, k3, k4;
};

template <int KIND, bool EXACT>
__device__ __forceinline__ float upd2(const Ctx2 &c, float m, float w, float e, float s, float n,
                                      float p)
{
    if (KIND == KDIFF)
        return diff5<EXACT>(m, w, e, s, n, c.k0, c.k1, c.k2, c.k3, c.k4);
    else
        return hot2<EXACT>(m, w, e, s, n, p, c.k0, c.k1, c.k2, c.k3, c.k4);
}

// the cell update with per-cell inputs q (Hotspot: power in q[0]; KVDIFF: cc, cw, ce, cs, cn)
template <int KIND, bool EXACT, int NPL>
__device__ __forceinline__ float upd2q(const Ctx2 &c, float m, float w, float e, float s, float n,
                                       const float (&q)[NPL])
{
    if (KIND == KVDIFF)
        return diff5<EXACT>(m, w, e, s, n, q[0], q[NPL > 1 ? 1 : 0], q[NPL > 2 ? 2 : 0],
                            q[NPL > 3 ? 3 : 0], q[NPL > 4 ? 4 : 0]);
    return upd2<KIND, EXACT>(c, m, w, e, s, n, q[0]);
}

// my V cells of per-cell input row `slot` of every plane
template <int V, int NPL, int NBP, int BX>
__device__ __forceinline__ void ld_planes(const float *ring, int slot, int o, float (&q)[NPL][V]);

template <int NT>
__device__ __forceinline__ void tb2_sync()
{
    if (NT == 32) __syncwarp();
    else __syncthreads();
}

// Issue the async copy of tile row y (field, and power for Hotspot) into ring slots.
template <int KIND, int BX, int NT, int NPL = 1, int NBP = 0>
__device__ __forceinline__ void tb2_load_row(const Ctx2 &c, int y, float *dstF, float *dstP)
{
    const float *srcF = c.in + (long long)y * c.ld_in;
    const float *srcP = (KIND != KDIFF) ? c.pw + (long long)y * c.ld_pw : nullptr;
#pragma unroll
    for (int qq = 0; qq < BX / 4 / NT; qq++) {
        const int q = c.tid + qq * NT;
        const int x = c.x0 + 4 * q;   // x is a multiple of 4: a chunk is all < 0 or all >= 0
        if (c.vec_in) {
            const int nb = (x >= 0 && x < c.nx) ? min(16, 4 * (c.nx - x)) : 0;
            cp_async16(dstF + 4 * q, nb ? srcF + x : srcF, nb);
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int xx = x + j;
                const int nb = (xx >= 0 && xx < c.nx) ? 4 : 0;
                cp_async4(dstF + 4 * q + j, nb ? srcF + xx : srcF, nb);
            }
        }
        if (KIND != KDIFF) {
#pragma unroll
            for (int pl = 0; pl < NPL; pl++) {
                const float *sp = srcP + pl * c.pw_plane;
                float *dp = dstP + pl * NBP * BX;
                if (c.vec_pw) {
                    const int nb = (x >= 0 && x < c.nx) ? min(16, 4 * (c.nx - x)) : 0;
                    cp_async16(dp + 4 * q, nb ? sp + x : sp, nb);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int xx = x + j;
                        const int nb = (xx >= 0 && xx < c.nx) ? 4 : 0;
                        cp_async4(dp + 4 * q + j, nb ? sp + xx : sp, nb);
                    }
                }
            }
        }
    }
}

template <int V>
__device__ __forceinline__ void ld_smem_row(const float *p, float (&v)[V])
{
#pragma unroll
    for (int q = 0; q < V / 4; q++) {
        float4 t = *reinterpret_cast<const float4 *>(p + 4 * q);
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}

template <int V, int NPL, int NBP, int BX>
__device__ __forceinline__ void ld_planes(const float *ring, int slot, int o, float (&q)[NPL][V])
{
#pragma unroll
    for (int pl = 0; pl < NPL; pl++) ld_smem_row<V>(ring + (pl * NBP + slot) * BX + o, q[pl]);
}

// Neighbour values of my V cells of row `m`, given the cells just left and right of them.
template <int V, bool EDGE>
__device__ __forceinline__ void neighbours(const Ctx2 &c, const float (&m)[V], float w_in,
                                           float e_in, float (&wv)[V], float (&ev)[V])
{
    wv[0] = w_in;
    ev[V - 1] = e_in;
#pragma unroll
    for (int j = 1; j < V; j++) wv[j] = m[j - 1];
#pragma unroll
    for (int j = 0; j < V - 1; j++) ev[j] = m[j + 1];
    if (EDGE) {   // clamp x-1 at x = 0 and x+1 at x = nx-1 to the cell itself
#pragma unroll
        for (int j = 0; j < V; j++) {
            wv[j] = ((c.lmask >> j) & 1u) ? m[j] : wv[j];
            ev[j] = ((c.rmask >> j) & 1u) ? m[j] : ev[j];
        }
    }
}

template <int V>
__device__ __forceinline__ void store_row(const Ctx2 &c, int r, const float (&v)[V])
{
    float *dst = c.out + (long long)r * c.ld_out + c.xt;
    if (c.st_full) {
#pragma unroll
        for (int q = 0; q < V / 4; q++)
            *reinterpret_cast<float4 *>(dst + 4 * q) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < V; j++)
            if (j >= c.st_lo && j < c.st_hi) dst[j] = v[j];
    }
}

template <int KIND, bool EXACT, int T, int V, int W, int P, int MODE>
__device__ __forceinline__ void tb2_stages(const Ctx2 &c,
                                           float (&B)[TB2<KIND, EXACT, T, V, W>::NS][3][V], int i,
                                           int R0, float (&out)[V]);

// One row iteration in phase P (= i mod 3) and boundary mode MODE.
template <int KIND, bool EXACT, int T, int V, int W, int P, int MODE>
__device__ __forceinline__ void tb2_iter(const Ctx2 &c, float (&B)[TB2<KIND, EXACT, T, V, W>::NS][3][V],
                                         int i)
{
    using C = TB2<KIND, EXACT, T, V, W>;
    constexpr bool SP = MODE == MODE_SPECIAL;
    constexpr bool ED = MODE != MODE_PLAIN;
    const int R0 = c.y_start + i;   // row that arrived for this iteration

    // ---- stage 0: time 1 at row R0-1 from the time-0 rows in the ring -----------------------
    float out[V];
    {
        int du = -2, dd = 0;   // rows R-1 and R+1 relative to R0
        if (SP) {
            const int R = R0 - 1;
            du = max(R - 1, 0) - R0;
            dd = min(R0, c.ny - 1) - R0;
        }
        const float *fu = c.ringF + ((i + du) & (C::NBF - 1)) * C::BX;
        const float *fm = c.ringF + ((i - 1) & (C::NBF - 1)) * C::BX;
        const float *fd = c.ringF + ((i + dd) & (C::NBF - 1)) * C::BX;
        const int o = c.tid * V;
        float u[V], m[V], d[V], wv[V], ev[V];
        ld_smem_row<V>(fu + o, u);
        ld_smem_row<V>(fm + o, m);
        ld_smem_row<V>(fd + o, d);
        const float w_in = fm[o > 0 ? o - 1 : 0];
        const float e_in = fm[o + V < C::BX ? o + V : C::BX - 1];
        neighbours<V, ED>(c, m, w_in, e_in, wv, ev);
        float pv[C::NPL][V];
        if (KIND != KDIFF) ld_planes<V, C::NPL, C::NBP, C::BX>(c.ringP, (i - 1) & (C::NBP - 1), o, pv);
#pragma unroll
        for (int j = 0; j < V; j++) {
            float q[C::NPL];
#pragma unroll
            for (int pl = 0; pl < C::NPL; pl++) q[pl] = KIND != KDIFF ? pv[pl][j] : 0.f;
            out[j] = upd2q<KIND, EXACT, C::NPL>(c, m[j], wv[j], ev[j], d[j], u[j], q);
        }
    }
    if constexpr (T == 1) {
        const int R = R0 - 1;
        if (R >= c.s0 && R < c.s1) store_row<V>(c, R, out);
        return;
    } else {
        tb2_stages<KIND, EXACT, T, V, W, P, MODE>(c, B, i, R0, out);
    }
}

// Stages 1 .. T-1 of one row iteration (T > 1).
template <int KIND, bool EXACT, int T, int V, int W, int P, int MODE>
__device__ __forceinline__ void tb2_stages(const Ctx2 &c,
                                           float (&B)[TB2<KIND, EXACT, T, V, W>::NS][3][V], int i,
                                           int R0, float (&out)[V])
{
    using C = TB2<KIND, EXACT, T, V, W>;
    constexpr bool SP = MODE == MODE_SPECIAL;
    constexpr bool ED = MODE != MODE_PLAIN;
    constexpr int PU = P, PM = (P + 1) % 3, PD = (P + 2) % 3;
    // exchange blocks: this row's outputs go to parity i&1, the rows read now came from (i-1)&1
    float *xw = c.xch + (i & 1) * (C::NX > 0 ? C::NX : 1) * C::XB + c.xw_off;
    const float *xr = c.xch + ((i - 1) & 1) * (C::NX > 0 ? C::NX : 1) * C::XB + c.xr_off;

    // hand stage 0's row to stage 1
#pragma unroll
    for (int j = 0; j < V; j++) B[0][PD][j] = out[j];
    if (C::NX > 0) xw[0] = c.is0 ? out[0] : out[V - 1];

#pragma unroll
    for (int s = 1; s < T; s++) {
        const int R = R0 - 1 - s;   // row this stage produces (time s+1)
        float(&Ws)[3][V] = B[s - 1];
        if (SP && s >= c.tsteps) {
            // beyond this pass's step count: forward the time-s row unchanged
#pragma unroll
            for (int j = 0; j < V; j++) out[j] = Ws[PM][j];
        } else {
            if (SP && R == c.ny - 1) {   // bottom edge: row ny is row ny-1
#pragma unroll
                for (int j = 0; j < V; j++) Ws[PD][j] = Ws[PM][j];
            }
            float w_in, e_in;
            {
                float vw = Ws[PM][V - 1], ve = Ws[PM][0];
                if (C::NX > 0) {
                    const float X = xr[(s - 1) * C::XB];
                    vw = c.is31 ? X : vw;
                    ve = c.is0 ? X : ve;
                }
                w_in = __shfl_sync(0xffffffffu, vw, (c.lane + 31) & 31);
                e_in = __shfl_sync(0xffffffffu, ve, (c.lane + 1) & 31);
            }
            float wv[V], ev[V];
            neighbours<V, ED>(c, Ws[PM], w_in, e_in, wv, ev);
            float pv[C::NPL][V];
            if (KIND != KDIFF)
                ld_planes<V, C::NPL, C::NBP, C::BX>(c.ringP, (i - 1 - s) & (C::NBP - 1), c.tid * V, pv);
#pragma unroll
            for (int j = 0; j < V; j++) {
                float q[C::NPL];
#pragma unroll
                for (int pl = 0; pl < C::NPL; pl++) q[pl] = KIND != KDIFF ? pv[pl][j] : 0.f;
                out[j] = upd2q<KIND, EXACT, C::NPL>(c, Ws[PM][j], wv[j], ev[j], Ws[PD][j],
                                                    Ws[PU][j], q);
            }
            if (SP && R == -1) {   // top edge: the next window's row -1 is row 0
#pragma unroll
                for (int j = 0; j < V; j++) Ws[PM][j] = Ws[PD][j];
            }
        }
        if (s < T - 1) {
#pragma unroll
            for (int j = 0; j < V; j++) B[s][PD][j] = out[j];
            if (C::NX > 0) xw[s * C::XB] = c.is0 ? out[0] : out[V - 1];
        } else {
            if (R >= c.s0 && R < c.s1) store_row<V>(c, R, out);
        }
    }
}

template <int KIND, bool EXACT, int T, int V, int W>
__global__ void __launch_bounds__(32 * W) k_tb2d(const Pass2D p)
{
    using C = TB2<KIND, EXACT, T, V, W>;
    extern __shared__ __align__(16) float smem[];
    Ctx2 c;
    c.in = p.in;
    c.out = p.out;
    c.pw = p.pw;
    c.ld_in = p.ld_in;
    c.ld_out = p.ld_out;
    c.ld_pw = p.ld_pw;
    c.pw_plane = p.pw_plane;
    c.ringF = smem;
    c.ringP = smem + C::NBF * C::BX;
    c.xch = c.ringP + C::NPL * C::NBP * C::BX;
    c.nx = p.nx;
    c.ny = p.ny;
    c.tsteps = p.tsteps;
    c.vec_in = p.vec_in;
    c.vec_out = p.vec_out;
    c.vec_pw = p.vec_pw;
    c.tid = threadIdx.x;
    c.lane = threadIdx.x & 31;
    c.wid = threadIdx.x >> 5;
    c.is0 = c.lane == 0;
    c.is31 = c.lane == 31;
    c.k0 = p.k[0]; c.k1 = p.k[1]; c.k2 = p.k[2]; c.k3 = p.k[3]; c.k4 = p.k[4];
    // exchange slots: 2*(w+1) = left edge of warp w, 2*(w+1)+1 = its right edge; slot 2*(W+2)
    // is the spare one that lanes 1..30 write.  Lane 31 reads the left warp's right edge,
    // lane 0 (and, harmlessly, every other lane) the right warp's left edge.
    c.xr_off = c.is31 ? (c.wid * 2 + 1) : ((c.wid + 2) * 2 + 0);
    c.xw_off = c.is0 ? (c.wid + 1) * 2 : (c.is31 ? (c.wid + 1) * 2 + 1 : (W + 2) * 2);

    float B[C::NS][3][V];
#pragma unroll
    for (int s = 0; s < C::NS; s++)
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int j = 0; j < V; j++) B[s][q][j] = 0.f;

    long long f = (long long)blockIdx.x * p.rows_per_cta;
    const long long fend = min(f + p.rows_per_cta, p.total_rows);
    while (f < fend) {
        const int tx = (int)(f / p.ny);
        const int s0 = (int)(f - (long long)tx * p.ny);
        const int s1 = (int)min((long long)p.ny, (long long)s0 + (fend - f));
        f += s1 - s0;

        c.s0 = s0;
        c.s1 = s1;
        c.x0 = tx * C::CX - C::H;
        c.xt = c.x0 + c.tid * V;
        c.y_start = max(0, s0 - c.tsteps);
        c.last_row = min(c.ny - 1, s1 - 1 + c.tsteps);
        {
            const int lcl = (c.xt <= 0 && 0 < c.xt + V) ? -c.xt : -1;
            const int rcl = (c.xt <= c.nx - 1 && c.nx - 1 < c.xt + V) ? (c.nx - 1 - c.xt) : -1;
            c.lmask = lcl >= 0 ? (1u << lcl) : 0u;
            c.rmask = rcl >= 0 ? (1u << rcl) : 0u;
            c.edge = __any_sync(0xffffffffu, lcl >= 0 || rcl >= 0);
        }
        {
            const int lo = max(c.x0 + C::H, 0), hi = min(c.x0 + C::H + C::CX, c.nx);
            c.st_lo = min(max(lo - c.xt, 0), V);
            c.st_hi = min(max(hi - c.xt, 0), V);
            c.st_full = c.vec_out && c.st_lo == 0 && c.st_hi == V;
        }
        const int n_it = s1 + T - c.y_start;   // stage T-1 emits row s1-1 at i = n_it-1
        const int bot_i = c.ny - c.y_start;    // from here on a stage may sit on row ny-1
        const bool top = (c.y_start == 0);
        const bool partial = (c.tsteps < T);

#pragma unroll 1
        for (int j = 0; j < C::PF; j++) {
            const int y = c.y_start + j;
            if (y <= c.last_row)
                tb2_load_row<KIND, C::BX, C::NT, C::NPL, C::NBP>(c, y, c.ringF + (j & (C::NBF - 1)) * C::BX,
                                                 c.ringP + (j & (C::NBP > 0 ? C::NBP - 1 : 0)) * C::BX);
            cp_async_commit();
        }

        int i = 0;
#define STN_TB2_STEP(PH)                                                                       \
    if (i < n_it) {                                                                            \
        cp_async_wait<C::PF - 1>();                                                            \
        tb2_sync<C::NT>();                                                                     \
        if (partial || (top && i <= T) || i >= bot_i)                                          \
            tb2_iter<KIND, EXACT, T, V, W, PH, MODE_SPECIAL>(c, B, i);                         \
        else if (c.edge)                                                                       \
            tb2_iter<KIND, EXACT, T, V, W, PH, MODE_EDGE>(c, B, i);                            \
        else                                                                                   \
            tb2_iter<KIND, EXACT, T, V, W, PH, MODE_PLAIN>(c, B, i);                           \
        {                                                                                      \
            const int y = c.y_start + i + C::PF;                                               \
            if (y <= c.last_row)                                                               \
                tb2_load_row<KIND, C::BX, C::NT, C::NPL, C::NBP>(                              \
                    c, y, c.ringF + ((i + C::PF) & (C::NBF - 1)) * C::BX,                      \
                    c.ringP + ((i + C::PF) & (C::NBP > 0 ? C::NBP - 1 : 0)) * C::BX);          \
            cp_async_commit();                                                                 \
        }                                                                                      \
        ++i;                                                                                   \
    }
#pragma unroll 1
        while (i < n_it) {
            STN_TB2_STEP(0)
            STN_TB2_STEP(1)
            STN_TB2_STEP(2)
        }
#undef STN_TB2_STEP
        cp_async_wait<0>();
        tb2_sync<C::NT>();
    }
}

}  // namespace stn
