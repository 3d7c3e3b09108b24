// Reverse-mode gradient of a 2D run: the adjoint (transposed-stencil) sweep.
//
// One Jacobi step (arXiv 1802.00438, Sec. 2.1, Table 2 updates, clamped boundary) is affine in
// the field: u_{t+1} = A u_t + b(theta, p).  For a scalar loss with upstream gradient
// w = dL/du_N the adjoint recursion is
//     lambda_N = w,   lambda_t = A^T lambda_{t+1},   dL/du_0 = lambda_0,
//     dL/dtheta = sum_{t<N} sum_i lambda_{t+1}[i] dF_i/dtheta(u_t),
//     dL/dp_i   = k_dt * sum_{t=1..N} lambda_t[i]            (Hotspot: dF_i/dp_i = k_dt).
// A^T is again a five-point stencil with the forward weights moved to the mirrored neighbours:
//     (A^T l)_j = wc l_j + ww l_{x+1} + we l_{x-1} + ws l_{y-1} + wn l_{y+1}
// with out-of-domain l = 0, plus, at the domain edges, the weight of every clamped neighbour
// that the forward step folded into cell j (x = 0: ww, x = nx-1: we, y = 0: wn, y = ny-1: ws).
//
// GPU design.  The reverse sweep is temporally blocked like the forward sweep (Sec. 3.2): a
// pass loads a 128 x 32 tile of lambda_{t+TA} with a halo of TA cells into shared memory and
// applies TA transposed steps there (ping-pong buffers, redundant halo work, only the compute
// block written).  With rows on 16-byte boundaries the lambda tile, the power tile and the
// state tile u_t of every fused step arrive by tensor-map bulk copies (one elected thread,
// mbarrier completion, every step's state tile requested when the tile starts);
// otherwise the kernel reads them with plain loads.  The same pass accumulates the coefficient
// and power gradients of its compute block from the forward states u_t, which are recomputed
// from checkpoints every K steps into a K-state buffer (one trajectory run of this library per
// segment: 8 fused steps per launch, every step written out).  Coefficient gradients
// are float32 sums in a fixed order: each thread sums its own cells and steps of a pass (at most
// 64 terms, fused multiply-adds), then blocks and two final launches combine those partial sums
// as (hi, lo) pairs with error-free transformations (TwoSum) in a fixed tree, so results are
// deterministic and the rounding of the combination is negligible beside the per-thread sums.  Alongside each gradient the
// same reduction yields sum |term|, the scale its rounding error is relative to.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

namespace {

// 128 x 32 tiles in 256-thread blocks, two blocks per SM: one block's copies land while the
// other computes (128 x 64 tiles in one 512-thread block per SM left HBM idle between tiles)
constexpr int AX = 128, AY = 32, ANT = 256, ACPT = AX * AY / ANT;   // tile, threads, cells/thread
static_assert(AX == 4 * 32 && AY == 4 * (ANT / 32), "a lane owns 4 x 4 cells of the tile");
constexpr int ATA = 4;                                                // fused adjoint steps
// halos: ATA rows in y; in x at least ATA cells and a multiple of 4, so that every tile origin
// (a tensor-map copy's innermost coordinate) stays on a 16-byte boundary
constexpr int AHX = (ATA + 3) / 4 * 4;
constexpr int ACX = AX - 2 * AHX, ACY = AY - 2 * ATA;                // compute block
// tile origin x = tx * ACX - AHX: a multiple of 4 floats for every tile (an unaligned innermost
// coordinate of a tensor-map copy is an illegal instruction)
static_assert(AHX % 4 == 0 && ACX % 4 == 0 && AHX >= ATA, "tile origins on 16-byte boundaries");
constexpr int NG = 5;                                                 // coefficients
constexpr int NPART = 3 * NG;                                         // (hi, lo, |.|) x 5

// dynamic shared memory of a pass: two lambda tiles, one state tile per fused step, and the
// power tile for Hotspot (7 x 16 KiB: two blocks and their static arrays fit in one SM)
constexpr int adj_smem(int kind)
{
    return (2 + ATA + (kind == ST_THERMAL ? 1 : 0)) * AX * AY * (int)sizeof(float);
}

struct AdjPass {
    const float *lam_in;     // lambda_{t_hi}
    float *lam_out;          // lambda_{t_lo}
    const float *states;     // u_{t0 + k} at states + k * n
    long long n;             // cells per grid
    int k_hi;                // index of u_{t_hi - 1} in states
    int nsteps;              // t_hi - t_lo, 1..ATA
    const float *pw;         // Hotspot power map
    float *gpw;              // Hotspot dL/dp (accumulated)
    int nx, ny, ntx;
    float wc, ww, we, ws, wn;   // forward weights of c, w, e, s, n
    float k[5];
    float *partials;         // this pass's [block][NPART]
    int use_tma;             // stage lambda, u and power tiles by tensor-map copies
    int *err;                // device flag: a bounded wait gave up
};

__device__ __forceinline__ uint32_t sm32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// bounded wait for phase `parity` (false: gave up)
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    for (int n = 0; n < (1 << 22); n++) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// one (AX x AY) box of plane z of a tensor map into shared memory, completing on `bar`
__device__ __forceinline__ void tile_copy(uint32_t dst, const CUtensorMap *m, int x, int y, int z,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void add_pair(float &hi, float &lo, float bhi, float blo)
{
    float s, e;
    two_sum(hi, bhi, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, blo));
    two_sum(s, e, hi, lo);
}

template <int KIND>
__device__ __forceinline__ void dfdtheta(const AdjPass &a, float c, float w, float e, float s,
                                         float n, float p, float (&g)[NG])
{
    if (KIND == ST_DIFFUSION) {   // [cc, cw, ce, cs, cn]
        g[0] = c; g[1] = w; g[2] = e; g[3] = s; g[4] = n;
    } else {                      // [k_dt, Rx, Ry, Rz, amb]
        const float c2 = __fmul_rn(2.0f, c);
        const float t1 = __fsub_rn(__fadd_rn(n, s), c2);
        const float t2 = __fsub_rn(__fadd_rn(e, w), c2);
        const float t3 = __fsub_rn(a.k[4], c);
        float q = __fmaf_rn(t1, a.k[2], p);
        q = __fmaf_rn(t2, a.k[1], q);
        q = __fmaf_rn(t3, a.k[3], q);
        g[0] = q;
        g[1] = __fmul_rn(a.k[0], t2);
        g[2] = __fmul_rn(a.k[0], t1);
        g[3] = __fmul_rn(a.k[0], t3);
        g[4] = __fmul_rn(a.k[0], a.k[3]);
    }
}

// Thread layout of a tile: lane L owns cells 4L .. 4L+3 of rows 4w .. 4w+3 of warp w; its
// cells are visited row by row, left to right (cell c = 4 r + j), on every path, so every
// path accumulates the same terms in the same order.
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// One transposed step on my 4 x 4 cells of a staged tile: the rows by 16-byte loads, the
// x-neighbours across lanes by shuffles; per cell the operations and their order are those of
// the general path.  EDGE = false: the tile lies inside the grid and off its edges (no clamp,
// no mask).  EDGE = true: any staged tile; cells off the grid are masked and the clamped
// neighbours of cells on the grid's edges are applied per cell (out-of-grid cells of the
// staged tiles arrive as zeros, as the general path reads them).
template <int KIND, bool ABS, bool EDGE>
__device__ __forceinline__ void adj_block(const AdjPass &a, int lane, int ly0, int x0, int y0,
                                          const float *cur, float *nxt, const float *ut,
                                          const float *ptile, float (&hi)[NG], float (&ab)[NG],
                                          float (&pacc)[ACPT])
{
    const int lx0 = 4 * lane;
    float L[6][4];   // lambda rows ly0-1 .. ly0+4 (zero beyond the tile)
#pragma unroll
    for (int rr = 0; rr < 6; rr++) {
        const int row = ly0 - 1 + rr;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row >= 0 && row < AY) v = lds4(cur + row * AX + lx0);
        L[rr][0] = v.x; L[rr][1] = v.y; L[rr][2] = v.z; L[rr][3] = v.w;
    }
    float wl[4], er[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        wl[r] = __shfl_sync(0xffffffffu, L[r + 1][3], (lane + 31) & 31);
        er[r] = __shfl_sync(0xffffffffu, L[r + 1][0], (lane + 1) & 31);
        if (lane == 0) wl[r] = 0.f;
        if (lane == 31) er[r] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        float o[4];
        const int gy = y0 + ly0 + r;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int gx = x0 + lx0 + j;
            const float le = j < 3 ? L[r + 1][j + 1] : er[r];
            const float lw = j > 0 ? L[r + 1][j - 1] : wl[r];
            float cs = a.wc;
            if (EDGE) {   // the weights of clamped neighbours fold into the diagonal
                if (gx == 0) cs = __fadd_rn(cs, a.ww);
                if (gx == a.nx - 1) cs = __fadd_rn(cs, a.we);
                if (gy == 0) cs = __fadd_rn(cs, a.wn);
                if (gy == a.ny - 1) cs = __fadd_rn(cs, a.ws);
            }
            float v = __fmul_rn(cs, L[r + 1][j]);
            v = __fmaf_rn(a.ww, le, v);
            v = __fmaf_rn(a.we, lw, v);
            v = __fmaf_rn(a.ws, L[r][j], v);
            v = __fmaf_rn(a.wn, L[r + 2][j], v);
            if (EDGE && !(gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny)) v = 0.f;
            o[j] = v;
        }
        *reinterpret_cast<float4 *>(nxt + (ly0 + r) * AX + lx0) = make_float4(o[0], o[1], o[2], o[3]);
    }
    // gradient terms of the compute block (its cells and their neighbours are in the tile);
    // the condition is warp-uniform, so every lane takes part in the shuffles below
    const bool rows_any = ly0 + 3 >= ATA && ly0 < ATA + ACY;
    if (rows_any) {
        float U[6][4];
#pragma unroll
        for (int rr = 0; rr < 6; rr++) {
            const int row = min(max(ly0 - 1 + rr, 0), AY - 1);   // only own cells' rows are used
            const float4 v = lds4(ut + row * AX + lx0);
            U[rr][0] = v.x; U[rr][1] = v.y; U[rr][2] = v.z; U[rr][3] = v.w;
        }
        float uw[4], ue[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            uw[r] = __shfl_sync(0xffffffffu, U[r + 1][3], (lane + 31) & 31);
            ue[r] = __shfl_sync(0xffffffffu, U[r + 1][0], (lane + 1) & 31);
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int ly = ly0 + r, gy = y0 + ly;
            if (ly < ATA || ly >= ATA + ACY) continue;
            if (EDGE && gy >= a.ny) continue;
            float pr[4] = {0.f, 0.f, 0.f, 0.f};
            if (KIND == ST_THERMAL) {
                const float4 v = lds4(ptile + ly * AX + lx0);
                pr[0] = v.x; pr[1] = v.y; pr[2] = v.z; pr[3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int lx = lx0 + j, gx = x0 + lx;
                if (lx < AHX || lx >= AHX + ACX) continue;
                if (EDGE && gx >= a.nx) continue;
                const float uc = U[r + 1][j];
                float uwj = j > 0 ? U[r + 1][j - 1] : uw[r];
                float uej = j < 3 ? U[r + 1][j + 1] : ue[r];
                float usj = U[r + 2][j], unj = U[r][j];
                if (EDGE) {   // clamp at the domain edges (own cells are never off the grid's start)
                    if (gx == 0) uwj = uc;
                    if (gx == a.nx - 1) uej = uc;
                    if (gy == 0) unj = uc;
                    if (gy == a.ny - 1) usj = uc;
                }
                float g[NG];
                dfdtheta<KIND>(a, uc, uwj, uej, usj, unj, pr[j], g);
                const float l = L[r + 1][j];
#pragma unroll
                for (int m = 0; m < NG; m++) {
                    hi[m] = __fmaf_rn(l, g[m], hi[m]);
                    if (ABS) ab[m] = __fmaf_rn(fabsf(l), fabsf(g[m]), ab[m]);
                }
                if (KIND == ST_THERMAL) pacc[4 * r + j] = __fadd_rn(pacc[4 * r + j], l);
            }
        }
    }
}

// ABS: also accumulate sum |term| per coefficient (only when the caller asks for it; the
// gradients themselves are the same sums in the same order either way)
template <int KIND, bool ABS>
__global__ void __launch_bounds__(ANT, 2) k_adj2d(const AdjPass a, const __grid_constant__ CUtensorMap tl,
                                               const __grid_constant__ CUtensorMap tu,
                                               const __grid_constant__ CUtensorMap tp)
{
    extern __shared__ __align__(128) float sm[];
    constexpr uint32_t TILE_B = 4u * AX * AY;
    float *buf0 = sm, *buf1 = sm + AX * AY;
    float *ubuf = sm + 2 * AX * AY;             // one state tile per fused step
    float *ptile = sm + (2 + ATA) * AX * AY;    // power tile (Hotspot)
    __shared__ float red[ANT / 32][NPART];
    __shared__ __align__(8) uint64_t bars[2 + ATA];   // lambda, power, state tiles 0 .. ATA-1
    const int tid = threadIdx.x;
    const int tx = blockIdx.x % a.ntx, ty = blockIdx.x / a.ntx;
    const int x0 = tx * ACX - AHX, y0 = ty * ACY - ATA;
    const bool tma = a.use_tma != 0;
    const uint32_t b0 = sm32(&bars[0]);
    // block-uniform: the whole tile is in the grid and no cell of it lies on the grid's edge
    const bool interior = tma && x0 >= 1 && y0 >= 1 && x0 + AX <= a.nx - 1 && y0 + AY <= a.ny - 1;

    // every copy of the tile is requested at once (lambda, power and the state tile of each
    // fused step, each on its own barrier, used once): the steps then wait only for their own
    // state tile, and one block keeps the whole tile's bytes in flight
    const auto drain = [&](int j0) {   // after a failed wait: let the copies in flight land
        for (int j = j0; j < a.nsteps; j++) (void)bar_wait(b0 + 8u * (2 + j), 0);
    };
    if (tma) {
        if (tid == 0) {
            for (int b = 0; b < 2 + ATA; b++) bar_init(b0 + 8u * b);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            bar_expect(b0, TILE_B);
            tile_copy(sm32(buf0), &tl, x0, y0, 0, b0);
            if (KIND == ST_THERMAL) {
                bar_expect(b0 + 8u, TILE_B);
                tile_copy(sm32(ptile), &tp, x0, y0, 0, b0 + 8u);
            }
            for (int j = 0; j < a.nsteps; j++) {
                bar_expect(b0 + 8u * (2 + j), TILE_B);
                tile_copy(sm32(ubuf + j * AX * AY), &tu, x0, y0, a.k_hi - j, b0 + 8u * (2 + j));
            }
        }
        __syncthreads();   // barriers initialised before anyone polls them
        bool ok = bar_wait(b0, 0);
        if (KIND == ST_THERMAL) ok = bar_wait(b0 + 8u, 0) && ok;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(a.err, 1);
                (void)bar_wait(b0, 0);
                if (KIND == ST_THERMAL) (void)bar_wait(b0 + 8u, 0);
                drain(0);
            }
            return;
        }
    } else {
#pragma unroll
        for (int q = 0; q < ACPT; q++) {
            const int idx = tid + q * ANT, lx = idx % AX, ly = idx / AX;
            const int gx = x0 + lx, gy = y0 + ly;
            const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
            buf0[idx] = in ? a.lam_in[(long long)gy * a.nx + gx] : 0.f;
        }
        __syncthreads();
    }

    const int lane = tid & 31, lx0 = 4 * lane, ly0 = 4 * (tid >> 5);   // my 4 x 4 cells
    float hi[NG], lo[NG], ab[NG], pacc[ACPT];
#pragma unroll
    for (int m = 0; m < NG; m++) hi[m] = lo[m] = ab[m] = 0.f;
#pragma unroll
    for (int q = 0; q < ACPT; q++) pacc[q] = 0.f;

    float *cur = buf0, *nxt = buf1;
    for (int j = 0; j < a.nsteps; j++) {
        const float *u = a.states + (long long)(a.k_hi - j) * a.n;   // u_t, t = t_hi - 1 - j
        const float *ut = ubuf + j * AX * AY;                        // its tile (staged path)
        if (tma) {
            const bool ok = bar_wait(b0 + 8u * (2 + j), 0);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicExch(a.err, 1);
                    drain(j);
                }
                return;
            }
        }
        if (interior) {
            adj_block<KIND, ABS, false>(a, lane, ly0, x0, y0, cur, nxt, ut, ptile, hi, ab, pacc);
        } else if (tma) {
            adj_block<KIND, ABS, true>(a, lane, ly0, x0, y0, cur, nxt, ut, ptile, hi, ab, pacc);
        } else {
#pragma unroll
            for (int c = 0; c < ACPT; c++) {
                const int lx = lx0 + (c & 3), ly = ly0 + (c >> 2), idx = ly * AX + lx;
                const int gx = x0 + lx, gy = y0 + ly;
                const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
                const float l = cur[idx];   // lambda_{t+1}
                const float le = lx + 1 < AX ? cur[idx + 1] : 0.f;
                const float lw = lx > 0 ? cur[idx - 1] : 0.f;
                const float ln = ly > 0 ? cur[idx - AX] : 0.f;
                const float ls = ly + 1 < AY ? cur[idx + AX] : 0.f;
                float cs = a.wc;
                if (gx == 0) cs = __fadd_rn(cs, a.ww);
                if (gx == a.nx - 1) cs = __fadd_rn(cs, a.we);
                if (gy == 0) cs = __fadd_rn(cs, a.wn);
                if (gy == a.ny - 1) cs = __fadd_rn(cs, a.ws);
                float r = __fmul_rn(cs, l);
                r = __fmaf_rn(a.ww, le, r);
                r = __fmaf_rn(a.we, lw, r);
                r = __fmaf_rn(a.ws, ln, r);
                r = __fmaf_rn(a.wn, ls, r);
                nxt[idx] = in ? r : 0.f;
                const bool own = in && lx >= AHX && lx < AHX + ACX && ly >= ATA && ly < ATA + ACY;
                if (own) {
                    float g[NG];
                    if (tma) {
                        // own cells are ATA >= 1 cells inside the tile; clamp at the domain edges
                        const int dw = gx > 0 ? 1 : 0, de = gx < a.nx - 1 ? 1 : 0;
                        const int dn = gy > 0 ? AX : 0, dsn = gy < a.ny - 1 ? AX : 0;
                        const float p = KIND == ST_THERMAL ? ptile[idx] : 0.f;
                        dfdtheta<KIND>(a, ut[idx], ut[idx - dw], ut[idx + de], ut[idx + dsn],
                                       ut[idx - dn], p, g);
                    } else {
                        const long long o = (long long)gy * a.nx;
                        const int xw = gx > 0 ? gx - 1 : 0, xe = gx < a.nx - 1 ? gx + 1 : a.nx - 1;
                        const long long on = (long long)(gy > 0 ? gy - 1 : 0) * a.nx;
                        const long long os = (long long)(gy < a.ny - 1 ? gy + 1 : a.ny - 1) * a.nx;
                        const float p = KIND == ST_THERMAL ? __ldg(a.pw + o + gx) : 0.f;
                        dfdtheta<KIND>(a, __ldg(u + o + gx), __ldg(u + o + xw), __ldg(u + o + xe),
                                       __ldg(u + os + gx), __ldg(u + on + gx), p, g);
                    }
#pragma unroll
                    for (int m = 0; m < NG; m++) {
                        hi[m] = __fmaf_rn(l, g[m], hi[m]);
                        if (ABS) ab[m] = __fmaf_rn(fabsf(l), fabsf(g[m]), ab[m]);
                    }
                    if (KIND == ST_THERMAL) pacc[c] = __fadd_rn(pacc[c], l);
                }
            }
        }
        __syncthreads();
        float *t = cur;
        cur = nxt;
        nxt = t;
    }

#pragma unroll
    for (int c = 0; c < ACPT; c++) {
        const int lx = lx0 + (c & 3), ly = ly0 + (c >> 2), idx = ly * AX + lx;
        const int gx = x0 + lx, gy = y0 + ly;
        const bool own = gx < a.nx && gy < a.ny && lx >= AHX && lx < AHX + ACX && ly >= ATA &&
                         ly < ATA + ACY;
        if (own) {
            const long long o = (long long)gy * a.nx + gx;
            a.lam_out[o] = cur[idx];
            if (KIND == ST_THERMAL) a.gpw[o] = __fmaf_rn(a.k[0], pacc[c], a.gpw[o]);
        }
    }

    // block reduction of the (hi, lo) pairs and the magnitudes, fixed order
    const int wid = tid >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int m = 0; m < NG; m++) {
            const float bh = __shfl_down_sync(0xffffffffu, hi[m], off);
            const float bl = __shfl_down_sync(0xffffffffu, lo[m], off);
            const float bb = __shfl_down_sync(0xffffffffu, ab[m], off);
            add_pair(hi[m], lo[m], bh, bl);
            ab[m] = __fadd_rn(ab[m], bb);
        }
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < NG; m++) {
            red[wid][3 * m + 0] = hi[m];
            red[wid][3 * m + 1] = lo[m];
            red[wid][3 * m + 2] = ab[m];
        }
    __syncthreads();
    if (wid == 0) {
        constexpr int NWP = ANT / 32;
#pragma unroll
        for (int m = 0; m < NG; m++) {
            hi[m] = lane < NWP ? red[lane][3 * m + 0] : 0.f;
            lo[m] = lane < NWP ? red[lane][3 * m + 1] : 0.f;
            ab[m] = lane < NWP ? red[lane][3 * m + 2] : 0.f;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int m = 0; m < NG; m++) {
                const float bh = __shfl_down_sync(0xffffffffu, hi[m], off);
                const float bl = __shfl_down_sync(0xffffffffu, lo[m], off);
                const float bb = __shfl_down_sync(0xffffffffu, ab[m], off);
                add_pair(hi[m], lo[m], bh, bl);
                ab[m] = __fadd_rn(ab[m], bb);
            }
        if (lane == 0)
#pragma unroll
            for (int m = 0; m < NG; m++) {
                a.partials[(long long)blockIdx.x * NPART + 3 * m + 0] = hi[m];
                a.partials[(long long)blockIdx.x * NPART + 3 * m + 1] = lo[m];
                a.partials[(long long)blockIdx.x * NPART + 3 * m + 2] = ab[m];
            }
    }
}

// Combine partial triples per coefficient in a fixed order, in two launches: block b of the
// first takes the `chunk` entries from b * chunk on and writes one triple to out[b]; the second
// (one block, out == nullptr) combines those and writes the gradients.  Within a block thread
// t takes entries t, t + 256, ... sequentially, then a fixed shuffle / shared-memory tree.  The
// partition depends only on the entry count, so the result is deterministic.
constexpr int ADJ_SUM_BLOCKS = 256;   // blocks of the first launch, at most

__global__ void __launch_bounds__(256) k_adj_final(const float *partials, long long count,
                                                   long long chunk, float *out, float *grad,
                                                   float *grad_abs)
{
    __shared__ float red[8][NPART];
    float hi[NG], lo[NG], ab[NG];
#pragma unroll
    for (int m = 0; m < NG; m++) hi[m] = lo[m] = ab[m] = 0.f;
    const long long i0 = (long long)blockIdx.x * chunk, i1 = min(count, i0 + chunk);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x)
#pragma unroll
        for (int m = 0; m < NG; m++) {
            add_pair(hi[m], lo[m], partials[i * NPART + 3 * m], partials[i * NPART + 3 * m + 1]);
            ab[m] = __fadd_rn(ab[m], partials[i * NPART + 3 * m + 2]);
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int m = 0; m < NG; m++) {
            const float bh = __shfl_down_sync(0xffffffffu, hi[m], off);
            const float bl = __shfl_down_sync(0xffffffffu, lo[m], off);
            const float bb = __shfl_down_sync(0xffffffffu, ab[m], off);
            add_pair(hi[m], lo[m], bh, bl);
            ab[m] = __fadd_rn(ab[m], bb);
        }
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < NG; m++) {
            red[wid][3 * m] = hi[m];
            red[wid][3 * m + 1] = lo[m];
            red[wid][3 * m + 2] = ab[m];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int m = 0; m < NG; m++) {
            float h = red[0][3 * m], l = red[0][3 * m + 1], s = red[0][3 * m + 2];
            for (int w = 1; w < 8; w++) {
                add_pair(h, l, red[w][3 * m], red[w][3 * m + 1]);
                s = __fadd_rn(s, red[w][3 * m + 2]);
            }
            if (out) {
                out[(long long)blockIdx.x * NPART + 3 * m] = h;
                out[(long long)blockIdx.x * NPART + 3 * m + 1] = l;
                out[(long long)blockIdx.x * NPART + 3 * m + 2] = s;
            } else {
                grad[m] = __fadd_rn(h, l);
                if (grad_abs) grad_abs[m] = s;
            }
        }
    }
}

int status(cudaError_t e)
{
    if (e == cudaSuccess) return ST_OK;
    if (e == cudaErrorMemoryAllocation) return ST_ERR_OOM;
    return ST_ERR_CUDA;
}

}  // namespace

struct stencil_adjoint_s {
    int kind = 0, nx = 0, ny = 0, steps = 0, ckpt = 0, nseg = 0;
    cudaStream_t stream = nullptr;
    stencil_plan fwd = nullptr;   // forward runs and the trajectories between checkpoints
    float *ck = nullptr;      // nseg checkpoints: u at 0, K, 2K, ...
    float *seg = nullptr;     // K recomputed states of one segment
    float *lam[2] = {nullptr, nullptr};
    float *partials = nullptr;
    long long blocks = 0, passes = 0;
    float coef[5] = {0, 0, 0, 0, 0};
    bool have_forward = false;
    int *err = nullptr;       // device flag set by a kernel whose bounded wait gave up
};

extern "C" {

int stencil_adjoint_create(stencil_adjoint *out, int kind, int nx, int ny, int steps, int ckpt,
                           void *stream)
{
    if (!out) return ST_ERR_INVALID_ARG;
    *out = nullptr;
    if ((kind != ST_DIFFUSION && kind != ST_THERMAL) || nx < 1 || ny < 1 || steps < 0 ||
        ckpt < 1)
        return ST_ERR_INVALID_ARG;
    if ((long long)nx * ny > (1LL << 31)) return ST_ERR_INVALID_ARG;
    stencil_adjoint_s *a = new (std::nothrow) stencil_adjoint_s;
    if (!a) return ST_ERR_OOM;
    a->kind = kind;
    a->nx = nx;
    a->ny = ny;
    a->steps = steps;
    a->ckpt = std::min(ckpt, std::max(steps, 1));
    a->nseg = steps > 0 ? (steps + a->ckpt - 1) / a->ckpt : 0;
    a->stream = static_cast<cudaStream_t>(stream);
    const int ntx = (nx + ACX - 1) / ACX, nty = (ny + ACY - 1) / ACY;
    a->blocks = (long long)ntx * nty;
    for (int sg = 0; sg < a->nseg; sg++) {
        const int len = std::min(steps, (sg + 1) * a->ckpt) - sg * a->ckpt;
        a->passes += (len + ATA - 1) / ATA;
    }
    int rc = ST_OK;
    stencil_desc d = {};
    d.kind = kind;
    d.ndim = 2;
    d.nx = nx;
    d.ny = ny;
    d.nz = 1;
    d.storage = ST_F32;
    d.stream = stream;
    rc = stencil_plan_create(&a->fwd, &d);
    const size_t n = (size_t)nx * ny * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (rc == ST_OK && a->nseg > 0) {
        e = stn::dev_malloc(&a->ck, n * a->nseg);
        if (e == cudaSuccess) e = stn::dev_malloc(&a->seg, n * a->ckpt);
        if (e == cudaSuccess) e = stn::dev_malloc(&a->lam[0], n);
        if (e == cudaSuccess) e = stn::dev_malloc(&a->lam[1], n);
        if (e == cudaSuccess)
            e = stn::dev_malloc(&a->partials, sizeof(float) * NPART *
                                             (size_t)(a->blocks * a->passes + ADJ_SUM_BLOCKS));
        if (e == cudaSuccess) e = stn::dev_malloc(&a->err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(a->err, 0, sizeof(int));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_adj2d<ST_DIFFUSION, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     adj_smem(ST_DIFFUSION));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_adj2d<ST_DIFFUSION, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     adj_smem(ST_DIFFUSION));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_adj2d<ST_THERMAL, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     adj_smem(ST_THERMAL));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_adj2d<ST_THERMAL, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     adj_smem(ST_THERMAL));
        if (e != cudaSuccess) rc = status(e);
    }
    if (rc != ST_OK) {
        stencil_adjoint_destroy(a);
        return rc;
    }
    *out = a;
    return ST_OK;
}

int stencil_adjoint_forward(stencil_adjoint a, const float *u0, const float *power,
                            const float *coeffs, float *u_out)
{
    if (!a || !u0 || !coeffs || !u_out) return ST_ERR_INVALID_ARG;
    if (a->kind == ST_THERMAL && !power) return ST_ERR_INVALID_ARG;
    if (a->kind == ST_DIFFUSION && power) return ST_ERR_INVALID_ARG;
    const stn::NvtxRange r("stencil_adjoint_forward");
    const size_t n = (size_t)a->nx * a->ny * sizeof(float);
    for (int i = 0; i < 5; i++) a->coef[i] = coeffs[i];
    a->have_forward = false;
    if (a->nseg == 0) {
        if (u_out != u0) {
            cudaError_t e = cudaMemcpyAsync(u_out, u0, n, cudaMemcpyDeviceToDevice, a->stream);
            if (e != cudaSuccess) return status(e);
        }
        a->have_forward = true;
        return ST_OK;
    }
    cudaError_t e = cudaMemcpyAsync(a->ck, u0, n, cudaMemcpyDeviceToDevice, a->stream);
    if (e != cudaSuccess) return status(e);
    const long long cells = (long long)a->nx * a->ny;
    for (int sg = 0; sg < a->nseg; sg++) {
        const int len = std::min(a->steps, (sg + 1) * a->ckpt) - sg * a->ckpt;
        float *dst = sg + 1 < a->nseg ? a->ck + (sg + 1) * cells : u_out;
        const int rc = stencil_run(a->fwd, a->ck + sg * cells, dst, power, a->coef, a->nx, a->ny,
                                   1, len);
        if (rc != ST_OK) return rc;
    }
    a->have_forward = true;
    return ST_OK;
}

int stencil_adjoint_backward(stencil_adjoint a, const float *grad_out, const float *power,
                             float *grad_u0, float *grad_coeffs, float *grad_coeffs_abs,
                             float *grad_power)
{
    if (!a || !grad_out || !grad_u0 || !grad_coeffs) return ST_ERR_INVALID_ARG;
    if (!a->have_forward) return ST_ERR_INVALID_ARG;
    if (a->kind == ST_THERMAL && (!power || !grad_power)) return ST_ERR_INVALID_ARG;
    if (a->kind == ST_DIFFUSION && (power || grad_power)) return ST_ERR_INVALID_ARG;
    const stn::NvtxRange r("stencil_adjoint_backward");
    const long long cells = (long long)a->nx * a->ny;
    const size_t n = (size_t)cells * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (grad_power) e = cudaMemsetAsync(grad_power, 0, n, a->stream);
    if (e == cudaSuccess && a->nseg == 0) {
        e = cudaMemcpyAsync(grad_u0, grad_out, n, cudaMemcpyDeviceToDevice, a->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(grad_coeffs, 0, NG * sizeof(float), a->stream);
        if (e == cudaSuccess && grad_coeffs_abs)
            e = cudaMemsetAsync(grad_coeffs_abs, 0, NG * sizeof(float), a->stream);
        return status(e);
    }
    if (e != cudaSuccess) return status(e);

    AdjPass p = {};
    p.n = cells;
    p.pw = power;
    p.gpw = grad_power;
    p.nx = a->nx;
    p.ny = a->ny;
    p.ntx = (a->nx + ACX - 1) / ACX;
    for (int i = 0; i < 5; i++) p.k[i] = a->coef[i];
    if (a->kind == ST_DIFFUSION) {
        p.wc = a->coef[0];
        p.ww = a->coef[1];
        p.we = a->coef[2];
        p.ws = a->coef[3];
        p.wn = a->coef[4];
    } else {
        // Hotspot: F = c + k_dt (p + (n+s-2c) Ry + (e+w-2c) Rx + (amb-c) Rz)
        const double kdt = a->coef[0], rx = a->coef[1], ry = a->coef[2], rz = a->coef[3];
        p.wc = (float)(1.0 - kdt * (2.0 * ry + 2.0 * rx + rz));
        p.ww = p.we = (float)(kdt * rx);
        p.ws = p.wn = (float)(kdt * ry);
    }
    // tensor maps of the adjoint grids, the state buffer and the power map (rows on 16-byte
    // boundaries only; otherwise the kernel reads with plain loads)
    stn::Tma3D mo, m0, m1, ms, mp;
    std::memset(&mo, 0, sizeof(mo));
    m0 = m1 = ms = mp = mo;
    bool tma = stn::tma3d_encode(&mo.in, grad_out, a->nx, a->ny, 1, AX, AY) &&
               stn::tma3d_encode(&m0.in, a->lam[0], a->nx, a->ny, 1, AX, AY) &&
               stn::tma3d_encode(&m1.in, a->lam[1], a->nx, a->ny, 1, AX, AY) &&
               stn::tma3d_encode(&ms.in, a->seg, a->nx, a->ny, a->ckpt, AX, AY);
    if (tma && power) tma = stn::tma3d_encode(&mp.in, power, a->nx, a->ny, 1, AX, AY);
    p.use_tma = tma ? 1 : 0;
    p.err = a->err;
    const int smem = adj_smem(a->kind);
    const float *lin = grad_out;
    int which = 0;
    long long pass = 0;
    for (int sg = a->nseg - 1; sg >= 0 && e == cudaSuccess; sg--) {
        const int t0 = sg * a->ckpt, t1 = std::min(a->steps, t0 + a->ckpt), len = t1 - t0;
        // recompute u_{t0} .. u_{t1-1} into the segment buffer
        e = cudaMemcpyAsync(a->seg, a->ck + sg * cells, n, cudaMemcpyDeviceToDevice, a->stream);
        if (len > 1 && e == cudaSuccess) {   // u_{t0+1} .. u_{t1-1}: one trajectory run
            const int rc = stencil_run_trajectory(a->fwd, a->seg, a->seg + cells, cells, power,
                                                  a->coef, len - 1);
            if (rc != ST_OK) return rc;
        }
        int t_hi = t1;
        while (t_hi > t0 && e == cudaSuccess) {
            const int ns = std::min(ATA, t_hi - t0);
            p.lam_in = lin;
            p.lam_out = a->lam[which];
            p.states = a->seg;
            p.k_hi = t_hi - 1 - t0;
            p.nsteps = ns;
            p.partials = a->partials + (size_t)pass * a->blocks * NPART;
            const CUtensorMap &tl = lin == grad_out ? mo.in : (lin == a->lam[0] ? m0.in : m1.in);
            const bool abs_sums = grad_coeffs_abs != nullptr;
            const dim3 grid((unsigned)a->blocks);
            if (a->kind == ST_DIFFUSION) {
                if (abs_sums)
                    k_adj2d<ST_DIFFUSION, true><<<grid, ANT, smem, a->stream>>>(p, tl, ms.in, mp.in);
                else
                    k_adj2d<ST_DIFFUSION, false><<<grid, ANT, smem, a->stream>>>(p, tl, ms.in, mp.in);
            } else {
                if (abs_sums)
                    k_adj2d<ST_THERMAL, true><<<grid, ANT, smem, a->stream>>>(p, tl, ms.in, mp.in);
                else
                    k_adj2d<ST_THERMAL, false><<<grid, ANT, smem, a->stream>>>(p, tl, ms.in, mp.in);
            }
            e = cudaGetLastError();
            lin = a->lam[which];
            which ^= 1;
            t_hi -= ns;
            pass++;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad_u0, lin, n, cudaMemcpyDeviceToDevice, a->stream);
    if (e == cudaSuccess) {
        const long long count = pass * a->blocks;
        const long long chunk = std::max<long long>(1, (count + ADJ_SUM_BLOCKS - 1) / ADJ_SUM_BLOCKS);
        const long long nb = (count + chunk - 1) / chunk;   // <= ADJ_SUM_BLOCKS
        float *stage = a->partials + (size_t)a->blocks * a->passes * NPART;
        k_adj_final<<<(unsigned)std::max<long long>(nb, 1), 256, 0, a->stream>>>(
            a->partials, count, chunk, stage, nullptr, nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_adj_final<<<1, 256, 0, a->stream>>>(stage, nb, std::max<long long>(nb, 1), nullptr,
                                                  grad_coeffs, grad_coeffs_abs);
            e = cudaGetLastError();
        }
    }
    return status(e);
}

int stencil_adjoint_sync(stencil_adjoint a)
{
    if (!a) return ST_ERR_INVALID_ARG;
    cudaError_t e = a->stream ? cudaStreamSynchronize(a->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return status(e);
    int flag = 0;
    e = cudaMemcpy(&flag, a->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status(e);
    if (flag) {
        (void)cudaMemset(a->err, 0, sizeof(int));
        return ST_ERR_TIMEOUT;
    }
    return ST_OK;
}

int stencil_adjoint_destroy(stencil_adjoint a)
{
    if (!a) return ST_OK;
    if (a->stream) cudaStreamSynchronize(a->stream);
    else cudaDeviceSynchronize();
    if (a->fwd) stencil_plan_destroy(a->fwd);
    if (a->ck) stn::dev_free(a->ck);
    if (a->seg) stn::dev_free(a->seg);
    for (float *l : a->lam)
        if (l) stn::dev_free(l);
    if (a->partials) stn::dev_free(a->partials);
    if (a->err) stn::dev_free(a->err);
    delete a;
    return ST_OK;
}

}  // extern "C"
