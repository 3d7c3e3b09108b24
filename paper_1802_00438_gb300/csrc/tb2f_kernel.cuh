// 2D temporally-blocked Jacobi sweep, contracted arithmetic (fused multiply-adds): one pass
// advances the grid by `tsteps` (<= T) steps.
//
// Same blocking as the exact kernel (tb2d_kernel.cuh; arXiv 1802.00438 Sec. 3.1-3.2, Eq. 2):
// an overlapped x-tile streamed along y through a chain of T stages, stage s computing time
// step s+1 one row behind stage s-1, halos computed redundantly, only the compute block stored,
// trailing stages forwarding when the pass fuses fewer than T steps, clamped boundary
// (Sec. 5.1) at every stage.
//
// What differs is how a stage holds its window.  When row y of time s reaches stage s it
// completes row y-1 and starts rows y and y+1:
//   out(y-1) = P + cs * d                      (the only operation on the stage-to-stage path)
//   P'       = Q + cc * d + cw * d_w + ce * d_e  (row y, missing only its south term)
//   Q'       = cn * d                           (row y+1's north term)
// Hotspot 2D, c + sdc*(p + (n+s-2c)*Ry + (e+w-2c)*Rx + (amb-c)*Rz), uses the same split of its
// expansion cc*c + cx*(e+w) + cy*(n+s) - cz*c + src (cx = sdc*Rx, cy = sdc*Ry, cz = sdc*Rz,
// cc = 1 - 2cx - 2cy exact in float32, src = sdc*(p + amb*Rz) a per-cell map built once per run):
//   out(y-1) = P + cy * d
//   P'       = Q + cx * (d_e + d_w) + cc * d - cz * d
//   Q'       = cy * d + src(y+1)
// P' accumulates on top of Q and Q' is written where P was, so the two partial rows trade
// places every row: the row loop is unrolled twice with the roles swapped and every update is
// in place (no register copies).  Counted work per cell is unchanged (Table 2: 9 and 15 flops,
// issued as 5 and 6 operations; the plain-power Hotspot instances of the allocation-free entry
// point issue 9).
//
// GPU mapping: one warp per block; a tile is BX = 32*V cells wide incl. halos of
// H = roundup(T, 4) cells per side; thread = V consecutive cells; x-neighbours of a thread's
// edge cells by shuffle (the warp edge is the tile edge, inside the halo).  Field and power
// rows arrive through shared-memory rings filled by cp.async PF rows ahead.  The power ring
// keeps a mirrored copy of its first PW-1 slots, so the PW = max(T, 2) power rows an
// iteration reads are
// consecutive slots: one base address per row, constant offsets per stage.  Stage 0 needs no
// partial rows: its three time-0 rows are all in the field ring, and it evaluates the update
// from them directly.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tb2d_kernel.cuh"

namespace stn {

enum { STOR_F32 = 0, STOR_BF16 = 1, STOR_F16 = 2 };
// Flag added to STOR (Hotspot): the power ring holds the source map sdc*(p + amb*Rz) instead of
// p, and the coefficients are the expanded weights (hot_coeffs_src), so a stage issues six
// operations per cell instead of nine.  Float32 plans stage a map built once per run; 16-bit
// plans code the map itself in place of the power map.
__host__ __device__ constexpr int stor_fmt(int s) { return s & 3; }
__host__ __device__ constexpr bool stor_src(int s) { return (s & STOR_SRC) != 0; }
__host__ __device__ constexpr bool stor_all(int s) { return (s & STOR_ALL) != 0; }

template <int KIND, int T, int V, int STOR = STOR_F32>
struct TB2F {
    static constexpr int BX = 32 * V;
    static constexpr int H = (T + 3) / 4 * 4;
    static constexpr int CX = BX - 2 * H;
    static constexpr int PF = 4;                                    // rows requested ahead
    // 16-bit storage: the rows in flight wait in the staging rings, so the float rings hold
    // only the rows in use (decoded on arrival); float32 rows land in the float rings directly
    static constexpr bool Q16 = stor_fmt(STOR) != STOR_F32;
    static constexpr int NBF = Q16 ? 3 : PF + 3;                    // field rows i-2 .. i(+PF)
    static constexpr int PW = T > 1 ? T : 2;                        // power rows read per row:
                                                                    // i-PW+1 .. i
    static constexpr int NBP = (KIND == KTHERM) ? (Q16 ? PW : PW + PF + 1) : 0;   // power ring
    static constexpr int NBPX = (KIND == KTHERM) ? (NBP + PW - 1) : 0;  // incl. mirror
    static constexpr int NS = T > 1 ? T - 1 : 1;                    // partial-sum stages
    static constexpr int ROWB = BX * 4;                             // bytes per ring row
    // 16-bit storage: rows arrive raw (32-byte header of block codes + 2 bytes per cell) in a
    // staging ring of PF+1 rows per input and are decoded into the float rings once
    static constexpr int NBR = Q16 ? PF + 1 : 0;
    static constexpr int RAWB = 32 + 2 * BX;
    static constexpr size_t SMEM = (size_t)(NBF + NBPX) * ROWB +
                                   (size_t)NBR * RAWB * (KIND == KTHERM ? 2 : 1);
    static_assert(V % 4 == 0 && V <= 8, "V must be 4 or 8");
    // 16-bit storage: a lane decodes its V cells with one block code, so block boundaries
    // (every CX cells from the tile's first compute cell, H cells in) must fall between lanes
    static_assert(stor_fmt(STOR) == STOR_F32 || H % V == 0, "16-bit blocks split a lane's cells");
    static_assert(CX > 0, "tile narrower than its halos");
};

struct CoefF {
    // diffusion: cc, cw, ce, cs, cn; Hotspot: sdc, Rx, Ry, Rz, amb, sdc*Ry, -2*Ry; source-map
    // Hotspot kernels (STOR_SRC): cc, cx, cy, cz, amb, cy, 0 (host-made, hot_coeffs_src)
    float a0, a1, a2, a3, a4, a5, a6;
};

__device__ __forceinline__ float4 lds128(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}

__device__ __forceinline__ float lds32(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
    return v;
}

// Ring rows are stored with their 16-byte chunks rotated inside each 128-byte group: chunk g
// (cells 4g .. 4g+3) sits at chunk position ring_pos(g).  A warp's 16-byte accesses are served
// eight lanes at a time, so they are conflict-free when those eight lanes hit eight different
// 16-byte bank groups.  The copies into a row (lane L writes chunk L + 32q) and, with V = 8,
// the reads of a thread's own cells (lane L reads chunks 2L and 2L + 1) would otherwise meet
// only four bank groups per eight lanes; with the rotation both meet all eight.
__host__ __device__ constexpr uint32_t ring_pos(uint32_t g)
{
    return (g & ~7u) | ((g + (g >> 3)) & 7u);
}

// byte offset of cell x in a ring row
__host__ __device__ constexpr uint32_t ring_cell(uint32_t x)
{
    return 16u * ring_pos(x >> 2) + 4u * (x & 3u);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, int nbytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
                 : "memory");
}

__device__ __forceinline__ void cp4(uint32_t dst, const void *src, int nbytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
                 : "memory");
}

__device__ __forceinline__ void cp8(uint32_t dst, const void *src, int nbytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
                 : "memory");
}

__device__ __forceinline__ uint2 lds64u(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts128(uint32_t a, float x, float y, float z, float w)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(x), "f"(y), "f"(z),
                 "f"(w)
                 : "memory");
}

// 16-bit codes: bf16 / fp16 bit patterns of q in [-1, 1]
template <int STOR>
__device__ __forceinline__ float q2f(unsigned q)
{
    if (stor_fmt(STOR) == STOR_BF16) return __uint_as_float(q << 16);
    return __half2float(__ushort_as_half((unsigned short)q));
}

// two codes packed in one word (first argument in the low half), each rounded to nearest even
template <int STOR>
__device__ __forceinline__ unsigned f2q2(float a, float b)
{
    if (stor_fmt(STOR) == STOR_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const unsigned *>(&h);
    }
    // fp16 stops at 65504: a block whose cells lie further than that from its offset
    // saturates instead of storing an infinity
    const __half2 h = __floats2half2_rn(fminf(fmaxf(a, -65504.f), 65504.f),
                                        fminf(fmaxf(b, -65504.f), 65504.f));
    return *reinterpret_cast<const unsigned *>(&h);
}

struct CtxF {
    const float *__restrict__ in;
    float *__restrict__ out;
    const float *__restrict__ pw;
    long long ld_in, ld_out, ld_pw;
    uint32_t sF, sP;       // shared byte addresses of the field and power rings
    int nx, ny, tsteps;
    int x0, xt;
    int y_start, last_row, s0, s1;
    unsigned lmask, rmask;
    int st_lo, st_hi;
    bool st_full, st_any, edge;
    int vec_in, vec_out, vec_pw;
    int lane;
    uint32_t oq[2];        // byte offsets in a ring row of my cells' 16-byte chunks
    uint32_t wq[2];        // byte offsets of the chunks I copy into a ring row
    uint32_t ow4, oe4;     // byte offsets of the cells left and right of mine (clamped)
    // 16-bit storage
    uint32_t sRF, sRP;     // staging rings (raw field / raw power rows)
    const uint16_t *qin, *qpw;
    uint16_t *qout;
    const float2 *min_, *mpw;   // block codes (offset, scale) per (row, tile column)
    float2 *mout;
    long long ld_q;        // row pitch of 16-bit grids (cells)
    int ntx, tx;           // tile columns; my tile column
    int msel;              // which of the three blocks of a loaded row my cells belong to
    float *st_states;      // trajectory passes (STOR_ALL): where step t's rows go
    long long st_stride;
};

// my V cells of the ring row at byte address row
template <int V>
__device__ __forceinline__ void lds_row(uint32_t row, const CtxF &c, float (&v)[V])
{
#pragma unroll
    for (int q = 0; q < V / 4; q++) {
        const float4 t = lds128(row + c.oq[q]);
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}

template <int V, bool EDGE>
__device__ __forceinline__ void nbf(const CtxF &c, const float (&d)[V], float w_in, float e_in,
                                    float (&dw)[V], float (&de)[V])
{
    dw[0] = w_in;
    de[V - 1] = e_in;
#pragma unroll
    for (int j = 1; j < V; j++) dw[j] = d[j - 1];
#pragma unroll
    for (int j = 0; j < V - 1; j++) de[j] = d[j + 1];
    if (EDGE) {
#pragma unroll
        for (int j = 0; j < V; j++) {
            dw[j] = ((c.lmask >> j) & 1u) ? d[j] : dw[j];
            de[j] = ((c.rmask >> j) & 1u) ? d[j] : de[j];
        }
    }
}

// Start row y+1: Xq = its north term (+ its power for Hotspot), written over the finished P.
template <int KIND, int V>
__device__ __forceinline__ void qf(const CtxF &c, const CoefF &k, const float (&d)[V],
                                   uint32_t p_next, float (&Xq)[V])
{
    if (KIND == KDIFF) {
#pragma unroll
        for (int j = 0; j < V; j++) Xq[j] = __fmul_rn(k.a4, d[j]);
    } else {
        float p[V];
        lds_row<V>(p_next, c, p);
#pragma unroll
        for (int j = 0; j < V; j++) Xq[j] = __fmaf_rn(k.a2, d[j], p[j]);
    }
}

// One stage on the arrival of row y (values d, time s).  Xp holds P (row y-1, all but its
// south term), Xq holds Q (row y's north term).  Emits out = row y-1 at time s+1, leaves
// row y's P in Xq and row y+1's Q in Xp.
// SWAP = true: P' is built on top of Q in Xq and Q' is written to Xp (the caller alternates the
// arrays every row).  SWAP = false: P' goes back to Xp and Q' to Xq (no alternation; the
// register allocator decides whether that needs copies).
template <int KIND, int V, int MODE, bool SWAP, bool SRC = false>
__device__ __forceinline__ void stf(const CtxF &c, const CoefF &k, int y, bool fwd, float (&Xp)[V],
                                    float (&Xq)[V], const float (&d)[V], float w_in, float e_in,
                                    uint32_t p_y, uint32_t p_next, float (&out)[V])
{
    constexpr bool SP = MODE == MODE_SPECIAL;
    constexpr bool ED = MODE != MODE_PLAIN;
    if (SP && fwd) {   // beyond this pass's step count: row y-1 of time s passes unchanged
#pragma unroll
        for (int j = 0; j < V; j++) {
            out[j] = Xp[j];
            if (SWAP) Xq[j] = d[j];   // becomes "P" of the next row: forwarded one row later
            else Xp[j] = d[j];
        }
        return;
    }
    const float cs = (KIND == KDIFF) ? k.a3 : k.a5;
#pragma unroll
    for (int j = 0; j < V; j++) out[j] = __fmaf_rn(cs, d[j], Xp[j]);
    if (SP && y == c.ny) {   // row ny-1 was completed on arrival (its south is itself)
#pragma unroll
        for (int j = 0; j < V; j++) out[j] = Xp[j];
    }
    if (SP && y == 0) qf<KIND, V>(c, k, d, p_y, Xq);   // top: the row above row 0 is row 0
    float dw[V], de[V];
    nbf<V, ED>(c, d, w_in, e_in, dw, de);
    float(&Pn)[V] = SWAP ? Xq : Xp;   // where row y's P goes
    float(&Qn)[V] = SWAP ? Xp : Xq;   // where row y+1's Q goes
    if (KIND == KDIFF) {
#pragma unroll
        for (int j = 0; j < V; j++) {
            Pn[j] = __fmaf_rn(k.a0, d[j], Xq[j]);
            Pn[j] = __fmaf_rn(k.a1, dw[j], Pn[j]);
            Pn[j] = __fmaf_rn(k.a2, de[j], Pn[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; j++) {
            if (SRC) {
                // Q (cy*n + src) + cx*(e + w) + cc*c - cz*c: the expanded weights, cc exact
                Pn[j] = __fmaf_rn(k.a1, __fadd_rn(de[j], dw[j]), Xq[j]);
                Pn[j] = __fmaf_rn(k.a0, d[j], Pn[j]);
                Pn[j] = __fmaf_rn(-k.a3, d[j], Pn[j]);
            } else {
                const float t2 = __fmaf_rn(-2.0f, d[j], __fadd_rn(de[j], dw[j]));
                Pn[j] = __fmaf_rn(t2, k.a1, Xq[j]);
                const float t3 = __fsub_rn(k.a4, d[j]);
                Pn[j] = __fmaf_rn(t3, k.a3, Pn[j]);
                Pn[j] = __fmaf_rn(k.a6, d[j], Pn[j]);
                Pn[j] = __fmaf_rn(k.a0, Pn[j], d[j]);
            }
        }
    }
    qf<KIND, V>(c, k, d, p_next, Qn);
    if (SP && y == c.ny - 1) {   // bottom: complete row ny-1 now with south = itself
#pragma unroll
        for (int j = 0; j < V; j++) Pn[j] = __fmaf_rn(cs, d[j], Pn[j]);
    }
}

// Per-thread, per-segment state of the row loop.
struct RowF {
    const float *gF, *gP;   // field / power pointers at column x0 + 4*lane of the next row to load
    float *gO;              // output pointer at my first cell of the next row to store
    int colq[4];            // per 16-byte chunk: column offset to copy from (0 when off-grid)
    int nbq[4];             // per chunk: bytes inside the grid (0..16)
    int rf, rp;             // ring slots of field row i / of power row i
    int i_store;            // first iteration that stores a row
    int i_load_end;         // iterations i < i_load_end queue row i+PF
    // 16-bit storage
    const uint16_t *qF, *qP;     // raw rows of the next row to load (at column x0)
    const float2 *mF, *mP;       // block-code rows of the next row to load
    uint16_t *qO;                // raw output at my first cell of the next row to store
    float2 *mO;                  // block-code row of the next row to store
    int rr;                      // staging slot of row i
    int nbr;                     // my raw bytes inside the grid (0 .. 2V), colr: my column
    int colr;
};

// Trajectory passes: the row `row` of step t+1 of the pass (stage t's output) into state t,
// for the steps before the pass's last (whose rows go to the pass output) and the rows of
// this segment, compute-block cells only.
template <int V>
__device__ __forceinline__ void tbf_store_state(const CtxF &c, int t, int row, const float (&v)[V])
{
    if (t >= c.tsteps - 1 || row < c.s0 || row >= c.s1) return;
    float *g = c.st_states + (long long)t * c.st_stride + (long long)row * c.ld_out + c.xt;
    if (c.st_full) {
#pragma unroll
        for (int q = 0; q < V / 4; q++)
            *reinterpret_cast<float4 *>(g + 4 * q) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if (c.st_any) {
#pragma unroll
        for (int j = 0; j < V; j++)
            if (j >= c.st_lo && j < c.st_hi) g[j] = v[j];
    }
}

// One row iteration.  PH selects which of A/B holds P (PH = 0: A) for every stage.
template <int KIND, int T, int V, int MODE, int PH, bool SWAP, int STOR>
__device__ __forceinline__ void tbf_iter(const CtxF &c, const CoefF &k,
                                         float (&A)[TB2F<KIND, T, V>::NS][V],
                                         float (&B)[TB2F<KIND, T, V>::NS][V], int i,
                                         uint32_t fu, uint32_t fm, uint32_t fd, uint32_t pbase,
                                         float *gO, const RowF &r, bool store)
{
    using C = TB2F<KIND, T, V, STOR>;
    constexpr bool ED = MODE != MODE_PLAIN;
    const int R0 = c.y_start + i;
    float d[V], out[V];
    // stage 0: row R0-1 at time 1 straight from the time-0 rows R0-2, R0-1, R0 in the ring
    // (fu, fm, fd are those rows, already clamped to the grid for the boundary rows)
    {
        float u[V], m[V], dd[V], w[V], e[V];
        lds_row<V>(fu, c, u);
        lds_row<V>(fm, c, m);
        lds_row<V>(fd, c, dd);
        nbf<V, ED>(c, m, lds32(fm + c.ow4), lds32(fm + c.oe4), w, e);
        if (KIND == KDIFF) {
#pragma unroll
            for (int j = 0; j < V; j++)
                out[j] = diff5<false>(m[j], w[j], e[j], dd[j], u[j], k.a0, k.a1, k.a2, k.a3, k.a4);
        } else {
            float pv[V];
            lds_row<V>(pbase - C::ROWB, c, pv);   // power of row R0-1
            if (stor_src(STOR)) {
                // the source-map form of the Hotspot update (see stf): src + cx*(e + w) +
                // cy*(n + s) + cc*c - cz*c
#pragma unroll
                for (int j = 0; j < V; j++) {
                    float q = __fmaf_rn(k.a1, __fadd_rn(e[j], w[j]), pv[j]);
                    q = __fmaf_rn(k.a2, __fadd_rn(u[j], dd[j]), q);
                    q = __fmaf_rn(k.a0, m[j], q);
                    out[j] = __fmaf_rn(-k.a3, m[j], q);
                }
            } else {
#pragma unroll
                for (int j = 0; j < V; j++)
                    out[j] = hot2<false>(m[j], w[j], e[j], dd[j], u[j], pv[j], k.a0, k.a1, k.a2,
                                         k.a3, k.a4);
            }
        }
    }
    // stages 1 .. T-1: stage s receives row R0-s of time s; pbase is the slot of power row
    // R0 (ring-relative i), row i-t sits t slots below it
#pragma unroll
    for (int s = 1; s < T; s++) {
        if (stor_all(STOR)) tbf_store_state<V>(c, s - 1, R0 - s, out);
#pragma unroll
        for (int j = 0; j < V; j++) d[j] = out[j];
        const float w_in = __shfl_sync(0xffffffffu, d[V - 1], (c.lane + 31) & 31);
        const float e_in = __shfl_sync(0xffffffffu, d[0], (c.lane + 1) & 31);
        stf<KIND, V, MODE, SWAP, stor_src(STOR)>(c, k, R0 - s, s >= c.tsteps, PH == 0 ? A[s - 1] : B[s - 1],
                                 PH == 0 ? B[s - 1] : A[s - 1], d, w_in, e_in,
                           pbase - s * C::ROWB, pbase - (s - 1) * C::ROWB, out);
    }
    if (store) {
        if (stor_fmt(STOR) == STOR_F32) {
            if (c.st_full) {
#pragma unroll
                for (int q = 0; q < V / 4; q++)
                    *reinterpret_cast<float4 *>(gO + 4 * q) =
                        make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
            } else if (c.st_any) {
#pragma unroll
                for (int j = 0; j < V; j++)
                    if (j >= c.st_lo && j < c.st_hi) gO[j] = out[j];
            }
        } else {
            // encode the row segment of this tile as q = x - offset with the offset the value of
            // the block's first cell (tile column tx*CX: lane H/V, its cell 0, in the grid for
            // every tile) and scale 1.  bf16 and fp16 are floating-point formats, so q keeps 8
            // (11) significant bits of each cell's distance from the offset at any magnitude:
            // the error per cell is at most half an ulp of |x - offset| <= the block's spread,
            // and no block-wide minimum and maximum are needed
            const float mid = __shfl_sync(0xffffffffu, out[0], C::H / V);
            unsigned q2[V / 2];   // pairs of codes, cell 2i in the low half
#pragma unroll
            for (int j = 0; j < V / 2; j++) q2[j] = f2q2<STOR>(out[2 * j] - mid, out[2 * j + 1] - mid);
            if (c.st_full) {
#pragma unroll
                for (int t = 0; t < V / 4; t++)
                    *reinterpret_cast<uint2 *>(r.qO + 4 * t) = make_uint2(q2[2 * t], q2[2 * t + 1]);
            } else if (c.st_any) {
#pragma unroll
                for (int j = 0; j < V; j++)
                    if (j >= c.st_lo && j < c.st_hi)
                        r.qO[j] = (uint16_t)((j & 1) ? (q2[j / 2] >> 16) : (q2[j / 2] & 0xffffu));
            }
            if (c.lane == 0) r.mO[c.tx] = make_float2(mid, 1.0f);
        }
    }
}

// Decode my V cells of a staged raw row (header: codes of the blocks tx-1, tx, tx+1) into a
// float ring row (and into its mirror when mirror != 0).
template <int V, int STOR>
__device__ __forceinline__ void tbf_decode(const CtxF &c, uint32_t raw, uint32_t dst, uint32_t mirror)
{
    const uint2 cw = lds64u(raw + 8u * c.msel);
    const float mid = __uint_as_float(cw.x), sc = __uint_as_float(cw.y);
#pragma unroll
    for (int t = 0; t < V / 4; t++) {
        const uint2 w = lds64u(raw + 32u + 2u * V * c.lane + 8u * t);
        float x0 = __fmaf_rn(sc, q2f<STOR>(w.x & 0xffffu), mid);
        float x1 = __fmaf_rn(sc, q2f<STOR>(w.x >> 16), mid);
        float x2 = __fmaf_rn(sc, q2f<STOR>(w.y & 0xffffu), mid);
        float x3 = __fmaf_rn(sc, q2f<STOR>(w.y >> 16), mid);
        sts128(dst + c.oq[t], x0, x1, x2, x3);
        if (mirror) sts128(mirror + c.oq[t], x0, x1, x2, x3);
    }
}

// Queue tile row (row pointers in r) into field slot lf and power slot lp (plus its mirror);
// with 16-bit storage, into staging slot lr instead.
template <int KIND, int T, int V, int STOR>
__device__ __forceinline__ void tbf_queue(const CtxF &c, const RowF &r, int lf, int lp, int lr)
{
    using C = TB2F<KIND, T, V, STOR>;
    if (stor_fmt(STOR) != STOR_F32) {
#pragma unroll
        for (int in = 0; in < (KIND == KTHERM ? 2 : 1); in++) {
            const uint32_t dr = (in == 0 ? c.sRF : c.sRP) + lr * C::RAWB;
            const uint16_t *src = in == 0 ? r.qF : r.qP;
            const float2 *m = in == 0 ? r.mF : r.mP;
#pragma unroll
            for (int t = 0; t < V / 4; t++) {
                const int nb = max(0, min(8, r.nbr - 8 * t));
                cp8(dr + 32u + 2u * V * c.lane + 8u * t, nb ? src + r.colr + 4 * t : src, nb);
            }
            if (c.lane < 6) {
                const int b = min(max(c.tx - 1 + (c.lane >> 1), 0), c.ntx - 1);
                cp4(dr + 4u * c.lane, reinterpret_cast<const float *>(m + b) + (c.lane & 1), 4);
            }
        }
        return;
    }
    const uint32_t df = c.sF + lf * C::ROWB;
    const uint32_t dp = c.sP + lp * C::ROWB;
    if (c.vec_in && (KIND == KDIFF || c.vec_pw)) {
#pragma unroll
        for (int q = 0; q < V / 4; q++) {
            cp16(df + c.wq[q], r.gF + r.colq[q], r.nbq[q]);
            if (KIND == KTHERM) {
                cp16(dp + c.wq[q], r.gP + r.colq[q], r.nbq[q]);
                if (lp < C::PW - 1) cp16(dp + C::NBP * C::ROWB + c.wq[q], r.gP + r.colq[q], r.nbq[q]);
            }
        }
    } else {   // rows not 16-byte aligned: element-wise copies
#pragma unroll
        for (int q = 0; q < V / 4; q++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int nb = (4 * j < r.nbq[q]) ? 4 : 0;
                const int col = nb ? r.colq[q] + j : 0;
                cp4(df + c.wq[q] + 4 * j, r.gF + col, nb);
                if (KIND == KTHERM) {
                    cp4(dp + c.wq[q] + 4 * j, r.gP + col, nb);
                    if (lp < C::PW - 1) cp4(dp + C::NBP * C::ROWB + c.wq[q] + 4 * j, r.gP + col, nb);
                }
            }
    }
}

// One row: wait for row i, run the stages, queue row i+PF, advance pointers and rings.
template <int KIND, int T, int V, int MODE, int PH, bool SWAP, int STOR>
__device__ __forceinline__ void tbf_step(const CtxF &c, const CoefF &k,
                                         float (&A)[TB2F<KIND, T, V>::NS][V],
                                         float (&B)[TB2F<KIND, T, V>::NS][V], int i, RowF &r)
{
    using C = TB2F<KIND, T, V, STOR>;
    cp_async_wait<C::PF - 1>();   // row i has landed
    __syncwarp();
    if (stor_fmt(STOR) != STOR_F32) {       // decode row i into the float rings
        tbf_decode<V, STOR>(c, c.sRF + r.rr * C::RAWB, c.sF + r.rf * C::ROWB, 0u);
        if (KIND == KTHERM)   // (for STOR_SRC the coded map is the source map itself)
            tbf_decode<V, STOR>(c, c.sRP + r.rr * C::RAWB, c.sP + r.rp * C::ROWB,
                                r.rp < C::PW - 1 ? c.sP + (C::NBP + r.rp) * C::ROWB : 0u);
        __syncwarp();
    }
    // field ring slots of rows i-2, i-1, i (rows above or below the grid clamp to its edge)
    int su = r.rf - 2, sm = r.rf - 1, sd = r.rf;
    su += (su < 0) ? C::NBF : 0;
    sm += (sm < 0) ? C::NBF : 0;
    if (MODE == MODE_SPECIAL) {
        const int R = c.y_start + i - 1;    // stage 0's row
        if (R == 0) su = sm;                // row -1 is row 0
        if (R == c.ny - 1) sd = sm;         // row ny is row ny-1
    }
    const uint32_t pbase = c.sP + ((KIND == KTHERM && r.rp < C::PW - 1) ? C::NBP + r.rp : r.rp) * C::ROWB;
    const bool store = i >= r.i_store;
    tbf_iter<KIND, T, V, MODE, PH, SWAP, STOR>(c, k, A, B, i, c.sF + su * C::ROWB,
                                               c.sF + sm * C::ROWB, c.sF + sd * C::ROWB, pbase,
                                               r.gO, r, store);
    if (store) {
        if (stor_fmt(STOR) == STOR_F32) r.gO += c.ld_out;
        else {
            r.qO += c.ld_q;
            r.mO += c.ntx;
        }
    }
    __syncwarp();
    int lf = 0, lp = 0, lr = 0;   // slots of row i+PF: float rings, or the staging ring
    if (!C::Q16) {
        lf = r.rf + C::PF;
        lf -= (lf >= C::NBF) ? C::NBF : 0;
        if (KIND == KTHERM) {
            lp = r.rp + C::PF;
            lp -= (lp >= C::NBP) ? C::NBP : 0;
        }
    } else {
        lr = r.rr + C::PF;
        lr -= (lr >= C::NBR) ? C::NBR : 0;
    }
    if (i < r.i_load_end) {
        tbf_queue<KIND, T, V, STOR>(c, r, lf, lp, lr);
        if (stor_fmt(STOR) == STOR_F32) {
            r.gF += c.ld_in;
            if (KIND == KTHERM) r.gP += c.ld_pw;
        } else {
            r.qF += c.ld_q;
            r.mF += c.ntx;
            if (KIND == KTHERM) {
                r.qP += c.ld_q;
                r.mP += c.ntx;
            }
        }
    }
    cp_async_commit();
    r.rf = (r.rf + 1 == C::NBF) ? 0 : r.rf + 1;
    if (KIND == KTHERM) r.rp = (r.rp + 1 == C::NBP) ? 0 : r.rp + 1;
    if (stor_fmt(STOR) != STOR_F32) r.rr = (r.rr + 1 == C::NBR) ? 0 : r.rr + 1;
}

template <int KIND, int T, int V, int MODE, bool SWAP, int STOR>
__device__ __forceinline__ void tbf_step_rt(const CtxF &c, const CoefF &k,
                                            float (&A)[TB2F<KIND, T, V>::NS][V],
                                            float (&B)[TB2F<KIND, T, V>::NS][V], int i, RowF &r)
{
    if (SWAP && (i & 1)) tbf_step<KIND, T, V, MODE, 1, SWAP, STOR>(c, k, A, B, i, r);
    else tbf_step<KIND, T, V, MODE, 0, SWAP, STOR>(c, k, A, B, i, r);
}

// Work units [f, fend) of one grid's pass: unit f = (tile column f / ny, row f % ny); a block
// walks them as segments of consecutive rows of one tile column.
template <int KIND, int T, int V, bool SWAP, int STOR>
__device__ __forceinline__ void tbf_range(const Pass2D &p, long long f, const long long fend,
                                          float (&A)[TB2F<KIND, T, V>::NS][V],
                                          float (&B)[TB2F<KIND, T, V>::NS][V], float *smem)
{
    using C = TB2F<KIND, T, V, STOR>;
    CtxF c;
    c.in = p.in;
    c.out = p.out;
    c.pw = p.pw;
    c.ld_in = p.ld_in;
    c.ld_out = p.ld_out;
    c.ld_pw = p.ld_pw;
    c.sF = smem_u32(smem);
    c.sP = c.sF + C::NBF * C::ROWB;
    c.sRF = c.sP + C::NBPX * C::ROWB;
    c.sRP = c.sRF + C::NBR * C::RAWB;
    c.qin = static_cast<const uint16_t *>(p.qin);
    c.qpw = static_cast<const uint16_t *>(p.qpw);
    c.qout = static_cast<uint16_t *>(p.qout);
    c.min_ = p.min_;
    c.mpw = p.mpw;
    c.mout = p.mout;
    c.ld_q = p.ld_q;
    c.ntx = p.ntx;
    c.nx = p.nx;
    c.ny = p.ny;
    c.tsteps = p.tsteps;
    c.vec_in = p.vec_in;
    c.vec_out = p.vec_out;
    c.vec_pw = p.vec_pw;
    c.lane = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        c.oq[q] = 16u * ring_pos(min(V / 4 * c.lane + q, V / 4 * c.lane + V / 4 - 1));
        c.wq[q] = 16u * ring_pos(c.lane + 32 * min(q, V / 4 - 1));
    }
    c.ow4 = ring_cell(c.lane > 0 ? V * c.lane - 1 : 0);
    c.oe4 = ring_cell(c.lane < 31 ? V * c.lane + V : V * c.lane + V - 1);
    CoefF k;
    k.a0 = p.kf[0]; k.a1 = p.kf[1]; k.a2 = p.kf[2]; k.a3 = p.kf[3]; k.a4 = p.kf[4];
    k.a5 = p.kf[5];   // Hotspot: sdc * Ry
    k.a6 = p.kf[6];   // Hotspot: -2 Ry (source-map kernels: unused)
    c.st_states = p.states;
    c.st_stride = p.state_stride;

    while (f < fend) {
        const int tx = (int)(f / p.ny);
        const int s0 = (int)(f - (long long)tx * p.ny);
        const int s1 = (int)min((long long)p.ny, (long long)s0 + (fend - f));
        f += s1 - s0;

        c.s0 = s0;
        c.s1 = s1;
        c.x0 = tx * C::CX - C::H;
        c.xt = c.x0 + c.lane * V;
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
            c.st_any = c.st_hi > c.st_lo;
        }
        RowF r;
#pragma unroll
        for (int q = 0; q < V / 4; q++) {
            const int x = c.x0 + 4 * (c.lane + 32 * q);   // chunk q of my lane
            r.nbq[q] = (x >= 0 && x < c.nx) ? min(16, 4 * (c.nx - x)) : 0;
            r.colq[q] = r.nbq[q] ? x : 0;
        }
        c.tx = tx;
        c.msel = (c.xt < tx * C::CX) ? 0 : ((c.xt >= (tx + 1) * C::CX) ? 2 : 1);
        if (stor_fmt(STOR) != STOR_F32) {
            r.qF = c.qin + (long long)c.y_start * c.ld_q;
            r.mF = c.min_ + (long long)c.y_start * c.ntx;
            r.qP = (KIND == KTHERM) ? c.qpw + (long long)c.y_start * c.ld_q : nullptr;
            r.mP = (KIND == KTHERM) ? c.mpw + (long long)c.y_start * c.ntx : nullptr;
            r.qO = c.qout + (long long)s0 * c.ld_q + c.xt;
            r.mO = c.mout + (long long)s0 * c.ntx;
            r.rr = 0;
            r.colr = (c.xt >= 0 && c.xt < c.nx) ? c.xt : 0;
            r.nbr = (c.xt >= 0 && c.xt < c.nx) ? 2 * min(V, c.nx - c.xt) : 0;
        }
        r.gF = c.in + (long long)c.y_start * c.ld_in;
        r.gP = (KIND == KTHERM) ? c.pw + (long long)c.y_start * c.ld_pw : nullptr;
        r.rf = 0;
        r.rp = 0;
        const int n_it = s1 + T - c.y_start;           // the last stage emits row s1-1 last
        r.i_store = s0 - c.y_start + T;                 // it emits row s0 at this iteration
        r.gO = c.out + (long long)s0 * c.ld_out + c.xt;
        r.i_load_end = c.last_row - c.y_start - C::PF + 1;

        // queue the first PF rows
#pragma unroll 1
        for (int j = 0; j < C::PF; j++) {
            if (c.y_start + j <= c.last_row) {
                tbf_queue<KIND, T, V, STOR>(c, r, C::Q16 ? 0 : j, (KIND == KTHERM && !C::Q16) ? j : 0, j);
                if (stor_fmt(STOR) == STOR_F32) {
                    r.gF += c.ld_in;
                    if (KIND == KTHERM) r.gP += c.ld_pw;
                } else {
                    r.qF += c.ld_q;
                    r.mF += c.ntx;
                    if (KIND == KTHERM) {
                        r.qP += c.ld_q;
                        r.mP += c.ntx;
                    }
                }
            }
            cp_async_commit();
        }

        // rows that need boundary handling: the grid's top rows (for every stage), its bottom
        // rows, and every row of a pass that forwards trailing stages
        const bool partial = (c.tsteps < T);
        const int i_a = partial ? n_it : ((c.y_start == 0) ? min(T + 1, n_it) : 0);
        // (a stage meets row 0 at i <= T when the segment starts at the top, and rows ny-1 / ny
        // from i = ny - y_start on; the bounds below keep one row of margin)
        const int i_b = partial ? n_it : max(i_a, min(n_it, c.ny - 1 - c.y_start));
        int i = 0;
#pragma unroll 1
        for (; i < i_a; i++) tbf_step_rt<KIND, T, V, MODE_SPECIAL, SWAP, STOR>(c, k, A, B, i, r);
        if (SWAP) {
            if (i < i_b && (i & 1)) {
                if (c.edge) tbf_step<KIND, T, V, MODE_EDGE, 1, SWAP, STOR>(c, k, A, B, i, r);
                else tbf_step<KIND, T, V, MODE_PLAIN, 1, SWAP, STOR>(c, k, A, B, i, r);
                i++;
            }
            if (c.edge) {
#pragma unroll 1
                for (; i + 1 < i_b; i += 2) {
                    tbf_step<KIND, T, V, MODE_EDGE, 0, SWAP, STOR>(c, k, A, B, i, r);
                    tbf_step<KIND, T, V, MODE_EDGE, 1, SWAP, STOR>(c, k, A, B, i + 1, r);
                }
            } else {
#pragma unroll 1
                for (; i + 1 < i_b; i += 2) {
                    tbf_step<KIND, T, V, MODE_PLAIN, 0, SWAP, STOR>(c, k, A, B, i, r);
                    tbf_step<KIND, T, V, MODE_PLAIN, 1, SWAP, STOR>(c, k, A, B, i + 1, r);
                }
            }
        } else {
            if (c.edge) {
#pragma unroll 1
                for (; i < i_b; i++) tbf_step<KIND, T, V, MODE_EDGE, 0, SWAP, STOR>(c, k, A, B, i, r);
            } else {
#pragma unroll 1
                for (; i < i_b; i++) tbf_step<KIND, T, V, MODE_PLAIN, 0, SWAP, STOR>(c, k, A, B, i, r);
            }
        }
#pragma unroll 1
        for (; i < n_it; i++) tbf_step_rt<KIND, T, V, MODE_SPECIAL, SWAP, STOR>(c, k, A, B, i, r);
        cp_async_wait<0>();
        __syncwarp();
    }
}


template <int KIND, int T, int V, bool SWAP, int STOR>
__global__ void __launch_bounds__(32) k_tb2f(const Pass2D p)
{
    using C = TB2F<KIND, T, V, STOR>;
    extern __shared__ __align__(16) float smem[];
    float A[C::NS][V], B[C::NS][V];
#pragma unroll
    for (int s = 0; s < C::NS; s++)
#pragma unroll
        for (int j = 0; j < V; j++) A[s][j] = B[s][j] = 0.f;
    long long f, fend;
    if (p.starts) {
        f = __ldg(p.starts + blockIdx.x);
        fend = __ldg(p.starts + blockIdx.x + 1);
    } else {
        f = (long long)blockIdx.x * p.rows_per_cta;
        fend = min(f + p.rows_per_cta, p.total_rows);
    }
    tbf_range<KIND, T, V, SWAP, STOR>(p, f, fend, A, B, smem);
}

}  // namespace stn
