// 3D temporally-blocked Jacobi sweep, contracted arithmetic, partial sums along z.
//
// Method (arXiv 1802.00438): 2D spatial blocking in x and y with streaming along z (Sec. 3.1),
// overlapped tiles with halos of width >= rad*T (Eq. 2), a chain of T stages where stage t
// computes time step t one plane behind stage t-1 (Sec. 3.2), redundant halo computation with
// only the compute block written (Sec. 3.2), trailing stages forwarding when a pass fuses fewer
// than T steps (Sec. 3.2), clamped boundaries at every stage (Sec. 5.1).
//
// GPU mapping: tile 32*VX x NW*VY cells incl. halos; a thread owns VX adjacent x cells of VY
// consecutive rows, a warp spans the tile's width, warps are stacked along y.
//   Stage 0 evaluates plane z-1 directly from a cp.async ring of input planes in shared memory.
//   Stages 1..T-1 consume the plane the previous stage has just produced, in the same z
//   iteration, and keep only two partial sums per cell instead of a three-plane window: when
//   plane z of its input arrives, a stage
//     finishes output plane z-1:   out = P + ca*d
//     starts   output plane z:     P   = Q + cc*d + cw*w + ce*e + cs*s + cn*n (+ sdc*p(z))
//     starts   output plane z+1:   Q   = cb*d (+ ca*amb)
//   The rows above and below a warp's rows come from its neighbour warps through a small
//   shared-memory exchange (one barrier per stage and plane); x neighbours are warp shuffles.
//   Clamped z boundaries: at z = 0 the missing plane z-1 is plane 0 itself (Q is started from
//   d before it is used), and the missing plane nz is plane nz-1: a stage that reaches the
//   virtual plane nz finishes plane nz-1 from the repeated input and then repeats that output
//   so that the next stage sees the same clamp.
//   Power (Hotspot 3D) is staged with the field: a second cp.async ring holds the power planes
//   of every stage's current plane, so each power value is read from HBM once per pass.
//   Ring slots advance with the z iteration as rolling indices (no integer division in the
//   steady state); shared memory is addressed with 32-bit shared-window addresses.
#pragma once
#include <type_traits>
#include "common.cuh"
#include "internal.h"

namespace stn {

template <int KIND, int T, int VX, int VY, int NW>
struct TB3F {
    static constexpr int NT = 32 * NW;
    static constexpr int BX = 32 * VX;
    static constexpr int BY = NW * VY;
    static constexpr int HX = (T + 3) / 4 * 4;   // 16-byte aligned tile origins
    static constexpr int HY = T;
    static constexpr int CX = BX - 2 * HX;
    static constexpr int CY = BY - 2 * HY;
    static constexpr int NS = T > 1 ? T - 1 : 1;
    static constexpr int PLANE = BX * BY;
    static constexpr uint32_t PLANE_B = 4u * PLANE;
    static constexpr size_t XCH = (size_t)NS * NW * 2 * BX;   // [stage][warp][top/bottom][BX]
    // shared memory with PF planes in flight past the newest read: field ring of planes z-1,
    // z, z+1 and PF more; power ring of planes z-max(T-1,1) .. z+PF (stage 0 reads plane z-1
    // also when T = 1); exchange; one mbarrier per field slot (tensor-map staging)
    static constexpr size_t smem_for(int pf)
    {
        return sizeof(float) * ((size_t)((pf + 3) + (KIND == KTHERM ? (T > 1 ? T : 2) + pf : 0)) *
                                    PLANE + XCH) + 8 * (pf + 3);
    }
    // blocks of up to 8 warps run two per SM, larger ones one
    static constexpr int MINB = NT <= 256 ? 2 : 1;
    // the deepest prefetch (2..5 planes) whose shared memory fits MINB blocks per SM (1 KiB of
    // each block's share is reserved by the hardware)
    static constexpr size_t BUDGET = MINB == 2 ? 113 * 1024 : 227 * 1024;
    static constexpr int PF = smem_for(5) <= BUDGET ? 5 : smem_for(4) <= BUDGET ? 4
                            : smem_for(3) <= BUDGET ? 3 : 2;
    static constexpr int NBF = PF + 3;
    static constexpr int NBP = KIND == KTHERM ? (T > 1 ? T : 2) + PF : 0;
    static constexpr size_t SMEM = smem_for(PF);
    static_assert(CX > 0 && CY > 0, "tile smaller than its halos");
    static_assert(VX == 2 || VX == 4, "cells per lane");
    static_assert(VX * VY <= 32, "store mask");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Per-thread context of one tile column.
struct CtxF3 {
    const float *__restrict__ in;
    float *__restrict__ out;
    const float *__restrict__ pw;
    int nx, ny, nz, tsteps, vec, vec_pw;
    long long plane;       // nx * ny
    int x0, y0;            // tile origin
    int gx, gy;            // my first cell
    int z_start, last_plane, z0, z1;
    bool edge_x, edge_y;   // warp touches a domain edge in x / in y
    bool lx0;              // my cell 0 is x = 0
    unsigned rxm;          // bit j: my cell j is x = nx-1 (a mask, not an index: a compare of
                           // the index per cell would become an indexed store to memory)
    unsigned ym0, ymn;     // bit k: my row k is y = 0 / y = ny-1
    unsigned st_mask;      // bit (k*VX + j): my cell (row k, x j) is stored
    unsigned st_rows;      // bit k: my row k is stored whole
    bool st_fast;          // vector stores: every row whole or empty, aligned rows
    long long st_off;      // gy * nx + gx
    int tid, lane, wid;
    float k[9];
    float ca_amb;
};

template <int VX>
struct VecF;
template <>
struct VecF<2> {
    float v[2];
};
template <>
struct VecF<4> {
    float v[4];
};

template <int VX>
__device__ __forceinline__ VecF<VX> ldsv(uint32_t a)
{
    VecF<VX> r;
    if constexpr (VX == 2)
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(r.v[0]), "=f"(r.v[1]) : "r"(a));
    else
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
                     : "r"(a));
    return r;
}

template <int VX>
__device__ __forceinline__ void stsv(uint32_t a, const float *x)
{
    if constexpr (VX == 2)
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x[0]), "f"(x[1]) : "memory");
    else
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(x[0]), "f"(x[1]),
                     "f"(x[2]), "f"(x[3])
                     : "memory");
}

__device__ __forceinline__ void cpa16(uint32_t dst, const void *src, int nbytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
                 : "memory");
}

__device__ __forceinline__ void cpa4(uint32_t dst, const void *src, int nbytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes)
                 : "memory");
}

// ---- tensor-map bulk copies completing on an mbarrier ---------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier; gives up (false) after a bounded number of polls
// (each poll may suspend the thread for a while), so a lost copy cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (int n = 0; n < (1 << 22); n++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_plane(uint32_t dst, const CUtensorMap *m, int x, int y, int z,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Stage the tile's window of one plane (z-plane base `src`) into the slot at `dst`; cells
// outside the domain arrive as zeros.
template <int BX, int BY, int NT>
__device__ __forceinline__ void tbf3_load(const CtxF3 &c, const float *src, int vec, uint32_t dst)
{
    constexpr int CH = BX / 4;
    constexpr int NCH = CH * BY;
#pragma unroll
    for (int qq = 0; qq < (NCH + NT - 1) / NT; qq++) {
        const int q = c.tid + qq * NT;
        if (NCH % NT == 0 || q < NCH) {
            const int row = q / CH, ch = q % CH;
            const int y = c.y0 + row, x = c.x0 + 4 * ch;
            const uint32_t d = dst + 4u * (row * BX + 4 * ch);
            const bool yok = (y >= 0 && y < c.ny);
            const float *rs = src + (long long)(yok ? y : 0) * c.nx;
            if (vec) {
                const int nb = (yok && x >= 0 && x < c.nx) ? min(16, 4 * (c.nx - x)) : 0;
                cpa16(d, nb ? rs + x : src, nb);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int xx = x + j;
                    const int nb = (yok && xx >= 0 && xx < c.nx) ? 4 : 0;
                    cpa4(d + 4u * j, nb ? rs + xx : src, nb);
                }
            }
        }
    }
}

// Neighbours of my cells in a plane held as m[VY][VX]: w/e inside my cells or by shuffle,
// n/s from my rows or the rows of the warps above (nt) and below (sb).
// Clamped domain edges are applied to the plane, not to the neighbour arrays: in a warp that
// touches an edge, the out-of-domain cell next to each edge cell (a ghost: its own value is
// never used) takes the edge cell's value, inside my cells (m, in place) or in the value that
// arrives from another lane or warp (wl, er, nt, sb).  The neighbour arrays stay pure renames of
// m, so the common path keeps no second copy of them.
template <int VX, int VY, bool EDGE>
__device__ __forceinline__ void nbf3(const CtxF3 &c, float (&m)[VY][VX], float (&nt)[VX],
                                     float (&sb)[VX], float (&w)[VY][VX], float (&e)[VY][VX],
                                     float (&n)[VY][VX], float (&s)[VY][VX])
{
    float wl[VY], er[VY];
#pragma unroll
    for (int k = 0; k < VY; k++) {
        wl[k] = __shfl_sync(0xffffffffu, m[k][VX - 1], (c.lane + 31) & 31);
        er[k] = __shfl_sync(0xffffffffu, m[k][0], (c.lane + 1) & 31);
    }
    if (EDGE && c.edge_y) {
        // y = 0 at my row k: ghost row k-1 (or the row above, nt) := row k; likewise below
#pragma unroll
        for (int j = 0; j < VX; j++) {
            nt[j] = (c.ym0 & 1u) ? m[0][j] : nt[j];
            sb[j] = ((c.ymn >> (VY - 1)) & 1u) ? m[VY - 1][j] : sb[j];
        }
#pragma unroll
        for (int k = 1; k < VY; k++)
#pragma unroll
            for (int j = 0; j < VX; j++) m[k - 1][j] = ((c.ym0 >> k) & 1u) ? m[k][j] : m[k - 1][j];
#pragma unroll
        for (int k = 0; k < VY - 1; k++)
#pragma unroll
            for (int j = 0; j < VX; j++) m[k + 1][j] = ((c.ymn >> k) & 1u) ? m[k][j] : m[k + 1][j];
    }
    if (EDGE && c.edge_x) {
        // x = 0 is always my cell 0 (tile origins are multiples of 4); x = nx-1 is my cell j
#pragma unroll
        for (int k = 0; k < VY; k++) {
            wl[k] = c.lx0 ? m[k][0] : wl[k];
            er[k] = ((c.rxm >> (VX - 1)) & 1u) ? m[k][VX - 1] : er[k];
#pragma unroll
            for (int j = 1; j < VX; j++) m[k][j] = ((c.rxm >> (j - 1)) & 1u) ? m[k][j - 1] : m[k][j];
        }
    }
    // (every index below stays in range even in code the unrolling discards: an out-of-range
    // constant index, even in a dead branch, makes the compiler keep the array in memory)
#pragma unroll
    for (int k = 0; k < VY; k++) {
        w[k][0] = wl[k];
        e[k][VX - 1] = er[k];
#pragma unroll
        for (int j = 1; j < VX; j++) w[k][j] = m[k][j - 1];
#pragma unroll
        for (int j = 0; j < VX - 1; j++) e[k][j] = m[k][j + 1];
    }
#pragma unroll
    for (int j = 0; j < VX; j++) {
        n[0][j] = nt[j];
        s[VY - 1][j] = sb[j];
    }
#pragma unroll
    for (int k = 1; k < VY; k++)
#pragma unroll
        for (int j = 0; j < VX; j++) n[k][j] = m[k - 1][j];
#pragma unroll
    for (int k = 0; k < VY - 1; k++)
#pragma unroll
        for (int j = 0; j < VX; j++) s[k][j] = m[k + 1][j];
}

template <int VX, int VY>
__device__ __forceinline__ void tbf3_store(const CtxF3 &c, int z, const float (&v)[VY][VX])
{
    float *dst = c.out + (long long)z * c.plane + c.st_off;
    if (c.st_fast) {
        // every row of mine is stored whole or not at all, with aligned vector stores
#pragma unroll
        for (int k = 0; k < VY; k++) {
            float *d = dst + (long long)k * c.nx;
            if ((c.st_rows >> k) & 1u) {
                if constexpr (VX == 2) *reinterpret_cast<float2 *>(d) = make_float2(v[k][0], v[k][1]);
                else *reinterpret_cast<float4 *>(d) = make_float4(v[k][0], v[k][1], v[k][2], v[k][3]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < VY; k++)
#pragma unroll
            for (int j = 0; j < VX; j++)
                if ((c.st_mask >> (VX * k + j)) & 1u) dst[(long long)k * c.nx + j] = v[k][j];
    }
}

template <int N>
__device__ __forceinline__ int slot_of(int rel)   // rel >= -2N
{
    return (rel + 2 * N) % N;
}

template <int N>
__device__ __forceinline__ int slot_back(int s, int k)   // (s - k) mod N for 0 <= k <= N
{
    const int r = s - k;
    return r < 0 ? r + N : r;
}

// Ring slots of the current iteration: field plane Z0 and power plane Z0-1.
struct Slots3 {
    int f0;
    int p1;
};

template <int KIND>
__device__ __forceinline__ float upd3f(const CtxF3 &c, float m, float w, float e, float s,
                                       float n, float b, float a, float p)
{
    if (KIND == KDIFF) return diff7<false>(m, w, e, s, n, b, a, c.k);
    else return hot3<false>(m, w, e, s, n, b, a, p, c.k, c.ca_amb);
}

template <int KIND, int T, int VX, int VY, int NW, bool SPECIAL, bool EDGE>
__device__ __forceinline__ void tbf3_iter(const CtxF3 &c, uint32_t sring, uint32_t spw,
                                          uint32_t sxch, const Slots3 &sl,
                                          const float (&P)[TB3F<KIND, T, VX, VY, NW>::NS][VY][VX],
                                          const float (&Q)[TB3F<KIND, T, VX, VY, NW>::NS][VY][VX],
                                          float (&Pn)[TB3F<KIND, T, VX, VY, NW>::NS][VY][VX],
                                          float (&Qn)[TB3F<KIND, T, VX, VY, NW>::NS][VY][VX], int i)
{
    using C = TB3F<KIND, T, VX, VY, NW>;
    const int Z0 = c.z_start + i;   // newest plane in the ring
    const float cc = c.k[0], cw = c.k[1], ce = c.k[2], cs = c.k[3], cn = c.k[4], cb = c.k[5],
                ca = c.k[6];
    const uint32_t own = 4u * (c.wid * VY * C::BX + VX * c.lane);   // my row 0, cell 0
    float d[VY][VX];

    // ---- stage 0: plane R = Z0 - 1 from the ring ------------------------------------------
    {
        int fu, fm, fd, pm;
        if (SPECIAL) {
            const int R = min(Z0 - 1, c.nz - 1);   // past the bottom: repeat plane nz-1
            fu = slot_of<C::NBF>(max(R - 1, 0) - c.z_start);
            fm = slot_of<C::NBF>(R - c.z_start);
            fd = slot_of<C::NBF>(min(R + 1, c.nz - 1) - c.z_start);
            pm = KIND == KTHERM ? slot_of<C::NBP ? C::NBP : 1>(max(R, 0) - c.z_start) : 0;
        } else {
            fd = sl.f0;
            fm = slot_back<C::NBF>(fd, 1);
            fu = slot_back<C::NBF>(fd, 2);
            pm = sl.p1;
        }
        const uint32_t au = sring + fu * C::PLANE_B + own;
        const uint32_t am = sring + fm * C::PLANE_B + own;
        const uint32_t ad = sring + fd * C::PLANE_B + own;
        float u[VY][VX], m[VY][VX], a[VY][VX], w[VY][VX], e[VY][VX], n[VY][VX], s[VY][VX];
        float p[VY][VX];
#pragma unroll
        for (int k = 0; k < VY; k++) {
            const VecF<VX> x = ldsv<VX>(au + 4u * k * C::BX);
            const VecF<VX> y = ldsv<VX>(am + 4u * k * C::BX);
            const VecF<VX> z = ldsv<VX>(ad + 4u * k * C::BX);
#pragma unroll
            for (int j = 0; j < VX; j++) {
                u[k][j] = x.v[j];
                m[k][j] = y.v[j];
                a[k][j] = z.v[j];
            }
        }
        float nt[VX], sb[VX];
        {
            const int up = c.wid > 0 ? -1 : 0, dn = c.wid < NW - 1 ? VY : VY - 1;
            const VecF<VX> x = ldsv<VX>(am + 4 * up * C::BX);
            const VecF<VX> y = ldsv<VX>(am + 4 * dn * C::BX);
#pragma unroll
            for (int j = 0; j < VX; j++) {
                nt[j] = x.v[j];
                sb[j] = y.v[j];
            }
        }
        nbf3<VX, VY, EDGE>(c, m, nt, sb, w, e, n, s);
        if (KIND == KTHERM) {
            const uint32_t ap = spw + pm * C::PLANE_B + own;
#pragma unroll
            for (int k = 0; k < VY; k++) {
                const VecF<VX> x = ldsv<VX>(ap + 4u * k * C::BX);
#pragma unroll
                for (int j = 0; j < VX; j++) p[k][j] = x.v[j];
            }
        }
#pragma unroll
        for (int k = 0; k < VY; k++)
#pragma unroll
            for (int j = 0; j < VX; j++)
                d[k][j] = upd3f<KIND>(c, m[k][j], w[k][j], e[k][j], s[k][j], n[k][j], u[k][j],
                                      a[k][j], KIND == KTHERM ? p[k][j] : 0.f);
    }
    if constexpr (T == 1) {
        const int R = Z0 - 1;
        if (R >= c.z0 && R < c.z1) tbf3_store<VX, VY>(c, R, d);
    } else {
        constexpr uint32_t XS = 4u * NW * 2 * C::BX;   // bytes per stage in the exchange
        const uint32_t xo = 4u * VX * c.lane;
        const int wt = c.wid > 0 ? c.wid - 1 : 0;   // warp above (tile edge: any in-bounds row)
        const int wb = c.wid < NW - 1 ? c.wid + 1 : NW - 1;
#pragma unroll
        for (int st = 1; st < T; st++) {
            const int zc = Z0 - st;   // plane of d (output of stage st-1)
            float o[VY][VX];
            if (SPECIAL && st >= c.tsteps) {
                // forwarding stage: one plane of delay, no arithmetic
#pragma unroll
                for (int k = 0; k < VY; k++)
#pragma unroll
                    for (int j = 0; j < VX; j++) {
                        o[k][j] = Q[st - 1][k][j];
                        Qn[st - 1][k][j] = d[k][j];
                        Pn[st - 1][k][j] = P[st - 1][k][j];
                    }
            } else {
                const uint32_t xw = sxch + (st - 1) * XS + xo;
                stsv<VX>(xw + 4u * (c.wid * 2 + 0) * C::BX, d[0]);
                stsv<VX>(xw + 4u * (c.wid * 2 + 1) * C::BX, d[VY - 1]);
                __syncthreads();
                float nt[VX], sb[VX];
                {
                    const VecF<VX> x = ldsv<VX>(xw + 4u * (wt * 2 + 1) * C::BX);
                    const VecF<VX> y = ldsv<VX>(xw + 4u * (wb * 2 + 0) * C::BX);
#pragma unroll
                    for (int j = 0; j < VX; j++) {
                        nt[j] = x.v[j];
                        sb[j] = y.v[j];
                    }
                }
                float w[VY][VX], e[VY][VX], n[VY][VX], s[VY][VX], p[VY][VX];
                nbf3<VX, VY, EDGE>(c, d, nt, sb, w, e, n, s);
                if (KIND == KTHERM) {
                    int ps;
                    if (SPECIAL)
                        ps = slot_of<C::NBP ? C::NBP : 1>(min(max(zc, 0), c.nz - 1) - c.z_start);
                    else
                        ps = slot_back<C::NBP ? C::NBP : 1>(sl.p1, st - 1);
                    const uint32_t ap = spw + ps * C::PLANE_B + own;
#pragma unroll
                    for (int k = 0; k < VY; k++) {
                        const VecF<VX> x = ldsv<VX>(ap + 4u * k * C::BX);
#pragma unroll
                        for (int j = 0; j < VX; j++) p[k][j] = x.v[j];
                    }
                }
                const float(&Ps)[VY][VX] = P[st - 1];
                const float(&Qs)[VY][VX] = Q[st - 1];
                float(&Pw)[VY][VX] = Pn[st - 1];
                float(&Qw)[VY][VX] = Qn[st - 1];
                if (!SPECIAL || zc < c.nz) {
                    const bool first = SPECIAL && zc == 0;   // clamp: plane -1 is plane 0
#pragma unroll
                    for (int k = 0; k < VY; k++)
#pragma unroll
                        for (int j = 0; j < VX; j++) {
                            const float dv = d[k][j];
                            float qn;
                            if (KIND == KTHERM) qn = __fmaf_rn(cb, dv, c.ca_amb);
                            else qn = __fmul_rn(cb, dv);
                            const float qi = first ? qn : Qs[k][j];
                            o[k][j] = __fmaf_rn(ca, dv, Ps[k][j]);
                            float r = qi;
                            if (KIND == KTHERM) r = __fmaf_rn(c.k[7], p[k][j], r);
                            r = __fmaf_rn(cc, dv, r);
                            r = __fmaf_rn(cn, n[k][j], r);
                            r = __fmaf_rn(cs, s[k][j], r);
                            r = __fmaf_rn(ce, e[k][j], r);
                            r = __fmaf_rn(cw, w[k][j], r);
                            Pw[k][j] = r;
                            Qw[k][j] = qn;
                        }
                } else if (zc == c.nz) {
                    // virtual plane nz (= plane nz-1): finish plane nz-1 and keep it
#pragma unroll
                    for (int k = 0; k < VY; k++)
#pragma unroll
                        for (int j = 0; j < VX; j++) {
                            o[k][j] = __fmaf_rn(ca, d[k][j], Ps[k][j]);
                            Pw[k][j] = o[k][j];
                            Qw[k][j] = Qs[k][j];
                        }
                } else {
#pragma unroll
                    for (int k = 0; k < VY; k++)
#pragma unroll
                        for (int j = 0; j < VX; j++) {
                            o[k][j] = Ps[k][j];
                            Pw[k][j] = Ps[k][j];
                            Qw[k][j] = Qs[k][j];
                        }
                }
            }
#pragma unroll
            for (int k = 0; k < VY; k++)
#pragma unroll
                for (int j = 0; j < VX; j++) d[k][j] = o[k][j];
        }
        const int R = Z0 - T;
        if (R >= c.z0 && R < c.z1) tbf3_store<VX, VY>(c, R, d);
    }
}

template <int KIND, int T, int VX, int VY, int NW>
__global__ void __launch_bounds__(32 * NW, (TB3F<KIND, T, VX, VY, NW>::MINB))
    k_tb3f(const Pass3D p, const __grid_constant__ CUtensorMap tin,
           const __grid_constant__ CUtensorMap tpw)
{
    using C = TB3F<KIND, T, VX, VY, NW>;
    extern __shared__ __align__(128) float smem[];
    const uint32_t sring = smem_u32(smem);
    const uint32_t spw = sring + C::NBF * C::PLANE_B;
    const uint32_t sxch = spw + C::NBP * C::PLANE_B;
    const uint32_t sbar = sxch + (uint32_t)(4 * C::XCH);   // NBF mbarriers, 8 bytes each
    const bool tma = p.use_tma != 0;
    if (tma) {
        if (threadIdx.x == 0) {
            for (int b = 0; b < C::NBF; b++) mbar_init(sbar + 8u * b, 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        __syncthreads();
    }
    unsigned phase = 0;     // bit b: parity of the next completion of barrier b
    unsigned pending = 0;   // bit b: a copy on barrier b has not been waited for
    CtxF3 c;
    c.in = p.in;
    c.out = p.out;
    c.pw = p.pw;
    c.nx = p.nx;
    c.ny = p.ny;
    c.nz = p.nz;
    c.plane = (long long)p.nx * p.ny;
    c.tsteps = p.tsteps;
    c.vec = p.vec;
    c.vec_pw = p.vec_pw;
    c.tid = threadIdx.x;
    c.lane = threadIdx.x & 31;
    c.wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 9; j++) c.k[j] = p.k[j];
    c.ca_amb = (KIND == KTHERM) ? __fmul_rn(p.k[6], p.k[8]) : 0.f;

    float PA[C::NS][VY][VX], QA[C::NS][VY][VX], PB[C::NS][VY][VX], QB[C::NS][VY][VX];
#pragma unroll
    for (int s = 0; s < C::NS; s++)
#pragma unroll
        for (int k = 0; k < VY; k++)
#pragma unroll
            for (int j = 0; j < VX; j++) PA[s][k][j] = QA[s][k][j] = PB[s][k][j] = QB[s][k][j] = 0.f;

    // segments: zslab > 0 -- pieces (tile column, z-slab), taken round-robin, so that the
    // blocks of one round stream neighbouring tile columns through the same z-planes together
    // and the halo one of them re-reads is still in L2; else a contiguous range of
    // (tile column, plane) units per block, balanced by cost on the host
    long long f = (long long)blockIdx.x * p.planes_per_cta, pc = blockIdx.x;
    const long long total = p.total_cols * p.nz;
    long long fend = min(f + p.planes_per_cta, total);
    if (p.starts) {   // cost-balanced ranges
        f = __ldg(p.starts + blockIdx.x);
        fend = __ldg(p.starts + blockIdx.x + 1);
    }
    for (;;) {
        long long col;
        int z0, z1;
        if (p.zslab > 0) {
            if (pc >= p.pieces) break;
            const long long sl = pc / p.total_cols;
            col = pc - sl * p.total_cols;
            z0 = (int)(sl * p.zslab);
            z1 = min(p.nz, z0 + p.zslab);
            pc += gridDim.x;
        } else {
            if (f >= fend) break;
            col = f / p.nz;
            z0 = (int)(f - col * p.nz);
            z1 = (int)min((long long)p.nz, (long long)z0 + (fend - f));
            f += z1 - z0;
        }
        const int ty = (int)(col / p.ntx), tx = (int)(col - (long long)ty * p.ntx);

        c.z0 = z0;
        c.z1 = z1;
        c.x0 = tx * C::CX - C::HX;
        c.y0 = ty * C::CY - C::HY;
        c.gx = c.x0 + VX * c.lane;
        c.gy = c.y0 + c.wid * VY;
        c.z_start = max(0, z0 - c.tsteps);
        c.last_plane = min(c.nz - 1, z1 - 1 + c.tsteps);
        c.lx0 = (c.gx == 0);
        const int rxj = (c.gx <= c.nx - 1 && c.nx - 1 < c.gx + VX) ? (c.nx - 1 - c.gx) : -1;
        c.rxm = rxj >= 0 ? (1u << rxj) : 0u;
        const int ky0 = (c.gy <= 0 && 0 < c.gy + VY) ? -c.gy : -1;
        const int kyn = (c.gy <= c.ny - 1 && c.ny - 1 < c.gy + VY) ? (c.ny - 1 - c.gy) : -1;
        c.ym0 = ky0 >= 0 ? (1u << ky0) : 0u;
        c.ymn = kyn >= 0 ? (1u << kyn) : 0u;
        c.edge_x = __any_sync(0xffffffffu, c.lx0 || rxj >= 0);
        c.edge_y = __any_sync(0xffffffffu, ky0 >= 0 || kyn >= 0);
        {
            const int xl = max(c.x0 + C::HX, 0), xh = min(c.x0 + C::HX + C::CX, c.nx);
            const int yl = max(c.y0 + C::HY, 0), yh = min(c.y0 + C::HY + C::CY, c.ny);
            unsigned msk = 0;
#pragma unroll
            for (int k = 0; k < VY; k++)
#pragma unroll
                for (int j = 0; j < VX; j++) {
                    const int x = c.gx + j, y = c.gy + k;
                    if (x >= xl && x < xh && y >= yl && y < yh) msk |= 1u << (VX * k + j);
                }
            c.st_mask = msk;
            constexpr unsigned ALL = (1u << VX) - 1u;
            unsigned rows = 0;
            bool fast = c.vec != 0;
#pragma unroll
            for (int k = 0; k < VY; k++) {
                const unsigned b = (msk >> (VX * k)) & ALL;
                if (b == ALL) rows |= 1u << k;
                else if (b != 0) fast = false;
            }
            c.st_rows = rows;
            c.st_fast = fast;
            c.st_off = (long long)c.gy * c.nx + c.gx;
        }
        const int n_it = z1 + T - c.z_start;
        const int bot_i = c.nz - c.z_start;
        const bool top = (c.z_start == 0);
        const bool partial = (c.tsteps < T);

        // load plane z into field slot `fs` (and power slot `ps`), on barrier fs when staged
        // by tensor-map copies (one elected thread), else by per-thread cp.async (one group)
        auto load = [&](int z, int fs, int ps) {
            if (z <= c.last_plane) {
                if (tma) {
                    if (threadIdx.x == 0) {
                        const uint32_t bar = sbar + 8u * fs;
                        mbar_expect_tx(bar, (KIND == KTHERM ? 2u : 1u) * C::PLANE_B);
                        tma_plane(sring + fs * C::PLANE_B, &tin, c.x0, c.y0, z, bar);
                        if (KIND == KTHERM) tma_plane(spw + ps * C::PLANE_B, &tpw, c.x0, c.y0, z, bar);
                    }
                    pending |= 1u << fs;
                } else {
                    tbf3_load<C::BX, C::BY, C::NT>(c, c.in + (long long)z * c.plane, c.vec,
                                                   sring + fs * C::PLANE_B);
                    if (KIND == KTHERM)
                        tbf3_load<C::BX, C::BY, C::NT>(c, c.pw + (long long)z * c.plane,
                                                       c.vec_pw, spw + ps * C::PLANE_B);
                }
            }
            if (!tma) cp_async_commit();
        };
        // on a failed wait: flag it, give the copies in flight a bounded chance to land, leave
        auto bail = [&]() {
            if (threadIdx.x == 0) atomicExch(p.err, 1);
            for (int b = 0; b < C::NBF; b++)
                if ((pending >> b) & 1u) (void)mbar_wait_bounded(sbar + 8u * b, (phase >> b) & 1u);
        };
#pragma unroll 1
        for (int j = 0; j < C::PF; j++) load(c.z_start + j, j, KIND == KTHERM ? j : 0);
        Slots3 sl;
        sl.f0 = 0;
        sl.p1 = KIND == KTHERM ? C::NBP - 1 : 0;
        int lf = C::PF, lp = KIND == KTHERM ? C::PF : 0;   // slots the next loads fill
        // wait for plane z_start + i, then refill the slot last read one iteration ago (plane
        // z-1 of stage 0; for power, plane z-T+1 of stage T-1) with plane z_start + i + PF
        auto prologue = [&](int i) -> bool {
            bool bad = false;
            if (tma) {
                const int b = sl.f0;
                if ((pending >> b) & 1u) {
                    bad = !mbar_wait_bounded(sbar + 8u * b, (phase >> b) & 1u);
                    phase ^= 1u << b;
                    pending &= ~(1u << b);
                }
            } else {
                cp_async_wait<C::PF - 1>();
            }
            if (__syncthreads_or(bad)) return false;
            // the slot refilled below was read through the generic proxy before the barrier
            if (tma && threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            load(c.z_start + i + C::PF, lf, lp);
            return true;
        };
        auto advance = [&]() {
            sl.f0 = sl.f0 + 1 == C::NBF ? 0 : sl.f0 + 1;
            lf = lf + 1 == C::NBF ? 0 : lf + 1;
            if (KIND == KTHERM) {
                sl.p1 = sl.p1 + 1 == C::NBP ? 0 : sl.p1 + 1;
                lp = lp + 1 == C::NBP ? 0 : lp + 1;
            }
        };
        auto special = [&](int i) { return partial || (top && i <= T) || i >= bot_i; };
        auto copy_back = [&]() {
#pragma unroll
            for (int s = 0; s < C::NS; s++)
#pragma unroll
                for (int k = 0; k < VY; k++)
#pragma unroll
                    for (int j = 0; j < VX; j++) {
                        PA[s][k][j] = PB[s][k][j];
                        QA[s][k][j] = QB[s][k][j];
                    }
        };
        // The partial sums alternate between two register sets (A -> B, then B -> A) so that
        // no iteration copies them; the rare special iterations run A -> B and copy back.
        // Tile columns away from the x and y domain edges run an instance without the clamp
        // fix-ups: their in-place updates of the plane otherwise cost register copies on every
        // path.  Returns false when a wait gave up.
        auto run = [&](auto edge_tag) -> bool {
            constexpr bool EDGE = decltype(edge_tag)::value;
            int i = 0;
#pragma unroll 1
            while (i < n_it) {
                if (!prologue(i)) return false;
                if (special(i)) {
                    tbf3_iter<KIND, T, VX, VY, NW, true, EDGE>(c, sring, spw, sxch, sl, PA, QA, PB, QB, i);
                    advance();
                    copy_back();
                    ++i;
                    continue;
                }
                tbf3_iter<KIND, T, VX, VY, NW, false, EDGE>(c, sring, spw, sxch, sl, PA, QA, PB, QB, i);
                advance();
                ++i;
                if (i < n_it && !special(i)) {
                    if (!prologue(i)) return false;
                    tbf3_iter<KIND, T, VX, VY, NW, false, EDGE>(c, sring, spw, sxch, sl, PB, QB, PA, QA, i);
                    advance();
                    ++i;
                } else {
                    copy_back();
                }
            }
            return true;
        };
        const bool edge = __syncthreads_or(c.edge_x || c.edge_y) != 0;
        if (!(edge ? run(std::true_type{}) : run(std::false_type{}))) {
            bail();
            return;
        }
        if (!tma) cp_async_wait<0>();
        __syncthreads();
    }
}

}  // namespace stn
