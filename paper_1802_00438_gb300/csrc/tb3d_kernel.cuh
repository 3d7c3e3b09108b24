// 3D temporally-blocked Jacobi sweep ("3.5D" blocking: 2D spatial blocking in x and y,
// streaming along z, temporal blocking by a chain of stages), one pass = `tsteps` (<= T) steps.
//
// Method (arXiv 1802.00438): 2D spatial blocking for 3D stencils with no blocking along z
// (Sec. 3.1), overlapped tiles whose halos have width >= rad*T (Eq. 2), stage t computing time
// step t a fixed number of planes behind stage t-1 (Sec. 3.2), halo computed redundantly and
// only the compute block written (Sec. 3.2), trailing stages forwarding when the pass fuses
// fewer than T steps (Sec. 3.2), clamped boundary at every stage (Sec. 5.1).
//
// GPU mapping.
//   Block  = NW warps stacked along y; tile = 64 (x) by BY = NW*VY (y) cells incl. halos
//            HX = roundup(T, 4) in x and HY = T in y.
//   Thread = 2 adjacent x cells of VY consecutive rows; a warp spans the whole tile width, so
//            x-neighbours are warp shuffles and the warp edges are the tile edges (halo).
//   y-neighbours inside a thread's rows are registers; the rows just above and below come
//            from the neighbouring warps through a shared-memory exchange of every thread's
//            first and last row, published one plane earlier (one barrier per plane).
//   Stage 0 reads its three planes (z-1, z, z+1 at time 0) from a shared-memory ring filled
//            by cp.async PF planes ahead; stages 1..T-1 keep their three-plane window of own
//            cells in registers, rotating through three register sets (three-phase unroll).
//   Power (Hotspot 3D) is read per stage from global memory (L2-resident across stages).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace stn {

template <int KIND, bool EXACT, int T, int VY, int NW>
struct TB3 {
    static constexpr int NT = 32 * NW;
    static constexpr int BX = 64;
    static constexpr int BY = NW * VY;
    static constexpr int HX = (T + 3) / 4 * 4;
    static constexpr int HY = T;
    static constexpr int CX = BX - 2 * HX;
    static constexpr int CY = BY - 2 * HY;
    static constexpr int PF = 2;
    static constexpr int NBF = PF + 3;
    static constexpr int NS = T > 1 ? T - 1 : 1;
    static constexpr int NXS = T > 1 ? T - 1 : 1;   // exchanged stage outputs
    static constexpr int PLANE = BX * BY;
    // exchange: [parity][stage][warp][top/bottom][BX]
    static constexpr size_t XCH = (size_t)2 * NXS * NW * 2 * BX;
    static constexpr size_t SMEM = sizeof(float) * ((size_t)NBF * PLANE + XCH);
    static_assert(CX > 0 && CY > 0, "tile smaller than its halos");
    static_assert(VY >= 1, "VY");
};

struct Ctx3 {
    const float *__restrict__ in;
    float *__restrict__ out;
    const float *__restrict__ pw;
    float *ring, *xch;
    int nx, ny, nz, tsteps;
    long long plane;       // nx * ny
    int x0, y0;            // tile origin
    int gx, gy;            // my first cell (global x, global y of row 0)
    int z_start, last_plane, z0, z1;
    bool edge;             // warp touches a domain edge in x or y
    int lx0, rx1;          // my cell 0 is x = 0 / my cell 1 is x = nx-1
    int ky0, kyn;          // my row index at y = 0 / y = ny-1, or -1
    unsigned ym0, ymn;     // the same as bit masks (a mask, not an index, keeps the rows in
                           // registers: a per-row compare would become an indexed store)
    unsigned st_mask;      // bit (k*2 + j): my cell (row k, x j) is stored
    int vec;
    int tid, lane, wid;
    float k[9];
    float ca_amb;
};

template <int KIND, bool EXACT>
__device__ __forceinline__ float upd3(const Ctx3 &c, float m, float w, float e, float s, float n,
                                      float b, float a, float p)
{
    if (KIND == KDIFF) return diff7<EXACT>(m, w, e, s, n, b, a, c.k);
    else return hot3<EXACT>(m, w, e, s, n, b, a, p, c.k, c.ca_amb);
}

template <int BX, int BY, int NT>
__device__ __forceinline__ void tb3_load_plane(const Ctx3 &c, int z, float *dst)
{
    constexpr int CH = BX / 4;           // 16-byte chunks per tile row
    constexpr int NCH = CH * BY;
    const float *src = c.in + (long long)z * c.plane;
#pragma unroll
    for (int qq = 0; qq < (NCH + NT - 1) / NT; qq++) {
        const int q = c.tid + qq * NT;
        if (NCH % NT == 0 || q < NCH) {
            const int row = q / CH, ch = q % CH;
            const int y = c.y0 + row, x = c.x0 + 4 * ch;
            float *d = dst + row * BX + 4 * ch;
            const bool yok = (y >= 0 && y < c.ny);
            const float *rs = src + (long long)(yok ? y : 0) * c.nx;
            if (c.vec) {
                const int nb = (yok && x >= 0 && x < c.nx) ? min(16, 4 * (c.nx - x)) : 0;
                cp_async16(d, nb ? rs + x : src, nb);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int xx = x + j;
                    const int nb = (yok && xx >= 0 && xx < c.nx) ? 4 : 0;
                    cp_async4(d + j, nb ? rs + xx : src, nb);
                }
            }
        }
    }
}

// Neighbours of my cells in a plane held as m[VY][2]: w/e by shuffle, n/s from my rows or the
// rows published by the warps above (nt) and below (sb); domain-edge clamps when c.edge.
template <int VY>
__device__ __forceinline__ void nb3(const Ctx3 &c, const float (&m)[VY][2], const float (&nt)[2],
                                    const float (&sb)[2], float (&w)[VY][2], float (&e)[VY][2],
                                    float (&n)[VY][2], float (&s)[VY][2])
{
#pragma unroll
    for (int k = 0; k < VY; k++) {
        const float wl = __shfl_sync(0xffffffffu, m[k][1], (c.lane + 31) & 31);
        const float er = __shfl_sync(0xffffffffu, m[k][0], (c.lane + 1) & 31);
        w[k][0] = wl;
        w[k][1] = m[k][0];
        e[k][0] = m[k][1];
        e[k][1] = er;
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
        n[0][j] = nt[j];
        s[VY - 1][j] = sb[j];
    }
#pragma unroll
    for (int k = 1; k < VY; k++)
#pragma unroll
        for (int j = 0; j < 2; j++) n[k][j] = m[k - 1][j];
#pragma unroll
    for (int k = 0; k < VY - 1; k++)
#pragma unroll
        for (int j = 0; j < 2; j++) s[k][j] = m[k + 1][j];
    if (c.edge) {
#pragma unroll
        for (int k = 0; k < VY; k++) {
            w[k][0] = c.lx0 ? m[k][0] : w[k][0];
            e[k][0] = (c.rx1 == 0) ? m[k][0] : e[k][0];
            e[k][1] = (c.rx1 == 1) ? m[k][1] : e[k][1];
#pragma unroll
            for (int j = 0; j < 2; j++) {
                n[k][j] = ((c.ym0 >> k) & 1u) ? m[k][j] : n[k][j];
                s[k][j] = ((c.ymn >> k) & 1u) ? m[k][j] : s[k][j];
            }
        }
    }
}

template <int VY>
__device__ __forceinline__ void tb3_store(const Ctx3 &c, int z, const float (&v)[VY][2])
{
    float *dst = c.out + (long long)z * c.plane + (long long)c.gy * c.nx + c.gx;
#pragma unroll
    for (int k = 0; k < VY; k++) {
        const unsigned b = (c.st_mask >> (2 * k)) & 3u;
        float *d = dst + (long long)k * c.nx;
        if (b == 3u && c.vec) {
            *reinterpret_cast<float2 *>(d) = make_float2(v[k][0], v[k][1]);
        } else {
            if (b & 1u) d[0] = v[k][0];
            if (b & 2u) d[1] = v[k][1];
        }
    }
}

template <int KIND, bool EXACT, int T, int VY, int NW>
__device__ __forceinline__ void tb3_power(const Ctx3 &c, int z, float (&p)[VY][2])
{
    if (KIND == KTHERM) {
        const int zz = min(max(z, 0), c.nz - 1);
        const float *src = c.pw + (long long)zz * c.plane;
#pragma unroll
        for (int k = 0; k < VY; k++) {
            const int y = min(max(c.gy + k, 0), c.ny - 1);
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int x = min(max(c.gx + j, 0), c.nx - 1);
                p[k][j] = __ldg(src + (long long)y * c.nx + x);
            }
        }
    }
}

template <int KIND, bool EXACT, int T, int VY, int NW, int P, bool SPECIAL>
__device__ __forceinline__ void tb3_iter(const Ctx3 &c,
                                         float (&B)[TB3<KIND, EXACT, T, VY, NW>::NS][3][VY][2],
                                         int i)
{
    using C = TB3<KIND, EXACT, T, VY, NW>;
    constexpr int PU = P, PM = (P + 1) % 3, PD = (P + 2) % 3;
    const int Z0 = c.z_start + i;
    float out[VY][2];

    // ---- stage 0 from the ring ---------------------------------------------------------------
    {
        const int R = Z0 - 1;
        int ru = R - 1, rd = Z0;
        if (SPECIAL) {
            ru = max(ru, 0);
            rd = min(rd, c.nz - 1);
        }
        const float *pu = c.ring + ((ru - c.z_start + 2 * C::NBF) % C::NBF) * C::PLANE;
        const float *pm = c.ring + ((R - c.z_start + 2 * C::NBF) % C::NBF) * C::PLANE;
        const float *pd = c.ring + ((rd - c.z_start + 2 * C::NBF) % C::NBF) * C::PLANE;
        const int r0 = c.wid * VY, xo = 2 * c.lane;
        float u[VY][2], m[VY][2], d[VY][2], w[VY][2], e[VY][2], n[VY][2], s[VY][2], p[VY][2];
#pragma unroll
        for (int k = 0; k < VY; k++) {
            const float2 a = *reinterpret_cast<const float2 *>(pu + (r0 + k) * C::BX + xo);
            const float2 b = *reinterpret_cast<const float2 *>(pm + (r0 + k) * C::BX + xo);
            const float2 f = *reinterpret_cast<const float2 *>(pd + (r0 + k) * C::BX + xo);
            u[k][0] = a.x; u[k][1] = a.y;
            m[k][0] = b.x; m[k][1] = b.y;
            d[k][0] = f.x; d[k][1] = f.y;
        }
        float nt[2], sb[2];
        {
            const int rn = r0 > 0 ? r0 - 1 : 0, rs = r0 + VY < C::BY ? r0 + VY : C::BY - 1;
            const float2 a = *reinterpret_cast<const float2 *>(pm + rn * C::BX + xo);
            const float2 b = *reinterpret_cast<const float2 *>(pm + rs * C::BX + xo);
            nt[0] = a.x; nt[1] = a.y;
            sb[0] = b.x; sb[1] = b.y;
        }
        nb3<VY>(c, m, nt, sb, w, e, n, s);
        tb3_power<KIND, EXACT, T, VY, NW>(c, R, p);
#pragma unroll
        for (int k = 0; k < VY; k++)
#pragma unroll
            for (int j = 0; j < 2; j++)
                out[k][j] = upd3<KIND, EXACT>(c, m[k][j], w[k][j], e[k][j], s[k][j], n[k][j],
                                              u[k][j], d[k][j], p[k][j]);
    }
    if constexpr (T == 1) {
        const int R = Z0 - 1;
        if (R >= c.z0 && R < c.z1) tb3_store<VY>(c, R, out);
        return;
    } else {
        float *X = c.xch;
        constexpr int XS = NW * 2 * C::BX;                 // floats per (parity, stage)
        const int xo = 2 * c.lane;
        const int wt = c.wid > 0 ? c.wid - 1 : 0;         // warp above (tile edge: any)
        const int wb = c.wid < NW - 1 ? c.wid + 1 : NW - 1;
        // publish stage 0's first and last rows, hand its plane to stage 1
        {
            float *o = X + ((i & 1) * C::NXS + 0) * XS + c.wid * 2 * C::BX + xo;
            *reinterpret_cast<float2 *>(o) = make_float2(out[0][0], out[0][1]);
            *reinterpret_cast<float2 *>(o + C::BX) = make_float2(out[VY - 1][0], out[VY - 1][1]);
        }
#pragma unroll
        for (int k = 0; k < VY; k++) {
            B[0][PD][k][0] = out[k][0];
            B[0][PD][k][1] = out[k][1];
        }
#pragma unroll
        for (int st = 1; st < T; st++) {
            const int R = Z0 - 1 - st;
            float(&Ws)[3][VY][2] = B[st - 1];
            if (SPECIAL && st >= c.tsteps) {
#pragma unroll
                for (int k = 0; k < VY; k++) {
                    out[k][0] = Ws[PM][k][0];
                    out[k][1] = Ws[PM][k][1];
                }
            } else {
                if (SPECIAL && R == c.nz - 1) {
#pragma unroll
                    for (int k = 0; k < VY; k++) {
                        Ws[PD][k][0] = Ws[PM][k][0];
                        Ws[PD][k][1] = Ws[PM][k][1];
                    }
                }
                float nt[2], sb[2];
                {
                    const float *rx = X + (((i - 1) & 1) * C::NXS + (st - 1)) * XS + xo;
                    const float2 a = *reinterpret_cast<const float2 *>(rx + (wt * 2 + 1) * C::BX);
                    const float2 b = *reinterpret_cast<const float2 *>(rx + (wb * 2 + 0) * C::BX);
                    nt[0] = a.x; nt[1] = a.y;
                    sb[0] = b.x; sb[1] = b.y;
                }
                float w[VY][2], e[VY][2], n[VY][2], s[VY][2], p[VY][2];
                nb3<VY>(c, Ws[PM], nt, sb, w, e, n, s);
                tb3_power<KIND, EXACT, T, VY, NW>(c, R, p);
#pragma unroll
                for (int k = 0; k < VY; k++)
#pragma unroll
                    for (int j = 0; j < 2; j++)
                        out[k][j] = upd3<KIND, EXACT>(c, Ws[PM][k][j], w[k][j], e[k][j], s[k][j],
                                                      n[k][j], Ws[PU][k][j], Ws[PD][k][j], p[k][j]);
                if (SPECIAL && R == -1) {
#pragma unroll
                    for (int k = 0; k < VY; k++) {
                        Ws[PM][k][0] = Ws[PD][k][0];
                        Ws[PM][k][1] = Ws[PD][k][1];
                    }
                }
            }
            if (st < T - 1) {
#pragma unroll
                for (int k = 0; k < VY; k++) {
                    B[st][PD][k][0] = out[k][0];
                    B[st][PD][k][1] = out[k][1];
                }
                float *o = X + ((i & 1) * C::NXS + st) * XS + c.wid * 2 * C::BX + xo;
                *reinterpret_cast<float2 *>(o) = make_float2(out[0][0], out[0][1]);
                *reinterpret_cast<float2 *>(o + C::BX) =
                    make_float2(out[VY - 1][0], out[VY - 1][1]);
            } else {
                if (R >= c.z0 && R < c.z1) tb3_store<VY>(c, R, out);
            }
        }
    }
}

template <int KIND, bool EXACT, int T, int VY, int NW>
__global__ void __launch_bounds__(32 * NW) k_tb3d(const Pass3D p)
{
    using C = TB3<KIND, EXACT, T, VY, NW>;
    // 128-byte aligned as in the 3D contracted kernel: both 3D kernels share translation
    // units, where the declarations of the dynamic shared array must agree
    extern __shared__ __align__(128) float smem[];
    Ctx3 c;
    c.in = p.in;
    c.out = p.out;
    c.pw = p.pw;
    c.ring = smem;
    c.xch = smem + C::NBF * C::PLANE;
    c.nx = p.nx;
    c.ny = p.ny;
    c.nz = p.nz;
    c.plane = (long long)p.nx * p.ny;
    c.tsteps = p.tsteps;
    c.vec = p.vec;
    c.tid = threadIdx.x;
    c.lane = threadIdx.x & 31;
    c.wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 9; j++) c.k[j] = p.k[j];
    c.ca_amb = (KIND == KTHERM) ? __fmul_rn(p.k[6], p.k[8]) : 0.f;

    float B[C::NS][3][VY][2];
#pragma unroll
    for (int s = 0; s < C::NS; s++)
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int k = 0; k < VY; k++) B[s][q][k][0] = B[s][q][k][1] = 0.f;

    long long f = (long long)blockIdx.x * p.planes_per_cta;
    const long long total = p.total_cols * p.nz;
    const long long fend = min(f + p.planes_per_cta, total);
    while (f < fend) {
        const long long col = f / p.nz;
        const int z0 = (int)(f - col * p.nz);
        const int z1 = (int)min((long long)p.nz, (long long)z0 + (fend - f));
        f += z1 - z0;
        const int ty = (int)(col / p.ntx), tx = (int)(col - (long long)ty * p.ntx);

        c.z0 = z0;
        c.z1 = z1;
        c.x0 = tx * C::CX - C::HX;
        c.y0 = ty * C::CY - C::HY;
        c.gx = c.x0 + 2 * c.lane;
        c.gy = c.y0 + c.wid * VY;
        c.z_start = max(0, z0 - c.tsteps);
        c.last_plane = min(c.nz - 1, z1 - 1 + c.tsteps);
        c.lx0 = (c.gx == 0);
        c.rx1 = (c.gx == c.nx - 1) ? 0 : ((c.gx + 1 == c.nx - 1) ? 1 : -1);
        c.ky0 = (c.gy <= 0 && 0 < c.gy + VY) ? -c.gy : -1;
        c.kyn = (c.gy <= c.ny - 1 && c.ny - 1 < c.gy + VY) ? (c.ny - 1 - c.gy) : -1;
        c.ym0 = c.ky0 >= 0 ? (1u << c.ky0) : 0u;
        c.ymn = c.kyn >= 0 ? (1u << c.kyn) : 0u;
        c.edge = __any_sync(0xffffffffu, c.lx0 || c.rx1 >= 0 || c.ky0 >= 0 || c.kyn >= 0);
        {
            const int xl = max(c.x0 + C::HX, 0), xh = min(c.x0 + C::HX + C::CX, c.nx);
            const int yl = max(c.y0 + C::HY, 0), yh = min(c.y0 + C::HY + C::CY, c.ny);
            unsigned msk = 0;
#pragma unroll
            for (int k = 0; k < VY; k++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const int x = c.gx + j, y = c.gy + k;
                    if (x >= xl && x < xh && y >= yl && y < yh) msk |= 1u << (2 * k + j);
                }
            c.st_mask = msk;
        }
        const int n_it = z1 + T - c.z_start;
        const int bot_i = c.nz - c.z_start;
        const bool top = (c.z_start == 0);
        const bool partial = (c.tsteps < T);

#pragma unroll 1
        for (int j = 0; j < C::PF; j++) {
            const int z = c.z_start + j;
            if (z <= c.last_plane)
                tb3_load_plane<C::BX, C::BY, C::NT>(c, z, c.ring + (j % C::NBF) * C::PLANE);
            cp_async_commit();
        }
        int i = 0;
#define STN_TB3_STEP(PH)                                                                       \
    if (i < n_it) {                                                                            \
        cp_async_wait<C::PF - 1>();                                                            \
        __syncthreads();                                                                       \
        if (partial || (top && i <= T) || i >= bot_i)                                          \
            tb3_iter<KIND, EXACT, T, VY, NW, PH, true>(c, B, i);                               \
        else                                                                                   \
            tb3_iter<KIND, EXACT, T, VY, NW, PH, false>(c, B, i);                              \
        {                                                                                      \
            const int z = c.z_start + i + C::PF;                                               \
            if (z <= c.last_plane)                                                             \
                tb3_load_plane<C::BX, C::BY, C::NT>(c, z,                                      \
                                                    c.ring + ((i + C::PF) % C::NBF) * C::PLANE); \
            cp_async_commit();                                                                 \
        }                                                                                      \
        ++i;                                                                                   \
    }
#pragma unroll 1
        while (i < n_it) {
            STN_TB3_STEP(0)
            STN_TB3_STEP(1)
            STN_TB3_STEP(2)
        }
#undef STN_TB3_STEP
        cp_async_wait<0>();
        __syncthreads();
    }
}

}  // namespace stn
