// 3D temporally-blocked Jacobi sweep, contracted arithmetic, partial sums along z.
//
// Method (arXiv 1802.00438): 2D spatial blocking in x and y with streaming along z (Sec. 3.1),
// overlapped tiles with halos of width >= rad*T (Eq. 2), a chain of T stages where stage t
// computes time step t one plane behind stage t-1 (Sec. 3.2), redundant halo computation with
// only the compute block written (Sec. 3.2), trailing stages forwarding when a pass fuses fewer
// than T steps (Sec. 3.2), clamped boundaries at every stage (Sec. 5.1).
//
// GPU mapping (same tile and thread layout as k_tb3d: tile 64 x NW*VY cells, a thread owns 2
// adjacent x cells of VY consecutive rows, warps stacked along y).
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
#include "tb3d_kernel.cuh"

namespace stn {

template <int KIND, int T, int VY, int NW>
struct TB3F {
    static constexpr int NT = 32 * NW;
    static constexpr int BX = 64;
    static constexpr int BY = NW * VY;
    static constexpr int HX = (T + 3) / 4 * 4;
    static constexpr int HY = T;
    static constexpr int CX = BX - 2 * HX;
    static constexpr int CY = BY - 2 * HY;
    static constexpr int PF = KIND == KTHERM ? 2 : 3;   // planes in flight past the newest read
    static constexpr int NBF = PF + 3;                   // field ring: planes z-1, z, z+1 + PF
    // power ring: planes z-max(T-1,1) .. z+PF (stage 0 reads plane z-1 also when T = 1)
    static constexpr int NBP = KIND == KTHERM ? (T > 1 ? T : 2) + PF : 0;
    static constexpr int NS = T > 1 ? T - 1 : 1;
    static constexpr int PLANE = BX * BY;
    static constexpr uint32_t PLANE_B = 4u * PLANE;
    static constexpr size_t XCH = (size_t)NS * NW * 2 * BX;   // [stage][warp][top/bottom][BX]
    static constexpr size_t SMEM = sizeof(float) * ((size_t)(NBF + NBP) * PLANE + XCH);
    static_assert(CX > 0 && CY > 0, "tile smaller than its halos");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ float2 lds2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts2(uint32_t a, float x, float y)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x), "f"(y) : "memory");
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

// Stage the tile's window of one plane (z-plane base `src`) into the slot at `dst`; cells
// outside the domain arrive as zeros.
template <int BX, int BY, int NT>
__device__ __forceinline__ void tbf3_load(const Ctx3 &c, const float *src, int vec, uint32_t dst)
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

// Ring slots of the current iteration: field planes Z0-2, Z0-1, Z0 and power plane Z0-1.
struct Slots3 {
    int f0;   // field slot of Z0
    int p1;   // power slot of Z0 - 1
};

template <int KIND, int T, int VY, int NW, bool SPECIAL>
__device__ __forceinline__ void tbf3_iter(const Ctx3 &c, uint32_t sring, uint32_t spw,
                                          uint32_t sxch, const Slots3 &sl,
                                          float (&P)[TB3F<KIND, T, VY, NW>::NS][VY][2],
                                          float (&Q)[TB3F<KIND, T, VY, NW>::NS][VY][2], int i)
{
    using C = TB3F<KIND, T, VY, NW>;
    const int Z0 = c.z_start + i;   // newest plane in the ring
    const float cc = c.k[0], cw = c.k[1], ce = c.k[2], cs = c.k[3], cn = c.k[4], cb = c.k[5],
                ca = c.k[6];
    const uint32_t own = 4u * (c.wid * VY * C::BX + 2 * c.lane);   // my row 0, cell 0
    float d[VY][2];

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
        float u[VY][2], m[VY][2], a[VY][2], w[VY][2], e[VY][2], n[VY][2], s[VY][2], p[VY][2];
#pragma unroll
        for (int k = 0; k < VY; k++) {
            const float2 x = lds2(au + 4u * k * C::BX);
            const float2 y = lds2(am + 4u * k * C::BX);
            const float2 z = lds2(ad + 4u * k * C::BX);
            u[k][0] = x.x; u[k][1] = x.y;
            m[k][0] = y.x; m[k][1] = y.y;
            a[k][0] = z.x; a[k][1] = z.y;
        }
        float nt[2], sb[2];
        {
            const int up = c.wid > 0 ? -1 : 0, dn = c.wid < NW - 1 ? VY : VY - 1;
            const float2 x = lds2(am + 4 * up * C::BX);
            const float2 y = lds2(am + 4 * dn * C::BX);
            nt[0] = x.x; nt[1] = x.y;
            sb[0] = y.x; sb[1] = y.y;
        }
        nb3<VY>(c, m, nt, sb, w, e, n, s);
        if (KIND == KTHERM) {
            const uint32_t ap = spw + pm * C::PLANE_B + own;
#pragma unroll
            for (int k = 0; k < VY; k++) {
                const float2 x = lds2(ap + 4u * k * C::BX);
                p[k][0] = x.x;
                p[k][1] = x.y;
            }
        }
#pragma unroll
        for (int k = 0; k < VY; k++)
#pragma unroll
            for (int j = 0; j < 2; j++)
                d[k][j] = upd3<KIND, false>(c, m[k][j], w[k][j], e[k][j], s[k][j], n[k][j],
                                            u[k][j], a[k][j], KIND == KTHERM ? p[k][j] : 0.f);
    }
    if constexpr (T == 1) {
        const int R = Z0 - 1;
        if (R >= c.z0 && R < c.z1) tb3_store<VY>(c, R, d);
    } else {
        constexpr uint32_t XS = 4u * NW * 2 * C::BX;   // bytes per stage in the exchange
        const uint32_t xo = 8u * c.lane;
        const int wt = c.wid > 0 ? c.wid - 1 : 0;   // warp above (tile edge: any in-bounds row)
        const int wb = c.wid < NW - 1 ? c.wid + 1 : NW - 1;
#pragma unroll
        for (int st = 1; st < T; st++) {
            const int zc = Z0 - st;   // plane of d (output of stage st-1)
            float o[VY][2];
            if (SPECIAL && st >= c.tsteps) {
                // forwarding stage: one plane of delay, no arithmetic
#pragma unroll
                for (int k = 0; k < VY; k++)
#pragma unroll
                    for (int j = 0; j < 2; j++) {
                        o[k][j] = Q[st - 1][k][j];
                        Q[st - 1][k][j] = d[k][j];
                    }
            } else {
                const uint32_t xw = sxch + (st - 1) * XS + xo;
                sts2(xw + 4u * (c.wid * 2 + 0) * C::BX, d[0][0], d[0][1]);
                sts2(xw + 4u * (c.wid * 2 + 1) * C::BX, d[VY - 1][0], d[VY - 1][1]);
                __syncthreads();
                float nt[2], sb[2];
                {
                    const float2 x = lds2(xw + 4u * (wt * 2 + 1) * C::BX);
                    const float2 y = lds2(xw + 4u * (wb * 2 + 0) * C::BX);
                    nt[0] = x.x; nt[1] = x.y;
                    sb[0] = y.x; sb[1] = y.y;
                }
                float w[VY][2], e[VY][2], n[VY][2], s[VY][2], p[VY][2];
                nb3<VY>(c, d, nt, sb, w, e, n, s);
                if (KIND == KTHERM) {
                    int ps;
                    if (SPECIAL)
                        ps = slot_of<C::NBP ? C::NBP : 1>(min(max(zc, 0), c.nz - 1) - c.z_start);
                    else
                        ps = slot_back<C::NBP ? C::NBP : 1>(sl.p1, st - 1);
                    const uint32_t ap = spw + ps * C::PLANE_B + own;
#pragma unroll
                    for (int k = 0; k < VY; k++) {
                        const float2 x = lds2(ap + 4u * k * C::BX);
                        p[k][0] = x.x;
                        p[k][1] = x.y;
                    }
                }
                float(&Ps)[VY][2] = P[st - 1];
                float(&Qs)[VY][2] = Q[st - 1];
                if (!SPECIAL || zc < c.nz) {
                    const bool first = SPECIAL && zc == 0;   // clamp: plane -1 is plane 0
#pragma unroll
                    for (int k = 0; k < VY; k++)
#pragma unroll
                        for (int j = 0; j < 2; j++) {
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
                            Ps[k][j] = r;
                            Qs[k][j] = qn;
                        }
                } else if (zc == c.nz) {
                    // virtual plane nz (= plane nz-1): finish plane nz-1 and keep it
#pragma unroll
                    for (int k = 0; k < VY; k++)
#pragma unroll
                        for (int j = 0; j < 2; j++) {
                            o[k][j] = __fmaf_rn(ca, d[k][j], Ps[k][j]);
                            Ps[k][j] = o[k][j];
                        }
                } else {
#pragma unroll
                    for (int k = 0; k < VY; k++)
#pragma unroll
                        for (int j = 0; j < 2; j++) o[k][j] = Ps[k][j];
                }
            }
#pragma unroll
            for (int k = 0; k < VY; k++)
#pragma unroll
                for (int j = 0; j < 2; j++) d[k][j] = o[k][j];
        }
        const int R = Z0 - T;
        if (R >= c.z0 && R < c.z1) tb3_store<VY>(c, R, d);
    }
}

template <int KIND, int T, int VY, int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_tb3f(const Pass3D p)
{
    using C = TB3F<KIND, T, VY, NW>;
    extern __shared__ __align__(16) float smem[];
    const uint32_t sring = smem_u32(smem);
    const uint32_t spw = sring + C::NBF * C::PLANE_B;
    const uint32_t sxch = spw + C::NBP * C::PLANE_B;
    Ctx3 c;
    c.in = p.in;
    c.out = p.out;
    c.pw = p.pw;
    c.ring = nullptr;
    c.xch = nullptr;
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

    float P[C::NS][VY][2], Q[C::NS][VY][2];
#pragma unroll
    for (int s = 0; s < C::NS; s++)
#pragma unroll
        for (int k = 0; k < VY; k++)
#pragma unroll
            for (int j = 0; j < 2; j++) P[s][k][j] = Q[s][k][j] = 0.f;

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
            if (z <= c.last_plane) {
                tbf3_load<C::BX, C::BY, C::NT>(c, c.in + (long long)z * c.plane, c.vec,
                                               sring + j * C::PLANE_B);
                if (KIND == KTHERM)
                    tbf3_load<C::BX, C::BY, C::NT>(c, c.pw + (long long)z * c.plane, p.vec_pw,
                                                   spw + j * C::PLANE_B);
            }
            cp_async_commit();
        }
        Slots3 sl;
        sl.f0 = 0;
        sl.p1 = KIND == KTHERM ? C::NBP - 1 : 0;
        int lf = C::PF, lp = KIND == KTHERM ? C::PF : 0;   // slots the next loads fill
#pragma unroll 1
        for (int i = 0; i < n_it; i++) {
            cp_async_wait<C::PF - 1>();
            __syncthreads();
            {
                // the field slot refilled here was last read (as plane z-1 of stage 0) one
                // iteration ago, and the power slot (plane z-T+1 of stage T-1) too
                const int z = c.z_start + i + C::PF;
                if (z <= c.last_plane) {
                    tbf3_load<C::BX, C::BY, C::NT>(c, c.in + (long long)z * c.plane, c.vec,
                                                   sring + lf * C::PLANE_B);
                    if (KIND == KTHERM)
                        tbf3_load<C::BX, C::BY, C::NT>(c, c.pw + (long long)z * c.plane,
                                                       p.vec_pw, spw + lp * C::PLANE_B);
                }
                cp_async_commit();
            }
            if (partial || (top && i <= T) || i >= bot_i)
                tbf3_iter<KIND, T, VY, NW, true>(c, sring, spw, sxch, sl, P, Q, i);
            else
                tbf3_iter<KIND, T, VY, NW, false>(c, sring, spw, sxch, sl, P, Q, i);
            sl.f0 = sl.f0 + 1 == C::NBF ? 0 : sl.f0 + 1;
            lf = lf + 1 == C::NBF ? 0 : lf + 1;
            if (KIND == KTHERM) {
                sl.p1 = sl.p1 + 1 == C::NBP ? 0 : sl.p1 + 1;
                lp = lp + 1 == C::NBP ? 0 : lp + 1;
            }
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

}  // namespace stn
