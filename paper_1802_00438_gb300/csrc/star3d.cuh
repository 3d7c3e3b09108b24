// Star diffusion of radius R in 3D (6R+1 points; R = 2 is the 13-point stencil): spatial
// blocking in x and y with halos of width R*T, streaming along z, T fused steps per pass
// (arXiv 1802.00438, Eqs. 1-2 with rad = R > 1, the paper's named extension to higher-order
// stencils; Sec. 3.1's 2.5D blocking, Sec. 3.2's fused steps, Sec. 5.1's clamped boundary).
//
// One block per (64 x 64 tile incl. halos, z-segment).  A ring of shared-memory planes holds
// the time-0 planes z-R .. z+R of the tile plus PF planes in flight, each staged by one
// tensor-map copy (or per-thread loads when rows are not 16-byte aligned).  Stage 1 computes
// plane z at time 1 from them; with T = 2 its output goes to a second ring of 2R+1 planes and
// stage 2 computes plane z-R at time 2 from that ring.  The valid region shrinks by R per
// stage from the tile edges (redundant halo work, Sec. 3.2); only the compute block is
// stored.  A thread owns 4 x-cells of 4 rows: per row it reads the 4-cell chunks on either
// side (x-neighbours), its column from R rows above to R rows below (y-neighbours) and, per
// distance, the same 4 cells of planes z-d and z+d (z-neighbours), all 16-byte shared loads,
// and evaluates each cell from the centre outwards in the oracle's order (exact: one rounding
// per operation; contracted: fused multiply-adds in the same order).
// Clamped edges: in a tile that reaches past the grid in x or y, every out-of-grid cell of a
// plane is set to the value of the grid cell its coordinates clamp to before the plane is
// read; a star never reads a corner, so each in-grid cell sees its clamped neighbours.  Planes
// beyond the grid in z are the edge plane itself (the ring index clamps).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace stn {

constexpr int S3X = 64, S3Y = 64, S3NT = 256;   // tile (halos included), threads

template <int R, int T>
struct STAR3 {
    static constexpr int HX = (R * T + 3) / 4 * 4;   // 16-byte aligned tile origins
    static constexpr int HY = R * T;
    static constexpr int CX = S3X - 2 * HX;
    static constexpr int CY = S3Y - 2 * HY;
    static constexpr int PF = 2;                     // planes requested ahead
    static constexpr int N0 = 2 * R + 1 + PF;        // time-0 ring
    static constexpr int N1 = T > 1 ? 2 * R + 1 : 0; // time-1 ring
    static constexpr int PLANE = S3X * S3Y;          // floats per plane
    static constexpr size_t SMEM = (size_t)(N0 + N1) * PLANE * sizeof(float);
    // two resident blocks where their rings fit (1 KiB per block is reserved by the hardware)
    static constexpr int MINB = 2 * (SMEM + 1024 + 256) <= 227 * 1024 ? 2 : 1;
    static_assert(CX > 0 && CY > 0, "halos wider than the tile");
    static_assert(R >= 2 && R <= 4 && (T == 1 || T == 2), "radius / fused steps");
    static_assert(N0 <= 32, "pending-copy mask");
};

__device__ __forceinline__ float4 s3ld4(const float *a) { return *reinterpret_cast<const float4 *>(a); }

__device__ __forceinline__ void s3mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool s3mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded: a copy that never completes cannot hang the GPU
__device__ __forceinline__ bool s3mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int n = 0; n < (1 << 22); n++)
        if (s3mbar_try(bar, parity)) return true;
    return false;
}

// out-of-grid cells of my 4 x 4 block of a plane take the value of the grid cell they clamp to
__device__ __forceinline__ void s3_ghosts(float *pl, int x0, int y0, int lx, int ly, int nx, int ny)
{
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int gy = y0 + ly + r;
        const int cy = min(max(gy, 0), ny - 1) - y0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int gx = x0 + lx + j;
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
            const int cx = min(max(gx, 0), nx - 1) - x0;
            pl[(ly + r) * S3X + lx + j] = pl[cy * S3X + cx];
        }
    }
}

// One stage on plane z: my 16 cells from the ring plane `ctr` and the planes zb[d-1] (z-d)
// and za[d-1] (z+d), rows clamped into the tile (rows past its edge feed halo cells only).
template <bool EXACT, int R>
__device__ __forceinline__ void s3_stage(const float *k, const float *ctr, const float *const *zb,
                                         const float *const *za, int lx, int ly, float (&o)[4][4])
{
    // my column from R rows above to R rows below, centre chunk
    float col[4 + 2 * R][4];
#pragma unroll
    for (int r = 0; r < 4 + 2 * R; r++) {
        const int row = min(max(ly - R + r, 0), S3Y - 1);
        const float4 v = s3ld4(ctr + row * S3X + lx);
        col[r][0] = v.x; col[r][1] = v.y; col[r][2] = v.z; col[r][3] = v.w;
    }
    const int lxl = lx > 0 ? lx - 4 : lx, lxr = lx < S3X - 4 ? lx + 4 : lx;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const float *rowp = ctr + (ly + r) * S3X;
        const float4 a = s3ld4(rowp + lxl), b = s3ld4(rowp + lxr);
        const float seg[12] = {a.x, a.y, a.z, a.w, col[R + r][0], col[R + r][1], col[R + r][2],
                               col[R + r][3], b.x, b.y, b.z, b.w};
        float acc[4];
#pragma unroll
        for (int j = 0; j < 4; j++) acc[j] = __fmul_rn(k[0], seg[4 + j]);
#pragma unroll
        for (int d = 1; d <= R; d++) {
            const float *kd = k + 1 + 6 * (d - 1);
            const float4 vb = s3ld4(zb[d - 1] + (ly + r) * S3X + lx);
            const float4 va = s3ld4(za[d - 1] + (ly + r) * S3X + lx);
            const float pb[4] = {vb.x, vb.y, vb.z, vb.w}, pa[4] = {va.x, va.y, va.z, va.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float w = seg[4 + j - d], e = seg[4 + j + d];
                const float s = col[R + r + d][j], n = col[R + r - d][j];
                if (EXACT) {
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(kd[0], w));
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(kd[1], e));
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(kd[2], s));
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(kd[3], n));
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(kd[4], pb[j]));
                    acc[j] = __fadd_rn(acc[j], __fmul_rn(kd[5], pa[j]));
                } else {
                    acc[j] = __fmaf_rn(kd[0], w, acc[j]);
                    acc[j] = __fmaf_rn(kd[1], e, acc[j]);
                    acc[j] = __fmaf_rn(kd[2], s, acc[j]);
                    acc[j] = __fmaf_rn(kd[3], n, acc[j]);
                    acc[j] = __fmaf_rn(kd[4], pb[j], acc[j]);
                    acc[j] = __fmaf_rn(kd[5], pa[j], acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) o[r][j] = acc[j];
    }
}

template <bool EXACT, int R, int T>
__global__ void __launch_bounds__(S3NT, (STAR3<R, T>::MINB))
    k_star3d(const PassStar3D p, const __grid_constant__ CUtensorMap tin)
{
    using C = STAR3<R, T>;
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bars[C::N0];
    float *ring0 = sm, *ring1 = sm + C::N0 * C::PLANE;
    const int tid = threadIdx.x;
    const int lx = 4 * (tid & 15), ly = 4 * (tid >> 4);

    const int seg = blockIdx.x % p.nseg, colid = blockIdx.x / p.nseg;
    const int tx = colid % p.ntx, ty = colid / p.ntx;
    const int x0 = tx * C::CX - C::HX, y0 = ty * C::CY - C::HY;
    const int nz = p.nz;
    const int s0 = seg * p.zseg, s1 = min(nz, s0 + p.zseg);   // planes this block stores
    if (s0 >= s1) return;
    const int z1_lo = max(0, s0 - R * (T - 1)), z1_hi = min(nz - 1, s1 - 1 + R * (T - 1));
    const int z0_lo = max(0, z1_lo - R), z0_hi = min(nz - 1, z1_hi + R);
    const bool edge = x0 < 0 || y0 < 0 || x0 + S3X > p.nx || y0 + S3Y > p.ny;   // block-uniform
    float k[1 + 6 * R];
#pragma unroll
    for (int i = 0; i < 1 + 6 * R; i++) k[i] = p.k[i];

    const uint32_t bar0 = static_cast<uint32_t>(__cvta_generic_to_shared(&bars[0]));
    const bool tma = p.use_tma != 0;
    if (tma && tid == 0) {
        for (int b = 0; b < C::N0; b++) s3mbar_init(bar0 + 8u * b);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();   // barriers initialised before anyone polls them
    uint32_t pending = 0, phase = 0;   // per slot: a copy in flight; its completion parity

    auto slot0 = [&](int q) { return (q - z0_lo) % C::N0; };
    auto plane0 = [&](int q) { return ring0 + slot0(min(max(q, 0), nz - 1)) * C::PLANE; };
    auto slot1 = [&](int q) { return (q - z1_lo) % (C::N1 > 0 ? C::N1 : 1); };
    auto plane1 = [&](int q) { return ring1 + (C::N1 ? slot1(min(max(q, 0), nz - 1)) : 0) * C::PLANE; };

    // stage the time-0 plane q into its slot (tensor map: one elected thread, completion on the
    // slot's barrier; otherwise every thread copies its cells, clamped into the grid)
    auto issue = [&](int q) {
        const int b = slot0(q);
        if (tma) {
            if (tid == 0) {
                const uint32_t bar = bar0 + 8u * b;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                             "r"((uint32_t)(4 * C::PLANE))
                             : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(static_cast<uint32_t>(
                        __cvta_generic_to_shared(ring0 + b * C::PLANE))),
                    "l"(reinterpret_cast<uint64_t>(&tin)), "r"(x0), "r"(y0), "r"(q), "r"(bar)
                    : "memory");
            }
            pending |= 1u << b;
        } else {
            float *dst = ring0 + b * C::PLANE;
            const float *src = p.in + (long long)q * p.nx * p.ny;
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int gy = min(max(y0 + ly + r, 0), p.ny - 1);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int gx = min(max(x0 + lx + j, 0), p.nx - 1);
                    dst[(ly + r) * S3X + lx + j] = __ldg(src + (long long)gy * p.nx + gx);
                }
            }
        }
    };
    // wait for plane q; false if the bounded wait gave up
    auto land = [&](int q) -> bool {
        if (!tma) return true;
        const int b = slot0(q);
        bool ok = true;
        if ((pending >> b) & 1u) {
            ok = s3mbar_wait(bar0 + 8u * b, (phase >> b) & 1u);
            phase ^= 1u << b;
            pending &= ~(1u << b);
        }
        return ok;
    };
    // on a failed wait: flag it, give the copies in flight a bounded chance to land, leave
    auto bail = [&]() {
        if (tid == 0) atomicExch(p.err, 1);
        for (int b = 0; b < C::N0; b++)
            if ((pending >> b) & 1u) (void)s3mbar_wait(bar0 + 8u * b, (phase >> b) & 1u);
    };

    int next = z0_lo;    // next time-0 plane to stage
    int ready = z0_lo - 1;   // time-0 planes up to here have landed (and carry ghost cells)
    while (next <= min(z0_hi, z1_lo + R + C::PF)) issue(next++);

    for (int z1 = z1_lo;; z1++) {
        const bool do1 = z1 <= z1_hi;
        const int z2 = z1 - R * (T - 1);   // the plane the last stage emits
        if (!do1 && (T == 1 || z2 >= s1)) break;
        if (do1) {
            const int need = min(z1 + R, z0_hi);
            bool ok = true;
            while (ready < need) {
                ready++;
                ok = land(ready) && ok;
                if (!tma) __syncthreads();
                if (edge) s3_ghosts(plane0(ready), x0, y0, lx, ly, p.nx, p.ny);
            }
            if (__syncthreads_or(!ok)) {
                bail();
                return;
            }
            const float *zb[R], *za[R];
#pragma unroll
            for (int d = 1; d <= R; d++) {
                zb[d - 1] = plane0(z1 - d);
                za[d - 1] = plane0(z1 + d);
            }
            float o[4][4];
            s3_stage<EXACT, R>(k, plane0(z1), zb, za, lx, ly, o);
            if (T == 1) {
                if (z1 >= s0 && z1 < s1 && lx >= C::HX && lx < C::HX + C::CX) {
                    const int gx = x0 + lx;
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const int ry = ly + r, gy = y0 + ry;
                        if (ry < C::HY || ry >= C::HY + C::CY || gy >= p.ny) continue;
                        float *dst = p.out + ((long long)z1 * p.ny + gy) * p.nx + gx;
                        if (p.vec_out && gx + 3 < p.nx) {
                            *reinterpret_cast<float4 *>(dst) = make_float4(o[r][0], o[r][1], o[r][2], o[r][3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; j++)
                                if (gx + j < p.nx) dst[j] = o[r][j];
                        }
                    }
                }
            } else {
                float *dst = ring1 + slot1(z1) * C::PLANE;
#pragma unroll
                for (int r = 0; r < 4; r++)
                    *reinterpret_cast<float4 *>(dst + (ly + r) * S3X + lx) =
                        make_float4(o[r][0], o[r][1], o[r][2], o[r][3]);
            }
            __syncthreads();   // ring-0 reads done (its slots may refill), ring-1 plane complete
            if (T > 1 && edge) {
                s3_ghosts(ring1 + slot1(z1) * C::PLANE, x0, y0, lx, ly, p.nx, p.ny);
                __syncthreads();
            }
            while (next <= min(z0_hi, z1 + 1 + R + C::PF)) issue(next++);
        }
        if (T > 1 && z2 >= s0 && z2 < s1) {
            const float *zb[R], *za[R];
#pragma unroll
            for (int d = 1; d <= R; d++) {
                zb[d - 1] = plane1(z2 - d);
                za[d - 1] = plane1(z2 + d);
            }
            float o[4][4];
            if (p.tsteps >= 2) {
                s3_stage<EXACT, R>(k, plane1(z2), zb, za, lx, ly, o);
            } else {   // a one-step pass: the time-1 plane is the result
                const float *c1 = plane1(z2);
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int j = 0; j < 4; j++) o[r][j] = c1[(ly + r) * S3X + lx + j];
            }
            if (lx >= C::HX && lx < C::HX + C::CX) {
                const int gx = x0 + lx;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int ry = ly + r, gy = y0 + ry;
                    if (ry < C::HY || ry >= C::HY + C::CY || gy >= p.ny) continue;
                    float *dst = p.out + ((long long)z2 * p.ny + gy) * p.nx + gx;
                    if (p.vec_out && gx + 3 < p.nx) {
                        *reinterpret_cast<float4 *>(dst) = make_float4(o[r][0], o[r][1], o[r][2], o[r][3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (gx + j < p.nx) dst[j] = o[r][j];
                    }
                }
            }
        }
    }
    if (tma) {   // nothing may still be landing in the ring when the block retires
        bool ok = true;
        for (int b = 0; b < C::N0; b++)
            if ((pending >> b) & 1u) ok = s3mbar_wait(bar0 + 8u * b, (phase >> b) & 1u) && ok;
        if (!ok && tid == 0) atomicExch(p.err, 1);
    }
}

}  // namespace stn
