// Star diffusion of radius R in 2D (4R+1 points): combined spatial and temporal blocking with
// halos of width R*T (arXiv 1802.00438, Eqs. 1-2 with rad = R > 1, the paper's named
// extension to higher-order stencils; Sec. 3.2's fused steps; Sec. 5.1's clamped boundary).
//
// Persistent blocks, one per SM, take the 128 x 128 tiles (halos included) round-robin.  A tile
// arrives in shared memory by one tensor-map copy (or plain loads when rows are not 16-byte
// aligned), then `tsteps` steps run in shared memory between two buffers, the valid region
// shrinking by R per step from the tile edges (redundant halo work, Sec. 3.2), and only the
// compute block is stored.  Three tile buffers rotate: tile k lands in buffer k mod 3, steps
// between it and buffer (k+2) mod 3, while the next tile's copy lands in buffer (k+1) mod 3.  A thread owns
// 4 x-cells of 8 rows: per step it reads its column from R rows above to R rows below and, per
// row, the 4 cells on either side (16-byte shared loads), and evaluates each cell from the
// centre outwards in the oracle's order (exact: one rounding per operation; contracted: fused
// multiply-adds in the same order).
// Clamped edges: in a tile that reaches past the grid, every out-of-grid cell is set, before
// each step, to the value of the grid cell its coordinates clamp to; a star never reads a
// corner, so each in-grid cell then sees exactly its clamped neighbours at every distance.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace stn {

constexpr int SBX = 128, SBY = 128, SNW = 16, SVY = 8;   // tile, warps, rows per thread

template <int R, int T>
struct STAR {
    static constexpr int HX = (R * T + 3) / 4 * 4;   // 16-byte aligned tile origins
    static constexpr int HY = R * T;
    static constexpr int CX = SBX - 2 * HX;
    static constexpr int CY = SBY - 2 * HY;
    static constexpr size_t SMEM = 3 * (size_t)SBX * SBY * sizeof(float);   // three tiles
    static_assert(CX > 0 && CY > 0, "halos wider than the tile");
    static_assert(R >= 1 && R <= 4, "radius");
};

__device__ __forceinline__ float4 sld4(const float *a)
{
    return *reinterpret_cast<const float4 *>(a);
}

template <bool EXACT, int R>
__device__ __forceinline__ float star_cell(const float *k, float c, const float (&seg)[12], int j,
                                           const float *colv, int row)
{
    // colv[(R + row + dy) * 4 + j] is the cell dy rows below; seg[4 + j + dx] dx to the right
    float r = __fmul_rn(k[0], c);
#pragma unroll
    for (int d = 1; d <= R; d++) {
        const float *kd = k + 1 + 4 * (d - 1);
        const float w = seg[4 + j - d], e = seg[4 + j + d];
        const float s = colv[(R + row + d) * 4 + j], n = colv[(R + row - d) * 4 + j];
        if (EXACT) {
            r = __fadd_rn(r, __fmul_rn(kd[0], w));
            r = __fadd_rn(r, __fmul_rn(kd[1], e));
            r = __fadd_rn(r, __fmul_rn(kd[2], s));
            r = __fadd_rn(r, __fmul_rn(kd[3], n));
        } else {
            r = __fmaf_rn(kd[0], w, r);
            r = __fmaf_rn(kd[1], e, r);
            r = __fmaf_rn(kd[2], s, r);
            r = __fmaf_rn(kd[3], n, r);
        }
    }
    return r;
}

// out-of-grid cells of my 4 x 8 block take the value of the grid cell they clamp to
__device__ __forceinline__ void star_ghosts(float *buf, int x0, int y0, int lx, int ly, int nx,
                                            int ny)
{
#pragma unroll
    for (int k = 0; k < SVY; k++) {
        const int gy = y0 + ly + k;
        const int cy = min(max(gy, 0), ny - 1) - y0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int gx = x0 + lx + j;
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
            const int cx = min(max(gx, 0), nx - 1) - x0;
            buf[(ly + k) * SBX + lx + j] = buf[cy * SBX + cx];
        }
    }
}

template <bool EXACT, int R, int T>
__global__ void __launch_bounds__(32 * SNW, 1)
    k_star2d(const PassStar2D p, const __grid_constant__ CUtensorMap tin)
{
    using C = STAR<R, T>;
    constexpr int TS = SBX * SBY;
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bar[3];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int lx = 4 * lane, ly = SVY * wid;
    const int G = gridDim.x, ntiles = p.ntx * p.nty;
    const int nk = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    float k[1 + 4 * R];
#pragma unroll
    for (int i = 0; i < 1 + 4 * R; i++) k[i] = p.k[i];
    const uint32_t b0 = static_cast<uint32_t>(__cvta_generic_to_shared(&bar[0]));
    auto origin = [&](int kk, int &x0, int &y0) {
        const int t = (int)blockIdx.x + kk * G;
        x0 = (t % p.ntx) * C::CX - C::HX;
        y0 = (t / p.ntx) * C::CY - C::HY;
    };
    // thread 0: tile kk's copy into buffer kk mod 3, completing on that buffer's barrier
    auto issue = [&](int kk) {
        int x0, y0;
        origin(kk, x0, y0);
        const int s = kk % 3;
        const uint32_t b = b0 + 8u * s;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b),
                     "r"((uint32_t)(4 * TS))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
                static_cast<uint32_t>(__cvta_generic_to_shared(sm + s * TS))),
            "l"(reinterpret_cast<uint64_t>(&tin)), "r"(x0), "r"(y0), "r"(0), "r"(b)
            : "memory");
    };
    // bounded wait for tile kk's copy (phase (kk / 3) & 1 of its buffer's barrier)
    auto landed = [&](int kk) -> bool {
        const uint32_t b = b0 + 8u * (kk % 3), par = (uint32_t)((kk / 3) & 1);
        for (int n = 0; n < (1 << 22); n++) {
            uint32_t r;
            asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                         " selp.u32 %0, 1, 0, q;\n}\n"
                         : "=r"(r)
                         : "r"(b), "r"(par)
                         : "memory");
            if (r) return true;
        }
        return false;
    };

    if (p.use_tma) {
        if (tid == 0) {
            for (int s = 0; s < 3; s++)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b0 + 8u * s) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            if (nk > 0) issue(0);
        }
        __syncthreads();   // barriers initialised before anyone polls them
    }

    for (int kk = 0; kk < nk; kk++) {
        int x0, y0;
        origin(kk, x0, y0);
        float *cur = sm + (kk % 3) * TS, *nxt = sm + ((kk + 2) % 3) * TS;
        if (p.use_tma) {
            // the buffer of tile kk+1 was last read by tile kk-2's steps, before the barrier
            // that ended tile kk-1
            if (tid == 0 && kk + 1 < nk) issue(kk + 1);
            const bool ok = landed(kk);
            if (__syncthreads_or(!ok)) {   // a copy never completed: flag it and leave
                if (tid == 0) {
                    atomicExch(p.err, 1);
                    if (kk + 1 < nk) {   // give the next copy a bounded chance to land
                        (void)landed(kk + 1);
                    }
                }
                return;
            }
        } else {
#pragma unroll
            for (int kr = 0; kr < SVY; kr++) {
                const int gy = y0 + ly + kr;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int gx = x0 + lx + j;
                    const bool in = gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny;
                    cur[(ly + kr) * SBX + lx + j] = in ? __ldg(p.in + (long long)gy * p.ld_in + gx) : 0.f;
                }
            }
            __syncthreads();
        }
        const bool edge = x0 < 0 || y0 < 0 || x0 + SBX > p.nx || y0 + SBY > p.ny;   // block-uniform
        if (edge) {
            star_ghosts(cur, x0, y0, lx, ly, p.nx, p.ny);
            __syncthreads();
        }

        for (int t = 0; t < p.tsteps; t++) {
            // my column from R rows above to R rows below (clamped into the tile: rows past the
            // tile edge only feed halo cells, whose values are never stored)
            float colv[(SVY + 2 * R) * 4];
#pragma unroll
            for (int r = 0; r < SVY + 2 * R; r++) {
                const int row = min(max(ly - R + r, 0), SBY - 1);
                const float4 v = sld4(cur + row * SBX + lx);
                colv[4 * r] = v.x;
                colv[4 * r + 1] = v.y;
                colv[4 * r + 2] = v.z;
                colv[4 * r + 3] = v.w;
            }
            const int lxl = lane > 0 ? lx - 4 : lx, lxr = lane < 31 ? lx + 4 : lx;
#pragma unroll
            for (int kr = 0; kr < SVY; kr++) {
                const float *rowp = cur + (ly + kr) * SBX;
                const float4 a = sld4(rowp + lxl), c = sld4(rowp + lxr);
                float seg[12] = {a.x, a.y, a.z, a.w, colv[(R + kr) * 4], colv[(R + kr) * 4 + 1],
                                 colv[(R + kr) * 4 + 2], colv[(R + kr) * 4 + 3], c.x, c.y, c.z, c.w};
                float o[4];
#pragma unroll
                for (int j = 0; j < 4; j++) o[j] = star_cell<EXACT, R>(k, seg[4 + j], seg, j, colv, kr);
                *reinterpret_cast<float4 *>(nxt + (ly + kr) * SBX + lx) = make_float4(o[0], o[1], o[2], o[3]);
            }
            __syncthreads();
            if (edge) {
                star_ghosts(nxt, x0, y0, lx, ly, p.nx, p.ny);
                __syncthreads();
            }
            float *tt = cur;
            cur = nxt;
            nxt = tt;
        }

        // store my cells of the compute block that lie in the grid
        if (lx >= C::HX && lx < C::HX + C::CX) {
            const int gx = x0 + lx;
#pragma unroll
            for (int kr = 0; kr < SVY; kr++) {
                const int ry = ly + kr, gy = y0 + ry;
                if (ry < C::HY || ry >= C::HY + C::CY || gy >= p.ny) continue;
                const float4 v = sld4(cur + ry * SBX + lx);
                float *dst = p.out + (long long)gy * p.ld_out + gx;
                if (p.vec_out && gx + 3 < p.nx) {
                    *reinterpret_cast<float4 *>(dst) = v;
                } else {
                    if (gx < p.nx) dst[0] = v.x;
                    if (gx + 1 < p.nx) dst[1] = v.y;
                    if (gx + 2 < p.nx) dst[2] = v.z;
                    if (gx + 3 < p.nx) dst[3] = v.w;
                }
            }
        }
        __syncthreads();   // both buffers of this tile free before the next tile's copy
    }
}

}  // namespace stn
