// Block codec of the 16-bit grid storage (bf16 or fp16 with a float32 code per block), and the
// Hotspot source map p + amb*Rz that the contracted kernels stage instead of the power map.
//
// A block is the segment of one row that one tile column computes: cells
// [b*cx, min((b+1)*cx, nx)) of row y, with cx the compute width of the plan's tiling, so the
// kernel that writes a block is the only writer of its code.  Each block stores
// (offset, scale) = (mid-range, half-range) of its cells and every cell as q = (x - offset) /
// scale in [-1, 1] rounded to bf16 / fp16; x = offset + scale * q on load.  Precision is
// relative to the block's spread rather than to the values' magnitude, which matters for
// fields like temperatures (~330 K) whose bf16 ulp alone would be 2 K.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace stn {
namespace {

template <int STOR>
__device__ __forceinline__ unsigned enc(float x)
{
    if (STOR == 1) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

template <int STOR>
__device__ __forceinline__ float dec(unsigned q)
{
    if (STOR == 1) return __uint_as_float(q << 16);
    return __half2float(__ushort_as_half((unsigned short)q));
}

// one warp per block (row y, block b)
template <int STOR>
__global__ void __launch_bounds__(256) k_lp_encode(const float *__restrict__ src, long long ld_src,
                                                   uint16_t *__restrict__ dst, long long ld_q,
                                                   float2 *__restrict__ meta, int nx, int ny,
                                                   int cx, int ntx)
{
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)ny * ntx) return;
    const int y = (int)(wid / ntx), b = (int)(wid % ntx);
    const int x0 = b * cx, x1 = min(x0 + cx, nx);
    const float *row = src + (long long)y * ld_src;
    float lo = __int_as_float(0x7f800000), hi = -lo;
    for (int x = x0 + lane; x < x1; x += 32) {
        const float v = row[x];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    asm volatile("redux.sync.min.f32 %0, %0, 0xffffffff;\n" : "+f"(lo));
    asm volatile("redux.sync.max.f32 %0, %0, 0xffffffff;\n" : "+f"(hi));
    const float mid = 0.5f * (lo + hi);
    float sc = 0.5f * (hi - lo);
    sc = (sc > 0.f) ? sc : 1.f;
    const float inv = __frcp_rn(sc);
    uint16_t *q = dst + (long long)y * ld_q;
    for (int x = x0 + lane; x < x1; x += 32)
        q[x] = (uint16_t)enc<STOR>((row[x] - mid) * inv);   // |q| <= 1 + 3 * 2^-24: rounds to 1
    if (lane == 0) meta[(long long)y * ntx + b] = make_float2(mid, sc);
}

template <int STOR>
__global__ void __launch_bounds__(256) k_lp_decode(const uint16_t *__restrict__ src, long long ld_q,
                                                   const float2 *__restrict__ meta,
                                                   float *__restrict__ dst, long long ld_dst,
                                                   int nx, int ny, int cx, int ntx)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    const float2 m = meta[(long long)y * ntx + x / cx];
    dst[(long long)y * ld_dst + x] = __fmaf_rn(m.y, dec<STOR>(src[(long long)y * ld_q + x]), m.x);
}

// Hotspot source row: p + amb*Rz (the product rounded once, as the kernels round it)
__global__ void __launch_bounds__(256) k_hot_source(const float *__restrict__ p, long long ld_p,
                                                    float *__restrict__ dst, int nx, int ny,
                                                    float amb, float rz)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    dst[i] = __fadd_rn(p[(long long)y * ld_p + x], __fmul_rn(amb, rz));
}

}  // namespace

cudaError_t hot_source(const float *p, long long ld_p, float *dst, int nx, int ny, float amb,
                       float rz, cudaStream_t st)
{
    const long long n = (long long)nx * ny;
    k_hot_source<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, ld_p, dst, nx, ny, amb, rz);
    return cudaGetLastError();
}

cudaError_t lp_encode(int stor, const float *src, long long ld_src, void *dst, long long ld_q,
                      float2 *meta, int nx, int ny, int cx, cudaStream_t st)
{
    const int ntx = (nx + cx - 1) / cx;
    const long long warps = (long long)ny * ntx;
    const int blocks = (int)((warps * 32 + 255) / 256);
    uint16_t *q = static_cast<uint16_t *>(dst);
    if (stor == 1) k_lp_encode<1><<<blocks, 256, 0, st>>>(src, ld_src, q, ld_q, meta, nx, ny, cx, ntx);
    else k_lp_encode<2><<<blocks, 256, 0, st>>>(src, ld_src, q, ld_q, meta, nx, ny, cx, ntx);
    return cudaGetLastError();
}

cudaError_t lp_decode(int stor, const void *src, long long ld_q, const float2 *meta, float *dst,
                      long long ld_dst, int nx, int ny, int cx, cudaStream_t st)
{
    const int ntx = (nx + cx - 1) / cx;
    const long long n = (long long)nx * ny;
    const int blocks = (int)((n + 255) / 256);
    const uint16_t *q = static_cast<const uint16_t *>(src);
    if (stor == 1) k_lp_decode<1><<<blocks, 256, 0, st>>>(q, ld_q, meta, dst, ld_dst, nx, ny, cx, ntx);
    else k_lp_decode<2><<<blocks, 256, 0, st>>>(q, ld_q, meta, dst, ld_dst, nx, ny, cx, ntx);
    return cudaGetLastError();
}

}  // namespace stn
