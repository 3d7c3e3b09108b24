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

#include <algorithm>
#include <cmath>
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

// Hotspot source row: p + amb*Rz (the product rounded once, as the kernels round it); one
// block row per grid row, four cells per thread (16-byte accesses when rows are aligned)
__global__ void __launch_bounds__(256) k_hot_source(const float *__restrict__ p, long long ld_p,
                                                    float *__restrict__ dst, int nx, float amb,
                                                    float rz, int vec)
{
    const int y = blockIdx.y;
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= nx) return;
    const float a = __fmul_rn(amb, rz);
    const float *src = p + (long long)y * ld_p + x;
    float *d = dst + (long long)y * nx + x;
    if (vec) {
        const float4 v = *reinterpret_cast<const float4 *>(src);
        *reinterpret_cast<float4 *>(d) =
            make_float4(__fadd_rn(v.x, a), __fadd_rn(v.y, a), __fadd_rn(v.z, a), __fadd_rn(v.w, a));
    } else {
        for (int j = 0; j < 4 && x + j < nx; j++) d[j] = __fadd_rn(src[j], a);
    }
}

}  // namespace

void hot_coeffs_src(const float *k, float *kf)
{
    // kf = [sdc, Rx', Ry', Rz, amb, fl(sdc*Ry'), -(2Rx' + 2Ry')] where Rx', Ry' are Rx, Ry with
    // the bits below half an ulp of 2Rx + 2Ry cleared, so that 2Rx' + 2Ry' is exact in float32:
    // the centre weight then cancels the four neighbour weights exactly on a uniform field and
    // the folded constant moves no fixed point (Rx', Ry' differ from Rx, Ry by < 1e-7 relative)
    const double rx = k[1], ry = k[2];
    double ul = std::ldexp(1.0, std::ilogb((float)(2.0 * rx + 2.0 * ry)) - 23);
    double rxq = 0, ryq = 0;
    for (int i = 0; i < 3; i++) {
        rxq = std::nearbyint(rx / (ul / 2)) * (ul / 2);
        ryq = std::nearbyint(ry / (ul / 2)) * (ul / 2);
        const double sum = 2 * rxq + 2 * ryq;
        if ((double)(float)sum == sum) break;
        ul *= 2;   // the sum crossed into the next binade
    }
    kf[0] = k[0];
    kf[1] = (float)rxq;
    kf[2] = (float)ryq;
    kf[3] = k[3];
    kf[4] = k[4];
    kf[5] = kf[0] * kf[2];
    kf[6] = -(float)(2 * rxq + 2 * ryq);
}

cudaError_t hot_source(const float *p, long long ld_p, float *dst, int nx, int ny, float amb,
                       float rz, cudaStream_t st)
{
    if (nx < 1 || ny < 1) return cudaErrorInvalidValue;
    const int vec = ((uintptr_t)p % 16 == 0) && ((uintptr_t)dst % 16 == 0) && (nx % 4 == 0) &&
                    (ld_p % 4 == 0);
    const unsigned bx = (unsigned)((nx + 1023) / 1024);
    // grid rows beyond the 65535 limit of gridDim.y go in slices
    for (long long y0 = 0; y0 < ny; y0 += 65535) {
        const unsigned rows = (unsigned)std::min<long long>(65535, ny - y0);
        k_hot_source<<<dim3(bx, rows), 256, 0, st>>>(p + y0 * ld_p, ld_p, dst + y0 * nx, nx, amb,
                                                     rz, vec);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
