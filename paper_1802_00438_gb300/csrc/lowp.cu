// Block codec of the 16-bit grid storage (bf16 or fp16 with a float32 code per block), and the
// Hotspot source map sdc*(p + amb*Rz) that the contracted kernels stage instead of the power map.
//
// A block is the segment of one row that one tile column computes: cells
// [b*cx, min((b+1)*cx, nx)) of row y, with cx the compute width of the plan's tiling, so the
// kernel that writes a block is the only writer of its code.  Each block stores a float32
// (offset, scale) and every cell as q = (x - offset) / scale rounded to bf16 / fp16;
// x = offset + scale * q on load.  The encoder here (before the first pass) takes the block's
// mid-range and half-range, q in [-1, 1]; the passes take the block's first cell and scale 1,
// which needs no block-wide minimum and maximum (bf16 and fp16 are floating point, so q keeps
// its 8 or 11 significant bits at any size).  Either way the precision is relative to the
// block's spread rather than to the values' magnitude, which matters for fields like
// temperatures (~330 K) whose bf16 ulp alone would be 2 K.
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
// with src_mul != 0 the values coded are the Hotspot source map sdc*(p + amb*Rz) of the power
// map src (src_mul = sdc, src_add = amb*Rz), rounded as k_hot_source rounds them
template <int STOR>
__global__ void __launch_bounds__(256) k_lp_encode(const float *__restrict__ src, long long ld_src,
                                                   uint16_t *__restrict__ dst, long long ld_q,
                                                   float2 *__restrict__ meta, int nx, int ny,
                                                   int cx, int ntx, float src_add, float src_mul)
{
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)ny * ntx) return;
    const int y = (int)(wid / ntx), b = (int)(wid % ntx);
    const int x0 = b * cx, x1 = min(x0 + cx, nx);
    const float *row = src + (long long)y * ld_src;
    float lo = __int_as_float(0x7f800000), hi = -lo;
    auto val = [&](int x) {
        const float v = row[x];
        return src_mul != 0.f ? __fmul_rn(src_mul, __fadd_rn(v, src_add)) : v;
    };
    for (int x = x0 + lane; x < x1; x += 32) {
        const float v = val(x);
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
        q[x] = (uint16_t)enc<STOR>((val(x) - mid) * inv);   // |q| <= 1 + 3 * 2^-24: rounds to 1
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

// Hotspot source row: sdc*(p + amb*Rz), each operation rounded once; one block row per grid
// row, four cells per thread (16-byte accesses when rows are aligned)
__global__ void __launch_bounds__(256) k_hot_source(const float *__restrict__ p, long long ld_p,
                                                    float *__restrict__ dst, long long ld_d, int nx,
                                                    float amb, float rz, float sdc, int vec)
{
    const int y = blockIdx.y;
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= nx) return;
    const float a = __fmul_rn(amb, rz);
    const float *src = p + (long long)y * ld_p + x;
    float *d = dst + (long long)y * ld_d + x;
    if (vec) {
        const float4 v = *reinterpret_cast<const float4 *>(src);
        *reinterpret_cast<float4 *>(d) =
            make_float4(__fmul_rn(sdc, __fadd_rn(v.x, a)), __fmul_rn(sdc, __fadd_rn(v.y, a)),
                        __fmul_rn(sdc, __fadd_rn(v.z, a)), __fmul_rn(sdc, __fadd_rn(v.w, a)));
    } else {
        for (int j = 0; j < 4 && x + j < nx; j++) d[j] = __fmul_rn(sdc, __fadd_rn(src[j], a));
    }
}

}  // namespace

void hot_coeffs_src(const float *k, float *kf)
{
    // The Hotspot update c + sdc*(p + (n+s-2c)*Ry + (e+w-2c)*Rx + (amb-c)*Rz) (Table 2) as
    //   cc*c + cx*(e+w) + cy*(n+s) - cz*c + src,   src = sdc*(p + amb*Rz) (a per-cell map)
    // with cx = sdc*Rx, cy = sdc*Ry, cz = sdc*Rz and cc = 1 - 2cx - 2cy.  cx and cy are sdc*Rx,
    // sdc*Ry rounded to multiples of half an ulp of cc, so that cc is exact in float32 and
    // cc + 2cx + 2cy = 1 holds exactly: a uniform field then loses exactly cz*c per step to the
    // ambient term and gains src, with no drift from rounded weights (the weights move by less
    // than 2e-7 relative).  kf = [cc, cx, cy, cz, amb, cy, 0].
    const double sdc = k[0], rx = k[1], ry = k[2], rz = k[3];
    const double cx0 = sdc * rx, cy0 = sdc * ry;
    double cxq = cx0, cyq = cy0, cc = 1.0 - 2 * cx0 - 2 * cy0;
    if (cc > 0.0) {
        double ul = std::ldexp(1.0, std::ilogb((float)cc) - 23);
        for (int i = 0; i < 4; i++) {
            cxq = std::nearbyint(cx0 / (ul / 2)) * (ul / 2);
            cyq = std::nearbyint(cy0 / (ul / 2)) * (ul / 2);
            cc = 1.0 - 2 * cxq - 2 * cyq;
            if ((double)(float)cc == cc && (double)(float)cxq == cxq && (double)(float)cyq == cyq)
                break;
            ul /= 2;   // cc fell into the binade below
        }
    }
    kf[0] = (float)cc;
    kf[1] = (float)cxq;
    kf[2] = (float)cyq;
    kf[3] = (float)(sdc * rz);
    kf[4] = k[4];
    kf[5] = (float)cyq;
    kf[6] = 0.f;
}

cudaError_t hot_source(const float *p, long long ld_p, float *dst, long long ld_d, int nx, int ny,
                       float amb, float rz, float sdc, cudaStream_t st)
{
    if (nx < 1 || ny < 1) return cudaErrorInvalidValue;
    const int vec = ((uintptr_t)p % 16 == 0) && ((uintptr_t)dst % 16 == 0) && (nx % 4 == 0) &&
                    (ld_p % 4 == 0) && (ld_d % 4 == 0);
    const unsigned bx = (unsigned)((nx + 1023) / 1024);
    // grid rows beyond the 65535 limit of gridDim.y go in slices
    for (long long y0 = 0; y0 < ny; y0 += 65535) {
        const unsigned rows = (unsigned)std::min<long long>(65535, ny - y0);
        k_hot_source<<<dim3(bx, rows), 256, 0, st>>>(p + y0 * ld_p, ld_p, dst + y0 * ld_d, ld_d, nx,
                                                     amb, rz, sdc, vec);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t lp_encode(int stor, const float *src, long long ld_src, void *dst, long long ld_q,
                      float2 *meta, int nx, int ny, int cx, cudaStream_t st, float src_add,
                      float src_mul)
{
    const int ntx = (nx + cx - 1) / cx;
    const long long warps = (long long)ny * ntx;
    const int blocks = (int)((warps * 32 + 255) / 256);
    uint16_t *q = static_cast<uint16_t *>(dst);
    if (stor == 1)
        k_lp_encode<1><<<blocks, 256, 0, st>>>(src, ld_src, q, ld_q, meta, nx, ny, cx, ntx, src_add,
                                               src_mul);
    else
        k_lp_encode<2><<<blocks, 256, 0, st>>>(src, ld_src, q, ld_q, meta, nx, ny, cx, ntx, src_add,
                                               src_mul);
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
