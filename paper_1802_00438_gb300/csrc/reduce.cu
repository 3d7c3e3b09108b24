// Float64 verification reductions over grids: sums, energies, maximum magnitudes and the
// L2 / L-infinity norms of a difference.  Deterministic: a fixed block partition that depends
// only on n, fixed-order shuffle trees inside blocks, and one fixed-order pass over the
// per-block partials in a second kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stencil.h"

namespace {

constexpr int kBlocks = 1024;   // partial slots (grid of the first kernel is at most this)
constexpr int kThreads = 256;
constexpr int kVals = 8;        // sum_a, sumsq_a, max|a|, sum_b, sumsq_b, max|b|, sumsq_d, max|d|

template <int TYPE>
__device__ __forceinline__ double load(const void *p, long long i)
{
    if (TYPE == ST_F64) return static_cast<const double *>(p)[i];
    return (double)static_cast<const float *>(p)[i];
}

__device__ __forceinline__ void warp_reduce(double (&v)[kVals])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < kVals; k++) {
            const double o = __shfl_down_sync(0xffffffffu, v[k], off);
            const bool is_max = (k == 2 || k == 5 || k == 7);
            v[k] = is_max ? fmax(v[k], o) : v[k] + o;
        }
    }
}

__device__ __forceinline__ void block_reduce(double (&v)[kVals], double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_reduce(v);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kVals; k++) sh[wid * kVals + k] = v[k];
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x / 32;
#pragma unroll
        for (int k = 0; k < kVals; k++) v[k] = lane < nw ? sh[lane * kVals + k] : 0.0;
        warp_reduce(v);
    }
}

template <int TA, int TB>
__global__ void __launch_bounds__(kThreads) k_reduce_partial(const void *a, const void *b,
                                                             long long n, long long chunk,
                                                             double *partials)
{
    __shared__ double sh[(kThreads / 32) * kVals];
    double v[kVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double x = load<TA>(a, i);
        v[0] += x;
        v[1] += x * x;
        v[2] = fmax(v[2], fabs(x));
        if (TB >= 0) {
            const double y = load<TB>(b, i);
            const double d = x - y;
            v[3] += y;
            v[4] += y * y;
            v[5] = fmax(v[5], fabs(y));
            v[6] += d * d;
            v[7] = fmax(v[7], fabs(d));
        }
    }
    block_reduce(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kVals; k++) partials[blockIdx.x * kVals + k] = v[k];
}

__global__ void __launch_bounds__(kBlocks) k_reduce_final(const double *partials, int nblocks,
                                                          double *out)
{
    __shared__ double sh[(kBlocks / 32) * kVals];
    double v[kVals];
#pragma unroll
    for (int k = 0; k < kVals; k++)
        v[k] = (int)threadIdx.x < nblocks ? partials[threadIdx.x * kVals + k] : 0.0;
    block_reduce(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kVals; k++) out[k] = v[k];
}

template <int TA, int TB>
cudaError_t launch(const void *a, const void *b, long long n, double *out, double *ws,
                   cudaStream_t st)
{
    long long blocks = (n + 4LL * kThreads - 1) / (4LL * kThreads);
    if (blocks > kBlocks) blocks = kBlocks;
    if (blocks < 1) blocks = 1;
    const long long chunk = (n + blocks - 1) / blocks;
    k_reduce_partial<TA, TB><<<(int)blocks, kThreads, 0, st>>>(a, b, n, chunk, ws);
    k_reduce_final<<<1, kBlocks, 0, st>>>(ws, (int)blocks, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t stencil_reduce_workspace_bytes(void) { return (size_t)kBlocks * kVals * sizeof(double); }

int stencil_reduce(const void *a, int a_type, const void *b, int b_type, long long n,
                   double *out, void *workspace, void *stream)
{
    if (!a || !out || !workspace || n < 1) return ST_ERR_INVALID_ARG;
    if (a_type != ST_F32 && a_type != ST_F64) return ST_ERR_INVALID_ARG;
    if (b && b_type != ST_F32 && b_type != ST_F64) return ST_ERR_INVALID_ARG;
    if ((uintptr_t)workspace % 8 || (uintptr_t)out % 8) return ST_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *ws = static_cast<double *>(workspace);
    cudaError_t e;
    if (!b) e = a_type == ST_F32 ? launch<ST_F32, -1>(a, b, n, out, ws, st)
                                 : launch<ST_F64, -1>(a, b, n, out, ws, st);
    else if (a_type == ST_F32)
        e = b_type == ST_F32 ? launch<ST_F32, ST_F32>(a, b, n, out, ws, st)
                             : launch<ST_F32, ST_F64>(a, b, n, out, ws, st);
    else
        e = b_type == ST_F32 ? launch<ST_F64, ST_F32>(a, b, n, out, ws, st)
                             : launch<ST_F64, ST_F64>(a, b, n, out, ws, st);
    return e == cudaSuccess ? ST_OK : ST_ERR_CUDA;
}

}  // extern "C"
