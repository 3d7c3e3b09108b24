// Compiled instances of the batched (many-grid) 2D contracted sweep and their dispatch:
// (T, V) in {(4, 4), (8, 4), (4, 8), (8, 8)} for Diffusion 2D and Hotspot 2D.
#include "tb2f_kernel.cuh"

namespace stn {
namespace {

struct BatchEntry {
    int kind, T, V;
    const void *fn;
    size_t smem;
};

#define STN_TB2FB_ENTRY(K, T_, V_)                                                           \
    { K, T_, V_, reinterpret_cast<const void *>(&k_tb2f_batch<K, T_, V_, true>),           \
      TB2F<K, T_, V_, ((K) == 1 ? STOR_SRC : 0)>::SMEM }

const BatchEntry kBatch[] = {
    STN_TB2FB_ENTRY(0, 4, 4), STN_TB2FB_ENTRY(0, 8, 4), STN_TB2FB_ENTRY(0, 4, 8), STN_TB2FB_ENTRY(0, 8, 8),
    STN_TB2FB_ENTRY(1, 4, 4), STN_TB2FB_ENTRY(1, 8, 4), STN_TB2FB_ENTRY(1, 4, 8), STN_TB2FB_ENTRY(1, 8, 8),
};

const BatchEntry *find(const Shape2D &s)
{
    if (s.exact || s.stor || s.W != 1) return nullptr;
    for (const BatchEntry &e : kBatch)
        if (e.kind == s.kind && e.T == s.T && e.V == s.V) return &e;
    return nullptr;
}

}  // namespace

bool tb2d_batch_available(const Shape2D &s) { return find(s) != nullptr; }

cudaError_t tb2d_batch_prepare(const Shape2D &s, int *blocks_per_sm)
{
    const BatchEntry *e = find(s);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)e->smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, 32, e->smem);
}

cudaError_t tb2d_batch_launch(const Shape2D &s, const BatchPass2D &bp, cudaStream_t st)
{
    const BatchEntry *e = find(s);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<BatchPass2D *>(&bp)};
    return cudaLaunchKernel(e->fn, dim3(bp.ctas), dim3(32), args, e->smem, st);
}

}  // namespace stn
