// Compiled instances of the 3D star diffusion (radius R = 2 with T in {1, 2}; R = 3, 4 with
// T = 1 -- deeper fusion does not fit the shared-memory plane rings) and their dispatch.
#include "star3d.cuh"

namespace stn {
namespace {

struct Star3Entry {
    int R, exact, T;
    const void *fn;
    size_t smem;
    int hx, hy, cx, cy;
};

#define STN_STAR3(R_, E, T_)                                                                 \
    { R_, E, T_, reinterpret_cast<const void *>(&k_star3d<(E != 0), R_, T_>),              \
      STAR3<R_, T_>::SMEM, STAR3<R_, T_>::HX, STAR3<R_, T_>::HY, STAR3<R_, T_>::CX,          \
      STAR3<R_, T_>::CY }

const Star3Entry kStar3[] = {
    STN_STAR3(2, 0, 1), STN_STAR3(2, 0, 2), STN_STAR3(3, 0, 1), STN_STAR3(4, 0, 1),
    STN_STAR3(2, 1, 1), STN_STAR3(2, 1, 2), STN_STAR3(3, 1, 1), STN_STAR3(4, 1, 1),
};

const Star3Entry *find(int R, int exact, int T)
{
    for (const Star3Entry &e : kStar3)
        if (e.R == R && e.exact == (exact ? 1 : 0) && e.T == T) return &e;
    return nullptr;
}

}  // namespace

bool star3d_available(int R, int exact, int T) { return find(R, exact, T) != nullptr; }

void star3d_tile(int R, int T, int *cx, int *cy)
{
    const Star3Entry *e = find(R, 0, T);
    *cx = e ? e->cx : 0;
    *cy = e ? e->cy : 0;
}

cudaError_t star3d_prepare(int R, int exact, int T, int *blocks_per_sm)
{
    const Star3Entry *e = find(R, exact, T);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)e->smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, S3NT, e->smem);
}

cudaError_t star3d_launch(int R, int exact, int T, const PassStar3D &p, const CUtensorMap &tin,
                          cudaStream_t st)
{
    const Star3Entry *e = find(R, exact, T);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<PassStar3D *>(&p), const_cast<CUtensorMap *>(&tin)};
    const long long blocks = (long long)p.ntx * p.nty * p.nseg;
    return cudaLaunchKernel(e->fn, dim3((unsigned)blocks), dim3(S3NT), args, e->smem, st);
}

}  // namespace stn
