// Compiled instances of the 2D star diffusion (radius R in {2, 3, 4}, fused steps T in
// {1, 2, 4}, exact and contracted) and their dispatch.
#include <algorithm>

#include "star2d.cuh"

namespace stn {
namespace {

struct StarEntry {
    int R, exact, T;
    const void *fn;
    size_t smem;
    int hx, hy;
};

#define STN_STAR(R_, E, T_)                                                                  \
    { R_, E, T_, reinterpret_cast<const void *>(&k_star2d<(E != 0), R_, T_>),              \
      STAR<R_, T_>::SMEM, STAR<R_, T_>::HX, STAR<R_, T_>::HY }
#define STN_STAR_T(R_, E) STN_STAR(R_, E, 1), STN_STAR(R_, E, 2), STN_STAR(R_, E, 4)

const StarEntry kStar[] = {
    STN_STAR_T(2, 0), STN_STAR_T(3, 0), STN_STAR_T(4, 0),
    STN_STAR_T(2, 1), STN_STAR_T(3, 1), STN_STAR_T(4, 1),
};

const StarEntry *find(int R, int exact, int T)
{
    for (const StarEntry &e : kStar)
        if (e.R == R && e.exact == (exact ? 1 : 0) && e.T == T) return &e;
    return nullptr;
}

}  // namespace

bool star2d_available(int R, int exact, int T) { return find(R, exact, T) != nullptr; }

int star2d_halo_x(int R, int T)
{
    const StarEntry *e = find(R, 0, T);
    return e ? e->hx : 0;
}

int star2d_halo_y(int R, int T)
{
    const StarEntry *e = find(R, 0, T);
    return e ? e->hy : 0;
}

cudaError_t star2d_prepare(int R, int exact, int T)
{
    const StarEntry *e = find(R, exact, T);
    if (!e) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem);
}

cudaError_t star2d_launch(int R, int exact, int T, const PassStar2D &p, const CUtensorMap &tin,
                          cudaStream_t st)
{
    const StarEntry *e = find(R, exact, T);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<PassStar2D *>(&p), const_cast<CUtensorMap *>(&tin)};
    // persistent blocks, one per SM (three tile buffers fill its shared memory)
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    const long long tiles = (long long)p.ntx * p.nty;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, sms));
    return cudaLaunchKernel(e->fn, dim3(grid), dim3(32 * SNW), args,
                            e->smem, st);
}

}  // namespace stn
