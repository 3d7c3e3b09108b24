// Dispatch over the compiled 2D kernel instances.
#include "tb2d_table.cuh"

namespace stn {

static const Tb2dEntry *tb2d_find(const Shape2D &s)
{
    const Tb2dEntry *tabs[3] = {tb2d_table_diff, tb2d_table_therm, tb2d_table_vdiff};
    const int ns[3] = {tb2d_table_diff_n, tb2d_table_therm_n, tb2d_table_vdiff_n};
    if (s.kind < 0 || s.kind > 2) return nullptr;
    const Tb2dEntry *t = tabs[s.kind];
    for (int i = 0; i < ns[s.kind]; i++)
        if (t[i].exact == s.exact && t[i].T == s.T && t[i].V == s.V && t[i].W == s.W &&
            t[i].stor == s.stor)
            return &t[i];
    return nullptr;
}

bool tb2d_available(const Shape2D &s) { return tb2d_find(s) != nullptr; }
int tb2d_block_threads(const Shape2D &s) { return 32 * (s.W > 0 ? s.W : 1); }   // W <= 0: one warp
int tb2d_tile_width(const Shape2D &s) { return 32 * s.V * (s.W > 0 ? s.W : 1); }
int tb2d_halo(const Shape2D &s) { return (s.T + 3) / 4 * 4; }

size_t tb2d_smem_bytes(const Shape2D &s)
{
    const Tb2dEntry *e = tb2d_find(s);
    return e ? e->smem : 0;
}

cudaError_t tb2d_prepare(const Shape2D &s, int *blocks_per_sm)
{
    const Tb2dEntry *e = tb2d_find(s);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)e->smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, tb2d_block_threads(s),
                                                         e->smem);
}

cudaError_t tb2d_launch(const Shape2D &s, const Pass2D &p, cudaStream_t st)
{
    const Tb2dEntry *e = tb2d_find(s);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<Pass2D *>(&p)};
    return cudaLaunchKernel(e->fn, dim3(p.ctas), dim3(tb2d_block_threads(s)), args, e->smem, st);
}

}  // namespace stn
