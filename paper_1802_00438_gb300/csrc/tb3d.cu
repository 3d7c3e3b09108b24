// Dispatch over the compiled 3D kernel instances.
#include "tb3d_table.cuh"

namespace stn {

static const Tb3dEntry *find_in(const Tb3dEntry *t, int n, const Shape3D &s)
{
    for (int i = 0; i < n; i++) {
        const Tb3dEntry &e = t[i];
        if (e.kind == s.kind && e.exact == s.exact && e.T == s.T && e.VY == s.VY &&
            e.NW == s.NW && e.alg == s.alg)
            return &e;
    }
    return nullptr;
}

static const Tb3dEntry *tb3d_find(const Shape3D &s)
{
    if (s.alg == 0) return find_in(tb3d_table, tb3d_table_n, s);
    return s.kind == 0 ? find_in(tb3f_table_diff, tb3f_table_diff_n, s)
                       : find_in(tb3f_table_therm, tb3f_table_therm_n, s);
}

bool tb3d_available(const Shape3D &s) { return tb3d_find(s) != nullptr; }

int tb3d_block_threads(const Shape3D &s)
{
    const Tb3dEntry *e = tb3d_find(s);
    return e ? 32 * e->NW : 0;
}

int tb3d_halo(const Shape3D &s) { return s.T; }

size_t tb3d_smem_bytes(const Shape3D &s)
{
    const Tb3dEntry *e = tb3d_find(s);
    return e ? e->smem : 0;
}

cudaError_t tb3d_prepare(const Shape3D &s, int *blocks_per_sm)
{
    const Tb3dEntry *e = tb3d_find(s);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)e->smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, 32 * e->NW,
                                                         e->smem);
}

cudaError_t tb3d_launch(const Shape3D &s, const Pass3D &p, cudaStream_t st)
{
    const Tb3dEntry *e = tb3d_find(s);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<Pass3D *>(&p)};
    return cudaLaunchKernel(e->fn, dim3(p.ctas), dim3(32 * e->NW), args, e->smem, st);
}

}  // namespace stn
