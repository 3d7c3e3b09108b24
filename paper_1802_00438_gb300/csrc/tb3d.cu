// Dispatch over the compiled 3D kernel instances.
#include <cstdint>

#include "tb3d_table.cuh"

namespace stn {

static const Tb3dEntry *find_in(const Tb3dEntry *t, int n, const Shape3D &s)
{
    for (int i = 0; i < n; i++) {
        const Tb3dEntry &e = t[i];
        if (e.kind == s.kind && e.exact == s.exact && e.T == s.T && e.VY == s.VY &&
            e.NW == s.NW && e.alg == s.alg && e.VX == s.VX)
            return &e;
    }
    return nullptr;
}

static const Tb3dEntry *tb3d_find(const Shape3D &s)
{
    if (s.alg == 0) return find_in(tb3d_table, tb3d_table_n, s);
    const Tb3dList lists[] = {{tb3f_table_diff_a, &tb3f_table_diff_a_n},
                              {tb3f_table_diff_b, &tb3f_table_diff_b_n},
                              {tb3f_table_therm_a, &tb3f_table_therm_a_n},
                              {tb3f_table_therm_b, &tb3f_table_therm_b_n}};
    for (const Tb3dList &l : lists)
        if (const Tb3dEntry *e = find_in(l.e, *l.n, s)) return e;
    return nullptr;
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

cudaError_t tb3d_launch(const Shape3D &s, const Pass3D &p, const Tma3D &t, cudaStream_t st)
{
    const Tb3dEntry *e = tb3d_find(s);
    if (!e) return cudaErrorInvalidValue;
    if (e->alg == 0) {
        void *args[] = {const_cast<Pass3D *>(&p)};
        return cudaLaunchKernel(e->fn, dim3(p.ctas), dim3(32 * e->NW), args, e->smem, st);
    }
    void *args[] = {const_cast<Pass3D *>(&p), const_cast<CUtensorMap *>(&t.in),
                    const_cast<CUtensorMap *>(&t.pw)};
    return cudaLaunchKernel(e->fn, dim3(p.ctas), dim3(32 * e->NW), args, e->smem, st);
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}
}  // namespace

bool tma3d_encode(CUtensorMap *m, const float *base, int nx, int ny, int nz, int bx, int by)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || !base || (uintptr_t)base % 16 != 0 || nx % 4 != 0) return false;
    const cuuint64_t dim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t stride[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    // out-of-bound cells of a box arrive as zeros (FLOAT_OOB_FILL_NONE)
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dim, stride, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace stn
