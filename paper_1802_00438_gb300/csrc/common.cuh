// Device helpers shared by the stencil kernels: the Table 2 cell updates and the async-copy
// staging primitives.  sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace stn {

// stencil kinds: Table 2's diffusion and Hotspot, and diffusion whose five coefficients are
// per-cell arrays (Table 2 row 1 with Sec. 5.1's array arguments)
enum { KDIFF = 0, KTHERM = 1, KVDIFF = 2 };

// ---------------------------------------------------------------------------------------
// Cell updates (arXiv 1802.00438, Table 2).  EXACT = true evaluates the printed expression
// left to right with one rounding per operation (the __f*_rn intrinsics are never fused);
// EXACT = false contracts the same expression into fused multiply-adds, ordered so that the
// term of the neighbour the streaming kernels receive last (s in 2D, a in 3D: the row or
// plane the previous stage has just produced) enters last.  Everything else of the update
// is then ready before that neighbour arrives, and a fused stage adds only two dependent
// operations to the chain between consecutive stages.
// Neighbours: w = x-1, e = x+1, n = y-1, s = y+1, b = z-1, a = z+1.
// ---------------------------------------------------------------------------------------

// Diffusion 2D: cc*c + cw*w + ce*e + cs*s + cn*n
template <bool EXACT>
__device__ __forceinline__ float diff5(float c, float w, float e, float s, float n, float cc,
                                       float cw, float ce, float cs, float cn)
{
    if (EXACT) {
        float r = __fmul_rn(cc, c);
        r = __fadd_rn(r, __fmul_rn(cw, w));
        r = __fadd_rn(r, __fmul_rn(ce, e));
        r = __fadd_rn(r, __fmul_rn(cs, s));
        return __fadd_rn(r, __fmul_rn(cn, n));
    } else {
        float r = __fmul_rn(cc, c);
        r = __fmaf_rn(cw, w, r);
        r = __fmaf_rn(ce, e, r);
        r = __fmaf_rn(cn, n, r);
        return __fmaf_rn(cs, s, r);
    }
}

// Diffusion 3D: ... + cb*b + ca*a
template <bool EXACT>
__device__ __forceinline__ float diff7(float c, float w, float e, float s, float n, float b,
                                       float a, const float *k)
{
    if (EXACT) {
        float r = __fmul_rn(k[0], c);
        r = __fadd_rn(r, __fmul_rn(k[1], w));
        r = __fadd_rn(r, __fmul_rn(k[2], e));
        r = __fadd_rn(r, __fmul_rn(k[3], s));
        r = __fadd_rn(r, __fmul_rn(k[4], n));
        r = __fadd_rn(r, __fmul_rn(k[5], b));
        return __fadd_rn(r, __fmul_rn(k[6], a));
    } else {
        float r = __fmul_rn(k[0], c);
        r = __fmaf_rn(k[1], w, r);
        r = __fmaf_rn(k[2], e, r);
        r = __fmaf_rn(k[3], s, r);
        r = __fmaf_rn(k[4], n, r);
        r = __fmaf_rn(k[5], b, r);
        return __fmaf_rn(k[6], a, r);
    }
}

// Hotspot 2D: c + sdc*(p + (n+s-2c)*Ry + (e+w-2c)*Rx + (amb-c)*Rz).
// 2c is exact in binary floating point, so computing it once for both brackets changes no
// rounding; in the contracted form (n+s) - 2c is one fused multiply-add with the same single
// rounding as the subtraction.
template <bool EXACT>
__device__ __forceinline__ float hot2(float c, float w, float e, float s, float n, float p,
                                      float sdc, float rx, float ry, float rz, float amb)
{
    if (EXACT) {
        float c2 = __fmul_rn(2.0f, c);
        float t1 = __fsub_rn(__fadd_rn(n, s), c2);
        float t2 = __fsub_rn(__fadd_rn(e, w), c2);
        float t3 = __fsub_rn(amb, c);
        float q = __fadd_rn(p, __fmul_rn(t1, ry));
        q = __fadd_rn(q, __fmul_rn(t2, rx));
        q = __fadd_rn(q, __fmul_rn(t3, rz));
        return __fadd_rn(c, __fmul_rn(sdc, q));
    } else {
        // (n + s - 2c) Ry split as (n - 2c) Ry + s Ry so that s enters last
        float t2 = __fmaf_rn(-2.0f, c, __fadd_rn(e, w));
        float t3 = __fsub_rn(amb, c);
        float n2 = __fmaf_rn(-2.0f, c, n);
        float q = __fmaf_rn(t2, rx, p);
        q = __fmaf_rn(t3, rz, q);
        q = __fmaf_rn(n2, ry, q);
        q = __fmaf_rn(s, ry, q);
        return __fmaf_rn(sdc, q, c);
    }
}

// Hotspot 3D: c*cc + n*cn + s*cs + e*ce + w*cw + a*ca + b*cb + sdc*p + ca*amb.
// ca_amb = ca*amb is the same rounded product for every cell and is hoisted by the caller.
template <bool EXACT>
__device__ __forceinline__ float hot3(float c, float w, float e, float s, float n, float b,
                                      float a, float p, const float *k, float ca_amb)
{
    if (EXACT) {
        float r = __fmul_rn(c, k[0]);
        r = __fadd_rn(r, __fmul_rn(n, k[4]));
        r = __fadd_rn(r, __fmul_rn(s, k[3]));
        r = __fadd_rn(r, __fmul_rn(e, k[2]));
        r = __fadd_rn(r, __fmul_rn(w, k[1]));
        r = __fadd_rn(r, __fmul_rn(a, k[6]));
        r = __fadd_rn(r, __fmul_rn(b, k[5]));
        r = __fadd_rn(r, __fmul_rn(k[7], p));
        return __fadd_rn(r, ca_amb);
    } else {
        float r = __fmaf_rn(k[7], p, ca_amb);
        r = __fmaf_rn(c, k[0], r);
        r = __fmaf_rn(n, k[4], r);
        r = __fmaf_rn(s, k[3], r);
        r = __fmaf_rn(e, k[2], r);
        r = __fmaf_rn(w, k[1], r);
        r = __fmaf_rn(b, k[5], r);
        return __fmaf_rn(a, k[6], r);
    }
}

// ---------------------------------------------------------------------------------------
// Async global -> shared staging (cp.async).  `src_bytes` < copy size zero-fills the rest,
// so out-of-domain cells arrive as zeros without a branch in the copy.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace stn
