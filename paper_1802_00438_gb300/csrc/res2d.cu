// Resident tiles: a 2D grid small enough to stay on chip, advanced by ONE cooperative launch.
//
// The overlapped tiles of Sec. 3.1-3.2 (halos of width rad*T, T steps fused, redundant halo
// computation, only the compute block kept), except that the tiles never leave the SMs: each
// block holds its tile (compute block plus halos) in registers for the whole run.  After every
// T steps (an epoch) it publishes the cells of its compute block that its neighbours' halos
// cover and reloads its halos from its neighbours' cells of the same epoch (bounded waits).  A run therefore reads the grid once and writes it once, and an epoch costs one
// exchange through L2 instead of a pass over device memory; for grids that fit (up to a few
// million cells over the SMs) the run is bound by the SMs' issue rate, not by HBM.
//
// Geometry: block b = (bx, by) of nbx x nby owns [bx*cw, min(nx, (bx+1)*cw)) x
// [by*ch, min(ny, (by+1)*ch)); its tile is the (32*VX) x (NW*VY) window starting at
// (bx*cw - hx, by*ch - hy), hx = T rounded up to a multiple of VX, hy = T, cw = 32*VX - 2*hx.
// Lane L of warp w holds cells x0 + L*VX + [0, VX) of rows y0 + w*VY + [0, VY).  x-neighbours
// across lanes come by shuffle, y-neighbours across warps through shared memory (one barrier
// per step).
//
// Clamped edges (Sec. 5.1: an out-of-range neighbour is the boundary cell): tile origins are
// multiples of VX, so x = 0 is always cell 0 of a lane, whose west input is replaced by the
// cell itself; x = nx-1 as the last cell of a lane has its east input replaced the same way,
// elsewhere in a lane the ghost cell x = nx next to it is set equal to it after every step; the
// rows y = -1 and y = ny are ghost rows kept equal to the edge rows the same way (or the edge
// row's shared-memory input is replaced when it is a warp's first or last row).  Cells further
// outside the grid hold values that never reach a cell inside it.
//
// Exchange: two grid-sized buffers alternate by epoch parity.  A block overwrites its cells of
// epoch e (with epoch e+2) only after its neighbours have published epoch e+1, which they do
// only after reading epoch e.  flags[b] counts the epochs block b has published (growing
// across runs from the plan's epoch0, so no reset between runs): after the block's barrier
// one thread publishes it with a release store, and a waiting block polls its (up to 8)
// neighbours' counters with acquire loads before its barrier and its reads -- no further
// fences (measured on GB300: an exchange with a gpu-scope fence on either side took ~5 us,
// with release/acquire alone ~2.7 us).  Every wait is bounded: after wait_ns the waiting block
// sets the status word and leaves, and every other block leaves at its next wait, so a lost
// update cannot hang the GPU.  All blocks must be resident at once, hence the cooperative
// launch (which fails rather than starting a grid larger than the device can hold).
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace stn {
namespace {

constexpr int kResVY = 8;   // rows per thread

// Threads per block each instance is compiled for (its register budget: 65536 / threads), from
// the registers each needs without spilling (-Xptxas -v): 64 (Diffusion, 2 cells per row), 108
// (Diffusion, 4), 80 (Hotspot, 2), 128 and 188 (Hotspot, 4, contracted and exact).
constexpr int res_max_threads(int kind, int vx, bool exact)
{
    return kind == KDIFF ? (vx == 2 ? 1024 : 512) : (vx == 2 ? 768 : (exact ? 320 : 512));
}

__device__ __forceinline__ long long rs_timer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ int rs_ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int rs_ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void rs_st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// One cell of Table 2.  Diffusion: k = [cc, cw, ce, cs, cn].  Hotspot, exact: k = [sdc, Rx,
// Ry, Rz, amb] and q the power; contracted: k = [cc, cx, cy, cz] (the expanded weights of the
// streaming kernels, cc + 2cx + 2cy = 1 exactly) and q the source map sdc*(p + amb*Rz), the
// operations in the streaming kernels' first stage order.
template <int KIND, bool EXACT>
__device__ __forceinline__ float rcell(float c, float w, float e, float s, float n, float q,
                                       const float (&k)[5])
{
    if (KIND == KDIFF) return diff5<EXACT>(c, w, e, s, n, k[0], k[1], k[2], k[3], k[4]);
    if (EXACT) return hot2<true>(c, w, e, s, n, q, k[0], k[1], k[2], k[3], k[4]);
    float r = __fmaf_rn(k[1], __fadd_rn(e, w), q);
    r = __fmaf_rn(k[2], __fadd_rn(n, s), r);
    r = __fmaf_rn(k[0], c, r);
    return __fmaf_rn(-k[3], c, r);
}

template <int VX>
__device__ __forceinline__ void st_row(float *p, const float (&v)[VX])
{
    if (VX == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if (VX == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else
#pragma unroll
        for (int j = 0; j < VX; j++) p[j] = v[j];
}

template <int VX>
__device__ __forceinline__ void ld_row(const float *p, float (&v)[VX])
{
    if (VX == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if (VX == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int j = 0; j < VX; j++) v[j] = p[j];
    }
}

// Per-thread roles at the clamped edges (all fixed for the run).
struct Edges {
    bool wsel;   // x = 0 is my cell 0: its west input is itself
    bool esel;   // x = nx-1 is my cell VX-1: its east input is itself
    int efix;    // x = nx-1 is my cell efix < VX-1: ghost cell efix+1 copies it after each step
    int k0, k1;  // rows of y = 0 and y = ny-1 among my VY rows (outside [0, VY): none)
};

// Clamp work of a block at the x edges, one bit each, so that a block compiles and runs only
// what its own edges need (measured: with one edge path for both edges and the ghost-column
// fix-up, the x-edge blocks took ~15 % more cycles per step than the others, and every block
// waits for its neighbours at each exchange).
enum : int {
    XW = 1,   // x = 0 in the block: its west input is itself
    XS = 2,   // x = nx-1 is a lane's last cell: its east input is itself
    XF = 4,   // x = nx-1 inside a lane: the ghost cell after it copies it after each step
};

// One Jacobi step of the thread's VX x VY cells, in place.  xs: the block's row-exchange
// buffers [2][NW][2][32*VX] (parity, warp, top/bottom row); XM: the block's clamp work at the
// x edges (XW | XS | XF).
template <int KIND, int VX, int VY, bool EXACT, int XM>
__device__ __forceinline__ void rstep(float (&u)[VY][VX], const float (&q)[VY][VX],
                                      const float (&k)[5], float *xs, int &par, int nw, int w,
                                      int lane, const Edges &g)
{
    constexpr int RW = 32 * VX;
    float *mine = xs + ((par * nw + w) * 2) * RW + lane * VX;
    st_row<VX>(mine, u[0]);
    st_row<VX>(mine + RW, u[VY - 1]);
    __syncthreads();
    float nin[VX], sin[VX];
    if (w > 0) ld_row<VX>(mine - RW, nin);            // bottom row of the warp above
    else
#pragma unroll
        for (int j = 0; j < VX; j++) nin[j] = u[0][j];
    if (w < nw - 1) ld_row<VX>(mine + 2 * RW, sin);   // top row of the warp below
    else
#pragma unroll
        for (int j = 0; j < VX; j++) sin[j] = u[VY - 1][j];
    par ^= 1;
    if (g.k0 == 0)
#pragma unroll
        for (int j = 0; j < VX; j++) nin[j] = u[0][j];
    if (g.k1 == VY - 1)
#pragma unroll
        for (int j = 0; j < VX; j++) sin[j] = u[VY - 1][j];

    float prev[VX];
#pragma unroll
    for (int j = 0; j < VX; j++) prev[j] = nin[j];
#pragma unroll
    for (int r = 0; r < VY; r++) {
        float c[VX];
#pragma unroll
        for (int j = 0; j < VX; j++) c[j] = u[r][j];
        float win = __shfl_up_sync(0xffffffffu, c[VX - 1], 1);
        float ein = __shfl_down_sync(0xffffffffu, c[0], 1);
        if (XM & XW) win = g.wsel ? c[0] : win;
        if (XM & XS) ein = g.esel ? c[VX - 1] : ein;
#pragma unroll
        for (int j = 0; j < VX; j++) {
            const float wv = j > 0 ? c[j - 1] : win;
            const float ev = j < VX - 1 ? c[j + 1] : ein;
            const float sv = r < VY - 1 ? u[r + 1][j] : sin[j];
            u[r][j] = rcell<KIND, EXACT>(c[j], wv, ev, sv, prev[j], q[r][j], k);
        }
#pragma unroll
        for (int j = 0; j < VX; j++) prev[j] = c[j];
    }
    // ghost rows and columns follow the edge cells (warp-uniform rows; one lane for columns)
    if (g.k0 >= 1 && g.k0 < VY) {
#pragma unroll
        for (int r = 1; r < VY; r++)
            if (g.k0 == r)
#pragma unroll
                for (int j = 0; j < VX; j++) u[r - 1][j] = u[r][j];
    }
    if (g.k1 >= 0 && g.k1 < VY - 1) {
#pragma unroll
        for (int r = 0; r < VY - 1; r++)
            if (g.k1 == r)
#pragma unroll
                for (int j = 0; j < VX; j++) u[r + 1][j] = u[r][j];
    }
    if ((XM & XF) && g.efix >= 0) {
#pragma unroll
        for (int j = 0; j < VX - 1; j++)
            if (g.efix == j)
#pragma unroll
                for (int r = 0; r < VY; r++) u[r][j + 1] = u[r][j];
    }
}

template <int KIND, int VX, bool EXACT>
__global__ void __launch_bounds__(res_max_threads(KIND, VX, EXACT)) k_res2d(const Res2D p)
{
    constexpr int VY = kResVY;
    constexpr bool AUX = KIND == KTHERM;
    extern __shared__ __align__(16) float xs[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    const int bx = blockIdx.x % p.nbx, by = blockIdx.x / p.nbx;
    const int gx0 = bx * p.cw - p.hx + lane * VX;   // my first column
    const int gy0 = by * p.ch - p.hy + w * VY;      // my first row
    const int cx0 = bx * p.cw, cx1 = min(cx0 + p.cw, p.nx);
    const int cy0 = by * p.ch, cy1 = min(cy0 + p.ch, p.ny);
    float k[5];
#pragma unroll
    for (int i = 0; i < 5; i++) k[i] = p.k[i];

    // my cells in the compute block (kept; written out at the end), those of them a
    // neighbour's halo covers (published every epoch), and my halo cells (reloaded every
    // epoch; rows that round the tile up to whole warps lie beyond the halo and are neither:
    // they reach no compute cell within an epoch)
    unsigned own = 0, pub = 0, rld = 0;
#pragma unroll
    for (int r = 0; r < VY; r++)
#pragma unroll
        for (int j = 0; j < VX; j++) {
            const int x = gx0 + j, y = gy0 + r;
            const bool in = x >= cx0 && x < cx1 && y >= cy0 && y < cy1;
            const bool b = in && (x < cx0 + p.hx || x >= cx1 - p.hx || y < cy0 + p.hy || y >= cy1 - p.hy);
            const bool h = !in && x >= cx0 - p.hx && x < cx1 + p.hx && y >= cy0 - p.hy && y < cy1 + p.hy;
            own |= (in ? 1u : 0u) << (r * VX + j);
            pub |= (b ? 1u : 0u) << (r * VX + j);
            rld |= (h ? 1u : 0u) << (r * VX + j);
        }
    Edges g;
    g.wsel = gx0 == 0;
    const int r1 = p.nx - 1 - gx0;
    g.esel = r1 == VX - 1;
    g.efix = (r1 >= 0 && r1 < VX - 1) ? r1 : -1;
    g.k0 = -gy0;
    g.k1 = p.ny - 1 - gy0;
    const int xm = (__syncthreads_or(g.wsel) ? XW : 0) | (__syncthreads_or(g.esel) ? XS : 0) |
                   (__syncthreads_or(g.efix >= 0) ? XF : 0);

    // the tile at time 0 (coordinates clamped: ghost cells start equal to the edge cells)
    float u[VY][VX], q[VY][VX];
#pragma unroll
    for (int r = 0; r < VY; r++) {
        const int yc = min(max(gy0 + r, 0), p.ny - 1);
#pragma unroll
        for (int j = 0; j < VX; j++) {
            const int xc = min(max(gx0 + j, 0), p.nx - 1);
            u[r][j] = __ldg(p.in + (long long)yc * p.ld_in + xc);
            float v = AUX ? __ldg(p.aux + (long long)yc * p.ld_aux + xc) : 0.f;
            // contracted Hotspot: the source map, each operation rounded once (as the streaming
            // plans build it)
            if (AUX && !EXACT) v = __fmul_rn(p.src_sdc, __fadd_rn(v, p.src_a));
            q[r][j] = v;
        }
    }

    int par = 0;
    const int E = (p.steps + p.T - 1) / p.T;
    for (int e = 0; e < E; e++) {
        const int ts = (e == E - 1) ? p.steps - p.T * (E - 1) : p.T;
        // unrolled so that the rows updated in place need no register moves at the loop edge
        // (measured: 4 steps per iteration +7-9 % over 1)
        // interior blocks and blocks on one x edge (x = nx-1 on a lane's last cell), unrolled;
        // the rest (x = nx-1 inside a lane, a grid one block wide) in one general loop
        // (measured: more unrolled variants slowed the interior blocks' loop by ~2 %)
        if (xm == 0) {
#pragma unroll 4
            for (int t = 0; t < ts; t++) rstep<KIND, VX, VY, EXACT, 0>(u, q, k, xs, par, nw, w, lane, g);
        } else if (xm == XW) {
#pragma unroll 4
            for (int t = 0; t < ts; t++) rstep<KIND, VX, VY, EXACT, XW>(u, q, k, xs, par, nw, w, lane, g);
        } else if (xm == XS) {
#pragma unroll 4
            for (int t = 0; t < ts; t++) rstep<KIND, VX, VY, EXACT, XS>(u, q, k, xs, par, nw, w, lane, g);
        } else {
#pragma unroll 1
            for (int t = 0; t < ts; t++)
                rstep<KIND, VX, VY, EXACT, XW | XS | XF>(u, q, k, xs, par, nw, w, lane, g);
        }
        if (e == E - 1) break;

        // publish my border cells of time (e+1)*T.  The coordinates pass through an empty asm
        // so that the compiler recomputes the addresses here instead of keeping 2 * VX * VY of
        // them live across the steps.
        float *X = p.xg + (long long)(e & 1) * p.xplane;
        int ox = gx0, oy = gy0;
        unsigned pb = pub, rl = rld;
        asm volatile("" : "+r"(ox), "+r"(oy), "+r"(pb), "+r"(rl));
        constexpr unsigned ALL = (1u << VX) - 1u;
#pragma unroll
        for (int r = 0; r < VY; r++) {
            float *row = X + (long long)(oy + r) * p.ld_x + ox;
            const unsigned bits = (pb >> (r * VX)) & ALL;
            if (bits == ALL) {   // the lane's cells of this row whole: one aligned vector store
                st_row<VX>(row, u[r]);
            } else if (bits) {
#pragma unroll
                for (int j = 0; j < VX; j++)
                    if ((bits >> j) & 1u) row[j] = u[r][j];
            }
        }
        // the block's stores, then one release store of its counter (cumulative over the
        // stores the barrier ordered before it); counters only grow, across runs too
        const int want = p.epoch0 + e + 1;
        __syncthreads();
        if (tid == 0 && !(p.hold_block == (int)blockIdx.x && e >= p.hold_epoch))
            rs_st_release(p.flags + blockIdx.x, want);
        // threads 0..8 wait (acquire) for the 3 x 3 neighbourhood's counters
        bool failed = false;
        if (tid < 9) {
            const int nbx_ = bx + tid % 3 - 1, nby_ = by + tid / 3 - 1;
            if (tid != 4 && nbx_ >= 0 && nbx_ < p.nbx && nby_ >= 0 && nby_ < p.nby) {
                const int *f = p.flags + nby_ * p.nbx + nbx_;
                const long long deadline = rs_timer() + p.wait_ns;
                while (rs_ld_acquire(f) < want) {
                    if (rs_ld_relaxed(p.status) != 0) {
                        failed = true;
                        break;
                    }
                    if (rs_timer() > deadline) {
                        atomicCAS(p.status, 0, 1);
                        failed = true;
                        break;
                    }
                    __nanosleep(20);
                }
            }
        }
        if (__syncthreads_or(failed)) return;   // block-uniform; no copy in flight
        // reload the halos (clamped: ghost cells take the edge cells' new values), from L2
        asm volatile("" : "+r"(ox), "+r"(oy), "+r"(rl));
        const bool xin = ox >= 0 && ox + VX <= p.nx;   // my columns need no clamp
#pragma unroll
        for (int r = 0; r < VY; r++) {
            const int y = oy + r;
            const float *row = X + (long long)min(max(y, 0), p.ny - 1) * p.ld_x;
            const unsigned bits = (rl >> (r * VX)) & ALL;
            if (bits == ALL && xin && y >= 0 && y < p.ny) {   // one aligned vector load
                if (VX == 4) {
                    const float4 v = __ldcg(reinterpret_cast<const float4 *>(row + ox));
                    u[r][0] = v.x; u[r][1] = v.y; u[r][VX > 2 ? 2 : 0] = v.z; u[r][VX > 3 ? 3 : 0] = v.w;
                } else {
                    const float2 v = __ldcg(reinterpret_cast<const float2 *>(row + ox));
                    u[r][0] = v.x; u[r][1] = v.y;
                }
            } else if (bits) {
#pragma unroll
                for (int j = 0; j < VX; j++)
                    if ((bits >> j) & 1u) u[r][j] = __ldcg(row + min(max(ox + j, 0), p.nx - 1));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < VY; r++)
#pragma unroll
        for (int j = 0; j < VX; j++)
            if ((own >> (r * VX + j)) & 1u) p.out[(long long)(gy0 + r) * p.nx + gx0 + j] = u[r][j];
}

struct REntry {
    int kind, exact, vx;
    const void *fn;
};

#define STN_RES(K, VX, E) \
    { K, E, VX, reinterpret_cast<const void *>(&k_res2d<K, VX, (E) != 0>) }

const REntry kRes[] = {STN_RES(KDIFF, 4, 0), STN_RES(KDIFF, 4, 1), STN_RES(KDIFF, 2, 0),
                       STN_RES(KDIFF, 2, 1), STN_RES(KTHERM, 4, 0), STN_RES(KTHERM, 4, 1),
                       STN_RES(KTHERM, 2, 0), STN_RES(KTHERM, 2, 1)};

const REntry *rfind(int kind, int exact, int vx)
{
    for (const REntry &e : kRes)
        if (e.kind == kind && e.exact == (exact ? 1 : 0) && e.vx == vx) return &e;
    return nullptr;
}

}  // namespace

int res2d_rows_per_thread() { return kResVY; }

int res2d_max_warps(int kind, int exact, int vx) { return res_max_threads(kind, vx, exact != 0) / 32; }

size_t res2d_smem(int vx, int nw) { return (size_t)2 * nw * 2 * 32 * vx * sizeof(float); }

bool res2d_available(int kind, int exact, int vx) { return rfind(kind, exact, vx) != nullptr; }

cudaError_t res2d_occupancy(int kind, int exact, int vx, int nw, int *blocks_per_sm)
{
    const REntry *e = rfind(kind, exact, vx);
    if (!e || nw < 1 || nw > res2d_max_warps(kind, exact, vx)) return cudaErrorInvalidValue;
    const size_t sm = res2d_smem(vx, nw);
    cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)res2d_smem(vx, res2d_max_warps(kind, exact, vx)));
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, 32 * nw, sm);
}

cudaError_t res2d_launch(int kind, int exact, int vx, int nw, const Res2D &a, cudaStream_t st)
{
    const REntry *e = rfind(kind, exact, vx);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<Res2D *>(&a)};
    return cudaLaunchCooperativeKernel(e->fn, dim3(a.nbx * a.nby), dim3(32 * nw), args,
                                       res2d_smem(vx, nw), st);
}

}  // namespace stn
