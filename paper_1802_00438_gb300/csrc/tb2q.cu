// Many 2D grids in one persistent launch fed by a tile work queue.
//
// The temporally-blocked pass of the paper (Sec. 3.1-3.2: overlapped tiles with halos of width
// >= rad*T, T fused steps, redundant halo compute, only the compute block stored, the last pass
// fusing the remainder) is split into items of one tile column x L rows.  The items of every
// grid of a batch, all passes, sit in one queue in pass-major order (Eq. 8 gives each grid its
// own ceil(steps/T) passes); the blocks of ONE launch pop items one after another (one queue per
// stencil kind, each SM starting on one of them: see QueueBatch2D).  A pass of a
// grid depends on the previous pass of the same grid only where the tiles overlap, so an item
// waits, before it reads anything, for the neighbouring tiles' previous pass (tx +- 1, seg +- 1:
// the halo it reads and the cells it overwrites in the ping-pong buffer).
//
// Why no item can wait forever: items are popped in queue order and depend only on items
// earlier in the same queue, so the earliest unfinished item of each queue always has its
// dependencies finished and is held by a running block.  Every wait is bounded all the same (a lost update would otherwise
// hang the GPU): after QueueCtl::wait_ns a block sets the batch's status word and leaves, and
// every other block leaves at its next poll or pop.  Waits happen before an item issues any
// copy, so no block leaves with copies in flight.
//
// Ordering: every lane of the finishing warp fences its own stores (gpu scope), then lane 0
// publishes the tile's counter with a release store; every lane of a waiting warp observes the
// counter itself (relaxed loads) and fences before it reads (acquire).
#include "tb2f_kernel.cuh"

namespace stn {
namespace {

__device__ __forceinline__ long long gtimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// The whole warp waits until flags[y * row + x] >= need for x in [x0, x1], y in [y0, y1] (every
// lane polls the same flag: one broadcast load; decisions are lane 0's, so the warp stays
// converged).  Returns false when the batch's status is set (another block gave up) or when
// the deadline passes (this warp sets the status).  On success every lane has issued a
// gpu-scope fence after observing the flags (acquire).
__device__ bool q_wait(const int *flags, int row, int x0, int x1, int y0, int y1, int need,
                       int *status, long long deadline)
{
    const int lane = threadIdx.x & 31;
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
            const int *f = flags + (long long)y * row + x;
            unsigned ns = 32;
            while (__shfl_sync(0xffffffffu, ld_relaxed(f) < need ? 1 : 0, 0)) {
                int outcome = 0;   // 1: another block gave up, 2: our deadline passed
                if (lane == 0) {
                    if (ld_relaxed(status) != 0) outcome = 1;
                    else if (gtimer() > deadline) {
                        atomicCAS(status, 0, 1);
                        outcome = 2;
                    }
                }
                if (__shfl_sync(0xffffffffu, outcome, 0)) return false;
                __nanosleep(ns);
                ns = ns < 1024 ? 2 * ns : ns;
            }
        }
    __threadfence();
    return true;
}

template <int T, int V>
__global__ void __launch_bounds__(32) k_tb2f_queue(const QueueBatch2D q)
{
    using CD = TB2F<KDIFF, T, V, STOR_F32>;
    // partial rows updated in place (no two-row unroll; measured on the 64-grid workload:
    // 1980 against 1729 GCell/s with 192-row items)
    constexpr bool SW = false;
    extern __shared__ __align__(16) float smem[];
    float A[CD::NS][V], B[CD::NS][V];
#pragma unroll
    for (int s = 0; s < CD::NS; s++)
#pragma unroll
        for (int j = 0; j < V; j++) A[s][j] = B[s][j] = 0.f;
    const int lane = threadIdx.x;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;\n" : "=r"(smid));
    int qs = (int)smid < q.split ? 0 : 1;   // this SM's queue first, then the other one
    for (int tries = 0; tries < 2;) {
        int it = 0;
        if (lane == 0) it = ld_relaxed(q.status) ? q.total[qs] : (int)atomicAdd(q.head + qs, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= q.total[qs]) {
            if (ld_relaxed(q.status)) break;
            qs ^= 1;
            tries++;
            continue;
        }
        const QItem w = q.items[qs][it];
        // read from global memory where used: little stays live across the pass
        const QGrid &G = q.grids[w.g];
        bool ok = true;
        {
            const long long deadline =
                __shfl_sync(0xffffffffu, gtimer(), 0) + q.ctl->wait_ns;
            const int s0 = max(w.seg - 1, 0), s1 = min(w.seg + 1, G.nseg - 1);
            if (w.k == 0 && G.P > 0 && G.kind == KTHERM)
                ok = q_wait(q.srcf + G.srcf_off, G.ntx, max(w.tx - 1, 0), min(w.tx + 1, G.ntx - 1),
                            s0, s1, 1, q.status, deadline);
            else if (w.k > 0 && w.k < G.P)
                ok = q_wait(q.done + G.done_off, G.ntx, max(w.tx - 1, 0), min(w.tx + 1, G.ntx - 1),
                            s0, s1, w.k, q.status, deadline);
        }
        if (!ok) break;
        const int r0 = w.seg * q.L, r1 = min(G.ny, r0 + q.L);
        if (w.k < 0) {
            // source map of the tile's compute block: sdc*(p + amb*Rz), each operation rounded
            // once (the plans' k_hot_source); 16-byte accesses where the rows allow, the warp's
            // lanes spread over the block's rows and columns so many loads are in flight
            const float a = __fmul_rn(G.amb, G.rz), sdc = G.sdc;
            constexpr int CXQ = 32 * V - 2 * ((T + 3) / 4 * 4);
            const int x0 = w.tx * CXQ, x1 = min(G.nx, x0 + CXQ);
            const int nq = (x1 - x0 + 3) / 4;               // 4-cell chunks per row
            const bool vec = (G.nx % 4 == 0);   // the source rows are padded: aligned always
            for (int c = lane; c < nq * (r1 - r0); c += 32) {
                const int y = r0 + c / nq, x = x0 + 4 * (c % nq);
                const float *pr = G.power + (long long)y * G.nx + x;
                float *d = G.src + (long long)y * G.ld_src + x;
                if (vec) {
                    const float4 v = *reinterpret_cast<const float4 *>(pr);
                    *reinterpret_cast<float4 *>(d) =
                        make_float4(__fmul_rn(sdc, __fadd_rn(v.x, a)), __fmul_rn(sdc, __fadd_rn(v.y, a)),
                                    __fmul_rn(sdc, __fadd_rn(v.z, a)), __fmul_rn(sdc, __fadd_rn(v.w, a)));
                } else {
                    for (int j = 0; j < 4 && x + j < x1; j++) d[j] = __fmul_rn(sdc, __fadd_rn(pr[j], a));
                }
            }
        } else if (w.k < G.P) {
            const Pass2D &p = q.passes[G.pass_base + w.k];
            const long long lo = (long long)w.tx * G.ny + r0;
            const long long hi = lo + (r1 - r0);
            if (G.kind == KDIFF) tbf_range<KDIFF, T, V, SW, STOR_F32>(p, lo, hi, A, B, smem);
            else tbf_range<KTHERM, T, V, SW, STOR_SRC>(p, lo, hi, A, B, smem);
        } else {
            for (int y = r0; y < r1; y++) {
                const float *s = G.copy_from + (long long)y * G.ld_copy;
                float *d = G.copy_to + (long long)y * G.nx;
                for (int x = lane; x < G.nx; x += 32) d[x] = __ldcg(s + x);
            }
        }
        // every lane fences its own stores, then one lane publishes (release)
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            if (w.k < 0)
                st_release(q.srcf + G.srcf_off + (long long)w.seg * G.ntx + w.tx, 1);
            else if (w.k < G.P && w.k != q.ctl->hold_pass)
                st_release(q.done + G.done_off + (long long)w.seg * G.ntx + w.tx, w.k + 1);
        }
    }
}

struct QEntry {
    int T, V;
    const void *fn;
    size_t smem;
};

template <int T, int V>
constexpr size_t q_smem()
{
    return TB2F<KDIFF, T, V, STOR_F32>::SMEM > TB2F<KTHERM, T, V, STOR_SRC>::SMEM
               ? TB2F<KDIFF, T, V, STOR_F32>::SMEM
               : TB2F<KTHERM, T, V, STOR_SRC>::SMEM;
}

#define STN_TB2Q_ENTRY(T_, V_) \
    { T_, V_, reinterpret_cast<const void *>(&k_tb2f_queue<T_, V_>), q_smem<T_, V_>() }

const QEntry kQueue[] = {STN_TB2Q_ENTRY(8, 4)};

const QEntry *qfind(int T, int V)
{
    for (const QEntry &e : kQueue)
        if (e.T == T && e.V == V) return &e;
    return nullptr;
}

}  // namespace

bool tb2q_available(int T, int V) { return qfind(T, V) != nullptr; }

cudaError_t tb2q_prepare(int T, int V, int *blocks_per_sm)
{
    const QEntry *e = qfind(T, V);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)e->smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, 32, e->smem);
}

cudaError_t tb2q_launch(int T, int V, const QueueBatch2D &q, cudaStream_t st)
{
    const QEntry *e = qfind(T, V);
    if (!e) return cudaErrorInvalidValue;
    void *args[] = {const_cast<QueueBatch2D *>(&q)};
    return cudaLaunchKernel(e->fn, dim3(q.ctas), dim3(32), args, e->smem, st);
}

}  // namespace stn
