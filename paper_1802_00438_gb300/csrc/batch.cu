// Many 2D grids of uneven sizes and step counts advanced by ONE persistent kernel launch fed by a
// tile work queue, captured in a CUDA graph.
//
// Every grid runs ceil(steps/T) temporally-blocked passes like stencil_run (Eq. 8, Sec. 3.2: the
// last pass fuses the remainder) with its own ping-pong scratch; one (T, cells per thread) for
// the whole batch comes from the GPU restatement of the paper's model (Eqs. 3-9), the choice that
// minimises the predicted total time.  The passes are cut into items (one tile column x L rows),
// queued pass by pass on a levelled timeline with the Hotspot source-map rows first and the
// copies of grids with no steps last; the blocks of one launch (one warp each, as many as are
// resident) pop them and wait, bounded, for the neighbouring tiles of the previous pass
// (tb2q.cu).  The graph is: reset of the queue head, status and per-tile counters; the launch; a
// copy of the status word to host memory that stencil_batch_sync reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

using namespace stn;

namespace stn {
double batch_model_gcells(int kind, int nx, int ny, int steps, int sms, int T, int V, int bps,
                          int seg_rows);
}

struct stencil_batch_s {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    int qT = 0, qV = 0;
    std::vector<stencil_batch_grid> grid;
    std::vector<int> passes;
    std::vector<float *> scratch;     // two per grid: the passes between the first and the last
    std::vector<float *> src;         // Hotspot grids: the source map sdc*(p + amb*Rz)
    std::vector<long long> ld_scratch;
    void *dev = nullptr;              // items, grids, pass descriptors, counters, control
    QueueCtl *ctl = nullptr;          // inside dev
    int *h_status = nullptr;          // pinned: the status word after the last replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    long long items = 0;
};

namespace {

// rows per queue item (L), by default: each item streams 2T rows more than it stores, and
// fewer, longer items leave more blocks waiting for their neighbours (measured on the 64-grid
// workload, T = 8: 1921 / 1973 / 1980 / 1978 / 1961 GCell/s for L = 128 / 160 / 192 / 224 / 256)
constexpr int kRows = 192;
constexpr long long kWaitNs = 1000LL * 1000 * 1000;   // 1 s: a wait of a healthy batch is far shorter
// (T, V) of the compiled queue kernel: 4 cells per lane (with 8, the launch ran at half the
// rate on the 64-grid workload: 816 against 1713 GCell/s, one 255-register block per SMSP pair;
// T = 12 with 4 cells, 255 registers, 1763 against 1980 for T = 8)
const int kCand[][2] = {{8, 4}};

int status(cudaError_t e)
{
    if (e == cudaSuccess) return ST_OK;
    return e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

extern "C" {

int stencil_batch_create(stencil_batch *out, const stencil_batch_grid *grids, int count,
                         void *stream)
{
    return stencil_batch_create_ex(out, grids, count, stream, 0, 0, 0);
}

int stencil_batch_create_ex(stencil_batch *out, const stencil_batch_grid *grids, int count,
                            void *stream, int rows_per_item, int force_T, int force_vec)
{
    if (!out) return ST_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grids || count < 1 || rows_per_item < 0 || force_T < 0 || force_vec < 0)
        return ST_ERR_INVALID_ARG;
    const int L = rows_per_item ? rows_per_item : kRows;
    for (int g = 0; g < count; g++) {
        const stencil_batch_grid &q = grids[g];
        if ((q.kind != ST_DIFFUSION && q.kind != ST_THERMAL) || q.nx < 1 || q.ny < 1 ||
            q.steps < 0 || !q.grid_in || !q.grid_out)
            return ST_ERR_INVALID_ARG;
        if ((q.kind == ST_THERMAL) != (q.power != nullptr)) return ST_ERR_INVALID_ARG;
        const size_t bytes = (size_t)q.nx * q.ny * sizeof(float);
        const uintptr_t a = (uintptr_t)q.grid_in, b = (uintptr_t)q.grid_out;
        if (a != b && a < b + bytes && b < a + bytes) return ST_ERR_INVALID_ARG;
        if (q.power) {
            const uintptr_t p = (uintptr_t)q.power;
            if (p < b + bytes && b < p + bytes) return ST_ERR_INVALID_ARG;
        }
    }
    stencil_batch_s *B = new (std::nothrow) stencil_batch_s();
    if (!B) return ST_ERR_OOM;
    B->stream = static_cast<cudaStream_t>(stream);
    if (!B->stream) {
        // graphs cannot be captured on the legacy default stream: use an owned stream that
        // synchronises with it (cudaStreamCreate's default, blocking flag)
        cudaError_t se = cudaStreamCreate(&B->stream);
        if (se != cudaSuccess) {
            delete B;
            return status(se);
        }
        B->own_stream = true;
    }
    B->grid.assign(grids, grids + count);
    int dev = 0, rc = ST_OK;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = stn::host_malloc(&B->h_status, sizeof(int));
    if (e != cudaSuccess) {
        stencil_batch_destroy(B);
        return status(e);
    }
    *B->h_status = 0;

    // one (T, V) for the launch: the compiled candidate with the least predicted total time
    int bps = 0;
    {
        double best = -1.0;
        for (const auto &tv : kCand) {
            int b = 0;
            if ((force_T && tv[0] != force_T) || (force_vec && tv[1] != force_vec)) continue;
            if (tv[0] > L) continue;   // an item's halo rows must come from its neighbours
            if (tb2q_prepare(tv[0], tv[1], &b) != cudaSuccess || b < 1) continue;
            double t = 0.0;
            for (const stencil_batch_grid &q : B->grid) {
                if (q.steps <= 0) continue;
                const double m = batch_model_gcells(q.kind, q.nx, q.ny, q.steps, B->sms, tv[0],
                                                    tv[1], b, L);
                t += (double)q.nx * q.ny * q.steps / std::max(m, 1e-9);
            }
            if (best < 0 || t < best) {
                best = t;
                B->qT = tv[0];
                B->qV = tv[1];
                bps = b;
            }
        }
        (void)cudaGetLastError();
        if (best < 0) rc = ST_ERR_UNSUPPORTED;
    }
    const int T = B->qT, V = B->qV;
    const int halo = (T + 3) / 4 * 4, cx = 32 * V - 2 * halo;

    // Buffers: pass 0 reads grid_in, the last pass writes grid_out, every pass between them
    // reads and writes two grid-sized scratch buffers with rows padded to 32 cells.  So the
    // launch never reads data it wrote itself except from the padded scratch, through
    // 16-byte copies that bypass L1 (a row of the caller's grids may be unaligned and would be
    // read through L1, which other SMs' writes do not update), and a grid run in place needs no
    // final copy.
    B->passes.assign(count, 0);
    B->scratch.assign(2 * count, nullptr);
    B->src.assign(count, nullptr);
    B->ld_scratch.assign(count, 0);
    for (int g = 0; g < count && rc == ST_OK; g++) {
        const stencil_batch_grid &q = B->grid[g];
        B->passes[g] = q.steps > 0 ? (q.steps + T - 1) / T : 0;
        B->ld_scratch[g] = ((long long)q.nx + 31) / 32 * 32;
        const size_t sb = (size_t)B->ld_scratch[g] * q.ny * sizeof(float);
        if (B->passes[g] > 1) e = stn::dev_malloc(&B->scratch[2 * g], sb);
        if (e == cudaSuccess && B->passes[g] > 2) e = stn::dev_malloc(&B->scratch[2 * g + 1], sb);
        if (e == cudaSuccess && B->passes[g] > 0 && q.kind == ST_THERMAL)   // padded rows too
            e = stn::dev_malloc(&B->src[g], sb);
        if (e != cudaSuccess) rc = status(e);
    }

    // grids, pass descriptors and the queue
    std::vector<QGrid> qg(count);
    std::vector<Pass2D> desc;
    std::vector<QItem> items;
    int ndone = 0, nsrcf = 0, maxp = 0;
    for (int g = 0; g < count && rc == ST_OK; g++) {
        const stencil_batch_grid &q = B->grid[g];
        const int P = B->passes[g];
        QGrid &G = qg[g];
        G.kind = q.kind;
        G.ntx = (q.nx + cx - 1) / cx;
        G.nseg = (q.ny + L - 1) / L;
        G.P = P;
        G.nx = q.nx;
        G.ny = q.ny;
        G.done_off = ndone;
        ndone += G.ntx * G.nseg;
        G.srcf_off = nsrcf;
        if (q.kind == ST_THERMAL && P > 0) nsrcf += G.ntx * G.nseg;
        G.pass_base = (int)desc.size();
        G.power = static_cast<const float *>(q.power);
        G.src = B->src[g];
        G.ld_src = B->ld_scratch[g];
        G.amb = q.coeffs[4];
        G.rz = q.coeffs[3];
        G.sdc = q.coeffs[0];
        G.copy_from = nullptr;
        G.ld_copy = q.nx;
        G.copy_to = static_cast<float *>(q.grid_out);
        maxp = std::max(maxp, P);
        const int last = P > 0 ? q.steps - T * (P - 1) : 0;
        for (int p = 0; p < P; p++) {
            Pass2D a = {};
            a.in = p == 0 ? static_cast<const float *>(q.grid_in) : B->scratch[2 * g + (p - 1) % 2];
            a.ld_in = p == 0 ? q.nx : B->ld_scratch[g];
            a.out = p == P - 1 ? static_cast<float *>(q.grid_out) : B->scratch[2 * g + p % 2];
            a.ld_out = p == P - 1 ? q.nx : B->ld_scratch[g];
            a.pw = B->src[g];   // Hotspot: sdc*(p + amb*Rz), rebuilt at every replay
            a.ld_pw = B->ld_scratch[g];
            a.nx = q.nx;
            a.ny = q.ny;
            a.tsteps = (p == P - 1) ? last : T;
            a.ntx = G.ntx;
            a.total_rows = (long long)a.ntx * q.ny;
            for (int i = 0; i < 5; i++) a.k[i] = a.kf[i] = q.coeffs[i];
            a.kf[5] = q.coeffs[0] * q.coeffs[2];
            a.kf[6] = -2.0f * q.coeffs[2];
            if (q.kind == ST_THERMAL) hot_coeffs_src(q.coeffs, a.kf);   // source-map kernels
            a.vec_in = ((uintptr_t)a.in % 16 == 0) && (a.ld_in % 4 == 0);
            a.vec_out = ((uintptr_t)a.out % 16 == 0) && (a.ld_out % 4 == 0);
            a.vec_pw = a.pw ? (((uintptr_t)a.pw % 16 == 0) && (a.ld_pw % 4 == 0)) : 0;
            desc.push_back(a);
        }
        if (P == 0 && q.grid_in != q.grid_out) {
            G.copy_from = static_cast<const float *>(q.grid_in);   // no steps: a plain copy
            G.ld_copy = q.nx;
        }
    }
    // Two queues, one per kind.  Within a queue each grid's pass chain is placed on a timeline
    // of `maxp` slots so that the work per slot is level: the grids with the most work first,
    // each at the start slot that keeps the heaviest slot it touches lightest (a grid of few
    // passes fills in beside the long chains, which start at once: they set the critical path).
    // Items go in slot order (source-map tiles first, copies last); within a slot by grid, row
    // segment, tile column.  Every item depends only on items before it in its queue: its
    // grid's previous pass sits in an earlier slot.
    std::vector<QItem> kitems[2];
    double kwork[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2 && rc == ST_OK; kind++) {
        std::vector<QItem> &its = kitems[kind];
        std::vector<int> start(count, 0), order;
        std::vector<double> load(std::max(maxp, 1), 0.0);
        for (int g = 0; g < count; g++)
            if (qg[g].P > 0 && qg[g].kind == kind) order.push_back(g);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            const double wa = (double)qg[a].nx * qg[a].ny * qg[a].P;
            const double wb = (double)qg[b].nx * qg[b].ny * qg[b].P;
            return wa != wb ? wa > wb : a < b;
        });
        for (int g : order) {
            const int P = qg[g].P;
            const double wgt = (double)qg[g].nx * qg[g].ny;
            int best_s = 0;
            double best_m = 1e300, best_sum = 1e300;
            for (int s0 = 0; s0 + P <= maxp; s0++) {
                double m = 0.0, sum = 0.0;
                for (int k = s0; k < s0 + P; k++) {
                    m = std::max(m, load[k]);
                    sum += load[k];
                }
                if (m < best_m || (m == best_m && sum < best_sum)) {
                    best_m = m;
                    best_sum = sum;
                    best_s = s0;
                }
            }
            start[g] = best_s;
            for (int k = best_s; k < best_s + P; k++) load[k] += wgt;
            const stencil_batch_grid &q = B->grid[g];
            kwork[kind] += (double)q.nx * q.ny * q.steps /
                           std::max(batch_model_gcells(q.kind, q.nx, q.ny, q.steps, B->sms, T, V,
                                                       bps, L), 1e-9);
        }
        if (kind == ST_THERMAL)
            for (int g : order)
                for (int s = 0; s < qg[g].nseg; s++)
                    for (int tx = 0; tx < qg[g].ntx; tx++) its.push_back(QItem{g, -1, tx, s});
        for (int slot = 0; slot < maxp; slot++)
            for (int g = 0; g < count; g++) {
                if (qg[g].kind != kind) continue;
                const int p = slot - start[g];
                if (p < 0 || p >= qg[g].P) continue;
                for (int s = 0; s < qg[g].nseg; s++)
                    for (int tx = 0; tx < qg[g].ntx; tx++) its.push_back(QItem{g, p, tx, s});
            }
        for (int g = 0; g < count; g++)
            if (qg[g].kind == kind && qg[g].copy_from)
                for (int s = 0; s < qg[g].nseg; s++) its.push_back(QItem{g, qg[g].P, 0, s});
    }
    items = kitems[0];
    items.insert(items.end(), kitems[1].begin(), kitems[1].end());
    B->items = (long long)items.size();

    // device table: [items | grids | descriptors | control | counters (reset per replay)]
    const size_t o_items = 0;
    const size_t o_grids = o_items + align256(items.size() * sizeof(QItem));
    const size_t o_desc = o_grids + align256(qg.size() * sizeof(QGrid));
    const size_t o_ctl = o_desc + align256(std::max<size_t>(1, desc.size()) * sizeof(Pass2D));
    const size_t o_cnt = o_ctl + align256(sizeof(QueueCtl));
    const size_t cnt_bytes = (size_t)(3 + ndone + nsrcf) * sizeof(int);   // heads, status, counters
    const size_t table = o_cnt + align256(cnt_bytes);
    if (rc == ST_OK) {
        e = stn::dev_malloc(&B->dev, table);
        if (e != cudaSuccess) rc = status(e);
    }
    char *d = static_cast<char *>(B->dev);
    QueueBatch2D qb = {};
    if (rc == ST_OK) {
        std::vector<unsigned char> host(o_cnt, 0);
        if (!items.empty()) std::memcpy(host.data() + o_items, items.data(), items.size() * sizeof(QItem));
        std::memcpy(host.data() + o_grids, qg.data(), qg.size() * sizeof(QGrid));
        if (!desc.empty()) std::memcpy(host.data() + o_desc, desc.data(), desc.size() * sizeof(Pass2D));
        QueueCtl ctl = {kWaitNs, -1, 0};
        std::memcpy(host.data() + o_ctl, &ctl, sizeof(ctl));
        e = cudaMemcpy(B->dev, host.data(), o_cnt, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = status(e);
        B->ctl = reinterpret_cast<QueueCtl *>(d + o_ctl);
        int *cnt = reinterpret_cast<int *>(d + o_cnt);
        qb.items[0] = reinterpret_cast<const QItem *>(d + o_items);
        qb.items[1] = qb.items[0] + kitems[0].size();
        qb.total[0] = (int)kitems[0].size();
        qb.total[1] = (int)kitems[1].size();
        // SMs per kind in proportion to the kind's predicted time (each SM runs one kind's loop)
        const double wsum = kwork[0] + kwork[1];
        qb.split = wsum > 0 ? (int)std::lround(B->sms * kwork[0] / wsum) : 0;
        qb.L = L;
        qb.grids = reinterpret_cast<const QGrid *>(d + o_grids);
        qb.passes = reinterpret_cast<const Pass2D *>(d + o_desc);
        qb.head = reinterpret_cast<unsigned *>(cnt);
        qb.status = cnt + 2;
        qb.done = cnt + 3;
        qb.srcf = cnt + 3 + ndone;
        qb.ctl = B->ctl;
        // as many one-warp blocks as are resident at once (no more: the rest would only pop
        // items once earlier blocks leave)
        qb.ctas = (int)std::max<long long>(1, std::min<long long>((long long)B->sms * bps,
                                                                   (long long)items.size()));
    }
    // the graph: reset, the one launch, the status word back to the host
    if (rc == ST_OK) {
        e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = cudaMemsetAsync(d + o_cnt, 0, cnt_bytes, B->stream);
            if (le == cudaSuccess && !items.empty()) {
                le = tb2q_launch(T, V, qb, B->stream);
                B->launches = 1;
            }
            if (le == cudaSuccess)
                le = cudaMemcpyAsync(B->h_status, qb.status, sizeof(int), cudaMemcpyDeviceToHost,
                                     B->stream);
            e = cudaStreamEndCapture(B->stream, &B->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
        if (e != cudaSuccess) rc = status(e);
    }
    if (rc != ST_OK) {
        (void)cudaGetLastError();
        stencil_batch_destroy(B);
        return rc;
    }
    *out = B;
    return ST_OK;
}

int stencil_batch_run(stencil_batch b)
{
    if (!b || !b->exec) return ST_ERR_INVALID_ARG;
    const stn::NvtxRange r("stencil_batch_run");
    return status(cudaGraphLaunch(b->exec, b->stream));
}

int stencil_batch_sync(stencil_batch b)
{
    if (!b) return ST_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return ST_ERR_CUDA;
    return *b->h_status ? ST_ERR_TIMEOUT : ST_OK;
}

int stencil_batch_set_wait(stencil_batch b, long long wait_ns, int hold_pass)
{
    if (!b || !b->ctl || wait_ns < 1 || hold_pass < -1) return ST_ERR_INVALID_ARG;
    QueueCtl ctl = {wait_ns, hold_pass, 0};
    cudaError_t e = cudaMemcpyAsync(b->ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? ST_OK : ST_ERR_CUDA;
}

int stencil_batch_get_grid(stencil_batch b, int g, int *T, int *vec, int *passes)
{
    if (!b || g < 0 || g >= (int)b->grid.size() || !T || !vec || !passes) return ST_ERR_INVALID_ARG;
    *T = b->qT;
    *vec = b->qV;
    *passes = b->passes[g];
    return ST_OK;
}

int stencil_batch_launch_count(stencil_batch b)
{
    return b ? b->launches : ST_ERR_INVALID_ARG;
}

int stencil_batch_destroy(stencil_batch b)
{
    if (!b) return ST_OK;
    if (b->exec) {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->exec);
    }
    if (b->graph) cudaGraphDestroy(b->graph);
    for (float *s : b->scratch)
        if (s) stn::dev_free(s);
    for (float *s : b->src)
        if (s) stn::dev_free(s);
    if (b->dev) stn::dev_free(b->dev);
    if (b->h_status) stn::host_free(b->h_status);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return ST_OK;
}

}  // extern "C"
