// Many 2D grids of uneven sizes and step counts advanced by one CUDA-graph launch.
//
// Each grid gets its own (T, cells per thread) from the GPU restatement of the paper's model
// (Eqs. 3-9, model.cu) and its own ping-pong scratch, and runs ceil(steps/T) temporally-blocked
// passes like stencil_run (Sec. 3.2; the last pass fuses the remainder).  Grids that share a
// kernel instance (stencil kind, T, V) form a group; pass p of a group is one persistent launch
// over a work queue of all its grids' (tile column, row) units that run a pass in that launch,
// split evenly over the blocks, so small and large grids are served in the same launch without
// idle blocks; each grid's chain of passes starts at the launch slot that levels the work of
// the group's launches (a grid with few passes fills in where long-running grids leave room).
// All launches (and the final copies of grids run in place with an odd pass count) are
// captured once into a CUDA graph with one branch per group; stencil_batch_run replays it.
// The order of passes of one grid is the order of launches on its branch: no device-side
// waiting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

using namespace stn;

namespace stn {
double batch_model_gcells(int kind, int nx, int ny, int steps, int sms, int T, int V, int bps);
}

struct stencil_batch_s {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    std::vector<stencil_batch_grid> grid;
    std::vector<int> T, V, passes;
    std::vector<float *> scratch;
    std::vector<float *> src;         // Hotspot grids: the source map p + amb*Rz
    std::vector<long long> ld_scratch;
    void *dev = nullptr;              // descriptors and prefix arrays of every (group, pass)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

namespace {

int status(cudaError_t e)
{
    if (e == cudaSuccess) return ST_OK;
    return e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA;
}

const int kCand[][2] = {{4, 4}, {8, 4}, {4, 8}, {8, 8}};   // (T, V) compiled for batches

struct LaunchRec {
    int group;                     // branch of the graph the launch is captured on
    Shape2D shape;
    BatchPass2D bp;
    size_t desc_off, prefix_off;   // byte offsets into the device table
    std::vector<Pass2D> desc;
    std::vector<long long> prefix;
};

}  // namespace

extern "C" {

int stencil_batch_create(stencil_batch *out, const stencil_batch_grid *grids, int count,
                         void *stream)
{
    if (!out) return ST_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grids || count < 1) return ST_ERR_INVALID_ARG;
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
    if (e != cudaSuccess) {
        delete B;
        return status(e);
    }
    // per-grid parameters from the model
    B->T.resize(count);
    B->V.resize(count);
    B->passes.resize(count);
    B->scratch.assign(count, nullptr);
    B->src.assign(count, nullptr);
    B->ld_scratch.resize(count);
    // One (T, V) per kind: the grids that share a kernel run together in each launch slot, so
    // a split of one kind over several kernels multiplies the launches and leaves each of them
    // small.  The choice minimises the kind's predicted total time, sum over its grids of
    // cells x steps / modelled rate.
    int kind_T[2] = {0, 0}, kind_V[2] = {0, 0};
    for (int kind = 0; kind < 2; kind++) {
        double best = -1.0;
        for (const auto &tv : kCand) {
            const Shape2D sh{kind, 0, tv[0], tv[1], 1};
            int bps = 0;
            if (tb2d_batch_prepare(sh, &bps) != cudaSuccess || bps < 1) continue;
            double t = 0.0;
            for (int g = 0; g < count; g++) {
                const stencil_batch_grid &q = B->grid[g];
                if (q.kind != kind || q.steps <= 0) continue;
                const double m = batch_model_gcells(q.kind, q.nx, q.ny, q.steps, B->sms, tv[0], tv[1], bps);
                t += (double)q.nx * q.ny * q.steps / std::max(m, 1e-9);
            }
            if (best < 0 || t < best) {
                best = t;
                kind_T[kind] = tv[0];
                kind_V[kind] = tv[1];
            }
        }
        (void)cudaGetLastError();
        if (best < 0) rc = ST_ERR_UNSUPPORTED;
    }
    for (int g = 0; g < count && rc == ST_OK; g++) {
        const stencil_batch_grid &q = B->grid[g];
        B->T[g] = kind_T[q.kind];
        B->V[g] = kind_V[q.kind];
        B->passes[g] = q.steps > 0 ? (q.steps + B->T[g] - 1) / B->T[g] : 0;
        B->ld_scratch[g] = ((long long)q.nx + 31) / 32 * 32;
        if (rc == ST_OK && B->passes[g] > 0) {
            e = cudaMalloc(&B->scratch[g], (size_t)B->ld_scratch[g] * q.ny * sizeof(float));
            if (e == cudaSuccess && q.kind == ST_THERMAL)
                e = cudaMalloc(&B->src[g], (size_t)q.nx * q.ny * sizeof(float));
            if (e != cudaSuccess) rc = status(e);
        }
    }
    // launches: group (kind, T, V) x pass index
    std::vector<LaunchRec> recs;
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    for (int g = 0; g < count; g++)
        if (B->passes[g] > 0) groups[std::make_tuple(B->grid[g].kind, B->T[g], B->V[g])].push_back(g);
    // Level the work of a group's launches: grid g's P_g passes occupy launch slots
    // [start_g, start_g + P_g) of the group's timeline of max P slots; largest grids first, each
    // at the start that keeps the heaviest slot it touches lightest.
    std::vector<int> start(count, 0);
    int maxp = 0;
    for (int g = 0; g < count; g++) maxp = std::max(maxp, B->passes[g]);
    for (auto &kv : groups) {
        int S = 0;
        for (int g : kv.second) S = std::max(S, B->passes[g]);
        std::vector<double> load(S, 0.0);
        std::vector<int> order = kv.second;
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            return (double)B->grid[a].nx * B->grid[a].ny * B->passes[a] >
                   (double)B->grid[b].nx * B->grid[b].ny * B->passes[b];
        });
        for (int g : order) {
            const int P = B->passes[g];
            const double wgt = (double)B->grid[g].nx * B->grid[g].ny;
            int best_s = 0;
            double best_m = 1e300, best_sum = 1e300;
            for (int s0 = 0; s0 + P <= S; s0++) {
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
        }
    }
    size_t table = 0;
    std::vector<int> group_of(count, -1);
    {
        int gi = 0;
        for (auto &kv : groups) {
            for (int g : kv.second) group_of[g] = gi;
            gi++;
        }
    }
    for (int slot = 0; slot < maxp && rc == ST_OK; slot++) {
        int gi = -1;
        for (auto &kv : groups) {
            gi++;
            const int kind = std::get<0>(kv.first), T = std::get<1>(kv.first), V = std::get<2>(kv.first);
            LaunchRec r;
            r.group = gi;
            r.shape = Shape2D{kind, 0, T, V, 1};
            const int bx = 32 * V, h = (T + 3) / 4 * 4, cx = bx - 2 * h;
            r.prefix.push_back(0);
            for (int g : kv.second) {
                const stencil_batch_grid &q = B->grid[g];
                const int P = B->passes[g];
                const int p = slot - start[g];   // this grid's pass in this slot
                if (p < 0 || p >= P) continue;
                const int last = q.steps - T * (P - 1);
                const bool shift = (q.grid_in == q.grid_out) && (P % 2 == 1);
                auto to_out = [&](int i) { return shift ? ((P - i) % 2 == 0) : ((P - 1 - i) % 2 == 0); };
                Pass2D a = {};
                const bool src_in = (p == 0);
                const bool src_out = !src_in && to_out(p - 1);
                a.in = src_in ? static_cast<const float *>(q.grid_in)
                              : (src_out ? static_cast<const float *>(q.grid_out) : B->scratch[g]);
                a.ld_in = (src_in || src_out) ? q.nx : B->ld_scratch[g];
                a.out = to_out(p) ? static_cast<float *>(q.grid_out) : B->scratch[g];
                a.ld_out = to_out(p) ? q.nx : B->ld_scratch[g];
                a.pw = B->src[g];   // Hotspot: p + amb*Rz, rebuilt at every replay
                a.ld_pw = q.nx;
                a.nx = q.nx;
                a.ny = q.ny;
                a.tsteps = (p == P - 1) ? last : T;
                a.ntx = (q.nx + cx - 1) / cx;
                a.total_rows = (long long)a.ntx * q.ny;
                for (int i = 0; i < 5; i++) a.k[i] = a.kf[i] = q.coeffs[i];
                a.kf[5] = q.coeffs[0] * q.coeffs[2];
                a.kf[6] = -2.0f * q.coeffs[2];
                if (q.kind == ST_THERMAL) hot_coeffs_src(q.coeffs, a.kf);   // source-map kernels
                a.vec_in = ((uintptr_t)a.in % 16 == 0) && (a.ld_in % 4 == 0);
                a.vec_out = ((uintptr_t)a.out % 16 == 0) && (a.ld_out % 4 == 0);
                a.vec_pw = a.pw ? (((uintptr_t)a.pw % 16 == 0) && (q.nx % 4 == 0)) : 0;
                r.desc.push_back(a);
                r.prefix.push_back(r.prefix.back() + a.total_rows);
            }
            if (r.desc.empty()) continue;
            int bps = 0;
            e = tb2d_batch_prepare(r.shape, &bps);
            if (e != cudaSuccess || bps < 1) {
                rc = e != cudaSuccess ? status(e) : ST_ERR_UNSUPPORTED;
                break;
            }
            r.bp.ngrids = (int)r.desc.size();
            r.bp.total_units = r.prefix.back();
            const long long min_rows = 4;   // short segments keep small grids parallel
            const long long ctas = std::min<long long>((long long)B->sms * bps,
                                                       std::max<long long>(1, r.bp.total_units / min_rows));
            r.bp.units_per_cta = (r.bp.total_units + ctas - 1) / ctas;
            r.bp.ctas = (int)((r.bp.total_units + r.bp.units_per_cta - 1) / r.bp.units_per_cta);
            r.desc_off = table;
            table += (r.desc.size() * sizeof(Pass2D) + 255) / 256 * 256;
            r.prefix_off = table;
            table += (r.prefix.size() * sizeof(long long) + 255) / 256 * 256;
            recs.push_back(std::move(r));
        }
    }
    if (rc == ST_OK && table) {
        e = cudaMalloc(&B->dev, table);
        if (e != cudaSuccess) rc = status(e);
    }
    if (rc == ST_OK && table) {
        std::vector<unsigned char> host(table, 0);
        for (LaunchRec &r : recs) {
            std::memcpy(host.data() + r.desc_off, r.desc.data(), r.desc.size() * sizeof(Pass2D));
            std::memcpy(host.data() + r.prefix_off, r.prefix.data(), r.prefix.size() * sizeof(long long));
            r.bp.grids = reinterpret_cast<const Pass2D *>(static_cast<char *>(B->dev) + r.desc_off);
            r.bp.prefix = reinterpret_cast<const long long *>(static_cast<char *>(B->dev) + r.prefix_off);
        }
        e = cudaMemcpy(B->dev, host.data(), table, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = status(e);
    }
    // Capture every launch (and the in-place copies) into one graph.  Each group is a branch
    // of its own (captured on its own stream, forked from and joined back into B->stream), so
    // the groups' launches overlap on the GPU and one group's launch tails fill with another's
    // work; within a branch, launch order is pass order.
    if (rc == ST_OK) {
        const int ng = (int)groups.size();
        std::vector<cudaStream_t> gs(ng, nullptr);
        std::vector<cudaEvent_t> join(ng, nullptr);
        cudaEvent_t fork = nullptr;
        e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int i = 0; i < ng && e == cudaSuccess; i++) {
            e = cudaStreamCreateWithFlags(&gs[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            // Hotspot source maps from the power maps' current contents, before any pass
            cudaError_t le = cudaSuccess;
            for (int g = 0; g < count && le == cudaSuccess; g++)
                if (B->src[g]) {
                    const stencil_batch_grid &q = B->grid[g];
                    le = hot_source(static_cast<const float *>(q.power), q.nx, B->src[g], q.nx,
                                    q.ny, q.coeffs[4], q.coeffs[3], B->stream);
                    B->launches++;
                }
            if (le == cudaSuccess) le = cudaEventRecord(fork, B->stream);
            for (int i = 0; i < ng && le == cudaSuccess; i++) le = cudaStreamWaitEvent(gs[i], fork, 0);
            for (const LaunchRec &r : recs) {
                if (le == cudaSuccess) le = tb2d_batch_launch(r.shape, r.bp, gs[r.group]);
                B->launches++;
            }
            for (int g = 0; g < count && le == cudaSuccess; g++) {
                const stencil_batch_grid &q = B->grid[g];
                const int P = B->passes[g];
                if (P == 0 && q.grid_in != q.grid_out)
                    le = cudaMemcpyAsync(q.grid_out, q.grid_in, (size_t)q.nx * q.ny * sizeof(float),
                                         cudaMemcpyDeviceToDevice, B->stream);
                else if (P > 0 && q.grid_in == q.grid_out && P % 2 == 1)
                    le = cudaMemcpy2DAsync(q.grid_out, (size_t)q.nx * sizeof(float), B->scratch[g],
                                           (size_t)B->ld_scratch[g] * sizeof(float),
                                           (size_t)q.nx * sizeof(float), q.ny,
                                           cudaMemcpyDeviceToDevice, gs[group_of[g]]);
            }
            for (int i = 0; i < ng; i++) {
                cudaError_t je = cudaEventRecord(join[i], gs[i]);
                if (je == cudaSuccess) je = cudaStreamWaitEvent(B->stream, join[i], 0);
                if (le == cudaSuccess) le = je;
            }
            e = cudaStreamEndCapture(B->stream, &B->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
        for (int i = 0; i < ng; i++) {
            if (join[i]) cudaEventDestroy(join[i]);
            if (gs[i]) cudaStreamDestroy(gs[i]);
        }
        if (fork) cudaEventDestroy(fork);
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
    return status(cudaGraphLaunch(b->exec, b->stream));
}

int stencil_batch_get_grid(stencil_batch b, int g, int *T, int *vec, int *passes)
{
    if (!b || g < 0 || g >= (int)b->grid.size() || !T || !vec || !passes) return ST_ERR_INVALID_ARG;
    *T = b->T[g];
    *vec = b->V[g];
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
        if (s) cudaFree(s);
    for (float *s : b->src)
        if (s) cudaFree(s);
    if (b->dev) cudaFree(b->dev);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return ST_OK;
}

}  // extern "C"
