// Allocation-free variant of stencil_run for 2D grids: stencil_run_noalloc.
//
// Who needs it: code that may not allocate device memory at the point where it advances a grid,
// for example a caller running inside a memory pool or arena it does not own, a real-time or
// signal-driven path where cudaMalloc's implicit device synchronisation and unbounded latency
// are not acceptable, or a host whose allocator is locked down.  stencil_plan_create allocates a
// grid-sized ping-pong buffer; this entry point instead uses one fixed buffer that the library
// reserves when it is loaded.
//
// The buffer is a file-scope __device__ array of kStaticScratchCells floats (16 MiB): every GPU
// on which the library is loaded holds it until the process exits.  Grids larger than that are
// rejected with ST_ERR_TOO_LARGE.  All calls on a device share the one buffer and it keeps
// whatever the previous call left in it; nothing read from it is assumed to start at zero (each
// pass writes every cell it later reads).  Calls whose work overlaps on the GPU (on different
// streams, or from different host threads without ordering) race on the buffer.
//
// Host code cannot use the array's name as a device address: on the host it names a shadow
// variable.  The first call on each device therefore looks the device address up once with
// cudaGetSymbolAddress (with that device current) and caches it; make that first call before
// any stream capture.  The cache entry remembers the CUDA context it was looked up in: after a
// cudaDeviceReset (or any release and re-creation of the device's primary context) the module
// is loaded again and the array may move, so the next call looks the address up again; that
// call, too, should come before any stream capture.  No call allocates: no cudaMalloc,
// cudaFree or allocating library routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/stencil.h"
#include "internal.h"

using namespace stn;

namespace {

constexpr long long kStaticScratchCells = 4LL * 1024 * 1024;   // 16 MiB of float32
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_static_scratch[kStaticScratchCells];

struct DeviceSlot {
    float *scratch = nullptr;   // device address of g_static_scratch on this device
    int sms = 0;
    unsigned long long ctx_id = 0;   // the context the address was looked up in
};

DeviceSlot g_dev[kMaxDevices];
std::mutex g_mu;

int to_status(cudaError_t e)
{
    if (e == cudaSuccess) return ST_OK;
    return ST_ERR_CUDA;
}

// Unique ID of the calling thread's current context (0 when there is none yet or the driver
// cannot tell), through the driver entry points the runtime hands out (no link to libcuda).
unsigned long long current_ctx_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {   // called under g_mu
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f);
            get_id = reinterpret_cast<GetId>(g);
        }
        resolved = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// once per device and context, with that device current: the scratch array's device address,
// the SM count
int device_slot(DeviceSlot **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return to_status(e);
    if (dev < 0 || dev >= kMaxDevices) return ST_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSlot &s = g_dev[dev];
    const unsigned long long ctx = current_ctx_id();
    if (!s.scratch || (ctx && ctx != s.ctx_id)) {
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_static_scratch);   // makes the context current
        if (e != cudaSuccess) return to_status(e);
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return to_status(e);
        s.sms = sms;
        s.scratch = static_cast<float *>(addr);
        s.ctx_id = current_ctx_id();
    }
    *out = &s;
    return ST_OK;
}

const int kTs[] = {1, 2, 4, 6, 8, 12};

int pass2(const DeviceSlot &dv, int kind, int exact, int V, int W, int T, const float *src,
          float *dst, const float *pw, const float *k, int nx, int ny, int tsteps,
          cudaStream_t st)
{
    // the kernel of the smallest compiled T >= tsteps in this (kind, exact, V, W) family
    int Tk = 0;
    for (int t : kTs)
        if (t >= tsteps && t <= T && tb2d_available(Shape2D{kind, exact, t, V, W})) {
            Tk = t;
            break;
        }
    if (!Tk) return ST_ERR_UNSUPPORTED;
    const Shape2D sh{kind, exact, Tk, V, W};
    int bps = 0;
    cudaError_t e = tb2d_prepare(sh, &bps);
    if (e != cudaSuccess) return to_status(e);
    if (bps < 1) return ST_ERR_UNSUPPORTED;
    const int bx = tb2d_tile_width(sh), h = tb2d_halo(sh), cx = bx - 2 * h;
    Pass2D a = {};
    a.in = src;
    a.out = dst;
    a.pw = pw;
    a.ld_in = nx;
    a.ld_out = nx;
    a.ld_pw = nx;
    a.nx = nx;
    a.ny = ny;
    a.tsteps = tsteps;
    a.ntx = (nx + cx - 1) / cx;
    a.total_rows = (long long)a.ntx * ny;
    const long long min_rows = 4;   // short segments keep small grids parallel
    const long long ctas = std::min<long long>((long long)dv.sms * bps,
                                               std::max<long long>(1, a.total_rows / min_rows));
    a.rows_per_cta = (a.total_rows + ctas - 1) / ctas;
    a.ctas = (int)((a.total_rows + a.rows_per_cta - 1) / a.rows_per_cta);
    for (int i = 0; i < 5; i++) a.k[i] = a.kf[i] = k[i];
    a.kf[5] = k[0] * k[2];    // Hotspot: sdc * Ry, rounded once (float32)
    a.kf[6] = -2.0f * k[2];   // Hotspot: -2 Ry (exact)
    a.vec_in = ((uintptr_t)src % 16 == 0) && (nx % 4 == 0);
    a.vec_out = ((uintptr_t)dst % 16 == 0) && (nx % 4 == 0);
    a.vec_pw = pw ? (((uintptr_t)pw % 16 == 0) && (nx % 4 == 0)) : 0;
    return to_status(tb2d_launch(sh, a, st));
}

}  // namespace

extern "C" int stencil_run_noalloc(int kind, const void *grid_in, void *grid_out,
                                   const void *power, const float *coeffs, int nx, int ny,
                                   int steps, int exact, int T, void *stream)
{
    if (kind != ST_DIFFUSION && kind != ST_THERMAL) return ST_ERR_INVALID_ARG;
    if (!grid_in || !grid_out || !coeffs || nx < 1 || ny < 1 || steps < 0 || T < 0)
        return ST_ERR_INVALID_ARG;
    if ((kind == ST_THERMAL) != (power != nullptr)) return ST_ERR_INVALID_ARG;
    const long long cells = (long long)nx * ny;
    if (cells > kStaticScratchCells) return ST_ERR_TOO_LARGE;
    const size_t bytes = (size_t)cells * sizeof(float);
    const uintptr_t pi = (uintptr_t)grid_in, po = (uintptr_t)grid_out;
    if (pi != po && pi < po + bytes && po < pi + bytes) return ST_ERR_INVALID_ARG;
    if (power) {
        const uintptr_t pp = (uintptr_t)power;
        if (pp < po + bytes && po < pp + bytes) return ST_ERR_INVALID_ARG;
    }
    const stn::NvtxRange r("stencil_run_noalloc");
    DeviceSlot *dv = nullptr;
    int rc = device_slot(&dv);
    if (rc != ST_OK) return rc;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *in = static_cast<const float *>(grid_in);
    float *out = static_cast<float *>(grid_out);
    const float *pw = static_cast<const float *>(power);
    if (steps == 0) {
        if (in == out) return ST_OK;
        return to_status(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st));
    }
    // same tile families as a default plan: exact -> rotating windows (V = 4, four warps on
    // wide grids), contracted -> partial-sum stages in one warp (Hotspot V = 4, Diffusion V = 8)
    const int ex = exact ? 1 : 0;
    const int V = (ex || kind == ST_THERMAL) ? 4 : 8;
    const int W = (ex && nx >= 512) ? 4 : 1;
    int Tp = T ? T : 8;
    if (!tb2d_available(Shape2D{kind, ex, Tp, V, W})) return ST_ERR_UNSUPPORTED;

    const int passes = (steps + Tp - 1) / Tp;
    const int last = steps - Tp * (passes - 1);
    // pass i writes the output when (passes-1-i) is even, else the static scratch; in place
    // with an odd pass count every pass shifts by one and a final copy lands the result
    const bool shift = (in == out) && (passes % 2 == 1);
    float *scratch = dv->scratch;
    const float *src = in;
    for (int i = 0; i < passes; i++) {
        const int ts = (i == passes - 1) ? last : Tp;
        const bool to_out = shift ? ((passes - i) % 2 == 0) : ((passes - 1 - i) % 2 == 0);
        float *dst = to_out ? out : scratch;
        rc = pass2(*dv, kind, ex, V, W, Tp, src, dst, pw, coeffs, nx, ny, ts, st);
        if (rc != ST_OK) return rc;
        src = dst;
    }
    if (shift) return to_status(cudaMemcpyAsync(out, scratch, bytes, cudaMemcpyDeviceToDevice, st));
    return ST_OK;
}
