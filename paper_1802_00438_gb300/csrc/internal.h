// Interface between the host runtime (api.cu) and the kernel translation units.
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/stencil.h"

namespace stn {

// One pass of the 2D temporally-blocked sweep (tb2d.cu).
struct Pass2D {
    const float *in;
    float *out;
    const float *pw;       // power map (thermal), coefficient planes (per-cell diffusion) or nullptr
    long long ld_in, ld_out, ld_pw;   // row pitches in floats
    long long pw_plane;    // per-cell diffusion: floats from one coefficient plane to the next
    int nx, ny;
    int tsteps;            // steps fused in this pass, 1..T
    int ntx;               // tiles along x
    long long total_rows;  // ntx * ny: the (tile column, row) pairs of the pass
    long long rows_per_cta;
    const long long *starts;   // contracted kernel: block b takes pairs [starts[b], starts[b+1])
                               // (nullptr: rows_per_cta pairs each)
    int ctas;
    float k[5];
    // contracted kernel's coefficients, derived on the host from k: diffusion cc, cw, ce, cs, cn;
    // Hotspot sdc, Rx, Ry, Rz, amb, sdc*Ry (rounded once), -2*Ry (exact)
    float kf[7];
    int vec_in, vec_out, vec_pw;   // 1: rows start on 16-byte boundaries
    // 16-bit storage (contracted kernel, stor != 0): raw grids, block codes per (row, tile)
    int stor;                      // 0 float32, 1 bf16, 2 fp16
    const void *qin;
    void *qout;
    const void *qpw;
    const float2 *min_;
    float2 *mout;
    const float2 *mpw;
    long long ld_q;                // row pitch of the 16-bit grids, cells (multiple of 8)
    // trajectory passes (STOR_ALL): step t < tsteps-1 of the pass goes to states + t*state_stride
    float *states;
    long long state_stride;
};

// stor: storage format (0 float32, 1 bf16, 2 fp16) plus 4 when the kernel stages the Hotspot
// source map sdc*(p + amb*Rz) instead of the power map (every contracted Hotspot plan and batch)
struct Shape2D { int kind, exact, T, V, W; int stor = 0; };
enum { STOR_SRC = 4,     // Hotspot: the power rows carry sdc*(p + amb*Rz) (source map)
       STOR_ALL = 8 };    // every fused step's rows are also written (trajectory passes)

// Many 2D grids in ONE persistent launch fed by a work queue (k_tb2f_queue).  Items are
// popped in queue order by the launch's blocks; an item is
//   k = -1      : grid g's Hotspot source map sdc*(p + amb*Rz) over tile tx's compute columns,
//                 rows [seg*L, seg*L + L)
//   0 <= k < P  : pass k of grid g over tile column tx, rows [seg*L, seg*L + L)
//   k = P = 0   : copy of those rows from copy_from (grid_in) to copy_to (grid_out), for a grid
//                 with no steps
// and it waits (bounded) for what it reads and overwrites: pass k > 0 needs pass k-1 of the
// neighbouring tiles (tx +- 1, seg +- 1) finished (RAW on the halo, WAR on the ping-pong buffer
// it writes), pass 0 of a Hotspot grid needs the source map of tiles (tx +- 1, seg +- 1).
// done[g][seg][tx] holds the number of passes finished, srcf[g][seg][tx] 1 once the tile's
// source map is written.
struct QItem { int g, k, tx, seg; };
struct QGrid {
    int kind, ntx, nseg, P, nx, ny;
    int done_off, srcf_off, pass_base;
    const float *power;       // Hotspot: the power map (dense rows of nx)
    float *src;               // Hotspot: the source map it builds (rows ld_src apart)
    long long ld_src;
    float amb, rz, sdc;
    const float *copy_from;   // k = P items
    long long ld_copy;
    float *copy_to;
};
struct QueueCtl {
    long long wait_ns;        // a dependency wait gives up after this long (status = 1)
    int hold_pass;            // test hook, -1 = off: items of this pass never report finished
    int pad;
};
// Two queues, one per stencil kind (their items never depend on each other's): a block starts
// on the queue of its SM (SMs below `split` take diffusion items, the others Hotspot items,
// so each SM's instruction cache holds one kind's loop) and moves to the other queue once its
// own is empty.
struct QueueBatch2D {
    const QItem *items[2];
    int total[2];
    int split;
    int L;                    // rows per item
    const QGrid *grids;
    const Pass2D *passes;     // grids[g].pass_base + k
    int *done;
    int *srcf;
    unsigned *head;           // next item of each queue (two counters)
    int *status;              // 0, or 1 once a wait gave up (every block then leaves)
    const QueueCtl *ctl;
    int ctas;
};
bool tb2q_available(int T, int V);
cudaError_t tb2q_prepare(int T, int V, int *blocks_per_sm);
cudaError_t tb2q_launch(int T, int V, const QueueBatch2D &q, cudaStream_t st);


// Block codec of the 16-bit storage: one (offset, scale) per (row, tile column) of the tiling
// with compute width cx; x = offset + scale * q, q in [-1, 1].
// src_mul != 0: code the Hotspot source map sdc*(p + amb*Rz) of the power map src instead
// (src_mul = sdc, src_add = amb*Rz rounded once)
cudaError_t lp_encode(int stor, const float *src, long long ld_src, void *dst, long long ld_q,
                      float2 *meta, int nx, int ny, int cx, cudaStream_t st, float src_add = 0.f,
                      float src_mul = 0.f);
cudaError_t lp_decode(int stor, const void *src, long long ld_q, const float2 *meta, float *dst,
                      long long ld_dst, int nx, int ny, int cx, cudaStream_t st);

// Contracted Hotspot coefficients of the source-map kernels (STOR_SRC) from [sdc, Rx, Ry, Rz,
// amb]: kf = [cc, cx, cy, cz, amb, cy, 0] with cx ~ sdc*Rx, cy ~ sdc*Ry rounded so that
// cc = 1 - 2cx - 2cy is exact, cz = sdc*Rz
void hot_coeffs_src(const float *k, float *kf);

// Hotspot source map dst = sdc*(p + amb*Rz) (rows ld_d floats apart), read by the contracted
// kernels
cudaError_t hot_source(const float *p, long long ld_p, float *dst, long long ld_d, int nx, int ny,
                       float amb, float rz, float sdc, cudaStream_t st);

bool tb2d_available(const Shape2D &s);
int tb2d_block_threads(const Shape2D &s);
int tb2d_tile_width(const Shape2D &s);   // cells per tile incl. halos
int tb2d_halo(const Shape2D &s);
size_t tb2d_smem_bytes(const Shape2D &s);
cudaError_t tb2d_prepare(const Shape2D &s, int *blocks_per_sm);   // smem opt-in + occupancy
cudaError_t tb2d_launch(const Shape2D &s, const Pass2D &p, cudaStream_t st);

// One pass of the radius-R star diffusion in 2D (star2d.cu): 128 x 128 tiles, halos R*T.
struct PassStar2D {
    const float *in;
    float *out;
    long long ld_in, ld_out;   // row pitches in floats
    int nx, ny;
    int tsteps;                // steps fused in this pass, 1..T
    int ntx, nty;              // tiles along x and y
    float k[17];               // cc, then cw, ce, cs, cn per distance 1..R
    int use_tma;               // stage the tile by one tensor-map copy
    int vec_out;               // output rows start on 16-byte boundaries
    int *err;                  // device flag: a bounded wait gave up
};

bool star2d_available(int R, int exact, int T);
int star2d_halo_x(int R, int T);
int star2d_halo_y(int R, int T);
cudaError_t star2d_prepare(int R, int exact, int T);
cudaError_t star2d_launch(int R, int exact, int T, const PassStar2D &p, const CUtensorMap &tin,
                          cudaStream_t st);

// One pass of the 3D star diffusion of radius R (star3d.cu): one block per (tile, z-segment).
struct PassStar3D {
    const float *in;
    float *out;
    int nx, ny, nz;            // dense grids: row pitch nx, plane pitch nx * ny
    int tsteps;                // steps fused in this pass, 1..T
    int ntx, nty;              // tiles along x and y
    int nseg, zseg;            // z-segments per tile column and their length in planes
    float k[25];               // cc, then cw, ce, cs, cn, cb, ca per distance 1..R
    int use_tma;               // stage planes by tensor-map copies
    int vec_out;               // output rows start on 16-byte boundaries
    int *err;                  // device flag: a bounded wait gave up
};

bool star3d_available(int R, int exact, int T);
void star3d_tile(int R, int T, int *cx, int *cy);   // compute block per tile
cudaError_t star3d_prepare(int R, int exact, int T, int *blocks_per_sm);
cudaError_t star3d_launch(int R, int exact, int T, const PassStar3D &p, const CUtensorMap &tin,
                          cudaStream_t st);

// One pass of the 3D sweep (tb3d.cu).
struct Pass3D {
    const float *in;
    float *out;
    const float *pw;
    int nx, ny, nz;
    int tsteps;
    int ntx, nty;          // tiles along x and y
    long long total_cols;  // ntx * nty tile columns (each streamed along z)
    long long planes_per_cta;
    int ctas;
    int zslab;             // partial-sum kernel: > 0 = pieces of zslab planes, round-robin
    long long pieces;      // total_cols * ceil(nz / zslab)
    const long long *starts;   // partial-sum kernel, zslab = 0: block b takes units
                               // [starts[b], starts[b+1]) (nullptr: planes_per_cta each)
    float k[9];
    int vec;               // 1: rows start on 16-byte boundaries
    int vec_pw;            // 1: the power map's rows start on 16-byte boundaries
    int use_tma;           // partial-sum kernel: stage planes with tensor-map bulk copies
    int *err;              // device flag: a bounded wait gave up (set to 1)
};

// Tensor maps of the field and power grids (x, y, z; box = one tile plane) for use_tma.
struct Tma3D {
    CUtensorMap in, pw;
};

// tile (32*VX) x (VY*NW) cells; alg 0: three-plane register windows (k_tb3d, VX = 2, exact or
// contracted), alg 1: partial sums along z (k_tb3f, contracted only)
struct Shape3D { int kind, exact, T, VY, NW; int alg = 0; int VX = 2; };

bool tb3d_available(const Shape3D &s);
int tb3d_block_threads(const Shape3D &s);
int tb3d_halo(const Shape3D &s);
size_t tb3d_smem_bytes(const Shape3D &s);
cudaError_t tb3d_prepare(const Shape3D &s, int *blocks_per_sm);
cudaError_t tb3d_launch(const Shape3D &s, const Pass3D &p, const Tma3D &t, cudaStream_t st);
// encode the tensor map of a (nx, ny, nz) float32 grid with a (bx, by, 1) box; false if the
// driver entry point or the encoding is unavailable
bool tma3d_encode(CUtensorMap *m, const float *base, int nx, int ny, int nz, int bx, int by);

// Resident tiles (res2d.cu): the whole 2D grid held on chip by nbx x nby co-resident blocks
// for a run of `steps` steps, halos exchanged through L2 every T steps (an epoch).
struct Res2D {
    const float *in;       // grid_in, rows of ld_in floats
    long long ld_in;
    float *out;            // grid_out, dense rows of nx
    const float *aux;      // Hotspot: the power map, rows of ld_aux floats
    long long ld_aux;
    float src_sdc, src_a;  // contracted Hotspot: the source map sdc*(p + amb*Rz), a = amb*Rz
    float *xg;             // two exchange grids (epoch parity), rows of ld_x floats
    long long xplane, ld_x;
    int *flags;            // per block: epochs published, as epoch0 + e + 1 (never reset)
    int epoch0;
    int *status;           // set to 1 by a wait that gave up
    long long wait_ns;     // bound of every wait
    int hold_block, hold_epoch;   // test hook: that block publishes no exchange >= hold_epoch
    int nx, ny, steps, T;
    int nbx, nby, cw, ch, hx, hy;   // blocks, compute block size, halo widths
    float k[5];            // Diffusion: cc cw ce cs cn; Hotspot exact: sdc Rx Ry Rz amb;
                           // Hotspot contracted: cc cx cy cz (expanded weights)
};

// A named range on the host timeline for tools (ncu --nvtx, Nsight Systems): NVTX3, header
// only; without a tool attached a push or pop returns at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device and pinned-host allocations of the library (alloc.cu): failure injection and live
// accounting for tests (stencil_debug_fail_alloc, stencil_debug_live_allocs).
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
cudaError_t host_malloc(void **p, size_t bytes);
void host_free(void *p);
template <class T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
template <class T>
cudaError_t host_malloc(T **p, size_t bytes)
{
    return host_malloc(reinterpret_cast<void **>(p), bytes);
}

int res2d_rows_per_thread();
int res2d_max_warps(int kind, int exact, int vx);
size_t res2d_smem(int vx, int nw);
bool res2d_available(int kind, int exact, int vx);
cudaError_t res2d_occupancy(int kind, int exact, int vx, int nw, int *blocks_per_sm);
cudaError_t res2d_launch(int kind, int exact, int vx, int nw, const Res2D &a, cudaStream_t st);

// tuning cache (tune.cu): the measured configuration for the desc's problem key, if any, as
// desc fields (force_T, force_bx, force_by, force_vec, partial_rows, resident)
bool tune_cache_lookup(const stencil_desc &d, int *f6);

}  // namespace stn
