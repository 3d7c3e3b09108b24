// Host runtime of the stencil engine: plans, parameter choice, pass scheduling, validation.
//
// A run of `steps` Jacobi steps is ceil(steps / T) passes over device memory (Eq. 8 of
// arXiv 1802.00438), each pass one launch of a temporally-blocked kernel that fuses up to T
// steps; the last pass fuses the remainder (Sec. 3.2).  Passes ping-pong between the caller's
// output buffer and one plan-owned scratch grid (Sec. 2.1's second buffer), ordered so that
// the last pass lands in the output.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

using namespace stn;

namespace {

struct PassCfg2D {
    Shape2D shape;
    int ntx = 0;
    long long total = 0, rows_per_cta = 0;
    int ctas = 0;
    long long *starts = nullptr;   // device: cost-balanced ranges (contracted kernel), or none
    bool ready = false;
};

// Ranges of (tile column, row or plane) units, one per block, balanced by cost rather than by
// count: a segment streams 2T rows (planes) of pipeline fill besides its own (Sec. 3.2), so a
// block whose range crosses a tile column pays the fill twice, and a unit of an edge tile column
// costs more (its warps run the clamp selects): w[col] per unit.  The slowest block sets the
// pass time.  Greedy cut at the mean cost.  Returns the ranges' largest cost and fills starts
// (ctas + 1 entries).
double balanced_ranges(long long len, int ctas, int fill, const std::vector<double> &w,
                       std::vector<long long> &st)
{
    const long long ncol = (long long)w.size(), total = ncol * len;
    double weighted = 0.0;
    for (double x : w) weighted += x * len;
    const double target = (weighted + (double)fill * (ctas + ncol - 1)) / ctas;
    st.assign(ctas + 1, total);
    long long u = 0;
    for (int b = 0; b < ctas; b++) {
        st[b] = u;
        double cost = 0.0;
        while (u < total) {
            const long long col = u / len, col_end = (col + 1) * len;
            const double room = target - cost - fill;
            if (room < w[col] && cost > 0.0) break;
            const long long take = std::min<long long>(col_end - u, std::max<long long>(1, (long long)std::ceil(room / w[col])));
            cost += fill + w[col] * (double)take;
            u += take;
            if (cost >= target) break;
        }
    }
    double worst = 0.0;
    for (int b = 0; b < ctas; b++) {   // the last block also takes whatever is left
        double c = 0.0;
        for (long long x = st[b]; x < st[b + 1];) {
            const long long e = std::min(st[b + 1], (x / len + 1) * len);
            c += fill + w[x / len] * (double)(e - x);
            x = e;
        }
        worst = std::max(worst, c);
    }
    return worst;
}

// the largest cost of ranges of `per` units each (same costs)
double even_ranges_cost(long long len, long long per, int fill, const std::vector<double> &w)
{
    const long long total = (long long)w.size() * len;
    double worst = 0.0;
    for (long long a = 0; a < total; a += per) {
        const long long e = std::min(total, a + per);
        double c = 0.0;
        for (long long x = a; x < e;) {
            const long long f = std::min(e, (x / len + 1) * len);
            c += fill + w[x / len] * (double)(f - x);
            x = f;
        }
        worst = std::max(worst, c);
    }
    return worst;
}

struct PassCfg3D {
    Shape3D shape;
    int ntx = 0, nty = 0;
    long long cols = 0, planes_per_cta = 0;
    int ctas = 0;
    int zslab = 0;          // > 0: round-robin pieces of zslab planes (partial-sum kernel)
    long long pieces = 0;
    long long *starts = nullptr;   // device: cost-balanced ranges (zslab = 0), or none
    bool ready = false;
};

}  // namespace

struct stencil_plan_s {
    stencil_desc d;
    cudaStream_t stream = nullptr;
    int device = 0, sms = 0;
    float *scratch = nullptr;
    long long ld_scratch = 0;   // row pitch of the scratch grid (2D), floats
    size_t scratch_bytes = 0;
    int T = 1;
    // 2D
    int V = 4, W = 4;
    std::vector<PassCfg2D> cfg2;   // indexed by kernel T
    // 3D
    int VY = 8, NW = 8, alg3 = 0, VX3 = 2;
    int *err = nullptr;   // device flag set by a kernel whose bounded wait gave up
    double model = 0.0;   // calibrated model's prediction for this plan (1000 steps), GCell/s
    int tuned = 0;        // configuration taken from the tuning cache
    PassCfg2D traj;       // trajectory passes (stencil_run_trajectory)
    float *src = nullptr;   // contracted float32 Hotspot 2D: the source map sdc*(p + amb*Rz)
    long long ld_src = 0;   // its row pitch, floats
    int ntx_star = 0, nty_star = 0;   // star diffusion (rad > 1): tiles along x and y
    int nseg_star = 1, zseg_star = 0; // 3D star: z-segments per tile column, their length
    std::vector<PassCfg3D> cfg3;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // pairs, reused
    size_t ev_used = 0;
    double ms_acc = 0.0;
    long long launches = 0;
    int sticky = ST_OK;
    // 16-bit storage (2D contracted plans): ping-pong grids and block codes, coded power map
    int stor = 0;
    long long ld_q = 0;
    int cx = 0, ntx = 0;
    void *q[2] = {nullptr, nullptr};
    float2 *qm[2] = {nullptr, nullptr};
    void *qp = nullptr;
    float2 *qpm = nullptr;
    // resident tiles (2D): the whole grid on chip for the run, one cooperative launch
    int res = 0, res_vx = 4, res_nw = 0, res_nbx = 0, res_nby = 0, res_cw = 0, res_ch = 0, res_hx = 0;
    float *res_xg = nullptr;      // two exchange grids, rows of res_ld floats
    long long res_ld = 0;
    int *res_flags = nullptr;     // per block: epochs published (grow across runs)
    int res_epoch = 0;            // epoch base of the next run
    long long res_wait_ns = 1000000000LL;
    int res_hold_block = -1, res_hold_epoch = -1;
};

namespace {

const int kTcand[] = {1, 2, 3, 4, 6, 8, 12, 16};

int map_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return ST_OK;
    if (e == cudaErrorMemoryAllocation) return ST_ERR_OOM;
    return ST_ERR_CUDA;
}

long long cells_of(const stencil_desc &d) { return (long long)d.nx * d.ny * d.nz; }

int ncoef(const stencil_desc &d)
{
    if (d.kind == ST_DIFFUSION_VAR) return 0;   // per-cell coefficient planes on the device
    if (d.rad > 1) return 1 + (d.ndim == 2 ? 4 : 6) * d.rad;
    if (d.ndim == 2) return 5;
    return d.kind == ST_DIFFUSION ? 7 : 9;
}

bool stor_src_bits(int stor) { return (stor & STOR_SRC) != 0; }

// storage bits of a plan's 2D kernel shape: the format, plus STOR_SRC for contracted Hotspot
// kernels (they stage p + amb*Rz instead of the power map)
int shape_stor(const stencil_plan_s *p)
{
    return p->stor | ((p->d.kind == ST_THERMAL && !p->d.exact) ? STOR_SRC : 0);
}

bool available(const stencil_plan_s *p, int T)
{
    if (p->d.ndim == 2)
        return tb2d_available(Shape2D{p->d.kind, p->d.exact ? 1 : 0, T, p->V, p->W, shape_stor(p)});
    return tb3d_available(Shape3D{p->d.kind, p->d.exact ? 1 : 0, T, p->VY, p->NW, p->alg3, p->VX3});
}

// ---- parameter choice seeded by the GPU restatement of the paper's model (Eqs. 3-9) -------
//
// Calibration (GB300 ncu counts of the contracted 2D kernels): each stage issues its Table 2
// operations (5 Diffusion, 9 Hotspot per cell) plus ~4 per thread (2 shuffles, power loads,
// addressing), each row ~100 more per thread (waits, copies, ring and pointer updates); issue
// efficiency grows with resident warps (0.69 at 8, 0.77 at 12 per SM); a hot loop beyond ~12 KB
// of code loses issue rate in proportion (instruction-cache misses); these kernels reach ~62 %
// of the measured copy bandwidth when they are memory-bound; every row segment streams 2T rows
// more than it stores, which dominates on small grids cut into many short segments.  With these factors the model
// ranks the compiled variants as measured on 16384^2 grids at T in {4, 6, 8, 12}.
struct Cand2D { int T, V, W; };

// seg_rows = 0: the plan's own launch geometry; > 0: a batch launch, whose segments hold about
// seg_rows rows across all its grids and whose launch cost the grids share
double model_gcells_2d(const stencil_desc &d, int sms, const Cand2D &k, int bps, int steps,
                       int seg_rows = 0)
{
    const bool swap = k.W == 1;
    const double fp = d.kind == ST_DIFFUSION ? 5.0 : 6.0;   // Hotspot: the expanded weights
    const double ops = fp + 4.0 / k.V + 100.0 / (k.T * k.V);
    const double code_kb = (swap ? 2.0 : 1.0) * k.T * (k.V * fp + 6.0) * 16.0 / 1024.0;
    // the launch geometry of prepare2: one-warp blocks over (tile column, row) units in
    // segments of at least 4 rows; each segment streams 2T extra rows (Sec. 3.2's pipeline
    // fill and drain), and a small grid leaves SMs with fewer resident warps
    const int halo = (k.T + 3) / 4 * 4;
    const long long cx = 32LL * k.V - 2 * halo;
    const long long units = (d.nx + cx - 1) / cx * (long long)d.ny;
    const long long ctas = std::min<long long>((long long)sms * bps, std::max<long long>(1, units / 4));
    const double rows_per_cta = seg_rows > 0 ? seg_rows : (double)units / ctas;
    const int warps = seg_rows > 0 ? std::min(bps, 16)
                                   : (int)std::min<long long>(std::min(bps, 16), (ctas + sms - 1) / sms);
    double eff = std::min(0.85, 0.45 + 0.027 * warps);
    if (code_kb > 12.0) eff *= 12.0 / code_kb;
    stencil_gpu_model_in m = {};
    m.ndim = 2;
    m.nx = d.nx;
    m.ny = d.ny;
    m.nz = 1;
    m.steps = steps > 0 ? steps : 1000;
    m.T = k.T;
    m.bx = 32 * k.V;
    m.halo_x = (k.T + 3) / 4 * 4;
    m.sms = sms;
    m.sm_hz = 2.07e9;
    m.hbm_gbs = 6800.0;
    m.bytes_per_cell = d.kind == ST_DIFFUSION ? 8.0 : 12.0;
    m.ops_per_cell = ops;
    m.issue_eff = eff;
    m.hbm_eff = 0.62;
    m.stream_overhead = 2.0 * k.T / rows_per_cta;
    m.launch_s = seg_rows > 0 ? 0.0 : 4e-6;
    stencil_gpu_model_out r;
    if (stencil_model_gpu(&m, &r) != ST_OK) return 0.0;
    return r.gcells;
}

// 3D partial-sum kernel: the same restatement.  Issued work: 17.3 (Diffusion) and 19.7
// (Hotspot) thread instructions per computed cell update including halos (ncu counts of the
// 512^3 and 512^2 x 256 runs with 2 x 4 cells per thread at T = 4), x(0.85 + 0.6/T) for the
// costlier first stage.  Issue efficiency 0.61 for one
// 16-warp block per SM, x1.10 for two 8-warp blocks (they wait at fewer barriers together),
// x0.80 for 32-warp blocks of 2 x 2 cells (twice the y exchange per cell).  Device memory: the
// tiles read their halos again (the tile fit's read factor, ntx*bx*nty*by / (nx*ny)), at 62 %
// of the measured copy bandwidth.  Calibrated on the 50-point sweep of bench.py --model-study
// (measured / predicted per configuration).
// 3D segments (tb3f): the z-slab length Z of round-robin (tile column, z-slab) pieces, or 0 for
// contiguous (tile column, plane) ranges.  Pieces read the tiles' halo planes from L2 and cut
// the pass's DRAM traffic to about the algorithmic bytes (ranges: 1.4-1.6x), which pays only
// where the pass is memory-bound: measured on GB300, T = 1 (512^3 diffusion: 578 GCell/s with
// pieces, 431 with ranges); from T = 2 on the kernel is issue-bound and the cost-balanced
// ranges are faster (T = 3: 963 against 935).  So pieces for T = 1, when their rounds cost at
// most 6 % more plane-times per block (planes plus T of pipeline fill per segment) than the
// ranges; *cost receives the chosen mode's plane-times per block.
int zslab_pick(long long cols, int nz, long long slots, int T, double *cost)
{
    const long long total = cols * nz;
    const long long ctas = std::min(slots, std::max<long long>(1, total / std::max(16, 8 * T)));
    const double range_cost = (double)((total + ctas - 1) / ctas) + T;
    double best = 0.0;
    int best_z = 0;
    for (int S = 1; S <= std::max(1, nz / (2 * T)); S++) {
        const int Z = (nz + S - 1) / S;
        const long long pieces = cols * ((nz + Z - 1) / Z);
        const long long G = std::min(slots, pieces);
        const double c = (double)((pieces + G - 1) / G) * (Z + T);
        if (!best_z || c < best) {
            best = c;
            best_z = Z;
        }
    }
    if (T == 1 && best_z > 0 && best <= 1.06 * range_cost) {
        if (cost) *cost = best;
        return best_z;
    }
    if (cost) *cost = range_cost;
    return 0;
}

double model_gcells_3d(const stencil_desc &d, int sms, int T, int VX, int VY, int NW)
{
    stencil_gpu_model_in m = {};
    m.ndim = 3;
    m.nx = d.nx;
    m.ny = d.ny;
    m.nz = d.nz;
    m.steps = 1000;
    m.T = T;
    m.bx = 32 * VX;
    m.by = VY * NW;
    m.halo_x = (T + 3) / 4 * 4;
    m.halo_y = T;
    m.sms = sms;
    m.sm_hz = 2.07e9;
    m.hbm_gbs = 6800.0;
    const double cx = m.bx - 2.0 * m.halo_x, cy = m.by - 2.0 * m.halo_y;
    if (cx < 1 || cy < 1) return 0.0;
    const long long cols = (long long)std::ceil(d.nx / cx) * (long long)std::ceil(d.ny / cy);
    double rf = std::ceil(d.nx / cx) * m.bx * std::ceil(d.ny / cy) * m.by / ((double)d.nx * d.ny);
    // the segments prepare3 will take: z-slab pieces read their halos again from L2, not DRAM
    const long long slots = (long long)sms * (NW <= 8 ? 2 : 1);
    double seg_cost = 0.0;
    const bool pieces = zslab_pick(cols, d.nz, slots, T, &seg_cost) > 0;
    if (pieces) rf = 1.0;
    const double alg = d.kind == ST_DIFFUSION ? 8.0 : 12.0;
    const double read = alg - 4.0;   // field (and power) in; the field out is written once
    m.bytes_per_cell = alg;
    m.hbm_eff = 0.62 * alg / (read * rf + 4.0);
    // stage 0 (three ring planes, their exchange) costs more than the partial-sum stages
    // (recalibrated after interior tile columns dropped the clamp fix-ups: measured / model
    // over the 3D configurations of the accuracy study was 1.11 (diffusion), 1.07 (Hotspot))
    m.ops_per_cell = (d.kind == ST_DIFFUSION ? 16.0 : 18.6) * (0.85 + 0.6 / T);
    m.issue_eff = 0.61 * (NW <= 8 ? 1.10 : NW >= 32 ? 0.80 : 1.0);
    // plane-times per block beyond an even share of the planes (fill, round quantisation)
    m.stream_overhead = pieces ? std::max(0.0, seg_cost * slots / ((double)cols * d.nz) - 1.0) : 0.04;
    m.launch_s = 4e-6;
    stencil_gpu_model_out r;
    if (stencil_model_gpu(&m, &r) != ST_OK) return 0.0;
    return r.gcells;
}

}  // namespace

namespace stn {
// the batch's (T, V) choice uses the same calibrated model; seg_rows: rows per queue item (each
// item streams 2T rows more than it stores)
double batch_model_gcells(int kind, int nx, int ny, int steps, int sms, int T, int V, int bps,
                          int seg_rows)
{
    stencil_desc d = {};
    d.kind = kind;
    d.ndim = 2;
    d.nx = nx;
    d.ny = ny;
    d.nz = 1;
    return model_gcells_2d(d, sms, Cand2D{T, V, 1}, bps, steps, std::min(seg_rows, ny));
}
}  // namespace stn

namespace {

// ---- resident tiles (res2d.cu) ---------------------------------------------------------------
// A 2D grid that fits the co-resident blocks is held on chip for the whole run; the chosen
// (T, cells per thread, block rows) minimises the same kind of restated run time as Eqs. 3-9:
//   t(steps) = steps * t_step + (epochs - 1) * t_x + t_launch + t_io,
//   t_step   = (cells held per SM) * ops / (issue rate of an SM) + t_bar,
// a cell held being one of a tile incl. its halos (Sec. 3.2's redundant compute), ops the issued
// thread instructions per cell and step (the Table 2 operations, the shuffles of the lane edges,
// the row exchange between warps, loop overhead), t_bar the per-step barrier of that exchange,
// t_x one exchange through L2 after every T steps (publish, neighbour wait, halo reload), t_io
// the single read and write of the grid.  Calibrated on GB300: first by least squares over 93
// measured configurations of 512^2 and 1024^2 grids (T = 1..16, 2 and 4 cells per lane, both
// kinds, exact and contracted); then, after the step loop was unrolled and the x-edge work split
// by edge, on the step loops' clock64 cycles and the run times of 1024^2 at T = 12..20 (both
// kinds, exact and contracted, within 0.9-1.05): issue efficiency 0.73, t_x = 7.8 us, and two
// more operations per cell for exact plans (Table 2 order, no fused multiply-adds).
struct ResGeom {
    int T = 0, vx = 0, nw = 0, nbx = 0, nby = 0, cw = 0, ch = 0, hx = 0;
    double t = 0.0;   // predicted seconds for 1000 steps
};

double res_time(const stencil_desc &d, int sms, const ResGeom &g, int steps)
{
    const int VY = res2d_rows_per_thread();
    const double per_sm = std::ceil((double)g.nbx * g.nby / sms);
    const double cells = per_sm * g.nw * 32.0 * g.vx * VY;
    double fp = d.kind == ST_DIFFUSION ? 5.0 : 6.0;
    if (d.exact) fp = d.kind == ST_DIFFUSION ? 11.0 : 15.0;
    const double ops = fp + 2.0 / g.vx + 4.0 / (g.vx * VY) + 1.0;
    const double t_step = cells * ops / (128.0 * 0.73 * 2.07e9) + 0.1e-6;
    const double t_x = 7.8e-6;
    const int epochs = (steps + g.T - 1) / g.T;
    return steps * t_step + (epochs - 1) * t_x + 5e-6 + (double)d.nx * d.ny * 8.0 / 6.8e12;
}

// The fastest resident geometry with T steps per exchange and vx cells per thread along x;
// false when the grid does not fit the co-resident blocks of the device.
bool res_geometry(const stencil_desc &d, int sms, int T, int vx, ResGeom *out)
{
    const int kind = d.kind;
    if (T < 1 || !res2d_available(kind, d.exact, vx)) return false;
    const int VY = res2d_rows_per_thread(), maxw = res2d_max_warps(kind, d.exact, vx);
    const int hx = (T + vx - 1) / vx * vx, hy = T;   // x-halo a multiple of vx: x = 0 is a cell 0
    const int cw = 32 * vx - 2 * hx;
    if (cw < 1) return false;
    const int nbx = (d.nx + cw - 1) / cw;
    if (nbx > 1 && cw < hx) return false;   // a halo must not reach past the next block
    std::vector<int> bps(maxw + 1, 0);
    bool found = false;
    ResGeom best;
    for (int nby = 1; nby <= d.ny; nby++) {
        const int ch = (d.ny + nby - 1) / nby;
        if (nby > 1 && ch < hy) break;
        if ((long long)(nby - 1) * ch >= d.ny) continue;   // the last block would be empty
        const int nw = (ch + 2 * hy + VY - 1) / VY;
        if (nw > maxw) continue;
        if (!bps[nw]) {
            int b = 0;
            if (res2d_occupancy(kind, d.exact, vx, nw, &b) != cudaSuccess) {
                (void)cudaGetLastError();
                b = 0;
            }
            bps[nw] = b > 0 ? b : -1;
        }
        if (bps[nw] < 1 || (long long)nbx * nby > (long long)sms * bps[nw]) continue;
        ResGeom g;
        g.T = T;
        g.vx = vx;
        g.nw = nw;
        g.nbx = nbx;
        g.nby = nby;
        g.cw = cw;
        g.ch = ch;
        g.hx = hx;
        g.t = res_time(d, sms, g, 1000);
        if (!found || g.t < best.t) {
            best = g;
            found = true;
        }
    }
    if (found) *out = best;
    return found;
}

// the best resident geometry over the compiled cells per thread and the candidate T (forced
// values restrict the search)
bool res_choose(const stencil_desc &d, int sms, ResGeom *out)
{
    bool found = false;
    for (int vx : {2, 4}) {
        if (d.force_vec && d.force_vec != vx) continue;
        for (int t : {1, 2, 3, 4, 6, 8, 12, 16, 20, 24, 32}) {
            if (d.force_T && t != d.force_T) continue;
            ResGeom g;
            if (res_geometry(d, sms, t, vx, &g) && (!found || g.t < out->t)) {
                *out = g;
                found = true;
            }
        }
        if (d.force_T && !found) {   // a forced T outside the list above
            ResGeom g;
            if (res_geometry(d, sms, d.force_T, vx, &g) && (!found || g.t < out->t)) {
                *out = g;
                found = true;
            }
        }
    }
    return found;
}

// smallest compiled kernel T >= want for the plan's family (or the largest compiled one)
int kernel_T_for(const stencil_plan_s *p, int want)
{
    int best = 0;
    for (int t : kTcand) {
        if (!available(p, t)) continue;
        if (t >= want) return t;
        best = t;
    }
    return best;
}

int prepare2(stencil_plan_s *p, int Tk, PassCfg2D **out)
{
    if ((int)p->cfg2.size() <= Tk) p->cfg2.resize(Tk + 1);
    PassCfg2D &c = p->cfg2[Tk];
    if (!c.ready) {
        c.shape = Shape2D{p->d.kind, p->d.exact ? 1 : 0, Tk, p->V, p->W, shape_stor(p)};
        if (!tb2d_available(c.shape)) return ST_ERR_UNSUPPORTED;
        int bps = 0;
        cudaError_t e = tb2d_prepare(c.shape, &bps);
        if (e != cudaSuccess) return map_cuda(e);
        if (bps < 1) return ST_ERR_UNSUPPORTED;
        const int bx = tb2d_tile_width(c.shape), h = tb2d_halo(c.shape);
        const int cx = bx - 2 * h;
        c.ntx = (p->d.nx + cx - 1) / cx;
        c.total = (long long)c.ntx * p->d.ny;
        // each block streams at least ~8T rows so the y-halo (2T rows per segment) stays small
        const long long min_rows = 4;   // short segments keep small grids parallel
        long long ctas = std::min<long long>((long long)p->sms * bps,
                                             std::max<long long>(1, c.total / min_rows));
        c.rows_per_cta = (c.total + ctas - 1) / ctas;
        c.ctas = (int)((c.total + c.rows_per_cta - 1) / c.rows_per_cta);
        if (!c.shape.exact && c.shape.kind != ST_DIFFUSION_VAR) {
            // contracted kernel: cost-balanced ranges where they shorten the longest block
            std::vector<long long> st;
            const int fill = 2 * Tk;
            // a row of an edge tile column costs 1.25: its warps run the clamp selects
            // (measured on GB300 with the edge weight swept 1.0-1.4: 16384^2 Hotspot 2684 ->
            // 2948 GCell/s, diffusion 3337 -> 3753, flat between 1.2 and 1.4)
            std::vector<double> w(c.ntx, 1.0);
            w.front() = w.back() = 1.25;
            if (balanced_ranges(p->d.ny, (int)ctas, fill, w, st) <
                even_ranges_cost(p->d.ny, c.rows_per_cta, fill, w)) {
                e = stn::dev_malloc(&c.starts, st.size() * sizeof(long long));
                if (e == cudaSuccess)
                    e = cudaMemcpy(c.starts, st.data(), st.size() * sizeof(long long), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    if (c.starts) stn::dev_free(c.starts);
                    c.starts = nullptr;
                    return map_cuda(e);
                }
                c.ctas = (int)ctas;
            }
        }
        c.ready = true;
    }
    *out = &c;
    return ST_OK;
}

// Trajectory passes run the in-place T = 8, V = 8 contracted kernel that also writes every
// fused step; same launch geometry rules as the plan's own passes.
constexpr int kTrajT = 8;

int prepare_traj(stencil_plan_s *p, PassCfg2D **out)
{
    PassCfg2D &c = p->traj;
    if (!c.ready) {
        c.shape = Shape2D{p->d.kind, 0, kTrajT, 8, 0,
                          (p->d.kind == ST_THERMAL ? (int)STOR_SRC : 0) | (int)STOR_ALL};
        if (!tb2d_available(c.shape)) return ST_ERR_UNSUPPORTED;
        int bps = 0;
        cudaError_t e = tb2d_prepare(c.shape, &bps);
        if (e != cudaSuccess) return map_cuda(e);
        if (bps < 1) return ST_ERR_UNSUPPORTED;
        const int cx = tb2d_tile_width(c.shape) - 2 * tb2d_halo(c.shape);
        c.ntx = (p->d.nx + cx - 1) / cx;
        c.total = (long long)c.ntx * p->d.ny;
        const long long ctas = std::min<long long>((long long)p->sms * bps,
                                                   std::max<long long>(1, c.total / 4));
        c.rows_per_cta = (c.total + ctas - 1) / ctas;
        c.ctas = (int)((c.total + c.rows_per_cta - 1) / c.rows_per_cta);
        c.ready = true;
    }
    *out = &c;
    return ST_OK;
}

int prepare3(stencil_plan_s *p, int Tk, PassCfg3D **out)
{
    if ((int)p->cfg3.size() <= Tk) p->cfg3.resize(Tk + 1);
    PassCfg3D &c = p->cfg3[Tk];
    if (!c.ready) {
        c.shape = Shape3D{p->d.kind, p->d.exact ? 1 : 0, Tk, p->VY, p->NW, p->alg3, p->VX3};
        if (!tb3d_available(c.shape)) return ST_ERR_UNSUPPORTED;
        int bps = 0;
        cudaError_t e = tb3d_prepare(c.shape, &bps);
        if (e != cudaSuccess) return map_cuda(e);
        if (bps < 1) return ST_ERR_UNSUPPORTED;
        const int hx = (Tk + 3) / 4 * 4, hy = Tk;
        const int cx = 32 * p->VX3 - 2 * hx, cy = p->VY * p->NW - 2 * hy;
        c.ntx = (p->d.nx + cx - 1) / cx;
        c.nty = (p->d.ny + cy - 1) / cy;
        c.cols = (long long)c.ntx * c.nty;
        const long long total = c.cols * p->d.nz;
        const long long min_planes = std::max(16, 8 * Tk);
        long long ctas = std::min<long long>((long long)p->sms * bps,
                                             std::max<long long>(1, total / min_planes));
        c.planes_per_cta = (total + ctas - 1) / ctas;
        c.ctas = (int)((total + c.planes_per_cta - 1) / c.planes_per_cta);
        if (p->alg3) {
            // or pieces (tile column, z-slab) dealt round-robin (zslab_pick): the blocks of a
            // round stream neighbouring tile columns through the same planes together, so the
            // halo cells a tile reads again come from L2 (with contiguous ranges the neighbours
            // run far apart in z and every tile reads its halos from device memory: measured
            // on 512^2 x 256 diffusion, T = 3, DRAM bytes per pass 751 MB with ranges, 504 MB
            // with 52-plane pieces, 537 MB algorithmic).
            const long long slots = (long long)p->sms * bps;
            const int best_z = zslab_pick(c.cols, p->d.nz, slots, Tk, nullptr);
            // a plane of a tile column at the x edge costs 1.2, at the y edge 1.1 (only those
            // columns run the kernel instance with the clamp fix-ups; measured on GB300,
            // weights swept 1.0-1.45, T = 3: 512^3 diffusion 923 -> 1027 GCell/s, 512^2 x 256
            // Hotspot 752 -> 838)
            const double wx = 1.2, wy = 1.1;
            std::vector<double> w(c.cols, 1.0);
            for (long long col = 0; col < c.cols; col++) {
                const long long ty = col / c.ntx, tx = col - ty * c.ntx;
                if (tx == 0 || tx == c.ntx - 1) w[col] *= wx;
                if (ty == 0 || ty == c.nty - 1) w[col] *= wy;
            }
            if (best_z > 0) {
                c.zslab = best_z;
                c.pieces = c.cols * ((p->d.nz + best_z - 1) / best_z);
                c.ctas = (int)std::min(slots, c.pieces);
            } else {
                // contiguous ranges balanced by cost: edge tile columns weigh more
                std::vector<long long> st;
                if (balanced_ranges(p->d.nz, (int)ctas, Tk, w, st) <
                    even_ranges_cost(p->d.nz, c.planes_per_cta, Tk, w)) {
                    e = stn::dev_malloc(&c.starts, st.size() * sizeof(long long));
                    if (e == cudaSuccess)
                        e = cudaMemcpy(c.starts, st.data(), st.size() * sizeof(long long), cudaMemcpyHostToDevice);
                    if (e != cudaSuccess) {
                        if (c.starts) stn::dev_free(c.starts);
                        c.starts = nullptr;
                        return map_cuda(e);
                    }
                    c.ctas = (int)ctas;
                }
            }
        }
        c.ready = true;
    }
    *out = &c;
    return ST_OK;
}

bool ranges_overlap(const void *a, const void *b, size_t n)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
}

// [a, a + na) and [b, b + nb) share a byte
bool ranges_overlap2(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

bool stable(const stencil_desc &d, const float *k)
{
    const double eps = 1e-6;
    for (int i = 0; i < ncoef(d); i++)
        if (!std::isfinite(k[i])) return false;
    if (d.kind == ST_DIFFUSION) {
        double s = 0;
        for (int i = 0; i < ncoef(d); i++) {
            if (k[i] < 0) return false;
            s += k[i];
        }
        return s <= 1.0 + eps;
    }
    if (d.ndim == 2) {
        const double kdt = k[0], rx = k[1], ry = k[2], rz = k[3];
        if (kdt < 0 || rx < 0 || ry < 0 || rz < 0) return false;
        return kdt * (2 * rx + 2 * ry + rz) <= 1.0 + eps;
    }
    for (int i = 0; i < 8; i++)
        if (k[i] < 0) return false;
    return true;
}

cudaError_t record(stencil_plan_s *p, bool begin)
{
    if (!p->timing) return cudaSuccess;
    if (begin && p->ev_used + 2 > p->ev.size()) {
        for (int i = 0; i < 64; i++) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            p->ev.push_back(e);
        }
    }
    cudaError_t err = cudaEventRecord(p->ev[p->ev_used], p->stream);
    p->ev_used++;
    return err;
}

int flush_timing(stencil_plan_s *p)
{
    if (p->ev_used == 0) return ST_OK;
    cudaError_t e = cudaEventSynchronize(p->ev[p->ev_used - 1]);
    if (e != cudaSuccess) return map_cuda(e);
    for (size_t i = 0; i + 1 < p->ev_used; i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]);
        if (e != cudaSuccess) return map_cuda(e);
        p->ms_acc += ms;
        p->launches++;
    }
    p->ev_used = 0;
    return ST_OK;
}

// traj (trajectory passes): its configuration, and where the pass's intermediate steps go
int run_pass2(stencil_plan_s *p, const float *src, long long lds, float *dst, long long ldd,
              const float *pw, const float *k, int tsteps, PassCfg2D *traj = nullptr,
              float *states = nullptr, long long stride = 0)
{
    PassCfg2D *c = traj;
    int rc = traj ? ST_OK : prepare2(p, kernel_T_for(p, tsteps), &c);
    if (rc != ST_OK) return rc;
    Pass2D a = {};
    a.states = states;
    a.state_stride = stride;
    a.in = src;
    a.out = dst;
    a.pw = pw;
    a.ld_in = lds;
    a.ld_out = ldd;
    a.ld_pw = (p->src && pw == p->src) ? p->ld_src : p->d.nx;
    a.pw_plane = (long long)p->d.nx * p->d.ny;   // per-cell coefficient planes, dense
    a.nx = p->d.nx;
    a.ny = p->d.ny;
    a.tsteps = tsteps;
    a.ntx = c->ntx;
    a.total_rows = c->total;
    a.rows_per_cta = c->rows_per_cta;
    a.starts = c->starts;
    a.ctas = c->ctas;
    for (int i = 0; i < 5; i++) a.k[i] = a.kf[i] = k[i];
    a.kf[5] = k[0] * k[2];    // Hotspot: sdc * Ry, rounded once (float32)
    a.kf[6] = -2.0f * k[2];   // Hotspot: -2 Ry (exact)
    if (stor_src_bits(c->shape.stor)) hot_coeffs_src(k, a.kf);
    a.vec_in = ((uintptr_t)src % 16 == 0) && (lds % 4 == 0);
    a.vec_out = ((uintptr_t)dst % 16 == 0) && (ldd % 4 == 0) &&
                (!states || ((uintptr_t)states % 16 == 0 && stride % 4 == 0));
    a.vec_pw = pw ? (((uintptr_t)pw % 16 == 0) && (a.ld_pw % 4 == 0)) : 0;
    if (p->timing && p->ev_used + 2 > 2 * 1024) {
        rc = flush_timing(p);
        if (rc != ST_OK) return rc;
    }
    cudaError_t e = record(p, true);
    if (e == cudaSuccess) e = tb2d_launch(c->shape, a, p->stream);
    if (e == cudaSuccess) e = record(p, false);
    return map_cuda(e);
}

// a run of a resident-tile plan: one cooperative launch (after zeroing the blocks' epoch
// counters)
int run_resident(stencil_plan_s *p, const float *in, float *out, const float *pw, const float *k,
                 int steps)
{
    const stencil_desc &d = p->d;
    Res2D a = {};
    a.in = in;
    a.ld_in = d.nx;
    a.out = out;
    cudaError_t e = cudaSuccess;
    const int epochs = (steps + p->T - 1) / p->T;
    if (in == out && epochs == 1) {
        // in place with no exchange between the blocks' first read and last write: a block
        // could overwrite cells a neighbour has yet to read, so the run reads a copy (in the
        // exchange grids, unused by a single epoch)
        float *cp = p->res_xg;
        e = cudaMemcpy2DAsync(cp, (size_t)p->res_ld * sizeof(float), in, (size_t)d.nx * sizeof(float),
                              (size_t)d.nx * sizeof(float), d.ny, cudaMemcpyDeviceToDevice, p->stream);
        if (e != cudaSuccess) return map_cuda(e);
        a.in = cp;
        a.ld_in = p->res_ld;
    }
    a.aux = pw;
    a.ld_aux = d.nx;
    a.xg = p->res_xg;
    a.xplane = p->res_ld * d.ny;
    a.ld_x = p->res_ld;
    if (epochs > 1) {
        if (p->res_epoch > 0x7fffffff - epochs) {
            // the counters would overflow: start again from zero
            e = cudaMemsetAsync(p->res_flags, 0, (size_t)p->res_nbx * p->res_nby * sizeof(int), p->stream);
            if (e != cudaSuccess) return map_cuda(e);
            p->res_epoch = 0;
        }
        a.epoch0 = p->res_epoch;
        p->res_epoch += epochs;
    }
    a.flags = p->res_flags;
    a.status = p->err;
    a.wait_ns = p->res_wait_ns;
    a.hold_block = p->res_hold_block;
    a.hold_epoch = p->res_hold_epoch;
    a.nx = d.nx;
    a.ny = d.ny;
    a.steps = steps;
    a.T = p->T;
    a.nbx = p->res_nbx;
    a.nby = p->res_nby;
    a.cw = p->res_cw;
    a.ch = p->res_ch;
    a.hx = p->res_hx;
    a.hy = p->T;
    if (d.kind == ST_THERMAL && !d.exact) {
        // the expanded weights cc, cx, cy, cz of the contracted Hotspot kernels
        float kf[7];
        hot_coeffs_src(k, kf);
        for (int i = 0; i < 4; i++) a.k[i] = kf[i];
        a.src_sdc = k[0];
        a.src_a = k[4] * k[3];   // amb * Rz, rounded once
    } else {
        for (int i = 0; i < 5; i++) a.k[i] = k[i];
    }
    if (p->timing && p->ev_used + 2 > 2 * 1024) {
        const int rc = flush_timing(p);
        if (rc != ST_OK) return rc;
    }
    e = record(p, true);
    if (e == cudaSuccess)
        e = res2d_launch(d.kind, d.exact, p->res_vx, p->res_nw, a,
                         p->stream);
    if (e == cudaSuccess) e = record(p, false);
    return map_cuda(e);
}

// one pass of a 16-bit plan: coded grid q[src] -> q[dst], always the plan's T kernel (the
// trailing stages forward when tsteps < T), so the block codes keep the plan's tiling
int run_pass2q(stencil_plan_s *p, int src, int dst, const float *k, int tsteps)
{
    PassCfg2D *c = nullptr;
    int rc = prepare2(p, p->T, &c);
    if (rc != ST_OK) return rc;
    Pass2D a = {};
    a.nx = p->d.nx;
    a.ny = p->d.ny;
    a.tsteps = tsteps;
    a.ntx = c->ntx;
    a.total_rows = c->total;
    a.rows_per_cta = c->rows_per_cta;
    a.starts = c->starts;
    a.ctas = c->ctas;
    for (int i = 0; i < 5; i++) a.k[i] = a.kf[i] = k[i];
    a.kf[5] = k[0] * k[2];
    a.kf[6] = -2.0f * k[2];
    if (stor_src_bits(c->shape.stor)) hot_coeffs_src(k, a.kf);
    a.vec_in = a.vec_out = a.vec_pw = 1;
    a.stor = p->stor;
    a.qin = p->q[src];
    a.qout = p->q[dst];
    a.min_ = p->qm[src];
    a.mout = p->qm[dst];
    a.qpw = p->qp;
    a.mpw = p->qpm;
    a.ld_q = p->ld_q;
    cudaError_t e = record(p, true);
    if (e == cudaSuccess) e = tb2d_launch(c->shape, a, p->stream);
    if (e == cudaSuccess) e = record(p, false);
    return map_cuda(e);
}

int run_pass_star3(stencil_plan_s *p, const float *src, float *dst, const float *k, int tsteps)
{
    PassStar3D a = {};
    a.in = src;
    a.out = dst;
    a.nx = p->d.nx;
    a.ny = p->d.ny;
    a.nz = p->d.nz;
    a.tsteps = tsteps;
    a.ntx = p->ntx_star;
    a.nty = p->nty_star;
    a.nseg = p->nseg_star;
    a.zseg = p->zseg_star;
    for (int i = 0; i < ncoef(p->d) && i < 25; i++) a.k[i] = k[i];
    a.vec_out = ((uintptr_t)dst % 16 == 0) && (p->d.nx % 4 == 0);
    a.err = p->err;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof(tm));
    a.use_tma = tma3d_encode(&tm, src, p->d.nx, p->d.ny, p->d.nz, 64, 64) ? 1 : 0;
    if (p->timing && p->ev_used + 2 > 2 * 1024) {
        const int rc = flush_timing(p);
        if (rc != ST_OK) return rc;
    }
    cudaError_t e = record(p, true);
    if (e == cudaSuccess) e = star3d_launch(p->d.rad, p->d.exact, p->T, a, tm, p->stream);
    if (e == cudaSuccess) e = record(p, false);
    return map_cuda(e);
}

int run_pass_star(stencil_plan_s *p, const float *src, float *dst, const float *k, int tsteps)
{
    if (p->d.ndim == 3) return run_pass_star3(p, src, dst, k, tsteps);
    PassStar2D a = {};
    a.in = src;
    a.out = dst;
    a.ld_in = p->d.nx;
    a.ld_out = p->d.nx;
    a.nx = p->d.nx;
    a.ny = p->d.ny;
    a.tsteps = tsteps;
    a.ntx = p->ntx_star;
    a.nty = p->nty_star;
    for (int i = 0; i < ncoef(p->d) && i < 17; i++) a.k[i] = k[i];
    a.vec_out = ((uintptr_t)dst % 16 == 0) && (p->d.nx % 4 == 0);
    a.err = p->err;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof(tm));
    a.use_tma = tma3d_encode(&tm, src, p->d.nx, p->d.ny, 1, 128, 128) ? 1 : 0;
    if (p->timing && p->ev_used + 2 > 2 * 1024) {
        const int rc = flush_timing(p);
        if (rc != ST_OK) return rc;
    }
    cudaError_t e = record(p, true);
    if (e == cudaSuccess) e = star2d_launch(p->d.rad, p->d.exact, p->T, a, tm, p->stream);
    if (e == cudaSuccess) e = record(p, false);
    return map_cuda(e);
}

int run_pass3(stencil_plan_s *p, const float *src, float *dst, const float *pw, const float *k,
              int tsteps)
{
    PassCfg3D *c = nullptr;
    int rc = prepare3(p, kernel_T_for(p, tsteps), &c);
    if (rc != ST_OK) return rc;
    Pass3D a;
    a.in = src;
    a.out = dst;
    a.pw = pw;
    a.nx = p->d.nx;
    a.ny = p->d.ny;
    a.nz = p->d.nz;
    a.tsteps = tsteps;
    a.ntx = c->ntx;
    a.nty = c->nty;
    a.total_cols = c->cols;
    a.planes_per_cta = c->planes_per_cta;
    a.ctas = c->ctas;
    a.zslab = c->zslab;
    a.pieces = c->pieces;
    a.starts = c->starts;
    for (int i = 0; i < 9; i++) a.k[i] = i < ncoef(p->d) ? k[i] : 0.f;
    a.vec = ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0) && (p->d.nx % 4 == 0);
    a.vec_pw = pw && ((uintptr_t)pw % 16 == 0) && (p->d.nx % 4 == 0);
    a.err = p->err;
    a.use_tma = 0;
    Tma3D tm;
    std::memset(&tm, 0, sizeof(tm));
    if (p->alg3 && a.vec) {
        const int bx = 32 * p->VX3, by = p->VY * p->NW;
        bool ok = tma3d_encode(&tm.in, src, p->d.nx, p->d.ny, p->d.nz, bx, by);
        if (ok && pw) ok = a.vec_pw && tma3d_encode(&tm.pw, pw, p->d.nx, p->d.ny, p->d.nz, bx, by);
        a.use_tma = ok ? 1 : 0;
    }
    if (p->timing && p->ev_used + 2 > 2 * 1024) {
        rc = flush_timing(p);
        if (rc != ST_OK) return rc;
    }
    cudaError_t e = record(p, true);
    if (e == cudaSuccess) e = tb3d_launch(c->shape, a, tm, p->stream);
    if (e == cudaSuccess) e = record(p, false);
    return map_cuda(e);
}

}  // namespace

extern "C" {

int stencil_abi_version(void) { return ST_ABI_VERSION; }

const char *stencil_strerror(int code)
{
    switch (code) {
    case ST_OK: return "ok";
    case ST_ERR_INVALID_ARG: return "invalid argument";
    case ST_ERR_DIMS_MISMATCH: return "grid dimensions differ from the plan's";
    case ST_ERR_UNSTABLE_COEFFS: return "coefficients violate the explicit stability bound";
    case ST_ERR_CUDA: return "CUDA runtime error";
    case ST_ERR_OOM: return "device memory allocation failed";
    case ST_ERR_TIMEOUT: return "bounded device wait timed out";
    case ST_ERR_UNSUPPORTED: return "unsupported parameter combination";
    case ST_ERR_TOO_LARGE: return "grid larger than the allocation-free entry point's fixed buffer";
    default: return "unknown status";
    }
}

int stencil_plan_destroy(stencil_plan p);

static int plan_create(stencil_plan *out, const stencil_desc *desc);

int stencil_plan_create(stencil_plan *out, const stencil_desc *desc)
{
    // nothing forced and a measured choice cached for this problem: take it (an entry this
    // build cannot make falls back to the model's choice)
    if (out && desc && !desc->force_T && !desc->force_bx && !desc->force_by && !desc->force_vec &&
        !desc->partial_rows && !desc->resident) {
        stencil_desc t = *desc;
        int f[6];
        if (tune_cache_lookup(t, f)) {
            t.force_T = f[0];
            t.force_bx = f[1];
            t.force_by = f[2];
            t.force_vec = f[3];
            t.partial_rows = f[4];
            t.resident = f[5];
            const int rc = plan_create(out, &t);
            if (rc == ST_OK) {
                (*out)->tuned = 1;
                return rc;
            }
            if (rc != ST_ERR_UNSUPPORTED) return rc;
        }
    }
    return plan_create(out, desc);
}

int stencil_plan_tuned(stencil_plan p) { return p ? p->tuned : 0; }

static int plan_create(stencil_plan *out, const stencil_desc *desc)
{
    if (!out) return ST_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc) return ST_ERR_INVALID_ARG;
    stencil_desc d = *desc;
    if (d.kind != ST_DIFFUSION && d.kind != ST_THERMAL && d.kind != ST_DIFFUSION_VAR)
        return ST_ERR_INVALID_ARG;
    if (d.ndim != 2 && d.ndim != 3) return ST_ERR_INVALID_ARG;
    if (d.ndim == 2) d.nz = 1;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return ST_ERR_INVALID_ARG;
    if (d.storage != ST_F32 && d.storage != ST_BF16 && d.storage != ST_F16)
        return ST_ERR_INVALID_ARG;
    // 16-bit storage: 2D contracted plans only
    if (d.storage != ST_F32 && (d.ndim != 2 || d.exact)) return ST_ERR_UNSUPPORTED;
    if (d.force_T < 0 || d.force_bx < 0 || d.force_by < 0 || d.force_vec < 0)
        return ST_ERR_INVALID_ARG;
    if (d.rad < 0) return ST_ERR_INVALID_ARG;
    if (d.partial_rows < 0 || d.partial_rows > 2 || d.resident < -1 || d.resident > 1)
        return ST_ERR_INVALID_ARG;
    if (d.ndim == 2 && d.rad <= 1 && d.force_by) return ST_ERR_INVALID_ARG;   // no 2D tile height
    if (d.partial_rows && (d.ndim != 2 || d.exact || d.kind == ST_DIFFUSION_VAR || d.rad > 1))
        return ST_ERR_UNSUPPORTED;
    if (d.resident == 1 && (d.ndim != 2 || d.rad > 1 || d.kind == ST_DIFFUSION_VAR ||
                            d.storage != ST_F32 || d.force_bx || d.partial_rows))
        return ST_ERR_UNSUPPORTED;
    // per-cell coefficients: 2D float32 plans of the windowed kernel (V = 4, 128 or 512 cells
    // wide); the stability check of strict plans needs host coefficients
    if (d.kind == ST_DIFFUSION_VAR &&
        (d.ndim != 2 || d.storage != ST_F32 || d.rad > 1 || d.strict || d.force_by ||
         (d.force_vec && d.force_vec != 4) || (d.force_bx && d.force_bx != 128 && d.force_bx != 512)))
        return ST_ERR_UNSUPPORTED;
    if (d.rad > 1) {
        const int tile = d.ndim == 2 ? 128 : 64;   // star tiles: 128 x 128 in 2D, 64 x 64 in 3D
        if (d.kind != ST_DIFFUSION || d.storage != ST_F32 || d.rad > 4 ||
            (d.force_bx && d.force_bx != tile) || (d.force_by && d.force_by != tile) ||
            (d.force_vec && d.force_vec != (d.ndim == 2 ? 4 : 16)))
            return ST_ERR_UNSUPPORTED;
    }

    stencil_plan_s *p = new (std::nothrow) stencil_plan_s();
    if (!p) return ST_ERR_OOM;
    p->d = d;
    p->stream = static_cast<cudaStream_t>(d.stream);
    int rc = ST_OK;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return map_cuda(e);
    }

    p->stor = d.storage == ST_BF16 ? 1 : (d.storage == ST_F16 ? 2 : 0);
    if (d.rad > 1 && d.ndim == 3) {
        // 3D star diffusion: 64 x 64 tiles streamed along z, T = 1 unless forced: measured on
        // 512^3, R = 2 (GB300), T = 1 runs at 382 GCell/s and T = 2 at 271 -- the second ring
        // of planes leaves one 8-warp block per SM and adds a barrier per plane
        const int T = d.force_T ? d.force_T : 1;
        int bps = 0;
        if (!star3d_available(d.rad, d.exact, T)) rc = ST_ERR_UNSUPPORTED;
        if (rc == ST_OK) {
            e = star3d_prepare(d.rad, d.exact, T, &bps);
            if (e != cudaSuccess) rc = map_cuda(e);
            else if (bps < 1) rc = ST_ERR_UNSUPPORTED;
        }
        if (rc == ST_OK) {
            p->T = T;
            int cx = 0, cy = 0;
            star3d_tile(d.rad, T, &cx, &cy);
            p->ntx_star = (d.nx + cx - 1) / cx;
            p->nty_star = (d.ny + cy - 1) / cy;
            // z-segments: the count that keeps the most block slots busy, discounted by the
            // planes a segment re-reads (R T at either end); segments at least 8 R T long
            const long long cols = (long long)p->ntx_star * p->nty_star;
            const long long slots = (long long)p->sms * bps;
            const int max_seg = std::max(1, d.nz / (8 * d.rad * T));
            double best = -1.0;
            long long nseg = 1;
            for (int n = 1; n <= max_seg; n++) {
                const long long blocks = cols * n, waves = (blocks + slots - 1) / slots;
                const double zs = (double)((d.nz + n - 1) / n);
                const double eff = (double)blocks / (double)(waves * slots) * zs / (zs + 2.0 * d.rad * T);
                if (eff > best + 1e-9) {
                    best = eff;
                    nseg = n;
                }
            }
            p->zseg_star = (int)((d.nz + nseg - 1) / nseg);
            p->nseg_star = (d.nz + p->zseg_star - 1) / p->zseg_star;
            p->scratch_bytes = (size_t)cells_of(d) * sizeof(float);
        }
    } else if (d.rad > 1) {
        // star diffusion: 128 x 128 tiles, T from {1, 2, 4} (default: the largest whose halos
        // leave at least 70 % of the tile's cells in its compute block)
        int T = d.force_T;
        if (!T) {
            T = 1;
            for (int t : {2, 4}) {
                const double cx = 128 - 2 * ((d.rad * t + 3) / 4 * 4), cy = 128 - 2 * d.rad * t;
                if (cx > 0 && cy > 0 && cx * cy >= 0.7 * 128 * 128) T = t;
            }
        }
        if (!star2d_available(d.rad, d.exact, T)) rc = ST_ERR_UNSUPPORTED;
        if (rc == ST_OK) {
            e = star2d_prepare(d.rad, d.exact, T);
            if (e != cudaSuccess) rc = map_cuda(e);
        }
        if (rc == ST_OK) {
            p->T = T;
            const int cx = 128 - 2 * star2d_halo_x(d.rad, T), cy = 128 - 2 * star2d_halo_y(d.rad, T);
            p->ntx_star = (d.nx + cx - 1) / cx;
            p->nty_star = (d.ny + cy - 1) / cy;
            p->ld_scratch = d.nx;   // dense rows: the tensor map of a grid uses the grid's pitch
            p->scratch_bytes = (size_t)d.nx * d.ny * sizeof(float);
        }
    } else if (d.ndim == 2) {
        // resident tiles: when asked for, or compared below with the passes when nothing else
        // is forced
        ResGeom rg;
        bool res = false;
        if (d.resident == 1) {
            res = res_choose(d, p->sms, &rg);
            if (!res) rc = ST_ERR_UNSUPPORTED;
        } else if (d.resident == 0 && !d.force_T && !d.force_vec && !d.force_bx && !d.partial_rows &&
                   d.kind != ST_DIFFUSION_VAR && !p->stor) {
            res = res_choose(d, p->sms, &rg);
        }
        const double res_g = res ? 1000.0 * d.nx * d.ny / rg.t / 1e9 : 0.0;
        if (d.resident != 1) {
            // Contracted plans run one-warp tiles of V = 8 cells per thread (bsize_x = 256) with
            // partial-sum stages; exact plans run the rotating-window kernel, V = 4, with W warps
            // per tile (bsize_x = 128 W).
            // measured on GB300 (16384^2, T = 8): Hotspot runs best with V = 4 (its V = 8 body
            // overflows the instruction cache), Diffusion with V = 8
            const bool var = d.kind == ST_DIFFUSION_VAR;   // windowed kernel, exact or contracted
            p->V = d.force_vec ? d.force_vec : ((d.exact || d.kind != ST_DIFFUSION) ? 4 : 8);
            if (d.force_bx) {
                if (d.force_bx % (32 * p->V)) rc = ST_ERR_UNSUPPORTED;
                p->W = d.force_bx / (32 * p->V);
            } else {
                p->W = 1;
                if (d.exact && d.nx >= 512) p->W = 4;
            }
            if (!d.exact && d.partial_rows == 1) p->W = 0;   // partial rows updated in place
            if (!d.exact && d.partial_rows == 2) p->W = 1;   // two alternating sets of partial rows
            if (p->stor && !d.force_T && !d.force_vec && !d.force_bx && !d.partial_rows) {
                // 16-bit storage, nothing forced: T = 8, 8 cells per lane, rows in place (measured
                // on 16384^2: Hotspot 1990 GCell/s against 1802 for V = 4 two-row; diffusion 2720
                // against 2380 for V = 8 two-row)
                p->V = 8;
                p->W = 0;
            }
            if (!d.exact && !var && !p->stor && !d.force_T && !d.force_vec && !d.force_bx && !d.partial_rows) {
                // contracted, nothing forced: the compiled (T, V, variant) the model rates best
                const Cand2D cands[] = {{4, 4, 1}, {8, 4, 1}, {12, 4, 1}, {4, 8, 1}, {6, 8, 1},
                                        {8, 8, 1}, {8, 8, 0}, {12, 4, 0}};
                double best = -1.0;
                for (const Cand2D &k : cands) {
                    const Shape2D sh{d.kind, 0, k.T, k.V, k.W, d.kind == ST_THERMAL ? STOR_SRC : 0};
                    if (!tb2d_available(sh)) continue;
                    int bps = 0;
                    if (tb2d_prepare(sh, &bps) != cudaSuccess || bps < 1) continue;
                    const double g = model_gcells_2d(d, p->sms, k, bps, 1000);
                    if (g > best) {
                        best = g;
                        p->V = k.V;
                        p->W = k.W;
                    }
                }
                (void)cudaGetLastError();
            }
            // per-cell coefficients: every fused step keeps five more weight rows per tile column in
            // shared memory, so deeper fusion costs resident warps; measured on 8192^2 (GB300):
            // T = 4 with one-warp tiles 608 GCell/s, T = 8 545, four-warp tiles 532 / 451
            const int want = d.force_T ? d.force_T : (var ? 4 : 8);
            p->T = kernel_T_for(p, want);
            if (!d.exact && !var && !p->stor && !d.force_T && !d.force_vec && !d.force_bx && !d.partial_rows) {
                // and the T the model rates best within that family
                double best = -1.0;
                for (int t : kTcand) {
                    const Shape2D sh{d.kind, 0, t, p->V, p->W, d.kind == ST_THERMAL ? STOR_SRC : 0};
                    if (!tb2d_available(sh)) continue;
                    int bps = 0;
                    if (tb2d_prepare(sh, &bps) != cudaSuccess || bps < 1) continue;
                    const double g = model_gcells_2d(d, p->sms, Cand2D{t, p->V, p->W}, bps, 1000);
                    if (g > best) {
                        best = g;
                        p->T = t;
                    }
                }
                (void)cudaGetLastError();
            }
            if (p->T == 0 || (d.force_T && p->T != d.force_T)) rc = ST_ERR_UNSUPPORTED;
            PassCfg2D *c = nullptr;
            if (rc == ST_OK) rc = prepare2(p, p->T, &c);
            if (rc == ST_OK && p->stor) {
                // coded grids: rows padded to 8 cells (16 bytes), codes per (row, tile column)
                p->cx = 32 * p->V - 2 * ((p->T + 3) / 4 * 4);
                p->ntx = (d.nx + p->cx - 1) / p->cx;
                p->ld_q = ((long long)d.nx + 7) / 8 * 8;
                const size_t qb = (size_t)p->ld_q * d.ny * 2, mb = (size_t)p->ntx * d.ny * sizeof(float2);
                for (int b = 0; b < 2 && rc == ST_OK; b++) {
                    e = stn::dev_malloc(&p->q[b], qb);
                    if (e == cudaSuccess) e = stn::dev_malloc(&p->qm[b], mb);
                    if (e != cudaSuccess) rc = map_cuda(e);
                }
                if (rc == ST_OK && d.kind == ST_THERMAL) {
                    e = stn::dev_malloc(&p->qp, qb);
                    if (e == cudaSuccess) e = stn::dev_malloc(&p->qpm, mb);
                    if (e != cudaSuccess) rc = map_cuda(e);
                }
                p->scratch_bytes = 0;   // no float32 scratch: the coded grids take its place
            } else if (rc == ST_OK) {
                p->ld_scratch = ((long long)d.nx + 31) / 32 * 32;
                p->scratch_bytes = (size_t)p->ld_scratch * d.ny * sizeof(float);
            }
        }
        if (res && d.resident == 0 && rc == ST_OK && !d.exact) {
            // contracted: resident tiles only where the model rates them above the passes
            // (exact plans: always when the grid fits; the exact passes have no calibration)
            int bps = 0;
            const Shape2D sh{d.kind, 0, p->T, p->V, p->W, d.kind == ST_THERMAL ? STOR_SRC : 0};
            if (tb2d_prepare(sh, &bps) == cudaSuccess && bps > 0 &&
                model_gcells_2d(d, p->sms, Cand2D{p->T, p->V, p->W}, bps, 1000) >= res_g)
                res = false;
            (void)cudaGetLastError();
        }
        if (res && rc == ST_OK) {
            p->res = 1;
            p->T = rg.T;
            p->res_vx = rg.vx;
            p->res_nw = rg.nw;
            p->res_nbx = rg.nbx;
            p->res_nby = rg.nby;
            p->res_cw = rg.cw;
            p->res_ch = rg.ch;
            p->res_hx = rg.hx;
            p->res_ld = ((long long)d.nx + 3) / 4 * 4;
            p->scratch_bytes = 0;   // the two exchange grids take the scratch grid's place
            p->model = res_g;
        }
    } else {
        // tile width 64 (2 cells per lane) or 128 (4 cells per lane), tile height, cells per
        // thread; 64 x 64 with 16 cells per thread is the three-plane-window kernel (exact or
        // contracted), every other shape the partial-sum kernel (contracted)
        const bool free_tile = !d.exact && !d.force_bx && !d.force_by && !d.force_vec;
        int bx = d.force_bx ? d.force_bx : 64;
        int by = d.force_by ? d.force_by : (bx == 128 || free_tile ? 32 : 64);
        int cells = d.force_vec ? d.force_vec : (d.exact ? 16 : 8);
        int model_T = 0;
        if (free_tile && !d.force_T && d.rad <= 1) {
            // nothing forced, contracted: the compiled partial-sum (tile, T) the calibrated
            // model rates best
            const int shapes[][3] = {{64, 64, 8}, {64, 64, 4}, {128, 32, 8}, {64, 32, 8}};
            double best = -1.0;
            for (const auto &sh : shapes)
                for (int t = 1; t <= 4; t++) {
                    const int vx = sh[0] / 32, vy = sh[2] / vx, nw = sh[1] / vy;
                    if (!tb3d_available(Shape3D{d.kind, 0, t, vy, nw, 1, vx})) continue;
                    const double g = model_gcells_3d(d, p->sms, t, vx, vy, nw);
                    if (g > best) {
                        best = g;
                        bx = sh[0];
                        by = sh[1];
                        cells = sh[2];
                        model_T = t;
                    }
                }
        }
        if (bx != 64 && bx != 128) rc = ST_ERR_UNSUPPORTED;
        p->VX3 = bx / 32;
        if (rc == ST_OK && (cells % p->VX3 != 0 || by % (cells / p->VX3) != 0))
            rc = ST_ERR_UNSUPPORTED;
        if (rc == ST_OK) {
            p->VY = cells / p->VX3;
            p->NW = by / p->VY;
            p->alg3 = (p->VX3 == 2 && p->VY == 8 && p->NW == 8) ? 0 : 1;
            if (p->alg3 && d.exact) rc = ST_ERR_UNSUPPORTED;
        }
        const int want = d.force_T ? d.force_T : (model_T ? model_T : 4);
        p->T = kernel_T_for(p, want);
        if (p->T == 0 || (d.force_T && p->T != d.force_T)) rc = ST_ERR_UNSUPPORTED;
        PassCfg3D *c = nullptr;
        if (rc == ST_OK) rc = prepare3(p, p->T, &c);
        p->scratch_bytes = (size_t)cells_of(d) * sizeof(float);
    }
    if (rc == ST_OK && p->scratch_bytes) {
        e = stn::dev_malloc(&p->scratch, p->scratch_bytes);
        if (e != cudaSuccess) rc = map_cuda(e);
    }
    if (rc == ST_OK && d.ndim == 2 && d.kind == ST_THERMAL && !d.exact && !p->stor) {
        // rows padded to 32 cells like the scratch grid: 16-byte aligned rows for any nx
        p->ld_src = ((long long)d.nx + 31) / 32 * 32;
        e = stn::dev_malloc(&p->src, (size_t)p->ld_src * d.ny * sizeof(float));
        if (e != cudaSuccess) rc = map_cuda(e);
    }
    if (rc == ST_OK && p->res) {
        const size_t fb = (size_t)p->res_nbx * p->res_nby * sizeof(int);
        e = stn::dev_malloc(&p->res_xg, (size_t)2 * p->res_ld * d.ny * sizeof(float));
        if (e == cudaSuccess) e = stn::dev_malloc(&p->res_flags, fb);
        if (e == cudaSuccess) e = cudaMemset(p->res_flags, 0, fb);
        if (e != cudaSuccess) rc = map_cuda(e);
    }
    if (rc == ST_OK && !p->res && !d.exact && !p->stor && d.rad <= 1 && d.kind != ST_DIFFUSION_VAR) {
        if (d.ndim == 2) {
            int bps = 0;
            const Shape2D sh{d.kind, 0, p->T, p->V, p->W, d.kind == ST_THERMAL ? STOR_SRC : 0};
            if (tb2d_prepare(sh, &bps) == cudaSuccess && bps > 0)
                p->model = model_gcells_2d(d, p->sms, Cand2D{p->T, p->V, p->W}, bps, 1000);
            (void)cudaGetLastError();
        } else if (p->alg3) {
            p->model = model_gcells_3d(d, p->sms, p->T, p->VX3, p->VY, p->NW);
        }
    }
    if (rc == ST_OK) {
        e = stn::dev_malloc(&p->err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->err, 0, sizeof(int));
        if (e != cudaSuccess) rc = map_cuda(e);
    }
    if (rc != ST_OK) {
        stencil_plan_destroy(p);
        return rc;
    }
    *out = p;
    return ST_OK;
}

int stencil_run(stencil_plan p, const void *grid_in, void *grid_out, const void *power,
                const float *coeffs, int nx, int ny, int nz, int steps)
{
    if (!p || !grid_in || !grid_out || steps < 0) return ST_ERR_INVALID_ARG;
    const stencil_desc &d = p->d;
    // per-cell coefficients come as device planes in `power`; host coefficients are unused
    static const float no_coeffs[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (!coeffs) {
        if (d.kind != ST_DIFFUSION_VAR) return ST_ERR_INVALID_ARG;
        coeffs = no_coeffs;
    }
    if (d.ndim == 2 && nz != 1) return ST_ERR_DIMS_MISMATCH;
    if (nx != d.nx || ny != d.ny || nz != d.nz) return ST_ERR_DIMS_MISMATCH;
    if ((d.kind != ST_DIFFUSION) != (power != nullptr)) return ST_ERR_INVALID_ARG;
    const size_t bytes = (size_t)cells_of(d) * sizeof(float);
    const size_t pw_bytes = d.kind == ST_DIFFUSION_VAR ? 5 * bytes : bytes;
    if (grid_in != grid_out && ranges_overlap(grid_in, grid_out, bytes)) return ST_ERR_INVALID_ARG;
    if (power && ranges_overlap2(power, pw_bytes, grid_out, bytes)) return ST_ERR_INVALID_ARG;
    if (d.strict && !stable(d, coeffs)) return ST_ERR_UNSTABLE_COEFFS;
    if (p->sticky != ST_OK) return p->sticky;
    const stn::NvtxRange r_run("stencil_run");

    const float *in = static_cast<const float *>(grid_in);
    float *out = static_cast<float *>(grid_out);
    const float *pw = static_cast<const float *>(power);
    cudaError_t e;
    if (steps == 0) {
        if (in == out) return ST_OK;
        e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, p->stream);
        return map_cuda(e);
    }
    if (p->res) {
        const int rc = run_resident(p, in, out, pw, coeffs, steps);
        if (rc != ST_OK) p->sticky = rc;
        return rc;
    }
    const int T = p->T;
    const int passes = (steps + T - 1) / T;
    const int last = steps - T * (passes - 1);
    if (p->stor) {
        // 16-bit storage: code the field (and the power map), run every pass on the coded
        // grids, decode into the output
        e = lp_encode(p->stor, in, d.nx, p->q[0], p->ld_q, p->qm[0], d.nx, d.ny, p->cx, p->stream);
        // the power map is coded as the Hotspot source map sdc*(p + amb*Rz) the kernels read
        if (e == cudaSuccess && pw)
            e = lp_encode(p->stor, pw, d.nx, p->qp, p->ld_q, p->qpm, d.nx, d.ny, p->cx, p->stream,
                          coeffs[4] * coeffs[3], coeffs[0]);
        if (e != cudaSuccess) return map_cuda(e);
        int cur = 0;
        for (int i = 0; i < passes; i++) {
            const stn::NvtxRange r_pass("pass");
            const int rc = run_pass2q(p, cur, 1 - cur, coeffs, (i == passes - 1) ? last : T);
            if (rc != ST_OK) {
                p->sticky = rc;
                return rc;
            }
            cur = 1 - cur;
        }
        e = lp_decode(p->stor, p->q[cur], p->ld_q, p->qm[cur], out, d.nx, d.nx, d.ny, p->cx,
                      p->stream);
        return map_cuda(e);
    }
    // buffer of pass i: the caller's output when (passes-1-i) is even, else the scratch grid;
    // in place with an odd pass count, pass 0 cannot write the input it reads, so every pass
    // shifts by one and a final copy brings the scratch result to the output.
    const bool shift = (in == out) && (passes % 2 == 1);
    const long long ldo = d.nx, ldsc = d.ndim == 2 ? p->ld_scratch : d.nx;
    if (p->src) {
        // contracted Hotspot 2D kernels stage sdc*(p + amb*Rz) (Table 2's source and ambient
        // terms folded into one map)
        e = hot_source(pw, d.nx, p->src, p->ld_src, d.nx, d.ny, coeffs[4], coeffs[3], coeffs[0],
                       p->stream);
        if (e != cudaSuccess) return map_cuda(e);
        pw = p->src;
    }
    const float *src = in;
    long long lds = d.nx;
    for (int i = 0; i < passes; i++) {
        const stn::NvtxRange r_pass("pass");
        const int ts = (i == passes - 1) ? last : T;
        const bool to_out = shift ? ((passes - i) % 2 == 0) : ((passes - 1 - i) % 2 == 0);
        float *dst = to_out ? out : p->scratch;
        const long long ldd = to_out ? ldo : ldsc;
        int rc = d.rad > 1     ? run_pass_star(p, src, dst, coeffs, ts)
                 : d.ndim == 2 ? run_pass2(p, src, lds, dst, ldd, pw, coeffs, ts)
                               : run_pass3(p, src, dst, pw, coeffs, ts);
        if (rc != ST_OK) {
            p->sticky = rc;
            return rc;
        }
        src = dst;
        lds = ldd;
    }
    if (shift) {
        if (d.ndim == 2)
            e = cudaMemcpy2DAsync(out, (size_t)d.nx * sizeof(float), p->scratch,
                                  (size_t)p->ld_scratch * sizeof(float), (size_t)d.nx * sizeof(float),
                                  d.ny, cudaMemcpyDeviceToDevice, p->stream);
        else
            e = cudaMemcpyAsync(out, p->scratch, bytes, cudaMemcpyDeviceToDevice, p->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    return ST_OK;
}

int stencil_run_trajectory(stencil_plan p, const void *grid_in, void *states, long long stride,
                           const void *power, const float *coeffs, int steps)
{
    if (!p || !grid_in || !states || !coeffs || steps < 1) return ST_ERR_INVALID_ARG;
    const stencil_desc &d = p->d;
    if (d.ndim != 2 || d.exact || p->stor || d.rad > 1 || d.kind == ST_DIFFUSION_VAR)
        return ST_ERR_UNSUPPORTED;
    const long long n = (long long)d.nx * d.ny;
    if (stride < n) return ST_ERR_INVALID_ARG;
    if ((d.kind == ST_THERMAL) != (power != nullptr)) return ST_ERR_INVALID_ARG;
    const size_t bytes = (size_t)n * sizeof(float);
    const size_t span = ((size_t)(steps - 1) * stride + n) * sizeof(float);
    if (ranges_overlap2(grid_in, bytes, states, span)) return ST_ERR_INVALID_ARG;
    if (power && ranges_overlap2(power, bytes, states, span)) return ST_ERR_INVALID_ARG;
    if (d.strict && !stable(d, coeffs)) return ST_ERR_UNSTABLE_COEFFS;
    if (p->sticky != ST_OK) return p->sticky;
    PassCfg2D *c = nullptr;
    int rc = prepare_traj(p, &c);
    if (rc != ST_OK) return rc;
    const float *pw = static_cast<const float *>(power);
    if (p->src) {
        // contracted Hotspot kernels stage sdc*(p + amb*Rz) (Table 2's source and ambient terms
        // folded into one map)
        const cudaError_t e = hot_source(pw, d.nx, p->src, p->ld_src, d.nx, d.ny, coeffs[4],
                                         coeffs[3], coeffs[0], p->stream);
        if (e != cudaSuccess) return map_cuda(e);
        pw = p->src;
    }
    float *st = static_cast<float *>(states);
    const int passes = (steps + kTrajT - 1) / kTrajT;
    for (int i = 0; i < passes; i++) {
        const int ts = std::min(kTrajT, steps - i * kTrajT);
        const float *src = i == 0 ? static_cast<const float *>(grid_in)
                                  : st + ((long long)i * kTrajT - 1) * stride;
        float *dst = st + ((long long)i * kTrajT + ts - 1) * stride;
        rc = run_pass2(p, src, d.nx, dst, d.nx, pw, coeffs, ts, c,
                       st + (long long)i * kTrajT * stride, stride);
        if (rc != ST_OK) {
            p->sticky = rc;
            return rc;
        }
    }
    return ST_OK;
}

int stencil_plan_sync(stencil_plan p)
{
    if (!p) return ST_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return map_cuda(e);
    if (p->err) {
        int flag = 0;
        e = cudaMemcpy(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return map_cuda(e);
        if (flag) {
            (void)cudaMemset(p->err, 0, sizeof(int));
            return ST_ERR_TIMEOUT;
        }
    }
    return p->sticky;
}

int stencil_plan_set_wait(stencil_plan p, long long wait_ns, int hold_block, int hold_epoch)
{
    if (!p || wait_ns <= 0 || hold_block < -1) return ST_ERR_INVALID_ARG;
    if (!p->res) return ST_ERR_UNSUPPORTED;
    p->res_wait_ns = wait_ns;
    p->res_hold_block = hold_block;
    p->res_hold_epoch = hold_block >= 0 ? hold_epoch : -1;
    return ST_OK;
}

int stencil_plan_get_info(stencil_plan p, stencil_plan_info *info)
{
    if (!p || !info) return ST_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->T = p->T;
    info->model_gcells = p->model;
    info->sms = p->sms;
    info->scratch_bytes = (long long)p->scratch_bytes;
    info->exact = p->d.exact;
    info->partial_rows = (p->d.ndim == 2 && !p->d.exact && p->d.rad <= 1 && !p->res &&
                          p->d.kind != ST_DIFFUSION_VAR) ? (p->W == 0 ? 1 : 2) : 0;
    if (p->res) {
        info->resident = 1;
        info->bx = 32 * p->res_vx;
        info->by = p->res_nw * res2d_rows_per_thread();
        info->halo = p->res_hx;
        info->vec = p->res_vx;
        info->warps = p->res_nw;
        info->ctas = p->res_nbx * p->res_nby;
        info->scratch_bytes = (long long)2 * p->res_ld * p->d.ny * sizeof(float);
        info->kernel_id = 7;
        return ST_OK;
    }
    if (p->d.rad > 1 && p->d.ndim == 3) {
        int cx = 0, cy = 0;
        star3d_tile(p->d.rad, p->T, &cx, &cy);
        info->bx = 64;
        info->by = 64;
        info->halo = (64 - cx) / 2;
        info->vec = 16;
        info->warps = 8;
        info->ctas = p->ntx_star * p->nty_star * p->nseg_star;
        info->kernel_id = 6;
    } else if (p->d.rad > 1) {
        info->bx = 128;
        info->by = 128;
        info->halo = star2d_halo_x(p->d.rad, p->T);
        info->vec = 4;
        info->warps = 16;
        info->ctas = std::min(p->ntx_star * p->nty_star, p->sms);   // persistent, one per SM
        info->kernel_id = 5;
    } else if (p->d.ndim == 2) {
        PassCfg2D *c = nullptr;
        int rc = prepare2(p, p->T, &c);
        if (rc != ST_OK) return rc;
        const int warps = std::max(p->W, 1);   // W = 0 marks the one-warp in-place variant
        info->bx = 32 * p->V * warps;
        info->by = 0;
        info->halo = (p->T + 3) / 4 * 4;
        info->vec = p->V;
        info->warps = warps;
        info->ctas = c->ctas;
        info->kernel_id = 2;
    } else {
        PassCfg3D *c = nullptr;
        int rc = prepare3(p, p->T, &c);
        if (rc != ST_OK) return rc;
        info->bx = 32 * p->VX3;
        info->by = p->VY * p->NW;
        info->halo = p->T;
        info->vec = p->VX3 * p->VY;
        info->warps = p->NW;
        info->ctas = c->ctas;
        info->kernel_id = p->alg3 ? 4 : 3;
    }
    return ST_OK;
}

int stencil_plan_set_timing(stencil_plan p, int enable)
{
    if (!p) return ST_ERR_INVALID_ARG;
    p->timing = enable != 0;
    return ST_OK;
}

int stencil_plan_kernel_time(stencil_plan p, double *ms, long long *launches, int reset)
{
    if (!p || !ms || !launches) return ST_ERR_INVALID_ARG;
    int rc = flush_timing(p);
    if (rc != ST_OK) return rc;
    *ms = p->ms_acc;
    *launches = p->launches;
    if (reset) {
        p->ms_acc = 0.0;
        p->launches = 0;
    }
    return ST_OK;
}

int stencil_plan_destroy(stencil_plan p)
{
    if (!p) return ST_OK;
    if (p->ev_used) cudaStreamSynchronize(p->stream);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    if (p->scratch) stn::dev_free(p->scratch);
    for (int b = 0; b < 2; b++) {
        if (p->q[b]) stn::dev_free(p->q[b]);
        if (p->qm[b]) stn::dev_free(p->qm[b]);
    }
    if (p->qp) stn::dev_free(p->qp);
    if (p->qpm) stn::dev_free(p->qpm);
    if (p->err) stn::dev_free(p->err);
    if (p->src) stn::dev_free(p->src);
    if (p->res_xg) stn::dev_free(p->res_xg);
    if (p->res_flags) stn::dev_free(p->res_flags);
    for (PassCfg2D &c : p->cfg2)
        if (c.starts) stn::dev_free(c.starts);
    for (PassCfg3D &c : p->cfg3)
        if (c.starts) stn::dev_free(c.starts);
    delete p;
    return ST_OK;
}

}  // extern "C"
