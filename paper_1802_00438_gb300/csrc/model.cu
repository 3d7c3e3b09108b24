// Performance models (host code): the paper's FPGA model and its GPU restatement.
//
// stencil_model_fpga: Sec. 4 of arXiv 1802.00438, Eqs. 3-9, in the paper's own terms (memory
// throughput from f_max, par_vec, cell size and accesses, capped by th_max; compute blocks,
// block counts, traversed cells, reads and writes per pass; run time over ceil(iter/par_time)
// passes; throughput in GB/s of num_acc * size_input * size_cell * iter).  The paper writes
// Eq. 7 for 2D only; for 3D the same out-of-bound subtraction is applied along x and y.
//
// stencil_model_gpu: the same structure for the GPU engine.  A pass moves the algorithmic bytes
// through HBM (overlapping halo re-reads of neighbouring tiles are served by L2) and computes
// every cell of every tile, halos included, for each fused step; its time is the larger of the
// HBM time and the issue time, each divided by a calibration factor as the paper calibrates its
// projection (Sec. 6.3).
#include <cmath>

#include "../../include/stencil.h"

extern "C" {

int stencil_model_fpga(const stencil_fpga_model_in *in, stencil_fpga_model_out *out)
{
    if (!in || !out) return ST_ERR_INVALID_ARG;
    const stencil_fpga_model_in &m = *in;
    if ((m.ndim != 2 && m.ndim != 3) || m.rad < 1 || m.par_vec < 1 || m.par_time < 1 ||
        m.size_cell < 1 || m.num_read < 0 || m.num_write < 0 || m.iter < 0 || m.dim_x < 1 ||
        m.dim_y < 1 || m.bsize_x < 1 || m.fmax_hz <= 0 || m.th_max_gbs <= 0)
        return ST_ERR_INVALID_ARG;
    if (m.ndim == 3 && (m.dim_z < 1 || m.bsize_y < 1)) return ST_ERR_INVALID_ARG;
    stencil_fpga_model_out r = {};
    const double num_acc = m.num_read + m.num_write;
    // Eq. 3
    r.th_mem_gbs = std::fmin(m.fmax_hz * m.par_vec * m.size_cell * num_acc / 1e9, m.th_max_gbs);
    // Eq. 2 and Eq. 4
    const long long halo = (long long)m.rad * m.par_time;
    r.csize_x = m.bsize_x - 2 * halo;
    r.csize_y = m.ndim == 3 ? m.bsize_y - 2 * halo : 0;
    if (r.csize_x < 1 || (m.ndim == 3 && r.csize_y < 1)) return ST_ERR_INVALID_ARG;
    // Eq. 5
    r.bnum_x = (m.dim_x + r.csize_x - 1) / r.csize_x;
    r.bnum_y = m.ndim == 3 ? (m.dim_y + r.csize_y - 1) / r.csize_y : 0;
    // Eq. 6 and Eq. 7 (traversed cells beyond the input are not read)
    const double trav_x = (double)r.bnum_x * r.csize_x + 2.0 * halo;
    double size_input;
    if (m.ndim == 2) {
        r.t_cell = (double)r.bnum_x * m.bsize_x * m.dim_y;
        r.t_read = (r.t_cell - (trav_x - m.dim_x) * m.dim_y) * m.num_read;
        size_input = (double)m.dim_x * m.dim_y;
    } else {
        const double trav_y = (double)r.bnum_y * r.csize_y + 2.0 * halo;
        r.t_cell = (double)r.bnum_x * m.bsize_x * r.bnum_y * m.bsize_y * m.dim_z;
        r.t_read = ((double)r.bnum_x * m.bsize_x - (trav_x - m.dim_x)) *
                   ((double)r.bnum_y * m.bsize_y - (trav_y - m.dim_y)) * m.dim_z * m.num_read;
        size_input = (double)m.dim_x * m.dim_y * m.dim_z;
    }
    r.t_write = size_input * m.num_write;
    // Eq. 8
    const double passes = (double)((m.iter + m.par_time - 1) / m.par_time);
    r.run_time_s = passes * (r.t_read + r.t_write) * m.size_cell / (1e9 * r.th_mem_gbs);
    // Eq. 9
    r.throughput_gbs = r.run_time_s > 0
                           ? num_acc * size_input * m.size_cell * (double)m.iter / (1e9 * r.run_time_s)
                           : 0.0;
    *out = r;
    return ST_OK;
}

int stencil_model_gpu(const stencil_gpu_model_in *in, stencil_gpu_model_out *out)
{
    if (!in || !out) return ST_ERR_INVALID_ARG;
    const stencil_gpu_model_in &m = *in;
    if ((m.ndim != 2 && m.ndim != 3) || m.nx < 1 || m.ny < 1 || m.nz < 1 || m.steps < 0 ||
        m.T < 1 || m.bx < 1 || m.halo_x < 0 || m.sms < 1 || m.sm_hz <= 0 || m.hbm_gbs <= 0 ||
        m.ops_per_cell <= 0 || m.issue_eff <= 0 || m.hbm_eff <= 0 || m.bytes_per_cell <= 0)
        return ST_ERR_INVALID_ARG;
    if (m.ndim == 3 && (m.by < 1 || m.halo_y < 0)) return ST_ERR_INVALID_ARG;
    stencil_gpu_model_out r = {};
    const long long cx = m.bx - 2LL * m.halo_x;
    const long long cy = m.ndim == 3 ? m.by - 2LL * m.halo_y : 1;
    if (cx < 1 || cy < 1) return ST_ERR_INVALID_ARG;
    const double ntx = std::ceil((double)m.nx / cx);
    const double cells = (double)m.nx * m.ny * (m.ndim == 3 ? m.nz : 1);
    // cells computed per fused step, halos included (the streamed axis carries the 2T-row
    // warm-up of every segment, folded into stream_overhead)
    double computed;
    if (m.ndim == 2) {
        computed = ntx * m.bx * (double)m.ny * (1.0 + m.stream_overhead);
    } else {
        const double nty = std::ceil((double)m.ny / cy);
        computed = ntx * m.bx * nty * m.by * (double)m.nz * (1.0 + m.stream_overhead);
    }
    r.passes = m.steps > 0 ? std::ceil((double)m.steps / m.T) : 0;
    r.bytes_per_pass = cells * m.bytes_per_cell;
    r.cells_computed_per_pass = computed * m.T;
    r.t_hbm_s = r.bytes_per_pass / (m.hbm_gbs * 1e9 * m.hbm_eff);
    const double lanes = (double)m.sms * 128.0 * m.sm_hz * m.issue_eff;
    r.t_alu_s = r.cells_computed_per_pass * m.ops_per_cell / lanes;
    r.t_pass_s = std::fmax(r.t_hbm_s, r.t_alu_s) + m.launch_s;
    r.run_time_s = r.passes * r.t_pass_s;
    r.gcells = r.run_time_s > 0 ? cells * m.steps / r.run_time_s / 1e9 : 0.0;
    *out = r;
    return ST_OK;
}

}  // extern "C"
