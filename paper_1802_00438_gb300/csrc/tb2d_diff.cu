// Compiled instances of the 2D temporally-blocked sweep, Diffusion 2D.
// Exact (Table 2 order, rotating register windows): T in {1,2,4,8}, V = 4, W in {1,4}.
// Contracted (partial-sum stages, one warp per block): V = 8 for T in {1,2,4,6,8}, V = 4 for
// T in {1,2,4,8,12}; larger T or V do not fit the register file.  In-place variants (no
// two-row unroll) for (T, V) = (8, 8) and (12, 4), and (8, 8) for trajectory passes that write
// every fused step.  16-bit block-coded storage (bf16, fp16)
// for (T, V) in {(1, 4), (2, 4), (4, 4), (8, 4), (8, 8)}, and (8, 8) with in-place rows.
#include "tb2d_table.cuh"

namespace stn {

#define STN_EXACT(T_) STN_TB2_ENTRY(0, 1, T_, 4, 1), STN_TB2_ENTRY(0, 1, T_, 4, 4)

const Tb2dEntry tb2d_table_diff[] = {
    STN_EXACT(1), STN_EXACT(2), STN_EXACT(4), STN_EXACT(8),
    STN_TB2F_ENTRY(0, 1, 8), STN_TB2F_ENTRY(0, 2, 8), STN_TB2F_ENTRY(0, 4, 8),
    STN_TB2F_ENTRY(0, 8, 8), STN_TB2F_ENTRY(0, 6, 8),
    STN_TB2F_ENTRY(0, 1, 4), STN_TB2F_ENTRY(0, 2, 4), STN_TB2F_ENTRY(0, 4, 4),
    STN_TB2F_ENTRY(0, 8, 4), STN_TB2F_ENTRY(0, 12, 4),
    STN_TB2F1_ENTRY(0, 8, 8), STN_TB2F1_ENTRY(0, 12, 4), STN_TB2FA_ENTRY(0, 8, 8),
    STN_TB2FQ_ENTRY(0, 4, 4, 1), STN_TB2FQ_ENTRY(0, 8, 4, 1), STN_TB2FQ_ENTRY(0, 8, 8, 1),
    STN_TB2FQ_ENTRY(0, 4, 4, 2), STN_TB2FQ_ENTRY(0, 8, 4, 2), STN_TB2FQ_ENTRY(0, 8, 8, 2),
    STN_TB2FQ1_ENTRY(0, 8, 8, 1), STN_TB2FQ1_ENTRY(0, 8, 8, 2),
    STN_TB2FQ_ENTRY(0, 1, 4, 1), STN_TB2FQ_ENTRY(0, 2, 4, 1), STN_TB2FQ_ENTRY(0, 1, 4, 2),
    STN_TB2FQ_ENTRY(0, 2, 4, 2),
};
const int tb2d_table_diff_n = sizeof(tb2d_table_diff) / sizeof(tb2d_table_diff[0]);

}  // namespace stn
