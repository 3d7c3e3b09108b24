// Compiled instances of the 2D temporally-blocked sweep, Diffusion 2D.
// Contracted (exact = 0): T in {1,2,4,8,12} with (V,W) in {(4,1),(4,2),(4,4)}, plus V = 8
// (one warp per block) for T <= 8; larger T or V would not fit the register file.
// Exact (Table 2 order, no fused multiply-add): T in {1,2,4,8} with (V,W) in {(4,1),(4,4)}.
#include "tb2d_table.cuh"

namespace stn {

#define STN_FAST(T_) STN_TB2_ENTRY(0, 0, T_, 4, 1), STN_TB2_ENTRY(0, 0, T_, 4, 2), \
                     STN_TB2_ENTRY(0, 0, T_, 4, 4)
#define STN_FAST8(T_) STN_TB2_ENTRY(0, 0, T_, 8, 1)
#define STN_EXACT(T_) STN_TB2_ENTRY(0, 1, T_, 4, 1), STN_TB2_ENTRY(0, 1, T_, 4, 4)

const Tb2dEntry tb2d_table_diff[] = {
    STN_FAST(1), STN_FAST(2), STN_FAST(4), STN_FAST(8), STN_FAST(12),
    STN_FAST8(1), STN_FAST8(2), STN_FAST8(4), STN_FAST8(8),
    STN_EXACT(1), STN_EXACT(2), STN_EXACT(4), STN_EXACT(8),
};
const int tb2d_table_diff_n = sizeof(tb2d_table_diff) / sizeof(tb2d_table_diff[0]);

}  // namespace stn
