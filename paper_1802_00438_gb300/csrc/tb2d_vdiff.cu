// Compiled instances of the 2D temporally-blocked sweep, diffusion with per-cell coefficients
// (Table 2 row 1 with its five coefficients as arrays): rotating register windows, V = 4, in
// Table 2 order (exact) or with fused multiply-adds (contracted), T in {1,2,4,8}, W in {1,4}.
#include "tb2d_table.cuh"

namespace stn {

#define STN_VD(E, T_) STN_TB2_ENTRY(2, E, T_, 4, 1), STN_TB2_ENTRY(2, E, T_, 4, 4)

const Tb2dEntry tb2d_table_vdiff[] = {
    STN_VD(1, 1), STN_VD(1, 2), STN_VD(1, 4), STN_VD(1, 8),
    STN_VD(0, 1), STN_VD(0, 2), STN_VD(0, 4), STN_VD(0, 8),
};
const int tb2d_table_vdiff_n = sizeof(tb2d_table_vdiff) / sizeof(tb2d_table_vdiff[0]);

}  // namespace stn
