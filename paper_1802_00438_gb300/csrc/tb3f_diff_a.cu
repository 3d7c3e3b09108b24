// Compiled instances of the contracted partial-sum 3D sweep (Diffusion 3D), 64 x 64 tiles:
// 2 x 4 cells per thread (16 warps, T = 1..4), 2 x 2 cells per thread (32 warps, T = 2..4), and
// 64 x 32 tiles of 2 x 4 cells per thread (8 warps, two blocks per SM, T = 2..4).
#include "tb3d_table.cuh"

namespace stn {

const Tb3dEntry tb3f_table_diff_a[] = {
    STN_TB3F_ENTRY(0, 1, 2, 4, 16), STN_TB3F_ENTRY(0, 2, 2, 4, 16), STN_TB3F_ENTRY(0, 3, 2, 4, 16),
    STN_TB3F_ENTRY(0, 4, 2, 4, 16), STN_TB3F_ENTRY(0, 2, 2, 2, 32), STN_TB3F_ENTRY(0, 3, 2, 2, 32),
    STN_TB3F_ENTRY(0, 4, 2, 2, 32),
    STN_TB3F_ENTRY(0, 2, 2, 4, 8), STN_TB3F_ENTRY(0, 3, 2, 4, 8), STN_TB3F_ENTRY(0, 4, 2, 4, 8),
};
const int tb3f_table_diff_a_n = sizeof(tb3f_table_diff_a) / sizeof(tb3f_table_diff_a[0]);

}  // namespace stn
