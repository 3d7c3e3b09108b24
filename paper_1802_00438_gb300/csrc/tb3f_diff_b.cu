// Compiled instances of the contracted partial-sum 3D sweep (Diffusion 3D), 128 x 32 tiles:
// 4 x 2 cells per thread (16 warps), T = 2..4.
#include "tb3d_table.cuh"

namespace stn {

const Tb3dEntry tb3f_table_diff_b[] = {
    STN_TB3F_ENTRY(0, 2, 4, 2, 16), STN_TB3F_ENTRY(0, 3, 4, 2, 16), STN_TB3F_ENTRY(0, 4, 4, 2, 16),
};
const int tb3f_table_diff_b_n = sizeof(tb3f_table_diff_b) / sizeof(tb3f_table_diff_b[0]);

}  // namespace stn
