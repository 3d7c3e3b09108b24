// Compiled instances of the contracted partial-sum 3D sweep (Diffusion 3D):
// T in {1,2,3,4}, tiles of 64 x 64 cells as 16 warps of 4 rows or 32 warps of 2 rows.
#include "tb3d_table.cuh"

namespace stn {

const Tb3dEntry tb3f_table_diff[] = {
    STN_TB3F_ENTRY(0, 1, 4, 16), STN_TB3F_ENTRY(0, 2, 4, 16), STN_TB3F_ENTRY(0, 3, 4, 16),
    STN_TB3F_ENTRY(0, 4, 4, 16), STN_TB3F_ENTRY(0, 1, 2, 32), STN_TB3F_ENTRY(0, 2, 2, 32),
    STN_TB3F_ENTRY(0, 3, 2, 32), STN_TB3F_ENTRY(0, 4, 2, 32),
};
const int tb3f_table_diff_n = sizeof(tb3f_table_diff) / sizeof(tb3f_table_diff[0]);

}  // namespace stn
