// Compiled instances of the contracted partial-sum 3D sweep (Hotspot 3D), 128 x 32 tiles:
// 4 x 2 cells per thread (16 warps), T = 2..4.
#include "tb3d_table.cuh"

namespace stn {

const Tb3dEntry tb3f_table_therm_b[] = {
    STN_TB3F_ENTRY(1, 2, 4, 2, 16), STN_TB3F_ENTRY(1, 3, 4, 2, 16), STN_TB3F_ENTRY(1, 4, 4, 2, 16),
};
const int tb3f_table_therm_b_n = sizeof(tb3f_table_therm_b) / sizeof(tb3f_table_therm_b[0]);

}  // namespace stn
