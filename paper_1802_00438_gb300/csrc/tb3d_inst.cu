// Compiled instances of the 3D temporally-blocked sweep (Diffusion 3D and Hotspot 3D).
// Contracted: T in {1,2,3,4}; tile 64 x 64 cells (8 warps, 8 rows per thread).
// Exact (Table 2 order): T in {1,2,4} with the 8-warp tile.
#include "tb3d_table.cuh"

namespace stn {

#define STN_F3(K, T_) STN_TB3_ENTRY(K, 0, T_, 8, 8)
#define STN_E3(K, T_) STN_TB3_ENTRY(K, 1, T_, 8, 8)

const Tb3dEntry tb3d_table[] = {
    STN_F3(0, 1), STN_F3(0, 2), STN_F3(0, 3), STN_F3(0, 4),
    STN_F3(1, 1), STN_F3(1, 2), STN_F3(1, 3), STN_F3(1, 4),
    STN_E3(0, 1), STN_E3(0, 2), STN_E3(0, 4),
    STN_E3(1, 1), STN_E3(1, 2), STN_E3(1, 4),
};
const int tb3d_table_n = sizeof(tb3d_table) / sizeof(tb3d_table[0]);

}  // namespace stn
