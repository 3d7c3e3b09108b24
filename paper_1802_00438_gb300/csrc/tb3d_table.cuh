// Registry of the compiled 3D kernel instances.
#pragma once
#include "tb3d_kernel.cuh"
#include "tb3f_kernel.cuh"

namespace stn {

struct Tb3dEntry {
    int kind, exact, T, VY, NW, alg, VX;
    const void *fn;
    size_t smem;
};

#define STN_TB3_ENTRY(K, E, T_, VY_, NW_)                                                       \
    { K, E, T_, VY_, NW_, 0, 2, reinterpret_cast<const void *>(&k_tb3d<K, (E != 0), T_, VY_, NW_>), \
      TB3<K, (E != 0), T_, VY_, NW_>::SMEM }

#define STN_TB3F_ENTRY(K, T_, VX_, VY_, NW_)                                                    \
    { K, 0, T_, VY_, NW_, 1, VX_, reinterpret_cast<const void *>(&k_tb3f<K, T_, VX_, VY_, NW_>), \
      TB3F<K, T_, VX_, VY_, NW_>::SMEM }

// registries of the partial-sum instances, one per translation unit
struct Tb3dList {
    const Tb3dEntry *e;
    const int *n;
};

extern const Tb3dEntry tb3d_table[];
extern const int tb3d_table_n;
extern const Tb3dEntry tb3f_table_diff_a[], tb3f_table_diff_b[], tb3f_table_therm_a[],
    tb3f_table_therm_b[];
extern const int tb3f_table_diff_a_n, tb3f_table_diff_b_n, tb3f_table_therm_a_n,
    tb3f_table_therm_b_n;

}  // namespace stn
