// Registry of the compiled 3D kernel instances.
#pragma once
#include "tb3d_kernel.cuh"
#include "tb3f_kernel.cuh"

namespace stn {

struct Tb3dEntry {
    int kind, exact, T, VY, NW, alg;
    const void *fn;
    size_t smem;
};

#define STN_TB3_ENTRY(K, E, T_, VY_, NW_)                                                       \
    { K, E, T_, VY_, NW_, 0, reinterpret_cast<const void *>(&k_tb3d<K, (E != 0), T_, VY_, NW_>), \
      TB3<K, (E != 0), T_, VY_, NW_>::SMEM }

#define STN_TB3F_ENTRY(K, T_, VY_, NW_)                                                         \
    { K, 0, T_, VY_, NW_, 1, reinterpret_cast<const void *>(&k_tb3f<K, T_, VY_, NW_>),         \
      TB3F<K, T_, VY_, NW_>::SMEM }

extern const Tb3dEntry tb3d_table[];
extern const int tb3d_table_n;
extern const Tb3dEntry tb3f_table_diff[];
extern const int tb3f_table_diff_n;
extern const Tb3dEntry tb3f_table_therm[];
extern const int tb3f_table_therm_n;

}  // namespace stn
