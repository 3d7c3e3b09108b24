// Registry of the compiled 3D kernel instances.
#pragma once
#include "tb3d_kernel.cuh"

namespace stn {

struct Tb3dEntry {
    int kind, exact, T, VY, NW;
    const void *fn;
    size_t smem;
};

#define STN_TB3_ENTRY(K, E, T_, VY_, NW_)                                                       \
    { K, E, T_, VY_, NW_, reinterpret_cast<const void *>(&k_tb3d<K, (E != 0), T_, VY_, NW_>), \
      TB3<K, (E != 0), T_, VY_, NW_>::SMEM }

extern const Tb3dEntry tb3d_table[];
extern const int tb3d_table_n;

}  // namespace stn
