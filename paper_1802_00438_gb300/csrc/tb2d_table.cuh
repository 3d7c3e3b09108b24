// Registry of the compiled 2D kernel instances.
#pragma once
#include "tb2d_kernel.cuh"
#include "tb2f_kernel.cuh"

namespace stn {

struct Tb2dEntry {
    int kind, exact, T, V, W;
    const void *fn;
    size_t smem;
    int stor;   // 0 float32 grids; 1 bf16, 2 fp16 block-coded grids; + STOR_SRC (Hotspot:
                // the power map arrives with amb*Rz folded in)
};

#define STN_TB2_ENTRY(K, E, T_, V_, W_)                                                      \
    { K, E, T_, V_, W_, reinterpret_cast<const void *>(&k_tb2d<K, (E != 0), T_, V_, W_>),  \
      TB2<K, (E != 0), T_, V_, W_>::SMEM, 0 }

// contracted path: one-warp blocks (W = 1), partial-sum stages
// W = 1: partial rows alternate between two register arrays (two-row unroll);
// W = 0 (a marker, still one warp): partial rows updated in place, no unroll
// Hotspot contracted kernels read the power map with amb*Rz folded in (STOR_SRC), except the
// plain-power instances (STN_TB2F0_ENTRY) that the allocation-free entry point uses
#define STN_TB2F_SRC(K) ((K) == 1 ? STOR_SRC : 0)
#define STN_TB2F_ENTRY(K, T_, V_)                                                            \
    { K, 0, T_, V_, 1,                                                                       \
      reinterpret_cast<const void *>(&k_tb2f<K, T_, V_, true, STN_TB2F_SRC(K)>),           \
      TB2F<K, T_, V_, STN_TB2F_SRC(K)>::SMEM, STN_TB2F_SRC(K) }
#define STN_TB2F1_ENTRY(K, T_, V_)                                                           \
    { K, 0, T_, V_, 0,                                                                       \
      reinterpret_cast<const void *>(&k_tb2f<K, T_, V_, false, STN_TB2F_SRC(K)>),          \
      TB2F<K, T_, V_, STN_TB2F_SRC(K)>::SMEM, STN_TB2F_SRC(K) }
#define STN_TB2F0_ENTRY(K, T_, V_)                                                           \
    { K, 0, T_, V_, 1, reinterpret_cast<const void *>(&k_tb2f<K, T_, V_, true, 0>),        \
      TB2F<K, T_, V_>::SMEM, 0 }
// trajectory passes (every fused step's rows written too): in-place partial rows
#define STN_TB2FA_ENTRY(K, T_, V_)                                                           \
    { K, 0, T_, V_, 0,                                                                       \
      reinterpret_cast<const void *>(&k_tb2f<K, T_, V_, false, STN_TB2F_SRC(K) | STOR_ALL>), \
      TB2F<K, T_, V_, STN_TB2F_SRC(K) | STOR_ALL>::SMEM, STN_TB2F_SRC(K) | STOR_ALL }
// 16-bit block-coded storage (S = 1 bf16, 2 fp16), two-row unroll
#define STN_TB2FQ_ENTRY(K, T_, V_, S)                                                        \
    { K, 0, T_, V_, 1,                                                                       \
      reinterpret_cast<const void *>(&k_tb2f<K, T_, V_, true, (S) | STN_TB2F_SRC(K)>),     \
      TB2F<K, T_, V_, (S) | STN_TB2F_SRC(K)>::SMEM, (S) | STN_TB2F_SRC(K) }

// 16-bit block-coded storage, partial rows updated in place (W = 0 marker)
#define STN_TB2FQ1_ENTRY(K, T_, V_, S)                                                       \
    { K, 0, T_, V_, 0,                                                                       \
      reinterpret_cast<const void *>(&k_tb2f<K, T_, V_, false, (S) | STN_TB2F_SRC(K)>),    \
      TB2F<K, T_, V_, (S) | STN_TB2F_SRC(K)>::SMEM, (S) | STN_TB2F_SRC(K) }

extern const Tb2dEntry tb2d_table_diff[];
extern const int tb2d_table_diff_n;
extern const Tb2dEntry tb2d_table_therm[];
extern const int tb2d_table_therm_n;
extern const Tb2dEntry tb2d_table_vdiff[];
extern const int tb2d_table_vdiff_n;

}  // namespace stn
