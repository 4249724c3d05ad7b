// tl_persist_sizes.h -- shared-memory sizes of the single persistent
// ragged launch (tl_persist.cuh), for the launch code and the tuner.
#pragma once
#include "tl_smem.cuh"

namespace tl {

// Shared-memory slice of one warp (doubles) unless a size's choice needs
// more: 2 systems of n = 32 with 16 lanes each, which also holds the
// measured best lanes of every smaller n (one thread up to n = 7, 2 lanes
// at 8, 4 up to 14, 8 up to 22, 16 above).  With it 12 warps stay resident
// per SM, and 12 warps leave 170 registers to a thread, enough for the
// one-thread register path.
constexpr int kPersistSliceDoubles = 2 * (32 * 33 + 32 + 16);

// Largest n of the one-thread register path.
constexpr int kPersistRegMaxN = 7;

// Doubles of shared memory one warp's item needs: 32 systems stored one
// after another with an odd stride for one thread per system, else 32 / T
// blocks of the element-walk solver.
__host__ __device__ constexpr int persist_reg_stride(int n) { return (n * n + n) | 1; }
__host__ __device__ constexpr int persist_need(int n, int T)
{
    return T == 1 ? 32 * persist_reg_stride(n) : (32 / T) * smem_sys_doubles(n, T);
}

}  // namespace tl
