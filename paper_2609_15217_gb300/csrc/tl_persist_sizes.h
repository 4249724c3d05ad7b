// tl_persist_sizes.h -- shared-memory sizes of the single persistent
// ragged launch (tl_persist.cuh), for the launch code and the tuner.
#pragma once
#include "tl_smem.cuh"

namespace tl {

// Resident warps (one-warp blocks) per SM the launch is built for: the
// kernel's register limit (a sub-partition's 16,384 registers over its
// warps: 170 per thread for 12, 128 for 16) and the shared-memory slice of
// a warp follow from it.  Measured on GB300 with the benchmark's ragged
// mix: 16 warps (no one-thread register path at n = 7, wider lane groups
// at n = 7, 13, 19 and 32 to fit the smaller slice) is 2.5% slower than 12.
constexpr int kPersistWarps = 12;

// Shared-memory slice of one warp in doubles: an equal share of the SM's
// 228 KiB less the 1 KiB the hardware reserves per block and the block's
// static arrays.  12 warps: 2272 doubles (2 systems of n = 32 with 16 lanes
// each fit).
constexpr int kPersistSliceDoubles = (233472 / kPersistWarps - 1024 - 256) / 8;

// Doubles of shared memory one warp's item needs: 32 systems stored one
// after another with an odd stride for one thread per system, else 32 / T
// blocks of the element-walk solver.
__host__ __device__ constexpr int persist_reg_stride(int n) { return (n * n + n) | 1; }
__host__ __device__ constexpr int persist_need(int n, int T)
{
    return T == 1 ? 32 * persist_reg_stride(n) : (32 / T) * smem_sys_doubles(n, T);
}

// Largest n of the one-thread register path: 32 systems must fit in the
// slice (n = 7 with 12 warps).
constexpr int persist_reg_max_n()
{
    int n = 1;
    while (n < 9 && persist_need(n + 1, 1) <= kPersistSliceDoubles) ++n;
    return n;
}
constexpr int kPersistRegMaxN = persist_reg_max_n();

}  // namespace tl
