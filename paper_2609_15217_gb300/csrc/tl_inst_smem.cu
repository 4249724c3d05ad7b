// Shared-memory solver instantiations (run-time n): registered for every n
// from 2 to 32 as variants of kind 1 (lane tile for 2..8 lanes, element walk
// for 16 and 32) and kind 2 (element walk for 2..8 lanes), beside the per-n
// register kernels.
#include "tl_smem.cuh"

namespace tl {
namespace {

// ASYNC: cp.async loads into shared memory (the 2..8-lane kernels, 20-40%
// faster than staged loads); 16 and 32 lanes per system measured 4-8% faster
// with register-staged streaming loads.
template <int T, int L, bool WALK = (T >= 16), bool ASYNC = (T < 16)>
void reg_smem()
{
    constexpr int kind = (WALK && T < 16) ? 2 : 1;
    for (int n = 2; n <= TL_MAX_N; ++n) {
        register_variant(n, L, kOpGesv, T,
                         reinterpret_cast<const void *>(&k_smem_group<T, L, kGesv, false, WALK, ASYNC>), kind);
        register_variant(n, L, kOpGesvLU, T,
                         reinterpret_cast<const void *>(&k_smem_group<T, L, kGesv, true, WALK, ASYNC>), kind);
        register_variant(n, L, kOpGetrf, T,
                         reinterpret_cast<const void *>(&k_smem_group<T, L, kGetrf, true, WALK, ASYNC>), kind);
    }
}

template <int T>
void reg_smem_ragged()
{
    for (int n = 2; n <= TL_MAX_N; ++n)
        register_variant(n, kPerSystem, kOpRagged, T, reinterpret_cast<const void *>(&k_smem_ragged<T>), 1);
}

struct SmemRegistrar {
    SmemRegistrar()
    {
        reg_smem<2, kPerSystem>();
        reg_smem<4, kPerSystem>();
        reg_smem<8, kPerSystem>();
        reg_smem<16, kPerSystem>();
        reg_smem<32, kPerSystem>();
        reg_smem<2, kInterleaved>();
        reg_smem<4, kInterleaved>();
        reg_smem<8, kInterleaved>();
        reg_smem<16, kInterleaved>();
        reg_smem<32, kInterleaved>();
        reg_smem<2, kPerSystem, true>();
        reg_smem<4, kPerSystem, true>();
        reg_smem<8, kPerSystem, true>();
        reg_smem<2, kInterleaved, true>();
        reg_smem<4, kInterleaved, true>();
        reg_smem<8, kInterleaved, true>();
        reg_smem_ragged<2>();
        reg_smem_ragged<4>();
        reg_smem_ragged<8>();
        reg_smem_ragged<16>();
        reg_smem_ragged<32>();
    }
};
const SmemRegistrar smem_registrar_instance;

}  // namespace
}  // namespace tl
