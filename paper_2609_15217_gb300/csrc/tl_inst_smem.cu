// Shared-memory solver instantiations (run-time n): registered for every n
// from 2 to 32 as variants of kind 1, beside the per-n register kernels.
#include "tl_smem.cuh"

namespace tl {
namespace {

template <int T, int L>
void reg_smem()
{
    for (int n = 2; n <= TL_MAX_N; ++n) {
        register_variant(n, L, kOpGesv, T, reinterpret_cast<const void *>(&k_smem_group<T, L, kGesv, false>), 1);
        register_variant(n, L, kOpGesvLU, T, reinterpret_cast<const void *>(&k_smem_group<T, L, kGesv, true>), 1);
        register_variant(n, L, kOpGetrf, T, reinterpret_cast<const void *>(&k_smem_group<T, L, kGetrf, true>), 1);
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
        reg_smem_ragged<8>();
        reg_smem_ragged<16>();
        reg_smem_ragged<32>();
    }
};
const SmemRegistrar smem_registrar_instance;

}  // namespace
}  // namespace tl
