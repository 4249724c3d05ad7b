// Kernel instantiation unit: compiled once per (N, T) pair with
// -DTL_INST_N=<n> -DTL_INST_T=<lanes per system>, so the per-size kernels
// build in parallel.  The unit registers its kernels with the dispatcher
// when the library is loaded.
#include "tl_kernels.cuh"

#ifndef TL_INST_N
#error "TL_INST_N must be defined"
#endif
#ifndef TL_INST_T
#error "TL_INST_T must be defined"
#endif

namespace tl {
namespace {

template <int N, int T, int L>
void reg_one_layout()
{
    if constexpr (T == 1) {
        register_variant(N, L, kOpGesv, 1, reinterpret_cast<const void *>(&k_factor_thread<N, L, kGesv, false>), 0,
                         reinterpret_cast<const void *>(&k_fixup_thread<N, L, kGesv, false>));
        register_variant(N, L, kOpGesvLU, 1, reinterpret_cast<const void *>(&k_factor_thread<N, L, kGesv, true>), 0,
                         reinterpret_cast<const void *>(&k_fixup_thread<N, L, kGesv, true>));
        register_variant(N, L, kOpGetrf, 1, reinterpret_cast<const void *>(&k_factor_thread<N, L, kGetrf, true>), 0,
                         reinterpret_cast<const void *>(&k_fixup_thread<N, L, kGetrf, true>));
        register_variant(N, L, kOpGetrs, 1, reinterpret_cast<const void *>(&k_getrs_thread<N, L>));
    } else {
        register_variant(N, L, kOpGesv, T, reinterpret_cast<const void *>(&k_factor_group<N, T, L, kGesv, false>));
        register_variant(N, L, kOpGesvLU, T, reinterpret_cast<const void *>(&k_factor_group<N, T, L, kGesv, true>));
        register_variant(N, L, kOpGetrf, T, reinterpret_cast<const void *>(&k_factor_group<N, T, L, kGetrf, true>));
        register_variant(N, L, kOpGetrs, T, reinterpret_cast<const void *>(&k_getrs_group<N, T, L>));
    }
}

struct Registrar {
    Registrar()
    {
        reg_one_layout<TL_INST_N, TL_INST_T, kPerSystem>();
        reg_one_layout<TL_INST_N, TL_INST_T, kInterleaved>();
        // ragged batches are per-system storage only; registered in slot 0
        // (register groups only up to n = 16: above, the shared-memory
        // solvers are faster and the register groups spill)
        if constexpr (TL_INST_T == 1)
            register_variant(TL_INST_N, kPerSystem, kOpRagged, 1,
                             reinterpret_cast<const void *>(&k_ragged_thread<TL_INST_N>), 0,
                             reinterpret_cast<const void *>(&k_ragged_fixup<TL_INST_N>));
        else if constexpr (TL_INST_N <= 16)
            register_variant(TL_INST_N, kPerSystem, kOpRagged, TL_INST_T,
                             reinterpret_cast<const void *>(&k_ragged_group<TL_INST_N, TL_INST_T>));
    }
};
const Registrar registrar_instance;

}  // namespace
}  // namespace tl
