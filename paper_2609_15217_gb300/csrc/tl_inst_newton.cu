// Instantiation unit of the sub-warp tanh-law Newton kernel for one (N, T)
// pair, compiled with -DTL_INST_N=<n> -DTL_INST_T=<lanes per point>; it
// registers the kernel with the dispatcher when the library is loaded.
#include "tl_newton.cuh"

#ifndef TL_INST_N
#error "TL_INST_N must be defined"
#endif
#ifndef TL_INST_T
#error "TL_INST_T must be defined"
#endif

namespace tl {
namespace {

struct RegistrarNewton {
    RegistrarNewton()
    {
        register_variant(TL_INST_N, kPerSystem, kOpNewtonTanh, TL_INST_T,
                         reinterpret_cast<const void *>(&k_newton_tanh_group<TL_INST_N, TL_INST_T>));
    }
};
const RegistrarNewton registrar_newton_instance;

}  // namespace
}  // namespace tl
