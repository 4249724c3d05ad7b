// Instantiation unit of the mixed-precision ragged kernel for one (N, T)
// pair, compiled with -DTL_INST_N=<n> -DTL_INST_T=<lanes per system>; it
// registers the kernel with the dispatcher when the library is loaded.
#include "tl_ir.cuh"

#ifndef TL_INST_N
#error "TL_INST_N must be defined"
#endif
#ifndef TL_INST_T
#error "TL_INST_T must be defined"
#endif

namespace tl {
namespace {

struct RegistrarIr {
    RegistrarIr()
    {
        register_variant(TL_INST_N, kPerSystem, kOpRaggedIr, TL_INST_T,
                         reinterpret_cast<const void *>(&k_ragged_ir<TL_INST_N, TL_INST_T>));
    }
};
const RegistrarIr registrar_ir_instance;

}  // namespace
}  // namespace tl
