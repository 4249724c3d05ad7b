// Instantiation unit of the mixed-precision ragged kernels for one n,
// compiled with -DTL_INST_N=<n> -DTL_INST_T=<lanes per system of the
// register kernel>: the register group kernel and (n >= 2) the shared-memory
// warp kernel, registered with the dispatcher when the library is loaded.
#include "tl_ir.cuh"
#include "tl_ir_smem.cuh"

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
        if constexpr (TL_INST_N >= 2)
            register_variant(TL_INST_N, kPerSystem, kOpRaggedIr, 32,
                             reinterpret_cast<const void *>(&k_smem_ir<TL_INST_N>), 1);
    }
};
const RegistrarIr registrar_ir_instance;

}  // namespace
}  // namespace tl
