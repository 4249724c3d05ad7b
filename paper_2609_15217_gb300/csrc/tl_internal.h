// tl_internal.h -- types shared by the kernel instantiations and the C ABI
// implementation (not part of the public interface).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tl {

enum : int { kPerSystem = 0, kInterleaved = 1 };
enum : int { kGesv = 0, kGetrf = 1, kGetrs = 2 };

// Arguments of every batched solve kernel.  Unused pointers are null.
//   gesv : A, b in; x, ipiv, info out; LU out when factors are requested
//   getrf: LU in/out (A is ignored); ipiv, info out
//   getrs: A = factors in, ipiv in, x = right-hand sides in / solutions out
struct SolveArgs {
    const double *A;
    double *LU;
    const double *b;
    double *x;
    int32_t *ipiv;
    int32_t *info;
    int64_t ld;
    int64_t batch;
    int nrhs;
    // tile-local pivoting (shared-memory kernels only): 0 = textbook
    int tile;
    double threshold;
};

// Arguments of the ragged-batch kernels (tl_lupp_solve_batched): the
// systems of size N are listed in bucket[offsets[N] .. offsets[N+1]) -- or
// bucket[offsets[N] .. offsets[N] + counts[N]) when counts is set; each one
// lives at its own element offsets in per-system column-major storage.
// The mixed-precision kernels also write refine (nullable) and append the
// systems they hand to the binary64 kernels to fb_list[offsets[N] + ...],
// counting them in fb_count[N].
struct RaggedArgs {
    const int32_t *bucket;
    const int32_t *offsets;  // [TL_MAX_N + 2]
    const int64_t *a_off;
    const double *A;
    const int64_t *b_off;
    const double *b;
    double *x;
    const int64_t *piv_off;
    int32_t *ipiv;
    int32_t *info;
    const int32_t *counts;
    int32_t *refine;
    int32_t *fb_count;
    int32_t *fb_list;
};

// Kernel variant for one (n, layout, operation): how many lanes share a
// system (1 = one thread per system) and the launch entry.
//   kind 0: register kernel compiled for one n, kernel(SolveArgs)
//   kind 1: shared-memory kernel for any n, kernel(SolveArgs, int n) with
//           smem_sys_bytes(n) of dynamic shared memory per system
// The variant id is lanes + 100 * kind.
struct Variant {
    int lanes;                     // T
    const void *kernel;            // __global__ function, for occupancy queries
    int kind;
    const void *fixup;             // second pass for flagged systems (or null)
};
__host__ __device__ constexpr int variant_id(int lanes, int kind) { return lanes + 100 * kind; }

// Registry filled by the instantiation units (tl_inst.cu, one per (N, T)).
enum : int {
    kOpGesv = 0,
    kOpGesvLU = 1,
    kOpGetrf = 2,
    kOpGetrs = 3,
    kOpRagged = 4,
    kOpRaggedIr = 5,
    kOpNewtonTanh = 6
};
constexpr int kOps = 7;
constexpr int kMaxVariants = 12;
struct VariantList {
    int count;
    Variant v[kMaxVariants];
};
VariantList &registry(int n, int layout, int op);
void register_variant(int n, int layout, int op, int lanes, const void *kernel, int kind = 0,
                      const void *fixup = nullptr);

}  // namespace tl
