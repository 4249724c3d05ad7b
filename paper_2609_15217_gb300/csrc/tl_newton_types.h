// tl_newton_types.h -- job tables of the fused Newton kernels (shared by
// the kernels of tl_newton.cuh and the host code that builds the tables).
#pragma once
#include <cstdint>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_norton.cuh"

namespace tl {

// One request's points.  Field-major arrays with stride npoints:
// in[f*npoints + p], x[i*npoints + p], out[i*npoints + p].
struct NewtonJob {
    const double *in;
    double *x;
    double *out;  // nullable (Norton: end-of-step stress)
    double *tangent;  // nullable (Norton: consistent tangent, 36 rows)
    int32_t *iters;
    int32_t *status;
    int64_t npoints;
    int64_t start;  // index of the job's first point in the launch
    NortonParams P;  // Norton jobs only
};

// A launch: jobs[0..njobs) in device memory, or the single job `one` when
// jobs is null.  Points are numbered 0..total-1 across the jobs in order.
struct NewtonBatch {
    const NewtonJob *jobs;
    NewtonJob one;
    int njobs;
    int64_t total;
    double rtol;
    int max_iter;
};

// Launch the fused Newton kernel of a law (law_id, n) over B on stream.
tl_status newton_launch(tl_handle *h, int law_id, int n, const NewtonBatch &B, cudaStream_t stream);
// Shared-memory tanh-law kernel for 25 <= n <= 32: launches it and returns
// true with *out set, or returns false for other n.
bool newton_tanh_smem_launch(tl_handle *h, int n, const NewtonBatch &B, cudaStream_t stream, tl_status *out);
// Law parameters of a descriptor into a job (false: invalid descriptor).
bool law_params(const tl_law &law, NewtonJob *jb);

}  // namespace tl
