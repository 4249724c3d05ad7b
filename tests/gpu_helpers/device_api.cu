// Test helper: a user kernel that includes only the public device header
// (include/tinylu_device.cuh) and calls tl::lupp_solve / tl::lupp_solve_subwarp
// once per system (compiled by tests/test_gpu_device_api.py with -I include
// alone).  Storage: per-system column-major A[s*N*N + j*N + i], b[s*N + i].
#include <cstdint>

#include "tinylu_device.cuh"

template <int N>
__global__ void k_user_thread(const double *A, const double *b, double *x, int *ipiv, int *info, int64_t batch)
{
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    double a[N][N], bb[N];
    int p[N];
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) a[i][j] = A[s * N * N + j * N + i];
    for (int i = 0; i < N; ++i) bb[i] = b[s * N + i];
    info[s] = tl::lupp_solve<N>(a, bb, p);
    for (int i = 0; i < N; ++i) {
        x[s * N + i] = bb[i];
        ipiv[s * N + i] = p[i];
    }
}

template <int N, int T>
__global__ void k_user_group(const double *A, const double *b, double *x, int *ipiv, int *info, int64_t batch)
{
    constexpr int K = tl::dev::Group<N, T>::K;
    const int t = static_cast<int>(threadIdx.x) % T;
    const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / T;
    const bool active = s < batch;  // every lane calls the solve (shuffles inside)
    double a[K][N], bb[K];
    int p[K];
    for (int sl = 0; sl < K; ++sl) {
        const int i = t + sl * T;
        const bool ok = active && i < N;
        for (int j = 0; j < N; ++j) a[sl][j] = ok ? A[s * N * N + j * N + i] : 0.0;
        bb[sl] = ok ? b[s * N + i] : 0.0;
    }
    const int inf = tl::lupp_solve_subwarp<N, T>(a, bb, p);
    if (!active) return;
    for (int sl = 0; sl < K; ++sl) {
        const int i = t + sl * T;
        if (i < N) {
            x[s * N + i] = bb[sl];
            ipiv[s * N + i] = p[sl];
        }
    }
    if (t == 0) info[s] = inf;
}

template <int N, int T>
static int launch(const double *A, const double *b, double *x, int *ipiv, int *info, int64_t batch)
{
    const int64_t threads = batch * T;
    const unsigned grid = static_cast<unsigned>((threads + 127) / 128);
    if (T == 1) k_user_thread<N><<<grid, 128>>>(A, b, x, ipiv, info, batch);
    else k_user_group<N, T><<<grid, 128>>>(A, b, x, ipiv, info, batch);
    return static_cast<int>(cudaDeviceSynchronize());
}

// Returns a CUDA error code, or -1 for an (n, T) pair not built here.
extern "C" int device_api_solve(int n, int T, const double *A, const double *b, double *x, int *ipiv, int *info,
                                int64_t batch)
{
#define TL_CASE(NN, TT) \
    if (n == (NN) && T == (TT)) return launch<NN, TT>(A, b, x, ipiv, info, batch);
    TL_CASE(1, 1)
    TL_CASE(3, 1)
    TL_CASE(7, 1)
    TL_CASE(9, 1)
    TL_CASE(10, 2)
    TL_CASE(13, 4)
    TL_CASE(20, 8)
    TL_CASE(32, 16)
    TL_CASE(32, 32)
#undef TL_CASE
    return -1;
}
