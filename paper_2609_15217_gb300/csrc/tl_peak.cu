// tl_peak.cu -- tl_measure_fma_peak: the FMA throughput of the device,
// measured.  Every LU flop of this library runs on the binary64 FMA pipe,
// so its roofline is that pipe's rate on the GPU at hand, not a datasheet
// number.  The probe fills every SM with warps that each run kChains
// independent FMA chains (x = fma(x, a, c), a slightly below 1, so every
// value stays a normal number near c / (1 - a)), times the launch with CUDA
// events on the caller's stream and reads each block's SM cycle counter,
// which gives the FMA rate per SM and clock as well as the clock the probe
// ran at.  a and c are formed per thread so that they live in registers:
// measured on GB300, a DFMA that reads an operand from the constant bank
// (a kernel parameter or a literal) issues at 1.68 lanes per clock per SM
// instead of the 2.0 of an all-register DFMA.
#include <cmath>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"

namespace tl {
namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_peak_sink;
__device__ unsigned long long g_peak_cycles;

template <typename F>
__device__ __forceinline__ F fma_rn(F x, F a, F c);
template <>
__device__ __forceinline__ double fma_rn<double>(double x, double a, double c) { return __fma_rn(x, a, c); }
template <>
__device__ __forceinline__ float fma_rn<float>(float x, float a, float c) { return __fmaf_rn(x, a, c); }

template <typename F>
__global__ void __launch_bounds__(kBlock) k_fma_peak(int iters, F a, F c)
{
    F x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = static_cast<F>(threadIdx.x + 7 * i) * static_cast<F>(1e-3);
    // register operands (a thread-dependent perturbation far below an ulp of
    // the chains' values keeps the compiler from folding them into constants)
    a = a + static_cast<F>(threadIdx.x) * static_cast<F>(1e-30);
    c = c + static_cast<F>(threadIdx.x) * static_cast<F>(1e-30);
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; it += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma_rn<F>(x[i], a, c);
    }
    __syncthreads();
    const long long t1 = clock64();
    F s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == static_cast<F>(-1.0)) g_peak_sink = static_cast<double>(s);  // never true; keeps the chains
    if (threadIdx.x == 0) atomicMax(&g_peak_cycles, static_cast<unsigned long long>(t1 - t0));
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" tl_status tl_measure_fma_peak(tl_handle *h, int bits, double *tflops, double *fma_per_clk_per_sm,
                                         double *sm_mhz, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (bits != 64 && bits != 32) return fail_arg(h, 2);
    if (!tflops) return fail_arg(h, 3);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs != cudaStreamCaptureStatusNone) return TL_ERR_UNSUPPORTED;
    // about 60 ms per launch at the expected rates (binary32 is ~60x faster)
    const int iters = bits == 64 ? 24576 : 24576 * 48;
    const unsigned grid = static_cast<unsigned>(h->sm_count * kBlocksPerSm);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 1e30f;
    unsigned long long cycles = 0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // the first launch warms up
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbolAsync(g_peak_cycles, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) break;
        cudaEventRecord(e0, stream);
        if (bits == 64)
            k_fma_peak<double><<<grid, kBlock, 0, stream>>>(iters, 0.9999999, 1e-7);
        else
            k_fma_peak<float><<<grid, kBlock, 0, stream>>>(iters, 0.9999f, 1e-5f);
        cudaEventRecord(e1, stream);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        unsigned long long cyc = 0;
        if ((e = cudaMemcpyFromSymbol(&cyc, g_peak_cycles, sizeof(cyc))) != cudaSuccess) break;
        if (rep > 0 && ms < best_ms) {
            best_ms = ms;
            cycles = cyc;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail_cuda(h, e);
    const double fmas = static_cast<double>(grid) * kBlock * kChains * static_cast<double>(iters);
    const double secs = best_ms * 1e-3;
    *tflops = 2.0 * fmas / secs / 1e12;
    if (fma_per_clk_per_sm) *fma_per_clk_per_sm = cycles ? fmas / static_cast<double>(cycles) / h->sm_count : 0.0;
    if (sm_mhz) *sm_mhz = cycles ? static_cast<double>(cycles) / secs / 1e6 : 0.0;
    return TL_OK;
}
