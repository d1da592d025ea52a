// Measurement helper, not part of the method: chains of fused multiply-adds
// that keep the float32 or float64 pipe busy, so that a benchmark can time
// the device's arithmetic peak (the denominator of an arithmetic roofline)
// on the device it runs on.  Each thread runs kChains independent chains of
// `iters` steps, 2 * kChains * iters flops, and writes its sum so that
// nothing is optimised away.
#include "pt_common.cuh"

namespace ptk {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = T(1) + T(1e-3) * T(t % 97 + k);
    const T b = T(0.9999999), c = T(1e-7);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    out[t] = s;
}

}  // namespace
}  // namespace ptk

extern "C" pt_status pt_fma_probe(int32_t fp64, int32_t iters, int32_t n_threads, void *out, void *stream) {
    using namespace ptk;
    if (!out || iters < 1 || n_threads < kThreads || n_threads % kThreads || (fp64 != 0 && fp64 != 1))
        return PT_ERR_INVALID_ARG;
    const int blocks = n_threads / kThreads;
    cudaStream_t s = (cudaStream_t)stream;
    if (fp64) k_fma_probe<double><<<blocks, kThreads, 0, s>>>(iters, (double *)out);
    else k_fma_probe<float><<<blocks, kThreads, 0, s>>>(iters, (float *)out);
    return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
