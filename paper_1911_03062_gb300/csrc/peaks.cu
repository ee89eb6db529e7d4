// peaks.cu -- arithmetic-throughput probes for the roofline denominators that are
// not copy bandwidth or BF16 tensor throughput: FP32 FMA and FP64 FMA (DFMA) on the
// SIMT pipes.  Built as its own small library (libnpfem_peaks.so), used by the
// benchmark's peaks leg only; the solver does not link it.
//
// Each thread runs CHAINS independent fused multiply-add chains for `iters`
// rounds (a = a * b + c with runtime b, c, so nothing folds), then stores their
// sum so nothing is dead.  Flops per launch = blocks * threads * iters * CHAINS * 2.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(T *out, int iters, T b, T c) {
    T a[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) a[j] = T(threadIdx.x) * T(1e-3) + T(j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) a[j] = fma(a[j], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += a[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// Launch the FP32 (fp64 = 0) or FP64 (fp64 = 1) probe on `stream` with `blocks`
// blocks of 256 threads; out: device buffer of blocks * 256 values of the type.
// Returns the flops the launch performs, or -1 on a launch error.
double npfem_peak_fma(int fp64, void *stream, int blocks, int iters, void *out) {
    cudaStream_t s = (cudaStream_t)stream;
    if (fp64)
        k_fma_loop<double><<<blocks, 256, 0, s>>>((double *)out, iters, 0.9999999, 1e-7);
    else
        k_fma_loop<float><<<blocks, 256, 0, s>>>((float *)out, iters, 0.9999999f, 1e-7f);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return (double)blocks * 256.0 * iters * CHAINS * 2.0;
}

}  // extern "C"
