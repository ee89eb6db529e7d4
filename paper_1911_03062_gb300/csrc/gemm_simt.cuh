// gemm_simt.cuh -- FP64 (and FP32) CUDA-core kernels of the global step and
// of the one-time set-up:
//   * k_gemm_simt : Z[r][v] = sum_k Q[r][k] Pinv[v][k], the plain FP64 apply of
//                   P^{-1} to all stacked right-hand sides (the comparison form);
//   * k_gj_*      : in-place Gauss-Jordan inversion of the SPD matrix P in FP64,
//                   one pivot per launch pair (no pivoting: P is SPD and strongly
//                   diagonally dominant through M/h^2);
//   * k_convert_pinv : FP64 inverse -> FP32 (or TF32 high and low part) / BF16 (high and
//                      low part) operand copies.
#pragma once

#include "common.cuh"

namespace npfem {

constexpr int SG_T = 64;   // output tile (rows x vertices)
constexpr int SG_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(int rows, int nV, int nVp, const T *__restrict__ Q,
                                                   const T *__restrict__ Pinv, T *__restrict__ Z) {
    __shared__ T As[SG_K][SG_T + 1];
    __shared__ T Bs[SG_K][SG_T + 1];
    const int r0 = blockIdx.y * SG_T, v0 = blockIdx.x * SG_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < nV; k0 += SG_K) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int idx = threadIdx.x + i * 256;
            int rr = idx >> 4, kk = idx & 15;
            int gr = r0 + rr, gk = k0 + kk, gv = v0 + rr;
            As[kk][rr] = (gr < rows && gk < nV) ? Q[(long long)gr * nVp + gk] : T(0);
            Bs[kk][rr] = (gv < nV && gk < nV) ? Pinv[(long long)gv * nVp + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SG_K; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gr = r0 + ty * 4 + i;
        if (gr >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gv = v0 + tx * 4 + j;
            if (gv < nV) Z[(long long)gr * nVp + gv] = acc[i][j];
        }
    }
}

// Gauss-Jordan pivot k on the n x n matrix A (row major): save the scaled
// pivot row and the pivot column, then update every entry.
__global__ void k_gj_prep(int n, int k, const double *A, double *rowk, double *colk, int *bad) {
    const double p = A[(long long)k * n + k];
    if (!(p > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *bad = 1;
        return;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        rowk[j] = (j == k ? 1.0 : A[(long long)k * n + j]) / p;
        colk[j] = (j == k) ? 0.0 : A[(long long)j * n + k];
    }
}

__global__ void k_gj_update(int n, int k, double *A, const double *rowk, const double *colk, const int *bad) {
    if (*bad) return;
    long long total = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
        if (i == k) A[idx] = rowk[j];
        else A[idx] = (j == k ? 0.0 : A[idx]) - colk[i] * rowk[j];
    }
}

// dense n x n FP64 -> padded [n][nVp] copies (FP64, FP32, BF16; null = skip)
__global__ void k_convert_pinv(int n, int nVp, const double *A, double *P64, float *P32, __nv_bfloat16 *P16,
                               __nv_bfloat16 *P16lo, float *P32lo) {
    long long total = (long long)n * nVp;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx / nVp), j = (int)(idx - (long long)i * nVp);
        double v = j < n ? 0.5 * (A[(long long)i * n + j] + A[(long long)j * n + i]) : 0.0;
        if (P64) P64[idx] = v;
        if (P32) P32[idx] = P32lo ? tf32_hi((float)v) : (float)v;
        if (P32lo) P32lo[idx] = (float)(v - (double)P32[idx]);   // TF32 split: low part
        if (P16) P16[idx] = __float2bfloat16_rn((float)v);
        if (P16lo) {   // low part: v - hi, rounded to BF16 (hi + lo carries ~16 bits)
            const double hi = (double)__bfloat162float(__float2bfloat16_rn((float)v));
            P16lo[idx] = __float2bfloat16_rn((float)(v - hi));
        }
    }
}

}  // namespace npfem
