// gemm_simt.cuh -- FP64 (and FP32) CUDA-core kernels of the global step and
// of the one-time set-up:
//   * k_gemm_simt : Z[r][v] = sum_k Q[r][k] Pinv[v][k], the plain FP64 apply of
//                   P^{-1} to all stacked right-hand sides (the comparison form);
//   * k_bgj_*     : in-place blocked Gauss-Jordan inversion of the SPD matrix P in
//                   FP64, 32 pivots per launch pair (no pivoting: P is SPD and
//                   strongly diagonally dominant through M/h^2);
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
// Blocked Gauss-Jordan inverse of an SPD matrix in place (no pivoting: the Schur
// complements of an SPD matrix keep positive pivots), A: [npad][npad] FP64 with
// npad a multiple of GJB; rows/columns beyond n carry the identity.  For each
// block column kb, with D = A_kk^{-1}, C = A[:, kb] and R = A[kb, :] (old values):
//   A_kk = D,  A_kj = D R_j,  A_ik = -C_i D,  A_ij -= C_i (D R_j)   (i, j != kb)
// -- the same eliminations as the pivot-by-pivot form, GJB pivots per launch pair.
// k_bgj_panel (one block per column tile b): D by an in-shared-memory Gauss-Jordan
// (every block computes it; block 0 stores it), DR_b = D R_b and the copy C_b.
// k_bgj_update (one block per tile): the four cases above.  A pivot <= 0 sets *bad.
// Both run with 256 threads.
constexpr int GJB = 32;

__global__ void __launch_bounds__(256) k_bgj_panel(int npad, int kb, const double *__restrict__ A,
                                                   double *__restrict__ D, double *__restrict__ C,
                                                   double *__restrict__ DR, int *bad) {
    __shared__ double M[GJB][GJB + 1], R[GJB][GJB + 1];
    const int b = blockIdx.x, t = threadIdx.x;
    const long long k0 = (long long)kb * GJB, b0 = (long long)b * GJB;
    for (int e = t; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        M[i][j] = A[(k0 + i) * npad + k0 + j];
        R[i][j] = A[(k0 + i) * npad + b0 + j];
        C[(b0 + i) * GJB + j] = A[(b0 + i) * npad + k0 + j];
    }
    constexpr int PER = GJB * GJB / 256;                   // elements per thread (launched with 256)
    double nv[PER];
    for (int p = 0; p < GJB; ++p) {
        __syncthreads();
        const double piv = M[p][p];
        if (!(piv > 0.0)) {
            if (t == 0) *bad = 1;
            return;                                        // uniform: every thread read the same pivot
        }
        const double ip = 1.0 / piv;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = t + 256 * r, i = e / GJB, j = e % GJB;
            if (i == p) nv[r] = (j == p) ? ip : M[p][j] * ip;
            else if (j == p) nv[r] = -M[i][p] * ip;
            else nv[r] = M[i][j] - M[i][p] * M[p][j] * ip;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) M[(t + 256 * r) / GJB][(t + 256 * r) % GJB] = nv[r];
    }
    __syncthreads();
    for (int e = t; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        if (b == 0) D[e] = M[i][j];
        double s = 0.0;
#pragma unroll 8
        for (int l = 0; l < GJB; ++l) s = fma(M[i][l], R[l][j], s);
        DR[(long long)i * npad + b0 + j] = s;
    }
}

__global__ void __launch_bounds__(256) k_bgj_update(int npad, int kb, double *__restrict__ A,
                                                    const double *__restrict__ D, const double *__restrict__ C,
                                                    const double *__restrict__ DR, const int *bad) {
    if (*bad) return;
    __shared__ double Cs[GJB][GJB + 1], X[GJB][GJB + 1];
    const int ti = blockIdx.y, tj = blockIdx.x, t = threadIdx.x;
    const long long i0 = (long long)ti * GJB, j0 = (long long)tj * GJB;
    if (ti == kb) {
        for (int e = t; e < GJB * GJB; e += blockDim.x) {
            const int i = e / GJB, j = e % GJB;
            A[(i0 + i) * npad + j0 + j] = (tj == kb) ? D[e] : DR[(long long)i * npad + j0 + j];
        }
        return;
    }
    for (int e = t; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        Cs[i][j] = C[(i0 + i) * GJB + j];
        X[i][j] = (tj == kb) ? D[e] : DR[(long long)i * npad + j0 + j];
    }
    __syncthreads();
    for (int e = t; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        double s = 0.0;
#pragma unroll 8
        for (int l = 0; l < GJB; ++l) s = fma(Cs[i][l], X[l][j], s);
        double &a = A[(i0 + i) * npad + j0 + j];
        a = (tj == kb) ? -s : a - s;
    }
}

// dense FP64 [n][lda] -> padded [n][nVp] copies (FP64, FP32, BF16; null = skip)
__global__ void k_convert_pinv(int n, int lda, int nVp, const double *A, double *P64, float *P32, __nv_bfloat16 *P16,
                               __nv_bfloat16 *P16lo, float *P32lo) {
    long long total = (long long)n * nVp;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx / nVp), j = (int)(idx - (long long)i * nVp);
        double v = j < n ? 0.5 * (A[(long long)i * lda + j] + A[(long long)j * lda + i]) : 0.0;
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
