// filters.cuh -- steps either side of the npFEM step (arXiv 1911.03062,
// Sec. 2.2): the one-ring median filter of the external forces (before the
// step) and the cap on vertex velocities (after it).
//
//   median : the force of vertex v becomes, per component, the median of the
//            forces of v and of its edge neighbours (closed one-ring); for an
//            even count the mean of the two middle values.  Selection on
//            order-preserving integer keys and one FP64 mean: exact.
//   cap    : |v| > u_max -> v u_max / |v| (direction kept), on the FP64 state.
#pragma once

#include "common.cuh"

namespace npfem {

constexpr int MEDIAN_FAST = 8;    // closed one-rings up to this size sort in registers
constexpr int MEDIAN_MAX = 32;    // largest closed one-ring accepted

// Order-preserving map of a double to a signed 64-bit key (involution): the
// comparisons of the selection run on the integer pipe, exactly.
__device__ __forceinline__ long long order_key(long long b) { return b ^ ((b >> 63) & 0x7fffffffffffffffll); }

// median of the first n of k[0..N) (the rest the largest key), compare-exchange network
template <int N>
__device__ __forceinline__ double median_keys(long long (&k)[N], int n) {
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int i = (r & 1); i + 1 < N; i += 2) {
            const long long a = k[i], b = k[i + 1];
            k[i] = a < b ? a : b;
            k[i + 1] = a < b ? b : a;
        }
    long long lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i == (n - 1) / 2) lo = k[i];
        if (i == n / 2) hi = k[i];
    }
    const double vh = __longlong_as_double(order_key(hi));
    return (n & 1) ? vh : 0.5 * (__longlong_as_double(order_key(lo)) + vh);
}

// One block per cell (grid-stride): the cell's forces (public layout, the
// caller's vertex numbering) are staged in shared memory by coalesced loads,
// each thread filters vertices tid, tid + B, ... (internal numbering) and the
// result leaves through shared memory by coalesced stores.  Dynamic shared
// memory: 2 x 3 nV doubles.
__global__ void __launch_bounds__(256) k_force_median(int ncells, int nV, const long long *__restrict__ pub_off,
                                                      const int *__restrict__ vpub, const int *__restrict__ adj_ptr,
                                                      const int *__restrict__ adj, const double *const *fslot,
                                                      double *out) {
    extern __shared__ __align__(16) unsigned char smem_med[];
    double *fin = reinterpret_cast<double *>(smem_med), *fout = fin + 3 * nV;
    const double *f = *fslot;
    const int n3 = 3 * nV;
    for (int cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
        const double *fc = f + pub_off[cell];
        for (int i = threadIdx.x; i < n3; i += blockDim.x) fin[i] = fc[i];
        __syncthreads();
        for (int v = threadIdx.x; v < nV; v += blockDim.x) {
            const int b = adj_ptr[v], n = adj_ptr[v + 1] - b + 1, pv = 3 * vpub[v];
            for (int c = 0; c < 3; ++c) {
                double med;
                if (n <= MEDIAN_FAST) {
                    long long k[MEDIAN_FAST];
#pragma unroll
                    for (int j = 0; j < MEDIAN_FAST; ++j)
                        k[j] = j == 0 ? order_key(__double_as_longlong(fin[pv + c]))
                                      : (j < n ? order_key(__double_as_longlong(fin[3 * vpub[adj[b + j - 1]] + c]))
                                               : 0x7fffffffffffffffll);
                    med = median_keys<MEDIAN_FAST>(k, n);
                } else {
                    long long k[MEDIAN_MAX];
                    k[0] = order_key(__double_as_longlong(fin[pv + c]));
                    for (int j = 1; j < n; ++j) k[j] = order_key(__double_as_longlong(fin[3 * vpub[adj[b + j - 1]] + c]));
                    for (int j = 1; j < n; ++j) {       // insertion sort
                        const long long x = k[j];
                        int i = j - 1;
                        while (i >= 0 && k[i] > x) { k[i + 1] = k[i]; --i; }
                        k[i + 1] = x;
                    }
                    const double vh = __longlong_as_double(order_key(k[n / 2]));
                    med = (n & 1) ? vh : 0.5 * (__longlong_as_double(order_key(k[n / 2 - 1])) + vh);
                }
                fout[pv + c] = med;
            }
        }
        __syncthreads();
        double *oc = out + pub_off[cell];
        for (int i = threadIdx.x; i < n3; i += blockDim.x) oc[i] = fout[i];
        __syncthreads();
    }
}

// One thread per (cell, vertex) of the FP64 SoA velocities [cell][3][nVp].
__global__ void k_vel_cap(int ncells, int nV, int nVp, double *vn, double umax) {
    const long long total = (long long)ncells * nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / nV), v = (int)(i - (long long)cell * nV);
        double *p = vn + (long long)cell * 3 * nVp + v;
        const double a = p[0], b = p[nVp], c = p[2 * nVp];
        const double s2 = a * a + b * b + c * c;
        if (s2 <= umax * umax * (1.0 - 1e-12)) continue;      // clearly below: no square root
        const double n = sqrt(s2);
        if (n > umax) {
            const double s = umax / n;
            p[0] = a * s;
            p[nVp] = b * s;
            p[2 * nVp] = c * s;
        }
    }
}

}  // namespace npfem
