// filters.cuh -- steps either side of the npFEM step (arXiv 1911.03062,
// Sec. 2.2): the one-ring median filter of the external forces (before the
// step) and the cap on vertex velocities (after it).
//
//   median : the force of vertex v becomes, per component, the median of the
//            forces of v and of its edge neighbours (closed one-ring); for an
//            even count the mean of the two middle values.  Selection on
//            order-preserving integer keys and one FP64 mean: exact.
//   cap    : |v| > u_max -> v u_max / |v| (direction kept), on the FP64 state.
//   PBD    : position-based-dynamics velocity damping (below), before the cap.
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

// Position-based-dynamics velocity damping (Mueller et al. 2007, Sec. 3.5), on
// the FP64 state after the step: per cell x_cm, v_cm, L = sum r x m v,
// I = sum m (|r|^2 E - r r^T), omega = I^{-1} L, then v += kappa (v_cm + omega x r - v).
// One block per cell (grid-stride), two FP64 block reductions, thread 0 inverts
// I by its adjugate (omega = 0 if I is singular).  mass: [nV] lumped masses.
__global__ void __launch_bounds__(256) k_pbd_damping(int ncells, int nV, int nVp, const double *__restrict__ mass,
                                                     const double *__restrict__ xn, double *vn, double kappa) {
    __shared__ double red[32 * 9];
    __shared__ double bc[9];   // x_cm, v_cm, omega
    for (int cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
        const double *x = xn + (long long)cell * 3 * nVp;
        double *v = vn + (long long)cell * 3 * nVp;
        Acc<double> a[7];
        for (int i = 0; i < 7; ++i) a[i].zero();
        for (int i = threadIdx.x; i < nV; i += blockDim.x) {
            const double m = mass[i];
            a[0].add(m);
            for (int c = 0; c < 3; ++c) {
                a[1 + c].add(m * x[c * nVp + i]);
                a[4 + c].add(m * v[c * nVp + i]);
            }
        }
        block_reduce_t0<double, 7>(a, red, [&](const double *s) {
            for (int c = 0; c < 3; ++c) {
                bc[c] = s[1 + c] / s[0];
                bc[3 + c] = s[4 + c] / s[0];
            }
        });
        Acc<double> b[9];   // L0 L1 L2 I00 I01 I02 I11 I12 I22
        for (int i = 0; i < 9; ++i) b[i].zero();
        for (int i = threadIdx.x; i < nV; i += blockDim.x) {
            const double m = mass[i];
            const double r0 = x[i] - bc[0], r1 = x[nVp + i] - bc[1], r2 = x[2 * nVp + i] - bc[2];
            const double p0 = m * v[i], p1 = m * v[nVp + i], p2 = m * v[2 * nVp + i];
            b[0].add(r1 * p2 - r2 * p1);
            b[1].add(r2 * p0 - r0 * p2);
            b[2].add(r0 * p1 - r1 * p0);
            const double rr = r0 * r0 + r1 * r1 + r2 * r2;
            b[3].add(m * (rr - r0 * r0));
            b[4].add(-m * r0 * r1);
            b[5].add(-m * r0 * r2);
            b[6].add(m * (rr - r1 * r1));
            b[7].add(-m * r1 * r2);
            b[8].add(m * (rr - r2 * r2));
        }
        block_reduce_t0<double, 9>(b, red, [&](const double *s) {
            const double I[9] = {s[3], s[4], s[5], s[4], s[6], s[7], s[5], s[7], s[8]};
            double C[9];
            C[0] = I[4] * I[8] - I[5] * I[7]; C[1] = I[2] * I[7] - I[1] * I[8]; C[2] = I[1] * I[5] - I[2] * I[4];
            C[3] = I[5] * I[6] - I[3] * I[8]; C[4] = I[0] * I[8] - I[2] * I[6]; C[5] = I[2] * I[3] - I[0] * I[5];
            C[6] = I[3] * I[7] - I[4] * I[6]; C[7] = I[1] * I[6] - I[0] * I[7]; C[8] = I[0] * I[4] - I[1] * I[3];
            const double det = I[0] * C[0] + I[1] * C[3] + I[2] * C[6];
            for (int r = 0; r < 3; ++r)
                bc[6 + r] = fabs(det) > 0 ? (C[3 * r] * s[0] + C[3 * r + 1] * s[1] + C[3 * r + 2] * s[2]) / det : 0.0;
        });
        for (int i = threadIdx.x; i < nV; i += blockDim.x) {
            const double r0 = x[i] - bc[0], r1 = x[nVp + i] - bc[1], r2 = x[2 * nVp + i] - bc[2];
            const double w0 = bc[6], w1 = bc[7], w2 = bc[8];
            const double g0 = bc[3] + w1 * r2 - w2 * r1, g1 = bc[4] + w2 * r0 - w0 * r2, g2 = bc[5] + w0 * r1 - w1 * r0;
            v[i] += kappa * (g0 - v[i]);
            v[nVp + i] += kappa * (g1 - v[nVp + i]);
            v[2 * nVp + i] += kappa * (g2 - v[2 * nVp + i]);
        }
        __syncthreads();
    }
}

// The same damping for the mixed forms: coordinates relative to vertex 0 are
// formed in FP64 and carried in FP32, moments are float-float sums, omega is
// formed in FP64 from them by thread 0, and only the velocity update touches
// FP64 (GB300 runs FP64 at ~1/64 of FP32).  Velocity change error ~1e-7 of
// itself.  inv_mtot: 1 / total mass of the type.
__global__ void __launch_bounds__(256) k_pbd_damping_f32(int ncells, int nV, int nVp, const double *__restrict__ mass,
                                                         double inv_mtot, const double *__restrict__ xn, double *vn,
                                                         float kappa) {
    __shared__ double red[32 * 9];
    __shared__ float bc[9];   // x_cm - x_0, v_cm, omega
    for (int cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
        const double *x = xn + (long long)cell * 3 * nVp;
        double *v = vn + (long long)cell * 3 * nVp;
        const double x00 = x[0], x01 = x[nVp], x02 = x[2 * nVp];
        Acc<float> a[6];
        for (int i = 0; i < 6; ++i) a[i].zero();
        for (int i = threadIdx.x; i < nV; i += blockDim.x) {
            const float m = (float)mass[i];
            a[0].add_prod(m, (float)(x[i] - x00));
            a[1].add_prod(m, (float)(x[nVp + i] - x01));
            a[2].add_prod(m, (float)(x[2 * nVp + i] - x02));
            a[3].add_prod(m, (float)v[i]);
            a[4].add_prod(m, (float)v[nVp + i]);
            a[5].add_prod(m, (float)v[2 * nVp + i]);
        }
        block_reduce_t0<float, 6>(a, red, [&](const double *s) {
            for (int c = 0; c < 6; ++c) bc[c] = (float)(s[c] * inv_mtot);
        });
        Acc<float> b[9];   // L0 L1 L2 I00 I01 I02 I11 I12 I22
        for (int i = 0; i < 9; ++i) b[i].zero();
        for (int i = threadIdx.x; i < nV; i += blockDim.x) {
            const float m = (float)mass[i];
            const float r0 = (float)(x[i] - x00) - bc[0], r1 = (float)(x[nVp + i] - x01) - bc[1],
                        r2 = (float)(x[2 * nVp + i] - x02) - bc[2];
            const float p0 = m * (float)v[i], p1 = m * (float)v[nVp + i], p2 = m * (float)v[2 * nVp + i];
            b[0].add(r1 * p2 - r2 * p1);
            b[1].add(r2 * p0 - r0 * p2);
            b[2].add(r0 * p1 - r1 * p0);
            b[3].add(m * (r1 * r1 + r2 * r2));
            b[4].add(-m * r0 * r1);
            b[5].add(-m * r0 * r2);
            b[6].add(m * (r0 * r0 + r2 * r2));
            b[7].add(-m * r1 * r2);
            b[8].add(m * (r0 * r0 + r1 * r1));
        }
        block_reduce_t0<float, 9>(b, red, [&](const double *s) {
            const double I[9] = {s[3], s[4], s[5], s[4], s[6], s[7], s[5], s[7], s[8]};
            double C[9];
            C[0] = I[4] * I[8] - I[5] * I[7]; C[1] = I[2] * I[7] - I[1] * I[8]; C[2] = I[1] * I[5] - I[2] * I[4];
            C[3] = I[5] * I[6] - I[3] * I[8]; C[4] = I[0] * I[8] - I[2] * I[6]; C[5] = I[2] * I[3] - I[0] * I[5];
            C[6] = I[3] * I[7] - I[4] * I[6]; C[7] = I[1] * I[6] - I[0] * I[7]; C[8] = I[0] * I[4] - I[1] * I[3];
            const double det = I[0] * C[0] + I[1] * C[3] + I[2] * C[6];
            for (int r = 0; r < 3; ++r)
                bc[6 + r] = fabs(det) > 0 ? (float)((C[3 * r] * s[0] + C[3 * r + 1] * s[1] + C[3 * r + 2] * s[2]) / det) : 0.f;
        });
        for (int i = threadIdx.x; i < nV; i += blockDim.x) {
            const float r0 = (float)(x[i] - x00) - bc[0], r1 = (float)(x[nVp + i] - x01) - bc[1],
                        r2 = (float)(x[2 * nVp + i] - x02) - bc[2];
            const float w0 = bc[6], w1 = bc[7], w2 = bc[8];
            const float g0 = bc[3] + w1 * r2 - w2 * r1, g1 = bc[4] + w2 * r0 - w0 * r2, g2 = bc[5] + w0 * r1 - w1 * r0;
            v[i] += (double)(kappa * (g0 - (float)v[i]));
            v[nVp + i] += (double)(kappa * (g1 - (float)v[nVp + i]));
            v[2 * nVp + i] += (double)(kappa * (g2 - (float)v[2 * nVp + i]));
        }
        __syncthreads();
    }
}

}  // namespace npfem
