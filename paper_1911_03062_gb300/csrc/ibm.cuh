// ibm.cuh -- immersed-boundary forces by multi-direct forcing (arXiv 1911.03062,
// supplementary IBM section, after Wang et al. and Ota et al.): the Lagrangian
// points are the vertices of every cell (positions x_n, velocities v_n, areas
// A_k = a third of the incident triangles' areas), the fluid velocity u* lives
// on a lattice of nodes x0 + (i, j, k) dx, and Peskin's four-point function
// phi4 (support 4 dx per axis) interpolates and spreads:
//
//   u(X)  = sum_x u(x) phi4 phi4 phi4,      F(x) = sum_k f_k phi4 phi4 phi4 / dx^2
//   f_0   = (U - u*(X)) A / dt
//   cycle: F = spread(f); f += (U - (u* + F dt)(X)) A / dt
//   F_imm = spread(f_C)
//
// (a point stands for the shell volume A dx; nodes outside the lattice are left
// out).  One call: k_ibm_init computes each point's stencil (first node and the
// 12 weights, kept for the call: 108 bytes per point) and f_0; then per cycle
// k_ibm_spread (FP64 atomics into F) and k_ibm_update; then the final spread.
// FP64 throughout: the state is FP64 and the weights are computed once.
#pragma once

#include "common.cuh"
#include "contact.cuh"

namespace npfem {

struct IbmLattice {
    int nx, ny, nz;
    double dx, x0, y0, z0;
};

// Peskin's four-point function
__device__ __forceinline__ double phi4(double r) {
    const double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
    return 0.0;
}

struct IbmPoint {                // a point's stencil: first node per axis and the weights
    double w[3][4];
    int first[3];
    int pad;
};

// u at a point: sum over the stencil of (u* + F dt) weights (F may be null)
__device__ __forceinline__ void ibm_interp(const IbmLattice &L, const double *__restrict__ u,
                                           const double *__restrict__ F, double dt, const IbmPoint &s,
                                           double out[3]) {
    const long long nn = (long long)L.nx * L.ny * L.nz;
    out[0] = out[1] = out[2] = 0.0;
    for (int k = 0; k < 4; ++k) {
        const int iz = s.first[2] + k;
        if (iz < 0 || iz >= L.nz) continue;
        for (int j = 0; j < 4; ++j) {
            const int iy = s.first[1] + j;
            if (iy < 0 || iy >= L.ny) continue;
            const double wyz = s.w[1][j] * s.w[2][k];
            for (int i = 0; i < 4; ++i) {
                const int ix = s.first[0] + i;
                if (ix < 0 || ix >= L.nx) continue;
                const long long n = ((long long)iz * L.ny + iy) * L.nx + ix;
                const double wt = s.w[0][i] * wyz;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double uv = u[c * nn + n];
                    if (F) uv += F[c * nn + n] * dt;
                    out[c] += uv * wt;
                }
            }
        }
    }
}

// stencils, areas and f_0 for the points of type ti (flat index vbase + cell nV + v);
// f in the public layout
__global__ void k_ibm_init(const PikTypes T, int ti, IbmLattice L, const double *__restrict__ u, double dt,
                           IbmPoint *__restrict__ st, double *__restrict__ area, double *__restrict__ f) {
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
        const double *x = P.xn + (long long)cell * 3 * P.nVp;
        const double X[3] = {x[v], x[P.nVp + v], x[2 * P.nVp + v]};
        const double o[3] = {L.x0, L.y0, L.z0};
        IbmPoint s;
        for (int d = 0; d < 3; ++d) {
            const double q = (X[d] - o[d]) / L.dx;
            const int i0 = (int)floor(fmin(fmax(q, -1e9), 1e9)) - 1;   // far outside: no node in range
            s.first[d] = i0;
            for (int j = 0; j < 4; ++j) s.w[d][j] = phi4(q - (double)(i0 + j));
        }
        s.pad = 0;
        double a = 0.0;                              // a third of the incident triangles' areas
        for (int k = P.ring_ptr[v]; k < P.ring_ptr[v + 1]; ++k) {
            const int vb = P.ring_bc[k] & 0xffff, vc = P.ring_bc[k] >> 16;
            const double b0 = x[vb] - X[0], b1 = x[P.nVp + vb] - X[1], b2 = x[2 * P.nVp + vb] - X[2];
            const double c0 = x[vc] - X[0], c1 = x[P.nVp + vc] - X[1], c2 = x[2 * P.nVp + vc] - X[2];
            const double n0 = b1 * c2 - b2 * c1, n1 = b2 * c0 - b0 * c2, n2 = b0 * c1 - b1 * c0;
            a += 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        }
        a /= 3.0;
        const long long flat = P.vbase + i;
        st[flat] = s;
        area[flat] = a;
        double ui[3];
        ibm_interp(L, u, nullptr, dt, s, ui);
        const double *vv = P.vn + (long long)cell * 3 * P.nVp;
        double *fo = f + P.pub_off[cell] + 3 * P.vpub[v];
        for (int c = 0; c < 3; ++c) fo[c] = (vv[c * P.nVp + v] - ui[c]) * a / dt;
    }
}

// F += f_k phi phi phi / dx^2 over each point's stencil (F zeroed before)
__global__ void k_ibm_spread(const PikTypes T, int ti, IbmLattice L, const IbmPoint *__restrict__ st,
                             const double *__restrict__ f, double *__restrict__ F) {
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV, nn = (long long)L.nx * L.ny * L.nz;
    const double sc = 1.0 / (L.dx * L.dx);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
        const IbmPoint s = st[P.vbase + i];
        const double *fi = f + P.pub_off[cell] + 3 * P.vpub[v];
        const double f0 = fi[0] * sc, f1 = fi[1] * sc, f2 = fi[2] * sc;
        for (int k = 0; k < 4; ++k) {
            const int iz = s.first[2] + k;
            if (iz < 0 || iz >= L.nz) continue;
            for (int j = 0; j < 4; ++j) {
                const int iy = s.first[1] + j;
                if (iy < 0 || iy >= L.ny) continue;
                const double wyz = s.w[1][j] * s.w[2][k];
                for (int q = 0; q < 4; ++q) {
                    const int ix = s.first[0] + q;
                    if (ix < 0 || ix >= L.nx) continue;
                    const long long node = ((long long)iz * L.ny + iy) * L.nx + ix;
                    const double wt = s.w[0][q] * wyz;
                    atomicAdd(F + node, f0 * wt);
                    atomicAdd(F + nn + node, f1 * wt);
                    atomicAdd(F + 2 * nn + node, f2 * wt);
                }
            }
        }
    }
}

// f += (U - (u* + F dt)(X)) A / dt
__global__ void k_ibm_update(const PikTypes T, int ti, IbmLattice L, const double *__restrict__ u,
                             const double *__restrict__ F, double dt, const IbmPoint *__restrict__ st,
                             const double *__restrict__ area, double *__restrict__ f) {
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
        const long long flat = P.vbase + i;
        const IbmPoint s = st[flat];
        double ui[3];
        ibm_interp(L, u, F, dt, s, ui);
        const double a = area[flat];
        const double *vv = P.vn + (long long)cell * 3 * P.nVp;
        double *fo = f + P.pub_off[cell] + 3 * P.vpub[v];
        for (int c = 0; c < 3; ++c) fo[c] += (vv[c * P.nVp + v] - ui[c]) * a / dt;
    }
}

}  // namespace npfem
