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
// k_ibm_spread_box (FP64 atomics into F, aggregated per block in shared memory),
// k_ibm_correct (F <- u* + F dt at the nodes, so the re-interpolation reads one
// field) and k_ibm_update; then the final spread.
// FP64 throughout: the state is FP64 and the weights are computed once.
#pragma once

#include "common.cuh"
#include "contact.cuh"

namespace npfem {

struct IbmLattice {
    int nx, ny, nz;
    double dx, x0, y0, z0;
};

// Peskin's four-point function at the offsets r + 1, r, r - 1, r - 2 of a point
// with fractional grid position r in [0, 1): the four branches share one square
// root, s = sqrt(1 + 4r - 4r^2) (the arguments of the |r| <= 1 and 1 <= |r| <= 2
// branches at these offsets reduce to it), so
//   phi(r+1) = (3 - 2r - s)/8, phi(r) = (3 - 2r + s)/8,
//   phi(r-1) = (1 + 2r + s)/8, phi(r-2) = (1 + 2r - s)/8.
__device__ __forceinline__ void phi4_weights(double r, double w[4]) {
    const double s = sqrt(1.0 + 4.0 * r - 4.0 * r * r);
    w[0] = (3.0 - 2.0 * r - s) * 0.125;
    w[1] = (3.0 - 2.0 * r + s) * 0.125;
    w[2] = (1.0 + 2.0 * r + s) * 0.125;
    w[3] = (1.0 + 2.0 * r - s) * 0.125;
}

struct IbmPoint {                // a point's stencil: first node per axis and the weights
    double w[3][4];
    int first[3];
    int pad;
};

// u at a point: the weighted sum over its stencil
__device__ __forceinline__ void ibm_interp(const IbmLattice &L, const double *__restrict__ u, const IbmPoint &s,
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
                for (int c = 0; c < 3; ++c) out[c] += u[c * nn + n] * wt;
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
            const double q = fmin(fmax((X[d] - o[d]) / L.dx, -1e9), 1e9);   // far outside: no node in range
            const double fq = floor(q);
            s.first[d] = (int)fq - 1;
            phi4_weights(q - fq, s.w[d]);
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
        ibm_interp(L, u, s, ui);
        const double *vv = P.vn + (long long)cell * 3 * P.nVp;
        double *fo = f + P.pub_off[cell] + 3 * P.vpub[v];
        for (int c = 0; c < 3; ++c) fo[c] = (vv[c * P.nVp + v] - ui[c]) * a / dt;
    }
}

// F += f_k phi phi phi / dx^2 over each point's stencil (F zeroed before), aggregated
// per block: the block's points (consecutive vertices of a cell, so their stencils
// overlap) first add into a shared-memory box of the lattice nodes their stencils
// cover, which is then flushed with one global atomic per non-zero node and
// component instead of one per point, node and component.  Blocks whose box exceeds
// the shared memory (points far apart) add straight into F.  Dynamic shared
// memory: IBM_BOX_DOUBLES doubles.
constexpr int IBM_BOX_DOUBLES = 8192;    // 64 KB: 3 components of up to 2730 nodes

__global__ void __launch_bounds__(256) k_ibm_spread_box(const PikTypes T, int ti, IbmLattice L,
                                                        const IbmPoint *__restrict__ st,
                                                        const double *__restrict__ f, double *__restrict__ F) {
    extern __shared__ double box[];
    __shared__ int lo_sh[3], hi_sh[3];
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV, nn = (long long)L.nx * L.ny * L.nz;
    const double sc = 1.0 / (L.dx * L.dx);
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < n; b0 += (long long)gridDim.x * blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const bool on = i < n;
        IbmPoint s;
        double fv[3] = {0.0, 0.0, 0.0};
        if (on) {
            const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
            s = st[P.vbase + i];
            const double *fi = f + P.pub_off[cell] + 3 * P.vpub[v];
            fv[0] = fi[0] * sc;
            fv[1] = fi[1] * sc;
            fv[2] = fi[2] * sc;
        }
        if (threadIdx.x < 3) { lo_sh[threadIdx.x] = INT_MAX; hi_sh[threadIdx.x] = INT_MIN; }
        __syncthreads();
        if (on)
            for (int d = 0; d < 3; ++d) {
                atomicMin(lo_sh + d, s.first[d]);
                atomicMax(hi_sh + d, s.first[d] + 3);
            }
        __syncthreads();
        const int bx = lo_sh[0], by = lo_sh[1], bz = lo_sh[2];
        const long long ex = (long long)hi_sh[0] - bx + 1, ey = (long long)hi_sh[1] - by + 1,
                        ez = (long long)hi_sh[2] - bz + 1;
        // each extent bounded before the product (stencils far outside the lattice can span ~1e9)
        const bool small = ex <= IBM_BOX_DOUBLES && ey <= IBM_BOX_DOUBLES && ez <= IBM_BOX_DOUBLES;
        const long long nb = small ? ex * ey * ez : 0;
        const bool tiled = small && nb > 0 && 3 * nb <= IBM_BOX_DOUBLES;
        if (tiled)
            for (long long k = threadIdx.x; k < 3 * nb; k += blockDim.x) box[k] = 0.0;
        __syncthreads();
        if (on) {
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
                        const double wt = s.w[0][q] * wyz;
                        if (tiled) {
                            const long long bnode = ((long long)(iz - bz) * ey + (iy - by)) * ex + (ix - bx);
                            atomicAdd(box + bnode, fv[0] * wt);
                            atomicAdd(box + nb + bnode, fv[1] * wt);
                            atomicAdd(box + 2 * nb + bnode, fv[2] * wt);
                        } else {
                            const long long node = ((long long)iz * L.ny + iy) * L.nx + ix;
                            atomicAdd(F + node, fv[0] * wt);
                            atomicAdd(F + nn + node, fv[1] * wt);
                            atomicAdd(F + 2 * nn + node, fv[2] * wt);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (tiled)
            for (long long k = threadIdx.x; k < 3 * nb; k += blockDim.x) {
                const double val = box[k];
                if (val == 0.0) continue;
                const long long c = k / nb, r = k - c * nb;
                const long long zz = r / (ex * ey), yy = (r / ex) % ey, xx = r % ex;
                const long long node = ((zz + bz) * L.ny + (yy + by)) * L.nx + (xx + bx);   // in range: only
                atomicAdd(F + c * nn + node, val);                                            // added nodes are non-zero
            }
        __syncthreads();
    }
}

// the corrected velocity at every node, in place: F <- u* + F dt
__global__ void k_ibm_correct(long long n3, const double *__restrict__ u, double *__restrict__ F, double dt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
        F[i] = u[i] + F[i] * dt;
}

// f += (U - uc(X)) A / dt, uc = u* + F dt formed at the nodes by k_ibm_correct
__global__ void k_ibm_update(const PikTypes T, int ti, IbmLattice L, const double *__restrict__ uc, double dt,
                             const IbmPoint *__restrict__ st,
                             const double *__restrict__ area, double *__restrict__ f) {
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
        const long long flat = P.vbase + i;
        const IbmPoint s = st[flat];
        double ui[3];
        ibm_interp(L, uc, s, ui);
        const double a = area[flat];
        const double *vv = P.vn + (long long)cell * 3 * P.nVp;
        double *fo = f + P.pub_off[cell] + 3 * P.vpub[v];
        for (int c = 0; c < 3; ++c) fo[c] += (vv[c * P.nVp + v] - ui[c]) * a / dt;
    }
}

}  // namespace npfem
