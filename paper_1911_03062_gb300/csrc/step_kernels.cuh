// step_kernels.cuh -- per-cell kernels of one npFEM time step (arXiv
// 1911.03062, Supplementary Sec. 2.1): the inertial predictor, the fused
// quasi-Newton iteration (L-BFGS second loop -> direction -> Armijo line
// search over local steps -> history update -> L-BFGS first loop), the
// descent fallback apply, the FP64 refinement residual of the global step,
// and the public <-> internal layout conversions.
//
// Internal layout of every per-cell vector: SoA [cell][3][nVp] (component
// major, vertex contiguous, nVp = nV rounded up to 8, padding kept zero).
// One thread block owns one cell at a time (grid-stride over cells).
#pragma once

#include "local.cuh"

namespace npfem {

template <typename T>
struct IterArgs {
    TypeConst<T> tc;
    int ncells, m, max_bt, last, use_allow, stash_T;
    double h, c1;
    double *xn, *vn;              // state, FP64 SoA
    const double *const *fptr;    // device slot holding the f_ext base (public layout)
    const long long *pub_off;     // [cell] offset of the cell in the public arrays (doubles)
    const double *minv;           // [nV] 1 / m_v
    T *yrel;                      // y - origin
    double *origin;               // [cell][3]
    T *delta, *grad, *q, *z;
    __nv_bfloat16 *q_bf16;        // GEMM operand copy of q (BF16 form), or null
    T *S, *Y;                     // history [cell][m][3][nVp]
    double *rho, *alpha;          // [cell][m]
    double *g;                    // [cell] energy at the current iterate
    double *allow;                // [cell] rounding allowance of g (FP32 local step)
    int *hcount, *hhead;          // [cell] ring state
    int *fb_list, *fb_count;      // cells whose direction failed the descent test
    DevStatus *st;
};

template <typename T, int EPT>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, T (&r)[EPT], int n3) {
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        int e = threadIdx.x + j * blockDim.x;
        r[j] = e < n3 ? p[e] : T(0);
    }
}

template <typename T, int EPT>
__device__ __forceinline__ void store_vec(T *__restrict__ p, const T (&r)[EPT], int n3) {
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        int e = threadIdx.x + j * blockDim.x;
        if (e < n3) p[e] = r[j];
    }
}

// y = x_n + h v_n + h^2 M^{-1} F_ext in FP64 for this thread's elements.
template <typename T, int EPT>
__device__ __forceinline__ void predictor64(const IterArgs<T> &a, int cell, double (&y)[EPT], double (&xo)[EPT]) {
    const int nVp = a.tc.nVp, nV = a.tc.nV, n3 = 3 * nVp;
    const double *f = *a.fptr + a.pub_off[cell];
    const long long base = (long long)cell * n3;
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        int e = threadIdx.x + j * blockDim.x, v;
        y[j] = 0.0;
        xo[j] = 0.0;
        if (e >= n3) continue;
        int c = elem_cv(e, nVp, v);
        if (v >= nV) continue;
        double x = a.xn[base + e];
        xo[j] = x;
        y[j] = x + a.h * a.vn[base + e] + a.h * a.h * a.minv[v] * f[3 * v + c];
    }
}

// Start of a step: y, origin (centroid of y), y_rel, delta = 0, history
// cleared, g and grad g at x^0 = y, and q = grad g (the first apply's RHS).
template <typename T, int EPT, int MAXB>
__global__ void __launch_bounds__(MAXB, MAXB <= 256 ? 3 : 1) k_predict(IterArgs<T> a) {
    const Smem<T> S = smem_layout<T>(a.tc.nVp);
    const int nVp = a.tc.nVp, n3 = 3 * nVp;
    for (int cell = blockIdx.x; cell < a.ncells; cell += gridDim.x) {
        const long long base = (long long)cell * n3;
        double y[EPT], xo[EPT];
        predictor64<T, EPT>(a, cell, y, xo);
        // centroid of y, per component
        Acc<double> s[3];
        s[0].zero(); s[1].zero(); s[2].zero();
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = threadIdx.x + j * blockDim.x, v;
            if (e >= n3) continue;
            int c = elem_cv(e, nVp, v);
            if (v >= a.tc.nV) continue;
            s[c].add(y[j]);
        }
        block_reduce_t0<double, 3>(s, S.red, [&](const double *o) {
            for (int c = 0; c < 3; ++c) {
                S.bc->d[c] = o[c] / a.tc.nV;
                a.origin[3 * cell + c] = S.bc->d[c];
            }
        });
        T yr[EPT], dl[EPT], gr[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = threadIdx.x + j * blockDim.x, v;
            yr[j] = T(0);
            dl[j] = T(0);
            if (e >= n3) continue;
            int c = elem_cv(e, nVp, v);
            if (v >= a.tc.nV) continue;
            yr[j] = T(y[j] - S.bc->d[c]);
        }
        store_vec<T, EPT>(a.yrel + base, yr, n3);
        store_vec<T, EPT>(a.delta + base, dl, n3);
        __syncthreads();
        local_eval<T, EPT>(a.tc, a.yrel + base, dl, gr, S, a.stash_T, [&](double g, double allow) {
            a.g[cell] = g;
            a.allow[cell] = allow;
            a.hcount[cell] = 0;
            a.hhead[cell] = 0;
            if (!isfinite(g)) dev_raise(a.st, DEV_ENONFINITE, cell);
        });
        store_vec<T, EPT>(a.grad + base, gr, n3);
        store_vec<T, EPT>(a.q + base, gr, n3);
        if (a.q_bf16) {
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                int e = threadIdx.x + j * blockDim.x;
                if (e < n3) a.q_bf16[base + e] = __float2bfloat16_rn((float)gr[j]);
            }
        }
    }
}

// One quasi-Newton iteration of every listed cell (all cells when list is
// null).  z = P^{-1} q from the global step must be in a.z.
//   second loop : r = z; for i oldest -> newest: beta = rho_i y_i.r; r += s_i (alpha_i - beta)
//   direction   : d = -r; if grad.d >= 0 with history: clear it, queue the cell for
//                 d = -P^{-1} grad (fallback list) and stop here
//   line search : alpha = 1, halve while g(x + alpha d) > g + c1 alpha grad.d
//                 (at most max_bt halvings, then the last trial is taken)
//   history     : s = x_new - x, y = grad_new - grad, kept if s.y > 1e-12 |s||y|
//   last        : x_{n+1} = y + delta, v_{n+1} = (x_{n+1} - x_n)/h  (Eq. vel)
//   otherwise   : first loop  q = grad; for i newest -> oldest: alpha_i = rho_i s_i.q;
//                 q -= alpha_i y_i  -> the next global step's RHS.
// Scalars (dots, coefficients, the Armijo and curvature tests) are formed by
// thread 0 in FP64 and broadcast through shared memory.
template <typename T, int EPT, int MAXB>
__global__ void __launch_bounds__(MAXB, MAXB <= 256 ? 3 : 1) k_iterate(IterArgs<T> a, const int *list,
                                                                      const int *list_count) {
    const Smem<T> S = smem_layout<T>(a.tc.nVp);
    const int nVp = a.tc.nVp, n3 = 3 * nVp, m = a.m;
    const int nitems = list ? *list_count : a.ncells;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int cell = list ? list[item] : item;
        const long long base = (long long)cell * n3;
        T *Sh = a.S + (long long)cell * m * n3;
        T *Yh = a.Y + (long long)cell * m * n3;
        double *rho = a.rho + (long long)cell * m, *alp = a.alpha + (long long)cell * m;
        int cnt = a.hcount[cell], head = a.hhead[cell];
        T r[EPT], d[EPT], gr[EPT], dl[EPT];
        load_vec<T, EPT>(a.z + base, r, n3);
        for (int l = cnt - 1; l >= 0; --l) {
            const int i = ((head - 1 - l) % m + m) % m;
            T yi[EPT], si[EPT];
            load_vec<T, EPT>(Yh + (long long)i * n3, yi, n3);
            load_vec<T, EPT>(Sh + (long long)i * n3, si, n3);
            Acc<T> ac[1];
            ac[0].zero();
#pragma unroll
            for (int j = 0; j < EPT; ++j) ac[0].add_prod(yi[j], r[j]);
            block_reduce_t0<T, 1>(ac, S.red, [&](const double *s) { S.bc->t[0] = T(alp[i] - rho[i] * s[0]); });
            const T coef = S.bc->t[0];
#pragma unroll
            for (int j = 0; j < EPT; ++j) r[j] += si[j] * coef;
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) d[j] = -r[j];
        load_vec<T, EPT>(a.grad + base, gr, n3);
        {
            Acc<T> ac[1];
            ac[0].zero();
#pragma unroll
            for (int j = 0; j < EPT; ++j) ac[0].add_prod(gr[j], d[j]);
            block_reduce_t0<T, 1>(ac, S.red, [&](const double *s) {
                S.bc->d[1] = s[0];                       // grad . d
                S.bc->d[2] = 1.0;                        // alpha
                S.bc->i[2] = 0;                          // halvings
                S.bc->i[1] = (s[0] >= 0.0 && cnt > 0);   // not a descent direction
                if (S.bc->i[1]) {
                    a.hcount[cell] = 0;
                    a.hhead[cell] = 0;
                    a.fb_list[atomicAdd(a.fb_count, 1)] = cell;
                    atomicAdd(&a.st->fallbacks, 1ull);
                }
            });
        }
        if (S.bc->i[1]) {
            store_vec<T, EPT>(a.q + base, gr, n3);
            __syncthreads();
            continue;
        }
        load_vec<T, EPT>(a.delta + base, dl, n3);
        T dt[EPT], gt[EPT];
        T alpha = T(1);
        for (;;) {
#pragma unroll
            for (int j = 0; j < EPT; ++j) dt[j] = dl[j] + alpha * d[j];
            local_eval<T, EPT>(a.tc, a.yrel + base, dt, gt, S, a.stash_T, [&](double g, double allow) {
                const double al = S.bc->d[2], gd = S.bc->d[1];
                const double slack = a.use_allow ? (a.allow[cell] + allow) : 0.0;
                S.bc->d[3] = g;
                S.bc->d[4] = allow;
                if (g <= a.g[cell] + a.c1 * al * gd + slack) {
                    S.bc->i[3] = 1;
                } else if (S.bc->i[2] == a.max_bt) {
                    S.bc->i[3] = 2;
                    atomicAdd(&a.st->capped, 1ull);
                } else {
                    S.bc->i[3] = 0;
                    S.bc->d[2] = 0.5 * al;
                    S.bc->t[2] = T(0.5 * al);
                    S.bc->i[2] += 1;
                }
            });
            if (S.bc->i[3]) break;
            alpha = S.bc->t[2];
        }
        // history pair
        T sv[EPT], yv[EPT];
        Acc<T> h3[3];
        h3[0].zero(); h3[1].zero(); h3[2].zero();
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            sv[j] = dt[j] - dl[j];
            yv[j] = gt[j] - gr[j];
            h3[0].add_prod(sv[j], yv[j]);
            h3[1].add_prod(sv[j], sv[j]);
            h3[2].add_prod(yv[j], yv[j]);
        }
        block_reduce_t0<T, 3>(h3, S.red, [&](const double *hs) {
            const int keep = m > 0 && hs[0] > 1e-12 * sqrt(hs[1]) * sqrt(hs[2]);
            S.bc->i[4] = keep;
            if (keep) rho[head] = 1.0 / hs[0];
            const double gtv = S.bc->d[3];
            a.g[cell] = gtv;
            a.allow[cell] = S.bc->d[4];
            if (S.bc->i[2]) atomicAdd(&a.st->backtracks, (unsigned long long)S.bc->i[2]);
            if (!isfinite(gtv)) dev_raise(a.st, DEV_ENONFINITE, cell);
            if (a.last) atomicAdd(&a.st->energy_sum, gtv);
        });
        if (S.bc->i[4]) {
            store_vec<T, EPT>(Sh + (long long)head * n3, sv, n3);
            store_vec<T, EPT>(Yh + (long long)head * n3, yv, n3);
            head = (head + 1) % m;
            if (cnt < m) ++cnt;
        }
        store_vec<T, EPT>(a.delta + base, dt, n3);
        store_vec<T, EPT>(a.grad + base, gt, n3);
        if (threadIdx.x == 0) {
            a.hcount[cell] = cnt;
            a.hhead[cell] = head;
        }
        if (a.last) {
            double y[EPT], xo[EPT];
            predictor64<T, EPT>(a, cell, y, xo);
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                int e = threadIdx.x + j * blockDim.x;
                if (e >= n3) continue;
                double x = y[j] + (double)dt[j];
                a.xn[base + e] = x;
                a.vn[base + e] = (x - xo[j]) / a.h;
            }
        } else {
            T qv[EPT];
#pragma unroll
            for (int j = 0; j < EPT; ++j) qv[j] = gt[j];
            for (int l = 0; l < cnt; ++l) {
                const int i = ((head - 1 - l) % m + m) % m;
                T si[EPT], yi[EPT];
                load_vec<T, EPT>(Sh + (long long)i * n3, si, n3);
                load_vec<T, EPT>(Yh + (long long)i * n3, yi, n3);
                Acc<T> ac[1];
                ac[0].zero();
#pragma unroll
                for (int j = 0; j < EPT; ++j) ac[0].add_prod(si[j], qv[j]);
                block_reduce_t0<T, 1>(ac, S.red, [&](const double *s) {
                    const double al = rho[i] * s[0];
                    alp[i] = al;
                    S.bc->t[0] = T(al);
                });
                const T ca = S.bc->t[0];
#pragma unroll
                for (int j = 0; j < EPT; ++j) qv[j] -= ca * yi[j];
            }
            store_vec<T, EPT>(a.q + base, qv, n3);
            if (a.q_bf16) {
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    int e = threadIdx.x + j * blockDim.x;
                    if (e < n3) a.q_bf16[base + e] = __float2bfloat16_rn((float)qv[j]);
                }
            }
        }
        __syncthreads();
    }
}

// z = P^{-1} q for the cells of the fallback list, with the full-precision
// inverse (FP64 path: FP64; FP32 path: FP32 copy of the FP64 inverse).
template <typename T>
__global__ void k_fallback_apply(int nV, int nVp, const T *__restrict__ Pinv, const T *__restrict__ q,
                                 T *__restrict__ z, const int *list, const int *count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *qs = reinterpret_cast<T *>(smem_raw);
    const int n3 = 3 * nVp;
    for (int item = blockIdx.x; item < *count; item += gridDim.x) {
        const long long base = (long long)list[item] * n3;
        for (int e = threadIdx.x; e < n3; e += blockDim.x) qs[e] = q[base + e];
        __syncthreads();
        for (int e = threadIdx.x; e < n3; e += blockDim.x) {
            int v, c = elem_cv(e, nVp, v);
            T acc = T(0);
            if (v < nV) {
                const T *row = Pinv + (long long)v * nVp;
                const T *qc = qs + c * nVp;
                for (int k = 0; k < nV; ++k) acc += row[k] * qc[k];
            }
            z[base + e] = acc;
        }
        __syncthreads();
    }
}

// Refinement residual of the global step (mixed forms), r = q - P z with
// P = diag(P) + offdiag(P).  The cancellation sits in q - diag(P) z (r is
// ~1e-3 of q after a BF16 apply), so that part must be exact:
//   FP64R = true : r = (q - diag z) in FP64, minus offdiag z in FP32;
//   FP64R = false: diag(P) held as a float pair hi + lo, r = fma(-lo, z,
//                  fma(-hi, z, q)) - offdiag z.  Both products are exact in
//                  the fused multiply-adds and q, z are FP32 values, so the
//                  result carries one rounding of r itself, not of q.
// The off-diagonal part is ~1% of q; its FP32 rounding puts the floor of the
// residual near 1e-9 |q| in both variants.  The residual is written in the
// GEMM operand type for the correction apply; per cell conv = |r| <= tol |q|
// (2-norms over the cell's three components).  first: evaluate every cell;
// otherwise cells already converged are skipped (the correction GEMM leaves
// their rows untouched).  final_pass: norms only, for the statistics of
// cells that never converged.
struct ResidArgs {
    int ncells, nV, nVp, first, final_pass;
    double tol;
    const double *diag;      // [nV] diag(P)
    const float *dhi, *dlo;  // [nV] diag(P) = dhi + dlo (+ O(2^-48))
    const int *op, *oj;      // off-diagonal CSR
    const float *ov;
    const float *q, *z;
    __nv_bfloat16 *r_bf16;   // BF16 form
    float *r_f32;            // TF32 form
    int *conv;               // [cell]
    int *any_active;         // set when a cell is not converged
    DevStatus *st;
};

template <bool FP64R>
__global__ void __launch_bounds__(256) k_residual(ResidArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *red = reinterpret_cast<double *>(smem_raw);
    float *zs = reinterpret_cast<float *>(smem_raw + 128 * sizeof(double) + 16);
    const int nVp = a.nVp, n3 = 3 * nVp;
    for (int cell = blockIdx.x; cell < a.ncells; cell += gridDim.x) {
        if (!a.first && a.conv[cell]) continue;
        const long long base = (long long)cell * n3;
        for (int e = threadIdx.x; e < n3; e += blockDim.x) zs[e] = a.z[base + e];
        __syncthreads();
        Acc<float> s[2];
        s[0].zero(); s[1].zero();
        for (int e = threadIdx.x; e < n3; e += blockDim.x) {
            int v, c = elem_cv(e, nVp, v);
            float r = 0.f;
            if (v < a.nV) {
                const float qv = a.q[base + e], zv = zs[e];
                float off = 0.f;
                const float *zc = zs + c * nVp;
                for (int k = a.op[v]; k < a.op[v + 1]; ++k) off = fmaf(a.ov[k], zc[a.oj[k]], off);
                if (FP64R) {
                    r = (float)(fma(-a.diag[v], (double)zv, (double)qv) - (double)off);
                } else {
                    r = __fmaf_rn(-a.dhi[v], zv, qv);
                    r = __fmaf_rn(-a.dlo[v], zv, r);
                    r = __fsub_rn(r, off);
                }
                s[0].add_prod(r, r);
                s[1].add_prod(qv, qv);
            }
            if (!a.final_pass) {
                if (a.r_bf16) a.r_bf16[base + e] = __float2bfloat16_rn(r);
                else a.r_f32[base + e] = r;
            }
        }
        block_reduce_t0<float, 2>(s, red, [&](const double *nr) {
            const bool ok = nr[0] <= a.tol * a.tol * nr[1];
            const float ratio = nr[1] > 0 ? (float)sqrt(nr[0] / nr[1]) : 0.f;
            if (a.final_pass || ok) atomicMax(&a.st->max_resid_bits, __float_as_uint(ratio));
            if (!a.final_pass) {
                a.conv[cell] = ok ? 1 : 0;
                if (!ok) {
                    atomicOr(a.any_active, 1);
                    atomicAdd(&a.st->refine_sweeps, 1ull);
                }
            }
        });
    }
}

// z += dz (correction of one refinement sweep) where the cell is not converged.
__global__ void k_axpy_unconverged(int ncells, int n3, float *z, const float *dz, const int *conv) {
    long long total = (long long)ncells * n3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int cell = (int)(i / n3);
        if (!conv[cell]) z[i] += dz[i];
    }
}

// public [cell][nV][3] (FP64) <-> internal SoA [cell][3][nVp]
__global__ void k_pub_to_soa(int ncells, int nV, int nVp, const long long *pub_off, const double *src,
                             double *dst) {
    const int n3 = 3 * nVp;
    long long total = (long long)ncells * n3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int cell = (int)(i / n3), e = (int)(i - (long long)cell * n3), v;
        int c = elem_cv(e, nVp, v);
        dst[i] = v < nV ? (src ? src[pub_off[cell] + 3 * v + c] : 0.0) : 0.0;
    }
}

__global__ void k_soa_to_pub(int ncells, int nV, int nVp, const long long *pub_off, const double *src,
                             double *dst) {
    long long total = (long long)ncells * nV * 3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int cell = (int)(i / (3 * nV)), k = (int)(i - (long long)cell * 3 * nV);
        int v = k / 3, c = k - 3 * v;
        dst[pub_off[cell] + k] = src[(long long)cell * 3 * nVp + c * nVp + v];
    }
}

// internal SoA (T) [rows][nVp] <-> FP64 column block [rows][nV] (apply entry)
template <typename T>
__global__ void k_cols_in(int rows, int nV, int nVp, const double *src, T *dst, __nv_bfloat16 *dst16) {
    long long total = (long long)rows * nVp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / nVp), v = (int)(i - (long long)r * nVp);
        double x = v < nV ? src[(long long)r * nV + v] : 0.0;
        dst[i] = T(x);
        if (dst16) dst16[i] = __float2bfloat16_rn((float)x);
    }
}

template <typename T>
__global__ void k_cols_out(int rows, int nV, int nVp, const T *src, double *dst) {
    long long total = (long long)rows * nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / nV), v = (int)(i - (long long)r * nV);
        dst[i] = (double)src[(long long)r * nVp + v];
    }
}

__global__ void k_check_finite(long long n, const double *p, DevStatus *st, int ndof_per_cell_hint) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(p[i])) dev_raise(st, DEV_ENONFINITE, (long long)(i / (ndof_per_cell_hint > 0 ? ndof_per_cell_hint : 1)));
}

}  // namespace npfem
