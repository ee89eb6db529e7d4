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
#include "npfem.h"

namespace npfem {

template <typename T>
struct IterArgs {
    TypeConst<T> tc;
    int ncells, m, max_bt, last, use_allow, stash_T;
    int cell0;                    // k_predict: first cell of the launch (it steps cells cell0 .. ncells - 1)
    int pf_dist;                  // k_predict: L2 prefetch of cell + pf_dist (one resident wave ahead), 0: off
    double h, inv_h, c1;
    double curv_tol, curv_tol2;   // history admits a pair if s.y > curv_tol |s||y| (and its square)
    double *xn, *vn;              // state, FP64 SoA
    const double *const *fptr;    // device slot holding the f_ext base (public layout)
    const long long *pub_off;     // [cell] offset of the cell in the public arrays (doubles)
    const int *vpub;              // [nV] the caller's index of internal vertex v
    const double *minv;           // [nV] 1 / m_v
    const T *zpred;               // Rayleigh-damped type: Mt^{-1}(M v_n + h F_ext) per cell (SoA), else null
    const T *kcol;                // PIK collisions: [cell][nVp] stiffness (0: no contact), else null
    T *ccol;                      // PIK: [cell][3][nVp] push p - x_n, turned into p - y by k_predict
    T *yrel;                      // y - origin
    double *y64;                  // [cell][3][nVp] y in FP64 (k_predict writes it, the last iteration reads it)
    double *origin;               // [cell][3]
    T *delta, *grad, *q, *z;
    __nv_bfloat16 *q_bf16;        // GEMM operand copy of q (BF16 form), or null
    T *S, *Y;                     // history [cell][m][3][nVp]
    double *rho, *alpha;          // [cell][m]
    double *M;                    // [cell][m][m]: M[i][j] = s_i . y_j for pair i older than pair j
    double *g;                    // [cell] energy at the current iterate
    double *allow;                // [cell] rounding allowance of g (FP32 local step)
    int *hcount, *hhead;          // [cell] ring state
    int *fb_list, *fb_count;      // cells whose direction failed the descent test
    DevStatus *st;
};

// this thread's elements (granules of 4, see elem_of) of a per-cell vector
template <typename T, int EPT>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, T (&r)[EPT], int n3) {
#pragma unroll
    for (int g = 0; g < EPT / 4; ++g) {
        const int e0 = 4 * (threadIdx.x + g * blockDim.x);
        T v[4] = {T(0), T(0), T(0), T(0)};
        if (e0 < n3) ld4(p + e0, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) r[4 * g + i] = v[i];
    }
}

template <typename T, int EPT>
__device__ __forceinline__ void store_vec(T *__restrict__ p, const T (&r)[EPT], int n3) {
#pragma unroll
    for (int g = 0; g < EPT / 4; ++g) {
        const int e0 = 4 * (threadIdx.x + g * blockDim.x);
        if (e0 >= n3) continue;
        const T v[4] = {r[4 * g], r[4 * g + 1], r[4 * g + 2], r[4 * g + 3]};
        st4(p + e0, v);
    }
}

// BF16 copy of this thread's elements (the GEMM operand of q)
template <typename T, int EPT>
__device__ __forceinline__ void store_vec_bf16(__nv_bfloat16 *__restrict__ p, const T (&r)[EPT], int n3) {
#pragma unroll
    for (int g = 0; g < EPT / 4; ++g) {
        const int e0 = 4 * (threadIdx.x + g * blockDim.x);
        if (e0 >= n3) continue;
        __nv_bfloat162 lo = __floats2bfloat162_rn((float)r[4 * g], (float)r[4 * g + 1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn((float)r[4 * g + 2], (float)r[4 * g + 3]);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&lo);
        u.y = *reinterpret_cast<unsigned *>(&hi);
        *reinterpret_cast<uint2 *>(p + e0) = u;
    }
}

// y = x_n + h v_n + h^2 M^{-1} F_ext in FP64 for this thread's elements; with
// Rayleigh damping y = x_n + h Mt^{-1}(M v_n + h F_ext), the solve done before.
// y is also stored (a.y64) for the step's last iteration, which forms
// x_{n+1} = y + delta from it.
template <typename T, int EPT>
__device__ __forceinline__ void predictor64(const IterArgs<T> &a, int cell, double (&y)[EPT]) {
    const int nVp = a.tc.nVp, nV = a.tc.nV, n3 = 3 * nVp;
    const double *f = *a.fptr + a.pub_off[cell];
    const long long base = (long long)cell * n3;
#pragma unroll
    for (int g = 0; g < EPT / 4; ++g) {
        const int e0 = 4 * (threadIdx.x + g * blockDim.x);
#pragma unroll
        for (int i = 0; i < 4; ++i) y[4 * g + i] = 0.0;
        if (e0 >= n3) continue;
        int v0;
        const int c = elem_cv(e0, nVp, v0);
        double xv[4], vv[4];
        ld4(a.xn + base + e0, xv);
        if (a.zpred) {
            T zv[4];
            ld4(a.zpred + base + e0, zv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (v0 + i >= nV) continue;
                y[4 * g + i] = xv[i] + a.h * (double)zv[i];
            }
            const double yv[4] = {y[4 * g], y[4 * g + 1], y[4 * g + 2], y[4 * g + 3]};
            st4(a.y64 + base + e0, yv);
            continue;
        }
        ld4(a.vn + base + e0, vv);
        T kc4[4] = {T(0), T(0), T(0), T(0)};
        if (a.kcol) ld4(a.kcol + (long long)cell * nVp + v0, kc4);   // contact: the fluid force is dropped
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int v = v0 + i;
            if (v >= nV) continue;
            const double fv = kc4[i] != T(0) ? 0.0 : f[3 * a.vpub[v] + c];
            y[4 * g + i] = xv[i] + a.h * vv[i] + a.h * a.h * a.minv[v] * fv;
        }
        // kept for the last iteration's x_{n+1} = y + delta
        const double yv[4] = {y[4 * g], y[4 * g + 1], y[4 * g + 2], y[4 * g + 3]};
        st4(a.y64 + base + e0, yv);
    }
}

// L2 prefetch hint of n bytes at p (rounded down to 16-byte multiples; p must be
// 16-byte aligned): cp.async.bulk.prefetch, no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t n) {
    const uint32_t b = (uint32_t)(n & ~(size_t)15);
    if (b && !(reinterpret_cast<uintptr_t>(p) & 15))
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(b) : "memory");
}

// Sums over the block of n per-thread partials at once (the dot products of
// one L-BFGS pass): partials are written transposed to shared memory, warp w
// reduces values w, w + nwarps, ... in float-float (FP64 in the FP64 path)
// in a fixed order, and out[i] (shared memory) holds the totals, rounded once
// to T, for every thread on return.  scratch: NMAX * blockDim.x values of T
// (the per-cell kernels use their local-step buffers, idle outside local_eval).
template <typename T, int NMAX>
__device__ __forceinline__ void block_sum_many(const T (&part)[NMAX], int n1, int n2, T *scratch, T *out) {
    // values [0, n1) and [n2, NMAX) are summed; the others are skipped
    const int B = blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (B + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
        if (i < n1 || i >= n2) scratch[i * B + threadIdx.x] = part[i];
    __syncthreads();
    for (int i = warp; i < NMAX; i += nw) {
        if (i >= n1 && i < n2) continue;
        Acc<T> acc;
        acc.zero();
        for (int k = lane; k < B; k += 32) acc.add(scratch[i * B + k]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc.merge_shfl(0xffffffffu, off);
        if (lane == 0) out[i] = (T)acc.nearest();
    }
    __syncthreads();
}

// Start of a step: y, origin (midpoint of y at two far-apart vertices), y_rel, delta = 0, history
// cleared, g and grad g at x^0 = y, and q = grad g (the first apply's RHS).
// Right-hand side of the damped predictor, b = M v_n + h F_ext (SoA rows of nVp,
// zero padding), as the apply's operand: q in the form's type and split into a
// high and a low part for the tensor cores: BF16 form hi/lo in BF16 (~16 bits),
// TF32 form q = its TF32 high part and lo32 the FP32 rest (~21 bits).
template <typename T>
__global__ void k_damp_rhs(int ncells, int nV, int nVp, const double *__restrict__ mass, const double *__restrict__ vn,
                           const double *const *fptr, const long long *__restrict__ pub_off,
                           const int *__restrict__ vpub, double h, T *__restrict__ q, __nv_bfloat16 *__restrict__ hi,
                           __nv_bfloat16 *__restrict__ lo, float *__restrict__ lo32, const T *__restrict__ kcol) {
    const long long n3 = 3ll * nVp, total = (long long)ncells * n3;
    const double *f = *fptr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long cell = i / n3;
        const int e = (int)(i - cell * n3), c = e / nVp, v = e - c * nVp;
        double b = 0.0;
        if (v < nV) {
            const bool contact = kcol && kcol[cell * nVp + v] != T(0);   // PIK: fluid force dropped
            b = mass[v] * vn[i] + (contact ? 0.0 : h * f[pub_off[cell] + 3 * vpub[v] + c]);
        }
        q[i] = (T)b;
        if (lo32) {
            const float bh = tf32_hi((float)b);
            q[i] = (T)bh;
            lo32[i] = (float)(b - (double)bh);
        }
        if (hi) {
            const __nv_bfloat16 bh = __float2bfloat16_rn((float)b);
            hi[i] = bh;
            lo[i] = __float2bfloat16_rn((float)(b - (double)__bfloat162float(bh)));
        }
    }
}

template <typename T, int EPT, int MAXB>
__global__ void __launch_bounds__(MAXB, MAXB <= 256 ? (sizeof(T) == 8 ? 2 : 4) : 1) k_predict(IterArgs<T> a) {
    const Smem<T> S = smem_layout<T>(a.tc.nVp);
    const int nVp = a.tc.nVp, n3 = 3 * nVp;
    for (int cell = a.cell0 + blockIdx.x; cell < a.ncells; cell += gridDim.x) {
        const long long base = (long long)cell * n3;
        if (a.pf_dist && threadIdx.x < 3) {
            const int fut = cell + a.pf_dist;        // one resident wave ahead
            if (fut < a.ncells) {
                const size_t vb = (size_t)n3 * sizeof(double);
                if (threadIdx.x == 0) prefetch_l2(a.xn + (long long)fut * n3, vb);
                else if (threadIdx.x == 1) prefetch_l2(a.vn + (long long)fut * n3, vb);
                else prefetch_l2(*a.fptr + a.pub_off[fut], (size_t)3 * a.tc.nV * sizeof(double));
            }
        }
        double y[EPT];
        predictor64<T, EPT>(a, cell, y);
        if (a.ccol) {
            // collision targets relative to y: p - y = (p - x_n) - (y - x_n)
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const int e = elem_of(j);
                int v;
                if (e >= n3) continue;
                elem_cv(e, nVp, v);
                if (v >= a.tc.nV) continue;
                a.ccol[base + e] = T((double)a.ccol[base + e] - (y[j] - a.xn[base + e]));
            }
        }
        // origin of the FP32 offsets: the midpoint of y at two vertices that are far apart
        // at rest, near the middle of the cell (any fixed point serves; it is stored and y
        // is re-formed in FP64 at the end): no block reduction in FP64, whose rate is 1/62
        // of FP32's on this GPU
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = elem_of(j), v;
            if (e >= n3) continue;
            int c = elem_cv(e, nVp, v);
            if (v == a.tc.ova) S.bc->d[c] = y[j];
            if (v == a.tc.ovb) S.bc->d[3 + c] = y[j];
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            const int c = threadIdx.x;
            const double o = 0.5 * (S.bc->d[c] + S.bc->d[3 + c]);
            a.origin[3 * cell + c] = o;
            S.bc->d[c] = o;                  // thread c alone reads d[c] and d[3 + c] here
        }
        __syncthreads();
        T yr[EPT], dl[EPT], gr[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = elem_of(j), v;
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
        const Contact<T> ct{a.kcol ? a.kcol + (long long)cell * nVp : nullptr, a.ccol ? a.ccol + base : nullptr};
        local_eval<T, EPT>(a.tc, a.yrel + base, ct, dl, gr, S, a.stash_T, T(0), [&](double g, double allow, double) {
            a.g[cell] = g;
            a.allow[cell] = allow;
            a.hcount[cell] = 0;
            a.hhead[cell] = 0;
            if (!isfinite(g)) dev_raise(a.st, DEV_ENONFINITE, cell);
        });
        store_vec<T, EPT>(a.grad + base, gr, n3);
        store_vec<T, EPT>(a.q + base, gr, n3);
        if (a.q_bf16) store_vec_bf16<T, EPT>(a.q_bf16 + base, gr, n3);
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
// Both loops are evaluated in their dot-product form: with r_{i-1} and q_i
// written as combinations of z (or grad) and the history vectors,
//   y_i . r_{i-1} = y_i . z + sum_{j older than i} (alpha_j - beta_j) s_j . y_i
//   s_i . q_i     = s_i . grad - sum_{j newer than i} alpha_j s_i . y_j,
// so each loop needs one batched reduction (y_i . z, resp. s_i . grad) plus the
// stored products M[i][j] = s_i . y_j (i older than j), which a new pair adds
// in the same batch.  Scalars are formed by thread 0 in FP64 and broadcast.
constexpr int MH = NPFEM_MAX_HISTORY;

template <typename T, int EPT, int MAXB>
__global__ void __launch_bounds__(MAXB, MAXB <= 256 ? (sizeof(T) == 8 ? 2 : 4) : 1) k_iterate(IterArgs<T> a, const int *list,
                                                                      const int *list_count) {
    const Smem<T> S = smem_layout<T>(a.tc.nVp);
    const int nVp = a.tc.nVp, n3 = 3 * nVp, m = a.m;
    const int nitems = list ? *list_count : a.ncells;
    // batched sums (up to 2 MH + 4) and the cell's L-BFGS scalars in the arithmetic of T:
    // the dots are summed in float-float and rounded once to FP32 in the FP32 path, whose
    // coefficients then act on FP32 vectors (FP64 throughout in the FP64 path)
    T *out = reinterpret_cast<T *>(S.red);
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int cell = list ? list[item] : item;
        const long long base = (long long)cell * n3;
        T *Sh = a.S + (long long)cell * m * n3;
        T *Yh = a.Y + (long long)cell * m * n3;
        T *rho = reinterpret_cast<T *>(a.rho) + (long long)cell * m, *alp = reinterpret_cast<T *>(a.alpha) + (long long)cell * m;
        T *Mc = reinterpret_cast<T *>(a.M) + (long long)cell * m * m;
        const int cnt = a.hcount[cell], head = a.hhead[cell];
        // ring slot of history position l (0 = oldest): (head - cnt + l) mod m by a compare
        // and subtract (an integer division has a 74-cycle latency on this GPU)
        const int s0 = head - cnt < 0 ? head - cnt + m : head - cnt;
        auto slot = [&](int l) { const int v = s0 + l; return v >= m ? v - m : v; };
        // the cell's vectors read later in this iteration, requested into L2 now: the
        // gradient, the iterate, y (local steps) and the history pairs
        if ((int)threadIdx.x < 3 + 2 * cnt) {
            const int i = threadIdx.x;
            const T *src = i == 0 ? a.grad + base : i == 1 ? a.delta + base : i == 2 ? a.yrel + base
                         : (i - 3) < cnt ? Sh + (long long)slot(i - 3) * n3 : Yh + (long long)slot(i - 3 - cnt) * n3;
            prefetch_l2(src, (size_t)n3 * sizeof(T));
        }
        // the cell's scalars that thread 0 uses between barriers, fetched up front into
        // shared memory (red[RED_SCALARS ..), above every reduction's scratch): M, rho, alpha, g, allow
        T *sM = reinterpret_cast<T *>(S.red + RED_SCALARS), *srho = sM + MH * MH, *salp = srho + MH;
        static_assert(RED_SCALARS + MH * MH + 2 * MH <= RED_DOUBLES, "L-BFGS scalars exceed the reduction area");
        for (int i = threadIdx.x; i < m * m + 2 * m; i += blockDim.x) {
            if (i < m * m) sM[i] = Mc[i];
            else if (i < m * m + m) srho[i - m * m] = rho[i - m * m];
            else salp[i - m * m - m] = alp[i - m * m - m];
        }
        if (threadIdx.x == 0) {
            S.bc->d[5] = a.g[cell];
            S.bc->d[6] = a.allow[cell];
            S.bc->d[2] = 1.0;                        // alpha
            S.bc->i[2] = 0;                          // halvings
            S.bc->i[1] = 0;                          // not a descent direction
        }
        T r[EPT], d[EPT], gr[EPT], dl[EPT];
        load_vec<T, EPT>(a.z + base, r, n3);
        if (cnt > 0) {
            // second loop, pass A: y_i . z for all pairs
            T pa[MH];
#pragma unroll
            for (int l = 0; l < MH; ++l) {
                pa[l] = T(0);
                if (l < cnt) {
                    T yi[EPT];
                    load_vec<T, EPT>(Yh + (long long)slot(l) * n3, yi, n3);
#pragma unroll
                    for (int j = 0; j < EPT; ++j) pa[l] += yi[j] * r[j];
                }
            }
            block_sum_many<T, MH>(pa, cnt, MH, S.pos, out);
            if (threadIdx.x == 0) {                     // coefficients kept in S.bc->t
                T *coef = S.bc->t;
                for (int l = 0; l < cnt; ++l) {
                    const int i = slot(l);
                    T dot = out[l];
                    for (int k = 0; k < l; ++k) dot += coef[k] * sM[slot(k) * m + i];
                    coef[l] = salp[i] - srho[i] * dot;
                }
            }
            __syncthreads();
            // pass B: r = z + sum_l coef_l s_l
#pragma unroll
            for (int l = 0; l < MH; ++l) {
                if (l < cnt) {
                    T si[EPT];
                    load_vec<T, EPT>(Sh + (long long)slot(l) * n3, si, n3);
                    const T cf = S.bc->t[l];
#pragma unroll
                    for (int j = 0; j < EPT; ++j) r[j] += cf * si[j];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) d[j] = -r[j];
        // grad . d: this thread's partial, reduced with the first trial's energy
        T gdp = T(0);
        {
            load_vec<T, EPT>(a.grad + base, gr, n3);
#pragma unroll
            for (int j = 0; j < EPT; ++j) gdp = fma(gr[j], d[j], gdp);
        }
        load_vec<T, EPT>(a.delta + base, dl, n3);
        T dt[EPT], gt[EPT];
        T alpha = T(1);
#pragma unroll
        for (int j = 0; j < EPT; ++j) dt[j] = dl[j] + alpha * d[j];
        // d waits in the q buffer (dead until this iteration writes the next q) and the
        // iterate in delta, so neither they nor the trial point hold registers through
        // the local steps: a backtracking trial, and the end of the search, re-form the
        // trial point from them (the same expression, so the same bits)
        store_vec<T, EPT>(a.q + base, d, n3);
        for (;;) {
            const Contact<T> ct{a.kcol ? a.kcol + (long long)cell * nVp : nullptr, a.ccol ? a.ccol + base : nullptr};
            local_eval<T, EPT>(a.tc, a.yrel + base, ct, dt, gt, S, a.stash_T, gdp,
                               [&](double g, double allow, double gds) {
                if (S.bc->i[2] == 0) {                   // first trial: grad . d arrives here
                    S.bc->d[1] = gds;
                    if (gds >= 0.0 && cnt > 0) {         // not a descent direction: clear the
                        S.bc->i[1] = 1;                  // history, queue the cell for
                        S.bc->i[3] = 1;                  // d = -P^{-1} grad, end the search
                        a.hcount[cell] = 0;
                        a.hhead[cell] = 0;
                        a.fb_list[atomicAdd(a.fb_count, 1)] = cell;
                        atomicAdd(&a.st->fallbacks, 1ull);
                        return;
                    }
                }
                const double al = S.bc->d[2], gd = S.bc->d[1];
                const double slack = a.use_allow ? (S.bc->d[6] + allow) : 0.0;
                S.bc->d[3] = g;
                S.bc->d[4] = allow;
                if (g <= S.bc->d[5] + a.c1 * al * gd + slack) {
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
            gdp = T(0);
            load_vec<T, EPT>(a.delta + base, dl, n3);
            load_vec<T, EPT>(a.q + base, d, n3);
#pragma unroll
            for (int j = 0; j < EPT; ++j) dt[j] = dl[j] + alpha * d[j];
        }
        load_vec<T, EPT>(a.grad + base, gr, n3);      // old gradient and iterate (dead during the search)
        load_vec<T, EPT>(a.delta + base, dl, n3);
        load_vec<T, EPT>(a.q + base, d, n3);
#pragma unroll
        for (int j = 0; j < EPT; ++j) dt[j] = dl[j] + alpha * d[j];
        if (S.bc->i[1]) {                              // fallback: the apply's RHS is grad g
            store_vec<T, EPT>(a.q + base, gr, n3);
            __syncthreads();
            continue;
        }
        store_vec<T, EPT>(a.delta + base, dt, n3);
        store_vec<T, EPT>(a.grad + base, gt, n3);
        if (a.last) {
            if (threadIdx.x == 0) {
                const double gtv = S.bc->d[3];
                a.g[cell] = gtv;
                if (S.bc->i[2]) atomicAdd(&a.st->backtracks, (unsigned long long)S.bc->i[2]);
                if (!isfinite(gtv)) dev_raise(a.st, DEV_ENONFINITE, cell);
                atomicAdd(&a.st->energy_sum, gtv);
            }
            double y[EPT], xo[EPT];
            load_vec<double, EPT>(a.y64 + base, y, n3);       // y as the predictor formed it
            load_vec<double, EPT>(a.xn + base, xo, n3);
#pragma unroll
            for (int g = 0; g < EPT / 4; ++g) {
                const int e0 = 4 * (threadIdx.x + g * blockDim.x);
                if (e0 >= n3) continue;
                double xv[4], vv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = 4 * g + i;
                    xv[i] = y[j] + (double)dt[j];
                    vv[i] = (xv[i] - xo[j]) * a.inv_h;
                }
                st4(a.xn + base + e0, xv);
                st4(a.vn + base + e0, vv);
            }
            __syncthreads();
            continue;
        }
        // history pair and the first loop's dots (pass C): for every old pair
        // s_l . grad_new and s_l . y_new; for the new pair s.y, s.s, y.y, s.grad_new
        T sv[EPT], yv[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            sv[j] = dt[j] - dl[j];
            yv[j] = gt[j] - gr[j];
        }
        T pc[2 * MH + 4];
#pragma unroll
        for (int l = 0; l < MH; ++l) {
            pc[2 * l] = T(0);
            pc[2 * l + 1] = T(0);
            if (l < cnt) {
                T si[EPT];
                load_vec<T, EPT>(Sh + (long long)slot(l) * n3, si, n3);
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    pc[2 * l] += si[j] * gt[j];
                    pc[2 * l + 1] += si[j] * yv[j];
                }
            }
        }
        T nsy = T(0), nss = T(0), nyy = T(0), nsg = T(0);
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            nsy += sv[j] * yv[j];
            nss += sv[j] * sv[j];
            nyy += yv[j] * yv[j];
            nsg += sv[j] * gt[j];
        }
        pc[2 * MH] = nsy;
        pc[2 * MH + 1] = nss;
        pc[2 * MH + 2] = nyy;
        pc[2 * MH + 3] = nsg;
        block_sum_many<T, 2 * MH + 4>(pc, 2 * cnt, 2 * MH, S.pos, out);
        if (threadIdx.x == 0) {
            const T sy = out[2 * MH], ss = out[2 * MH + 1], yy = out[2 * MH + 2], sg = out[2 * MH + 3];
            // curvature test sy > tol |s| |y|, squared (no square roots): for tol >= 0 it
            // needs sy > 0 and sy^2 > tol^2 |s|^2 |y|^2; for tol < 0 a pair with sy <= 0 passes
            // when sy^2 < tol^2 |s|^2 |y|^2 (tol = -inf: any pair with s, y != 0)
            const T tol2 = (T)a.curv_tol2;
            const int keep = m > 0 && (a.curv_tol >= 0.0 ? (sy > T(0) && sy * sy > tol2 * ss * yy)
                                                         : (sy > T(0) || sy * sy < tol2 * ss * yy));
            const double gtv = S.bc->d[3];
            a.g[cell] = gtv;
            a.allow[cell] = S.bc->d[4];
            if (S.bc->i[2]) atomicAdd(&a.st->backtracks, (unsigned long long)S.bc->i[2]);
            if (!isfinite(gtv)) dev_raise(a.st, DEV_ENONFINITE, cell);
            // the history after this iteration, oldest first: old pairs (minus the
            // evicted oldest when full) then the new one
            int first_old = 0, ncnt = cnt;
            T rr = T(0);
            if (keep) {
                if (cnt == m) first_old = 1; else ncnt = cnt + 1;
                const int ns = head;                         // the new pair's slot
                rr = T(1) / sy;
                rho[ns] = rr;
                srho[ns] = rr;
                for (int l = first_old; l < cnt; ++l) {
                    Mc[slot(l) * m + ns] = out[2 * l + 1];
                    sM[slot(l) * m + ns] = out[2 * l + 1];
                }
            }
            // alpha_i = rho_i (s_i . grad - sum_{j newer} alpha_j s_i . y_j), newest first:
            // the new pair's (p = nold), then the kept old ones (p = l - first_old), kept
            // in S.bc->t[p] (the coefficients pass D applies)
            const int nold = cnt - first_old;
            T *al = S.bc->t;
            const T aln = keep ? rr * sg : T(0);
            if (keep) al[nold] = aln;
            for (int l = cnt - 1; l >= first_old; --l) {
                const int i = slot(l), p = l - first_old;
                T dot = out[2 * l];
                for (int k = p + 1; k < nold; ++k) dot -= al[k] * sM[i * m + slot(k + first_old)];
                if (keep) dot -= aln * out[2 * l + 1];
                al[p] = srho[i] * dot;
                alp[i] = al[p];
            }
            if (keep) alp[head] = aln;
            S.bc->i[4] = keep;
            S.bc->i[5] = first_old;
            a.hcount[cell] = ncnt;
            a.hhead[cell] = keep ? (head + 1) % m : head;
        }
        __syncthreads();
        const int keep = S.bc->i[4], first_old = S.bc->i[5], nold = cnt - first_old;
        // pass D: q = grad - sum alpha_l y_l over the new history
        T qv[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) qv[j] = gt[j];
#pragma unroll
        for (int l = 0; l < MH; ++l) {
            if (l >= first_old && l < cnt) {
                T yi[EPT];
                load_vec<T, EPT>(Yh + (long long)slot(l) * n3, yi, n3);
                const T ca = S.bc->t[l - first_old];
#pragma unroll
                for (int j = 0; j < EPT; ++j) qv[j] -= ca * yi[j];
            }
        }
        if (keep) {
            const T ca = S.bc->t[nold];
#pragma unroll
            for (int j = 0; j < EPT; ++j) qv[j] -= ca * yv[j];
            store_vec<T, EPT>(Sh + (long long)head * n3, sv, n3);
            store_vec<T, EPT>(Yh + (long long)head * n3, yv, n3);
        }
        store_vec<T, EPT>(a.q + base, qv, n3);
        if (a.q_bf16) store_vec_bf16<T, EPT>(a.q_bf16 + base, qv, n3);
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
    const int *op;           // [nV + 1] off-diagonal CSR row starts
    const int2 *oe;          // (column, value bits) per off-diagonal entry
    const float *q, *z;
    __nv_bfloat16 *r_bf16;   // BF16 form (high part when r_lo is set)
    __nv_bfloat16 *r_lo;     // split corrections: r - r_hi in BF16, or null
    float *r_f32;            // TF32 form
    int *conv;               // [cell]
    const int *prev_active;  // the previous sweep left no cell unconverged if 0 here (null: run)
    int *any_active;         // set when a cell is not converged
    DevStatus *st;
};

// One warp per cell, no block-wide barriers: the warp stages its cell's z in
// shared memory (float4 loads), then each lane evaluates all components of
// vertices lane, lane + 32, ... from one pass over the vertex's CSR row (the
// CSR of the type, shared by all cells, stays in L1), and the warp reduces
// the two norms by shuffles.
template <bool FP64R>
__global__ void __launch_bounds__(256) k_residual(ResidArgs a) {
    if (a.prev_active && *a.prev_active == 0) return;   // uniform: every cell already converged
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nVp = a.nVp, n3 = 3 * nVp, nV = a.nV;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *zw = reinterpret_cast<float *>(smem_raw) + (size_t)warp * n3;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int cell = blockIdx.x * (blockDim.x >> 5) + warp; cell < a.ncells; cell += nwarps) {
        if (!a.first && a.conv[cell]) continue;
        const long long base = (long long)cell * n3;
        {
            const float4 *src = reinterpret_cast<const float4 *>(a.z + base);
            float4 *dst = reinterpret_cast<float4 *>(zw);
            for (int i = lane; i < n3 / 4; i += 32) dst[i] = __ldg(src + i);
        }
        __syncwarp();
        // squared norms for the convergence test (|r| <= tol |q| needs ~1% accuracy):
        // FP32 per lane, float-float across the warp
        float nr = 0.f, nq = 0.f;
        for (int v = lane; v < nVp; v += 32) {
            float r[3] = {0.f, 0.f, 0.f};
            if (v < nV) {
                float off[3] = {0.f, 0.f, 0.f};
                const int kend = __ldg(a.op + v + 1);
                for (int k = __ldg(a.op + v); k < kend; ++k) {
                    const int2 e = __ldg(a.oe + k);          // (column, value bits)
                    const int u = e.x;
                    const float w = __int_as_float(e.y);
                    off[0] = fmaf(w, zw[u], off[0]);
                    off[1] = fmaf(w, zw[nVp + u], off[1]);
                    off[2] = fmaf(w, zw[2 * nVp + u], off[2]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float qv = __ldg(a.q + base + c * nVp + v), zv = zw[c * nVp + v];
                    if (FP64R) {
                        r[c] = (float)(fma(-a.diag[v], (double)zv, (double)qv) - (double)off[c]);
                    } else {
                        float t = __fmaf_rn(-__ldg(a.dhi + v), zv, qv);
                        t = __fmaf_rn(-__ldg(a.dlo + v), zv, t);
                        r[c] = __fsub_rn(t, off[c]);
                    }
                    nr = fmaf(r[c], r[c], nr);
                    nq = fmaf(qv, qv, nq);
                }
            }
            if (!a.final_pass) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (a.r_bf16) {
                        const __nv_bfloat16 hi = __float2bfloat16_rn(r[c]);
                        a.r_bf16[base + c * nVp + v] = hi;
                        if (a.r_lo) a.r_lo[base + c * nVp + v] = __float2bfloat16_rn(r[c] - __bfloat162float(hi));
                    } else {
                        a.r_f32[base + c * nVp + v] = r[c];
                    }
                }
            }
        }
        Acc<float> s[2];
        s[0].zero();
        s[1].zero();
        s[0].add(nr);
        s[1].add(nq);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s[0].merge_shfl(0xffffffffu, off);
            s[1].merge_shfl(0xffffffffu, off);
        }
        if (lane == 0) {
            const double nr0 = s[0].get(), nr1 = s[1].get();
            const bool ok = nr0 <= a.tol * a.tol * nr1;
            const float ratio = nr1 > 0 ? (float)sqrt(nr0 / nr1) : 0.f;
            if (a.final_pass) {
                atomicMax(&a.st->max_resid_bits, __float_as_uint(ratio));
            } else {
                if (ok) atomicMax(&a.st->max_resid_bits, __float_as_uint(ratio));
                a.conv[cell] = ok ? 1 : 0;
                if (!ok) {
                    atomicOr(a.any_active, 1);
                    atomicAdd(&a.st->refine_sweeps, 1ull);
                }
            }
        }
        __syncwarp();
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
// vpub[v]: the caller's index of internal vertex v (vint: the inverse)
__global__ void k_pub_to_soa(int ncells, int nV, int nVp, const long long *pub_off, const double *src,
                             double *dst, const int *vpub) {
    const int n3 = 3 * nVp;
    long long total = (long long)ncells * n3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int cell = (int)(i / n3), e = (int)(i - (long long)cell * n3), v;
        int c = elem_cv(e, nVp, v);
        dst[i] = v < nV ? (src ? src[pub_off[cell] + 3 * vpub[v] + c] : 0.0) : 0.0;
    }
}

__global__ void k_soa_to_pub(int ncells, int nV, int nVp, const long long *pub_off, const double *src,
                             double *dst, const int *vint) {
    long long total = (long long)ncells * nV * 3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int cell = (int)(i / (3 * nV)), k = (int)(i - (long long)cell * 3 * nV);
        int v = k / 3, c = k - 3 * v;
        dst[pub_off[cell] + k] = src[(long long)cell * 3 * nVp + c * nVp + vint[v]];
    }
}

// internal SoA (T) [rows][nVp] <-> FP64 column block [rows][nV] (apply entry)
template <typename T>
__global__ void k_cols_in(int rows, int nV, int nVp, const double *src, T *dst, __nv_bfloat16 *dst16,
                          const int *vpub) {
    long long total = (long long)rows * nVp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / nVp), v = (int)(i - (long long)r * nVp);
        double x = v < nV ? src[(long long)r * nV + vpub[v]] : 0.0;
        dst[i] = T(x);
        if (dst16) dst16[i] = __float2bfloat16_rn((float)x);
    }
}

template <typename T>
__global__ void k_cols_out(int rows, int nV, int nVp, const T *src, double *dst, const int *vint) {
    long long total = (long long)rows * nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / nV), v = (int)(i - (long long)r * nV);
        dst[i] = (double)src[(long long)r * nVp + vint[v]];
    }
}

__global__ void k_check_finite(long long n, const double *p, DevStatus *st, int ndof_per_cell_hint) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(p[i])) dev_raise(st, DEV_ENONFINITE, (long long)(i / (ndof_per_cell_hint > 0 ? ndof_per_cell_hint : 1)));
}

}  // namespace npfem
