// local.cuh -- the local step of one cell, evaluated by one thread block:
// energy g(x) and gradient grad g(x) of the implicit-Euler objective
// (arXiv 1911.03062, Supplementary Sec. 2.1, Eq. (genericOptimizationNewton)),
//
//   g(x) = 1/(2h^2) sum_v m_v |x_v - y_v|^2 + sum_i w_i/2 |A_i x - p_i(x)|^2,
//   grad = M/h^2 (x - y) + sum_i w_i A_i^T (A_i x - p_i(x)),
//
// with the projective element energies (strain and area per triangle,
// bending per interior edge, volume per cell) and their closest-point
// projections p_i.  Layout: one cell's vectors are SoA [3][nVp] (component
// major, vertex contiguous); thread t owns elements t + j*blockDim (j < EPT).
// Positions are relative to a per-cell origin; x = y_rel + delta.
#pragma once

#include "common.cuh"

namespace npfem {

template <typename T>
struct TypeConst {
    int nV, nVp, nT, nH;
    const int4 *tri;      // nT: (i0, i1, i2, 0), outward CCW
    const T *dinv;        // nT x 4: inverse rest edge matrix D_m^{-1}, row major
    const T *wtri;        // nT x 2: (k_strain, k_area) x rest area
    const int4 *hv;       // nH: hinge (x0, x1, x2, x3)
    const T *hc;          // nH x 4: cotangent stencil
    const T *hrest;       // nH: |b| at rest
    const int *vt_ptr;    // nV + 1: vertex -> triangle incidences (sorted by triangle)
    const int *vt_inc;    //   (t << 2) | corner
    const T *vt_g;        //   (G[corner][0], G[corner][1])
    const int *vh_ptr;    // nV + 1: vertex -> hinge incidences (sorted by hinge)
    const int *vh_inc;    //   (h << 2) | slot
    const T *vh_c;        //   stencil coefficient of the vertex in that hinge
    const T *mh2;         // nV: m_v / h^2
    double V0;            // rest volume
    T kb, kv;             // bending and volume weights
};

__device__ __forceinline__ int elem_cv(int e, int nVp, int &v) {
    int c = (e >= nVp) + (e >= 2 * nVp);
    v = e - c * nVp;
    return c;
}

// ---------------------------------------------------------------- 3x2 SVD
// Closed-form eigen-decomposition of S = F^T F (2x2 symmetric):
// S = V diag(l1, l2) V^T, sigma = sqrt(l), u_i = F v_i / sigma_i; a collapsed
// triangle (sigma2 <= tol sigma1) gets a deterministic orthonormal u2.
template <typename T>
__device__ __forceinline__ void svd32(const T F[6], T U[6], T V[4], T s[2]) {
    T a = F[0] * F[0] + F[2] * F[2] + F[4] * F[4];
    T b = F[0] * F[1] + F[2] * F[3] + F[4] * F[5];
    T c = F[1] * F[1] + F[3] * F[3] + F[5] * F[5];
    T half = T(0.5) * (a + c);
    T dd = hypot(T(0.5) * (a - c), b);
    T l1 = half + dd;
    T det = a * c - b * b;
    T l2 = (l1 > T(0)) ? det / l1 : T(0);
    if (l2 < T(0)) l2 = T(0);
    T v1x, v1y;
    if (dd == T(0)) {
        v1x = T(1); v1y = T(0);
    } else {
        T w1x = l1 - c, w1y = b, w2x = b, w2y = l1 - a;
        T n1 = w1x * w1x + w1y * w1y, n2 = w2x * w2x + w2y * w2y;
        if (n1 >= n2) { T n = sqrt(n1); v1x = w1x / n; v1y = w1y / n; }
        else          { T n = sqrt(n2); v1x = w2x / n; v1y = w2y / n; }
    }
    T v2x = -v1y, v2y = v1x;
    V[0] = v1x; V[1] = v2x; V[2] = v1y; V[3] = v2y;
    s[0] = sqrt(l1);
    s[1] = sqrt(l2);
    T u1[3], u2[3];
    if (s[0] == T(0)) {
        u1[0] = 1; u1[1] = 0; u1[2] = 0;
        u2[0] = 0; u2[1] = 1; u2[2] = 0;
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) u1[r] = (F[2 * r] * v1x + F[2 * r + 1] * v1y) / s[0];
        if (s[1] > T(Prec<T>::degen_tol) * s[0]) {
#pragma unroll
            for (int r = 0; r < 3; ++r) u2[r] = (F[2 * r] * v2x + F[2 * r + 1] * v2y) / s[1];
        } else {
            int ax = 0;
            if (fabs(u1[1]) < fabs(u1[ax])) ax = 1;
            if (fabs(u1[2]) < fabs(u1[ax])) ax = 2;
            T e[3] = {0, 0, 0};
            e[ax] = T(1);
            T pr = e[0] * u1[0] + e[1] * u1[1] + e[2] * u1[2];
#pragma unroll
            for (int r = 0; r < 3; ++r) u2[r] = e[r] - pr * u1[r];
            T n = sqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
#pragma unroll
            for (int r = 0; r < 3; ++r) u2[r] /= n;
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) { U[2 * r] = u1[r]; U[2 * r + 1] = u2[r]; }
}

// Closest (d1, d2) to (s1, s2) on d1 d2 = 1: root of
// f(l) = (s1 + l s2)(s2 + l s1) - (1 - l^2)^2 in the bracket [-s2/s1, 0]
// (s1 s2 > 1) or [0, 1] (otherwise), Newton from 0 with bisection when a
// step leaves the bracket; d1 = (s1 + l s2)/(1 - l^2), d2 = (s2 + l s1)/(1 - l^2).
template <typename T>
__device__ __forceinline__ void area_target(T s1, T s2, T d[2]) {
    T f0 = s1 * s2 - T(1);
    T lam = T(0);
    if (f0 != T(0) && s1 > T(0)) {
        T lo, hi;
        if (f0 > T(0)) { lo = -s2 / s1; hi = T(0); } else { lo = T(0); hi = T(1); }
        for (int it = 0; it < 30; ++it) {
            T A = s1 + lam * s2, B = s2 + lam * s1, q = T(1) - lam * lam;
            T f = A * B - q * q;
            if (f == T(0)) break;
            if (f < T(0)) lo = lam; else hi = lam;
            T fp = s2 * B + s1 * A + T(4) * lam * q;
            T ln = (fp > T(0)) ? lam - f / fp : T(0.5) * (lo + hi);
            if (!(ln >= lo && ln <= hi)) ln = T(0.5) * (lo + hi);
            T step = fabs(ln - lam);
            lam = ln;
            if (step <= T(Prec<T>::area_tol)) break;
        }
    }
    T q = T(1) - lam * lam;
    d[0] = (s1 + lam * s2) / q;
    d[1] = (s2 + lam * s1) / q;
}

// Strain + area projection of one triangle.  R = w_s (F - T_s) + w_a (F - T_a)
// is stashed; the vertex gradient is sum_c R[:, c] G[corner][c].
template <typename T>
__device__ __forceinline__ void tri_local(const T *pos, int nVp, int4 tv, const T *Di, T ws, T wa,
                                          T R[6], Acc<T> &en, Acc<T> &al) {
    T F[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T *pc = pos + c * nVp;
        T x0 = pc[tv.x];
        T e1 = pc[tv.y] - x0, e2 = pc[tv.z] - x0;
        F[2 * c] = e1 * Di[0] + e2 * Di[2];
        F[2 * c + 1] = e1 * Di[1] + e2 * Di[3];
    }
    T U[6], V[4], s[2], d[2];
    svd32(F, U, V, s);
    area_target(s[0], s[1], d);
    T ns = T(0), na = T(0), nf = T(0);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            T u1v = U[2 * r] * V[c * 2 + 0], u2v = U[2 * r + 1] * V[c * 2 + 1];
            T rs = F[2 * r + c] - (u1v + u2v);
            T ra = F[2 * r + c] - (d[0] * u1v + d[1] * u2v);
            ns += rs * rs;
            na += ra * ra;
            nf += F[2 * r + c] * F[2 * r + c];
            R[2 * r + c] = ws * rs + wa * ra;
        }
    en.add(T(0.5) * ws * ns);
    en.add(T(0.5) * wa * na);
    T rf = sqrt(nf);
    al.add(ws * sqrt(ns) * rf + wa * sqrt(na) * rf);
}

// Bending of one hinge: b = sum_j c_j x_j, p = b |b_rest| / |b|; stash kb (b - p).
template <typename T>
__device__ __forceinline__ void hinge_local(const T *pos, int nVp, int4 hv, const T *hc, T rest, T kb,
                                            T R[3], Acc<T> &en, Acc<T> &al) {
    T b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T *pc = pos + c * nVp;
        b[c] = hc[0] * pc[hv.x] + hc[1] * pc[hv.y] + hc[2] * pc[hv.z] + hc[3] * pc[hv.w];
    }
    T nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    T sc = (nb > T(1e-12) * rest && nb > T(0)) ? rest / nb : T(1);
    T n2 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T r = b[c] - b[c] * sc;
        n2 += r * r;
        R[c] = kb * r;
    }
    en.add(T(0.5) * kb * n2);
    al.add(kb * sqrt(n2) * nb);
}

// -------------------------------------------------------- the local step
// dt: this thread's elements of delta (x = y_rel + delta); gr receives the
// gradient; returns g(x) (all threads) and, in allow, a bound on the rounding
// error of g for the FP32 path (8 u sum_i w_i |A_i x - p_i| |A_i x| + u * inertia).
// Shared memory: pos[3 nVp], stash[stash_T], red[reduction scratch].
template <typename T, int EPT>
__device__ double local_eval(const TypeConst<T> &tc, const T *__restrict__ yrel, const T (&dt)[EPT],
                             T (&gr)[EPT], double &allow, T *pos, T *stash, int stash_T, double *red) {
    const int B = blockDim.x, tid = threadIdx.x;
    const int nVp = tc.nVp, nV = tc.nV, n3 = 3 * nVp;
    T x[EPT];
    Acc<T> en, al;
    en.zero();
    al.zero();
    // 1. positions and the inertia term M/h^2 (x - y) = M/h^2 delta
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        int e = tid + j * B;
        int v;
        x[j] = T(0);
        gr[j] = T(0);
        if (e < n3) {
            elem_cv(e, nVp, v);
            if (v < nV) {
                x[j] = yrel[e] + dt[j];
                pos[e] = x[j];
                T mh = tc.mh2[v];
                gr[j] = mh * dt[j];
                T q = T(0.5) * mh * dt[j] * dt[j];
                en.add(q);
                al.add(q);
            }
        }
    }
    __syncthreads();
    // 2. triangles (strain + area), chunked through the stash
    {
        const int ct = stash_T / 6;
        int cur[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = tid + j * B, v;
            cur[j] = 0;
            if (e < n3) { elem_cv(e, nVp, v); if (v < nV) cur[j] = tc.vt_ptr[v]; }
        }
        for (int t0 = 0; t0 < tc.nT; t0 += ct) {
            const int t1 = min(tc.nT, t0 + ct);
            for (int t = t0 + tid; t < t1; t += B) {
                T R[6];
                const T *Di = tc.dinv + 4 * t;
                tri_local(pos, nVp, tc.tri[t], Di, tc.wtri[2 * t], tc.wtri[2 * t + 1], R, en, al);
                T *st = stash + 6 * (t - t0);
#pragma unroll
                for (int i = 0; i < 6; ++i) st[i] = R[i];
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                int e = tid + j * B, v;
                if (e >= n3) continue;
                int c = elem_cv(e, nVp, v);
                if (v >= nV) continue;
                const int end = tc.vt_ptr[v + 1];
                T acc = gr[j];
                int k = cur[j];
                for (; k < end; ++k) {
                    int tt = tc.vt_inc[k] >> 2;
                    if (tt >= t1) break;
                    const T *st = stash + 6 * (tt - t0) + 2 * c;
                    acc += st[0] * tc.vt_g[2 * k] + st[1] * tc.vt_g[2 * k + 1];
                }
                cur[j] = k;
                gr[j] = acc;
            }
            __syncthreads();
        }
    }
    // 3. hinges (bending), chunked through the stash
    {
        const int ch = stash_T / 3;
        int cur[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = tid + j * B, v;
            cur[j] = 0;
            if (e < n3) { elem_cv(e, nVp, v); if (v < nV) cur[j] = tc.vh_ptr[v]; }
        }
        for (int h0 = 0; h0 < tc.nH; h0 += ch) {
            const int h1 = min(tc.nH, h0 + ch);
            for (int h = h0 + tid; h < h1; h += B) {
                T R[3];
                hinge_local(pos, nVp, tc.hv[h], tc.hc + 4 * h, tc.hrest[h], tc.kb, R, en, al);
                T *st = stash + 3 * (h - h0);
                st[0] = R[0]; st[1] = R[1]; st[2] = R[2];
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                int e = tid + j * B, v;
                if (e >= n3) continue;
                int c = elem_cv(e, nVp, v);
                if (v >= nV) continue;
                const int end = tc.vh_ptr[v + 1];
                T acc = gr[j];
                int k = cur[j];
                for (; k < end; ++k) {
                    int hh = tc.vh_inc[k] >> 2;
                    if (hh >= h1) break;
                    acc += tc.vh_c[k] * stash[3 * (hh - h0) + c];
                }
                cur[j] = k;
                gr[j] = acc;
            }
            __syncthreads();
        }
    }
    // 4. volume: p = closest point with V(p) = V0 by the Gauss-Newton
    //    iteration p_{j+1} = x + lambda_j gV(p_j),
    //    lambda_j = (V0 - V(p_j) - gV(p_j).(x - p_j)) / |gV(p_j)|^2,
    //    stopped once |V(p_j) - V0| <= tol V0 or after 8 updates.  pos holds p.
    {
        T p[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) p[j] = x[j];
        for (int it = 0;; ++it) {
            const T o0 = pos[0], o1 = pos[nVp], o2 = pos[2 * nVp];
            Acc<T> a[3];
            a[0].zero(); a[1].zero(); a[2].zero();
            for (int t = tid; t < tc.nT; t += B) {
                int4 tv = tc.tri[t];
                T ax = pos[tv.x] - o0, ay = pos[nVp + tv.x] - o1, az = pos[2 * nVp + tv.x] - o2;
                T bx = pos[tv.y] - o0, by = pos[nVp + tv.y] - o1, bz = pos[2 * nVp + tv.y] - o2;
                T cx = pos[tv.z] - o0, cy = pos[nVp + tv.z] - o1, cz = pos[2 * nVp + tv.z] - o2;
                a[0].add(ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx));
            }
            T gV[EPT];
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                gV[j] = T(0);
                int e = tid + j * B, v;
                if (e >= n3) continue;
                int c = elem_cv(e, nVp, v);
                if (v >= nV) continue;
                const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                const T oc1 = c1 == 0 ? o0 : (c1 == 1 ? o1 : o2);
                const T oc2 = c2 == 0 ? o0 : (c2 == 1 ? o1 : o2);
                T acc = T(0);
                for (int k = tc.vt_ptr[v]; k < tc.vt_ptr[v + 1]; ++k) {
                    int inc = tc.vt_inc[k];
                    int4 tv = tc.tri[inc >> 2];
                    int corner = inc & 3;
                    int vb = corner == 0 ? tv.y : (corner == 1 ? tv.z : tv.x);
                    int vc = corner == 0 ? tv.z : (corner == 1 ? tv.x : tv.y);
                    // component c of (p_b - o) x (p_c - o)
                    T b1 = pos[c1 * nVp + vb] - oc1, b2 = pos[c2 * nVp + vb] - oc2;
                    T q1 = pos[c1 * nVp + vc] - oc1, q2 = pos[c2 * nVp + vc] - oc2;
                    acc += b1 * q2 - b2 * q1;
                }
                gV[j] = acc / T(6);
                a[1].add_prod(gV[j], gV[j]);
                a[2].add_prod(gV[j], x[j] - p[j]);
            }
            double r[3];
            block_reduce<T, 3>(a, r, red);
            const double V = r[0] / 6.0;
            if (fabs(V - tc.V0) <= Prec<T>::vol_tol * fabs(tc.V0) || it == 8) break;
            const T lam = T((tc.V0 - V - r[2]) / r[1]);
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                int e = tid + j * B, v;
                if (e >= n3) continue;
                elem_cv(e, nVp, v);
                if (v >= nV) continue;
                p[j] = x[j] + lam * gV[j];
                pos[e] = p[j];
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = tid + j * B, v;
            if (e >= n3) continue;
            elem_cv(e, nVp, v);
            if (v >= nV) continue;
            T r = x[j] - p[j];
            en.add(T(0.5) * tc.kv * r * r);
            al.add(tc.kv * fabs(r) * fabs(x[j]));
            gr[j] += tc.kv * r;
        }
    }
    Acc<T> fin[2] = {en, al};
    double out[2];
    block_reduce<T, 2>(fin, out, red);
    allow = 8.0 * Prec<T>::round_unit * out[1];
    return out[0];
}

}  // namespace npfem
