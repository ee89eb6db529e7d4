// local.cuh -- the local step of one cell, evaluated by one thread block:
// energy g(x) and gradient grad g(x) of the implicit-Euler objective
// (arXiv 1911.03062, Supplementary Sec. 2.1, Eq. (genericOptimizationNewton)),
//
//   g(x) = 1/(2h^2) (x - y)^T Mt (x - y) + sum_i w_i/2 |A_i x - p_i(x)|^2,
//   grad = Mt/h^2 (x - y) + sum_i w_i A_i^T (A_i x - p_i(x)),
//
// Mt = M undamped; with Rayleigh damping C = alpha M + beta L (Eq. (Newton2nd),
// L = sum_i w_i A_i^T A_i), Mt = M + h C: its diagonal part ((1 + h alpha) M +
// h beta k_vol I) is the per-vertex inertia coefficient, its element parts are
// evaluated with the elements on x - y.
//
// with the projective element energies (strain and area per triangle,
// bending per interior edge, volume per cell) and their closest-point
// projections p_i.  Layout: one cell's vectors are SoA [3][nVp] (component
// major, vertex contiguous); thread t owns elements t + j*blockDim (j < EPT).
// Positions are relative to a per-cell origin; x = y_rel + delta.
//
// Per-element contributions are gathered vertex by vertex through the
// one-ring incidence lists (all three components per visit), in a fixed
// order, so the result is deterministic.
#pragma once

#include "common.cuh"

namespace npfem {

// vertex -> triangle incidence: triangle, the two other vertices in CCW order
// from this one (vb | vc << 16), and G[corner][0..1] with F[:,c] = sum_j G[j][c] x_j
template <typename T> struct alignas(16) TriInc { int t; int bc; T g0, g1; };
// vertex -> hinge incidence: hinge and the vertex's stencil coefficient
template <typename T> struct alignas(2 * sizeof(T)) HingeInc { int h; T c; };

template <typename T>
struct TypeConst {
    int nV, nVp, nT, nH;
    const uint2 *tri;       // nT: i0 | i1 << 16, i2 (16-bit vertex indices), outward CCW
    const T *dinv;          // nT x 4: D_m^{-1}[0][0], D_m^{-1}[0][1], D_m^{-1}[1][1] (the rest frame's
                            // first axis is edge 0->1, so D_m and its inverse are upper triangular),
                            // rest area
    T ks, ka;               // strain and area stiffness (weights k x rest area)
    const uint4 *hv;        // nH: hinge x0 | x1 << 16, x2 | x3 << 16 (16-bit vertex indices), then |b| at
                            // rest (FP32 form: its bits in .z; FP64 form: low word .z, high word .w)
    const T *hc;            // nH x 4: cotangent stencil
    const int *vt_ptr;      // nV + 1: vertex -> triangle incidences (sorted by triangle)
    const TriInc<T> *vt;
    const int *vh_ptr;      // nV + 1: vertex -> hinge incidences (sorted by hinge)
    const HingeInc<T> *vh;
    const T *mh2;           // nV: m_v / h^2 (damped: (1 + h alpha) m_v / h^2 + (beta / h) k_vol)
    int ova, ovb;           // two vertices far apart at rest: the midpoint of their y is the origin
    double V0;              // rest volume
    double V0x6, vtol6;     // 6 V0 and 6 tol |V0| (the volume sums give 6 V)
    T kb, kv;               // bending and volume weights
    T cd;                   // Rayleigh beta / h (0: undamped)
    // slot-major padded copies of the incidence lists (slot q of vertex v at
    // [q * nV + v]; unused slots carry zero weights), for one-round gathers:
    int pad_t, pad_h;       // slots per vertex (0 = not available)
    int2 tri_vrange[4];     // triangle chunk c < 4 (of stash_T / 9 triangles): first and last vertex
                            // its triangles touch (x > y: none)
    const int *vt_pad;      // (t << 2) | corner; padding -1
    const int2 *vh_pad;     // (h, c) as bits; padding (0, 0)
};

constexpr int PAD_T = 8, PAD_H = 16;

// Elements of a per-cell vector owned by the calling thread: EPT / 4 granules
// of 4 consecutive elements, granule g at 4 (tid + g B), so vector loads and
// stores are 16 bytes (FP32) wide and a warp's granules are contiguous.
// Element j is lane j % 4 of granule j / 4; a granule lies in one component
// (nVp is a multiple of 8).
__device__ __forceinline__ int elem_of(int j) { return 4 * (threadIdx.x + (j >> 2) * blockDim.x) + (j & 3); }

// 4 consecutive values at p (16-byte aligned for FP32, 32-byte for FP64)
__device__ __forceinline__ void ld4(const float *p, float (&r)[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&r)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
}
__device__ __forceinline__ void ld2(const float *p, float (&r)[2]) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    r[0] = v.x; r[1] = v.y;
}
__device__ __forceinline__ void ld2(const double *p, double (&r)[2]) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    r[0] = v.x; r[1] = v.y;
}
__device__ __forceinline__ void st4(float *p, const float (&r)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&r)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(r[2], r[3]);
}

// 16-bit packed vertex indices of a triangle / hinge
__device__ __forceinline__ int4 tri_idx(uint2 p) { return make_int4(p.x & 0xffffu, p.x >> 16, p.y & 0xffffu, 0); }
__device__ __forceinline__ int4 hinge_idx(uint4 p) { return make_int4(p.x & 0xffffu, p.x >> 16, p.y & 0xffffu, p.y >> 16); }
__device__ __forceinline__ void hinge_rest(uint4 p, float &r) { r = __uint_as_float(p.z); }
__device__ __forceinline__ void hinge_rest(uint4 p, double &r) { r = __hiloint2double((int)p.w, (int)p.z); }

__device__ __forceinline__ int elem_cv(int e, int nVp, int &v) {
    int c = (e >= nVp) + (e >= 2 * nVp);
    v = e - c * nVp;
    return c;
}

// Values broadcast by thread 0 after a block reduction.
template <typename T>
struct Bcast {
    double d[8];
    T t[8];
    int i[8];
};

// Shared-memory layout of the per-cell kernels:
//   red[RED_DOUBLES] | Bcast | pos[3 nVp] | grad[3 nVp] | gva[3 nVp] | stash[stash_T]
// red: [0, 64) reduction scratch (block_reduce_t0 of up to 4 values over up to
// 16 warps; the batched L-BFGS sums), [64, 64 + 80) the iteration's per-cell
// L-BFGS scalars (k_iterate).
constexpr int RED_DOUBLES = 160;
constexpr int RED_SCALARS = 64;   // first double of the per-cell L-BFGS scalars

template <typename T>
struct Smem {
    double *red;
    Bcast<T> *bc;
    T *pos, *gsh, *gva, *stash;
};

template <typename T>
__device__ __forceinline__ Smem<T> smem_layout(int nVp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T> s;
    s.red = reinterpret_cast<double *>(smem_raw);
    s.bc = reinterpret_cast<Bcast<T> *>(smem_raw + RED_DOUBLES * sizeof(double));
    s.pos = reinterpret_cast<T *>(smem_raw + RED_DOUBLES * sizeof(double) + sizeof(Bcast<double>) + 64);
    s.gsh = s.pos + 3 * nVp;
    s.gva = s.gsh + 3 * nVp;
    s.stash = s.gva + 3 * nVp;
    return s;
}

__host__ __device__ constexpr size_t smem_header_bytes() { return RED_DOUBLES * sizeof(double) + sizeof(Bcast<double>) + 64; }
constexpr int SMEM_VECS = 3;   // pos, grad, gva: 3 nVp values each

// ---------------------------------------------------------------- 3x2 SVD
// Closed-form eigen-decomposition of S = F^T F (2x2 symmetric):
// S = V diag(l1, l2) V^T, sigma = sqrt(l), u_i = F v_i / sigma_i; a collapsed
// triangle (sigma2 <= tol sigma1) gets a deterministic orthonormal u2.
template <typename T>
__device__ __forceinline__ void sym_eig2(T a, T b, T c, T &l1, T &l2, T &v1x, T &v1y) {
    // [[a, b], [b, c]] = l1 v1 v1^T + l2 v2 v2^T, l1 >= l2 >= 0, v1 unit
    T half = T(0.5) * (a + c);
    T hd = T(0.5) * (a - c);
    T dd = sqrt(hd * hd + b * b);
    l1 = half + dd;
    T det = a * c - b * b;
    l2 = (l1 > T(0)) ? det / l1 : T(0);
    if (l2 < T(0)) l2 = T(0);
    if (dd == T(0)) {
        v1x = T(1); v1y = T(0);
    } else {
        T w1x = l1 - c, w1y = b, w2x = b, w2y = l1 - a;
        T n1 = w1x * w1x + w1y * w1y, n2 = w2x * w2x + w2y * w2y;
        if (n1 >= n2) { T n = T(1) / sqrt(n1); v1x = w1x * n; v1y = w1y * n; }
        else          { T n = T(1) / sqrt(n2); v1x = w2x * n; v1y = w2y * n; }
    }
}

template <typename T>
__device__ __forceinline__ void svd32(const T F[6], T U[6], T V[4], T s[2]) {
    T a = F[0] * F[0] + F[2] * F[2] + F[4] * F[4];
    T b = F[0] * F[1] + F[2] * F[3] + F[4] * F[5];
    T c = F[1] * F[1] + F[3] * F[3] + F[5] * F[5];
    T l1, l2, v1x, v1y;
    sym_eig2(a, b, c, l1, l2, v1x, v1y);
    T v2x = -v1y, v2y = v1x;
    V[0] = v1x; V[1] = v2x; V[2] = v1y; V[3] = v2y;
    s[0] = sqrt(l1);
    s[1] = sqrt(l2);
    T u1[3], u2[3];
    if (s[0] == T(0)) {
        u1[0] = 1; u1[1] = 0; u1[2] = 0;
        u2[0] = 0; u2[1] = 1; u2[2] = 0;
    } else {
        const T i0 = T(1) / s[0];
#pragma unroll
        for (int r = 0; r < 3; ++r) u1[r] = (F[2 * r] * v1x + F[2 * r + 1] * v1y) * i0;
        if (s[1] > T(Prec<T>::degen_tol) * s[0]) {
            const T i1 = T(1) / s[1];
#pragma unroll
            for (int r = 0; r < 3; ++r) u2[r] = (F[2 * r] * v2x + F[2 * r + 1] * v2y) * i1;
        } else {
            int ax = 0;
            if (fabs(u1[1]) < fabs(u1[ax])) ax = 1;
            if (fabs(u1[2]) < fabs(u1[ax])) ax = 2;
            T e[3] = {0, 0, 0};
            e[ax] = T(1);
            T pr = e[0] * u1[0] + e[1] * u1[1] + e[2] * u1[2];
#pragma unroll
            for (int r = 0; r < 3; ++r) u2[r] = e[r] - pr * u1[r];
            T n = T(1) / sqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
#pragma unroll
            for (int r = 0; r < 3; ++r) u2[r] *= n;
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
    T iq = T(1) / (T(1) - lam * lam);
    d[0] = (s1 + lam * s2) * iq;
    d[1] = (s2 + lam * s1) * iq;
}

// Rayleigh damping part of one element, returned by value: r = wd A(x - y),
// e = wd/2 |A(x - y)|^2, a = wd |A(x - y)| |A x| (rounding allowance).  Out of
// line, with scalar arguments, so the undamped path keeps its registers.
template <typename T>
struct Damp {
    T r[6];
    T e, a;
};

template <typename T>
__device__ __noinline__ Damp<T> tri_damp(const T *pos, const T *__restrict__ yr, int nVp, int4 tv, T D0, T D1, T D2,
                                         T D3, T wd, T nfx) {
    Damp<T> o;
    T nd = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T *pc = pos + c * nVp, *yc = yr + c * nVp;
        const T d0 = pc[tv.x] - yc[tv.x];
        const T e1 = (pc[tv.y] - yc[tv.y]) - d0, e2 = (pc[tv.z] - yc[tv.z]) - d0;
        const T f0 = e1 * D0 + e2 * D2, f1 = e1 * D1 + e2 * D3;
        o.r[2 * c] = wd * f0;
        o.r[2 * c + 1] = wd * f1;
        nd += f0 * f0 + f1 * f1;
    }
    o.e = T(0.5) * wd * nd;
    o.a = wd * sqrt(nd) * nfx;
    return o;
}

// Strain + area projection of one triangle, written to its 9 stash values:
// R = w_s (F - T_s) + w_a (F - T_a) (the vertex gradient is sum_c R[:, c]
// G[corner][c]) in st[0..5], or (corners) the gradients of corners 1 and 2,
// R G[1] and R G[2], in st[0..2] and st[3..5]; N = (e1 x e2) / 6 (each
// corner's share of the volume gradient) in st[6..8].  Returns the
// signed-volume term (x0 - o).(e1 x e2) of the triangle.
// Rayleigh damping (cd = beta/h != 0): the triangle's part of
// beta/(2h) (x - y)^T L (x - y), i.e. cd (w_s + w_a)/2 |F(x - y)|^2, adds
// cd (w_s + w_a) F(x - y) to R; yr holds y (same frame as pos).
template <typename T>
__device__ __forceinline__ T tri_local(const T *pos, const T *__restrict__ yr, int nVp, int4 tv, const T (&Di)[3], T ws,
                                       T wa, T cd, const T o[3], bool corners, T *st, T &en, T &al) {
    // F = [e1 e2] D_m^{-1} with D_m^{-1} = [[Di0, Di1], [0, Di2]]
    T F[6], E1[3], E2[3], A0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T *pc = pos + c * nVp;
        T x0 = pc[tv.x];
        E1[c] = pc[tv.y] - x0;
        E2[c] = pc[tv.z] - x0;
        A0[c] = x0 - o[c];
        F[2 * c] = E1[c] * Di[0];
        F[2 * c + 1] = E1[c] * Di[1] + E2[c] * Di[2];
    }
    // volume part first (the edge vectors are then dead)
    const T C0 = E1[1] * E2[2] - E1[2] * E2[1], C1 = E1[2] * E2[0] - E1[0] * E2[2], C2 = E1[0] * E2[1] - E1[1] * E2[0];
    const T vol = A0[0] * C0 + A0[1] * C1 + A0[2] * C2;
    T R[6];
    // S = F^T F = V diag(s^2) V^T.  For a triangle that has not collapsed,
    // R = ws (F - U V^T) + wa (F - U diag(d) V^T) = F G with the 2x2
    // G = V diag((ws + wa) - (ws + wa d_i) / s_i) V^T (U = F V diag(1/s)),
    // and |F - U V^T|^2 = sum (s_i - 1)^2, |F - U diag(d) V^T|^2 = sum (s_i - d_i)^2.
    const T sa = F[0] * F[0] + F[2] * F[2] + F[4] * F[4];
    const T sb = F[0] * F[1] + F[2] * F[3] + F[4] * F[5];
    const T sc = F[1] * F[1] + F[3] * F[3] + F[5] * F[5];
    T l1, l2, v1x, v1y;
    sym_eig2(sa, sb, sc, l1, l2, v1x, v1y);
    T s[2] = {sqrt(l1), sqrt(l2)}, d[2];
    T ns, na, nf = sa + sc;
    if (s[1] > T(Prec<T>::degen_tol) * s[0]) {
        area_target(s[0], s[1], d);
        const T g1 = (ws + wa) - (ws + wa * d[0]) / s[0], g2 = (ws + wa) - (ws + wa * d[1]) / s[1];
        const T G00 = g1 * v1x * v1x + g2 * v1y * v1y, G11 = g1 * v1y * v1y + g2 * v1x * v1x;
        const T G01 = (g1 - g2) * v1x * v1y;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R[2 * r] = F[2 * r] * G00 + F[2 * r + 1] * G01;
            R[2 * r + 1] = F[2 * r] * G01 + F[2 * r + 1] * G11;
        }
        ns = (s[0] - T(1)) * (s[0] - T(1)) + (s[1] - T(1)) * (s[1] - T(1));
        na = (s[0] - d[0]) * (s[0] - d[0]) + (s[1] - d[1]) * (s[1] - d[1]);
    } else {
        // collapsed: the polar factor needs the chosen second left vector
        T U[6], V[4];
        svd32(F, U, V, s);
        area_target(s[0], s[1], d);
        ns = T(0);
        na = T(0);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                T u1v = U[2 * r] * V[c * 2 + 0], u2v = U[2 * r + 1] * V[c * 2 + 1];
                T rs = F[2 * r + c] - (u1v + u2v);
                T ra = F[2 * r + c] - (d[0] * u1v + d[1] * u2v);
                ns += rs * rs;
                na += ra * ra;
                R[2 * r + c] = ws * rs + wa * ra;
            }
    }
    en += T(0.5) * ws * ns + T(0.5) * wa * na;
    al += ws * sqrt(ns * nf) + wa * sqrt(na * nf);
    if (cd != T(0)) {
        const Damp<T> dm = tri_damp(pos, yr, nVp, tv, Di[0], Di[1], T(0), Di[2], cd * (ws + wa), sqrt(nf));
#pragma unroll
        for (int i = 0; i < 6; ++i) R[i] += dm.r[i];
        en += dm.e;
        al += dm.a;
    }
    if (corners) {
        // the gradients of corners 1 and 2 (corner 0's is minus their sum: the three
        // G rows sum to zero), so that the gather's incidence entries carry no coefficients
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            st[r] = R[2 * r] * Di[0] + R[2 * r + 1] * Di[1];
            st[3 + r] = R[2 * r + 1] * Di[2];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) st[i] = R[i];
    }
    st[6] = C0 / T(6);
    st[7] = C1 / T(6);
    st[8] = C2 / T(6);
    return vol;
}

// Rayleigh damping part of one hinge (out of line, as tri_damp; r[0..2] used).
template <typename T>
__device__ __noinline__ Damp<T> hinge_damp(const T *pos, const T *__restrict__ yr, int nVp, int4 hv, T c0, T c1, T c2,
                                           T c3, T wd, T nb) {
    Damp<T> o;
    T nd = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T *pc = pos + c * nVp, *yc = yr + c * nVp;
        const T bd = c0 * (pc[hv.x] - yc[hv.x]) + c1 * (pc[hv.y] - yc[hv.y]) + c2 * (pc[hv.z] - yc[hv.z]) +
                     c3 * (pc[hv.w] - yc[hv.w]);
        o.r[c] = wd * bd;
        nd += bd * bd;
    }
    o.r[3] = o.r[4] = o.r[5] = T(0);
    o.e = T(0.5) * wd * nd;
    o.a = wd * sqrt(nd) * nb;
    return o;
}

// Bending of one hinge: b = sum_j c_j x_j, p = b |b_rest| / |b|; stash kb (b - p)
// (+ cd kb b(x - y) with Rayleigh damping, energy cd kb/2 |b(x - y)|^2).
template <typename T>
__device__ __forceinline__ void hinge_local(const T *pos, const T *__restrict__ yr, int nVp, int4 hv, const T (&hc)[4],
                                            T rest, T kb, T cd, T R[3], T &en, T &al) {
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
    en += T(0.5) * kb * n2;
    al += kb * fabs(nb - nb * sc) * nb;              // |b - p| = |b| |1 - sc| (no square root)
    if (cd != T(0)) {
        const Damp<T> dm = hinge_damp(pos, yr, nVp, hv, hc[0], hc[1], hc[2], hc[3], cd * kb, nb);
        R[0] += dm.r[0];
        R[1] += dm.r[1];
        R[2] += dm.r[2];
        en += dm.e;
        al += dm.a;
    }
}

// Signed volume (x 6) of the current positions in pos (relative to vertex 0): this
// thread's partial sum over its triangles (plain arithmetic of T; the block combines
// the partials in float-float / FP64).
template <typename T>
__device__ __forceinline__ T volume_pass(const TypeConst<T> &tc, const T *pos, int nVp, T *nst) {
    T aV = T(0);
    const T o0 = pos[0], o1 = pos[nVp], o2 = pos[2 * nVp];
    for (int t = threadIdx.x; t < tc.nT; t += blockDim.x) {
        const int4 tv = tri_idx(__ldg(tc.tri + t));
        T ax = pos[tv.x] - o0, ay = pos[nVp + tv.x] - o1, az = pos[2 * nVp + tv.x] - o2;
        T e1x = pos[tv.y] - pos[tv.x], e1y = pos[nVp + tv.y] - pos[nVp + tv.x], e1z = pos[2 * nVp + tv.y] - pos[2 * nVp + tv.x];
        T e2x = pos[tv.z] - pos[tv.x], e2y = pos[nVp + tv.z] - pos[nVp + tv.x], e2z = pos[2 * nVp + tv.z] - pos[2 * nVp + tv.x];
        const T cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
        aV += ax * cx + ay * cy + az * cz;
        if (nst) {                                   // the triangle's share of the volume gradient
            nst[3 * t] = cx / T(6);
            nst[3 * t + 1] = cy / T(6);
            nst[3 * t + 2] = cz / T(6);
        }
    }
    return aV;
}

// PIK collision term of one cell: kc[v] (0: no contact) and c = p - y ([3][nVp]);
// the local step adds kc/2 |x - p|^2 = kc/2 |delta - c|^2.  Null pointers: none.
template <typename T>
struct Contact {
    const T *kc;
    const T *c;
};

// -------------------------------------------------------- the local step
// dt: this thread's elements of delta (x = y_rel + delta); gr receives the
// gradient.  After the final reduction thread 0 calls done(g, allow, extra)
// with g(x), the rounding-error bound of g for the FP32 path
// (8 u sum_i w_i |A_i x - p_i| |A_i x| + u * inertia) and the block sum of the
// callers' `extra` partials (reduced with the energy, e.g. a dot product the
// caller needs at the same barrier); done writes what the caller needs into
// S.bc before the closing barrier.
// Per-thread partial sums (energy, volume, |gV|^2, the Gauss-Newton dots) are
// plain arithmetic of T over the thread's few terms; the block combines them in
// float-float (FP32 path) or FP64.
template <typename T, int EPT, typename Done>
__device__ void local_eval(const TypeConst<T> &tc, const T *__restrict__ yrel, const Contact<T> &ct,
                           const T (&dt)[EPT], T (&gr)[EPT], const Smem<T> &S, int stash_T, T extra, Done &&done) {
    const int B = blockDim.x, tid = threadIdx.x;
    const int nVp = tc.nVp, nV = tc.nV, n3 = 3 * nVp;
    T *pos = S.pos, *gsh = S.gsh, *gva = S.gva, *stash = S.stash;
    T x[EPT];
    T en = T(0), al = T(0);      // energy and allowance partials (per thread: a handful of terms)
    // 1. positions; gradient buffer starts with the inertia term M/h^2 (x - y)
#pragma unroll
    for (int g4 = 0; g4 < EPT / 4; ++g4) {
        const int e0 = 4 * (tid + g4 * B);
        T xv[4] = {T(0), T(0), T(0), T(0)}, gv[4] = {T(0), T(0), T(0), T(0)};
        if (e0 < n3) {
            int v0;
            elem_cv(e0, nVp, v0);
            T yr4[4], mh4[4];
            ld4(yrel + e0, yr4);
            ld4(tc.mh2 + v0, mh4);                      // zero beyond nV
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T dj = dt[4 * g4 + i];
                if (v0 + i < nV) {
                    xv[i] = yr4[i] + dj;
                    gv[i] = mh4[i] * dj;
                    T q = T(0.5) * mh4[i] * dj * dj;
                    en += q;
                    al += q;
                }
            }
            if (ct.kc) {                                // collision term (contact vertices only)
                T kc4[4], c4[4];
                ld4(ct.kc + v0, kc4);
                ld4(ct.c + e0, c4);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (v0 + i >= nV || kc4[i] == T(0)) continue;
                    const T r = dt[4 * g4 + i] - c4[i];
                    gv[i] += kc4[i] * r;
                    const T q = T(0.5) * kc4[i] * r * r;
                    en += q;
                    al += q;
                }
            }
            const T zero4[4] = {T(0), T(0), T(0), T(0)};
            st4(pos + e0, xv);
            st4(gsh + e0, gv);
            st4(gva + e0, zero4);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) x[4 * g4 + i] = xv[i];
    }
    __syncthreads();
    T aV = T(0), ag2 = T(0);   // signed 6V of x; |gV(x)|^2 (over the vertices this thread gathers)
    const T o[3] = {pos[0], pos[nVp], pos[2 * nVp]};
    // 2. triangles (strain + area, the volume of x and its gradient), chunked through the stash
    {
        const int ct = stash_T / 9;
        for (int t0 = 0; t0 < tc.nT; t0 += ct) {
            const int t1 = min(tc.nT, t0 + ct);
            for (int t = t0 + tid; t < t1; t += B) {
                const int4 tv = tri_idx(__ldg(tc.tri + t));
                T dq[4];
                ld4(tc.dinv + 4 * t, dq);
                const T Di[3] = {dq[0], dq[1], dq[2]}, w[2] = {tc.ks * dq[3], tc.ka * dq[3]};
                aV += tri_local(pos, yrel, nVp, tv, Di, w[0], w[1], tc.cd, o, sizeof(T) == 4 && tc.pad_t != 0,
                                stash + 9 * (t - t0), en, al);
            }
            __syncthreads();
            if (sizeof(T) == 4 && tc.pad_t) {
                // all slots of a vertex loaded at once (coalesced); a slot whose triangle lies
                // outside this chunk, or a padding slot (-1), adds nothing;
                // only the vertices this chunk's triangles touch are visited (a contiguous
                // range: vertices in RCM order, triangles sorted by their smallest vertex)
                const int nct = t1 - t0, chunk = t0 / ct;
                const int2 rg = chunk < 4 ? tc.tri_vrange[chunk] : make_int2(0, nV - 1);
                for (int v = rg.x + tid; v <= rg.y; v += B) {
                    T g0 = T(0), g1 = T(0), g2 = T(0), n0 = T(0), n1 = T(0), n2 = T(0);
#pragma unroll
                    for (int q0 = 0; q0 < PAD_T; q0 += 4) {
                        if (q0 >= tc.pad_t) break;
                        int inc[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            inc[q] = q0 + q < tc.pad_t ? __ldg(tc.vt_pad + (q0 + q) * nV + v) : -1;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int tt = (inc[q] >> 2) - t0;
                            if ((unsigned)tt >= (unsigned)nct) continue;
                            const T *st = stash + 9 * tt;
                            const int k = inc[q] & 3;
                            const T a0 = st[0], a1 = st[1], a2 = st[2], b0 = st[3], b1 = st[4], b2 = st[5];
                            g0 += k == 1 ? a0 : k == 2 ? b0 : -(a0 + b0);
                            g1 += k == 1 ? a1 : k == 2 ? b1 : -(a1 + b1);
                            g2 += k == 1 ? a2 : k == 2 ? b2 : -(a2 + b2);
                            n0 += st[6];
                            n1 += st[7];
                            n2 += st[8];
                        }
                    }
                    gsh[v] += g0;
                    gsh[nVp + v] += g1;
                    gsh[2 * nVp + v] += g2;
                    gva[v] += n0;                       // area-vector sums (zeroed with the positions)
                    gva[nVp + v] += n1;
                    gva[2 * nVp + v] += n2;
                }
                __syncthreads();
                continue;
            }
            for (int v = tid; v < nV; v += B) {
                T g0 = T(0), g1 = T(0), g2 = T(0), n0 = T(0), n1 = T(0), n2 = T(0);
                const int end = tc.vt_ptr[v + 1];
                for (int k = tc.vt_ptr[v]; k < end; ++k) {
                    const TriInc<T> inc = tc.vt[k];
                    if (inc.t < t0) continue;
                    if (inc.t >= t1) break;
                    const T *st = stash + 9 * (inc.t - t0);
                    g0 += st[0] * inc.g0 + st[1] * inc.g1;
                    g1 += st[2] * inc.g0 + st[3] * inc.g1;
                    g2 += st[4] * inc.g0 + st[5] * inc.g1;
                    n0 += st[6];
                    n1 += st[7];
                    n2 += st[8];
                }
                gsh[v] += g0;
                gsh[nVp + v] += g1;
                gsh[2 * nVp + v] += g2;
                const T f0 = (gva[v] += n0), f1 = (gva[nVp + v] += n1), f2 = (gva[2 * nVp + v] += n2);
                if (t1 == tc.nT) {                      // last chunk: the complete gradient
                    ag2 = fma(f0, f0, ag2);
                    ag2 = fma(f1, f1, ag2);
                    ag2 = fma(f2, f2, ag2);
                }
            }
            __syncthreads();
        }
    }
    if (sizeof(T) == 4 && tc.pad_t) {
        // |gV(x)|^2 over this thread's elements of the complete volume gradient
#pragma unroll
        for (int g4 = 0; g4 < EPT / 4; ++g4) {
            const int e0 = 4 * (tid + g4 * B);
            if (e0 >= n3) continue;
            T gv[4];
            ld4(gva + e0, gv);
#pragma unroll
            for (int i = 0; i < 4; ++i) ag2 = fma(gv[i], gv[i], ag2);
        }
    }
    // First volume reduction {6 V(x), |gV(x)|^2} on the hinge phase's barriers:
    // warp partials now, combined by warp 0 right after the hinge compute
    // barrier, lambda_0 visible after the hinge gather barrier.
    auto vol_first = [&](const double *s) {
        const double r6 = tc.V0x6 - s[0];                   // 6 (V0 - V(x))
        S.bc->i[0] = fabs(r6) <= tc.vtol6;                  // x satisfies the constraint: no update
        S.bc->t[0] = T(r6) / T(6.0 * s[1]);                 // p_0 = x: gV.(x - p_0) = 0
    };
    {
        Acc<T> a1[2];
        a1[0].zero();
        a1[1].zero();
        a1[0].add(aV);
        a1[1].add(ag2);
        warp_partials_store<T, 2>(a1, S.red);
    }
    // 3. hinges (bending), chunked through the stash
    {
        const int ch = stash_T / 3;
        for (int h0 = 0; h0 < tc.nH; h0 += ch) {
            const int h1 = min(tc.nH, h0 + ch);
            uint4 hv_n = make_uint4(0, 0, 0, 0);
            T hc_n[4] = {T(0), T(0), T(0), T(0)};
            if (h0 + tid < h1) {
                hv_n = __ldg(tc.hv + h0 + tid);
                ld4(tc.hc + 4 * (h0 + tid), hc_n);
            }
            for (int h = h0 + tid; h < h1; h += B) {
                const int4 hv = hinge_idx(hv_n);
                T rest;
                hinge_rest(hv_n, rest);
                const T hc[4] = {hc_n[0], hc_n[1], hc_n[2], hc_n[3]};
                if (h + B < h1) {
                    hv_n = __ldg(tc.hv + h + B);
                    ld4(tc.hc + 4 * (h + B), hc_n);
                }
                T R[3];
                hinge_local(pos, yrel, nVp, hv, hc, rest, tc.kb, tc.cd, R, en, al);
                T *st = stash + 3 * (h - h0);
                st[0] = R[0]; st[1] = R[1]; st[2] = R[2];
            }
            __syncthreads();
            if (h0 == 0) block_combine_t0<T, 2>(S.red, vol_first);
            if (sizeof(T) == 4 && tc.pad_h && h0 == 0 && h1 == tc.nH) {
                for (int v = tid; v < nV; v += B) {
                    T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
                    for (int q0 = 0; q0 < PAD_H; q0 += 4) {
                        if (q0 >= tc.pad_h) break;
                        int2 inc[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            inc[q] = q0 + q < tc.pad_h ? __ldg(tc.vh_pad + (q0 + q) * nV + v) : make_int2(0, 0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const T *st = stash + 3 * inc[q].x;
                            const T c = __int_as_float(inc[q].y);
                            g0 += c * st[0];
                            g1 += c * st[1];
                            g2 += c * st[2];
                        }
                    }
                    gsh[v] += g0;
                    gsh[nVp + v] += g1;
                    gsh[2 * nVp + v] += g2;
                }
                __syncthreads();
                continue;
            }
            for (int v = tid; v < nV; v += B) {
                T g0 = T(0), g1 = T(0), g2 = T(0);
                const int end = tc.vh_ptr[v + 1];
                for (int k = tc.vh_ptr[v]; k < end; ++k) {
                    const HingeInc<T> inc = tc.vh[k];
                    if (inc.h < h0) continue;
                    if (inc.h >= h1) break;
                    const T *st = stash + 3 * (inc.h - h0);
                    g0 += inc.c * st[0];
                    g1 += inc.c * st[1];
                    g2 += inc.c * st[2];
                }
                gsh[v] += g0;
                gsh[nVp + v] += g1;
                gsh[2 * nVp + v] += g2;
            }
            __syncthreads();
        }
    }
    if (tc.nH == 0) {                                       // no hinge barriers to ride on
        __syncthreads();
        block_combine_t0<T, 2>(S.red, vol_first);
        __syncthreads();
    }
    // 4. volume: p = closest point with V(p) = V0 by the Gauss-Newton
    //    iteration p_{j+1} = x + lambda_j gV(p_j),
    //    lambda_j = (V0 - V(p_j) - gV(p_j).(x - p_j)) / |gV(p_j)|^2,
    //    stopped once |V(p_j) - V0| <= tol V0 or after 8 updates.  gV(x) was
    //    gathered with the triangles (gva) and lambda_0 formed during the hinge
    //    phase; later gradients come from the triangles' (e1 x e2)/6 of the last
    //    volume pass (FP32 path) or the one-ring cross products (into gva).
    //    pos holds p (x until the first update); each thread reads back its own
    //    elements, so p needs no registers.
    {
        T *gV = gva;
        // FP32 path with the padded incidence table: each volume pass also leaves every
        // triangle's (e1 x e2)/6 in the stash, and the next gradient is their sum over the
        // vertex's triangles (the same sum as the triangle phase's)
        const bool nsum = sizeof(T) == 4 && tc.pad_t && stash_T >= 3 * tc.nT;
        for (int it = 0; !S.bc->i[0]; ++it) {
            if (it > 0 && nsum) {
                for (int v = tid; v < nV; v += B) {
                    T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
                    for (int q0 = 0; q0 < PAD_T; q0 += 4) {
                        if (q0 >= tc.pad_t) break;
                        int inc[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            inc[q] = q0 + q < tc.pad_t ? __ldg(tc.vt_pad + (q0 + q) * nV + v) : -1;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (inc[q] < 0) continue;
                            const T *nq = stash + 3 * (inc[q] >> 2);
                            g0 += nq[0];
                            g1 += nq[1];
                            g2 += nq[2];
                        }
                    }
                    gV[v] = g0;
                    gV[nVp + v] = g1;
                    gV[2 * nVp + v] = g2;
                }
            } else if (it > 0) {
                const T q0 = pos[0], q1 = pos[nVp], q2 = pos[2 * nVp];
                for (int v = tid; v < nV; v += B) {
                    T g[3] = {T(0), T(0), T(0)};
                    const int end = tc.vt_ptr[v + 1];
                    for (int k = tc.vt_ptr[v]; k < end; ++k) {
                        const int bc = tc.vt[k].bc;
                        const int vb = bc & 0xffff, vc = bc >> 16;
                        T bx = pos[vb] - q0, by = pos[nVp + vb] - q1, bz = pos[2 * nVp + vb] - q2;
                        T cx = pos[vc] - q0, cy = pos[nVp + vc] - q1, cz = pos[2 * nVp + vc] - q2;
                        g[0] += by * cz - bz * cy;
                        g[1] += bz * cx - bx * cz;
                        g[2] += bx * cy - by * cx;
                    }
                    gV[v] = g[0] / T(6);
                    gV[nVp + v] = g[1] / T(6);
                    gV[2 * nVp + v] = g[2] / T(6);
                }
            }
            if (it > 0) {
                __syncthreads();
                T qg2 = T(0), qd = T(0);
#pragma unroll
                for (int g4 = 0; g4 < EPT / 4; ++g4) {
                    const int e0 = 4 * (tid + g4 * B);
                    if (e0 >= n3) continue;
                    int v0;
                    elem_cv(e0, nVp, v0);
                    T gv[4], pv[4];
                    ld4(gV + e0, gv);
                    ld4(pos + e0, pv);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (v0 + i >= nV) continue;
                        qg2 = fma(gv[i], gv[i], qg2);
                        qd = fma(gv[i], x[4 * g4 + i] - pv[i], qd);
                    }
                }
                Acc<T> a2[2];
                a2[0].zero();
                a2[1].zero();
                a2[0].add(qg2);
                a2[1].add(qd);
                block_reduce_t0<T, 2>(a2, S.red, [&](const double *s) {
                    S.bc->t[0] = T(tc.V0x6 - S.bc->d[0] - 6.0 * s[1]) / T(6.0 * s[0]);
                });
            }
            const T lam = S.bc->t[0];
#pragma unroll
            for (int g4 = 0; g4 < EPT / 4; ++g4) {
                const int e0 = 4 * (tid + g4 * B);
                if (e0 >= n3) continue;
                int v0;
                elem_cv(e0, nVp, v0);
                T gv[4], pv[4];
                ld4(gV + e0, gv);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = 4 * g4 + i;
                    pv[i] = v0 + i < nV ? x[j] + lam * gv[i] : x[j];
                }
                st4(pos + e0, pv);
            }
            __syncthreads();
            Acc<T> a3[1];
            a3[0].zero();
            a3[0].add(volume_pass(tc, pos, nVp, nsum ? stash : nullptr));
            block_reduce_t0<T, 1>(a3, S.red, [&](const double *s) {
                S.bc->d[0] = s[0];
                S.bc->i[0] = fabs(tc.V0x6 - s[0]) <= tc.vtol6 || it == 7;
            });
        }
    }
    // 5. gradient to registers (+ volume term), energy
#pragma unroll
    for (int g4 = 0; g4 < EPT / 4; ++g4) {
        const int e0 = 4 * (tid + g4 * B);
#pragma unroll
        for (int i = 0; i < 4; ++i) gr[4 * g4 + i] = T(0);
        if (e0 >= n3) continue;
        int v0;
        elem_cv(e0, nVp, v0);
        T gs[4], pv[4];
        ld4(gsh + e0, gs);
        ld4(pos + e0, pv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (v0 + i >= nV) continue;
            const int j = 4 * g4 + i;
            T r = x[j] - pv[i];
            en += T(0.5) * tc.kv * r * r;
            al += tc.kv * fabs(r) * fabs(x[j]);
            gr[j] = gs[i] + tc.kv * r;
        }
    }
    Acc<T> fin[3];
    fin[0].zero();
    fin[1].zero();
    fin[2].zero();
    fin[0].add(en);
    fin[1].add(al);
    fin[2].add(extra);
    block_reduce_t0<T, 3>(fin, S.red, [&](const double *s) { done(s[0], 8.0 * Prec<T>::round_unit * s[1], s[2]); });
}

}  // namespace npfem
