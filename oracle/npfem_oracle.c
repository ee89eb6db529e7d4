/*
 * npfem_oracle.c -- plain, slow, FP64 CPU oracle of the npFEM solid-solver
 * time step (Kotsalos et al., as summarised in arXiv 1911.03062,
 * Supplementary Sec. 2.1, Eqs. (vel), (Newton2nd), (genericOptimizationNewton)
 * and the quasi-Newton update that follows them).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * The paper states the variational form and the quasi-Newton iteration but
 * defers the element energies, their projections, the Hessian approximation
 * and the line search to its npFEM reference.  This file follows the standard
 * projective-dynamics reading of those (each E_i = w_i/2 |A_i x - p_i(x)|^2,
 * p_i the closest point of a constraint set; the constant matrix
 * P = M/h^2 + sum_i w_i A_i^T A_i as H_0), with these concrete choices:
 *   strain  : per triangle, p = polar factor of the deformation gradient F
 *   area    : per triangle, p = U diag(d1,d2) V^T, closest (d1,d2) with d1 d2 = 1
 *   bending : per interior edge, cotangent hinge vector b, p = b |b_rest|/|b|
 *   volume  : per cell, p = closest point with V(p) = V_rest (Gauss-Newton)
 *   step    : L-BFGS (history m, H_0 = P^{-1}) + Armijo backtracking, fixed K.
 *   damping : optional Rayleigh C = alpha M + beta L, L = sum_i w_i A_i^T A_i
 *             (volume term included); Mt = M + h C replaces M in the inertia
 *             term and y = x_n + h Mt^{-1}(M v_n + h F_ext).
 *   contact : optional particle-in-kernel (PIK) collisions: brute-force search
 *             of the closest foreign vertex inside the kernel, its fluid force
 *             dropped, kc/2 |x - p|^2 toward a plane projection p (fixed per step).
 *   IBM     : multi-direct forcing with Peskin's four-point kernel (the producer
 *             of F_ext), brute force over each point's 4 x 4 x 4 lattice stencil.
 * The global solves use this file's own sparse (RCM + envelope) Cholesky.
 *
 * Public layout: positions, velocities, forces are [nV][3] doubles per cell.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ENOTSPD -3

#define AREA_MAX_IT 30
#define AREA_TOL 1e-15
#define VOL_MAX_UPDATES 8
#define VOL_TOL 1e-14
#define DEGEN_TOL 1e-12
#define BEND_TOL 1e-12
#define CURV_TOL 1e-12

typedef struct {
    int nV, nT, nH;
    int *tri;          /* nT*3 */
    double *rest;      /* nV*3 */
    double *mass;      /* nV */
    double ks, ka, kb, kv, h;
    double *Dinv;      /* nT*4, row-major 2x2 */
    double *area;      /* nT rest areas */
    int *hv;           /* nH*4 hinge vertices (x0,x1 hinge; x2 opp. in t1; x3 opp. in t2) */
    double *hc;        /* nH*4 stencil coefficients */
    double *hrest;     /* nH rest |b| */
    double V0;
    double ra, rb;     /* Rayleigh damping C = ra M + rb L (0, 0: none) */
    /* P in CSR (full symmetric pattern, sorted columns) */
    int *Pp, *Pj;
    double *Px;
    /* envelope Cholesky of P in RCM order */
    int *perm;         /* perm[new] = old */
    int *first;        /* first column (new numbering) of row i */
    long *rowstart;    /* offset of row i in env */
    double *env;       /* row i holds L[i][first[i] .. i] */
    /* damping only: L = sum_i w_i A_i^T A_i (with the volume term) in CSR, and the
       envelope Cholesky of Mt = (1 + h ra) M + h rb L */
    int *Lp, *Lj;
    double *Lx;
    int *mperm, *mfirst;
    long *mrowstart;
    double *menv;
} orc_type;

/* ---------------------------------------------------------------- helpers */
static double dot3(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void sub3(const double *a, const double *b, double *o) { o[0]=a[0]-b[0]; o[1]=a[1]-b[1]; o[2]=a[2]-b[2]; }
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1]*b[2] - a[2]*b[1];
    o[1] = a[2]*b[0] - a[0]*b[2];
    o[2] = a[0]*b[1] - a[1]*b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* cot of the angle at vertex a of triangle (a, b, c) */
static double cot_at(const double *a, const double *b, const double *c) {
    double u[3], v[3], w[3];
    sub3(b, a, u); sub3(c, a, v); cross3(u, v, w);
    return dot3(u, v) / norm3(w);
}

/* ------------------------------------------------------ element geometry */
/* Deformation gradient of triangle t: F = [x1-x0, x2-x0] Dinv, 3x2 row-major. */
static void tri_F(const orc_type *T, const double *x, int t, double F[6]) {
    const int *v = T->tri + 3*t;
    const double *Di = T->Dinv + 4*t;
    double e1[3], e2[3];
    sub3(x + 3*v[1], x + 3*v[0], e1);
    sub3(x + 3*v[2], x + 3*v[0], e2);
    for (int r = 0; r < 3; ++r) {
        F[2*r+0] = e1[r]*Di[0] + e2[r]*Di[2];
        F[2*r+1] = e1[r]*Di[1] + e2[r]*Di[3];
    }
}

/* Coefficients G[j][c] with F[:,c] = sum_j x_j G[j][c]. */
static void tri_G(const orc_type *T, int t, double G[3][2]) {
    const double *Di = T->Dinv + 4*t;
    for (int c = 0; c < 2; ++c) {
        G[1][c] = Di[0*2+c];
        G[2][c] = Di[1*2+c];
        G[0][c] = -G[1][c] - G[2][c];
    }
}

/*
 * Thin SVD of a 3x2 matrix through the closed-form eigen-decomposition of the
 * 2x2 symmetric S = F^T F: S = V diag(l1,l2) V^T, sigma_i = sqrt(l_i),
 * u_i = F v_i / sigma_i.  When sigma2 <= DEGEN_TOL * sigma1 the second left
 * vector is completed to an orthonormal pair deterministically.
 * Returns U (3x2 row-major), V (2x2, columns v1 v2, row-major), s[2].
 */
static void svd32(const double F[6], double U[6], double V[4], double s[2]) {
    double a = 0, b = 0, c = 0;
    for (int r = 0; r < 3; ++r) {
        a += F[2*r]*F[2*r];
        b += F[2*r]*F[2*r+1];
        c += F[2*r+1]*F[2*r+1];
    }
    double half = 0.5*(a + c);
    double dd = hypot(0.5*(a - c), b);
    double l1 = half + dd;
    double det = a*c - b*b;
    double l2 = (l1 > 0) ? det / l1 : 0.0;
    if (l2 < 0) l2 = 0;
    double v1[2];
    if (dd == 0.0) { v1[0] = 1; v1[1] = 0; }
    else {
        double w1x = l1 - c, w1y = b, w2x = b, w2y = l1 - a;
        double n1 = w1x*w1x + w1y*w1y, n2 = w2x*w2x + w2y*w2y;
        if (n1 >= n2) { double n = sqrt(n1); v1[0] = w1x/n; v1[1] = w1y/n; }
        else          { double n = sqrt(n2); v1[0] = w2x/n; v1[1] = w2y/n; }
    }
    double v2[2] = { -v1[1], v1[0] };
    V[0] = v1[0]; V[1] = v2[0];
    V[2] = v1[1]; V[3] = v2[1];
    s[0] = sqrt(l1); s[1] = sqrt(l2);
    double u1[3], u2[3];
    if (s[0] == 0.0) {
        u1[0] = 1; u1[1] = 0; u1[2] = 0;
        u2[0] = 0; u2[1] = 1; u2[2] = 0;
    } else {
        for (int r = 0; r < 3; ++r) u1[r] = (F[2*r]*v1[0] + F[2*r+1]*v1[1]) / s[0];
        if (s[1] > DEGEN_TOL * s[0]) {
            for (int r = 0; r < 3; ++r) u2[r] = (F[2*r]*v2[0] + F[2*r+1]*v2[1]) / s[1];
        } else {
            /* axis least aligned with u1, made orthogonal to it */
            int ax = 0;
            if (fabs(u1[1]) < fabs(u1[ax])) ax = 1;
            if (fabs(u1[2]) < fabs(u1[ax])) ax = 2;
            double e[3] = {0, 0, 0};
            e[ax] = 1.0;
            double pr = dot3(e, u1);
            for (int r = 0; r < 3; ++r) u2[r] = e[r] - pr*u1[r];
            double n = norm3(u2);
            for (int r = 0; r < 3; ++r) u2[r] /= n;
        }
    }
    for (int r = 0; r < 3; ++r) { U[2*r] = u1[r]; U[2*r+1] = u2[r]; }
}

/* U diag(d) V^T */
static void usv(const double U[6], const double V[4], const double d[2], double P[6]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 2; ++c)
            P[2*r+c] = U[2*r]*d[0]*V[c*2+0] + U[2*r+1]*d[1]*V[c*2+1];
}

/*
 * Closest (d1, d2) to (s1, s2) on d1 d2 = 1 (s1 >= s2 >= 0).  Stationarity
 * gives d1 = (s1 + l s2)/(1 - l^2), d2 = (s2 + l s1)/(1 - l^2) with
 * f(l) = (s1 + l s2)(s2 + l s1) - (1 - l^2)^2 = 0.  The root is bracketed by
 * [-s2/s1, 0] when s1 s2 > 1 and by [0, 1] otherwise; Newton from l = 0,
 * falling back to bisection when a step leaves the bracket, until
 * |dl| <= AREA_TOL or AREA_MAX_IT iterations.
 */
static void area_target(double s1, double s2, double d[2]) {
    double f0 = s1*s2 - 1.0;
    double lam = 0.0;
    if (f0 != 0.0 && s1 > 0.0) {
        double lo, hi;
        if (f0 > 0) { lo = -s2/s1; hi = 0.0; } else { lo = 0.0; hi = 1.0; }
        for (int it = 0; it < AREA_MAX_IT; ++it) {
            double A = s1 + lam*s2, B = s2 + lam*s1, q = 1.0 - lam*lam;
            double f = A*B - q*q;
            if (f == 0.0) break;
            if (f < 0) lo = lam; else hi = lam;
            double fp = s2*B + s1*A + 4.0*lam*q;
            double ln = (fp > 0) ? lam - f/fp : 0.5*(lo + hi);
            if (!(ln >= lo && ln <= hi)) ln = 0.5*(lo + hi);
            double step = fabs(ln - lam);
            lam = ln;
            if (step <= AREA_TOL) break;
        }
    }
    double q = 1.0 - lam*lam;
    d[0] = (s1 + lam*s2)/q;
    d[1] = (s2 + lam*s1)/q;
}

/* ------------------------------------------------------------------ volume */
/* V(p) = sum_t (p_a - o).((p_b - o) x (p_c - o)) / 6 with o = p_0 (same value in
 * exact arithmetic as the origin-based sum; the shift avoids cancellation). */
static double volume(const orc_type *T, const double *p) {
    const double *o = p;
    double V = 0;
    for (int t = 0; t < T->nT; ++t) {
        const int *v = T->tri + 3*t;
        double a[3], b[3], c[3], bc[3];
        sub3(p + 3*v[0], o, a); sub3(p + 3*v[1], o, b); sub3(p + 3*v[2], o, c);
        cross3(b, c, bc);
        V += dot3(a, bc) / 6.0;
    }
    return V;
}

/* dV/dp_v = sum over triangles (v, b, c) containing v (CCW from v) of (p_b x p_c)/6 */
static void volume_grad(const orc_type *T, const double *p, double *gV) {
    const double *o = p;
    memset(gV, 0, sizeof(double)*3*T->nV);
    for (int t = 0; t < T->nT; ++t) {
        const int *v = T->tri + 3*t;
        for (int k = 0; k < 3; ++k) {
            int a = v[k], b = v[(k+1)%3], c = v[(k+2)%3];
            double pb[3], pc[3], w[3];
            sub3(p + 3*b, o, pb); sub3(p + 3*c, o, pc);
            cross3(pb, pc, w);
            for (int r = 0; r < 3; ++r) gV[3*a+r] += w[r] / 6.0;
        }
    }
}

/*
 * Closest point p to x with V(p) = V0, by Gauss-Newton on the linearised
 * constraint: p_0 = x, lambda_j = (V0 - V(p_j) - gV(p_j).(x - p_j)) / |gV(p_j)|^2,
 * p_{j+1} = x + lambda_j gV(p_j); stop once |V(p_j) - V0| <= VOL_TOL |V0| or
 * after VOL_MAX_UPDATES updates.  Returns the number of updates.
 */
static int volume_project(const orc_type *T, const double *x, double *p, double *gV) {
    int n3 = 3*T->nV;
    memcpy(p, x, sizeof(double)*n3);
    int j = 0;
    for (;; ++j) {
        double V = volume(T, p);
        if (fabs(V - T->V0) <= VOL_TOL*fabs(T->V0) || j == VOL_MAX_UPDATES) break;
        volume_grad(T, p, gV);
        double G2 = 0, r = 0;
        for (int i = 0; i < n3; ++i) { G2 += gV[i]*gV[i]; r += gV[i]*(x[i] - p[i]); }
        double lam = (T->V0 - V - r) / G2;
        for (int i = 0; i < n3; ++i) p[i] = x[i] + lam*gV[i];
    }
    return j;
}

/* ------------------------------------------------------------------ energy */
#define TERM_INERTIA 1
#define TERM_STRAIN 2
#define TERM_AREA 4
#define TERM_BEND 8
#define TERM_VOLUME 16
#define TERM_ALL 31

/*
 * g(x) = 1/(2h^2) (x - y)^T Mt (x - y) + sum_i E_i(x)   (Eq. genericOptimizationNewton),
 * Mt = M + h C, C = ra M + rb L (Rayleigh; none: Mt = M), and its gradient
 * Mt/h^2 (x - y) + sum_i w_i A_i^T (A_i x - p_i).
 * terms[0..4] receive the inertia(+damping)/strain/area/bending/volume parts.
 */
/* PIK collision term of one cell: kc/2 |x_v - p_v|^2 for every vertex with hit[v] != 0. */
typedef struct {
    double kc;
    const int *hit;      /* [nV] */
    const double *p;     /* [nV][3] targets */
} orc_coll;

static double energy_impl(const orc_type *T, const double *x, const double *y, int mask,
                          double *grad, double *terms, const orc_coll *cc);

double orc_energy(const orc_type *T, const double *x, const double *y, int mask,
                  double *grad, double *terms) {
    return energy_impl(T, x, y, mask, grad, terms, NULL);
}

/* g with the PIK collision term (its energy is in the total, not in terms[]). */
double orc_energy_col(const orc_type *T, const double *x, const double *y, int mask,
                      double *grad, double *terms, double kc, const int *hit, const double *p) {
    orc_coll cc = {kc, hit, p};
    return energy_impl(T, x, y, mask, grad, terms, &cc);
}

static double energy_impl(const orc_type *T, const double *x, const double *y, int mask,
                          double *grad, double *terms, const orc_coll *cc) {
    int nV = T->nV;
    double e[5] = {0, 0, 0, 0, 0}, ecol = 0;
    if (grad) memset(grad, 0, sizeof(double)*3*nV);
    double ih2 = (1.0 + T->h*T->ra)/(T->h*T->h);      /* (1 + h ra)/h^2: Mt's mass part */
    if (mask & TERM_INERTIA) {
        for (int v = 0; v < nV; ++v) {
            double dx[3];
            sub3(x + 3*v, y + 3*v, dx);
            e[0] += 0.5*ih2*T->mass[v]*dot3(dx, dx);
            if (grad) for (int r = 0; r < 3; ++r) grad[3*v+r] += ih2*T->mass[v]*dx[r];
        }
        if (T->rb != 0) {
            /* Rayleigh stiffness part of 1/(2h^2) (x-y)^T Mt (x-y): rb/(2h) d^T L d, d = x - y */
            double c = T->rb/T->h;
            for (int v = 0; v < nV; ++v)
                for (int r = 0; r < 3; ++r) {
                    double Ld = 0;
                    for (int p = T->Lp[v]; p < T->Lp[v+1]; ++p)
                        Ld += T->Lx[p]*(x[3*T->Lj[p]+r] - y[3*T->Lj[p]+r]);
                    e[0] += 0.5*c*(x[3*v+r] - y[3*v+r])*Ld;
                    if (grad) grad[3*v+r] += c*Ld;
                }
        }
    }
    if (mask & (TERM_STRAIN | TERM_AREA)) {
        for (int t = 0; t < T->nT; ++t) {
            double F[6], U[6], V[4], s[2], G[3][2], R[6] = {0, 0, 0, 0, 0, 0};
            tri_F(T, x, t, F);
            svd32(F, U, V, s);
            tri_G(T, t, G);
            if (mask & TERM_STRAIN) {
                double one[2] = {1, 1}, Ps[6];
                usv(U, V, one, Ps);
                double w = T->ks*T->area[t], n2 = 0;
                for (int i = 0; i < 6; ++i) { n2 += (F[i]-Ps[i])*(F[i]-Ps[i]); R[i] += w*(F[i]-Ps[i]); }
                e[1] += 0.5*w*n2;
            }
            if (mask & TERM_AREA) {
                double d[2], Pa[6];
                area_target(s[0], s[1], d);
                usv(U, V, d, Pa);
                double w = T->ka*T->area[t], n2 = 0;
                for (int i = 0; i < 6; ++i) { n2 += (F[i]-Pa[i])*(F[i]-Pa[i]); R[i] += w*(F[i]-Pa[i]); }
                e[2] += 0.5*w*n2;
            }
            if (grad) {
                const int *v = T->tri + 3*t;
                for (int j = 0; j < 3; ++j)
                    for (int r = 0; r < 3; ++r)
                        grad[3*v[j]+r] += R[2*r]*G[j][0] + R[2*r+1]*G[j][1];
            }
        }
    }
    if (mask & TERM_BEND) {
        for (int hh = 0; hh < T->nH; ++hh) {
            const int *hv = T->hv + 4*hh;
            const double *c = T->hc + 4*hh;
            double b[3] = {0, 0, 0};
            for (int j = 0; j < 4; ++j)
                for (int r = 0; r < 3; ++r) b[r] += c[j]*x[3*hv[j]+r];
            double nb = norm3(b), p[3];
            if (nb > BEND_TOL*T->hrest[hh] && nb > 0) {
                for (int r = 0; r < 3; ++r) p[r] = b[r]*T->hrest[hh]/nb;
            } else {
                for (int r = 0; r < 3; ++r) p[r] = b[r];
            }
            double rr[3];
            sub3(b, p, rr);
            e[3] += 0.5*T->kb*dot3(rr, rr);
            if (grad)
                for (int j = 0; j < 4; ++j)
                    for (int r = 0; r < 3; ++r) grad[3*hv[j]+r] += T->kb*c[j]*rr[r];
        }
    }
    if (mask & TERM_VOLUME) {
        double *p = (double *)malloc(sizeof(double)*6*nV);
        double *gV = p + 3*nV;
        volume_project(T, x, p, gV);
        for (int i = 0; i < 3*nV; ++i) {
            double r = x[i] - p[i];
            e[4] += 0.5*T->kv*r*r;
            if (grad) grad[i] += T->kv*r;
        }
        free(p);
    }
    if (cc && cc->hit) {
        for (int v = 0; v < nV; ++v) {
            if (!cc->hit[v]) continue;
            for (int c = 0; c < 3; ++c) {
                double r = x[3*v+c] - cc->p[3*v+c];
                ecol += 0.5*cc->kc*r*r;
                if (grad) grad[3*v+c] += cc->kc*r;
            }
        }
    }
    if (terms) for (int i = 0; i < 5; ++i) terms[i] = e[i];
    return e[0] + e[1] + e[2] + e[3] + e[4] + ecol;
}

/* ----------------------------------------------------------- sparse matrix */
typedef struct { int i, j; double v; } trip;

static int trip_cmp(const void *a, const void *b) {
    const trip *x = (const trip *)a, *y = (const trip *)b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    return 0;
}

/*
 * wm M + wl (sum_t (w_strain + w_area) A_t^T A_t + sum_e w_bend A_e^T A_e + w_vol I).
 * P: wm = 1/h^2, wl = 1 (undamped; with Rayleigh damping (1 + h ra)/h^2 and
 * 1 + rb/h).  A_t maps the triangle's vertices to F (F[:,c] = sum_j G[j][c] x_j),
 * A_e to b = sum_j c_j x_j; the block for xyz is the same nV x nV matrix.
 */
static int assemble(const orc_type *T, double wm, double wl, int **Ap_, int **Aj_, double **Ax_) {
    int nV = T->nV;
    long cap = (long)nV + 9L*T->nT + 16L*T->nH;
    trip *tr = (trip *)malloc(sizeof(trip)*cap);
    if (!tr) return ORC_ENOMEM;
    long n = 0;
    for (int v = 0; v < nV; ++v) { tr[n].i = v; tr[n].j = v; tr[n].v = T->mass[v]*wm + T->kv*wl; ++n; }
    for (int t = 0; t < T->nT; ++t) {
        double G[3][2];
        tri_G(T, t, G);
        double w = wl*(T->ks + T->ka)*T->area[t];
        const int *v = T->tri + 3*t;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                tr[n].i = v[a]; tr[n].j = v[b];
                tr[n].v = w*(G[a][0]*G[b][0] + G[a][1]*G[b][1]);
                ++n;
            }
    }
    for (int hh = 0; hh < T->nH; ++hh) {
        const int *hv = T->hv + 4*hh;
        const double *c = T->hc + 4*hh;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                tr[n].i = hv[a]; tr[n].j = hv[b]; tr[n].v = wl*T->kb*c[a]*c[b]; ++n;
            }
    }
    qsort(tr, n, sizeof(trip), trip_cmp);
    int *Ap = (int *)calloc(nV + 1, sizeof(int));
    int *Aj = (int *)malloc(sizeof(int)*n);
    double *Ax = (double *)malloc(sizeof(double)*n);
    if (!Ap || !Aj || !Ax) { free(tr); free(Ap); free(Aj); free(Ax); return ORC_ENOMEM; }
    long m = 0;
    for (long k = 0; k < n; ++k) {
        if (m > 0 && Aj[m-1] == tr[k].j && k > 0 && tr[k-1].i == tr[k].i) {
            Ax[m-1] += tr[k].v;
        } else {
            Aj[m] = tr[k].j; Ax[m] = tr[k].v; Ap[tr[k].i + 1]++; ++m;
        }
    }
    for (int i = 0; i < nV; ++i) Ap[i+1] += Ap[i];
    free(tr);
    *Ap_ = Ap; *Aj_ = Aj; *Ax_ = Ax;
    return ORC_OK;
}

static int assemble_P(orc_type *T) {
    const double h = T->h;
    return assemble(T, (1.0 + h*T->ra)/(h*h), 1.0 + T->rb/h, &T->Pp, &T->Pj, &T->Px);
}

/* Reverse Cuthill-McKee ordering of a symmetric CSR pattern (start: lowest-degree
 * unvisited vertex; neighbours queued by increasing degree, then index). */
static void rcm(int n, const int *Ap, const int *Aj, int *perm) {
    int *deg = (int *)malloc(sizeof(int)*n);
    char *seen = (char *)calloc(n, 1);
    int *order = (int *)malloc(sizeof(int)*n);
    int *nb = (int *)malloc(sizeof(int)*n);
    for (int i = 0; i < n; ++i) deg[i] = Ap[i+1] - Ap[i] - 1;
    int head = 0, tail = 0;
    while (tail < n) {
        int s = -1;
        for (int i = 0; i < n; ++i)
            if (!seen[i] && (s < 0 || deg[i] < deg[s])) s = i;
        seen[s] = 1; order[tail++] = s;
        while (head < tail) {
            int u = order[head++], k = 0;
            for (int p = Ap[u]; p < Ap[u+1]; ++p) {
                int w = Aj[p];
                if (!seen[w]) { seen[w] = 1; nb[k++] = w; }
            }
            for (int a = 1; a < k; ++a) {          /* insertion sort by (deg, idx) */
                int w = nb[a], b = a - 1;
                while (b >= 0 && (deg[nb[b]] > deg[w] || (deg[nb[b]] == deg[w] && nb[b] > w))) {
                    nb[b+1] = nb[b]; --b;
                }
                nb[b+1] = w;
            }
            for (int a = 0; a < k; ++a) order[tail++] = nb[a];
        }
    }
    for (int i = 0; i < n; ++i) perm[i] = order[n - 1 - i];
    free(deg); free(seen); free(order); free(nb);
}

/* Envelope (profile) Cholesky of an RCM-permuted SPD CSR matrix, row by row.
 * Outputs (allocated here): perm[new] = old, first column of each row, row
 * offsets into env, env. */
static int factor_env(int n, const int *Ap, const int *Aj, const double *Ax, int **perm_, int **first_,
                      long **rowstart_, double **env_) {
    int *perm = (int *)malloc(sizeof(int)*n);
    int *iperm = (int *)malloc(sizeof(int)*n);
    int *first = (int *)malloc(sizeof(int)*n);
    long *rowstart = (long *)malloc(sizeof(long)*(n + 1));
    *perm_ = perm; *first_ = first; *rowstart_ = rowstart; *env_ = NULL;
    rcm(n, Ap, Aj, perm);
    for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
    for (int i = 0; i < n; ++i) {
        int old = perm[i], f = i;
        for (int p = Ap[old]; p < Ap[old+1]; ++p) {
            int j = iperm[Aj[p]];
            if (j < f) f = j;
        }
        first[i] = f;
    }
    rowstart[0] = 0;
    for (int i = 0; i < n; ++i) rowstart[i+1] = rowstart[i] + (i - first[i] + 1);
    double *env = (double *)calloc(rowstart[n], sizeof(double));
    *env_ = env;
    if (!env) { free(iperm); return ORC_ENOMEM; }
#define L(i, j) env[rowstart[i] + ((j) - first[i])]
    for (int i = 0; i < n; ++i) {
        int old = perm[i];
        for (int p = Ap[old]; p < Ap[old+1]; ++p) {
            int j = iperm[Aj[p]];
            if (j <= i) L(i, j) = Ax[p];
        }
    }
    for (int i = 0; i < n; ++i) {
        int fi = first[i];
        for (int j = fi; j < i; ++j) {
            double s = L(i, j);
            int k0 = fi > first[j] ? fi : first[j];
            for (int k = k0; k < j; ++k) s -= L(i, k)*L(j, k);
            L(i, j) = s / L(j, j);
        }
        double s = L(i, i);
        for (int k = fi; k < i; ++k) s -= L(i, k)*L(i, k);
        if (!(s > 0)) { free(iperm); return ORC_ENOTSPD; }
        L(i, i) = sqrt(s);
    }
    free(iperm);
    return ORC_OK;
}

static int factor_P(orc_type *T) {
    return factor_env(T->nV, T->Pp, T->Pj, T->Px, &T->perm, &T->first, &T->rowstart, &T->env);
}

/* x = A^{-1} b for each of the 3 components (b, x: [nV][3]) with an envelope factor. */
static void solve_env(int n, const int *perm, const int *first, const long *rowstart, const double *env,
                      const double *b, double *x) {
    double *z = (double *)malloc(sizeof(double)*n);
    for (int c = 0; c < 3; ++c) {
        for (int i = 0; i < n; ++i) z[i] = b[3*perm[i] + c];
        for (int i = 0; i < n; ++i) {                 /* L z = b */
            double s = z[i];
            for (int k = first[i]; k < i; ++k) s -= L(i, k)*z[k];
            z[i] = s / L(i, i);
        }
        for (int i = n - 1; i >= 0; --i) {            /* L^T w = z */
            z[i] /= L(i, i);
            for (int k = first[i]; k < i; ++k) z[k] -= L(i, k)*z[i];
        }
        for (int i = 0; i < n; ++i) x[3*perm[i] + c] = z[i];
    }
    free(z);
}
#undef L

/* x = P^{-1} b for each of the 3 components (b, x: [nV][3]). */
void orc_solve(const orc_type *T, const double *b, double *x) {
    solve_env(T->nV, T->perm, T->first, T->rowstart, T->env, b, x);
}

/* ------------------------------------------------------------ type set-up */
void orc_type_destroy(orc_type *T) {
    if (!T) return;
    free(T->tri); free(T->rest); free(T->mass); free(T->Dinv); free(T->area);
    free(T->hv); free(T->hc); free(T->hrest); free(T->Pp); free(T->Pj); free(T->Px);
    free(T->perm); free(T->first); free(T->rowstart); free(T->env);
    free(T->Lp); free(T->Lj); free(T->Lx); free(T->mperm); free(T->mfirst); free(T->mrowstart); free(T->menv);
    free(T);
}

/*
 * Hinges: every undirected edge of a closed, consistently oriented mesh is
 * seen once as a->b (triangle t1 = (a, b, c)) and once as b->a (t2 = (b, a, d)).
 * Stencil (cotangent hinge vector, scaled by sqrt(3/(A1+A2))) with
 * alpha_{t,v} = rest angle of triangle t at hinge vertex v:
 *   c0 = cot a_{1,1} + cot a_{2,1},  c1 = cot a_{1,0} + cot a_{2,0},
 *   c2 = -(cot a_{1,0} + cot a_{1,1}),  c3 = -(cot a_{2,0} + cot a_{2,1}).
 */
static int build_hinges(orc_type *T) {
    int nT = T->nT, nV = T->nV;
    int ne = 3*nT;
    /* directed half-edges (a, b, opposite, triangle) sorted by (min, max) key */
    long *key = (long *)malloc(sizeof(long)*ne);
    int *idx = (int *)malloc(sizeof(int)*ne);
    for (int t = 0; t < nT; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = T->tri[3*t+k], b = T->tri[3*t+(k+1)%3];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            key[3*t+k] = (long)lo*nV + hi;
            idx[3*t+k] = 3*t + k;
        }
    /* pair each half-edge with its twin through an open-addressing table on the key */
    long hsz = 1;
    while (hsz < 4L*ne) hsz <<= 1;
    int *tab = (int *)malloc(sizeof(int)*hsz);
    for (long i = 0; i < hsz; ++i) tab[i] = -1;
    int *twin = (int *)malloc(sizeof(int)*ne);
    int ok = 1;
    for (int e = 0; e < ne; ++e) {
        twin[e] = -1;
        long hpos = (long)((unsigned long)(key[e]*2654435761UL) & (hsz - 1));
        while (tab[hpos] >= 0 && key[tab[hpos]] != key[e]) hpos = (hpos + 1) & (hsz - 1);
        if (tab[hpos] < 0) tab[hpos] = e;
        else {
            int o = tab[hpos];
            if (twin[o] >= 0) { ok = 0; break; }       /* edge in > 2 triangles */
            int a = T->tri[e], b = T->tri[3*(e/3) + (e%3+1)%3];
            int oa = T->tri[o], ob = T->tri[3*(o/3) + (o%3+1)%3];
            if (!(a == ob && b == oa)) { ok = 0; break; } /* inconsistent orientation */
            twin[o] = e; twin[e] = o;
        }
    }
    if (ok) for (int e = 0; e < ne; ++e) if (twin[e] < 0) { ok = 0; break; }  /* open mesh */
    if (!ok) { free(key); free(idx); free(tab); free(twin); return ORC_EINVAL; }
    T->nH = ne/2;
    T->hv = (int *)malloc(sizeof(int)*4*T->nH);
    T->hc = (double *)malloc(sizeof(double)*4*T->nH);
    T->hrest = (double *)malloc(sizeof(double)*T->nH);
    int h = 0;
    for (int e = 0; e < ne; ++e) {
        int o = twin[e];
        if (o < e) continue;                  /* first appearance defines the hinge */
        int t1 = e/3, k1 = e%3, t2 = o/3, k2 = o%3;
        int x0 = T->tri[3*t1+k1], x1 = T->tri[3*t1+(k1+1)%3], x2 = T->tri[3*t1+(k1+2)%3];
        int x3 = T->tri[3*t2+(k2+2)%3];
        const double *X0 = T->rest + 3*x0, *X1 = T->rest + 3*x1, *X2 = T->rest + 3*x2, *X3 = T->rest + 3*x3;
        double c10 = cot_at(X0, X1, X2), c11 = cot_at(X1, X2, X0);
        double c20 = cot_at(X0, X3, X1), c21 = cot_at(X1, X0, X3);
        double A1 = T->area[t1], A2 = T->area[t2];
        double sc = sqrt(3.0/(A1 + A2));
        int *hv = T->hv + 4*h;
        double *c = T->hc + 4*h;
        hv[0] = x0; hv[1] = x1; hv[2] = x2; hv[3] = x3;
        c[0] = sc*(c11 + c21);
        c[1] = sc*(c10 + c20);
        c[2] = -sc*(c10 + c11);
        c[3] = -sc*(c20 + c21);
        double b[3] = {0, 0, 0};
        for (int j = 0; j < 4; ++j)
            for (int r = 0; r < 3; ++r) b[r] += c[j]*T->rest[3*hv[j]+r];
        T->hrest[h] = norm3(b);
        ++h;
    }
    free(key); free(idx); free(tab); free(twin);
    return ORC_OK;
}

int orc_type_create(int nV, const double *rest, int nT, const int *tris, const double *mass,
                    double ks, double ka, double kb, double kv, double dt, orc_type **out) {
    *out = NULL;
    if (nV < 4 || nT < 4 || !(dt > 0)) return ORC_EINVAL;
    for (int i = 0; i < 3*nT; ++i) if (tris[i] < 0 || tris[i] >= nV) return ORC_EINVAL;
    orc_type *T = (orc_type *)calloc(1, sizeof(orc_type));
    if (!T) return ORC_ENOMEM;
    T->nV = nV; T->nT = nT;
    T->ks = ks; T->ka = ka; T->kb = kb; T->kv = kv; T->h = dt;
    T->tri = (int *)malloc(sizeof(int)*3*nT);
    T->rest = (double *)malloc(sizeof(double)*3*nV);
    T->mass = (double *)malloc(sizeof(double)*nV);
    T->Dinv = (double *)malloc(sizeof(double)*4*nT);
    T->area = (double *)malloc(sizeof(double)*nT);
    memcpy(T->tri, tris, sizeof(int)*3*nT);
    memcpy(T->rest, rest, sizeof(double)*3*nV);
    for (int v = 0; v < nV; ++v) T->mass[v] = mass ? mass[v] : 1.0/nV;
    for (int t = 0; t < nT; ++t) {
        const int *v = T->tri + 3*t;
        double E1[3], E2[3], n[3];
        sub3(T->rest + 3*v[1], T->rest + 3*v[0], E1);
        sub3(T->rest + 3*v[2], T->rest + 3*v[0], E2);
        cross3(E1, E2, n);
        double nn = norm3(n), l1 = norm3(E1);
        if (!(nn > 0) || !(l1 > 0)) { orc_type_destroy(T); return ORC_EINVAL; }
        double u[3] = {E1[0]/l1, E1[1]/l1, E1[2]/l1};
        double nh[3] = {n[0]/nn, n[1]/nn, n[2]/nn}, w[3];
        cross3(nh, u, w);
        /* D_m = [[E1.u, E2.u], [E1.w, E2.w]] */
        double a = dot3(E1, u), b = dot3(E2, u), c = dot3(E1, w), d = dot3(E2, w);
        double det = a*d - b*c;
        double *Di = T->Dinv + 4*t;
        Di[0] = d/det; Di[1] = -b/det; Di[2] = -c/det; Di[3] = a/det;
        T->area[t] = 0.5*nn;
    }
    int rc = build_hinges(T);
    if (rc) { orc_type_destroy(T); return rc; }
    T->V0 = volume(T, T->rest);
    rc = assemble_P(T);
    if (!rc) rc = factor_P(T);
    if (rc) { orc_type_destroy(T); return rc; }
    *out = T;
    return ORC_OK;
}

/* Rayleigh damping C = ra M + rb L (paper Sec. 2.1, Eq. Newton2nd; Table Params
 * gives alpha_D = 0, beta_D = 0.01).  Reading: L = sum_i w_i A_i^T A_i (with the
 * volume term), the constant stiffness of the quadratic energies.  Rebuilds P =
 * Mt/h^2 + L = (1 + h ra) M/h^2 + (1 + rb/h) L and factors Mt = (1 + h ra) M + h rb L
 * for the predictor.  ra = rb = 0 restores the undamped type. */
int orc_type_set_damping(orc_type *T, double ra, double rb) {
    if (!(ra >= 0) || !(rb >= 0)) return ORC_EINVAL;
    free(T->Pp); free(T->Pj); free(T->Px); free(T->perm); free(T->first); free(T->rowstart); free(T->env);
    free(T->Lp); free(T->Lj); free(T->Lx); free(T->mperm); free(T->mfirst); free(T->mrowstart); free(T->menv);
    T->Pp = T->Pj = T->perm = T->first = T->Lp = T->Lj = T->mperm = T->mfirst = NULL;
    T->Px = T->env = T->Lx = T->menv = NULL;
    T->rowstart = T->mrowstart = NULL;
    T->ra = ra; T->rb = rb;
    int rc = assemble_P(T);
    if (!rc) rc = factor_P(T);
    if (!rc && (ra != 0 || rb != 0)) {
        rc = assemble(T, 0.0, 1.0, &T->Lp, &T->Lj, &T->Lx);
        int *Mp = NULL, *Mj = NULL;
        double *Mx = NULL;
        if (!rc) rc = assemble(T, 1.0 + T->h*ra, T->h*rb, &Mp, &Mj, &Mx);
        if (!rc) rc = factor_env(T->nV, Mp, Mj, Mx, &T->mperm, &T->mfirst, &T->mrowstart, &T->menv);
        free(Mp); free(Mj); free(Mx);
    }
    return rc;
}

void orc_type_info(const orc_type *T, int *nH, double *V0, int *nnzP, long *nnzL) {
    if (nH) *nH = T->nH;
    if (V0) *V0 = T->V0;
    if (nnzP) *nnzP = T->Pp[T->nV];
    if (nnzL) *nnzL = T->rowstart[T->nV];
}

void orc_P_dense(const orc_type *T, double *P) {
    int n = T->nV;
    memset(P, 0, sizeof(double)*n*n);
    for (int i = 0; i < n; ++i)
        for (int p = T->Pp[i]; p < T->Pp[i+1]; ++p) P[(long)i*n + T->Pj[p]] = T->Px[p];
}

void orc_hinges(const orc_type *T, int *hv, double *hc, double *hrest) {
    memcpy(hv, T->hv, sizeof(int)*4*T->nH);
    memcpy(hc, T->hc, sizeof(double)*4*T->nH);
    memcpy(hrest, T->hrest, sizeof(double)*T->nH);
}

/* ------------------------------------------------- single-element entries */
void orc_polar(const double F[6], double T[6], double s[2]) {
    double U[6], V[4], one[2] = {1, 1};
    svd32(F, U, V, s);
    usv(U, V, one, T);
}

void orc_area_project(const double F[6], double Pa[6], double d[2]) {
    double U[6], V[4], s[2];
    svd32(F, U, V, s);
    area_target(s[0], s[1], d);
    usv(U, V, d, Pa);
}

void orc_area_target(double s1, double s2, double d[2]) { area_target(s1, s2, d); }

int orc_volume_project(const orc_type *T, const double *x, double *p) {
    double *gV = (double *)malloc(sizeof(double)*3*T->nV);
    int j = volume_project(T, x, p, gV);
    free(gV);
    return j;
}

double orc_volume(const orc_type *T, const double *p) { return volume(T, p); }
void orc_volume_grad(const orc_type *T, const double *p, double *g) { volume_grad(T, p, g); }

/* ------------------------------------------------------------- time step */
static double vdot(const double *a, const double *b, int n) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += a[i]*b[i];
    return s;
}

/* Optional per-iteration record of one step (every array nullable):
 *   x, g : [K+1][n3] the iterates x^0 (= y) .. x^K and the gradients at them
 *   d    : [K][n3]   the direction taken at iteration k (after the descent test)
 *   kept : [K]       1 where the pair (x^{k+1} - x^k, g^{k+1} - g^k) entered the history */
typedef struct {
    double *x, *g, *d;
    int *kept;
} orc_trace;

/*
 * One implicit-Euler step of one cell (Eqs. vel, Newton2nd via the
 * minimisation of g):
 *   y = x_n + h v_n + h^2 M^{-1} F_ext,  x^0 = y
 *   for k < K:  d = -H grad g(x^k)  (L-BFGS two-loop, H_0 = P^{-1}, history m;
 *                                    plain -P^{-1} grad when the history is empty)
 *               if grad.d >= 0: clear history, d = -P^{-1} grad
 *               Armijo backtracking from alpha = 1 (c1, halving, <= max_bt halvings,
 *               the last trial is taken when the cap is hit)
 *               store (s, dgrad) when s.dgrad > CURV_TOL |s||dgrad|
 *   x_{n+1} = x^K,  v_{n+1} = (x_{n+1} - x_n)/h.
 * Traces (nullable): g_tr[K+1] energies, a_tr[K] accepted alphas,
 * bt_tr[K] halvings, fb_tr[K] 1 where the descent fallback ran.
 * Returns the number of iterations whose line search hit the cap.
 */
static int step_impl(const orc_type *T, const double *xn, const double *vn, const double *f_in,
                     int K, int m, double c1, int max_bt, const orc_coll *cc,
                     double *x_out, double *v_out,
                     double *g_tr, double *a_tr, int *bt_tr, int *fb_tr,
                     double curv_tol, const orc_trace *tr);

int orc_step(const orc_type *T, const double *xn, const double *vn, const double *f,
             int K, int m, double c1, int max_bt,
             double *x_out, double *v_out,
             double *g_tr, double *a_tr, int *bt_tr, int *fb_tr) {
    return step_impl(T, xn, vn, f, K, m, c1, max_bt, NULL, x_out, v_out, g_tr, a_tr, bt_tr, fb_tr,
                     CURV_TOL, NULL);
}

/* orc_step with the per-iteration record (orc_trace) and the curvature threshold
 * of the history as a parameter (CURV_TOL = 1e-12 is the method's; a test that
 * needs indefinite updates to reach the descent fallback passes -INFINITY). */
int orc_step_trace(const orc_type *T, const double *xn, const double *vn, const double *f,
                   int K, int m, double c1, int max_bt, double curv_tol,
                   double *x_out, double *v_out,
                   double *g_tr, double *a_tr, int *bt_tr, int *fb_tr,
                   double *xs, double *gs, double *ds, int *kept) {
    orc_trace tr = {xs, gs, ds, kept};
    return step_impl(T, xn, vn, f, K, m, c1, max_bt, NULL, x_out, v_out, g_tr, a_tr, bt_tr, fb_tr,
                     curv_tol, &tr);
}

/* The step with the PIK collision framework (Sec. 2.2, Supp. PIK): the
 * external (fluid) force of every vertex with hit[v] != 0 is disregarded and
 * the term kc/2 |x_v - p_v|^2 joins g, with the targets p fixed over the step. */
int orc_step_col(const orc_type *T, const double *xn, const double *vn, const double *f,
                 int K, int m, double c1, int max_bt, double kc, const int *hit, const double *p,
                 double *x_out, double *v_out) {
    orc_coll cc = {kc, hit, p};
    return step_impl(T, xn, vn, f, K, m, c1, max_bt, &cc, x_out, v_out, NULL, NULL, NULL, NULL,
                     CURV_TOL, NULL);
}

static int step_impl(const orc_type *T, const double *xn, const double *vn, const double *f_in,
                     int K, int m, double c1, int max_bt, const orc_coll *cc,
                     double *x_out, double *v_out,
                     double *g_tr, double *a_tr, int *bt_tr, int *fb_tr,
                     double curv_tol, const orc_trace *tr) {
    int nV = T->nV, n3 = 3*nV;
    double h = T->h;
    int mm = m > 0 ? m : 1;
    double *buf = (double *)malloc(sizeof(double)*n3*(8 + 2*mm));
    double *y = buf, *x = y + n3, *gr = x + n3, *d = gr + n3, *xt = d + n3, *gt = xt + n3;
    double *q = gt + n3, *r = q + n3;
    double *S = r + n3, *Y = S + n3*mm;
    double *rho = (double *)malloc(sizeof(double)*mm), *al = (double *)malloc(sizeof(double)*mm);
    double *fz = NULL;
    const double *f = f_in;
    if (cc && cc->hit) {                    /* PIK: contaminated vertices lose their fluid force */
        fz = (double *)malloc(sizeof(double)*n3);
        for (int v = 0; v < nV; ++v)
            for (int c = 0; c < 3; ++c) fz[3*v+c] = cc->hit[v] ? 0.0 : f_in[3*v+c];
        f = fz;
    }
    if (T->ra == 0 && T->rb == 0) {
        for (int v = 0; v < nV; ++v)
            for (int c = 0; c < 3; ++c)
                y[3*v+c] = xn[3*v+c] + h*vn[3*v+c] + h*h/T->mass[v]*f[3*v+c];
    } else {
        /* y = x_n + h Mt^{-1} (M v_n + h F_ext)  (x buffer as scratch) */
        memset(x, 0, sizeof(double)*n3);
        for (int v = 0; v < nV; ++v)
            for (int c = 0; c < 3; ++c) x[3*v+c] = T->mass[v]*vn[3*v+c] + h*f[3*v+c];
        solve_env(nV, T->mperm, T->mfirst, T->mrowstart, T->menv, x, y);
        for (int i = 0; i < n3; ++i) y[i] = xn[i] + h*y[i];
    }
    memcpy(x, y, sizeof(double)*n3);
    double g = energy_impl(T, x, y, TERM_ALL, gr, NULL, cc);
    if (g_tr) g_tr[0] = g;
    if (tr && tr->x) memcpy(tr->x, x, sizeof(double)*n3);
    if (tr && tr->g) memcpy(tr->g, gr, sizeof(double)*n3);
    int cnt = 0, head = 0, caps = 0;    /* ring: newest at (head-1) mod m */
    for (int k = 0; k < K; ++k) {
        int fb = 0;
        if (cnt == 0) {
            orc_solve(T, gr, d);
            for (int i = 0; i < n3; ++i) d[i] = -d[i];
        } else {
            memcpy(q, gr, sizeof(double)*n3);
            for (int l = 0; l < cnt; ++l) {             /* newest -> oldest */
                int i = ((head - 1 - l) % mm + mm) % mm;
                al[i] = rho[i]*vdot(S + (long)i*n3, q, n3);
                for (int e = 0; e < n3; ++e) q[e] -= al[i]*Y[(long)i*n3 + e];
            }
            orc_solve(T, q, r);
            for (int l = cnt - 1; l >= 0; --l) {        /* oldest -> newest */
                int i = ((head - 1 - l) % mm + mm) % mm;
                double be = rho[i]*vdot(Y + (long)i*n3, r, n3);
                for (int e = 0; e < n3; ++e) r[e] += S[(long)i*n3 + e]*(al[i] - be);
            }
            for (int i = 0; i < n3; ++i) d[i] = -r[i];
        }
        double gd = vdot(gr, d, n3);
        if (gd >= 0 && cnt > 0) {
            cnt = 0; fb = 1;
            orc_solve(T, gr, d);
            for (int i = 0; i < n3; ++i) d[i] = -d[i];
            gd = vdot(gr, d, n3);
        }
        if (tr && tr->d) memcpy(tr->d + (long)k*n3, d, sizeof(double)*n3);
        double alpha = 1.0, gtv;
        int bt = 0;
        for (;;) {
            for (int i = 0; i < n3; ++i) xt[i] = x[i] + alpha*d[i];
            gtv = energy_impl(T, xt, y, TERM_ALL, gt, NULL, cc);
            if (gtv <= g + c1*alpha*gd) break;
            if (bt == max_bt) { ++caps; break; }
            alpha *= 0.5; ++bt;
        }
        double *s_new = q, *y_new = r;          /* free here: the pair enters the ring only if kept */
        for (int i = 0; i < n3; ++i) { s_new[i] = xt[i] - x[i]; y_new[i] = gt[i] - gr[i]; }
        double sy = vdot(s_new, y_new, n3);
        double ns = sqrt(vdot(s_new, s_new, n3)), ny = sqrt(vdot(y_new, y_new, n3));
        memcpy(x, xt, sizeof(double)*n3);
        memcpy(gr, gt, sizeof(double)*n3);
        g = gtv;
        const int keep = m > 0 && sy > curv_tol*ns*ny;
        if (tr && tr->kept) tr->kept[k] = keep;
        if (tr && tr->x) memcpy(tr->x + (long)(k+1)*n3, x, sizeof(double)*n3);
        if (tr && tr->g) memcpy(tr->g + (long)(k+1)*n3, gr, sizeof(double)*n3);
        if (keep) {
            memcpy(S + (long)head*n3, s_new, sizeof(double)*n3);
            memcpy(Y + (long)head*n3, y_new, sizeof(double)*n3);
            rho[head] = 1.0/sy;
            head = (head + 1) % mm;
            if (cnt < m) ++cnt;
        }
        if (g_tr) g_tr[k+1] = g;
        if (a_tr) a_tr[k] = alpha;
        if (bt_tr) bt_tr[k] = bt;
        if (fb_tr) fb_tr[k] = fb;
    }
    for (int i = 0; i < n3; ++i) {
        x_out[i] = x[i];
        v_out[i] = (x[i] - xn[i]) / h;
    }
    free(buf); free(rho); free(al); free(fz);
    return caps;
}

/* ------------------------------------------------ pre- and post-step filters
 * One-ring median filter of the external forces (paper Sec. 2.2: a median in the
 * one-ring neighbourhood of every Lagrangian point attenuates force spikes).
 * Reading: the force of vertex v becomes, component by component, the median of
 * the forces of v and of the vertices sharing an edge with v; for an even count
 * the mean of the two middle values.  f, out: [nV][3]. */
static int dbl_cmp(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int orc_force_median(const orc_type *T, const double *f, double *out) {
    int nV = T->nV, nT = T->nT;
    int *deg = (int *)calloc((size_t)nV + 1, sizeof(int));
    int *nb = (int *)malloc(sizeof(int) * 6 * (size_t)nT);
    double *val = (double *)malloc(sizeof(double) * ((size_t)nV + 1));
    int *start = (int *)malloc(sizeof(int) * ((size_t)nV + 1));
    if (!deg || !nb || !val || !start) { free(deg); free(nb); free(val); free(start); return ORC_ENOMEM; }
    /* directed edges (each triangle edge both ways), bucketed by source vertex */
    for (int t = 0; t < nT; ++t)
        for (int k = 0; k < 3; ++k) { deg[T->tri[3*t+k]] += 2; }
    start[0] = 0;
    for (int v = 0; v < nV; ++v) start[v+1] = start[v] + deg[v];
    for (int v = 0; v < nV; ++v) deg[v] = 0;
    for (int t = 0; t < nT; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = T->tri[3*t+k], b = T->tri[3*t+(k+1)%3];
            nb[start[a] + deg[a]++] = b;
            nb[start[b] + deg[b]++] = a;
        }
    for (int v = 0; v < nV; ++v) {
        int *l = nb + start[v], n = deg[v], u = 0;
        /* unique neighbours (each appears twice in a closed manifold mesh) */
        for (int i = 0; i < n; ++i) {
            int dup = 0;
            for (int j = 0; j < u; ++j) if (l[j] == l[i]) { dup = 1; break; }
            if (!dup) l[u++] = l[i];
        }
        for (int c = 0; c < 3; ++c) {
            int cnt = 0;
            val[cnt++] = f[3*v + c];
            for (int i = 0; i < u; ++i) val[cnt++] = f[3*l[i] + c];
            qsort(val, (size_t)cnt, sizeof(double), dbl_cmp);
            out[3*v + c] = (cnt & 1) ? val[cnt/2] : 0.5 * (val[cnt/2 - 1] + val[cnt/2]);
        }
    }
    free(deg); free(nb); free(val); free(start);
    return ORC_OK;
}

/* Velocity cap (paper Sec. 2.2: an npFEM vertex velocity above U*_max is
 * truncated towards the threshold).  Reading: |v| > umax -> v * umax / |v|,
 * direction kept.  v: [nV][3], in place. */
void orc_velocity_cap(int nV, double *v, double umax) {
    for (int i = 0; i < nV; ++i) {
        double *w = v + 3*i;
        double n = sqrt(w[0]*w[0] + w[1]*w[1] + w[2]*w[2]);
        if (n > umax) {
            double sc = umax / n;
            w[0] *= sc; w[1] *= sc; w[2] *= sc;
        }
    }
}

/* Position-based-dynamics velocity damping (paper Sec. 2.1 cites it as the
 * second viscoelastic proxy; definition from Mueller et al. 2007, Sec. 3.5).
 * Reading: after the step, with the lumped masses m_i, total mass M:
 *   x_cm = sum m_i x_i / M, v_cm = sum m_i v_i / M, r_i = x_i - x_cm,
 *   L = sum r_i x (m_i v_i), I = sum m_i (|r_i|^2 E - r_i r_i^T), omega = I^{-1} L,
 *   v_i <- v_i + kappa (v_cm + omega x r_i - v_i).
 * The rigid part of the velocity field is kept, the rest scaled by (1 - kappa).
 * x, v: [nV][3]; v in place.  Returns ORC_EINVAL if I is singular. */
int orc_pbd_damping(const orc_type *T, const double *x, double *v, double kappa) {
    int nV = T->nV;
    double Mt = 0, xc[3] = {0, 0, 0}, vc[3] = {0, 0, 0};
    for (int i = 0; i < nV; ++i) {
        double m = T->mass[i];
        Mt += m;
        for (int c = 0; c < 3; ++c) { xc[c] += m * x[3*i+c]; vc[c] += m * v[3*i+c]; }
    }
    for (int c = 0; c < 3; ++c) { xc[c] /= Mt; vc[c] /= Mt; }
    double L[3] = {0, 0, 0}, I[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nV; ++i) {
        double m = T->mass[i], r[3], p[3];
        for (int c = 0; c < 3; ++c) { r[c] = x[3*i+c] - xc[c]; p[c] = m * v[3*i+c]; }
        L[0] += r[1]*p[2] - r[2]*p[1];
        L[1] += r[2]*p[0] - r[0]*p[2];
        L[2] += r[0]*p[1] - r[1]*p[0];
        double rr = r[0]*r[0] + r[1]*r[1] + r[2]*r[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                I[3*a+b] += m * ((a == b ? rr : 0.0) - r[a]*r[b]);
    }
    /* omega = I^{-1} L by the adjugate */
    double C[9];
    C[0] = I[4]*I[8] - I[5]*I[7]; C[1] = I[2]*I[7] - I[1]*I[8]; C[2] = I[1]*I[5] - I[2]*I[4];
    C[3] = I[5]*I[6] - I[3]*I[8]; C[4] = I[0]*I[8] - I[2]*I[6]; C[5] = I[2]*I[3] - I[0]*I[5];
    C[6] = I[3]*I[7] - I[4]*I[6]; C[7] = I[1]*I[6] - I[0]*I[7]; C[8] = I[0]*I[4] - I[1]*I[3];
    double det = I[0]*C[0] + I[1]*C[3] + I[2]*C[6];
    if (!(fabs(det) > 0)) return ORC_EINVAL;
    double w[3];
    for (int a = 0; a < 3; ++a) w[a] = (C[3*a]*L[0] + C[3*a+1]*L[1] + C[3*a+2]*L[2]) / det;
    for (int i = 0; i < nV; ++i) {
        double r[3];
        for (int c = 0; c < 3; ++c) r[c] = x[3*i+c] - xc[c];
        double rig[3] = {vc[0] + w[1]*r[2] - w[2]*r[1], vc[1] + w[2]*r[0] - w[0]*r[2], vc[2] + w[0]*r[1] - w[1]*r[0]};
        for (int c = 0; c < 3; ++c) v[3*i+c] += kappa * (rig[c] - v[3*i+c]);
    }
    return ORC_OK;
}

/* n cells of one type, one after another (arrays: [n][nV][3]). */
int orc_step_cells(const orc_type *T, int n, const double *xn, const double *vn, const double *f,
                   int K, int m, double c1, int max_bt, double *x_out, double *v_out) {
    long n3 = 3L*T->nV;
    int caps = 0;
    for (int c = 0; c < n; ++c)
        caps += orc_step(T, xn + c*n3, vn + c*n3, f + c*n3, K, m, c1, max_bt,
                         x_out + c*n3, v_out + c*n3, NULL, NULL, NULL, NULL);
    return caps;
}

/* n cells of one type with the PIK collision term (hit: [n][nV], p: [n][nV][3]). */
int orc_step_cells_col(const orc_type *T, int n, const double *xn, const double *vn, const double *f,
                       int K, int m, double c1, int max_bt, double kc, const int *hit, const double *p,
                       double *x_out, double *v_out) {
    long n3 = 3L*T->nV;
    int caps = 0;
    for (int c = 0; c < n; ++c)
        caps += orc_step_col(T, xn + c*n3, vn + c*n3, f + c*n3, K, m, c1, max_bt, kc, hit + c*(long)T->nV,
                             p + c*n3, x_out + c*n3, v_out + c*n3);
    return caps;
}

/* ---------------------------------------------------- PIK collision framework
 * Vertex normals of one cell: the sum over the incident triangles of
 * (x_b - x_a) x (x_c - x_a) (area-weighted outward normal), normalised.
 * x, n: [nV][3]. */
void orc_vertex_normals(const orc_type *T, const double *x, double *n) {
    int nV = T->nV;
    memset(n, 0, sizeof(double)*3*nV);
    for (int t = 0; t < T->nT; ++t) {
        const int *v = T->tri + 3*t;
        double e1[3], e2[3], cr[3];
        sub3(x + 3*v[1], x + 3*v[0], e1);
        sub3(x + 3*v[2], x + 3*v[0], e2);
        cross3(e1, e2, cr);
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) n[3*v[k]+c] += cr[c];
    }
    for (int i = 0; i < nV; ++i) {
        double l = sqrt(dot3(n + 3*i, n + 3*i));
        if (l > 0) for (int c = 0; c < 3; ++c) n[3*i+c] /= l;
    }
}

/* Particle-in-kernel search (paper Sec. 2.2 and the supplementary PIK section)
 * over ncells cells, cell c with nV[c] vertices at x[c] and normals nrm[c]
 * ([nV][3] each).  For every vertex i: among the vertices j of the other cells
 * inside the kernel, |x_j - x_i|^2 < rk^2, the closest one (ties: lower cell,
 * then lower vertex) is the colliding neighbour.  Reading of the projection:
 * p_i = x_i + (rk - s) n_j, s = (x_i - x_j).n_j, the closest point to x_i on the
 * far side of the plane through x_j + rk n_j normal to n_j.
 * Outputs, cells concatenated: hit_cell/hit_vert (-1 when no foreign vertex is in
 * the kernel) and p ([.][3]; x_i when none). */
int orc_pik(int ncells, const int *nV, const double *const *x, const double *const *nrm, double rk,
            int *hit_cell, int *hit_vert, double *p) {
    if (!(rk > 0)) return ORC_EINVAL;
    double r2 = rk*rk;
    long o = 0;
    for (int a = 0; a < ncells; ++a) {
        for (int i = 0; i < nV[a]; ++i, ++o) {
            const double *xi = x[a] + 3*i;
            double best = r2;
            int bc = -1, bv = -1;
            for (int b = 0; b < ncells; ++b) {
                if (b == a) continue;
                for (int j = 0; j < nV[b]; ++j) {
                    const double *xj = x[b] + 3*j;
                    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
                    double d2 = dx*dx + dy*dy + dz*dz;
                    /* cells and vertices are visited in increasing order: a strict
                       improvement keeps the lowest index among equal distances */
                    if (d2 < best) { best = d2; bc = b; bv = j; }
                }
            }
            hit_cell[o] = bc;
            hit_vert[o] = bv;
            for (int c = 0; c < 3; ++c) p[3*o+c] = xi[c];
            if (bc >= 0) {
                const double *xj = x[bc] + 3*bv, *nj = nrm[bc] + 3*bv;
                double s = (xi[0] - xj[0])*nj[0] + (xi[1] - xj[1])*nj[1] + (xi[2] - xj[2])*nj[2];
                for (int c = 0; c < 3; ++c) p[3*o+c] = xi[c] + (rk - s)*nj[c];
            }
        }
    }
    return ORC_OK;
}

/* --------------------------------------------- immersed boundary (IBM) forces
 * Multi-direct forcing of the supplementary IBM section (after Wang et al. and
 * Ota et al.) on a lattice of nx x ny x nz nodes at x0 + (i, j, k) dx, fluid
 * velocity u [3][nz][ny][nx].  Interpolation u(X) = sum_x u(x) W(x - X) dx^3,
 * W(r) = phi4(rx/dx) phi4(ry/dx) phi4(rz/dx) / dx^3.  Readings: a Lagrangian
 * point stands for the shell volume A_k dx, so the spread force density is
 * F(x) = sum_k f_k W(x - X_k) dx; nodes outside the lattice are left out.
 *   f_0 = (U - u*(X)) A / dt
 *   cycle c = 1..C: F = spread(f_{c-1}); u_c = u* + F dt at the nodes;
 *                   f_c = f_{c-1} + (U - u_c(X)) A / dt
 *   outputs: f_C per point ([N][3]) and F_imm = spread(f_C) ([3][nz][ny][nx]).
 * Peskin's four-point function:
 *   phi4(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8,   |r| <= 1
 *           = (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8, 1 <= |r| <= 2,  0 beyond. */
double orc_phi4(double r) {
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0*a + sqrt(1.0 + 4.0*a - 4.0*a*a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0*a - sqrt(-7.0 + 12.0*a - 4.0*a*a)) / 8.0;
    return 0.0;
}

/* Vertex areas: a third of the areas of the incident triangles.  x: [nV][3]. */
void orc_vertex_areas(const orc_type *T, const double *x, double *a) {
    memset(a, 0, sizeof(double)*T->nV);
    for (int t = 0; t < T->nT; ++t) {
        const int *v = T->tri + 3*t;
        double e1[3], e2[3], cr[3];
        sub3(x + 3*v[1], x + 3*v[0], e1);
        sub3(x + 3*v[2], x + 3*v[0], e2);
        cross3(e1, e2, cr);
        double ar = 0.5*sqrt(dot3(cr, cr));
        for (int k = 0; k < 3; ++k) a[v[k]] += ar / 3.0;
    }
}

typedef struct { int nx, ny, nz; double dx, x0, y0, z0; } orc_lattice;

/* the 4 x 4 x 4 stencil of point X: first node index per axis and weights phi4 */
static void ibm_stencil(const orc_lattice *L, const double *X, int first[3], double w[3][4]) {
    const double o[3] = {L->x0, L->y0, L->z0};
    for (int d = 0; d < 3; ++d) {
        double s = (X[d] - o[d]) / L->dx;
        int i0 = (int)floor(s) - 1;
        first[d] = i0;
        for (int j = 0; j < 4; ++j) w[d][j] = orc_phi4(s - (double)(i0 + j));
    }
}

static void ibm_interp(const orc_lattice *L, const double *u, const double *F, double dt, const double *X,
                       double out[3]) {
    int f[3];
    double w[3][4];
    long nn = (long)L->nx*L->ny*L->nz;
    ibm_stencil(L, X, f, w);
    out[0] = out[1] = out[2] = 0;
    for (int k = 0; k < 4; ++k) {
        int iz = f[2] + k;
        if (iz < 0 || iz >= L->nz) continue;
        for (int j = 0; j < 4; ++j) {
            int iy = f[1] + j;
            if (iy < 0 || iy >= L->ny) continue;
            for (int i = 0; i < 4; ++i) {
                int ix = f[0] + i;
                if (ix < 0 || ix >= L->nx) continue;
                long n = ((long)iz*L->ny + iy)*L->nx + ix;
                double wt = w[0][i]*w[1][j]*w[2][k];
                for (int c = 0; c < 3; ++c) {
                    double uv = u[c*nn + n];
                    if (F) uv += F[c*nn + n]*dt;
                    out[c] += uv*wt;
                }
            }
        }
    }
}

static void ibm_spread(const orc_lattice *L, int N, const double *X, const double *f, double *F) {
    long nn = (long)L->nx*L->ny*L->nz;
    double sc = 1.0 / (L->dx*L->dx);           /* W dx = phi phi phi / dx^2 */
    memset(F, 0, sizeof(double)*3*nn);
    for (int p = 0; p < N; ++p) {
        int fi[3];
        double w[3][4];
        ibm_stencil(L, X + 3*p, fi, w);
        for (int k = 0; k < 4; ++k) {
            int iz = fi[2] + k;
            if (iz < 0 || iz >= L->nz) continue;
            for (int j = 0; j < 4; ++j) {
                int iy = fi[1] + j;
                if (iy < 0 || iy >= L->ny) continue;
                for (int i = 0; i < 4; ++i) {
                    int ix = fi[0] + i;
                    if (ix < 0 || ix >= L->nx) continue;
                    long n = ((long)iz*L->ny + iy)*L->nx + ix;
                    double wt = w[0][i]*w[1][j]*w[2][k]*sc;
                    for (int c = 0; c < 3; ++c) F[c*nn + n] += f[3*p + c]*wt;
                }
            }
        }
    }
}

/* N Lagrangian points X, U ([N][3]), areas A ([N]); see the block comment above. */
int orc_ibm(int N, const double *X, const double *U, const double *A, int nx, int ny, int nz, double dx,
            double x0, double y0, double z0, const double *u, double dt, int cycles, double *f, double *Fimm) {
    if (N < 0 || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dt > 0) || cycles < 0) return ORC_EINVAL;
    orc_lattice L = {nx, ny, nz, dx, x0, y0, z0};
    for (int p = 0; p < N; ++p) {
        double ui[3];
        ibm_interp(&L, u, NULL, dt, X + 3*p, ui);
        for (int c = 0; c < 3; ++c) f[3*p + c] = (U[3*p + c] - ui[c]) * A[p] / dt;
    }
    for (int cyc = 0; cyc < cycles; ++cyc) {
        ibm_spread(&L, N, X, f, Fimm);
        for (int p = 0; p < N; ++p) {
            double ui[3];
            ibm_interp(&L, u, Fimm, dt, X + 3*p, ui);
            for (int c = 0; c < 3; ++c) f[3*p + c] += (U[3*p + c] - ui[c]) * A[p] / dt;
        }
    }
    ibm_spread(&L, N, X, f, Fimm);
    return ORC_OK;
}
