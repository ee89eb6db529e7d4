// contact.cuh -- particle-in-kernel (PIK) collision framework of the cell
// suspension (arXiv 1911.03062, Sec. 2.2 and the supplementary PIK section):
// every vertex looks for vertices of other cells inside its interpolation
// kernel (a sphere of radius rk); the closest one is its colliding neighbour,
// the vertex's fluid force is dropped and the step adds the collision energy
// kc/2 |x_i - p_i|^2 with the projection
//
//   p_i = x_i + (rk - s) n_j,   s = (x_i - x_j).n_j,
//
// n_j the neighbour's area-weighted vertex normal (the closest point to x_i on
// the far side of the plane through x_j + rk n_j), fixed over the step.
//
// Search: all vertices of all cells are binned on a grid of cells slightly
// larger than rk (so every neighbour within rk lies in the 27 surrounding grid
// cells), keyed by the grid coordinates wrapped into 2^bx x 2^by x 2^bz buckets
// (bx + by + bz = log2 of the bucket count, a power of two >= 2x the vertices;
// neighbours along x are adjacent buckets, so the 27-cell query reads 9 runs of
// 3 consecutive buckets), counting-sorted (count, scan, scatter), and queried
// in bucket order.  Candidates are screened in FP32 with a margin that covers
// the FP32 rounding of both points, and decided in FP64.  Ties in distance go
// to the lower public (cell, vertex) index, so the result does not depend on
// the scatter order.
#pragma once

#include <climits>

#include "common.cuh"

namespace npfem {

// One mesh type's cells, as the search and the target kernel see them.
struct PikType {
    const double *xn;            // state SoA [cell][3][nVp], internal vertex order
    const double *vn;            // velocities, same layout
    const long long *pub_off;    // [cell] offset of the cell in the public arrays (doubles)
    const int *vpub;             // [nV] public index of internal vertex v
    const int *ring_ptr;         // [nV + 1] vertex -> incident triangles
    const int *ring_bc;          // the two other vertices of each, CCW: vb | vc << 16
    int nV, nVp, ncells;
    int vbase;                   // first flat vertex id of the type (flat = vbase + cell nV + v)
    int cbase;                   // first global cell id of the type
};

constexpr int PIK_MAX_TYPES = 32;

struct PikTypes {
    PikType t[PIK_MAX_TYPES];
    int ntypes;
};

struct PikEntry {                // 24 bytes: a binned vertex (FP32 copy for the screen)
    float x, y, z;
    int pub;                     // public vertex index over all cells (tie-break order)
    int owner;                   // global cell id
    int flat;                    // flat vertex id
};

struct PikGrid {
    double inv_cell;             // 1 / grid cell edge
    int bx, by;                  // bits of the x and y grid coordinates in a key
    unsigned mask;               // buckets - 1 (a power of two)
};

__device__ __forceinline__ unsigned pik_key(long long ix, long long iy, long long iz, const PikGrid &g) {
    const unsigned mx = (1u << g.bx) - 1u, my = (1u << g.by) - 1u;
    const unsigned k = ((unsigned)ix & mx) | (((unsigned)iy & my) << g.bx) | ((unsigned)iz << (g.bx + g.by));
    return k & g.mask;
}

__device__ __forceinline__ long long pik_coord(double x, double inv_cell) { return (long long)floor(x * inv_cell); }

// |b - a|^2 without contraction: the same roundings as a plain C evaluation
__device__ __forceinline__ double dist2_rn(double ax, double ay, double az, double bx, double by, double bz) {
    const double dx = __dsub_rn(bx, ax), dy = __dsub_rn(by, ay), dz = __dsub_rn(bz, az);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// 1. bucket of every vertex of type ti; count per bucket
__global__ void k_pik_bin(const PikTypes T, int ti, PikGrid g, unsigned *__restrict__ cnt, unsigned *__restrict__ key) {
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
        const double *x = P.xn + (long long)cell * 3 * P.nVp;
        const unsigned k = pik_key(pik_coord(x[v], g.inv_cell), pik_coord(x[P.nVp + v], g.inv_cell),
                                   pik_coord(x[2 * P.nVp + v], g.inv_cell), g);
        key[P.vbase + i] = k;
        atomicAdd(cnt + k, 1u);
    }
}

// 2. exclusive scan of the counts (n + 1 entries with the last count zero, so
//    out[n] is the total): blocks of 4096, block sums, block offsets
constexpr int SCAN_B = 1024, SCAN_ITEMS = 4;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *wsum, unsigned &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) wsum[w] = s;
    __syncthreads();
    if (w == 0) {
        unsigned ws = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += t;
        }
        wsum[lane] = ws;                          // inclusive warp-sum prefix
    }
    __syncthreads();
    const unsigned before = (w > 0 ? wsum[w - 1] : 0u) + s - v;
    total = wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_B) k_scan_blocks(const unsigned *__restrict__ in, unsigned *__restrict__ out,
                                                        unsigned *__restrict__ bsum, long long n) {
    __shared__ unsigned wsum[32];
    const long long base = (long long)blockIdx.x * SCAN_B * SCAN_ITEMS + (long long)threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    unsigned total;
    unsigned run = block_excl_scan(s, wsum, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_B) k_scan_sums(unsigned *__restrict__ bsum, int nb) {
    __shared__ unsigned wsum[32];
    unsigned carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_B) {
        const int i = b0 + threadIdx.x;
        const unsigned v = i < nb ? bsum[i] : 0u;
        unsigned total;
        const unsigned e = block_excl_scan(v, wsum, total);
        if (i < nb) bsum[i] = carry + e;
        carry += total;
    }
}

__global__ void k_scan_add(unsigned *__restrict__ out, const unsigned *__restrict__ bsum, long long n) {
    const long long base = (long long)blockIdx.x * SCAN_B * SCAN_ITEMS;
    const unsigned add = bsum[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_B * SCAN_ITEMS; k += blockDim.x)
        if (base + k < n) out[base + k] += add;
}

// 3. scatter every vertex of type ti into its bucket's range
__global__ void k_pik_scatter(const PikTypes T, int ti, const unsigned *__restrict__ key,
                              const unsigned *__restrict__ start, unsigned *__restrict__ fill,
                              PikEntry *__restrict__ ent, double *__restrict__ pos64) {
    const PikType &P = T.t[ti];
    const long long n = (long long)P.ncells * P.nV;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nV), v = (int)(i - (long long)cell * P.nV);
        const double *x = P.xn + (long long)cell * 3 * P.nVp;
        const unsigned k = key[P.vbase + i];
        const unsigned pos = start[k] + atomicAdd(fill + k, 1u);
        const double px = x[v], py = x[P.nVp + v], pz = x[2 * P.nVp + v];
        PikEntry e;
        e.x = (float)px;
        e.y = (float)py;
        e.z = (float)pz;
        e.pub = (int)(P.pub_off[cell] / 3) + P.vpub[v];
        e.owner = P.cbase + cell;
        e.flat = (int)(P.vbase + i);
        ent[pos] = e;
        pos64[3ll * pos] = px;
        pos64[3ll * pos + 1] = py;
        pos64[3ll * pos + 2] = pz;
    }
}

// 4. closest foreign vertex inside the kernel, one binned vertex per thread in bucket order;
//    hit[flat] = flat id of the neighbour or -1; the number of contaminated vertices is
//    added to st->contacts.  Screen: |d_f32| against rk + tol, tol = 1e-6 (|x|+|y|+|z|+rk),
//    and, once a neighbour is found, against its distance + tol (FP64 only for candidates
//    that can still win)
//    (the FP32 copies are within 2^-24 |coordinate| of the FP64 values); the FP64 test
//    |d|^2 < rk^2 then decides.
__global__ void k_pik_query(const PikEntry *__restrict__ ent, const double *__restrict__ pos64,
                            const unsigned *__restrict__ start, long long n, PikGrid g, double rk,
                            int *__restrict__ hit, DevStatus *st) {
    const double r2 = rk * rk;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
        const long long p = base + threadIdx.x;
        int found = 0;
        if (p < n) {
            const PikEntry e = ent[p];
            const double ex = pos64[3 * p], ey = pos64[3 * p + 1], ez = pos64[3 * p + 2];
            const long long cx = pik_coord(ex, g.inv_cell), cy = pik_coord(ey, g.inv_cell), cz = pik_coord(ez, g.inv_cell);
            const float tol = 1e-6f * (fabsf(e.x) + fabsf(e.y) + fabsf(e.z) + (float)rk);
            const float rs = (float)rk + tol, rs2 = rs * rs;
            double best = r2;
            int bpub = INT_MAX, bflat = -1;
            float thr2 = rs2;       // screen: FP32 |d|^2 above it cannot be inside rk nor beat the best
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy) {
                    const unsigned b0 = pik_key(cx - 1, cy + dy, cz + dz, g), b1 = pik_key(cx, cy + dy, cz + dz, g),
                                   b2 = pik_key(cx + 1, cy + dy, cz + dz, g);
                    // the three x-neighbours as one range when their buckets are consecutive
                    unsigned lo[3], hi[3];
                    int nr;
                    if (b1 == b0 + 1 && b2 == b1 + 1) {
                        lo[0] = start[b0];
                        hi[0] = start[b2 + 1];
                        nr = 1;
                    } else {
                        lo[0] = start[b0]; hi[0] = start[b0 + 1];
                        lo[1] = start[b1]; hi[1] = start[b1 + 1];
                        lo[2] = start[b2]; hi[2] = start[b2 + 1];
                        nr = 3;
                    }
                    for (int r = 0; r < nr; ++r)
                        for (unsigned k = lo[r]; k < hi[r]; ++k) {
                            const PikEntry c = ent[k];
                            const float fx = c.x - e.x, fy = c.y - e.y, fz = c.z - e.z;
                            if (c.owner == e.owner || fx * fx + fy * fy + fz * fz > thr2) continue;
                            const double d2 = dist2_rn(ex, ey, ez, pos64[3ll * k], pos64[3ll * k + 1], pos64[3ll * k + 2]);
                            if (d2 < r2 && (d2 < best || (d2 == best && c.pub < bpub))) {
                                best = d2;
                                bpub = c.pub;
                                bflat = c.flat;
                                // later candidates need |d| <= sqrt(best): screen at (sqrt(best) + tol)^2,
                                // widened by 1e-6 twice for this bound's own FP32 roundings
                                const float sb = sqrtf((float)best) * (1.0f + 1e-6f) + tol;
                                thr2 = fminf(rs2, sb * sb * (1.0f + 1e-6f));
                            }
                        }
                }
            hit[e.flat] = bflat;
            found = bflat >= 0;
        }
        const unsigned b = __ballot_sync(0xffffffffu, found);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(&st->contacts, (unsigned long long)__popc(b));
    }
}

// 5. targets of type ti: kcol[cell][nVp] = kc on contaminated vertices (0 elsewhere),
//    ccol[cell][3][nVp] = p - x_n (the push, 0 elsewhere); k_predict turns the push into
//    p - y once y is known
template <typename T>
__global__ void k_pik_target(const PikTypes TT, int ti, const int *__restrict__ hit, double rk, double kc,
                             T *__restrict__ kcol, T *__restrict__ ccol) {
    const PikType &P = TT.t[ti];
    const long long n = (long long)P.ncells * P.nVp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i / P.nVp), v = (int)(i - (long long)cell * P.nVp);
        T *cc = ccol + (long long)cell * 3 * P.nVp;
        const int h = v < P.nV ? hit[P.vbase + (long long)cell * P.nV + v] : -1;
        if (h < 0) {
            kcol[i] = T(0);
            cc[v] = cc[P.nVp + v] = cc[2 * P.nVp + v] = T(0);
            continue;
        }
        int tj = 0;
        while (tj + 1 < TT.ntypes && h >= TT.t[tj + 1].vbase) ++tj;
        const PikType &Q = TT.t[tj];
        const int cj = (h - Q.vbase) / Q.nV, vj = h - Q.vbase - cj * Q.nV;
        const double *xq = Q.xn + (long long)cj * 3 * Q.nVp;
        const double *xi = P.xn + (long long)cell * 3 * P.nVp;
        const double a0 = xq[vj], a1 = xq[Q.nVp + vj], a2 = xq[2 * Q.nVp + vj];
        double n0 = 0, n1 = 0, n2 = 0;
        for (int k = Q.ring_ptr[vj]; k < Q.ring_ptr[vj + 1]; ++k) {
            const int vb = Q.ring_bc[k] & 0xffff, vc = Q.ring_bc[k] >> 16;
            const double b0 = xq[vb] - a0, b1 = xq[Q.nVp + vb] - a1, b2 = xq[2 * Q.nVp + vb] - a2;
            const double c0 = xq[vc] - a0, c1 = xq[Q.nVp + vc] - a1, c2 = xq[2 * Q.nVp + vc] - a2;
            n0 += b1 * c2 - b2 * c1;
            n1 += b2 * c0 - b0 * c2;
            n2 += b0 * c1 - b1 * c0;
        }
        const double l = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        if (l > 0) { n0 /= l; n1 /= l; n2 /= l; }
        const double s = (xi[v] - a0) * n0 + (xi[P.nVp + v] - a1) * n1 + (xi[2 * P.nVp + v] - a2) * n2;
        const double w = rk - s;
        kcol[i] = T(kc);
        cc[v] = T(w * n0);
        cc[P.nVp + v] = T(w * n1);
        cc[2 * P.nVp + v] = T(w * n2);
    }
}

}  // namespace npfem
