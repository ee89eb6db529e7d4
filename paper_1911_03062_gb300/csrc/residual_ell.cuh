// residual_ell.cuh -- refinement residual r = q - P z of the mixed global step
// (Supplementary Sec. 2.1: P is the constant system matrix of the quadratic
// energies, z the current approximation of P^{-1} q from the low-precision
// inverse), one block per cell, persistent over the cells of a mesh type.
//
// P's off-diagonal entries are a fixed-width row table (ELL, W slots per
// vertex row, rows with fewer entries padded with column 0 / value 0), the
// same for every cell: each thread keeps the rows of its vertices
// v = tid + k * blockDim.x (k < KR) in registers for the whole launch.
// Each cell's z and q (3 nVp FP32 each) are brought into a 4-stage shared
// ring by 1D bulk async copies (mbarrier complete_tx), so the loads of the
// next cells are in flight while the current one is evaluated.  The
// diagonal is the float pair dhi + dlo applied with exact FMAs, the sums of
// r^2 and q^2 are float-float accumulations reduced in warp order; warp 0
// takes the convergence decision and issues the next copies.
//
// Every wait is bounded: on expiry the kernel records NPFEM_ETIMEOUT, stops,
// waits (bounded) for the copies it issued, and returns.
#pragma once

#include "gemm_tc.cuh"

namespace npfem {

constexpr int RESID_STAGES = 4;
constexpr int RESID_MAX_THREADS = 256;

struct ResidEllArgs {
    int ncells, nV, nVp, first, final_pass;
    float tol2;                      // convergence: |r|^2 <= tol2 |q|^2
    const float *dhi, *dlo;          // [nVp] diag(P) = dhi + dlo, zero for v >= nV
    const unsigned short *ell_col;   // [W][nVp] column of slot w of row v
    const float *ell_val;            // [W][nVp] value of slot w of row v
    const float *q, *z;              // [cell][3][nVp]
    __nv_bfloat16 *r_bf16;           // BF16 form (high part when r_lo is set)
    __nv_bfloat16 *r_lo;             // split corrections: r - r_hi in BF16, or null
    float *r_f32;                    // TF32 form
    int *conv;                       // [cell]
    const int *prev_active;          // the previous sweep left no cell unconverged if 0 here (null: run)
    int *any_active;
    DevStatus *st;
};

template <int W, int KR>
__global__ void __launch_bounds__(RESID_MAX_THREADS, (KR * W <= 24) ? 3 : 2) k_residual_ell(ResidEllArgs a) {
    if (a.prev_active && *a.prev_active == 0) return;   // uniform: every cell already converged
    extern __shared__ __align__(16) unsigned char smem_res[];
    __shared__ uint64_t full[RESID_STAGES];
    __shared__ int cell_sh[RESID_STAGES];
    __shared__ float4 red[2][RESID_MAX_THREADS / 32];
    __shared__ int abort_sh;
    __shared__ int conv_sh;    // the current cell converged (deferred stores)

    const int nVp = a.nVp, n3 = 3 * nVp, nV = a.nV;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const uint32_t vec_bytes = (uint32_t)n3 * 4u;
    float *ring = reinterpret_cast<float *>(smem_res);   // stage s: z at 2 s n3, q at (2 s + 1) n3

    // this thread's rows of P (columns packed two per register)
    uint32_t colp[KR][W / 2];
    float val[KR][W], dh[KR], dl[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int v = tid + k * nt;
        const bool in = v < nVp;
#pragma unroll
        for (int w = 0; w < W; w += 2) {
            const uint32_t c0 = in ? __ldg(a.ell_col + (size_t)w * nVp + v) : 0u;
            const uint32_t c1 = in ? __ldg(a.ell_col + (size_t)(w + 1) * nVp + v) : 0u;
            colp[k][w / 2] = c0 | (c1 << 16);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) val[k][w] = in ? __ldg(a.ell_val + (size_t)w * nVp + v) : 0.f;
        dh[k] = in ? __ldg(a.dhi + v) : 0.f;
        dl[k] = in ? __ldg(a.dlo + v) : 0.f;
    }

    // producer (warp 0): next candidate cell of this block, uses of each stage.
    // The candidates' convergence flags are read 32 at a time and the first
    // active one is found by a ballot; lane 0 issues the copies.
    int next = blockIdx.x;
    int uses[RESID_STAGES] = {};
    auto issue = [&](int s) {
        int c = -1;
        while (next < a.ncells) {
            const int cand = next + lane * (int)gridDim.x;
            const bool act = cand < a.ncells && (a.first || !a.conv[cand]);
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (m) {
                c = next + (__ffs(m) - 1) * (int)gridDim.x;
                next = c + gridDim.x;
                break;
            }
            next += 32 * gridDim.x;
        }
        if (lane != 0) return;
        cell_sh[s] = c;
        if (c < 0) return;
        ++uses[s];
        float *dz = ring + (size_t)(2 * s) * n3;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::mbar_expect_tx(&full[s], 2u * vec_bytes);
        tc::bulk_g2s(dz, a.z + (size_t)c * n3, vec_bytes, &full[s]);
        tc::bulk_g2s(dz + n3, a.q + (size_t)c * n3, vec_bytes, &full[s]);
    };
    if (warp == 0) {
        if (lane == 0) {
            abort_sh = 0;
            for (int s = 0; s < RESID_STAGES; ++s) tc::mbar_init(&full[s], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        for (int s = 0; s < RESID_STAGES; ++s) issue(s);
    }
    __syncthreads();

    for (int it = 0;; ++it) {
        const int s = it % RESID_STAGES;
        const int cell = cell_sh[s];
        if (cell < 0) break;
        if (!tc::mbar_wait(&full[s], (uint32_t)(it / RESID_STAGES) & 1u)) abort_sh = 1;
        const float *zs = ring + (size_t)(2 * s) * n3;
        const float *qs = zs + n3;
        const size_t base = (size_t)cell * n3;
        // After the first pass most cells converge: there r is kept in registers and
        // stored only for a cell that did not (one extra barrier per cell).
        const bool defer = !a.first && !a.final_pass;
        auto store_r = [&](int v, const float (&r)[3]) {
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
        };
        float rk[KR][3];
        float nr = 0.f, nq = 0.f;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int v = tid + k * nt;
            if (v >= nVp) continue;
            float r[3] = {0.f, 0.f, 0.f};
            if (v < nV) {
                float off[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const int u = (w & 1) ? (int)(colp[k][w / 2] >> 16) : (int)(colp[k][w / 2] & 0xffffu);
                    off[0] = fmaf(val[k][w], zs[u], off[0]);
                    off[1] = fmaf(val[k][w], zs[nVp + u], off[1]);
                    off[2] = fmaf(val[k][w], zs[2 * nVp + u], off[2]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float qv = qs[c * nVp + v], zv = zs[c * nVp + v];
                    float t = __fmaf_rn(-dh[k], zv, qv);
                    t = __fmaf_rn(-dl[k], zv, t);
                    r[c] = __fsub_rn(t, off[c]);
                    nr = fmaf(r[c], r[c], nr);
                    nq = fmaf(qv, qv, nq);
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) rk[k][c] = r[c];
            if (!a.final_pass && !defer) store_r(v, r);
        }
        Acc<float> acc[2];
        acc[0].zero();
        acc[1].zero();
        acc[0].add(nr);
        acc[1].add(nq);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc[0].merge_shfl(0xffffffffu, off);
            acc[1].merge_shfl(0xffffffffu, off);
        }
        float4 *rb = red[it & 1];
        if (lane == 0) rb[warp] = make_float4(acc[0].v.hi, acc[0].v.lo, acc[1].v.hi, acc[1].v.lo);
        __syncthreads();
        if (abort_sh) break;
        if (warp == 0) {
            // warps' sums merged in warp order; the decision needs ~1 % accuracy
            const float4 p = lane < (nt >> 5) ? rb[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            Acc<float> t0{DF{p.x, p.y}}, t1{DF{p.z, p.w}};
#pragma unroll
            for (int off = RESID_MAX_THREADS / 64; off > 0; off >>= 1) {
                t0.merge_shfl(0xffffffffu, off);
                t1.merge_shfl(0xffffffffu, off);
            }
            if (lane == 0) {
                const float nr0 = t0.v.hi, nr1 = t1.v.hi;
                const bool ok = nr0 <= a.tol2 * nr1;
                const float ratio = nr1 > 0.f ? sqrtf(nr0 / nr1) : 0.f;
                if (a.final_pass) {
                    atomicMax(&a.st->max_resid_bits, __float_as_uint(ratio));
                } else {
                    if (ok) atomicMax(&a.st->max_resid_bits, __float_as_uint(ratio));
                    a.conv[cell] = ok ? 1 : 0;
                    conv_sh = ok ? 1 : 0;
                    if (!ok) {
                        atomicOr(a.any_active, 1);
                        atomicAdd(&a.st->refine_sweeps, 1ull);
                    }
                }
            }
            issue(s);       // every thread has finished reading stage s
        }
        if (defer) {
            __syncthreads();
            if (!conv_sh) {
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    const int v = tid + k * nt;
                    if (v < nVp) store_r(v, rk[k]);
                }
            }
        }
    }
    if (abort_sh) {
        if (tid == 0) {   // lane 0 of warp 0 holds the stage uses
            dev_raise(a.st, DEV_ETIMEOUT, 16);
            for (int s = 0; s < RESID_STAGES; ++s)
                if (cell_sh[s] >= 0 && !tc::mbar_wait(&full[s], (uint32_t)(uses[s] - 1) & 1u))
                    dev_raise(a.st, DEV_ETIMEOUT, 17);
        }
        __syncthreads();
    }
}

}  // namespace npfem
