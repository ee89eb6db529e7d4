// gemm_grouped.cuh -- the global step of all mesh types in one persistent
// tcgen05 launch:  Z_p[r][v] (+)= sum_k Q_p[r][k] * Pinv_p[v][k]  for every
// problem p (one mesh type: its stacked right-hand sides and its inverse).
//
// Split form (BF16): each stage also carries the low parts of both operands
// and the accumulator takes Q_hi P_hi + Q_lo P_hi + Q_hi P_lo (~16-bit
// operands, FP32 accumulation) for the refinement corrections.
//
// Work units are (problem, 128-row tile, N tile) triples, numbered problem by
// problem; each block (one per SM) takes units blockIdx.x, + gridDim.x, ...
// Roles (192 threads): warp 0 issues TMA loads of both operands through an
// S-stage shared-memory ring (mbarriers full/empty, phases continue across
// units), warp 1 issues tcgen05.mma into one of two TMEM accumulators
// (128 lanes x 256 columns each), warps 2..5 drain the other accumulator
// (tcgen05.ld) and store Z while the next unit is multiplied
// (mbarriers tfull/tempty).  In accumulate mode (refinement corrections) a
// unit whose cells are all converged is skipped by every role, and rows of
// converged cells are left untouched.  Every wait is bounded; on expiry the
// kernel records NPFEM_ETIMEOUT, stops issuing, waits (bounded) for its own
// copies, frees TMEM and returns.
#pragma once

#include "gemm_tc.cuh"

namespace npfem {
namespace tc {

constexpr int MAXG = 16;

struct GroupProblem {
    int rows, nV, nVp, n_tile, n_ntiles, m_tiles, kblocks, unit_begin;
    const int *conv;
};

struct GroupMaps {
    CUtensorMap q[MAXG];
    CUtensorMap p[MAXG];
    CUtensorMap q_lo[MAXG];   // split products only: low BF16 parts of Q and P^{-1}
    CUtensorMap p_lo[MAXG];
    CUtensorMap z[MAXG];      // Z (FP32, width nV, box 32 x 32, 128-byte swizzle): epilogue stores
};

constexpr uint32_t EPI_BOX_BYTES = 32 * 32 * 4;   // one epilogue warp's 32 rows x 32 columns
constexpr uint32_t EPI_SMEM = 4 * 2 * EPI_BOX_BYTES;   // 4 warps x double buffer

struct GroupArgs {
    int nprob, total_units, stages, accumulate, stage_bytes_b;   // B-tile bytes per stage (max n_tile)
    int split;   // 1: Z (+)= Q_hi P_hi + Q_lo P_hi + Q_hi P_lo (BF16 parts, FP32 accumulation)
    const int *active;   // corrections: 0 here = no cell left unconverged, nothing to do (null: run)
    GroupProblem pr[MAXG];
    DevStatus *st;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct Unit {
    int p, mt, nt;
};

__device__ __forceinline__ Unit decode_unit(const GroupArgs &a, int u) {
    int p = 0;
    while (p + 1 < a.nprob && u >= a.pr[p + 1].unit_begin) ++p;
    const int local = u - a.pr[p].unit_begin;
    Unit r;
    r.p = p;
    r.mt = local / a.pr[p].n_ntiles;
    r.nt = local - r.mt * a.pr[p].n_ntiles;
    return r;
}

// accumulate mode: a unit whose 128 rows belong only to converged cells does nothing
__device__ __forceinline__ bool unit_skipped(const GroupArgs &a, const Unit &w) {
    const GroupProblem &P = a.pr[w.p];
    if (!a.accumulate || !P.conv) return false;
    const int m0 = w.mt * BM;
    const int c0 = m0 / 3, c1 = min(P.rows - 1, m0 + BM - 1) / 3;
    for (int c = c0; c <= c1; ++c)
        if (!P.conv[c]) return false;
    return true;
}

template <bool TF32>
__global__ void __launch_bounds__(192, 1) k_gemm_grouped(const __grid_constant__ GroupMaps maps, GroupArgs a) {
    if (a.active && *a.active == 0) return;      // uniform: before any barrier or TMEM use
    extern __shared__ __align__(1024) uint8_t smem_g[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t base = smem_u32(smem_g);
    uint32_t pad = ((base + 1023u) & ~1023u) - base;
    uint8_t *tiles = smem_g + pad;
    // stage: A_hi | B_hi (| A_lo | B_lo when split); every tile 1024-byte aligned
    const uint32_t a_bytes = BM * KB_BYTES;
    const uint32_t half_bytes = a_bytes + (uint32_t)a.stage_bytes_b;
    const uint32_t stage_bytes = half_bytes * (a.split ? 2u : 1u);
    uint8_t *epi = tiles + (size_t)a.stages * stage_bytes;   // epilogue staging, 1024-byte aligned
    uint64_t *full = reinterpret_cast<uint64_t *>(epi + EPI_SMEM);
    uint64_t *empty = full + a.stages;
    uint64_t *tfull = empty + a.stages;      // [2]
    uint64_t *tempty = tfull + 2;            // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    __shared__ int abort_sh;
    volatile int &abort_flag = abort_sh;
    const int k_per_block = TF32 ? 32 : 64;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < a.stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            long long it = 0;
            int last_phase[16];
            for (int s = 0; s < 16; ++s) last_phase[s] = -1;
            for (int u = blockIdx.x; u < a.total_units && !abort_flag; u += gridDim.x) {
                const Unit w = decode_unit(a, u);
                if (unit_skipped(a, w)) continue;
                const GroupProblem &P = a.pr[w.p];
                const uint32_t bytes = (a_bytes + (uint32_t)P.n_tile * KB_BYTES) * (a.split ? 2u : 1u);
                for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
                    const int s = (int)(it % a.stages);
                    const uint32_t round = (uint32_t)(it / a.stages);
                    if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
                        dev_raise(a.st, DEV_ETIMEOUT, 11);
                        abort_flag = 1;
                        break;
                    }
                    uint8_t *sa = tiles + (size_t)s * stage_bytes;
                    mbar_expect_tx(&full[s], bytes);
                    tma_load_2d(sa, &maps.q[w.p], &full[s], kb * k_per_block, w.mt * BM);
                    tma_load_2d(sa + a_bytes, &maps.p[w.p], &full[s], kb * k_per_block, w.nt * P.n_tile);
                    if (a.split) {
                        tma_load_2d(sa + half_bytes, &maps.q_lo[w.p], &full[s], kb * k_per_block, w.mt * BM);
                        tma_load_2d(sa + half_bytes + a_bytes, &maps.p_lo[w.p], &full[s], kb * k_per_block,
                                    w.nt * P.n_tile);
                    }
                    last_phase[s] = round & 1;
                }
            }
            for (int s = 0; s < a.stages && s < 16; ++s)
                if (last_phase[s] >= 0 && !mbar_wait(&full[s], (uint32_t)last_phase[s])) dev_raise(a.st, DEV_ETIMEOUT, 12);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            long long it = 0;
            int tcount = 0;
            for (int u = blockIdx.x; u < a.total_units && !abort_flag; u += gridDim.x) {
                const Unit w = decode_unit(a, u);
                if (unit_skipped(a, w)) continue;
                const GroupProblem &P = a.pr[w.p];
                const int buf = tcount & 1, use = tcount >> 1;
                if (use > 0 && !mbar_wait(&tempty[buf], (use - 1) & 1)) {
                    dev_raise(a.st, DEV_ETIMEOUT, 13);
                    abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(buf * 256);
                const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, BM, P.n_tile);
                bool ok = true;
                for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
                    const int s = (int)(it % a.stages);
                    const uint32_t round = (uint32_t)(it / a.stages);
                    if (!mbar_wait(&full[s], round & 1) || abort_flag) {
                        dev_raise(a.st, DEV_ETIMEOUT, 14);
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = smem_u32(tiles + (size_t)s * stage_bytes), sb = sa + a_bytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        mma<TF32>(d_tmem, desc_sw128(sa + 32 * k), desc_sw128(sb + 32 * k), idesc,
                                  (kb > 0 || k > 0) ? 1u : 0u);
                    if (a.split) {
                        const uint32_t sal = sa + half_bytes, sbl = sal + a_bytes;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            mma<TF32>(d_tmem, desc_sw128(sal + 32 * k), desc_sw128(sb + 32 * k), idesc, 1u);
                            mma<TF32>(d_tmem, desc_sw128(sa + 32 * k), desc_sw128(sbl + 32 * k), idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[buf]);
                ++tcount;
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5 own TMEM lane quadrants (warp % 4).
        // Each 32-column chunk of the warp's 32 rows goes through a 128-byte-swizzled
        // shared box (chunk j of row r at 16-byte slot j ^ (r & 7): conflict-free) and
        // leaves by one TMA tile store (apply) or TMA reduce-add into Z (corrections:
        // the add happens at L2, no read of Z here); rows of converged cells are
        // staged as zeros.  Two boxes per warp alternate.
        const int quad = warp & 3;
        const uint32_t box0 = smem_u32(epi) + (uint32_t)quad * 2u * EPI_BOX_BYTES;
        int tcount = 0, sb = 0;
        for (int u = blockIdx.x; u < a.total_units; u += gridDim.x) {
            const Unit w = decode_unit(a, u);
            if (unit_skipped(a, w)) continue;
            const GroupProblem &P = a.pr[w.p];
            const int buf = tcount & 1, use = tcount >> 1;
            const bool have = mbar_wait(&tfull[buf], use & 1);
            __syncwarp();
            if (!have) {
                if (lane == 0) dev_raise(a.st, DEV_ETIMEOUT, 15);
                break;
            }
            fence_after();
            const int row = w.mt * BM + quad * 32 + lane;
            const int n0 = w.nt * P.n_tile;
            const bool zero_row = a.accumulate && (row >= P.rows || (P.conv && P.conv[row / 3]));
            for (int c0 = 0; c0 < P.n_tile; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + (uint32_t)(buf * 256) + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
                if (lane == 0) bulk_wait_read_1();          // this box's previous store has read it
                __syncwarp();
                const uint32_t box = box0 + (uint32_t)sb * EPI_BOX_BYTES;
                const uint32_t rbase = box + (uint32_t)lane * 128u;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t a16 = rbase + ((uint32_t)(j ^ (lane & 7)) << 4);
                    if (zero_row) st_shared_v4(a16, 0.f, 0.f, 0.f, 0.f);
                    else st_shared_v4(a16, v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (a.accumulate) tma_reduce_add_2d(&maps.z[w.p], box, n0 + c0, w.mt * BM + quad * 32);
                    else tma_store_2d(&maps.z[w.p], box, n0 + c0, w.mt * BM + quad * 32);
                    bulk_commit();
                }
                sb ^= 1;
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            ++tcount;
        }
        if (lane == 0) bulk_wait_all();
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace tc
}  // namespace npfem
