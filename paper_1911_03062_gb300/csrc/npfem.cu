// npfem.cu -- C ABI of the GB300 npFEM solver: context, mesh-type set-up,
// cell storage, the time-step schedule (CUDA-graph captured) and the
// global-step apply (FP64 SIMT, or tcgen05 TF32/BF16 with FP64-residual
// iterative refinement).  See include/npfem.h for the contract of each call.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "npfem.h"
#include "npfem_internal.h"
#include <fstream>
#include <sstream>

using namespace npfem;

// ------------------------------------------------------------ utilities
namespace {

struct Fail {
    int code;
};

void fail(npfem_ctx *ctx, int code, const char *fmt, ...);

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) fail(ctx, NPFEM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
constexpr int NPFEM_SWEEP_FLAGS = 16;   // per-sweep "a cell is still unconverged" flags (last one: final pass)
thread_local std::string g_create_error = "no error";   // message of the last failed npfem_create

}  // namespace

// ---------------------------------------------------------------- types
struct MeshTypeImpl {
    int nV = 0, nVp = 0, nT = 0, nH = 0;
    double h = 0, ks = 0, ka = 0, kb = 0, kv = 0, V0 = 0;
    // device constants
    std::vector<void *> owned;
    TypeConst<double> tc64{};
    TypeConst<float> tc32{};
    double *Pinv64 = nullptr;
    float *Pinv32 = nullptr;
    __nv_bfloat16 *Pinv16 = nullptr;
    __nv_bfloat16 *Pinv16lo = nullptr;          // split corrections: BF16 low part of P^{-1}
    // Rayleigh damping: Mt^{-1} (Mt = M + h C) for the predictor, in the form's operand type
    double ra = 0, rb = 0;
    bool damped = false;
    double *Minv64 = nullptr;
    float *Minv32 = nullptr, *Minv32lo = nullptr;   // TF32 form: TF32 high part and FP32 rest
    __nv_bfloat16 *Minv16 = nullptr, *Minv16lo = nullptr;
    double *diag = nullptr, *minv = nullptr, *mass = nullptr;
    double mtot = 0;                             // total mass of a cell
    float *dhi = nullptr, *dlo = nullptr;
    int *op = nullptr;
    int2 *oe = nullptr;
    // vertex numbering: vpub[i] = caller's index of internal vertex i, vint its inverse
    int *vpub = nullptr, *vint = nullptr;
    // edge neighbours of each (internal) vertex, CSR: the median filter's one-rings
    int *adj_ptr = nullptr, *adj = nullptr;
    // fixed-width row table of the off-diagonal entries for the block-per-cell
    // residual (ell_W = 0: rows too long or too many vertices, CSR kernel)
    unsigned short *ell_col = nullptr;
    float *ell_val = nullptr;
    int ell_W = 0, ell_KR = 0, ell_nt = 0, ell_grid = 0;
    // tensor-core GEMM configuration and the right-hand-side row count it was tuned for
    int n_tile = 0, stages = 0;
    long long tuned_rows = 0;
    CUtensorMap mapP{}, mapPlo{}, mapM{}, mapMlo{};
    // cells
    int ncells = 0, cap = 0;
    std::vector<long long> pub_off_h;
    long long *pub_off = nullptr;
    double *xn = nullptr, *vn = nullptr;        // state SoA FP64
    void *yrel = nullptr, *delta = nullptr, *grad = nullptr, *q = nullptr, *z = nullptr;
    void *S = nullptr, *Y = nullptr, *rlo = nullptr;
    void *zp = nullptr;                          // Rayleigh-damped type: Mt^{-1}(M v_n + h F_ext), kept for the step
    void *kcol = nullptr, *ccol = nullptr;       // PIK: [cell][nVp] stiffness (0: no contact), [cell][3][nVp] p - y
    int *ring_bc = nullptr;                      // vertex -> triangle incidences: the other two vertices
    __nv_bfloat16 *rlo_lo = nullptr;             // split corrections: BF16 low part of r
    __nv_bfloat16 *q16 = nullptr;
    double *y64 = nullptr, *origin = nullptr, *rho = nullptr, *alpha = nullptr, *M = nullptr, *g = nullptr, *allow = nullptr;
    int *hcount = nullptr, *hhead = nullptr, *conv = nullptr, *fb_list = nullptr, *fb_count = nullptr;
    CUtensorMap mapQ{}, mapR{}, mapRlo{}, mapZ{}, mapZp{};
    int ept = 8, block = 256, stash_T = 0;
    size_t smem_step = 0;
    int pf_iter = 0, pf_pred = 0;                // L2 prefetch distance: resident blocks of the kernel
};

constexpr int F_CHUNKS = 4;   // pieces of the host force copy (see npfem_step)

struct npfem_ctx {
    npfem_options opt{};
    int device = 0, nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<MeshTypeImpl *> types;
    long long ndofs = 0;
    double *d_f = nullptr;               // device copy of host forces (public layout)
    // host forces arrive in F_CHUNKS pieces on the copy stream (ev_chunk[i]: piece i is in),
    // each type's predictor launched per piece; ev_done: the last step has read d_f
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_chunk[F_CHUNKS] = {};
    cudaEvent_t ev_done = nullptr;
    double **d_fslot = nullptr;          // device slot: base of the forces read by the step
    double *d_stage = nullptr;           // staging for get/set (public layout)
    double *d_ffilt = nullptr;           // median-filtered forces (public layout), force_median only
    // particle-in-kernel search (pik_radius > 0): buckets, binned vertices, result per flat vertex
    unsigned *d_pik_cnt = nullptr, *d_pik_start = nullptr, *d_pik_fill = nullptr, *d_pik_key = nullptr;
    unsigned *d_pik_bsum = nullptr;
    PikEntry *d_pik_ent = nullptr;
    double *d_pik_pos = nullptr;         // FP64 positions of the binned vertices [pos][3]
    int *d_pik_hit = nullptr;
    long long pik_n = 0, pik_h = 0;
    // immersed-boundary forces: per-point stencils and areas of the last call
    IbmPoint *d_ibm_pts = nullptr;
    double *d_ibm_area = nullptr;
    long long ibm_cap = 0;
    DevStatus *d_st = nullptr;
    DevStatus *h_st = nullptr;           // pinned
    int *d_any = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_valid = false;
    bool graph_early = false;            // the graph was captured without the predictor
    bool stepped = false;
    int smem_optin = 0;
    // launch accounting and optional per-kernel CUDA-event timing
    long long launches_per_step = 0, launch_counter = 0;
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;       // start/end pairs, one pair per launch of a step
    std::vector<int> prof_cls;              // kernel class of each pair
    size_t prof_next = 0, graph_prof_pairs = 0;
    double prof_ms[NPFEM_KCLASSES] = {0};
    long long prof_n[NPFEM_KCLASSES] = {0};
    std::string err;
};

namespace {

void fail(npfem_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    throw Fail{code};
}

template <typename F>
int guard(npfem_ctx *ctx, F &&f) {
    try {
        f();
        return NPFEM_OK;
    } catch (Fail &e) {
        return e.code;
    } catch (std::bad_alloc &) {
        if (ctx) ctx->err = "host allocation failed";
        return NPFEM_ENOMEM;
    }
}

template <typename T>
T *dalloc(npfem_ctx *ctx, size_t n, std::vector<void *> *owned = nullptr) {
    if (n == 0) n = 1;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(ctx, e == cudaErrorMemoryAllocation ? NPFEM_ENOMEM : NPFEM_ECUDA, "cudaMalloc(%zu bytes): %s",
             n * sizeof(T), cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(p, 0, n * sizeof(T), ctx->stream);
    if (e != cudaSuccess) fail(ctx, NPFEM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    if (owned) owned->push_back(p);
    return reinterpret_cast<T *>(p);
}

template <typename T>
T *upload(npfem_ctx *ctx, const std::vector<T> &v, std::vector<void *> &owned) {
    T *p = dalloc<T>(ctx, v.size(), &owned);
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return p;
}

void dfree(void *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

bool mixed(const npfem_ctx *ctx) { return ctx->opt.precision != NPFEM_FP64; }
bool bf16(const npfem_ctx *ctx) { return ctx->opt.precision == NPFEM_MIXED_BF16; }
size_t esize(const npfem_ctx *ctx) { return mixed(ctx) ? sizeof(float) : sizeof(double); }

void get_encode(npfem_ctx *ctx) {
    if (g_encode) return;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        fail(ctx, NPFEM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

// 2D tensor map over a row-major [rows][stride] matrix whose first `inner`
// columns are valid; box = 128 bytes of K x box_rows, 128-byte swizzle.
CUtensorMap make_map(npfem_ctx *ctx, const void *base, bool is_bf16, int inner, long long rows, int stride,
                     int box_rows) {
    get_encode(ctx);
    CUtensorMap m;
    const int es = is_bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)stride * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(&m, is_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(ctx, NPFEM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return m;
}

int grid_for(long long n, int block, int cap = 1 << 20) {
    long long g = (n + block - 1) / block;
    return (int)std::max(1ll, std::min<long long>(g, cap));
}

// Every kernel launch of a step goes through prof_begin / prof_end: counts
// the launch and, when profiling, brackets it with a pair of CUDA events on
// the context stream (captured into the graph as event nodes).
// an event record on the context stream: an external record node when the
// stream is being captured (so that the graph records it at each replay)
void prof_record(npfem_ctx *ctx, cudaEvent_t e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) CK(cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal));
    else CK(cudaEventRecord(e, ctx->stream));
}

void prof_begin(npfem_ctx *ctx, int cls) {
    ctx->launch_counter++;
    if (!ctx->prof_on) return;
    if (ctx->prof_next + 2 > ctx->prof_ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            ctx->prof_ev.push_back(e);
        }
        ctx->prof_cls.resize(ctx->prof_ev.size() / 2);
    }
    ctx->prof_cls[ctx->prof_next / 2] = cls;
    prof_record(ctx, ctx->prof_ev[ctx->prof_next]);
}

void prof_end(npfem_ctx *ctx) {
    if (!ctx->prof_on) return;
    prof_record(ctx, ctx->prof_ev[ctx->prof_next + 1]);
    ctx->prof_next += 2;
}

void prof_harvest(npfem_ctx *ctx, size_t pairs) {
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < pairs; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        ctx->prof_ms[ctx->prof_cls[i]] += ms;
        ctx->prof_n[ctx->prof_cls[i]] += 1;
    }
}

}  // namespace

// ------------------------------------------------------ kernel dispatch
namespace {

template <typename T>
IterArgs<T> make_args(npfem_ctx *ctx, MeshTypeImpl *t) {
    IterArgs<T> a{};
    if constexpr (sizeof(T) == 8) a.tc = t->tc64;
    else a.tc = t->tc32;
    a.ncells = t->ncells;
    a.zpred = (const T *)t->zp;
    a.kcol = (const T *)t->kcol;
    a.ccol = (T *)t->ccol;
    a.m = ctx->opt.history;
    a.max_bt = ctx->opt.max_backtracks;
    a.use_allow = mixed(ctx) ? 1 : 0;
    a.stash_T = t->stash_T;
    a.h = t->h;
    a.inv_h = 1.0 / t->h;
    a.c1 = ctx->opt.armijo_c1;
    a.curv_tol = ctx->opt.curvature_tol;
    a.curv_tol2 = ctx->opt.curvature_tol * ctx->opt.curvature_tol;
    a.xn = t->xn;
    a.vn = t->vn;
    a.fptr = ctx->d_fslot;
    a.pub_off = t->pub_off;
    a.vpub = t->vpub;
    a.minv = t->minv;
    a.yrel = (T *)t->yrel;
    a.y64 = t->y64;
    a.origin = t->origin;
    a.delta = (T *)t->delta;
    a.grad = (T *)t->grad;
    a.q = (T *)t->q;
    a.z = (T *)t->z;
    a.q_bf16 = t->q16;
    a.S = (T *)t->S;
    a.Y = (T *)t->Y;
    a.rho = t->rho;
    a.alpha = t->alpha;
    a.M = t->M;
    a.g = t->g;
    a.allow = t->allow;
    a.hcount = t->hcount;
    a.hhead = t->hhead;
    a.fb_list = t->fb_list;
    a.fb_count = t->fb_count;
    a.st = ctx->d_st;
    return a;
}

// Resident blocks of the per-cell kernels (blocks per SM x SMs): a k_predict block
// prefetches into L2 the state and forces of the cell that many blocks ahead, which
// starts about when it ends.  (In k_iterate the same prefetch of the next wave's
// vectors evicted the history pairs the running blocks re-read from L2: +15 % at three
// blocks per SM; at four, where those re-reads miss L2 anyway, prefetching the next
// wave's z and y_i still measured +1.5 %.)
template <typename T, int EPT, int MAXB>
void prefetch_distance_t(npfem_ctx *ctx, MeshTypeImpl *t) {
    int bi = 0, bp = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bi, k_iterate<T, EPT, MAXB>, t->block, t->smem_step));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bp, k_predict<T, EPT, MAXB>, t->block, t->smem_step));
    t->pf_iter = bi * ctx->nsm;
    t->pf_pred = bp * ctx->nsm;
}

template <typename T, int EPT, int MAXB>
void run_predict_t(npfem_ctx *ctx, MeshTypeImpl *t, int c0, int c1) {
    IterArgs<T> a = make_args<T>(ctx, t);
    a.pf_dist = t->pf_pred;
    a.cell0 = c0;
    a.ncells = c1;
    prof_begin(ctx, NPFEM_K_PREDICT);
    k_predict<T, EPT, MAXB><<<c1 - c0, t->block, t->smem_step, ctx->stream>>>(a);
    CK(cudaGetLastError());
    prof_end(ctx);
}

template <typename T, int EPT, int MAXB>
void run_iterate_t(npfem_ctx *ctx, MeshTypeImpl *t, int last, bool fallback) {
    IterArgs<T> a = make_args<T>(ctx, t);
    a.last = last;
    prof_begin(ctx, fallback ? NPFEM_K_FALLBACK : NPFEM_K_ITERATE);
    if (!fallback) {
        k_iterate<T, EPT, MAXB><<<t->ncells, t->block, t->smem_step, ctx->stream>>>(a, nullptr, nullptr);
    } else {
        int grid = std::min(t->ncells, 2 * ctx->nsm);
        k_iterate<T, EPT, MAXB><<<grid, t->block, t->smem_step, ctx->stream>>>(a, t->fb_list, t->fb_count);
    }
    CK(cudaGetLastError());
    prof_end(ctx);
}

#define DISPATCH_EPT(T, FN, ...)                                         \
    do {                                                                 \
        if (t->ept == 4) FN<T, 4, 256>(__VA_ARGS__);                     \
        else if (t->ept == 8) FN<T, 8, 256>(__VA_ARGS__);                \
        else FN<T, 16, 512>(__VA_ARGS__);                                \
    } while (0)

void run_predict(npfem_ctx *ctx, MeshTypeImpl *t, int c0, int c1) {
    if (mixed(ctx)) DISPATCH_EPT(float, run_predict_t, ctx, t, c0, c1);
    else DISPATCH_EPT(double, run_predict_t, ctx, t, c0, c1);
}

void run_iterate(npfem_ctx *ctx, MeshTypeImpl *t, int last, bool fallback) {
    if (mixed(ctx)) DISPATCH_EPT(float, run_iterate_t, ctx, t, last, fallback);
    else DISPATCH_EPT(double, run_iterate_t, ctx, t, last, fallback);
}

void set_prefetch_distance(npfem_ctx *ctx, MeshTypeImpl *t) {
    if (mixed(ctx)) DISPATCH_EPT(float, prefetch_distance_t, ctx, t);
    else DISPATCH_EPT(double, prefetch_distance_t, ctx, t);
}

// --- global step: z = P^{-1} q for the stacked rows of every type (one grouped launch)
size_t grouped_smem(int stages, int max_ntile, bool split = false) {
    return 1024 + (size_t)stages * (tc::BM + max_ntile) * tc::KB_BYTES * (split ? 2 : 1) + tc::EPI_SMEM +
           (2 * stages + 4) * 8 + 16;
}
size_t gemm_smem(const MeshTypeImpl *t) { return grouped_smem(t->stages, t->n_tile); }

// Kernel attributes are set at set-up time (never inside a stream capture),
// to the device's opt-in maximum so that every type's request fits.
using ResidEllFn = void (*)(ResidEllArgs);

ResidEllFn resid_ell_fn(int W, int KR) {
    switch (W * 10 + KR) {
    case 121: return k_residual_ell<12, 1>;
    case 122: return k_residual_ell<12, 2>;
    case 123: return k_residual_ell<12, 3>;
    case 124: return k_residual_ell<12, 4>;
    case 161: return k_residual_ell<16, 1>;
    case 162: return k_residual_ell<16, 2>;
    case 163: return k_residual_ell<16, 3>;
    case 164: return k_residual_ell<16, 4>;
    default: return nullptr;
    }
}

size_t resid_ell_smem(int nVp) { return (size_t)RESID_STAGES * 2 * 3 * nVp * sizeof(float); }

bool split(const npfem_ctx *ctx) { return bf16(ctx) && ctx->opt.refine_split; }

void set_kernel_attrs(npfem_ctx *ctx) {
    int mx = 0;
    CK(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    auto all = [&](auto fn) {
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, fn));
        CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes));
    };
    {
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, k_ibm_spread_box));
        CK(cudaFuncSetAttribute(k_ibm_spread_box, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(IBM_BOX_DOUBLES * sizeof(double))));
    }
    if (mixed(ctx)) {
        all(k_predict<float, 4, 256>); all(k_predict<float, 8, 256>); all(k_predict<float, 16, 512>);
        all(k_iterate<float, 4, 256>); all(k_iterate<float, 8, 256>); all(k_iterate<float, 16, 512>);
        all(k_fallback_apply<float>);
        all(tc::k_gemm_grouped<false>);
        all(tc::k_gemm_grouped<true>);
    } else {
        all(k_predict<double, 4, 256>); all(k_predict<double, 8, 256>); all(k_predict<double, 16, 512>);
        all(k_iterate<double, 4, 256>); all(k_iterate<double, 8, 256>); all(k_iterate<double, 16, 512>);
        all(k_fallback_apply<double>);
    }
    all(k_residual<false>);
    all(k_residual<true>);
    for (int W : {12, 16})
        for (int KR = 1; KR <= 4; ++KR) all(resid_ell_fn(W, KR));
    all(k_force_median);
    ctx->smem_optin = mx;
}

struct GemmItem {
    const MeshTypeImpl *t;
    const CUtensorMap *mapQ;
    int rows;
    const CUtensorMap *mapZ;               // Z (FP32, width nV, 32 x 32 boxes)
    const int *conv;
    const CUtensorMap *mapQlo = nullptr;   // split form: low part of Q (P's low part from the type)
    const CUtensorMap *mapB = nullptr;     // the matrix instead of P^{-1} (Mt^{-1}: damped predictor)
    const CUtensorMap *mapBlo = nullptr;   // its low part (split form)
};

// One persistent launch (per MAXG items) over every item's (row tile, N tile) units.
void gemm_group(npfem_ctx *ctx, const std::vector<GemmItem> &items, int accumulate, bool split_form = false,
                const int *active = nullptr) {
    for (size_t i0 = 0; i0 < items.size(); i0 += tc::MAXG) {
        const size_t i1 = std::min(items.size(), i0 + tc::MAXG);
        tc::GroupArgs g{};
        tc::GroupMaps maps;
        int max_nt = 16, stages = 0, best_rows = -1, units = 0;
        for (size_t i = i0; i < i1; ++i) {
            const GemmItem &it = items[i];
            tc::GroupProblem &P = g.pr[g.nprob];
            P.rows = it.rows;
            P.nV = it.t->nV;
            P.nVp = it.t->nVp;
            P.n_tile = it.t->n_tile;
            P.n_ntiles = (it.t->nV + it.t->n_tile - 1) / it.t->n_tile;
            P.m_tiles = (it.rows + tc::BM - 1) / tc::BM;
            P.kblocks = (it.t->nV * (bf16(ctx) ? 2 : 4) + tc::KB_BYTES - 1) / tc::KB_BYTES;
            P.unit_begin = units;
            P.conv = it.conv;
            units += P.m_tiles * P.n_ntiles;
            maps.q[g.nprob] = *it.mapQ;
            maps.p[g.nprob] = it.mapB ? *it.mapB : it.t->mapP;
            maps.z[g.nprob] = *it.mapZ;
            if (split_form) {
                maps.q_lo[g.nprob] = *it.mapQlo;
                maps.p_lo[g.nprob] = it.mapBlo ? *it.mapBlo : it.t->mapPlo;
            }
            max_nt = std::max(max_nt, it.t->n_tile);
            if (it.rows > best_rows) { best_rows = it.rows; stages = it.t->stages; }
            ++g.nprob;
        }
        if (!units) continue;
        while (stages > 2 && grouped_smem(stages, max_nt, split_form) + 2048 > (size_t)ctx->smem_optin) --stages;
        g.total_units = units;
        g.stages = stages;
        g.accumulate = accumulate;
        g.split = split_form ? 1 : 0;
        g.active = active;
        g.stage_bytes_b = max_nt * tc::KB_BYTES;
        g.st = ctx->d_st;
        const int grid = std::min(units, ctx->nsm);
        const size_t smem = grouped_smem(stages, max_nt, split_form);
        prof_begin(ctx, accumulate ? NPFEM_K_GEMM_REFINE : NPFEM_K_GEMM);
        if (bf16(ctx)) tc::k_gemm_grouped<false><<<grid, 192, smem, ctx->stream>>>(maps, g);
        else tc::k_gemm_grouped<true><<<grid, 192, smem, ctx->stream>>>(maps, g);
        CK(cudaGetLastError());
        prof_end(ctx);
    }
}

void gemm_tc(npfem_ctx *ctx, MeshTypeImpl *t, const CUtensorMap &mapQ, int rows, const CUtensorMap &mapZ,
             int accumulate, const int *conv, const CUtensorMap *mapQlo = nullptr) {
    gemm_group(ctx, {GemmItem{t, &mapQ, rows, &mapZ, conv, mapQlo}}, accumulate, mapQlo != nullptr);
}

void residual(npfem_ctx *ctx, MeshTypeImpl *t, int rows_cells, const float *q, const float *z, void *r,
              int *conv, int first, int final_pass, __nv_bfloat16 *r_lo = nullptr, int *active = nullptr,
              const int *prev_active = nullptr) {
    ResidArgs a{};
    a.ncells = rows_cells;
    a.nV = t->nV;
    a.nVp = t->nVp;
    a.first = first;
    a.final_pass = final_pass;
    a.tol = ctx->opt.refine_tol;
    a.diag = t->diag;
    a.dhi = t->dhi;
    a.dlo = t->dlo;
    a.op = t->op;
    a.oe = t->oe;
    a.q = q;
    a.z = z;
    a.r_bf16 = bf16(ctx) ? (__nv_bfloat16 *)r : nullptr;
    a.r_f32 = bf16(ctx) ? nullptr : (float *)r;
    a.r_lo = r_lo;
    a.conv = conv;
    a.any_active = active ? active : ctx->d_any + NPFEM_SWEEP_FLAGS - 1;
    a.prev_active = prev_active;
    a.st = ctx->d_st;
    if (t->ell_W && !ctx->opt.residual_fp64) {
        ResidEllArgs e{};
        e.ncells = rows_cells;
        e.nV = t->nV;
        e.nVp = t->nVp;
        e.first = first;
        e.final_pass = final_pass;
        e.tol2 = (float)(ctx->opt.refine_tol * ctx->opt.refine_tol);
        e.dhi = t->dhi;
        e.dlo = t->dlo;
        e.ell_col = t->ell_col;
        e.ell_val = t->ell_val;
        e.q = q;
        e.z = z;
        e.r_bf16 = a.r_bf16;
        e.r_f32 = a.r_f32;
        e.r_lo = r_lo;
        e.conv = conv;
        e.any_active = a.any_active;
        e.prev_active = prev_active;
        e.st = ctx->d_st;
        const int grid = std::min(rows_cells, t->ell_grid);
        prof_begin(ctx, NPFEM_K_RESIDUAL);
        resid_ell_fn(t->ell_W, t->ell_KR)<<<grid, t->ell_nt, resid_ell_smem(t->nVp), ctx->stream>>>(e);
        CK(cudaGetLastError());
        prof_end(ctx);
        return;
    }
    // one warp per cell, up to 8 warps per block, each warp's z in shared memory
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / (12 * (size_t)t->nVp)));
    const size_t smem = (size_t)wpb * 3 * t->nVp * sizeof(float);
    const int grid = std::min((rows_cells + wpb - 1) / wpb, 3 * ctx->nsm);
    prof_begin(ctx, NPFEM_K_RESIDUAL);
    if (ctx->opt.residual_fp64) k_residual<true><<<grid, 32 * wpb, smem, ctx->stream>>>(a);
    else k_residual<false><<<grid, 32 * wpb, smem, ctx->stream>>>(a);
    CK(cudaGetLastError());
    prof_end(ctx);
}

// z = P^{-1} q for every cell of every type (q / z buffers of the types):
// FP64 form: one SIMT GEMM per type; mixed forms: grouped tensor-core applies
// and refinement sweeps (a residual per type between grouped corrections).
void apply_all(npfem_ctx *ctx) {
    if (!mixed(ctx)) {
        for (auto *t : ctx->types) {
            if (!t->ncells) continue;
            const int rows = 3 * t->ncells;
            dim3 grid((t->nV + SG_T - 1) / SG_T, (rows + SG_T - 1) / SG_T);
            prof_begin(ctx, NPFEM_K_GEMM);
            k_gemm_simt<double><<<grid, 256, 0, ctx->stream>>>(rows, t->nV, t->nVp, (const double *)t->q,
                                                               t->Pinv64, (double *)t->z);
            CK(cudaGetLastError());
            prof_end(ctx);
        }
        return;
    }
    std::vector<GemmItem> first, corr;
    for (auto *t : ctx->types) {
        if (!t->ncells) continue;
        first.push_back(GemmItem{t, &t->mapQ, 3 * t->ncells, &t->mapZ, nullptr});
        corr.push_back(GemmItem{t, &t->mapR, 3 * t->ncells, &t->mapZ, t->conv, split(ctx) ? &t->mapRlo : nullptr});
    }
    // per-sweep flags: residual pass s raises flag s when it leaves a cell unconverged;
    // the correction of sweep s and every later pass return at once while it is 0
    CK(cudaMemsetAsync(ctx->d_any, 0, NPFEM_SWEEP_FLAGS * sizeof(int), ctx->stream));
    auto flag = [&](int sweep) { return ctx->d_any + std::min(sweep, NPFEM_SWEEP_FLAGS - 2); };
    gemm_group(ctx, first, 0);
    for (int s = 0; s < ctx->opt.refine_max; ++s) {
        for (auto *t : ctx->types)
            if (t->ncells)
                residual(ctx, t, t->ncells, (const float *)t->q, (const float *)t->z, t->rlo, t->conv, s == 0, 0,
                         t->rlo_lo, flag(s), s == 0 ? nullptr : flag(s - 1));
        gemm_group(ctx, corr, 1, split(ctx), flag(s));
    }
    for (auto *t : ctx->types)
        if (t->ncells)
            residual(ctx, t, t->ncells, (const float *)t->q, (const float *)t->z, nullptr, t->conv,
                     ctx->opt.refine_max == 0, 1, nullptr, ctx->d_any + NPFEM_SWEEP_FLAGS - 1,
                     ctx->opt.refine_max == 0 ? nullptr : flag(ctx->opt.refine_max - 1));
}

void fallback_apply(npfem_ctx *ctx, MeshTypeImpl *t) {
    int grid = std::min(t->ncells, 2 * ctx->nsm);
    size_t smem = 3 * (size_t)t->nVp * esize(ctx);
    prof_begin(ctx, NPFEM_K_FALLBACK_APPLY);
    if (mixed(ctx))
        k_fallback_apply<float><<<grid, 256, smem, ctx->stream>>>(t->nV, t->nVp, t->Pinv32, (const float *)t->q,
                                                                  (float *)t->z, t->fb_list, t->fb_count);
    else
        k_fallback_apply<double><<<grid, 256, smem, ctx->stream>>>(t->nV, t->nVp, t->Pinv64, (const double *)t->q,
                                                                   (double *)t->z, t->fb_list, t->fb_count);
    CK(cudaGetLastError());
    prof_end(ctx);
}

__global__ void k_set_ptr(double **slot, const double *p) { *slot = const_cast<double *>(p); }

// Particle-in-kernel buffers for the current cells: buckets (a power of two >= 2x the
// vertices), binned vertices and the per-vertex result.
void pik_alloc(npfem_ctx *ctx) {
    long long n = 0;
    for (auto *t : ctx->types) n += (long long)t->ncells * t->nV;
    if (n > (1ll << 30)) fail(ctx, NPFEM_EINVAL, "%lld vertices exceed the collision search's 2^30", n);
    long long h = 1024;
    while (h < 2 * n) h <<= 1;
    void **bufs[] = {(void **)&ctx->d_pik_cnt, (void **)&ctx->d_pik_start, (void **)&ctx->d_pik_fill,
                     (void **)&ctx->d_pik_key, (void **)&ctx->d_pik_bsum, (void **)&ctx->d_pik_ent,
                     (void **)&ctx->d_pik_pos, (void **)&ctx->d_pik_hit};
    for (void **b : bufs) dfree(*b);
    ctx->pik_n = -1;                     // until every buffer is in place: a search refuses to run
    ctx->pik_h = 0;
    const long long nb = (h + 1 + SCAN_B * SCAN_ITEMS - 1) / (SCAN_B * SCAN_ITEMS);
    ctx->d_pik_cnt = dalloc<unsigned>(ctx, h + 1);
    ctx->d_pik_start = dalloc<unsigned>(ctx, h + 1);
    ctx->d_pik_fill = dalloc<unsigned>(ctx, h);
    ctx->d_pik_key = dalloc<unsigned>(ctx, std::max(1ll, n));
    ctx->d_pik_bsum = dalloc<unsigned>(ctx, nb);
    ctx->d_pik_ent = dalloc<PikEntry>(ctx, std::max(1ll, n));
    ctx->d_pik_pos = dalloc<double>(ctx, 3 * std::max(1ll, n));
    ctx->d_pik_hit = dalloc<int>(ctx, std::max(1ll, n));
    ctx->pik_n = n;
    ctx->pik_h = h;
}

// Descriptors of the types that hold cells (flat vertex ids: types in order, cells,
// internal vertices); returns the number of vertices.
long long point_types(npfem_ctx *ctx, PikTypes &pt, std::vector<MeshTypeImpl *> &tl) {
    pt = PikTypes{};
    tl.clear();
    long long vb = 0;
    int cb = 0;
    for (auto *t : ctx->types) {
        if (!t->ncells) continue;
        if (pt.ntypes == PIK_MAX_TYPES) fail(ctx, NPFEM_EINVAL, "at most %d mesh types with cells", PIK_MAX_TYPES);
        PikType &P = pt.t[pt.ntypes++];
        P.xn = t->xn;
        P.vn = t->vn;
        P.pub_off = t->pub_off;
        P.vpub = t->vpub;
        P.ring_ptr = mixed(ctx) ? t->tc32.vt_ptr : t->tc64.vt_ptr;
        P.ring_bc = t->ring_bc;
        P.nV = t->nV;
        P.nVp = t->nVp;
        P.ncells = t->ncells;
        P.vbase = (int)vb;
        P.cbase = cb;
        vb += (long long)t->ncells * t->nV;
        cb += t->ncells;
        tl.push_back(t);
    }
    if (vb > (1ll << 30)) fail(ctx, NPFEM_EINVAL, "%lld vertices exceed 2^30", vb);
    return vb;
}

// The collision search and targets of one step (positions at the start of the step):
// bin, scan, scatter, query, targets; see contact.cuh.
void pik_search(npfem_ctx *ctx) {
    PikTypes pt{};
    std::vector<MeshTypeImpl *> tl;
    const long long vb = point_types(ctx, pt, tl);
    if (vb != ctx->pik_n) fail(ctx, NPFEM_ESTATE, "collision search buffers out of date");
    const double rk = ctx->opt.pik_radius;
    int kb = 0;
    while ((1ll << kb) < ctx->pik_h) ++kb;
    const int bx = (kb + 2) / 3, by = (kb - bx + 1) / 2;
    const PikGrid g{1.0 / (rk * (1.0 + 1e-9)), bx, by, (unsigned)(ctx->pik_h - 1)};
    const long long H = ctx->pik_h, N = ctx->pik_n;
    CK(cudaMemsetAsync(ctx->d_pik_cnt, 0, (H + 1) * sizeof(unsigned), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_pik_fill, 0, H * sizeof(unsigned), ctx->stream));
    auto launch = [&](auto &&fn) {
        prof_begin(ctx, NPFEM_K_CONTACT);
        fn();
        CK(cudaGetLastError());
        prof_end(ctx);
    };
    for (int ti = 0; ti < pt.ntypes; ++ti) {
        const long long n = (long long)pt.t[ti].ncells * pt.t[ti].nV;
        launch([&] { k_pik_bin<<<grid_for(n, 256, 16 * ctx->nsm), 256, 0, ctx->stream>>>(pt, ti, g, ctx->d_pik_cnt,
                                                                                      ctx->d_pik_key); });
    }
    const int nb = (int)((H + 1 + SCAN_B * SCAN_ITEMS - 1) / (SCAN_B * SCAN_ITEMS));
    launch([&] { k_scan_blocks<<<nb, SCAN_B, 0, ctx->stream>>>(ctx->d_pik_cnt, ctx->d_pik_start, ctx->d_pik_bsum, H + 1); });
    launch([&] { k_scan_sums<<<1, SCAN_B, 0, ctx->stream>>>(ctx->d_pik_bsum, nb); });
    launch([&] { k_scan_add<<<nb, SCAN_B, 0, ctx->stream>>>(ctx->d_pik_start, ctx->d_pik_bsum, H + 1); });
    for (int ti = 0; ti < pt.ntypes; ++ti) {
        const long long n = (long long)pt.t[ti].ncells * pt.t[ti].nV;
        launch([&] { k_pik_scatter<<<grid_for(n, 256, 16 * ctx->nsm), 256, 0, ctx->stream>>>(
                         pt, ti, ctx->d_pik_key, ctx->d_pik_start, ctx->d_pik_fill, ctx->d_pik_ent, ctx->d_pik_pos); });
    }
    if (N > 0)
        launch([&] { k_pik_query<<<grid_for(N, 256, 16 * ctx->nsm), 256, 0, ctx->stream>>>(
                         ctx->d_pik_ent, ctx->d_pik_pos, ctx->d_pik_start, N, g, rk, ctx->d_pik_hit, ctx->d_st); });
    for (int ti = 0; ti < pt.ntypes; ++ti) {
        MeshTypeImpl *t = tl[ti];
        const long long n = (long long)t->ncells * t->nVp;
        if (mixed(ctx))
            launch([&] { k_pik_target<float><<<grid_for(n, 256, 16 * ctx->nsm), 256, 0, ctx->stream>>>(
                             pt, ti, ctx->d_pik_hit, rk, ctx->opt.collision_k, (float *)t->kcol, (float *)t->ccol); });
        else
            launch([&] { k_pik_target<double><<<grid_for(n, 256, 16 * ctx->nsm), 256, 0, ctx->stream>>>(
                             pt, ti, ctx->d_pik_hit, rk, ctx->opt.collision_k, (double *)t->kcol, (double *)t->ccol); });
    }
}

// Rayleigh-damped types: zp = Mt^{-1}(M v_n + h F_ext) for every cell, read by the
// predictor (y = x_n + h zp) and again where the last iteration re-forms y in FP64.
// FP64 form: SIMT FP64 apply; mixed forms: one grouped tensor-core apply of operands
// split into high and low parts (three products, FP32 accumulation), no refinement.
void damped_predictor_rhs(npfem_ctx *ctx) {
    std::vector<GemmItem> items;
    for (auto *t : ctx->types) {
        if (!t->ncells || !t->damped) continue;
        const long long total = 3ll * t->nVp * t->ncells;
        const int grid = grid_for(total, 256, 8 * ctx->nsm);
        prof_begin(ctx, NPFEM_K_PREDICT);
        if (mixed(ctx))
            k_damp_rhs<float><<<grid, 256, 0, ctx->stream>>>(t->ncells, t->nV, t->nVp, t->mass, t->vn, ctx->d_fslot,
                                                             t->pub_off, t->vpub, t->h, (float *)t->q,
                                                             bf16(ctx) ? t->q16 : nullptr, t->rlo_lo,
                                                             bf16(ctx) ? nullptr : (float *)t->rlo,
                                                             (const float *)t->kcol);
        else
            k_damp_rhs<double><<<grid, 256, 0, ctx->stream>>>(t->ncells, t->nV, t->nVp, t->mass, t->vn, ctx->d_fslot,
                                                              t->pub_off, t->vpub, t->h, (double *)t->q, nullptr,
                                                              nullptr, nullptr, (const double *)t->kcol);
        CK(cudaGetLastError());
        prof_end(ctx);
        if (!mixed(ctx)) {
            const int rows = 3 * t->ncells;
            dim3 g2((t->nV + SG_T - 1) / SG_T, (rows + SG_T - 1) / SG_T);
            prof_begin(ctx, NPFEM_K_GEMM);
            k_gemm_simt<double><<<g2, 256, 0, ctx->stream>>>(rows, t->nV, t->nVp, (const double *)t->q, t->Minv64,
                                                              (double *)t->zp);
            CK(cudaGetLastError());
            prof_end(ctx);
        } else {
            // low part of b: the BF16 low buffer, or (TF32) the FP32 residual buffer, free until
            // the first refinement sweep of the step
            GemmItem it{t, &t->mapQ, 3 * t->ncells, &t->mapZp, nullptr, bf16(ctx) ? &t->mapRlo : &t->mapR};
            it.mapB = &t->mapM;
            it.mapBlo = &t->mapMlo;
            items.push_back(it);
        }
    }
    if (!items.empty()) gemm_group(ctx, items, 0, true);
}

void enqueue_step(npfem_ctx *ctx, bool with_predict) {
    // counters only: a pending error word survives until a synchronising call reads it
    CK(cudaMemsetAsync(reinterpret_cast<char *>(ctx->d_st) + sizeof(unsigned long long), 0,
                       sizeof(DevStatus) - sizeof(unsigned long long), ctx->stream));
    if (ctx->opt.force_median) {
        // filtered copy of the forces; the step then reads it through the slot
        for (auto *t : ctx->types) {
            if (!t->ncells) continue;
            prof_begin(ctx, NPFEM_K_FILTER);
            k_force_median<<<std::min(t->ncells, 8 * ctx->nsm), 256, 2 * 3 * (size_t)t->nV * sizeof(double),
                             ctx->stream>>>(t->ncells, t->nV, t->pub_off, t->vpub, t->adj_ptr, t->adj, ctx->d_fslot,
                                            ctx->d_ffilt);
            CK(cudaGetLastError());
            prof_end(ctx);
        }
        prof_begin(ctx, NPFEM_K_FILTER);
        k_set_ptr<<<1, 1, 0, ctx->stream>>>(ctx->d_fslot, ctx->d_ffilt);
        CK(cudaGetLastError());
        prof_end(ctx);
    }
    if (ctx->opt.pik_radius > 0) pik_search(ctx);
    damped_predictor_rhs(ctx);
    if (with_predict)
        for (auto *t : ctx->types)
            if (t->ncells) run_predict(ctx, t, 0, t->ncells);
    const int K = ctx->opt.iters;
    for (int k = 0; k < K; ++k) {
        const int last = (k == K - 1);
        apply_all(ctx);
        for (auto *t : ctx->types) {
            if (!t->ncells) continue;
            CK(cudaMemsetAsync(t->fb_count, 0, sizeof(int), ctx->stream));
            run_iterate(ctx, t, last, false);
            fallback_apply(ctx, t);
            run_iterate(ctx, t, last, true);
        }
    }
    if (ctx->opt.pbd_kappa > 0) {
        for (auto *t : ctx->types) {
            if (!t->ncells) continue;
            prof_begin(ctx, NPFEM_K_FILTER);
            if (mixed(ctx))
                k_pbd_damping_f32<<<std::min(t->ncells, 8 * ctx->nsm), 256, 0, ctx->stream>>>(
                    t->ncells, t->nV, t->nVp, t->mass, 1.0 / t->mtot, t->xn, t->vn, (float)ctx->opt.pbd_kappa);
            else
                k_pbd_damping<<<std::min(t->ncells, 8 * ctx->nsm), 256, 0, ctx->stream>>>(
                    t->ncells, t->nV, t->nVp, t->mass, t->xn, t->vn, ctx->opt.pbd_kappa);
            CK(cudaGetLastError());
            prof_end(ctx);
        }
    }
    if (ctx->opt.u_max > 0) {
        for (auto *t : ctx->types) {
            if (!t->ncells) continue;
            prof_begin(ctx, NPFEM_K_FILTER);
            k_vel_cap<<<grid_for((long long)t->ncells * t->nV, 256, 8192), 256, 0, ctx->stream>>>(
                t->ncells, t->nV, t->nVp, t->vn, ctx->opt.u_max);
            CK(cudaGetLastError());
            prof_end(ctx);
        }
    }
}

}  // namespace

// ---------------------------------------------------------- mesh set-up
namespace {

struct V3 {
    double x, y, z;
};
V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 crs(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double dt3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
double nrm(V3 a) { return std::sqrt(dt3(a, a)); }

struct HostType {
    std::vector<int> tri;               // nT*3
    std::vector<double> dinv, area;     // nT*4, nT
    std::vector<int> hv;                // nH*4
    std::vector<double> hc, hrest;      // nH*4, nH
    std::vector<int> vt_ptr, vt_inc, vh_ptr, vh_inc;
    std::vector<double> vt_g, vh_c;
    std::vector<double> P;              // dense nV*nV
    std::vector<double> Mt;             // dense nV*nV, Rayleigh-damped types only: M + h C
    double V0 = 0;
};

// Internal vertex numbering: reverse Cuthill-McKee order of the vertex graph
// (bandwidth-reducing), so the vertices a warp touches in the element loops
// and vertex gathers have nearby indices, i.e. mostly distinct shared-memory
// banks.  Start of each component: a pseudo-peripheral vertex (two rounds of
// "minimum degree in the last BFS level"); ties by degree, then index.
// Returns pub[i] = caller's index of internal vertex i.
std::vector<int> rcm_order(int nV, int nT, const int32_t *tris) {
    std::vector<std::vector<int>> adj(nV);
    for (int t = 0; t < nT; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
            adj[a].push_back(b);
            adj[b].push_back(a);
        }
    for (auto &l : adj) {
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
    }
    auto deg = [&](int v) { return (int)adj[v].size(); };
    auto by_degree = [&](int a, int b) { return deg(a) != deg(b) ? deg(a) < deg(b) : a < b; };
    std::vector<int> order, level(nV, -1);
    order.reserve(nV);
    std::vector<char> placed(nV, 0);
    std::vector<int> q;
    auto bfs_last_level_min = [&](int s) {
        std::fill(level.begin(), level.end(), -1);
        q.assign(1, s);
        level[s] = 0;
        for (size_t i = 0; i < q.size(); ++i)
            for (int u : adj[q[i]])
                if (level[u] < 0) { level[u] = level[q[i]] + 1; q.push_back(u); }
        const int last = level[q.back()];
        int best = -1;
        for (int v : q)
            if (level[v] == last && (best < 0 || by_degree(v, best))) best = v;
        return best;
    };
    for (;;) {
        int s = -1;
        for (int v = 0; v < nV; ++v)
            if (!placed[v] && (s < 0 || by_degree(v, s))) s = v;
        if (s < 0) break;
        s = bfs_last_level_min(bfs_last_level_min(s));
        const size_t first = order.size();
        order.push_back(s);
        placed[s] = 1;
        for (size_t i = first; i < order.size(); ++i) {
            std::vector<int> nb;
            for (int u : adj[order[i]])
                if (!placed[u]) nb.push_back(u);
            std::sort(nb.begin(), nb.end(), by_degree);
            for (int u : nb) { placed[u] = 1; order.push_back(u); }
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// Validate the mesh and build the element constants:
//   triangles: D_m^{-1} in the triangle's rest frame, rest area;
//   hinges   : every edge shared by t1 = (a, b, c) and t2 = (b, a, d):
//              x0 = a, x1 = b, x2 = c, x3 = d, cotangent stencil scaled by
//              sqrt(3 / (A1 + A2)), rest |b|;
//   incidence lists per vertex (sorted by element), rest volume, dense P.
void build_host_type(npfem_ctx *ctx, int nV, const double *X, int nT, const int32_t *tris, const double *mass,
                     const npfem_material &m, const int *vpub, const int *tpub, HostType &H) {
    // vpub / tpub: the caller's number of each (internal) vertex / triangle, for messages
    auto P3 = [&](int i) { return V3{X[3 * i], X[3 * i + 1], X[3 * i + 2]}; };
    H.tri.assign(tris, tris + 3 * nT);
    for (int i = 0; i < 3 * nT; ++i)
        if (tris[i] < 0 || tris[i] >= nV) fail(ctx, NPFEM_EINVAL, "triangle index %d out of range", tris[i]);
    for (int t = 0; t < nT; ++t) {
        const int *v = &H.tri[3 * t];
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2])
            fail(ctx, NPFEM_EINVAL, "triangle %d repeats a vertex", tpub[t]);
    }
    // half-edge twins
    std::unordered_map<long long, int> he;
    he.reserve(6 * nT);
    for (int t = 0; t < nT; ++t)
        for (int k = 0; k < 3; ++k) {
            long long a = H.tri[3 * t + k], b = H.tri[3 * t + (k + 1) % 3];
            if (!he.emplace(a * nV + b, 3 * t + k).second)
                fail(ctx, NPFEM_EINVAL, "edge (%d,%d) used twice with the same orientation", vpub[a], vpub[b]);
        }
    for (auto &kv : he) {
        long long a = kv.first / nV, b = kv.first % nV;
        if (!he.count(b * nV + a))
            fail(ctx, NPFEM_EINVAL, "open or inconsistently oriented mesh at edge (%d,%d)", vpub[a], vpub[b]);
    }
    // triangle constants
    H.dinv.resize(4 * nT);
    H.area.resize(nT);
    for (int t = 0; t < nT; ++t) {
        const int *v = &H.tri[3 * t];
        V3 E1 = sub(P3(v[1]), P3(v[0])), E2 = sub(P3(v[2]), P3(v[0]));
        V3 n = crs(E1, E2);
        double nn = nrm(n), l1 = nrm(E1), l2 = nrm(E2);
        if (!(nn > 1e-14 * l1 * l2)) fail(ctx, NPFEM_EINVAL, "degenerate triangle %d", tpub[t]);
        V3 u = {E1.x / l1, E1.y / l1, E1.z / l1};
        V3 nh = {n.x / nn, n.y / nn, n.z / nn};
        V3 w = crs(nh, u);
        double a = dt3(E1, u), b = dt3(E2, u), c = dt3(E1, w), d = dt3(E2, w);
        double det = a * d - b * c;
        H.dinv[4 * t + 0] = d / det;
        H.dinv[4 * t + 1] = -b / det;
        H.dinv[4 * t + 2] = -c / det;
        H.dinv[4 * t + 3] = a / det;
        H.area[t] = 0.5 * nn;
    }
    // rest volume (relative to vertex 0); outward orientation required
    {
        V3 o = P3(0);
        double V = 0;
        for (int t = 0; t < nT; ++t) {
            const int *v = &H.tri[3 * t];
            V += dt3(sub(P3(v[0]), o), crs(sub(P3(v[1]), o), sub(P3(v[2]), o)));
        }
        H.V0 = V / 6.0;
        if (!(H.V0 > 0)) fail(ctx, NPFEM_EINVAL, "mesh is not outward oriented (rest volume %g)", H.V0);
    }
    // hinges in order of the first half-edge of each edge
    auto cot_at = [&](V3 a, V3 b, V3 c) {
        V3 u = sub(b, a), v = sub(c, a);
        return dt3(u, v) / nrm(crs(u, v));
    };
    for (int t = 0; t < nT; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = H.tri[3 * t + k], b = H.tri[3 * t + (k + 1) % 3], c = H.tri[3 * t + (k + 2) % 3];
            int tw = he[(long long)b * nV + a];
            if (tw < 3 * t + k) continue;   // the edge was met earlier as its twin
            int t2 = tw / 3, k2 = tw % 3;
            int d = H.tri[3 * t2 + (k2 + 2) % 3];
            V3 X0 = P3(a), X1 = P3(b), X2 = P3(c), X3 = P3(d);
            double c10 = cot_at(X0, X1, X2), c11 = cot_at(X1, X2, X0);
            double c20 = cot_at(X0, X3, X1), c21 = cot_at(X1, X0, X3);
            double sc = std::sqrt(3.0 / (H.area[t] + H.area[t2]));
            double cc[4] = {sc * (c11 + c21), sc * (c10 + c20), -sc * (c10 + c11), -sc * (c20 + c21)};
            int idx[4] = {a, b, c, d};
            V3 bb = {0, 0, 0};
            for (int j = 0; j < 4; ++j) {
                V3 p = P3(idx[j]);
                bb.x += cc[j] * p.x;
                bb.y += cc[j] * p.y;
                bb.z += cc[j] * p.z;
                H.hv.push_back(idx[j]);
                H.hc.push_back(cc[j]);
            }
            H.hrest.push_back(nrm(bb));
        }
    const int nH = (int)H.hrest.size();
    // incidence lists (counting sort keeps element order)
    H.vt_ptr.assign(nV + 1, 0);
    for (int i = 0; i < 3 * nT; ++i) H.vt_ptr[H.tri[i] + 1]++;
    for (int v = 0; v < nV; ++v) H.vt_ptr[v + 1] += H.vt_ptr[v];
    H.vt_inc.resize(3 * nT);
    H.vt_g.resize(6 * nT);
    {
        std::vector<int> fill(H.vt_ptr.begin(), H.vt_ptr.end() - 1);
        for (int t = 0; t < nT; ++t)
            for (int k = 0; k < 3; ++k) {
                int v = H.tri[3 * t + k], pos = fill[v]++;
                const double *Di = &H.dinv[4 * t];
                double g0, g1;
                if (k == 1) { g0 = Di[0]; g1 = Di[1]; }
                else if (k == 2) { g0 = Di[2]; g1 = Di[3]; }
                else { g0 = -Di[0] - Di[2]; g1 = -Di[1] - Di[3]; }
                H.vt_inc[pos] = (t << 2) | k;
                H.vt_g[2 * pos] = g0;
                H.vt_g[2 * pos + 1] = g1;
            }
    }
    H.vh_ptr.assign(nV + 1, 0);
    for (int i = 0; i < 4 * nH; ++i) H.vh_ptr[H.hv[i] + 1]++;
    for (int v = 0; v < nV; ++v) H.vh_ptr[v + 1] += H.vh_ptr[v];
    H.vh_inc.resize(4 * nH);
    H.vh_c.resize(4 * nH);
    {
        std::vector<int> fill(H.vh_ptr.begin(), H.vh_ptr.end() - 1);
        for (int h = 0; h < nH; ++h)
            for (int j = 0; j < 4; ++j) {
                int v = H.hv[4 * h + j], pos = fill[v]++;
                H.vh_inc[pos] = (h << 2) | j;
                H.vh_c[pos] = H.hc[4 * h + j];
            }
    }
    // L = k_vol I + sum_t (ws + wa) A_t^T A_t + sum_e kb A_e^T A_e (assembled in P),
    // then P = (1 + h alpha) M/h^2 + (1 + beta/h) L = Mt/h^2 + L and, when damped,
    // Mt = (1 + h alpha) M + h beta L
    const double h = m.dt, ra = m.rayleigh_alpha, rb = m.rayleigh_beta;
    const bool damped = ra != 0 || rb != 0;
    H.P.assign((size_t)nV * nV, 0.0);
    for (int v = 0; v < nV; ++v) H.P[(size_t)v * nV + v] += damped ? m.k_vol : mass[v] / (h * h) + m.k_vol;
    for (int t = 0; t < nT; ++t) {
        const double *Di = &H.dinv[4 * t];
        double G[3][2] = {{-Di[0] - Di[2], -Di[1] - Di[3]}, {Di[0], Di[1]}, {Di[2], Di[3]}};
        double w = (m.k_strain + m.k_area) * H.area[t];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                H.P[(size_t)H.tri[3 * t + i] * nV + H.tri[3 * t + j]] += w * (G[i][0] * G[j][0] + G[i][1] * G[j][1]);
    }
    for (int h = 0; h < nH; ++h)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                H.P[(size_t)H.hv[4 * h + i] * nV + H.hv[4 * h + j]] += m.k_bend * H.hc[4 * h + i] * H.hc[4 * h + j];
    if (damped) {
        H.Mt.resize(H.P.size());
        for (size_t i = 0; i < H.P.size(); ++i) H.Mt[i] = h * rb * H.P[i];
        for (int v = 0; v < nV; ++v) H.Mt[(size_t)v * nV + v] += (1.0 + h * ra) * mass[v];
        const double sl = 1.0 + rb / h, wm = (1.0 + h * ra) / (h * h);
        for (double &p : H.P) p *= sl;
        for (int v = 0; v < nV; ++v) H.P[(size_t)v * nV + v] += mass[v] * wm;
    }
}

template <typename T>
std::vector<T> cvt(const std::vector<double> &v) {
    return std::vector<T>(v.begin(), v.end());
}

template <typename T>
TypeConst<T> upload_consts(npfem_ctx *ctx, MeshTypeImpl *t, const HostType &H, const std::vector<double> &mass) {
    TypeConst<T> c{};
    c.nV = t->nV;
    c.nVp = t->nVp;
    c.nT = t->nT;
    c.nH = t->nH;
    std::vector<uint2> tri(t->nT);
    std::vector<uint4> hv(t->nH);
    auto u16 = [](int v) { return (unsigned)v & 0xffffu; };
    for (int i = 0; i < t->nT; ++i)
        tri[i] = make_uint2(u16(H.tri[3 * i]) | u16(H.tri[3 * i + 1]) << 16, u16(H.tri[3 * i + 2]));
    for (int i = 0; i < t->nH; ++i) {
        uint4 r = make_uint4(u16(H.hv[4 * i]) | u16(H.hv[4 * i + 1]) << 16, u16(H.hv[4 * i + 2]) | u16(H.hv[4 * i + 3]) << 16, 0, 0);
        if (sizeof(T) == 4) {
            const float rf = (float)H.hrest[i];
            std::memcpy(&r.z, &rf, 4);
        } else {
            const double rd = H.hrest[i];
            uint64_t b;
            std::memcpy(&b, &rd, 8);
            r.z = (unsigned)(b & 0xffffffffu);
            r.w = (unsigned)(b >> 32);
        }
        hv[i] = r;
    }
    std::vector<double> dq(4 * t->nT), mh2(t->nVp, 0.0);   // mh2 zero-padded for 4-wide loads
    for (int i = 0; i < t->nT; ++i) {
        dq[4 * i] = H.dinv[4 * i];
        dq[4 * i + 1] = H.dinv[4 * i + 1];
        dq[4 * i + 2] = H.dinv[4 * i + 3];
        dq[4 * i + 3] = H.area[i];
    }
    // inertia diagonal of the local step: m/h^2, damped (1 + h alpha) m/h^2 + (beta/h) k_vol
    // (Mt's mass part and the volume part of its beta L; the element parts of beta L are
    // evaluated with the elements, weighted by beta/h)
    for (int v = 0; v < t->nV; ++v)
        mh2[v] = t->damped ? (1.0 + t->h * t->ra) * mass[v] / (t->h * t->h) + t->rb / t->h * t->kv
                           : mass[v] / (t->h * t->h);
    c.tri = upload(ctx, tri, t->owned);
    c.dinv = upload(ctx, cvt<T>(dq), t->owned);
    c.ks = (T)t->ks;
    c.ka = (T)t->ka;
    c.hv = upload(ctx, hv, t->owned);
    c.hc = upload(ctx, cvt<T>(H.hc), t->owned);
    std::vector<TriInc<T>> vt(H.vt_inc.size());
    std::vector<int> ring(H.vt_inc.size());
    for (size_t k = 0; k < vt.size(); ++k) {
        const int tt = H.vt_inc[k] >> 2, corner = H.vt_inc[k] & 3;
        const int vb = H.tri[3 * tt + (corner + 1) % 3], vc = H.tri[3 * tt + (corner + 2) % 3];
        vt[k].t = tt;
        vt[k].bc = vb | (vc << 16);
        ring[k] = vt[k].bc;
        vt[k].g0 = (T)H.vt_g[2 * k];
        vt[k].g1 = (T)H.vt_g[2 * k + 1];
    }
    std::vector<HingeInc<T>> vh(H.vh_inc.size());
    for (size_t k = 0; k < vh.size(); ++k) {
        vh[k].h = H.vh_inc[k] >> 2;
        vh[k].c = (T)H.vh_c[k];
    }
    // slot-major padded incidence tables (FP32 path): a vertex's whole one-ring in one round of loads
    int maxt = 0, maxh = 0;
    for (int v = 0; v < t->nV; ++v) {
        maxt = std::max(maxt, H.vt_ptr[v + 1] - H.vt_ptr[v]);
        maxh = std::max(maxh, H.vh_ptr[v + 1] - H.vh_ptr[v]);
    }
    c.pad_t = (sizeof(T) == 4 && maxt <= PAD_T) ? maxt : 0;
    c.pad_h = (sizeof(T) == 4 && maxh <= PAD_H) ? maxh : 0;
    if (c.pad_t) {
        std::vector<int> vp((size_t)c.pad_t * t->nV, -1);
        for (int v = 0; v < t->nV; ++v)
            for (int k = H.vt_ptr[v], q = 0; k < H.vt_ptr[v + 1]; ++k, ++q)
                vp[(size_t)q * t->nV + v] = H.vt_inc[k];          // (t << 2) | corner
        c.vt_pad = upload(ctx, vp, t->owned);
    }
    if (c.pad_h) {
        std::vector<int2> hp((size_t)c.pad_h * t->nV, make_int2(0, 0));
        for (int v = 0; v < t->nV; ++v)
            for (int k = H.vh_ptr[v], q = 0; k < H.vh_ptr[v + 1]; ++k, ++q) {
                float cc = (float)H.vh_c[k];
                int2 e;
                e.x = H.vh_inc[k] >> 2;
                std::memcpy(&e.y, &cc, 4);
                hp[(size_t)q * t->nV + v] = e;
            }
        c.vh_pad = upload(ctx, hp, t->owned);
    }
    c.vt_ptr = upload(ctx, H.vt_ptr, t->owned);
    c.vt = upload(ctx, vt, t->owned);
    t->ring_bc = upload(ctx, ring, t->owned);
    c.vh_ptr = upload(ctx, H.vh_ptr, t->owned);
    c.vh = upload(ctx, vh, t->owned);
    c.mh2 = upload(ctx, cvt<T>(mh2), t->owned);
    c.V0 = H.V0;
    c.V0x6 = 6.0 * H.V0;
    c.vtol6 = 6.0 * Prec<T>::vol_tol * std::fabs(H.V0);
    c.kb = (T)t->kb;
    c.kv = (T)t->kv;
    c.cd = (T)(t->rb / t->h);
    return c;
}

// A^{-1} of an SPD matrix A (P, or Mt) in FP64 on the GPU (Gauss-Jordan), then the
// operand copies the form uses: FP64 (FP64 form), FP32 (mixed forms), BF16 (BF16
// form) and its BF16 low part (want_lo).
struct InvCopies {
    double *i64 = nullptr;
    float *i32 = nullptr, *i32lo = nullptr;
    __nv_bfloat16 *i16 = nullptr, *i16lo = nullptr;
};

InvCopies invert_on_gpu(npfem_ctx *ctx, MeshTypeImpl *t, const std::vector<double> &P, bool want64, bool want_lo,
                        const char *what) {
    InvCopies out;
    const int n = t->nV, nb = (n + GJB - 1) / GJB, npad = nb * GJB;
    std::vector<void *> tmp;
    try {
        // P padded to a multiple of the pivot block with the identity (its inverse is
        // blockdiag(P^{-1}, I)), then blocked Gauss-Jordan: 2 launches per GJB pivots
        std::vector<double> Ap((size_t)npad * npad, 0.0);
        for (int i = 0; i < npad; ++i)
            for (int j = 0; j < npad; ++j)
                Ap[(size_t)i * npad + j] = (i < n && j < n) ? P[(size_t)i * n + j] : (i == j ? 1.0 : 0.0);
        double *A = dalloc<double>(ctx, (size_t)npad * npad, &tmp);
        double *D = dalloc<double>(ctx, GJB * GJB, &tmp);
        double *C = dalloc<double>(ctx, (size_t)npad * GJB, &tmp), *DR = dalloc<double>(ctx, (size_t)npad * GJB, &tmp);
        int *bad = dalloc<int>(ctx, 1, &tmp);
        CK(cudaMemcpyAsync(A, Ap.data(), Ap.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        for (int kb = 0; kb < nb; ++kb) {
            k_bgj_panel<<<nb, 256, 0, ctx->stream>>>(npad, kb, A, D, C, DR, bad);
            k_bgj_update<<<dim3(nb, nb), 256, 0, ctx->stream>>>(npad, kb, A, D, C, DR, bad);
        }
        CK(cudaGetLastError());
        int hbad = 0;
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (hbad) fail(ctx, NPFEM_ENOTSPD, "%s is not positive definite", what);
        if (want64) out.i64 = dalloc<double>(ctx, (size_t)n * t->nVp, &t->owned);
        if (mixed(ctx)) out.i32 = dalloc<float>(ctx, (size_t)n * t->nVp, &t->owned);
        if (bf16(ctx)) out.i16 = dalloc<__nv_bfloat16>(ctx, (size_t)n * t->nVp, &t->owned);
        if (bf16(ctx) && want_lo) out.i16lo = dalloc<__nv_bfloat16>(ctx, (size_t)n * t->nVp, &t->owned);
        if (mixed(ctx) && !bf16(ctx) && want_lo) out.i32lo = dalloc<float>(ctx, (size_t)n * t->nVp, &t->owned);
        k_convert_pinv<<<grid_for((long long)n * t->nVp, 256, 4096), 256, 0, ctx->stream>>>(n, npad, t->nVp, A, out.i64,
                                                                                          out.i32, out.i16,
                                                                                          out.i16lo, out.i32lo);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        for (void *p : tmp) cudaFree(p);
        throw;
    }
    for (void *p : tmp) cudaFree(p);
    return out;
}

// GEMM tile autotuner: for each (device, nV, operand type, right-hand-side row
// bucket) time the grouped tensor-core apply for the N-tile widths that cover nV
// with the fewest (and one more) tiles and 2..6 pipeline stages, on operands
// filled with non-zero values, and keep the fastest.  The bucket is the type's
// row count 3 x cells rounded up to a power of two (at least 3 x 1024); a type is
// tuned at creation for 3 x 8192 rows and again, with its real row count, by the
// first step after its cell count changed bucket (before that step's graph is
// captured).  Timing runs on min(bucket, 3 x 32768) rows.  The grid is not a
// search dimension: every block holds both 256-column TMEM accumulators (512
// columns, the whole TMEM of an SM), so one block per SM, persistent over the
// units, is the only shape that runs all SMs concurrently.  Results are cached
// per process and, when npfem_options.autotune_cache names a file, read from /
// appended to it ("key n_tile stages microseconds" lines).
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tuned;

long long tune_bucket(long long rows) {
    long long b = 3 * 1024;
    while (b < rows) b <<= 1;
    return b;
}

std::string tune_key(npfem_ctx *ctx, int nV, long long bucket) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) prop.name[0] = 0;
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ') c = '_';
    return name + "|nV=" + std::to_string(nV) + "|" + (bf16(ctx) ? "bf16" : "tf32") + "|rows=" + std::to_string(bucket);
}

void choose_tiles(npfem_ctx *ctx, MeshTypeImpl *t, long long want_rows) {
    const void *pb = bf16(ctx) ? (const void *)t->Pinv16 : (const void *)t->Pinv32;
    const long long bucket = tune_bucket(want_rows);
    const std::string key = tune_key(ctx, t->nV, bucket);
    t->tuned_rows = bucket;
    auto use = [&](int nt, int st) {
        t->n_tile = nt;
        t->stages = st;
        t->mapP = make_map(ctx, pb, bf16(ctx), t->nV, t->nV, t->nVp, nt);
        if (t->Pinv16lo) t->mapPlo = make_map(ctx, t->Pinv16lo, true, t->nV, t->nV, t->nVp, nt);
        if (t->damped) {
            t->mapM = make_map(ctx, bf16(ctx) ? (const void *)t->Minv16 : (const void *)t->Minv32, bf16(ctx), t->nV,
                               t->nV, t->nVp, nt);
            if (t->Minv16lo) t->mapMlo = make_map(ctx, t->Minv16lo, true, t->nV, t->nV, t->nVp, nt);
            if (t->Minv32lo) t->mapMlo = make_map(ctx, t->Minv32lo, false, t->nV, t->nV, t->nVp, nt);
        }
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) { use(it->second.first, it->second.second); return; }
        if (ctx->opt.autotune_cache) {
            std::ifstream f(ctx->opt.autotune_cache);
            std::string line;
            while (std::getline(f, line)) {
                std::istringstream ls(line);
                std::string k;
                int nt = 0, st = 0;
                if (ls >> k >> nt >> st && k == key && nt >= 32 && nt <= 256 && nt % 32 == 0 && st >= 2 && st <= 8) {
                    g_tuned[key] = {nt, st};
                    use(nt, st);
                    return;
                }
            }
        }
    }
    const int rows = (int)std::min<long long>(bucket, 3 * 32768);
    std::vector<void *> tmp;
    float best = 1e30f;
    int best_nt = 0, best_st = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        const size_t qbytes = (size_t)rows * t->nVp * (bf16(ctx) ? 2 : 4);
        void *Q = dalloc<unsigned char>(ctx, qbytes, &tmp);
        CK(cudaMemsetAsync(Q, 0x3C, qbytes, ctx->stream));   // every element ~1.1e-2 (BF16 and FP32)
        float *Z = dalloc<float>(ctx, (size_t)rows * t->nVp, &tmp);
        CUtensorMap mq = make_map(ctx, Q, bf16(ctx), t->nV, rows, t->nVp, tc::BM);
        CUtensorMap mz = make_map(ctx, Z, false, t->nV, rows, t->nVp, 32);
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const int base_tiles = (t->nV + 255) / 256;
        for (int ntiles = base_tiles; ntiles <= base_tiles + 1; ++ntiles) {
            // N tile: a multiple of 32 (the epilogue's store box width), at most 256
            int nt = ((t->nV + ntiles - 1) / ntiles + 31) / 32 * 32;
            if (nt > 256 || nt < 16) continue;
            for (int st = 2; st <= 6; ++st) {
                if (grouped_smem(st, nt) + 2048 > (size_t)ctx->smem_optin) continue;
                use(nt, st);
                gemm_tc(ctx, t, mq, rows, mz, 0, nullptr);
                CK(cudaEventRecord(e0, ctx->stream));
                for (int r = 0; r < 5; ++r) gemm_tc(ctx, t, mq, rows, mz, 0, nullptr);
                CK(cudaEventRecord(e1, ctx->stream));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; best_nt = nt; best_st = st; }
            }
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamSynchronize(ctx->stream);
        for (void *p : tmp) cudaFree(p);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaStreamSynchronize(ctx->stream));
    for (void *p : tmp) cudaFree(p);
    if (!best_nt) fail(ctx, NPFEM_EINVAL, "no GEMM tile configuration fits nV = %d", t->nV);
    use(best_nt, best_st);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = {best_nt, best_st};
    if (ctx->opt.autotune_cache) {
        std::ofstream f(ctx->opt.autotune_cache, std::ios::app);
        f << key << " " << best_nt << " " << best_st << " " << (best * 1000.0f / 5.0f) << "\n";
    }
}

void fill_cells(npfem_ctx *ctx, MeshTypeImpl *t, const MeshTypeImpl *old_t, int cap);

void free_cells(MeshTypeImpl *t) {
    void **bufs[] = {(void **)&t->pub_off, (void **)&t->xn, (void **)&t->vn, &t->yrel, &t->delta, &t->grad, &t->q,
                     &t->z, &t->zp, &t->kcol, &t->ccol, &t->S, &t->Y, &t->rlo, (void **)&t->rlo_lo, (void **)&t->q16, (void **)&t->y64, (void **)&t->origin, (void **)&t->rho,
                     (void **)&t->alpha, (void **)&t->M, (void **)&t->g, (void **)&t->allow, (void **)&t->hcount,
                     (void **)&t->hhead, (void **)&t->conv, (void **)&t->fb_list, (void **)&t->fb_count};
    for (void **b : bufs) dfree(*b);
}

// (Re)allocate the per-cell arrays of a type for `cap` cells, keeping the state.  Every
// new array is allocated before the type changes: if one allocation fails, the new
// ones are freed and the type keeps its old arrays and state.
void alloc_cells(npfem_ctx *ctx, MeshTypeImpl *cur, int cap) {
    MeshTypeImpl nt = *cur;
    void **cell_ptrs[] = {(void **)&nt.pub_off, (void **)&nt.xn, (void **)&nt.vn, &nt.yrel, &nt.delta, &nt.grad,
                          &nt.q, &nt.z, &nt.zp, &nt.kcol, &nt.ccol, &nt.S, &nt.Y, &nt.rlo, (void **)&nt.rlo_lo,
                          (void **)&nt.q16, (void **)&nt.y64, (void **)&nt.origin, (void **)&nt.rho, (void **)&nt.alpha,
                          (void **)&nt.M, (void **)&nt.g, (void **)&nt.allow, (void **)&nt.hcount,
                          (void **)&nt.hhead, (void **)&nt.conv, (void **)&nt.fb_list, (void **)&nt.fb_count};
    for (void **b : cell_ptrs) *b = nullptr;
    try {
        fill_cells(ctx, &nt, cur, cap);
    } catch (...) {
        cudaStreamSynchronize(ctx->stream);
        free_cells(&nt);
        throw;
    }
    MeshTypeImpl old = *cur;
    *cur = nt;
    free_cells(&old);
}

// The arrays of alloc_cells for type t (per-cell pointers null on entry), the state
// of the cells of `old` copied over.
void fill_cells(npfem_ctx *ctx, MeshTypeImpl *t, const MeshTypeImpl *old_t, int cap) {
    const MeshTypeImpl &old = *old_t;
    const size_t n3 = 3 * (size_t)t->nVp, es = esize(ctx), m = std::max(1, ctx->opt.history);
    t->pub_off = dalloc<long long>(ctx, cap);
    t->xn = dalloc<double>(ctx, cap * n3);
    t->vn = dalloc<double>(ctx, cap * n3);
    auto vec = [&](void *&p) { p = dalloc<unsigned char>(ctx, cap * n3 * es); };
    vec(t->yrel); vec(t->delta); vec(t->grad); vec(t->q); vec(t->z);
    if (t->damped) vec(t->zp);
    if (ctx->opt.pik_radius > 0) {
        vec(t->ccol);
        t->kcol = dalloc<unsigned char>(ctx, cap * (size_t)t->nVp * es);
        CK(cudaMemsetAsync(t->kcol, 0, cap * (size_t)t->nVp * es, ctx->stream));
        CK(cudaMemsetAsync(t->ccol, 0, cap * n3 * es, ctx->stream));
    }
    t->S = dalloc<unsigned char>(ctx, cap * n3 * es * m);
    t->Y = dalloc<unsigned char>(ctx, cap * n3 * es * m);
    t->q16 = bf16(ctx) ? dalloc<__nv_bfloat16>(ctx, cap * n3) : nullptr;
    t->rlo = mixed(ctx) ? dalloc<unsigned char>(ctx, cap * n3 * (bf16(ctx) ? 2 : 4)) : nullptr;
    t->rlo_lo = (split(ctx) || (bf16(ctx) && t->damped)) ? dalloc<__nv_bfloat16>(ctx, cap * n3) : nullptr;
    t->y64 = dalloc<double>(ctx, cap * n3);
    t->origin = dalloc<double>(ctx, 3 * (size_t)cap);
    t->rho = dalloc<double>(ctx, m * cap);
    t->alpha = dalloc<double>(ctx, m * cap);
    t->M = dalloc<double>(ctx, m * m * cap);
    t->g = dalloc<double>(ctx, cap);
    t->allow = dalloc<double>(ctx, cap);
    t->hcount = dalloc<int>(ctx, cap);
    t->hhead = dalloc<int>(ctx, cap);
    t->conv = dalloc<int>(ctx, cap);
    t->fb_list = dalloc<int>(ctx, cap);
    t->fb_count = dalloc<int>(ctx, 1);
    t->cap = cap;
    if (old.ncells) {
        CK(cudaMemcpyAsync(t->xn, old.xn, old.ncells * n3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(t->vn, old.vn, old.ncells * n3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (mixed(ctx)) {
        t->mapQ = make_map(ctx, bf16(ctx) ? (const void *)t->q16 : t->q, bf16(ctx), t->nV, 3ll * cap, t->nVp, tc::BM);
        t->mapR = make_map(ctx, t->rlo, bf16(ctx), t->nV, 3ll * cap, t->nVp, tc::BM);
        if (t->rlo_lo) t->mapRlo = make_map(ctx, t->rlo_lo, true, t->nV, 3ll * cap, t->nVp, tc::BM);
        t->mapZ = make_map(ctx, t->z, false, t->nV, 3ll * cap, t->nVp, 32);
        if (t->zp) t->mapZp = make_map(ctx, t->zp, false, t->nV, 3ll * cap, t->nVp, 32);
    }
}

void invalidate_graph(npfem_ctx *ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->graph_valid = false;
}

int pending_error(npfem_ctx *ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) fail(ctx, NPFEM_ECUDA, "device error: %s", cudaGetErrorString(e));
    CK(cudaMemcpy(ctx->h_st, ctx->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    unsigned long long err = ctx->h_st->err;
    if (err) {
        int code = (int)(err >> 32);
        long long where = (long long)(err & 0xffffffffull);
        CK(cudaMemsetAsync(&ctx->d_st->err, 0, sizeof(unsigned long long), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (code == DEV_ENONFINITE) fail(ctx, NPFEM_ENONFINITE, "non-finite value in cell %lld (type-local index)", where);
        fail(ctx, NPFEM_ETIMEOUT, "a bounded device wait expired (site %lld)", where);
    }
    return NPFEM_OK;
}

}  // namespace

// ================================================================= C ABI
extern "C" {

void npfem_default_options(npfem_options *o) {
    std::memset(o, 0, sizeof *o);
    o->precision = NPFEM_FP64;
    o->iters = 10;
    o->history = 5;
    o->armijo_c1 = 1e-4;
    o->max_backtracks = 8;
    o->refine_tol = 1e-6;
    o->refine_max = 3;
    o->use_graph = 1;
    o->device = 0;
    o->cuda_stream = nullptr;
    o->autotune_cache = nullptr;
    o->residual_fp64 = 0;
    o->refine_split = 1;
    o->curvature_tol = 1e-12;
}

int npfem_create(const npfem_options *opt, npfem_ctx **out) {
    if (!out) return NPFEM_EINVAL;
    *out = nullptr;
    npfem_ctx *ctx = new (std::nothrow) npfem_ctx;
    if (!ctx) return NPFEM_ENOMEM;
    if (opt) ctx->opt = *opt;
    else npfem_default_options(&ctx->opt);
    int rc = guard(ctx, [&] {
        const npfem_options &o = ctx->opt;
        if (o.precision < 0 || o.precision > 2 || o.iters < 1 || o.history < 0 || o.history > NPFEM_MAX_HISTORY ||
            o.max_backtracks < 0 || !(o.armijo_c1 > 0 && o.armijo_c1 < 1) || o.refine_max < 0 || !(o.refine_tol > 0) ||
            o.force_median < 0 || o.force_median > 1 || !(o.u_max >= 0) || !std::isfinite(o.u_max) ||
            !(o.pbd_kappa >= 0 && o.pbd_kappa <= 1) || !(o.pik_radius >= 0) || !std::isfinite(o.pik_radius) ||
            (o.pik_radius > 0 && !(o.collision_k > 0 && std::isfinite(o.collision_k))) ||
            std::isnan(o.curvature_tol))
            fail(ctx, NPFEM_EINVAL, "invalid option value");
        CK(cudaSetDevice(o.device));
        ctx->device = o.device;
        CK(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, o.device));
        if (mixed(ctx)) {
            int major = 0, minor = 0;
            CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, o.device));
            CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, o.device));
            if (major != 10 || minor != 3)
                fail(ctx, NPFEM_EINVAL, "mixed-precision forms need tcgen05 on sm_103 (device is sm_%d%d)", major, minor);
        }
        if (o.cuda_stream) {
            ctx->stream = (cudaStream_t)o.cuda_stream;
        } else {
            CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
            ctx->own_stream = true;
        }
        ctx->d_st = dalloc<DevStatus>(ctx, 1);
        ctx->d_fslot = dalloc<double *>(ctx, 1);
        ctx->d_any = dalloc<int>(ctx, NPFEM_SWEEP_FLAGS);
        CK(cudaMallocHost(&ctx->h_st, sizeof(DevStatus)));
        set_kernel_attrs(ctx);
        CK(cudaStreamSynchronize(ctx->stream));
    });
    if (rc) {
        g_create_error = ctx->err;
        npfem_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return NPFEM_OK;
}

void npfem_destroy(npfem_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    invalidate_graph(ctx);
    for (auto *t : ctx->types) {
        free_cells(t);
        for (void *p : t->owned) cudaFree(p);
        delete t;
    }
    void *bufs[] = {ctx->d_f, ctx->d_fslot, ctx->d_stage, ctx->d_st, ctx->d_any, ctx->d_ffilt,
                    ctx->d_pik_cnt, ctx->d_pik_start, ctx->d_pik_fill, ctx->d_pik_key, ctx->d_pik_bsum,
                    ctx->d_pik_ent, ctx->d_pik_pos, ctx->d_pik_hit, ctx->d_ibm_pts, ctx->d_ibm_area};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    if (ctx->copy) {
        cudaStreamSynchronize(ctx->copy);
        cudaStreamDestroy(ctx->copy);
    }
    for (cudaEvent_t e : ctx->ev_chunk)
        if (e) cudaEventDestroy(e);
    if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *npfem_last_error(const npfem_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

size_t npfem_num_dofs(const npfem_ctx *ctx) { return ctx ? (size_t)ctx->ndofs : 0; }

int npfem_create_mesh_type(npfem_ctx *ctx, int nV, const double *rest_xyz, int nT, const int32_t *tris,
                           const double *vertex_mass, const npfem_material *mat, int *type_id) {
    if (!ctx) return NPFEM_EINVAL;
    auto *t = new (std::nothrow) MeshTypeImpl;
    if (!t) return NPFEM_ENOMEM;
    int rc = guard(ctx, [&] {
        if (!rest_xyz || !tris || !mat || nV < 4 || nT < 4) fail(ctx, NPFEM_EINVAL, "bad mesh arguments");
        if (nV > 2720) fail(ctx, NPFEM_EINVAL, "nV = %d exceeds the supported 2720 vertices per cell", nV);
        if (!(mat->dt > 0) || mat->k_strain < 0 || mat->k_area < 0 || mat->k_bend < 0 || mat->k_vol < 0)
            fail(ctx, NPFEM_EINVAL, "bad material");
        if (!(mat->rayleigh_alpha >= 0) || !(mat->rayleigh_beta >= 0) || !std::isfinite(mat->rayleigh_alpha) ||
            !std::isfinite(mat->rayleigh_beta))
            fail(ctx, NPFEM_EINVAL, "Rayleigh damping coefficients must be finite and >= 0");
        std::vector<double> mass(nV);
        for (int v = 0; v < nV; ++v) {
            mass[v] = vertex_mass ? vertex_mass[v] : 1.0 / nV;
            if (!(mass[v] > 0)) fail(ctx, NPFEM_EINVAL, "vertex mass must be positive");
        }
        for (int i = 0; i < 3 * nV; ++i)
            if (!std::isfinite(rest_xyz[i])) fail(ctx, NPFEM_ENONFINITE, "non-finite rest position");
        for (int i = 0; i < 3 * nT; ++i)
            if (tris[i] < 0 || tris[i] >= nV) fail(ctx, NPFEM_EINVAL, "triangle index %d out of range", tris[i]);
        // internal numbering: RCM vertex order; each triangle rotated (orientation kept)
        // to start at its smallest internal index, triangles sorted by their indices
        const std::vector<int> vpub = rcm_order(nV, nT, tris);
        std::vector<int> intl(nV);
        for (int i = 0; i < nV; ++i) intl[vpub[i]] = i;
        std::vector<double> rest_i(3 * (size_t)nV), mass_i(nV);
        for (int i = 0; i < nV; ++i) {
            for (int c = 0; c < 3; ++c) rest_i[3 * i + c] = rest_xyz[3 * vpub[i] + c];
            mass_i[i] = mass[vpub[i]];
        }
        std::vector<std::array<int, 3>> tr(nT);
        for (int k = 0; k < nT; ++k) {
            std::array<int, 3> a = {intl[tris[3 * k]], intl[tris[3 * k + 1]], intl[tris[3 * k + 2]]};
            for (int r = 0; r < 2 && (a[0] > a[1] || a[0] > a[2]); ++r) a = {a[1], a[2], a[0]};
            tr[k] = a;
        }
        std::vector<int> tpub(nT);
        for (int k = 0; k < nT; ++k) tpub[k] = k;
        std::stable_sort(tpub.begin(), tpub.end(), [&](int x, int y) { return tr[x] < tr[y]; });
        std::vector<int32_t> tris_i(3 * (size_t)nT);
        for (int k = 0; k < nT; ++k)
            for (int j = 0; j < 3; ++j) tris_i[3 * k + j] = tr[tpub[k]][j];
        mass.swap(mass_i);
        HostType H;
        build_host_type(ctx, nV, rest_i.data(), nT, tris_i.data(), mass.data(), *mat, vpub.data(), tpub.data(), H);
        t->vpub = upload(ctx, vpub, t->owned);
        t->vint = upload(ctx, intl, t->owned);
        {
            // edge neighbours in the internal numbering (the median filter's one-rings)
            std::vector<std::vector<int>> nb(nV);
            for (int k = 0; k < nT; ++k)
                for (int j = 0; j < 3; ++j) {
                    const int a = tris_i[3 * k + j], b = tris_i[3 * k + (j + 1) % 3];
                    nb[a].push_back(b);
                    nb[b].push_back(a);
                }
            std::vector<int> ap(nV + 1, 0), aj;
            for (int v = 0; v < nV; ++v) {
                std::sort(nb[v].begin(), nb[v].end());
                nb[v].erase(std::unique(nb[v].begin(), nb[v].end()), nb[v].end());
                if (ctx->opt.force_median && (int)nb[v].size() + 1 > MEDIAN_MAX)
                    fail(ctx, NPFEM_EINVAL, "vertex %d has %d neighbours; the median filter takes at most %d",
                         vpub[v], (int)nb[v].size(), MEDIAN_MAX - 1);
                aj.insert(aj.end(), nb[v].begin(), nb[v].end());
                ap[v + 1] = (int)aj.size();
            }
            t->adj_ptr = upload(ctx, ap, t->owned);
            t->adj = upload(ctx, aj, t->owned);
        }
        t->nV = nV;
        t->nVp = (nV + 7) / 8 * 8;
        t->nT = nT;
        t->nH = (int)H.hrest.size();
        t->h = mat->dt;
        t->ks = mat->k_strain;
        t->ka = mat->k_area;
        t->kb = mat->k_bend;
        t->kv = mat->k_vol;
        t->ra = mat->rayleigh_alpha;
        t->rb = mat->rayleigh_beta;
        t->damped = !H.Mt.empty();
        t->V0 = H.V0;
        if (mixed(ctx)) t->tc32 = upload_consts<float>(ctx, t, H, mass);
        else t->tc64 = upload_consts<double>(ctx, t, H, mass);
        {
            // the origin's two vertices: the one farthest from vertex 0 at rest, and the one
            // farthest from it
            auto far_from = [&](int a) {
                int best = 0;
                double bd = -1.0;
                for (int v = 0; v < nV; ++v) {
                    double d = 0.0;
                    for (int c = 0; c < 3; ++c) d += (rest_i[3 * v + c] - rest_i[3 * a + c]) * (rest_i[3 * v + c] - rest_i[3 * a + c]);
                    if (d > bd) { bd = d; best = v; }
                }
                return best;
            };
            const int va = far_from(0), vb = far_from(va);
            t->tc32.ova = t->tc64.ova = va;
            t->tc32.ovb = t->tc64.ovb = vb;
        }
        std::vector<double> minv(nV), diag(nV);
        std::vector<int> op(nV + 1, 0);
        std::vector<int2> oe;
        for (int v = 0; v < nV; ++v) {
            minv[v] = 1.0 / mass[v];
            diag[v] = H.P[(size_t)v * nV + v];
            for (int u = 0; u < nV; ++u) {
                double p = H.P[(size_t)v * nV + u];
                if (u != v && p != 0.0) {
                    const float pf = (float)p;
                    int bits;
                    std::memcpy(&bits, &pf, 4);
                    oe.push_back(make_int2(u, bits));
                }
            }
            op[v + 1] = (int)oe.size();
        }
        t->minv = upload(ctx, minv, t->owned);
        t->mass = upload(ctx, mass, t->owned);
        for (double mv : mass) t->mtot += mv;
        t->diag = upload(ctx, diag, t->owned);
        std::vector<float> dhi(t->nVp, 0.f), dlo(t->nVp, 0.f);
        for (int v = 0; v < nV; ++v) {
            dhi[v] = (float)diag[v];
            dlo[v] = (float)(diag[v] - (double)dhi[v]);
        }
        t->dhi = upload(ctx, dhi, t->owned);
        t->dlo = upload(ctx, dlo, t->owned);
        t->op = upload(ctx, op, t->owned);
        t->oe = upload(ctx, oe, t->owned);
        if (mixed(ctx)) {
            int wmax = 0;
            for (int v = 0; v < nV; ++v) wmax = std::max(wmax, op[v + 1] - op[v]);
            const int KR = (t->nVp + RESID_MAX_THREADS - 1) / RESID_MAX_THREADS;
            if (wmax <= 16 && KR <= 4 && nV < 65536) {
                const int W = wmax <= 12 ? 12 : 16;
                const int nVp = t->nVp;
                std::vector<unsigned short> col((size_t)W * nVp, 0);
                std::vector<float> val((size_t)W * nVp, 0.f);
                for (int v = 0; v < nV; ++v)
                    for (int k = op[v]; k < op[v + 1]; ++k) {
                        const int w = k - op[v];
                        col[(size_t)w * nVp + v] = (unsigned short)oe[k].x;
                        std::memcpy(&val[(size_t)w * nVp + v], &oe[k].y, 4);
                    }
                t->ell_col = upload(ctx, col, t->owned);
                t->ell_val = upload(ctx, val, t->owned);
                t->ell_W = W;
                t->ell_KR = KR;
                t->ell_nt = ((nVp + KR - 1) / KR + 31) / 32 * 32;
                int nb = 0;
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, resid_ell_fn(W, KR), t->ell_nt,
                                                                 resid_ell_smem(nVp)));
                if (nb < 1) fail(ctx, NPFEM_ECUDA, "residual kernel does not fit on an SM");
                t->ell_grid = nb * ctx->nsm;
            }
        }
        {
            const InvCopies pi = invert_on_gpu(ctx, t, H.P, true, bf16(ctx) && split(ctx), "system matrix P");
            t->Pinv64 = pi.i64;
            t->Pinv32 = pi.i32;
            t->Pinv16 = pi.i16;
            t->Pinv16lo = pi.i16lo;
        }
        if (t->damped) {
            // the predictor's Mt^{-1}: FP64 in the FP64 form; split in the mixed forms
            const InvCopies mi = invert_on_gpu(ctx, t, H.Mt, !mixed(ctx), true, "damped mass matrix M + hC");
            t->Minv64 = mi.i64;
            t->Minv32 = mi.i32;
            t->Minv32lo = mi.i32lo;
            t->Minv16 = mi.i16;
            t->Minv16lo = mi.i16lo;
        }
        // per-cell kernel shape: EPT elements per thread, block <= 256 (<= 512 for big meshes)
        const int n3 = 3 * t->nVp;
        if ((n3 + 3) / 4 <= 256) t->ept = 4;
        else if ((n3 + 7) / 8 <= 256) t->ept = 8;
        else t->ept = 16;
        t->block = ((n3 + t->ept - 1) / t->ept + 31) / 32 * 32;
        const size_t es = esize(ctx);
        // stash: 9 values per triangle of a chunk; as large as the shared memory left
        // after the header and the three vectors allows (capped), and with the vectors
        // at least the L-BFGS batch scratch ((2 m_max + 4) values per thread)
        const size_t fixed = smem_header_bytes() + 3 * SMEM_VECS * (size_t)t->nVp * es;
        const size_t cap = mixed(ctx) ? 16384 : 6144;
        size_t room = (size_t)ctx->smem_optin > fixed + 1024 ? ((size_t)ctx->smem_optin - fixed - 1024) / es : 0;
        size_t st = std::min<size_t>({9 * (size_t)nT, cap, room});
        if (mixed(ctx) && t->block <= 256) {
            // FP32 path, blocks of <= 256 threads (64 registers): size the stash so that four
            // blocks share an SM -- triangles in equal chunks of what fits, the hinges in one
            // chunk where that fits too (the padded gathers take chunks; a fourth resident
            // block measured faster than one stash for the whole mesh)
            int per_sm = 0, resv = 0;
            CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
            CK(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device));
            const size_t budget = (size_t)per_sm / 4 > (size_t)resv + fixed ? ((size_t)per_sm / 4 - resv - fixed) / es : 0;
            if (budget >= 9 * 32) {
                const size_t chunks = (9 * (size_t)nT + budget - 1) / budget;
                const size_t ct = ((size_t)nT + chunks - 1) / chunks;
                st = std::min(st, std::max<size_t>(9 * ct, 3 * (size_t)t->nH <= budget ? 3 * (size_t)t->nH : 0));
            }
        }
        const size_t need = (size_t)(2 * NPFEM_MAX_HISTORY + 4) * t->block;
        if (st + 3 * SMEM_VECS * (size_t)t->nVp < need) st = need - 3 * SMEM_VECS * (size_t)t->nVp;
        if (st < 9) st = 9;
        t->stash_T = (int)st;
        t->smem_step = smem_header_bytes() + (3 * SMEM_VECS * (size_t)t->nVp + t->stash_T) * es;
        if (mixed(ctx)) {
            // vertex range of each triangle chunk (the padded gather visits only those)
            const int ct = std::max(1, t->stash_T / 9);
            for (int c = 0; c < 4; ++c) {
                int lo = nV, hi = -1;
                for (int k = c * ct; k < std::min(nT, (c + 1) * ct); ++k)
                    for (int j = 0; j < 3; ++j) {
                        lo = std::min(lo, tris_i[3 * k + j]);
                        hi = std::max(hi, tris_i[3 * k + j]);
                    }
                t->tc32.tri_vrange[c] = make_int2(lo, hi);
            }
        }
        if (mixed(ctx)) choose_tiles(ctx, t, 3 * 8192);
        if (t->smem_step > (size_t)ctx->smem_optin || gemm_smem(t) + 2048 > (size_t)ctx->smem_optin)
            fail(ctx, NPFEM_EINVAL, "mesh type needs more shared memory than the device offers");
        set_prefetch_distance(ctx, t);
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->types.push_back(t);
        invalidate_graph(ctx);
        if (type_id) *type_id = (int)ctx->types.size() - 1;
    });
    if (rc) {
        free_cells(t);
        for (void *p : t->owned) cudaFree(p);
        delete t;
    }
    return rc;
}

int npfem_add_cells(npfem_ctx *ctx, int type_id, int n_cells, const double *x0, const double *v0,
                    int64_t *first_cell) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (type_id < 0 || type_id >= (int)ctx->types.size() || n_cells < 0 || (n_cells > 0 && !x0))
            fail(ctx, NPFEM_EINVAL, "bad add_cells arguments");
        MeshTypeImpl *t = ctx->types[type_id];
        const long long per = 3ll * t->nV, total = per * n_cells;
        for (long long i = 0; i < total; ++i)
            if (!std::isfinite(x0[i]) || (v0 && !std::isfinite(v0[i])))
                fail(ctx, NPFEM_ENONFINITE, "non-finite initial state in new cell %lld", i / per);
        // index of the first new cell in the public order = cells added so far
        long long first = 0;
        for (auto *u : ctx->types) first += u->ncells;
        if (first_cell) *first_cell = first;
        if (n_cells == 0) return;
        if (t->ncells + n_cells > t->cap) alloc_cells(ctx, t, std::max(t->ncells + n_cells, 2 * t->cap));
        // everything the grown context needs is allocated before anything is committed: on a
        // failure (ENOMEM) the context keeps its cells, sizes and buffers (a grown capacity
        // holds the same state)
        const long long ndofs_new = ctx->ndofs + total;
        std::vector<void *> tmp;
        std::vector<long long> pub_new = t->pub_off_h;
        for (int c = 0; c < n_cells; ++c) pub_new.push_back(ctx->ndofs + per * c);
        double *f_new = nullptr, *stage_new = nullptr, *ffilt_new = nullptr;
        try {
            f_new = dalloc<double>(ctx, ndofs_new, &tmp);
            stage_new = dalloc<double>(ctx, ndofs_new, &tmp);
            if (ctx->opt.force_median) ffilt_new = dalloc<double>(ctx, ndofs_new, &tmp);
        } catch (...) {
            cudaStreamSynchronize(ctx->stream);
            for (void *p : tmp) cudaFree(p);
            throw;
        }
        const std::vector<void *> keep = tmp;     // the new public-layout buffers
        tmp.clear();
        auto drop_new = [&] {
            cudaStreamSynchronize(ctx->stream);
            for (void *p : keep) cudaFree(p);
            for (void *p : tmp) cudaFree(p);
        };
        // stage x0 / v0 in the public layout and scatter into SoA (beyond the current cells)
        double *sx = nullptr, *sv = nullptr;
        long long *offs = nullptr;
        try {
            sx = dalloc<double>(ctx, total, &tmp);
            sv = dalloc<double>(ctx, total, &tmp);
            offs = dalloc<long long>(ctx, n_cells, &tmp);
            CK(cudaMemcpyAsync(t->pub_off, pub_new.data(), pub_new.size() * sizeof(long long),
                               cudaMemcpyHostToDevice, ctx->stream));
            std::vector<long long> lo(n_cells);
            for (int c = 0; c < n_cells; ++c) lo[c] = per * c;
            CK(cudaMemcpyAsync(offs, lo.data(), n_cells * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(sx, x0, total * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            if (v0) CK(cudaMemcpyAsync(sv, v0, total * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            const long long n3 = 3ll * t->nVp;
            k_pub_to_soa<<<grid_for(n_cells * n3, 256, 8192), 256, 0, ctx->stream>>>(n_cells, t->nV, t->nVp, offs, sx,
                                                                                   t->xn + t->ncells * n3, t->vpub);
            k_pub_to_soa<<<grid_for(n_cells * n3, 256, 8192), 256, 0, ctx->stream>>>(
                n_cells, t->nV, t->nVp, offs, v0 ? sv : nullptr, t->vn + t->ncells * n3, t->vpub);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(ctx->stream));
        } catch (...) {
            drop_new();
            throw;
        }
        for (void *p : tmp) cudaFree(p);
        // commit: the cells, the public layout and its buffers
        t->pub_off_h.swap(pub_new);
        t->ncells += n_cells;
        ctx->ndofs = ndofs_new;
        dfree((void *&)ctx->d_f);
        dfree((void *&)ctx->d_stage);
        dfree((void *&)ctx->d_ffilt);
        ctx->d_f = f_new;
        ctx->d_stage = stage_new;
        ctx->d_ffilt = ffilt_new;
        invalidate_graph(ctx);
        if (ctx->opt.pik_radius > 0) pik_alloc(ctx);   // on failure the search refuses to run (ESTATE)
    });
}

namespace {
// first value of piece i of the n-value public force array
long long force_chunk_lo(long long n, int i) { return n * i / F_CHUNKS; }

// the piece that holds the last force value of cell c of type t
int force_chunk_of_cell(const npfem_ctx *ctx, const MeshTypeImpl *t, int c) {
    const long long last = t->pub_off_h[c] + 3ll * t->nV - 1;
    int k = 0;
    while (k + 1 < F_CHUNKS && force_chunk_lo(ctx->ndofs, k + 1) <= last) ++k;
    return k;
}
}  // namespace

int npfem_step(npfem_ctx *ctx, const double *f_ext, int f_ext_on_device) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (ctx->ndofs == 0) fail(ctx, NPFEM_ESTATE, "no cells");
        if (!f_ext) fail(ctx, NPFEM_EINVAL, "f_ext is null");
        // With nothing ahead of the predictor that reads the forces (no force filter,
        // collision search or damped predictor), the predictor runs outside the graph, per
        // type in pieces that follow the public force array's F_CHUNKS pieces: host forces
        // are copied piece by piece on a second stream while the predictor works on the
        // pieces already in.
        const bool early = !ctx->opt.force_median && !(ctx->opt.pik_radius > 0) &&
                           std::none_of(ctx->types.begin(), ctx->types.end(), [](const MeshTypeImpl *t) { return t->damped; });
        const double *fd = f_ext;
        if (!f_ext_on_device) {
            if (early) {
                if (!ctx->copy) {
                    CK(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
                    for (cudaEvent_t &e : ctx->ev_chunk) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                    CK(cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming));
                }
                CK(cudaStreamWaitEvent(ctx->copy, ctx->ev_done, 0));      // the last step read d_f
                for (int i = 0; i < F_CHUNKS; ++i) {
                    const long long lo = force_chunk_lo(ctx->ndofs, i), hi = force_chunk_lo(ctx->ndofs, i + 1);
                    CK(cudaMemcpyAsync(ctx->d_f + lo, f_ext + lo, (hi - lo) * sizeof(double), cudaMemcpyHostToDevice,
                                       ctx->copy));
                    CK(cudaEventRecord(ctx->ev_chunk[i], ctx->copy));
                }
            } else {
                CK(cudaMemcpyAsync(ctx->d_f, f_ext, ctx->ndofs * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            }
            fd = ctx->d_f;
        }
        // tile choices for the real right-hand-side counts (outside any capture; a changed
        // choice rebuilds the graph)
        if (mixed(ctx))
            for (auto *t : ctx->types)
                if (t->ncells && tune_bucket(3ll * t->ncells) != t->tuned_rows) {
                    choose_tiles(ctx, t, 3ll * t->ncells);
                    invalidate_graph(ctx);
                }
        k_set_ptr<<<1, 1, 0, ctx->stream>>>(ctx->d_fslot, fd);
        CK(cudaGetLastError());
        ctx->prof_next = 0;
        ctx->launch_counter = 0;
        if (early) {
            for (auto *t : ctx->types) {
                if (!t->ncells) continue;
                for (int c0 = 0; c0 < t->ncells;) {
                    // the cells whose forces end in piece k: a run (the pieces grow with the cell)
                    const int k = force_chunk_of_cell(ctx, t, c0);
                    int c1 = c0 + 1, hi = t->ncells;
                    while (c1 < hi) {
                        const int mid = c1 + (hi - c1) / 2;
                        if (force_chunk_of_cell(ctx, t, mid) > k) hi = mid;
                        else c1 = mid + 1;
                    }
                    if (!f_ext_on_device) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_chunk[k], 0));
                    run_predict(ctx, t, c0, c1);
                    c0 = c1;
                }
            }
        }
        if (ctx->opt.use_graph) {
            if (!ctx->graph_valid || ctx->graph_early != early) {
                invalidate_graph(ctx);
                ctx->graph_early = early;
                CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
                try {
                    enqueue_step(ctx, !early);
                    ctx->launches_per_step = ctx->launch_counter + 1;   // + the force-pointer kernel
                } catch (...) {
                    cudaGraph_t g = nullptr;
                    cudaStreamEndCapture(ctx->stream, &g);
                    if (g) cudaGraphDestroy(g);
                    throw;
                }
                CK(cudaStreamEndCapture(ctx->stream, &ctx->graph));
                CK(cudaGraphInstantiate(&ctx->gexec, ctx->graph, 0));
                ctx->graph_valid = true;
                ctx->graph_prof_pairs = ctx->prof_next / 2;
            }
            CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
        } else {
            enqueue_step(ctx, !early);
            ctx->launches_per_step = ctx->launch_counter + 1;
        }
        if (early && !f_ext_on_device) CK(cudaEventRecord(ctx->ev_done, ctx->stream));
        if (ctx->prof_on) prof_harvest(ctx, ctx->opt.use_graph ? ctx->graph_prof_pairs : ctx->prof_next / 2);
        ctx->stepped = true;
    });
}

int npfem_sync(npfem_ctx *ctx) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] { pending_error(ctx); });
}

static int get_state(npfem_ctx *ctx, bool pos, double *out, size_t n, int on_device) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (!out || (long long)n != ctx->ndofs) fail(ctx, NPFEM_EINVAL, "output size %zu != %lld", n, ctx->ndofs);
        double *dst = on_device ? out : ctx->d_stage;
        for (auto *t : ctx->types) {
            if (!t->ncells) continue;
            long long tot = 3ll * t->nV * t->ncells;
            k_soa_to_pub<<<grid_for(tot, 256, 8192), 256, 0, ctx->stream>>>(t->ncells, t->nV, t->nVp, t->pub_off,
                                                                            pos ? t->xn : t->vn, dst, t->vint);
        }
        CK(cudaGetLastError());
        if (!on_device) CK(cudaMemcpyAsync(out, ctx->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        pending_error(ctx);
    });
}

int npfem_get_positions(npfem_ctx *ctx, double *out, size_t n, int on_device) {
    return get_state(ctx, true, out, n, on_device);
}

int npfem_get_velocities(npfem_ctx *ctx, double *out, size_t n, int on_device) {
    return get_state(ctx, false, out, n, on_device);
}

int npfem_set_state(npfem_ctx *ctx, const double *x, const double *v, size_t n) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (!x || (long long)n != ctx->ndofs) fail(ctx, NPFEM_EINVAL, "state size %zu != %lld", n, ctx->ndofs);
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(x[i]) || (v && !std::isfinite(v[i])))
                fail(ctx, NPFEM_ENONFINITE, "non-finite state value at %zu", i);
        for (int pass = 0; pass < 2; ++pass) {
            const double *src = pass == 0 ? x : v;
            if (src) CK(cudaMemcpyAsync(ctx->d_stage, src, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            for (auto *t : ctx->types) {
                if (!t->ncells) continue;
                long long tot = 3ll * t->nVp * t->ncells;
                k_pub_to_soa<<<grid_for(tot, 256, 8192), 256, 0, ctx->stream>>>(
                    t->ncells, t->nV, t->nVp, t->pub_off, src ? ctx->d_stage : nullptr, pass == 0 ? t->xn : t->vn, t->vpub);
            }
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(ctx->stream));
        }
    });
}

int npfem_stats(npfem_ctx *ctx, npfem_step_stats *out) {
    if (!ctx || !out) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        pending_error(ctx);
        const DevStatus &s = *ctx->h_st;
        long long cells = 0;
        for (auto *t : ctx->types) cells += t->ncells;
        out->cell_iterations = ctx->stepped ? cells * ctx->opt.iters : 0;
        out->backtracks = s.backtracks;
        out->capped_searches = s.capped;
        out->fallbacks = s.fallbacks;
        out->refine_sweeps = s.refine_sweeps;
        float r;
        std::memcpy(&r, &s.max_resid_bits, sizeof r);
        out->max_refine_residual = r;
        out->energy_sum = s.energy_sum;
        out->launches_per_step = ctx->launches_per_step;
        out->contacts = (int64_t)s.contacts;
    });
}

int npfem_profile(npfem_ctx *ctx, int enable) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        CK(cudaStreamSynchronize(ctx->stream));
        if ((bool)enable != ctx->prof_on) invalidate_graph(ctx);
        ctx->prof_on = enable != 0;
    });
}

int npfem_profile_read(npfem_ctx *ctx, npfem_kernel_times *out, int reset) {
    if (!ctx || !out) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        for (int i = 0; i < NPFEM_KCLASSES; ++i) {
            out->ms[i] = ctx->prof_ms[i];
            out->launches[i] = ctx->prof_n[i];
            if (reset) {
                ctx->prof_ms[i] = 0;
                ctx->prof_n[i] = 0;
            }
        }
    });
}

int npfem_ibm_forces(npfem_ctx *ctx, const npfem_lattice *lat, const double *u_fluid, double dt, int cycles,
                     double *f_lagr, double *f_grid) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (!lat || !u_fluid || !f_lagr || !f_grid) fail(ctx, NPFEM_EINVAL, "null argument");
        if (lat->nx < 1 || lat->ny < 1 || lat->nz < 1 || !(lat->dx > 0) || !std::isfinite(lat->dx) ||
            !std::isfinite(lat->x0) || !std::isfinite(lat->y0) || !std::isfinite(lat->z0) || !(dt > 0) ||
            !std::isfinite(dt) || cycles < 0)
            fail(ctx, NPFEM_EINVAL, "bad lattice, dt or cycles");
        const long long nn = (long long)lat->nx * lat->ny * lat->nz;
        if (nn > (1ll << 40)) fail(ctx, NPFEM_EINVAL, "lattice too large");
        if (ctx->ndofs == 0) fail(ctx, NPFEM_ESTATE, "no cells");
        PikTypes pt{};
        std::vector<MeshTypeImpl *> tl;
        const long long N = point_types(ctx, pt, tl);
        if (N > ctx->ibm_cap) {
            dfree((void *&)ctx->d_ibm_pts);
            dfree((void *&)ctx->d_ibm_area);
            ctx->ibm_cap = 0;
            ctx->d_ibm_pts = dalloc<IbmPoint>(ctx, N);
            ctx->d_ibm_area = dalloc<double>(ctx, N);
            ctx->ibm_cap = N;
        }
        const IbmLattice L{lat->nx, lat->ny, lat->nz, lat->dx, lat->x0, lat->y0, lat->z0};
        auto grid = [&](int ti) { return grid_for((long long)pt.t[ti].ncells * pt.t[ti].nV, 256, 16 * ctx->nsm); };
        auto spread = [&] {
            CK(cudaMemsetAsync(f_grid, 0, 3 * nn * sizeof(double), ctx->stream));
            for (int ti = 0; ti < pt.ntypes; ++ti)
                k_ibm_spread_box<<<grid(ti), 256, IBM_BOX_DOUBLES * sizeof(double), ctx->stream>>>(
                    pt, ti, L, ctx->d_ibm_pts, f_lagr, f_grid);
        };
        for (int ti = 0; ti < pt.ntypes; ++ti)
            k_ibm_init<<<grid(ti), 256, 0, ctx->stream>>>(pt, ti, L, u_fluid, dt, ctx->d_ibm_pts, ctx->d_ibm_area,
                                                          f_lagr);
        for (int c = 0; c < cycles; ++c) {
            spread();
            k_ibm_correct<<<grid_for(3 * nn, 256, 16 * ctx->nsm), 256, 0, ctx->stream>>>(3 * nn, u_fluid, f_grid, dt);
            for (int ti = 0; ti < pt.ntypes; ++ti)
                k_ibm_update<<<grid(ti), 256, 0, ctx->stream>>>(pt, ti, L, f_grid, dt, ctx->d_ibm_pts,
                                                                ctx->d_ibm_area, f_lagr);
        }
        spread();
        CK(cudaGetLastError());
    });
}

int npfem_check_wait(npfem_ctx *ctx, int limit_ms) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (limit_ms < 1 || limit_ms > 2000) fail(ctx, NPFEM_EINVAL, "limit_ms must be in [1, 2000]");
        tc::k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_st, (unsigned long long)limit_ms * 1000000ull);
        CK(cudaGetLastError());
    });
}

int npfem_apply_pinv(npfem_ctx *ctx, int type_id, const double *q, double *z, int n_cols) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (type_id < 0 || type_id >= (int)ctx->types.size() || n_cols < 0 || !q || !z)
            fail(ctx, NPFEM_EINVAL, "bad apply arguments");
        if (n_cols == 0) return;
        MeshTypeImpl *t = ctx->types[type_id];
        const int ncell = (n_cols + 2) / 3, rows = 3 * ncell;
        const size_t nvec = (size_t)rows * t->nVp;
        std::vector<void *> tmp;
        try {
            if (!mixed(ctx)) {
                double *qi = dalloc<double>(ctx, nvec, &tmp), *zi = dalloc<double>(ctx, nvec, &tmp);
                k_cols_in<double><<<grid_for(nvec, 256, 8192), 256, 0, ctx->stream>>>(n_cols, t->nV, t->nVp, q, qi, nullptr, t->vpub);
                dim3 grid((t->nV + SG_T - 1) / SG_T, (rows + SG_T - 1) / SG_T);
                k_gemm_simt<double><<<grid, 256, 0, ctx->stream>>>(rows, t->nV, t->nVp, qi, t->Pinv64, zi);
                k_cols_out<double><<<grid_for((long long)n_cols * t->nV, 256, 8192), 256, 0, ctx->stream>>>(
                    n_cols, t->nV, t->nVp, zi, z, t->vint);
            } else {
                float *qi = dalloc<float>(ctx, nvec, &tmp), *zi = dalloc<float>(ctx, nvec, &tmp);
                __nv_bfloat16 *q16 = bf16(ctx) ? dalloc<__nv_bfloat16>(ctx, nvec, &tmp) : nullptr;
                void *rl = dalloc<unsigned char>(ctx, nvec * (bf16(ctx) ? 2 : 4), &tmp);
                __nv_bfloat16 *rlo = split(ctx) ? dalloc<__nv_bfloat16>(ctx, nvec, &tmp) : nullptr;
                int *conv = dalloc<int>(ctx, ncell, &tmp);
                k_cols_in<float><<<grid_for(nvec, 256, 8192), 256, 0, ctx->stream>>>(n_cols, t->nV, t->nVp, q, qi, q16, t->vpub);
                CUtensorMap mq = make_map(ctx, bf16(ctx) ? (const void *)q16 : qi, bf16(ctx), t->nV, rows, t->nVp, tc::BM);
                CUtensorMap mr = make_map(ctx, rl, bf16(ctx), t->nV, rows, t->nVp, tc::BM);
                CUtensorMap mrl{};
                if (rlo) mrl = make_map(ctx, rlo, true, t->nV, rows, t->nVp, tc::BM);
                const CUtensorMap mz = make_map(ctx, zi, false, t->nV, rows, t->nVp, 32);
                gemm_tc(ctx, t, mq, rows, mz, 0, nullptr);
                for (int s = 0; s < ctx->opt.refine_max; ++s) {
                    residual(ctx, t, ncell, qi, zi, rl, conv, s == 0, 0, rlo);
                    gemm_tc(ctx, t, mr, rows, mz, 1, conv, rlo ? &mrl : nullptr);
                }
                residual(ctx, t, ncell, qi, zi, nullptr, conv, ctx->opt.refine_max == 0, 1);
                k_cols_out<float><<<grid_for((long long)n_cols * t->nV, 256, 8192), 256, 0, ctx->stream>>>(
                    n_cols, t->nV, t->nVp, zi, z, t->vint);
            }
            CK(cudaGetLastError());
            pending_error(ctx);
        } catch (...) {
            cudaStreamSynchronize(ctx->stream);
            for (void *p : tmp) cudaFree(p);
            throw;
        }
        for (void *p : tmp) cudaFree(p);
    });
}

// ---------------------------------------------------------------------------
// Allocation-free apply.  Its scratch is this file-scope device array: every
// GPU that loads the library holds it until the process exits.  Host code
// must not pass the symbol itself to a kernel (in host code it names a
// host-side stand-in); the device address is resolved once per device with
// cudaGetSymbolAddress and cached below.
#define NPFEM_NOALLOC_SCRATCH_BYTES ((size_t)NPFEM_NOALLOC_MAX_ELEMS * 16 + ((size_t)1 << 20))
static __device__ __align__(256) unsigned char g_noalloc_scratch[NPFEM_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
std::map<int, void *> g_noalloc_addr;   // device ordinal -> address of g_noalloc_scratch on it

void *noalloc_scratch(npfem_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(ctx->device);
    if (it != g_noalloc_addr.end()) return it->second;
    int prev = 0;
    CK(cudaGetDevice(&prev));
    CK(cudaSetDevice(ctx->device));
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess || !p) fail(ctx, NPFEM_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_addr[ctx->device] = p;
    return p;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

extern "C" int npfem_apply_pinv_noalloc(npfem_ctx *ctx, int type_id, const double *q, double *z, int n_cols) {
    if (!ctx) return NPFEM_EINVAL;
    return guard(ctx, [&] {
        if (type_id < 0 || type_id >= (int)ctx->types.size() || n_cols < 0 || !q || !z)
            fail(ctx, NPFEM_EINVAL, "bad apply arguments");
        if (n_cols == 0) return;
        MeshTypeImpl *t = ctx->types[type_id];
        const int ncell = (n_cols + 2) / 3, rows = 3 * ncell;
        const size_t nvec = (size_t)rows * t->nVp;
        if (nvec > (size_t)NPFEM_NOALLOC_MAX_ELEMS)
            fail(ctx, NPFEM_EINVAL,
                 "npfem_apply_pinv_noalloc: %d columns of a %d-vertex type need %zu scratch elements "
                 "(3 * ceil(n_cols / 3) * nVp, nVp = %d); the static scratch holds %d",
                 n_cols, t->nV, nvec, t->nVp, (int)NPFEM_NOALLOC_MAX_ELEMS);
        unsigned char *base = (unsigned char *)noalloc_scratch(ctx);
        const size_t es = esize(ctx);
        // carve: q, z (solver type), then the BF16 copy of q, the refinement operand (and its
        // low part for split corrections), then flags: at most 16 bytes per element
        size_t off = 0;
        void *qi = base + off;  off += up256(nvec * es);
        void *zi = base + off;  off += up256(nvec * es);
        __nv_bfloat16 *q16 = nullptr, *rlo = nullptr;
        void *rl = nullptr;
        int *conv = nullptr;
        if (mixed(ctx)) {
            if (bf16(ctx)) { q16 = (__nv_bfloat16 *)(base + off); off += up256(nvec * 2); }
            rl = base + off;  off += up256(nvec * (bf16(ctx) ? 2 : 4));
            if (split(ctx)) { rlo = (__nv_bfloat16 *)(base + off); off += up256(nvec * 2); }
            conv = (int *)(base + off);  off += up256((size_t)ncell * sizeof(int));
        }
        if (off > NPFEM_NOALLOC_SCRATCH_BYTES) fail(ctx, NPFEM_EINVAL, "scratch layout overflow");
        // The array keeps the previous call's contents: the rows after the last
        // column of a ragged final cell must start at zero (they enter the GEMM).
        if (rows > n_cols) {
            CK(cudaMemsetAsync((unsigned char *)qi + (size_t)n_cols * t->nVp * es, 0,
                               (size_t)(rows - n_cols) * t->nVp * es, ctx->stream));
            if (q16)
                CK(cudaMemsetAsync(q16 + (size_t)n_cols * t->nVp, 0, (size_t)(rows - n_cols) * t->nVp * 2, ctx->stream));
        }
        if (!mixed(ctx)) {
            k_cols_in<double><<<grid_for(nvec, 256, 8192), 256, 0, ctx->stream>>>(n_cols, t->nV, t->nVp, q,
                                                                                (double *)qi, nullptr, t->vpub);
            dim3 grid((t->nV + SG_T - 1) / SG_T, (rows + SG_T - 1) / SG_T);
            k_gemm_simt<double><<<grid, 256, 0, ctx->stream>>>(rows, t->nV, t->nVp, (const double *)qi, t->Pinv64,
                                                               (double *)zi);
            k_cols_out<double><<<grid_for((long long)n_cols * t->nV, 256, 8192), 256, 0, ctx->stream>>>(
                n_cols, t->nV, t->nVp, (const double *)zi, z, t->vint);
        } else {
            k_cols_in<float><<<grid_for(nvec, 256, 8192), 256, 0, ctx->stream>>>(n_cols, t->nV, t->nVp, q,
                                                                               (float *)qi, q16, t->vpub);
            CUtensorMap mq = make_map(ctx, bf16(ctx) ? (const void *)q16 : qi, bf16(ctx), t->nV, rows, t->nVp, tc::BM);
            CUtensorMap mr = make_map(ctx, rl, bf16(ctx), t->nV, rows, t->nVp, tc::BM);
            CUtensorMap mrl{};
            if (rlo) mrl = make_map(ctx, rlo, true, t->nV, rows, t->nVp, tc::BM);
            const CUtensorMap mz = make_map(ctx, zi, false, t->nV, rows, t->nVp, 32);
            gemm_tc(ctx, t, mq, rows, mz, 0, nullptr);
            for (int s = 0; s < ctx->opt.refine_max; ++s) {
                residual(ctx, t, ncell, (const float *)qi, (const float *)zi, rl, conv, s == 0, 0, rlo);
                gemm_tc(ctx, t, mr, rows, mz, 1, conv, rlo ? &mrl : nullptr);
            }
            residual(ctx, t, ncell, (const float *)qi, (const float *)zi, nullptr, conv, ctx->opt.refine_max == 0, 1);
            k_cols_out<float><<<grid_for((long long)n_cols * t->nV, 256, 8192), 256, 0, ctx->stream>>>(
                n_cols, t->nV, t->nVp, (const float *)zi, z, t->vint);
        }
        CK(cudaGetLastError());
        pending_error(ctx);
    });
}

}  // extern "C"
