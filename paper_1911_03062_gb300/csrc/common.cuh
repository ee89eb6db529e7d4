// common.cuh -- shared device helpers of the npFEM CUDA path: per-cell sums
// (FP64, or float-float compensated sums combined in FP64 for the FP32 local
// step), block reductions, bounded waits and the device error word.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace npfem {

// ---------------------------------------------------------------- errors
// First device error wins: code in the high 32 bits, cell/index in the low.
struct DevStatus {
    unsigned long long err;      // 0 = none
    unsigned long long backtracks;
    unsigned long long capped;
    unsigned long long fallbacks;
    unsigned long long refine_sweeps;
    unsigned long long contacts;  // vertices with a foreign vertex in their kernel (PIK)
    unsigned int max_resid_bits; // float bits of the largest final refinement ratio
    unsigned int pad;
    double energy_sum;
};

enum : int { DEV_ENONFINITE = 1, DEV_ETIMEOUT = 2 };

__device__ inline void dev_raise(DevStatus *st, int code, long long where) {
    unsigned long long v = ((unsigned long long)(unsigned)code << 32) | (unsigned long long)(unsigned)where;
    atomicCAS(&st->err, 0ull, v);
}

// ------------------------------------------------ float-float accumulation
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return {s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    float lo = __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo);
    float hi = __fadd_rn(s.hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s.hi));
    return {hi, lo};
}

// Sum accumulators: FP64 for the FP64 path; float-float (about 44 bits) for
// the FP32 path, whose per-thread partials are combined across the block in
// FP64 (see block_reduce_t0).
template <typename T> struct Acc;

template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ void merge_shfl(unsigned mask, int off) { v += __shfl_down_sync(mask, v, off); }
    __device__ __forceinline__ void merge(const Acc &o) { v += o.v; }
    __device__ __forceinline__ void store(double *p) const { *p = v; }
    __device__ __forceinline__ void load(const double *p) { v = *p; }
    __device__ __forceinline__ double get() const { return v; }
    __device__ __forceinline__ double nearest() const { return v; }
};

template <> struct Acc<float> {
    DF v;
    __device__ __forceinline__ void zero() { v.hi = 0.f; v.lo = 0.f; }
    __device__ __forceinline__ void add(float x) { v = df_add(v, DF{x, 0.f}); }
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p = __fmul_rn(a, b);
        float e = __fmaf_rn(a, b, -p);          // exact product p + e
        v = df_add(v, DF{p, e});
    }
    __device__ __forceinline__ void merge_shfl(unsigned mask, int off) {
        DF o{__shfl_down_sync(mask, v.hi, off), __shfl_down_sync(mask, v.lo, off)};
        v = df_add(v, o);
    }
    __device__ __forceinline__ void merge(const Acc &o) { v = df_add(v, o.v); }
    __device__ __forceinline__ void store(double *p) const { *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo); }
    __device__ __forceinline__ void load(const double *p) {
        float2 f = *reinterpret_cast<const float2 *>(p);
        v.hi = f.x;
        v.lo = f.y;
    }
    __device__ __forceinline__ double get() const { return (double)v.hi + (double)v.lo; }
    // the sum rounded to FP32: the high part of the normalised pair (no FP64 arithmetic)
    __device__ __forceinline__ float nearest() const { return v.hi; }
};

// Block-wide sums of N accumulators: each warp reduces by shuffles, warp 0
// combines the per-warp partials by a second shuffle tree (fixed order, so
// the result is deterministic), and thread 0 calls fn(sums) with the totals
// in FP64; fn writes the scalars the block needs to shared memory, visible
// to every thread when this returns.  Only thread 0 does FP64 arithmetic.
// Scratch: red[32 * N] doubles.
template <typename T, int N, typename F>
__device__ __forceinline__ void block_reduce_t0(Acc<T> (&a)[N], double *red, F &&fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i].merge_shfl(0xffffffffu, off);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i].store(red + warp * N + i);
    __syncthreads();
    if (warp == 0) {
        Acc<T> t[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (lane < nw) t[i].load(red + lane * N + i);
            else t[i].zero();
        }
        for (int off = 16; off > 0; off >>= 1) {
            if (off >= nw * 2) continue;       // lanes >= nw hold zeros: skip empty levels
#pragma unroll
            for (int i = 0; i < N; ++i) t[i].merge_shfl(0xffffffffu, off);
        }
        if (lane == 0) {
            double s[N];
#pragma unroll
            for (int i = 0; i < N; ++i) s[i] = t[i].get();
            fn(s);
        }
    }
    __syncthreads();
}

// The two halves of block_reduce_t0 for callers that already have barriers:
// warp_partials_store (every thread) before a __syncthreads, block_combine_t0
// (every thread; warp 0 merges, thread 0 calls fn) after it; fn's results are
// visible after the caller's next __syncthreads.  Same order as block_reduce_t0.
template <typename T, int N>
__device__ __forceinline__ void warp_partials_store(Acc<T> (&a)[N], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i].merge_shfl(0xffffffffu, off);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i].store(red + warp * N + i);
}

template <typename T, int N, typename F>
__device__ __forceinline__ void block_combine_t0(const double *red, F &&fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (warp != 0) return;
    Acc<T> t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (lane < nw) t[i].load(red + lane * N + i);
        else t[i].zero();
    }
    for (int off = 16; off > 0; off >>= 1) {
        if (off >= nw * 2) continue;
#pragma unroll
        for (int i = 0; i < N; ++i) t[i].merge_shfl(0xffffffffu, off);
    }
    if (lane == 0) {
        double s[N];
#pragma unroll
        for (int i = 0; i < N; ++i) s[i] = t[i].get();
        fn(s);
    }
}

// ------------------------------------------------------------ type traits
template <typename T> struct Prec;
template <> struct Prec<double> {
    static constexpr double area_tol = 1e-15;
    static constexpr double degen_tol = 1e-12;
    static constexpr double vol_tol = 1e-14;
    static constexpr double round_unit = 1.1102230246251565e-16;
};
template <> struct Prec<float> {
    static constexpr float area_tol = 2e-7f;
    static constexpr float degen_tol = 1e-6f;
    static constexpr double vol_tol = 2e-6;
    static constexpr double round_unit = 5.9604644775390625e-08;
};

// x rounded to the nearest value with a TF32 (10-bit) significand, ties away from
// zero: the high part of a TF32 split (exactly what the tensor core reads of it).
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

}  // namespace npfem
