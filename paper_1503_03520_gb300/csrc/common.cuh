// Device helpers shared by the l1ls kernels: SplitMix64 streams, value conversions,
// deterministic block reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace l1ls {

// ---- SplitMix64 (Steele, Lea & Flood 2014) as counter-based streams ------------------------
// The i-th output (0-based) of SplitMix64 started at state s0 is mix64(s0 + (i+1) * gamma);
// stream `tag` of `seed` starts at output `tag` of the generator seeded with `seed`.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm_output(uint64_t s0, uint64_t i) {
    return mix64(s0 + (i + 1ull) * kGamma);
}
__host__ __device__ __forceinline__ uint64_t sm_stream(uint64_t seed, uint64_t tag) {
    return sm_output(seed, tag);
}
// uniform double in [0, 1) from the top 53 bits
__host__ __device__ __forceinline__ double u01(uint64_t u) {
    return (double)(u >> 11) * (1.0 / 9007199254740992.0);
}

// stream tags (one stream per random quantity of the generator)
enum : uint64_t {
    kTagSigma = 1, kTagPerm = 2, kTagSupport = 3, kTagXVal = 4, kTagXSign = 5, kTagGOff = 6,
    kTagNRow = 7, kTagNVal = 8, kTagXi = 9
};

// ---- conversions ------------------------------------------------------------------------
template <class T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class Acc, class T> __device__ __forceinline__ Acc to_acc(T v);
template <> __device__ __forceinline__ double to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_acc<float, double>(double v) { return (float)v; }

template <class T> __device__ __forceinline__ T from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

// ---- reductions ---------------------------------------------------------------------------
template <bool IS_MAX> __device__ __forceinline__ double red_op(double a, double b) {
    if constexpr (IS_MAX) return fmax(a, b);
    else return a + b;
}

template <bool IS_MAX> __device__ __forceinline__ double warp_reduce(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = red_op<IS_MAX>(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of NP values; `maxmask` bit i selects max instead of sum for value i.
// Fixed order: lanes by shuffle tree, warps in index order.  Result valid in thread 0.
template <int BLOCK, int NP>
__device__ __forceinline__ void block_reduce(double (&v)[NP], unsigned maxmask, double* smem /*[NP*32]*/) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        v[i] = ((maxmask >> i) & 1) ? warp_reduce<true>(v[i]) : warp_reduce<false>(v[i]);
        if (lane == 0) smem[i * 32 + wid] = v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double a = smem[i * 32];
            for (int w = 1; w < NW; ++w) a = ((maxmask >> i) & 1) ? fmax(a, smem[i * 32 + w]) : a + smem[i * 32 + w];
            v[i] = a;
        }
    }
    __syncthreads();
}

// Grid-wide deterministic reduction through per-block partials and a "last block" step.
// Every block calls it with its block totals (valid in thread 0).  The block that arrives
// last reduces all partials in a fixed order and returns true with the totals in `tot`
// (valid in thread 0).  `counter` must be zero on entry to the launch; it is reset here.
template <int BLOCK, int NP>
__device__ __forceinline__ bool grid_reduce_last(const double (&blk)[NP], unsigned maxmask, double* partials,
                                                 unsigned* counter, double (&tot)[NP], double* smem) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) partials[(size_t)blockIdx.x * NP + i] = blk[i];
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double v[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) v[i] = ((maxmask >> i) & 1) ? -INFINITY : 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += BLOCK) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double p = __ldcg(&partials[(size_t)b * NP + i]);
            v[i] = ((maxmask >> i) & 1) ? fmax(v[i], p) : v[i] + p;
        }
    }
    block_reduce<BLOCK, NP>(v, maxmask, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) tot[i] = v[i];
        *counter = 0u;
    }
    return true;
}

__device__ __forceinline__ double soft_threshold(double v, double t) {
    double a = fabs(v) - t;
    return a > 0.0 ? copysign(a, v) : 0.0;
}

}  // namespace l1ls

namespace l1ls {

// ---- float-float arithmetic ---------------------------------------------------------------
// A value is hi + lo with |lo| <= ulp(hi)/2: about 48 significand bits, carried entirely on
// the FP32 pipes (the FP64 pipe of this part runs at a small fraction of the FP32 rate).
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971) and
// TwoProduct by a fused multiply-add; additions and products follow the double-word
// algorithms of Dekker (1971) and Bailey's double-double library.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
// Running sum of float-float terms: acc.hi is the FP32 sum, acc.lo collects the rounding error
// of every addition (TwoSum) and the low words of the terms.  Algorithm Sum2 of Ogita, Rump &
// Oishi ("Accurate sum and dot product", 2005): the result acc.hi + acc.lo is as accurate as
// a sum in twice the working precision, for 8 FP32 operations per term instead of the 20 of
// ff_add.  acc.lo is not normalised against acc.hi; read the total with ff_to_double.
__device__ __forceinline__ void sum2_add(ff& acc, ff p) {
    const ff t = two_sum(acc.hi, p.hi);
    acc.hi = t.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t.lo, p.lo));
}
// Double-word addition without the TwoSum of the low words (Dekker's "sloppy" addition,
// 11 FP32 operations instead of 20): the absolute error stays within a few units of
// 2^-48 (|a| + |b|), but under cancellation it is not small relative to the result.  Used for
// the FISTA iterate update, whose accuracy is absolute (relative to |x|) in any case.
__device__ __forceinline__ ff ff_add_sloppy(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}
// Square root and quotient of double-word numbers (Dekker 1971, "A floating-point technique for
// extending the available precision": sqrt2 and div2): the FP32 root (quotient) plus one
// correction from the exact remainder, which TwoProduct gives; relative error a few units of
// 2^-46.  For v > 0 (v = 0 gives 0) and b != 0 within the FP32 range.
__device__ __forceinline__ ff ff_sqrt(ff v) {
    const float s = __fsqrt_rn(v.hi);
    if (s == 0.0f) return {0.0f, 0.0f};
    const ff s2 = two_prod(s, s);
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(v.hi, s2.hi), s2.lo), v.lo);   // v - s^2 (first difference exact)
    return fast_two_sum(s, __fmul_rn(e, __fmul_rn(0.5f, __frcp_rn(s))));
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float r = __frcp_rn(b.hi);
    const float c = __fmul_rn(a.hi, r);
    const ff u = two_prod(c, b.hi);
    const float cc = __fmul_rn(__fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, u.hi), u.lo), a.lo), __fmul_rn(c, b.lo)), r);
    return fast_two_sum(c, cc);
}
__device__ __forceinline__ ff ff_from_float(float a) { return {a, 0.0f}; }
__device__ __forceinline__ ff ff_from_double(double d) {   // FP64 pipe: use outside hot loops
    const float hi = __double2float_rn(d);
    return {hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_abs(ff a) { return a.hi < 0.0f ? ff_neg(a) : a; }
// FISTA's step in float-float for one coordinate (Sec. 8.1): y = x1 + beta (x1 - x0),
// x = S_thr(y + g invL) with the shrinkage S_t(v) = sign(v) max(|v| - t, 0) of Sec. 2; also |x|
// for the l1 norm.  Additions without the low-word TwoSum
// (absolute errors of a few units of 2^-48 |x|: the iterate's own accuracy).
struct FfStep {
    ff y, x, mag;
};
__device__ __forceinline__ FfStep ff_fista_step(ff x1, ff x0, ff g, ff beta, ff invL, ff thr) {
    FfStep o;
    o.y = ff_add_sloppy(x1, ff_mul(beta, ff_add_sloppy(x1, ff_neg(x0))));
    ff gl = two_prod(g.hi, invL.hi);
    gl.lo = __fmaf_rn(g.hi, invL.lo, __fmaf_rn(g.lo, invL.hi, gl.lo));
    const ff v = ff_add_sloppy(o.y, fast_two_sum(gl.hi, gl.lo));
    const ff a = ff_add_sloppy(ff_abs(v), ff_neg(thr));
    if (a.hi > 0.0f) {
        o.mag = a;
        o.x = v.hi < 0.0f ? ff_neg(a) : a;
    } else {
        o.mag = o.x = {0.0f, 0.0f};
    }
    return o;
}

// Bounded grid barrier: every block's thread 0 arrives on count; the last one (count reaching
// gridDim.x + extra, extra = 0 in every solve) bumps gen.  A block that polls gen max_polls
// times without a change (sleeping sleep_ns between polls) sets *err = 2 and returns false
// (its block leaves the kernel).
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned* gen, int* err, uint32_t max_polls, unsigned extra,
                                          unsigned sleep_ns = 64) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *(volatile unsigned*)gen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == gridDim.x - 1 + extra) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            uint32_t polls = 0;
            while (*(volatile unsigned*)gen == g) {
                if (++polls > max_polls) {
                    ok = 0;
                    atomicExch(err, 2);
                    break;
                }
                if (sleep_ns) __nanosleep(sleep_ns);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace l1ls
