// FISTA (Sec. 8.1; Beck & Teboulle) with fused epilogues and a duality-gap certificate.
//
// Iteration k (k = 1, 2, ...) runs two kernels, each streaming one copy of A once:
//   K1  u = A x_{k-1};  A y_k = u + beta_k (u - A x_{k-2});  r_k = b - A y_k
//       writes u over A x_{k-2} and r_k; partial sums (u - b)^2, b.r_k, r_k^2  [FP64]
//   K2  g = A^T r_k;  y_k = x_{k-1} + beta_k (x_{k-1} - x_{k-2});
//       x_k = S_{tau/L}(y_k + g / L) written over x_{k-2}; partials max|g|, sum|x_k|
//       the last CTA certifies x_{k-1}: P = tau ||x_{k-1}||_1 + 1/2 ||u - b||^2,
//       D_k = s b.r_k - s^2/2 ||r_k||^2 with s = min(1, tau / ||g||_inf), gap = P - max_j D_j,
//       and either stops (flag in device memory) or advances t, beta.
// Every kernel returns at once when the stop flag is set, so chunks of iterations are
// captured in one CUDA graph and launched without host round trips.  x_{k-1} and x_{k-2}
// alternate between two buffers; a chunk holds an even number of iterations.
// FP64 values: all vectors FP64.  FP32 / BF16 values: products, residuals and A x in FP32
// (FP32 accumulation); the iterates are float-float pairs (hi, lo) updated in float-float
// arithmetic, K1 gathers the hi part, and the gap partials are accumulated in float-float
// and reduced across the grid in FP64.  (The FP64 pipe of this part is a small fraction of
// the FP32 rate; FP64 per row in these epilogues bounded both kernels before.)
#include <chrono>
#include <cmath>
#include <memory>

#include "internal.h"
#include <cstring>
#include "spmv.cuh"
#include "mfree.cuh"

namespace l1ls {

namespace {

constexpr int kBlock = 256;
// resident blocks per SM the K1 / K2 register allocations are sized for (build parameters;
// 4 caps a thread at 64 registers, the most that keeps 32 warps per SM)
#ifndef L1LS_K1_MIN_BLOCKS
#define L1LS_K1_MIN_BLOCKS 4
#endif
#ifndef L1LS_K2_MIN_BLOCKS
#define L1LS_K2_MIN_BLOCKS 4
#endif
// K1 loads A x_{k-2} and b and stores A x_{k-1} with evict-first hints (a build parameter;
// measured at C2: K1 0.297 -> 0.292 ms)
#ifndef L1LS_K1_STREAM_HINTS
#define L1LS_K1_STREAM_HINTS 1
#endif
// K2 loads the iterates x_{k-1}, x_{k-2} with evict-first hints (a build parameter; measured
// at C2: K2 0.315 -> 0.290 ms, the gathered residual stays in L2)
#ifndef L1LS_K2_STREAM_HINTS
#define L1LS_K2_STREAM_HINTS 1
#endif
// the same for the float-float kernels K1C / K2C (K2C at 64 registers spills; 3 blocks allow 85)
#ifndef L1LS_K1C_MIN_BLOCKS
#define L1LS_K1C_MIN_BLOCKS 4
#endif
#ifndef L1LS_K2C_MIN_BLOCKS
#define L1LS_K2C_MIN_BLOCKS 3
#endif

struct FistaState {
    double tau, L, tol;
    int64_t max_iter;
    double t, beta, best_d, l1_cur;
    double k1[3];
    int64_t iter, cert_iter, products;
    double P, D, gap, rel;
    int32_t stop, status;
    unsigned cnt1, cnt2;
    int32_t restart, stage_err;   // stage_err: kStageTimeout if a stage wait ran out
    int64_t restarts;
    // beta, 1/L and tau/L as float-float, refreshed with beta by the scalar step: the FP32
    // kernels read them instead of every thread converting (two FP64 divisions each)
    float beta_ff[2], invL_ff[2], thr_ff[2];
    double f_target;   // stop once P(x_{k-1}) <= f_target (-inf: off)
};
static_assert(sizeof(FistaState) <= Ctx::kPinnedSlotBytes, "the state read-back fits a pinned slot");

// host and device: the float-float scalars of the state
__host__ __device__ inline void split_ff(double d, float (&out)[2]) {
    out[0] = (float)d;
    out[1] = (float)(d - (double)out[0]);
}

template <class V, class Vec>
struct K1Args {
    const int32_t* ptr;
    const int32_t* col;
    const V* val;
    const Vec* x;        // x_{k-1} (gather source)
    Vec* ax;             // in: A x_{k-2}; out: A x_{k-1}
    Vec* res;            // out: r_k = b - A y_k
    const Vec* b;
    double* partials;
    FistaState* st;
    int64_t m;
};

template <class V, class Vec>
struct K2Args {
    const int32_t* ptr;
    const int32_t* col;
    const V* val;
    const Vec* res;
    const double* xc;    // x_{k-1} (FP64 values)
    double* xo;          // in: x_{k-2}; out: x_k (FP64 values)
    const float* xch;    // x_{k-1} as float-float (FP32 / BF16 values)
    const float* xcl;
    float* xoh;          // in: x_{k-2}; out: x_k as float-float
    float* xol;
    double* partials;
    FistaState* st;
    int64_t n;
};

// (FP64 vectors need more than 64 registers: 3 blocks per SM for them)
template <class V, class Vec, bool PAIRED>
__global__ void __launch_bounds__(kBlock, sizeof(Vec) == 8 ? 3 : L1LS_K1_MIN_BLOCKS) k_fista_k1(K1Args<V, Vec> a) {
    using Acc = Vec;
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    __shared__ double red[3 * 32];
    if (*(volatile int32_t*)&a.st->stop) return;
    const Vec beta = (Vec)a.st->beta;
    double p[3] = {0.0, 0.0, 0.0};
    ff q[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    struct Ops {
        Vec axo, bb;
    };
    rows_of<PAIRED, V, Vec, Acc>(
        a.ptr, a.col, a.val, a.x, a.m, sm, &a.st->stage_err,
        [&](int64_t r, bool has) {
            Ops o{Vec(0), Vec(0)};
            if (has) {
#if L1LS_K1_STREAM_HINTS
                // A x_{k-2} and b are not read again in this iteration: evict-first, so that the
                // gathered x (here) and the residual (K2) keep their place in L2
                o.axo = __ldcs(a.ax + r);
                o.bb = __ldcs(a.b + r);
#else
                o.axo = a.ax[r];
                o.bb = a.b[r];
#endif
            }
            return o;
        },
        [&](int64_t r, Acc u, const Ops& o) {
            const Vec ay = u + beta * (u - o.axo);
            const Vec rr = o.bb - ay;
#if L1LS_K1_STREAM_HINTS
            __stcs(a.ax + r, u);
#else
            a.ax[r] = u;
#endif
            a.res[r] = rr;
            if constexpr (sizeof(Vec) == 4) {
                const ff d = two_sum(u, -o.bb);                  // u - b exactly
                ff sq = two_prod(d.hi, d.hi);
                sq.lo = __fmaf_rn(2.0f * d.hi, d.lo, sq.lo);
                sum2_add(q[0], sq);
                sum2_add(q[1], two_prod(o.bb, rr));
                sum2_add(q[2], two_prod(rr, rr));
            } else {
                const double du = (double)u - (double)o.bb;
                p[0] += du * du;
                p[1] += (double)o.bb * (double)rr;
                p[2] += (double)rr * (double)rr;
            }
        });
    if constexpr (sizeof(Vec) == 4) {
        p[0] = ff_to_double(q[0]);
        p[1] = ff_to_double(q[1]);
        p[2] = ff_to_double(q[2]);
    }
    block_reduce<kBlock, 3>(p, 0u, red);
    double tot[3];
    if (grid_reduce_last<kBlock, 3>(p, 0u, a.partials, &a.st->cnt1, tot, red) && threadIdx.x == 0) {
        a.st->k1[0] = tot[0];
        a.st->k1[1] = tot[1];
        a.st->k1[2] = tot[2];
    }
}

__device__ void fista_finalize(FistaState* st, double amax, double l1_new, double restart_test) {
    const double tau = st->tau;
    const double P = __dadd_rn(__dmul_rn(tau, st->l1_cur), __dmul_rn(0.5, st->k1[0]));
    const double s = amax <= tau ? 1.0 : tau / amax;
    const double D = __dadd_rn(__dmul_rn(s, st->k1[1]), -__dmul_rn(__dmul_rn(__dmul_rn(0.5, s), s), st->k1[2]));
    st->best_d = fmax(st->best_d, D);
    const double gap = P - st->best_d;
    const double rel = gap / fmax(fabs(P), 1e-300);
    st->cert_iter = st->iter - 1;
    st->P = P;
    st->D = st->best_d;
    st->gap = gap;
    st->rel = rel;
    st->products += 2;
    if (!isfinite(P) || !isfinite(D)) {
        st->status = L1LS_ENUMERIC;
        st->stop = 1;
    } else if (rel <= st->tol || P <= st->f_target) {
        st->status = L1LS_OK;
        st->stop = 1;
    } else if (st->iter - 1 >= st->max_iter) {
        st->status = L1LS_ENOCONV;
        st->stop = 1;
    } else {
        if (st->restart && restart_test > 0.0) {     // momentum against the step: drop it
            st->t = 1.0;
            st->beta = 0.0;
            st->restarts += 1;
        } else {
            const double t = st->t;
            const double tn = __dmul_rn(0.5, __dadd_rn(1.0, sqrt(__dadd_rn(1.0, __dmul_rn(__dmul_rn(4.0, t), t)))));
            st->beta = (t - 1.0) / tn;
            st->t = tn;
        }
        split_ff(st->beta, st->beta_ff);
        st->l1_cur = l1_new;
        st->iter += 1;
    }
}

// (the gradient-restart partial needs more than 64 registers: 3 blocks per SM for that variant)
template <class V, class Vec, bool PAIRED, bool RESTART>
__global__ void __launch_bounds__(kBlock, RESTART ? 3 : L1LS_K2_MIN_BLOCKS) k_fista_k2(K2Args<V, Vec> a) {
    using Acc = Vec;
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    __shared__ double red[3 * 32];
    if (*(volatile int32_t*)&a.st->stop) return;
    const double beta = a.st->beta, L = a.st->L, tau = a.st->tau;
    const double invL = 1.0 / L, thr = tau / L;
    constexpr bool rs = RESTART;   // the gradient-restart partial (an instantiation per setting)
    double p[3] = {0.0, 0.0, 0.0};
    if constexpr (sizeof(Vec) == 4) {
        const ff beta_f = {a.st->beta_ff[0], a.st->beta_ff[1]}, invL_f = {a.st->invL_ff[0], a.st->invL_ff[1]},
                 thr_f = {a.st->thr_ff[0], a.st->thr_ff[1]};
        float gmax = 0.0f;
        ff l1 = {0.0f, 0.0f}, rt = {0.0f, 0.0f};
        struct Ops {
            ff x1, x0;
        };
        cols_of<PAIRED, V, Vec, Acc>(
            a.ptr, a.col, a.val, a.res, a.n, sm, &a.st->stage_err,
            [&](int64_t j, bool has) {
                Ops o{{0.f, 0.f}, {0.f, 0.f}};
                if (has) {
#if L1LS_K2_STREAM_HINTS
                    // read once in this iteration: evict-first, keeping the gathered residual in L2
                    o.x1 = {__ldcs(a.xch + j), __ldcs(a.xcl + j)};
                    o.x0 = {__ldcs(a.xoh + j), __ldcs(a.xol + j)};
#else
                    o.x1 = {a.xch[j], a.xcl[j]};
                    o.x0 = {a.xoh[j], a.xol[j]};
#endif
                }
                return o;
            },
            [&](int64_t j, Acc g, const Ops& o) {
                const FfStep f = ff_fista_step(o.x1, o.x0, ff_from_float(g), beta_f, invL_f, thr_f);
                a.xoh[j] = f.x.hi;
                a.xol[j] = f.x.lo;
                gmax = fmaxf(gmax, fabsf(g));
                sum2_add(l1, f.mag);
                if (rs) sum2_add(rt, ff_mul(ff_sub(f.y, f.x), ff_sub(f.x, o.x1)));
            });
        p[0] = (double)gmax;
        p[1] = ff_to_double(l1);
        p[2] = ff_to_double(rt);
    } else {
        struct Ops {
            double x1, x0;
        };
        cols_of<PAIRED, V, Vec, Acc>(
            a.ptr, a.col, a.val, a.res, a.n, sm, &a.st->stage_err,
            [&](int64_t j, bool has) {
                Ops o{0.0, 0.0};
                if (has) {
                    o.x1 = a.xc[j];
                    o.x0 = a.xo[j];
                }
                return o;
            },
            [&](int64_t j, Acc gacc, const Ops& o) {
                const double g = (double)gacc;
                const double y = o.x1 + beta * (o.x1 - o.x0);
                const double xn = soft_threshold(y + g * invL, thr);
                a.xo[j] = xn;
                p[0] = fmax(p[0], fabs(g));
                p[1] += fabs(xn);
                if (rs) p[2] += (y - xn) * (xn - o.x1);
            });
    }
    block_reduce<kBlock, 3>(p, 1u, red);
    double tot[3];
    if (grid_reduce_last<kBlock, 3>(p, 1u, a.partials, &a.st->cnt2, tot, red) && threadIdx.x == 0)
        fista_finalize(a.st, tot[0], tot[1], tot[2]);
}

// ---- compensated kernels (opts.accum = 1; FP32 / BF16 values) ----------------------------
// The same two kernels with both products accumulated in float-float (tile_ff): K1 gathers
// the high and low words of x_{k-1}, keeps A x in float-float and writes the residual in
// float-float (paired storage: one float4 {hi, hi, lo, lo} per row pair; plain: one float2
// per row); K2 gathers it and forms A^T r in float-float.  FP32 sums of the products put a floor of about 1e-5 .. 1e-2 under the relative
// gap at small tau (the residual is a small difference of large terms, and its rounding error
// does not shrink with the objective); these kernels remove that floor at about twice the
// arithmetic and 16 more bytes per row and 4 more per gathered column of traffic.

template <class V>
struct K1CArgs {
    const int32_t* ptr;
    const int32_t* col;
    const V* val;
    const float2* x;     // x_{k-1}, float-float {hi, lo} pairs (one 8-byte gather per entry)
    float2* ax;          // in: A x_{k-2}; out: A x_{k-1} (float-float)
    float* res;          // out: r_k (layout above)
    const float* b;
    double* partials;
    FistaState* st;
    int64_t m;
};

template <class V>
struct K2CArgs {
    const int32_t* ptr;
    const int32_t* pair;     // pair index (paired) or row index (plain) per entry
    const V* val;
    const float* res;
    const float2* x1;    // x_{k-1} as {hi, lo} pairs
    float2* x0;          // in: x_{k-2}; out: x_k
    double* partials;
    FistaState* st;
    int64_t n;
};

template <class V, bool PAIRED>
__global__ void __launch_bounds__(kBlock, L1LS_K1C_MIN_BLOCKS) k_fista_k1c(K1CArgs<V> a) {
    // paired storage: the staged traversal with float-float sums; plain CSR: lane runs
    __shared__ typename std::conditional<PAIRED, PairedSmem<V, kBlock>, CompSmem<kBlock>>::type sm;
    __shared__ double red[3 * 32];
    if (*(volatile int32_t*)&a.st->stop) return;
    const ff beta = ff_from_double(a.st->beta);
    float* resf = a.res;
    ff q[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    struct Ops {
        ff axo;
        float bb;
    };
    auto pre = [&](int64_t r, bool has) {
        Ops o{{0.f, 0.f}, 0.f};
        if (has) {   // not read again in this iteration (evict-first, as in K1)
            const float2 v = __ldcs(a.ax + r);
            o.axo = {v.x, v.y};
            o.bb = __ldcs(a.b + r);
        }
        return o;
    };
    auto epi = [&](int64_t r, ff u, const Ops& o) {
        const ff ay = ff_add(u, ff_mul(beta, ff_sub(u, o.axo)));
        const ff rr = ff_sub(ff_from_float(o.bb), ay);
        a.ax[r] = make_float2(u.hi, u.lo);
        if (PAIRED) {
            resf[4 * (r >> 1) + (r & 1)] = rr.hi;
            resf[4 * (r >> 1) + 2 + (r & 1)] = rr.lo;
        } else {
            resf[2 * r] = rr.hi;
            resf[2 * r + 1] = rr.lo;
        }
        const ff d = ff_sub(u, ff_from_float(o.bb));
        sum2_add(q[0], ff_mul(d, d));
        sum2_add(q[1], ff_mul(ff_from_float(o.bb), rr));
        sum2_add(q[2], ff_mul(rr, rr));
    };
    const int64_t nrows = PAIRED ? a.m / 2 : a.m;
    if constexpr (PAIRED) {
        warp_pcsr<true, V>(a.ptr, a.col, a.val, nrows, sm, &a.st->stage_err,
                           FFSum<true, V>{reinterpret_cast<const float*>(a.x), nullptr, nullptr}, pre, epi);
    } else {
        const int64_t nw = (int64_t)gridDim.x * (kBlock / 32), ntiles = (nrows + 31) >> 5;
        for (int64_t t = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); t < ntiles; t += nw)
            tile_ff<true, false, V>(t, a.ptr, a.col, a.val, reinterpret_cast<const float*>(a.x), nullptr, nullptr,
                                    nrows, sm.warp_buf(), pre, epi);
    }
    double p[3] = {ff_to_double(q[0]), ff_to_double(q[1]), ff_to_double(q[2])};
    block_reduce<kBlock, 3>(p, 0u, red);
    double tot[3];
    if (grid_reduce_last<kBlock, 3>(p, 0u, a.partials, &a.st->cnt1, tot, red) && threadIdx.x == 0) {
        a.st->k1[0] = tot[0];
        a.st->k1[1] = tot[1];
        a.st->k1[2] = tot[2];
    }
}

template <class V, bool PAIRED>
__global__ void __launch_bounds__(kBlock, L1LS_K2C_MIN_BLOCKS) k_fista_k2c(K2CArgs<V> a) {
    __shared__ typename std::conditional<PAIRED, PairedSmem<V, kBlock>, CompSmem<kBlock>>::type sm;
    __shared__ double red[3 * 32];
    if (*(volatile int32_t*)&a.st->stop) return;
    const bool rs = a.st->restart != 0;
    const ff beta_f = {a.st->beta_ff[0], a.st->beta_ff[1]}, invL_f = {a.st->invL_ff[0], a.st->invL_ff[1]},
             thr_f = {a.st->thr_ff[0], a.st->thr_ff[1]};
    float gmax = 0.0f;
    ff l1 = {0.0f, 0.0f}, rt = {0.0f, 0.0f};
    struct Ops {
        ff x1, x0;
    };
    auto pre = [&](int64_t j, bool has) {
        Ops o{{0.f, 0.f}, {0.f, 0.f}};
        if (has) {   // read once in this iteration (evict-first, as in K2)
            const float2 v1 = __ldcs(a.x1 + j), v0 = __ldcs(a.x0 + j);
            o.x1 = {v1.x, v1.y};
            o.x0 = {v0.x, v0.y};
        }
        return o;
    };
    auto epi = [&](int64_t j, ff g, const Ops& o) {
        const FfStep f = ff_fista_step(o.x1, o.x0, g, beta_f, invL_f, thr_f);
        a.x0[j] = make_float2(f.x.hi, f.x.lo);
        gmax = fmaxf(gmax, fabsf(g.hi));
        sum2_add(l1, f.mag);
        if (rs) sum2_add(rt, ff_mul(ff_sub(f.y, f.x), ff_sub(f.x, o.x1)));
    };
    if constexpr (PAIRED) {
        warp_pcsr<false, V>(a.ptr, a.pair, a.val, a.n, sm, &a.st->stage_err,
                            FFSum<false, V>{nullptr, nullptr, reinterpret_cast<const float4*>(a.res)}, pre, epi);
    } else {
        const int64_t nw = (int64_t)gridDim.x * (kBlock / 32), ntiles = (a.n + 31) >> 5;
        for (int64_t t = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); t < ntiles; t += nw)
            tile_ff<false, false, V>(t, a.ptr, a.pair, a.val, nullptr, nullptr, a.res, a.n, sm.warp_buf(), pre, epi);
    }
    double p[3] = {(double)gmax, ff_to_double(l1), ff_to_double(rt)};
    block_reduce<kBlock, 3>(p, 1u, red);
    double tot[3];
    if (grid_reduce_last<kBlock, 3>(p, 1u, a.partials, &a.st->cnt2, tot, red) && threadIdx.x == 0)
        fista_finalize(a.st, tot[0], tot[1], tot[2]);
}

// ---- matrix-free kernels (instances generated with matrix_free = 1) ------------------------
// K1 = z = Sigma R^T x_{k-1} (a stage sweep, mfree.cu) + k_fista_mf1: the rows of the left
// factor, K1's epilogue, and at once the first half of A^T r: the row pair's residual rotated
// by G~^T and scattered to P2^T order (zt), so the residual itself is never stored.  K2 =
// k_fista_mf2: R Sigma zt by a stage sweep with K2's epilogue and the certificate.  FP32
// products, float-float iterate.

constexpr int kMfUnroll = 4;   // row pairs per thread in flight in k_fista_mf1

struct MfK1Args {
    MfLeft L;
    const float* z;      // Sigma R^T x_{k-1}
    float* zt;           // out: the first n entries of P2^T G~^T r_k
    float* ax;           // in: A x_{k-2}; out: A x_{k-1}
    const float* b;
    double* partials;
    FistaState* st;
};

// read-only load and store with an L2 cache policy (createpolicy)
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float* p, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

__global__ void __launch_bounds__(kBlock, 3) k_fista_mf1(MfK1Args a) {
    __shared__ double red[3 * 32];
    if (*(volatile int32_t*)&a.st->stop) return;
    const float beta = (float)a.st->beta;
    const MfLeft& L = a.L;
    ff q[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    // r = b - A y with A y = u + beta (u - A x_{k-2}); gap partials (u - b)^2, b.r, r.r
    auto epi = [&](float u, float axo, float bb) {
        const float ay = u + beta * (u - axo);
        const float rr = bb - ay;
        const ff d = two_sum(u, -bb);
        ff sq = two_prod(d.hi, d.hi);
        sq.lo = __fmaf_rn(2.0f * d.hi, d.lo, sq.lo);
        sum2_add(q[0], sq);
        sum2_add(q[1], two_prod(bb, rr));
        sum2_add(q[2], two_prod(rr, rr));
        return rr;
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L.left) {
        const int64_t units = L.m / 2;
        const int2* perm2 = reinterpret_cast<const int2*>(L.perm);
        // z and zt with an L2 evict-last policy (the streams above are evict-first): the random
        // half of their accesses finds more of them in L2, and K2 reads zt from L2 (measured:
        // K1 0.2461 -> 0.2449 ms, K2 0.1209 -> 0.1184 ms at C2)
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
        float2* ax2 = reinterpret_cast<float2*>(a.ax);
        const float2* b2 = reinterpret_cast<const float2*>(a.b);
        for (int64_t t0 = gid; t0 < units; t0 += stride * kMfUnroll) {
            int2 pk[kMfUnroll];
            float2 axo[kMfUnroll], bb[kMfUnroll];
            float z0[kMfUnroll], z1[kMfUnroll];
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) {
                const int64_t t = t0 + k * stride;
                pk[k] = make_int2(INT32_MAX, INT32_MAX);
                if (t < units) {
                    pk[k] = __ldcs(perm2 + t);
                    axo[k] = __ldcs(ax2 + t);   // A x_{k-2}, b: streamed (evict-first), so that
                                                // z and zt keep their place in L2
                    bb[k] = __ldcs(b2 + t);
                }
            }
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) {
                z0[k] = 0.0f;
                z1[k] = 0.0f;
                if (pk[k].x < L.n) z0[k] = ld_hint(a.z + pk[k].x, pol);
                if (pk[k].y < L.n) z1[k] = ld_hint(a.z + pk[k].y, pol);
            }
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) {
                const int64_t t = t0 + k * stride;
                if (t >= units) break;
                const float u0 = __fmaf_rn(L.ct, z0[k], -L.st * z1[k]);
                const float u1 = __fmaf_rn(L.ct, z1[k], L.st * z0[k]);
                const float r0 = epi(u0, axo[k].x, bb[k].x);
                const float r1 = epi(u1, axo[k].y, bb[k].y);
                __stcs(ax2 + t, make_float2(u0, u1));
                if (pk[k].x < L.n) st_hint(a.zt + pk[k].x, __fmaf_rn(L.ct, r0, L.st * r1), pol);
                if (pk[k].y < L.n) st_hint(a.zt + pk[k].y, __fmaf_rn(L.ct, r1, -L.st * r0), pol);
            }
        }
    } else {
        for (int64_t t = gid; t < L.m; t += stride) {
            const float u = t < L.n ? __ldg(a.z + t) : 0.0f;
            const float rr = epi(u, a.ax[t], __ldcs(a.b + t));
            a.ax[t] = u;
            if (t < L.n) a.zt[t] = rr;
        }
    }
    double p[3] = {ff_to_double(q[0]), ff_to_double(q[1]), ff_to_double(q[2])};
    block_reduce<kBlock, 3>(p, 0u, red);
    double tot[3];
    if (grid_reduce_last<kBlock, 3>(p, 0u, a.partials, &a.st->cnt1, tot, red) && threadIdx.x == 0) {
        a.st->k1[0] = tot[0];
        a.st->k1[1] = tot[1];
        a.st->k1[2] = tot[2];
    }
}

struct MfK2Args {
    MfRight R;
    const float* sigma;
    const float* z;      // P2^T G~^T r_k (first n entries)
    const float* xch;
    const float* xcl;
    float* xoh;
    float* xol;
    double* partials;
    FistaState* st;
};

template <bool RESTART>
__global__ void __launch_bounds__(kMfThreads) k_fista_mf2(MfK2Args a) {
    __shared__ float buf[kMfLen];
    __shared__ double red[3 * 32];
    if (*(volatile int32_t*)&a.st->stop) return;
    const ff beta_f = {a.st->beta_ff[0], a.st->beta_ff[1]}, invL_f = {a.st->invL_ff[0], a.st->invL_ff[1]},
             thr_f = {a.st->thr_ff[0], a.st->thr_ff[1]};
    float gmax = 0.0f;
    ff l1 = {0.0f, 0.0f}, rt = {0.0f, 0.0f};
    // persistent blocks take tiles in turn (fewer per-block partials for the last block to sum)
    const int64_t ntiles = (a.R.n + kMfTile - 1) / kMfTile;
    constexpr int kPer = kMfTile / kMfThreads;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t a0 = tile * kMfTile;
        // this thread's iterates of the tile, loaded before the stage sweep so that their
        // latency overlaps the sweep (the new iterate overwrites x0 only after all are read)
        ff x1[kPer], x0[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int64_t j = a0 + (int)threadIdx.x + u * kMfThreads;
            x1[u] = x0[u] = ff{0.0f, 0.0f};
            if (j < a.R.n) {
                x1[u] = ff{__ldcs(a.xch + j), __ldcs(a.xcl + j)};
                x0[u] = ff{__ldcs(a.xoh + j), __ldcs(a.xol + j)};
            }
        }
        mf_load<true>(buf, a.z, a.sigma, a0 - kMfHalo, a.R.n);
        mf_stages<false>(buf, a0 - kMfHalo, a.R);
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int p = (int)threadIdx.x + u * kMfThreads;
            const int64_t j = a0 + p;
            if (j >= a.R.n) break;
            const float g = buf[kMfHalo + p];
            const FfStep f = ff_fista_step(x1[u], x0[u], ff_from_float(g), beta_f, invL_f, thr_f);
            a.xoh[j] = f.x.hi;
            a.xol[j] = f.x.lo;
            gmax = fmaxf(gmax, fabsf(g));
            sum2_add(l1, f.mag);
            if (RESTART) sum2_add(rt, ff_mul(ff_sub(f.y, f.x), ff_sub(f.x, x1[u])));
        }
        __syncthreads();   // the tile buffer is reloaded next
    }
    double pp[3] = {(double)gmax, ff_to_double(l1), ff_to_double(rt)};
    block_reduce<kMfThreads, 3>(pp, 1u, red);
    double tot[3];
    if (grid_reduce_last<kMfThreads, 3>(pp, 1u, a.partials, &a.st->cnt2, tot, red) && threadIdx.x == 0)
        fista_finalize(a.st, tot[0], tot[1], tot[2]);
}

__global__ void k_abs_sum(const double* __restrict__ x, int64_t n, double* __restrict__ partials,
                          unsigned* __restrict__ counter, double* __restrict__ out) {
    __shared__ double red[32];
    double v[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[0] += fabs(x[i]);
    block_reduce<kBlock, 1>(v, 0u, red);
    double tot[1];
    if (grid_reduce_last<kBlock, 1>(v, 0u, partials, counter, tot, red) && threadIdx.x == 0) *out = tot[0];
}

__global__ void k_d2ff(const double* __restrict__ in, int64_t n, float* __restrict__ hi, float* __restrict__ lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ff v = ff_from_double(in[i]);
    hi[i] = v.hi;
    lo[i] = v.lo;
}

__global__ void k_ff2d(const float* __restrict__ hi, const float* __restrict__ lo, int64_t n, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ff_to_double({hi[i], lo[i]});
}

// the same for the {hi, lo} pairs of the float-float kernels
__global__ void k_d2ff2(const double* __restrict__ in, int64_t n, float2* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ff v = ff_from_double(in[i]);
    out[i] = make_float2(v.hi, v.lo);
}

__global__ void k_ff22d(const float2* __restrict__ x, int64_t n, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ff_to_double({x[i].x, x[i].y});
}

template <class K>
int grid_of(const Inst* I, K kernel, int64_t rows) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = (rows + 31) / 32 / (kBlock / 32) + 1;   // blocks with one warp tile per warp
    const int64_t g = (int64_t)I->ctx->num_sms * per_sm;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, g));
}

// Per-instance FISTA work space and cached graph.
struct FistaWork {
    double* X[2] = {nullptr, nullptr};   // FP64 values: iterates
    float* Xh[2] = {nullptr, nullptr};   // FP32 / BF16 values: iterates as float-float
    float* Xl[2] = {nullptr, nullptr};
    double* tmp64 = nullptr;             // FP64 staging of x0 / x_out
    void* ax = nullptr;
    void* res = nullptr;
    float* zmf = nullptr;                // matrix-free products: Sigma R^T x, and P2^T G~^T r
    float* zt = nullptr;
    float2* ax_ff = nullptr;             // compensated kernels: A x and the residual (2m floats)
    float* res_ff = nullptr;
    float2* X2[2] = {nullptr, nullptr};  // compensated kernels: the iterates as {hi, lo} pairs
    int grid1c = 0, grid2c = 0;
    bool comp = false;                   // this run uses the compensated kernels
    bool restart = false;                // this run uses the gradient restart
    int exec_comp = -1, exec_restart = -1;
    double* part1 = nullptr;
    double* part2 = nullptr;
    FistaState* st = nullptr;
    FistaState* host_st = nullptr;   // host copy of the state
    int grid1 = 0, grid2 = 0;
    int grid2r = 0;                      // K2 with the gradient-restart partial (more registers)
    cudaGraphExec_t exec = nullptr;
    int exec_chunk = 0;
    int64_t enqueued = 0;           // iterations enqueued since begin (parity of the next one)
    bool active = false;
    cudaEvent_t ev[2][3] = {};
    Ctx* pin_ctx = nullptr;   // host_st is a pinned slot of this context (else pageable)
    ~FistaWork() {
        if (exec) cudaGraphExecDestroy(exec);
        if (pin_ctx) pin_ctx->pinned_put(host_st);
        else delete host_st;
        for (auto& row : ev)
            for (auto& e : row)
                if (e) cudaEventDestroy(e);
    }
};

template <class V, class Vec>
l1ls_status enqueue_k1(Inst* I, FistaWork* w, int parity, cudaStream_t st) {
    // parity 0: iteration k odd (x_{k-1} in X[0]); parity 1: k even (x_{k-1} in X[1])
    const int c = parity;
    K1Args<V, Vec> a1;
    a1.ptr = I->csr_ptr;
    a1.col = I->csr_col;
    a1.val = static_cast<const V*>(I->csr_val);
    if constexpr (sizeof(Vec) == 8) a1.x = reinterpret_cast<const Vec*>(w->X[c]);
    else a1.x = reinterpret_cast<const Vec*>(w->Xh[c]);   // hi part of the float-float iterate
    a1.ax = static_cast<Vec*>(w->ax);
    a1.res = static_cast<Vec*>(w->res);
    if constexpr (sizeof(Vec) == 8) a1.b = reinterpret_cast<const Vec*>(I->bhat);
    else a1.b = reinterpret_cast<const Vec*>(I->bhat32);
    a1.partials = w->part1;
    a1.st = w->st;
    a1.m = I->m;
    if (I->paired) {
        a1.ptr = I->prow_ptr;
        a1.col = I->prow_col;
        a1.val = static_cast<const V*>(I->prow_val);
        k_fista_k1<V, Vec, true><<<w->grid1, kBlock, 0, st>>>(a1);
    } else {
        k_fista_k1<V, Vec, false><<<w->grid1, kBlock, 0, st>>>(a1);
    }
    return L1LS_OK;
}

template <class V, class Vec>
l1ls_status enqueue_k2(Inst* I, FistaWork* w, int parity, cudaStream_t st) {
    const int c = parity, o = 1 - parity;
    K2Args<V, Vec> a2;
    a2.ptr = I->csc_ptr;
    a2.col = I->csc_row;
    a2.val = static_cast<const V*>(I->csc_val);
    a2.res = static_cast<const Vec*>(w->res);
    a2.xc = w->X[c];
    a2.xo = w->X[o];
    a2.xch = w->Xh[c];
    a2.xcl = w->Xl[c];
    a2.xoh = w->Xh[o];
    a2.xol = w->Xl[o];
    a2.partials = w->part2;
    a2.st = w->st;
    a2.n = I->n;
    if (I->paired) {
        a2.ptr = I->pcol_ptr;
        a2.col = I->pcol_pair;
        a2.val = static_cast<const V*>(I->pcol_val);
        if (w->restart) k_fista_k2<V, Vec, true, true><<<w->grid2r, kBlock, 0, st>>>(a2);
        else k_fista_k2<V, Vec, true, false><<<w->grid2, kBlock, 0, st>>>(a2);
    } else {
        if (w->restart) k_fista_k2<V, Vec, false, true><<<w->grid2r, kBlock, 0, st>>>(a2);
        else k_fista_k2<V, Vec, false, false><<<w->grid2, kBlock, 0, st>>>(a2);
    }
    return L1LS_OK;
}

template <class V>
void enqueue_k1c(Inst* I, FistaWork* w, int parity, cudaStream_t st) {
    K1CArgs<V> a;
    a.ptr = I->paired ? I->prow_ptr : I->csr_ptr;
    a.col = I->paired ? I->prow_col : I->csr_col;
    a.val = static_cast<const V*>(I->paired ? I->prow_val : I->csr_val);
    a.x = w->X2[parity];
    a.ax = w->ax_ff;
    a.res = w->res_ff;
    a.b = I->bhat32;
    a.partials = w->part1;
    a.st = w->st;
    a.m = I->m;
    if (I->paired) k_fista_k1c<V, true><<<w->grid1c, kBlock, 0, st>>>(a);
    else k_fista_k1c<V, false><<<w->grid1c, kBlock, 0, st>>>(a);
}

template <class V>
void enqueue_k2c(Inst* I, FistaWork* w, int parity, cudaStream_t st) {
    const int c = parity, o = 1 - parity;
    K2CArgs<V> a;
    a.ptr = I->paired ? I->pcol_ptr : I->csc_ptr;
    a.pair = I->paired ? I->pcol_pair : I->csc_row;
    a.val = static_cast<const V*>(I->paired ? I->pcol_val : I->csc_val);
    a.res = w->res_ff;
    a.x1 = w->X2[c];
    a.x0 = w->X2[o];
    a.partials = w->part2;
    a.st = w->st;
    a.n = I->n;
    if (I->paired) k_fista_k2c<V, true><<<w->grid2c, kBlock, 0, st>>>(a);
    else k_fista_k2c<V, false><<<w->grid2c, kBlock, 0, st>>>(a);
}

void enqueue_mf(Inst* I, FistaWork* w, int parity, int which, cudaStream_t st) {
    if (which == 0) {
        mf_apply_rt(I, w->Xh[parity], w->zmf, st);
        MfK1Args a;
        a.L = MfLeft{I->m, I->n, I->p.left_stages, I->mf_ct, I->mf_st, I->mf_pperm};
        a.z = w->zmf;
        a.zt = w->zt;
        a.ax = static_cast<float*>(w->ax);
        a.b = I->bhat32;
        a.partials = w->part1;
        a.st = w->st;
        k_fista_mf1<<<w->grid1, kBlock, 0, st>>>(a);
    } else {
        MfK2Args a;
        a.R = MfRight{I->n, I->p.right_stages, I->mf_c, I->mf_s};
        a.sigma = I->sigma32;
        a.z = w->zt;
        a.xch = w->Xh[parity];
        a.xcl = w->Xl[parity];
        a.xoh = w->Xh[1 - parity];
        a.xol = w->Xl[1 - parity];
        a.partials = w->part2;
        a.st = w->st;
        if (w->restart) k_fista_mf2<true><<<w->grid2, kMfThreads, 0, st>>>(a);
        else k_fista_mf2<false><<<w->grid2, kMfThreads, 0, st>>>(a);
    }
}

template <class V, class Vec>
l1ls_status enqueue_one(Inst* I, FistaWork* w, int parity, int which, cudaStream_t st) {
    if constexpr (sizeof(Vec) == 4) {
        if (I->matrix_free) {
            enqueue_mf(I, w, parity, which, st);
            return L1LS_OK;
        }
        if (w->comp) {
            if (which == 0) enqueue_k1c<V>(I, w, parity, st);
            else enqueue_k2c<V>(I, w, parity, st);
            return L1LS_OK;
        }
    }
    return which == 0 ? enqueue_k1<V, Vec>(I, w, parity, st) : enqueue_k2<V, Vec>(I, w, parity, st);
}

template <class V, class Vec>
l1ls_status enqueue_iteration(Inst* I, FistaWork* w, int parity, cudaStream_t st) {
    L1LS_TRY((enqueue_one<V, Vec>(I, w, parity, 0, st)));
    return enqueue_one<V, Vec>(I, w, parity, 1, st);
}

template <class V, class Vec>
l1ls_status begin(Inst* I, const l1ls_solve_opts* o, const double* x0, cudaStream_t st) {
    const int64_t m = I->m, n = I->n;
    if (o->accum != 0 && sizeof(Vec) == 8)
        return set_error(L1LS_EINVAL, "accum = 1 (float-float products) needs FP32 or BF16 values");
    if (o->accum != 0 && I->matrix_free)
        return set_error(L1LS_EINVAL, "accum = 1 is not available for matrix-free instances");
    if (o->accum != 0 && o->accum != 1) return set_error(L1LS_EINVAL, "accum must be 0 or 1");
    FistaWork* w = static_cast<FistaWork*>(I->fista_work);
    if (!w) {
        // the work space is attached to the instance only once complete: a failed allocation
        // leaves no partial work space for the next solve to use
        std::unique_ptr<FistaWork> fresh(new FistaWork());
        w = fresh.get();
        if (sizeof(Vec) == 8) {
            L1LS_TRY(I->alloc_n(&w->X[0], pad32(n)));
            L1LS_TRY(I->alloc_n(&w->X[1], pad32(n)));
        } else {
            for (int k = 0; k < 2; ++k) {
                L1LS_TRY(I->alloc_n(&w->Xh[k], pad32(n)));
                L1LS_TRY(I->alloc_n(&w->Xl[k], pad32(n)));
            }
        }
        L1LS_TRY(I->alloc_n(&w->tmp64, pad32(n)));
        L1LS_TRY(I->alloc(&w->ax, sizeof(Vec) * pad32(m)));
        L1LS_TRY(I->alloc(&w->res, sizeof(Vec) * pad32(m)));
        if (I->matrix_free) {
            L1LS_TRY(I->alloc_n(&w->zmf, pad32(n)));
            L1LS_TRY(I->alloc_n(&w->zt, pad32(n)));
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fista_mf1, kBlock, 0);
            const int64_t units = I->p.left_stages ? m / 2 : m;
            w->grid1 = (int)std::max<int64_t>(
                1, std::min<int64_t>((units + (int64_t)kBlock * kMfUnroll - 1) / ((int64_t)kBlock * kMfUnroll),
                                     (int64_t)I->ctx->num_sms * std::max(per_sm, 1)));
            int per_sm2 = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_fista_mf2<false>, kMfThreads, 0);
            w->grid2 = (int)std::max<int64_t>(1, std::min<int64_t>((n + kMfTile - 1) / kMfTile,
                                                                     (int64_t)I->ctx->num_sms * std::max(per_sm2, 1)));
        } else if (I->paired) {
            w->grid1 = grid_of(I, k_fista_k1<V, Vec, true>, m / 2);
            w->grid2 = grid_of(I, k_fista_k2<V, Vec, true, false>, n);
            w->grid2r = grid_of(I, k_fista_k2<V, Vec, true, true>, n);
        } else {
            w->grid1 = grid_of(I, k_fista_k1<V, Vec, false>, m);
            w->grid2 = grid_of(I, k_fista_k2<V, Vec, false, false>, n);
            w->grid2r = grid_of(I, k_fista_k2<V, Vec, false, true>, n);
        }
        L1LS_TRY(I->alloc_n(&w->part1, (int64_t)w->grid1 * 3));
        L1LS_TRY(I->alloc_n(&w->part2, (int64_t)w->grid2 * 3 + 1024));
        L1LS_TRY(I->alloc_n(&w->st, 1));
        // the state read back at every host check: a pinned slot of the context, else pageable
        if (void* slot = I->ctx->pinned_get(sizeof(FistaState))) {
            w->host_st = new (slot) FistaState();
            w->pin_ctx = I->ctx;
        } else {
            w->host_st = new FistaState();
        }
        for (int k = 0; k < 2; ++k) {
            L1LS_CUDA(cudaEventCreate(&w->ev[k][0]));
            L1LS_CUDA(cudaEventCreate(&w->ev[k][1]));
            L1LS_CUDA(cudaEventCreate(&w->ev[k][2]));
        }
        I->fista_work = fresh.release();
        I->fista_work_free = [](void* p) { delete static_cast<FistaWork*>(p); };
    }
    if constexpr (sizeof(Vec) == 4) {
        if (o->accum == 1 && !w->res_ff) {   // res_ff last: set only when all exist
            for (int k = 0; k < 2; ++k)
                if (!w->X2[k]) L1LS_TRY(I->alloc_n(&w->X2[k], pad32(n)));
            if (!w->ax_ff) L1LS_TRY(I->alloc_n(&w->ax_ff, pad32(m)));
            L1LS_TRY(I->alloc_n(&w->res_ff, 2 * pad32(m)));
            if (I->paired) {
                w->grid1c = grid_of(I, k_fista_k1c<V, true>, m / 2);
                w->grid2c = grid_of(I, k_fista_k2c<V, true>, n);
            } else {
                w->grid1c = grid_of(I, k_fista_k1c<V, false>, m);
                w->grid2c = grid_of(I, k_fista_k2c<V, false>, n);
            }
        }
    }
    w->comp = o->accum == 1;
    w->restart = o->restart != 0;
    FistaState h{};
    h.tau = o->tau;
    h.L = I->lipschitz;
    h.tol = o->rel_gap_tol;
    h.f_target = o->f_target;
    h.max_iter = o->max_iter;
    h.t = 1.0;
    h.beta = 0.0;
    h.best_d = -INFINITY;
    h.iter = 1;
    h.cert_iter = 0;
    h.stop = 0;
    h.status = L1LS_OK;
    h.restart = o->restart;
    h.restarts = 0;
    split_ff(0.0, h.beta_ff);
    split_ff(1.0 / h.L, h.invL_ff);
    split_ff(h.tau / h.L, h.thr_ff);
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (x0) {
        // x0 (device or host FP64) -> FP64 staging -> iterate buffers
        L1LS_CUDA(cudaMemcpyAsync(w->tmp64, x0, sizeof(double) * n, cudaMemcpyDefault, st));
        if (sizeof(Vec) == 8) {
            L1LS_CUDA(cudaMemcpyAsync(w->X[0], w->tmp64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            L1LS_CUDA(cudaMemcpyAsync(w->X[1], w->tmp64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        } else if (w->comp) {
            k_d2ff2<<<nb, 256, 0, st>>>(w->tmp64, n, w->X2[0]);
            k_d2ff2<<<nb, 256, 0, st>>>(w->tmp64, n, w->X2[1]);
        } else {
            k_d2ff<<<nb, 256, 0, st>>>(w->tmp64, n, w->Xh[0], w->Xl[0]);
            k_d2ff<<<nb, 256, 0, st>>>(w->tmp64, n, w->Xh[1], w->Xl[1]);
        }
        // ||x0||_1 into the state, A x0 into ax (relabelled rows)
        L1LS_CUDA(cudaMemsetAsync(&w->st->cnt1, 0, sizeof(unsigned), st));
        k_abs_sum<<<256, kBlock, 0, st>>>(w->tmp64, n, w->part2, &w->st->cnt1, &w->st->l1_cur);
        L1LS_CUDA(cudaGetLastError());
        if (w->comp) {
            // beta_1 = 0: A x_{k-2} is not used at k = 1 (any finite value will do)
            L1LS_CUDA(cudaMemsetAsync(w->ax_ff, 0, sizeof(float2) * m, st));
            h.products = 0;
        } else {
            const void* xsrc = sizeof(Vec) == 8 ? (const void*)w->X[0] : (const void*)w->Xh[0];
            L1LS_TRY(spmv_plain(I, false, xsrc, sizeof(Vec) == 8 ? L1LS_F64 : L1LS_F32, w->ax, false, st));
            h.products = 1;
        }
        L1LS_CUDA(cudaMemcpyAsync(&w->host_st->l1_cur, &w->st->l1_cur, sizeof(double), cudaMemcpyDeviceToHost, st));
        L1LS_CUDA(cudaStreamSynchronize(st));
        h.l1_cur = w->host_st->l1_cur;
    } else {
        if (sizeof(Vec) == 8) {
            L1LS_CUDA(cudaMemsetAsync(w->X[0], 0, sizeof(double) * n, st));
            L1LS_CUDA(cudaMemsetAsync(w->X[1], 0, sizeof(double) * n, st));
        } else if (w->comp) {
            for (int k = 0; k < 2; ++k) L1LS_CUDA(cudaMemsetAsync(w->X2[k], 0, sizeof(float2) * n, st));
        } else {
            for (int k = 0; k < 2; ++k) {
                L1LS_CUDA(cudaMemsetAsync(w->Xh[k], 0, sizeof(float) * n, st));
                L1LS_CUDA(cudaMemsetAsync(w->Xl[k], 0, sizeof(float) * n, st));
            }
        }
        L1LS_CUDA(cudaMemsetAsync(w->ax, 0, sizeof(Vec) * m, st));
        if (w->comp) L1LS_CUDA(cudaMemsetAsync(w->ax_ff, 0, sizeof(float2) * m, st));
        h.products = 0;
        h.l1_cur = 0.0;
    }
    h.cnt1 = h.cnt2 = 0;
    *w->host_st = h;
    L1LS_CUDA(cudaMemcpyAsync(w->st, w->host_st, sizeof(FistaState), cudaMemcpyHostToDevice, st));
    w->enqueued = 0;
    w->active = true;
    return L1LS_OK;
}

// Enqueue `iters` iterations one by one (parity tracked on the host).  With kernel_ms, CUDA
// events bracket K1 and K2 of every iteration and their summed durations are returned
// (the stream is synchronised for that).
template <class V, class Vec>
l1ls_status step(Inst* I, int64_t iters, float* kernel_ms, cudaStream_t st) {
    FistaWork* w = static_cast<FistaWork*>(I->fista_work);
    if (!w || !w->active) return set_error(L1LS_EINVAL, "l1ls_fista_step without l1ls_fista_begin");
    float acc[2] = {0.f, 0.f};
    for (int64_t i = 0; i < iters; ++i) {
        const int parity = (int)(w->enqueued & 1);
        if (kernel_ms) {
            cudaEvent_t* e = w->ev[i & 1];
            if (i >= 2) {   // collect the timings of the iteration that used these events
                L1LS_CUDA(cudaEventSynchronize(e[2]));
                float a = 0.f, b = 0.f;
                L1LS_CUDA(cudaEventElapsedTime(&a, e[0], e[1]));
                L1LS_CUDA(cudaEventElapsedTime(&b, e[1], e[2]));
                acc[0] += a;
                acc[1] += b;
            }
            L1LS_CUDA(cudaEventRecord(e[0], st));
            L1LS_TRY((enqueue_one<V, Vec>(I, w, parity, 0, st)));
            L1LS_CUDA(cudaEventRecord(e[1], st));
            L1LS_TRY((enqueue_one<V, Vec>(I, w, parity, 1, st)));
            L1LS_CUDA(cudaEventRecord(e[2], st));
        } else {
            L1LS_TRY(enqueue_iteration<V, Vec>(I, w, parity, st));
        }
        ++w->enqueued;
    }
    L1LS_CUDA(cudaGetLastError());
    if (kernel_ms) {
        for (int64_t i = std::max<int64_t>(0, iters - 2); i < iters; ++i) {
            cudaEvent_t* e = w->ev[i & 1];
            L1LS_CUDA(cudaEventSynchronize(e[2]));
            float a = 0.f, b = 0.f;
            L1LS_CUDA(cudaEventElapsedTime(&a, e[0], e[1]));
            L1LS_CUDA(cudaEventElapsedTime(&b, e[1], e[2]));
            acc[0] += a;
            acc[1] += b;
        }
        kernel_ms[0] = acc[0];
        kernel_ms[1] = acc[1];
    }
    return L1LS_OK;
}

l1ls_status end(Inst* I, double* x_out, l1ls_result* res, l1ls_status final_status, double seconds,
                cudaStream_t st) {
    FistaWork* w = static_cast<FistaWork*>(I->fista_work);
    if (!w || !w->active) return set_error(L1LS_EINVAL, "l1ls_fista_end without l1ls_fista_begin");
    L1LS_CUDA(cudaMemcpyAsync(w->host_st, w->st, sizeof(FistaState), cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    const FistaState& f = *w->host_st;
    if (final_status == L1LS_OK) final_status = f.stop ? (l1ls_status)f.status : L1LS_ENOCONV;
    if (f.stage_err && final_status == L1LS_OK)
        final_status = set_error(L1LS_ECUDA, "a bulk-copy stage wait ran out of polls (sums read directly)");
    if (x_out) {
        const int c = (int)(f.cert_iter & 1);
        if (w->X[c]) {
            L1LS_CUDA(cudaMemcpyAsync(x_out, w->X[c], sizeof(double) * I->n, cudaMemcpyDefault, st));
        } else if (w->comp) {
            k_ff22d<<<(unsigned)((I->n + 255) / 256), 256, 0, st>>>(w->X2[c], I->n, w->tmp64);
            L1LS_CUDA(cudaGetLastError());
            L1LS_CUDA(cudaMemcpyAsync(x_out, w->tmp64, sizeof(double) * I->n, cudaMemcpyDefault, st));
        } else {
            k_ff2d<<<(unsigned)((I->n + 255) / 256), 256, 0, st>>>(w->Xh[c], w->Xl[c], I->n, w->tmp64);
            L1LS_CUDA(cudaGetLastError());
            L1LS_CUDA(cudaMemcpyAsync(x_out, w->tmp64, sizeof(double) * I->n, cudaMemcpyDefault, st));
        }
    }
    L1LS_CUDA(cudaStreamSynchronize(st));
    w->active = false;
    if (res) {
        memset(res, 0, sizeof(*res));
        res->iters = f.cert_iter;
        res->products = f.products;
        res->f = f.P;
        res->dual = f.D;
        res->gap = f.gap;
        res->rel_gap = f.rel;
        res->status = final_status;
        res->seconds = seconds;
    }
    if (final_status != L1LS_OK) {
        const char* why = final_status == L1LS_ENOCONV ? "iteration limit reached"
                          : final_status == L1LS_ETIMEOUT ? "time limit reached"
                          : final_status == L1LS_ENUMERIC ? "NaN or Inf in the iteration"
                          : final_status == L1LS_ECANCELLED ? "cancelled"
                                                          : "internal error";
        return set_error(final_status, "FISTA: %s (rel_gap %.3e)", why, f.rel);
    }
    return L1LS_OK;
}

template <class V, class Vec>
l1ls_status graph_for(Inst* I, FistaWork* w, int chunk) {
    if (w->exec && w->exec_chunk == chunk && w->exec_comp == (int)w->comp && w->exec_restart == (int)w->restart)
        return L1LS_OK;
    if (w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
    }
    cudaStream_t cap;
    L1LS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph;
    L1LS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) enqueue_iteration<V, Vec>(I, w, i & 1, cap);
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
    }
    L1LS_CUDA(cudaGraphInstantiate(&w->exec, graph, 0));
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    w->exec_chunk = chunk;
    w->exec_comp = (int)w->comp;
    w->exec_restart = (int)w->restart;
    return L1LS_OK;
}

template <class V, class Vec>
l1ls_status run(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res,
                cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    L1LS_TRY(begin<V, Vec>(I, o, x0, st));
    FistaWork* w = static_cast<FistaWork*>(I->fista_work);
    int chunk = o->check_every > 0 ? o->check_every : 32;
    if (chunk & 1) ++chunk;
    L1LS_TRY(graph_for<V, Vec>(I, w, chunk));
    l1ls_status final_status = L1LS_OK;
    // the device stops by itself at max_iter; the host cap only guards against a stuck flag
    const int64_t max_launches = o->max_iter / chunk + 3;
    for (int64_t launch = 0;; ++launch) {
        if (launch >= max_launches) {
            final_status = L1LS_ECUDA;
            break;
        }
        L1LS_CUDA(cudaGraphLaunch(w->exec, st));
        w->enqueued += chunk;
        L1LS_CUDA(cudaMemcpyAsync(w->host_st, w->st, sizeof(FistaState), cudaMemcpyDeviceToHost, st));
        L1LS_CUDA(cudaStreamSynchronize(st));
        if (w->host_st->stop) break;
        if (cancel_requested()) {
            final_status = L1LS_ECANCELLED;
            break;
        }
        if (o->time_limit_s > 0) {
            double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > o->time_limit_s) {
                final_status = L1LS_ETIMEOUT;
                break;
            }
        }
    }
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return end(I, x_out, res, final_status, secs, st);
}

}  // namespace

l1ls_status fista_solve(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res,
                        cudaStream_t st) {
    switch (I->dtype) {
        case L1LS_F64: return run<double, double>(I, o, x0, x_out, res, st);
        case L1LS_F32: return run<float, float>(I, o, x0, x_out, res, st);
        default: return run<__nv_bfloat16, float>(I, o, x0, x_out, res, st);
    }
}

}  // namespace l1ls

using namespace l1ls;

static l1ls_status check_opts(const l1ls_solve_opts* o) {
    if (!o) return set_error(L1LS_EINVAL, "NULL options");
    if (!(o->tau > 0.0) || !(o->rel_gap_tol >= 0.0) || o->max_iter < 0)
        return set_error(L1LS_EINVAL, "bad solver options");
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_solve_fista(l1ls_inst* h, const l1ls_solve_opts* o, const double* x0, double* x_out,
                                        l1ls_result* res, void* stream) {
    if (!h) return set_error(L1LS_EINVAL, "NULL argument");
    L1LS_TRY(check_opts(o));
    Inst* I = reinterpret_cast<Inst*>(h);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    return fista_solve(I, o, x0, x_out, res, (cudaStream_t)stream);
}

extern "C" l1ls_status l1ls_fista_begin(l1ls_inst* h, const l1ls_solve_opts* o, const double* x0, void* stream) {
    if (!h) return set_error(L1LS_EINVAL, "NULL argument");
    L1LS_TRY(check_opts(o));
    Inst* I = reinterpret_cast<Inst*>(h);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    switch (I->dtype) {
        case L1LS_F64: return begin<double, double>(I, o, x0, st);
        case L1LS_F32: return begin<float, float>(I, o, x0, st);
        default: return begin<__nv_bfloat16, float>(I, o, x0, st);
    }
}

extern "C" l1ls_status l1ls_fista_step(l1ls_inst* h, int64_t iters, float* kernel_ms, void* stream) {
    if (!h || iters < 0) return set_error(L1LS_EINVAL, "bad argument");
    Inst* I = reinterpret_cast<Inst*>(h);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    switch (I->dtype) {
        case L1LS_F64: return step<double, double>(I, iters, kernel_ms, st);
        case L1LS_F32: return step<float, float>(I, iters, kernel_ms, st);
        default: return step<__nv_bfloat16, float>(I, iters, kernel_ms, st);
    }
}

extern "C" l1ls_status l1ls_fista_end(l1ls_inst* h, double* x_out, l1ls_result* res, void* stream) {
    if (!h) return set_error(L1LS_EINVAL, "NULL argument");
    Inst* I = reinterpret_cast<Inst*>(h);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    return end(I, x_out, res, L1LS_OK, 0.0, (cudaStream_t)stream);
}
