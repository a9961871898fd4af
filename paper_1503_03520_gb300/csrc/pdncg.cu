// pdNCG (Sec. 8.1, parameters of Sec. 8.3): primal-dual Newton-CG on the pseudo-Huber
// smoothing f^mu(x) = tau psi_mu(x) + 1/2 ||A x - b||^2 (Eqs. pseudoHuber, prob2, bd4).
//
// Newton step (one host round trip per phase; all arithmetic in the kernels):
//   N1  r = b - A x                               (partials ||r||^2, b.r)
//   N2  a = A^T r                                 (partials max|a|, ||x||_1); last CTA: gap
//       certificate at x, stop test, mu-continuation (mu /= 10 after a full Newton step
//       until the paper's mu; below it when a full step failed to halve the gap)
//   N3  w = sqrt(mu^2 + x^2), grad = tau x / w - a, h = tau (1 - g x / w) / w (primal-dual
//       curvature with the dual estimate g = clip(a / tau, -1, 1): the linear condition
//       tau g + A^T (A x - b) = 0 solved for g at the current x and projected onto the box),
//       M^{-1} = 1 / (h + diag(A^T A)), PCG start
//   PCG iteration (stopped when the residual in the preconditioner's norm falls to
//   pcg_rtol of its start, or at pcg_max), three kernels: the update of the search direction
//   p = z + beta p (z = M^{-1} res) is folded into the products, A p = A z + beta (A p_old),
//   so no pass of its own is needed:
//   C1  Ap = A z + beta Ap                     C2  p = z + beta p, Hp = h p + A^T Ap,
//                                                  alpha = rz / p.Hp
//   C3  d += alpha p, res -= alpha Hp, z = M^{-1} res, rz, beta
//   L1  Ad = A d (r.Ad, ||Ad||^2);  LT  Armijo trials, four halvings per pass, per-coordinate
//       psi differences;  L3  x += alpha d
// Precision: the iterate x, A^T r, the gradient and every reduction across blocks (the
// certificate, the CG inner products) are FP64.  The other CG vectors (h, M^{-1}, z, p, Hp,
// d) are held in the product precision: FP32 with FP32 / BF16 values, FP64 with FP64 values.
// The CG residual res is FP64 with FP64 values and float-float (hi, lo; about 48 bits) with
// FP32 / BF16 values, where its update and the per-thread sums of the inner products run as
// float-float arithmetic on the FP32 pipes: this GPU's FP64 pipe has a small fraction of the
// FP32 rate, and FP64 arithmetic per entry (with the conversions to and from FP32) made the
// vector update the slowest kernel of the iteration.
// Matrix-free instances (A in factored form) run the same Newton loop with the passes of
// run_mf below: the gradient and certificate in one FP64 sweep, the PCG product in one FP32
// sweep (A^T A = R Sigma^2 R^T), the line search's ||A d|| in one FP32 sweep.
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>

#include "internal.h"
#include "mfree.cuh"
#include "spmv.cuh"

namespace l1ls {

namespace {

constexpr int kBlock = 256;
constexpr int kTrialsPerPass = 4;

struct PdState {
    double tau, tol, mu, mu_target, mu_min, pcg_rtol, armijo, stall;
    int64_t max_newton, pcg_max, ls_max;
    double P, D, gap, rel, prev_gap;
    int32_t prev_full, stage_err;   // stage_err: kStageTimeout if a stage wait ran out
    double k1[2];
    double rz, rz0, alpha, beta;
    int32_t cg_done, pad1;
    int64_t cg_it;
    double rAd, AdAd, step;
    int32_t ls_done, pad2;
    int64_t ls_trial;
    int32_t stop, status;
    int64_t iter, products, cg_total, ls_total;
    unsigned cnt[8];
    double f_target;   // stop once P(x) <= f_target (-inf: off)
    double bb;         // ||b||^2 (matrix-free instances)
    double slope;      // grad.d of the current line search (float-float trials)
};
static_assert(sizeof(PdState) <= Ctx::kPinnedSlotBytes, "the state read-back fits a pinned slot");


__device__ __forceinline__ bool halted(const PdState* st) { return *(volatile const int32_t*)&st->stop != 0; }

// ---- N1 (Newton step of pdNCG, Sec. 8.1): r = b - A x --------------------------------------------------------------------
template <class V, class Vec, class X, bool PAIRED>
__global__ void __launch_bounds__(kBlock) k_pd_resid(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                     const V* __restrict__ val, const X* __restrict__ x,
                                                     const Vec* __restrict__ b, Vec* __restrict__ r, int64_t m,
                                                     double* partials, PdState* st) {
    using Acc = Vec;
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    __shared__ double red[2 * 32];
    if (halted(st)) return;
    double p[2] = {0.0, 0.0};
    rows_of<PAIRED, V, X, Acc>(
        ptr, col, val, x, m, sm, &st->stage_err, [&](int64_t i, bool has) { return has ? b[i] : Vec(0); },
        [&](int64_t i, Acc u, const Vec& bb) {
            const Vec rr = bb - u;
            r[i] = rr;
            p[0] += (double)rr * (double)rr;
            p[1] += (double)bb * (double)rr;
        });
    block_reduce<kBlock, 2>(p, 0u, red);
    double tot[2];
    if (grid_reduce_last<kBlock, 2>(p, 0u, partials, &st->cnt[0], tot, red) && threadIdx.x == 0) {
        st->k1[0] = tot[0];
        st->k1[1] = tot[1];
    }
}

// Certificate at x from ||r||^2, b.r (st->k1) and tot = {max |A^T r|, ||x||_1}, the stop test
// and the mu-continuation (last CTA of N2, thread 0)
__device__ void pd_certify(PdState* st, const double (&tot)[2]) {
    const double tau = st->tau;
    const double P = __dadd_rn(__dmul_rn(tau, tot[1]), __dmul_rn(0.5, st->k1[0]));
    const double s = tot[0] <= tau ? 1.0 : tau / tot[0];
    const double D = __dadd_rn(__dmul_rn(s, st->k1[1]), -__dmul_rn(__dmul_rn(__dmul_rn(0.5, s), s), st->k1[0]));
    const double gap = P - D;
    const double rel = gap / fmax(fabs(P), 1e-300);
    st->P = P;
    st->D = D;
    st->gap = gap;
    st->rel = rel;
    st->products += 2;
    if (!isfinite(P) || !isfinite(D)) {
        st->status = L1LS_ENUMERIC;
        st->stop = 1;
    } else if (rel <= st->tol || P <= st->f_target) {
        st->status = L1LS_OK;
        st->stop = 1;
    } else if (st->iter >= st->max_newton) {
        st->status = L1LS_ENOCONV;
        st->stop = 1;
    } else {
        if (st->prev_full && st->mu > st->mu_target) st->mu = fmax(st->mu * 0.1, st->mu_target);
        else if (st->prev_full && gap > st->stall * st->prev_gap) st->mu = fmax(st->mu * 0.1, st->mu_min);
        st->prev_gap = gap;
    }
}

// ---- N2: a = A^T r, certificate ---------------------------------------------------------
template <class V, class Vec, bool PAIRED>
__global__ void __launch_bounds__(kBlock) k_pd_atr(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                   const V* __restrict__ val, const Vec* __restrict__ r,
                                                   const double* __restrict__ x, double* __restrict__ atr, int64_t n,
                                                   double* partials, PdState* st) {
    using Acc = Vec;
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    __shared__ double red[2 * 32];
    if (halted(st)) return;
    double p[2] = {0.0, 0.0};
    cols_of<PAIRED, V, Vec, Acc>(
        ptr, col, val, r, n, sm, &st->stage_err, [&](int64_t j, bool has) { return has ? x[j] : 0.0; },
        [&](int64_t j, Acc a, const double& xj) {
            atr[j] = (double)a;
            p[0] = fmax(p[0], fabs((double)a));
            p[1] += fabs(xj);
        });
    block_reduce<kBlock, 2>(p, 1u, red);
    double tot[2];
    if (grid_reduce_last<kBlock, 2>(p, 1u, partials, &st->cnt[1], tot, red) && threadIdx.x == 0) pd_certify(st, tot);
}

// ---- N1 / N2 with float-float products (accum = 1; FP32 / BF16 values) ----------------
// At large kappa the residual b - A x is a small difference of large terms (e reaches
// 1 / sigma_min) and FP32 sums of A^T r lose the gradient to rounding; as in FISTA's
// compensated kernels, x is gathered as a float-float pair, A x and the residual are kept in
// float-float (paired storage: one float4 {hi, hi, lo, lo} per row pair; plain: float2 per
// row) and A^T r is summed in float-float.  The high words of r also go to the FP32 residual
// that the line search reads.
template <class V, bool PAIRED>
__global__ void __launch_bounds__(kBlock) k_pd_resid_ff(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                        const V* __restrict__ val, const float* __restrict__ xh,
                                                        const float* __restrict__ xl, const float* __restrict__ b,
                                                        float* __restrict__ rff, float* __restrict__ r, int64_t m,
                                                        double* partials, PdState* st) {
    __shared__ typename std::conditional<PAIRED, PairedSmem<V, kBlock>, CompSmem<kBlock>>::type sm;
    __shared__ double red[2 * 32];
    if (halted(st)) return;
    ff q0 = {0.0f, 0.0f}, q1 = {0.0f, 0.0f};
    auto pre = [&](int64_t i, bool has) { return has ? b[i] : 0.0f; };
    auto epi = [&](int64_t i, ff u, const float& bb) {
        const ff rr = ff_sub(ff_from_float(bb), u);
        if (PAIRED) {
            rff[4 * (i >> 1) + (i & 1)] = rr.hi;
            rff[4 * (i >> 1) + 2 + (i & 1)] = rr.lo;
        } else {
            rff[2 * i] = rr.hi;
            rff[2 * i + 1] = rr.lo;
        }
        r[i] = rr.hi;
        sum2_add(q0, ff_mul(rr, rr));
        sum2_add(q1, ff_mul(ff_from_float(bb), rr));
    };
    const int64_t nrows = PAIRED ? m / 2 : m;
    if constexpr (PAIRED) {
        warp_pcsr<true, V>(ptr, col, val, nrows, sm, &st->stage_err, FFSum<true, V>{xh, xl, nullptr}, pre, epi);
    } else {
        const int64_t nw = (int64_t)gridDim.x * (kBlock / 32), ntiles = (nrows + 31) >> 5;
        for (int64_t t = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); t < ntiles; t += nw)
            tile_ff<true, false, V>(t, ptr, col, val, xh, xl, nullptr, nrows, sm.warp_buf(), pre, epi);
    }
    double p[2] = {ff_to_double(q0), ff_to_double(q1)};
    block_reduce<kBlock, 2>(p, 0u, red);
    double tot[2];
    if (grid_reduce_last<kBlock, 2>(p, 0u, partials, &st->cnt[0], tot, red) && threadIdx.x == 0) {
        st->k1[0] = tot[0];
        st->k1[1] = tot[1];
    }
}

template <class V, bool PAIRED>
__global__ void __launch_bounds__(kBlock) k_pd_atr_ff(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                      const V* __restrict__ val, const float* __restrict__ rff,
                                                      const double* __restrict__ x, double* __restrict__ atr,
                                                      int64_t n, double* partials, PdState* st) {
    __shared__ typename std::conditional<PAIRED, PairedSmem<V, kBlock>, CompSmem<kBlock>>::type sm;
    __shared__ double red[2 * 32];
    if (halted(st)) return;
    double p[2] = {0.0, 0.0};
    auto pre = [&](int64_t j, bool has) { return has ? x[j] : 0.0; };
    auto epi = [&](int64_t j, ff g, const double& xj) {
        const double a = ff_to_double(g);
        atr[j] = a;
        p[0] = fmax(p[0], fabs(a));
        p[1] += fabs(xj);
    };
    if constexpr (PAIRED) {
        warp_pcsr<false, V>(ptr, col, val, n, sm, &st->stage_err,
                            FFSum<false, V>{nullptr, nullptr, reinterpret_cast<const float4*>(rff)}, pre, epi);
    } else {
        const int64_t nw = (int64_t)gridDim.x * (kBlock / 32), ntiles = (n + 31) >> 5;
        for (int64_t t = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); t < ntiles; t += nw)
            tile_ff<false, false, V>(t, ptr, col, val, nullptr, nullptr, rff, n, sm.warp_buf(), pre, epi);
    }
    block_reduce<kBlock, 2>(p, 1u, red);
    double tot[2];
    if (grid_reduce_last<kBlock, 2>(p, 1u, partials, &st->cnt[1], tot, red) && threadIdx.x == 0) pd_certify(st, tot);
}

// x as a float-float pair for the compensated N1
__global__ void __launch_bounds__(kBlock) k_pd_split(const double* __restrict__ x, float* __restrict__ xh,
                                                     float* __restrict__ xl, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
        const ff v = ff_from_double(x[j]);
        xh[j] = v.hi;
        xl[j] = v.lo;
    }
}

// ---- N3: gradient, primal-dual curvature, preconditioner, PCG start --------------------
// the CG residual: FP64 with FP64 vectors, float-float pairs with FP32 vectors
template <class CV> struct CgRes { using type = double; };
template <> struct CgRes<float> { using type = float2; };

template <class CV>
__global__ void __launch_bounds__(kBlock) k_pd_init(const double* __restrict__ x, const double* __restrict__ atr,
                                                    const double* __restrict__ cn2,
                                                    double* __restrict__ grad, CV* __restrict__ hd,
                                                    CV* __restrict__ minv, typename CgRes<CV>::type* __restrict__ rcg,
                                                    CV* __restrict__ z, CV* __restrict__ d,
                                                    int64_t n, double* partials, PdState* st) {
    __shared__ double red[32];
    if (halted(st)) return;
    const double mu = st->mu, tau = st->tau, itau = 1.0 / tau;
    double q[1] = {0.0};
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
        const double xj = x[j], aj = atr[j];
        // one reciprocal square root instead of a square root and three divisions (FP64 pipe)
        const double iw = rsqrt(mu * mu + xj * xj);
        const double xw = xj * iw;
        const double gr = tau * xw - aj;
        const double gj = fmin(1.0, fmax(-1.0, aj * itau));
        const double h = tau * (1.0 - gj * xw) * iw;
        // the preconditioner needs only the precision of the CG vectors
        CV mi;
        if constexpr (sizeof(CV) == 8) mi = 1.0 / (h + cn2[j]);
        else mi = __frcp_rn((float)(h + cn2[j]));
        const double rc = -gr;
        const CV zj = (CV)((double)mi * rc);
        grad[j] = gr;
        hd[j] = (CV)h;
        minv[j] = mi;
        if constexpr (sizeof(CV) == 8) {
            rcg[j] = rc;
        } else {
            const ff r = ff_from_double(rc);
            rcg[j] = make_float2(r.hi, r.lo);
        }
        z[j] = zj;
        d[j] = CV(0);
        q[0] += rc * (double)zj;
    }
    block_reduce<kBlock, 1>(q, 0u, red);
    double tot[1];
    if (grid_reduce_last<kBlock, 1>(q, 0u, partials, &st->cnt[2], tot, red) && threadIdx.x == 0) {
        st->rz = tot[0];
        st->rz0 = tot[0];
        st->beta = 0.0;
        st->cg_done = 0;
        st->cg_it = 0;
    }
}

// ---- C1: Ap = A z + beta Ap, i.e. A p for p = z + beta p (also L1: Ad = A d with partials)
template <class V, class Vec, class X, bool LS, bool PAIRED>
__global__ void __launch_bounds__(kBlock) k_pd_ax(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                  const V* __restrict__ val, const X* __restrict__ x,
                                                  Vec* __restrict__ out, const Vec* __restrict__ r, int64_t m,
                                                  double* partials, PdState* st) {
    using Acc = Vec;
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    __shared__ double red[2 * 32];
    if (halted(st)) return;
    if (!LS && *(volatile int32_t*)&st->cg_done) return;
    // beta = 0 (first CG iteration): out holds no previous A p, and is not read
    const Vec beta = LS ? Vec(0) : (Vec)st->beta;
    double p[2] = {0.0, 0.0};
    rows_of<PAIRED, V, X, Acc>(
        ptr, col, val, x, m, sm, &st->stage_err,
        [&](int64_t i, bool has) { return !has ? Vec(0) : LS ? r[i] : (beta != Vec(0) ? out[i] : Vec(0)); },
        [&](int64_t i, Acc u, const Vec& ri) {
            if (LS) {
                out[i] = u;
                p[0] += (double)ri * (double)u;
                p[1] += (double)u * (double)u;
            } else {
                out[i] = beta != Vec(0) ? u + beta * ri : u;
            }
        });
    if (!LS) return;
    block_reduce<kBlock, 2>(p, 0u, red);
    double tot[2];
    if (grid_reduce_last<kBlock, 2>(p, 0u, partials, &st->cnt[3], tot, red) && threadIdx.x == 0) {
        st->rAd = tot[0];
        st->AdAd = tot[1];
        st->products += 1;
        st->ls_done = 0;
        st->ls_trial = 0;
        st->step = 1.0;
    }
}

// ---- C2 (PCG product, Sec. 8.1): p = z + beta p, Hp = h p + A^T Ap, alpha ---------------------------------------
template <class V, class Vec, bool PAIRED>
__global__ void __launch_bounds__(kBlock) k_pd_hp(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                  const V* __restrict__ val, const Vec* __restrict__ ap,
                                                  const Vec* __restrict__ hd, const Vec* __restrict__ z,
                                                  Vec* __restrict__ p, Vec* __restrict__ hp, int64_t n,
                                                  double* partials, PdState* st) {
    using Acc = Vec;
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    __shared__ double red[32];
    if (halted(st) || *(volatile int32_t*)&st->cg_done) return;
    const Vec beta = (Vec)st->beta;
    double q[1] = {0.0};
    ff qf = {0.0f, 0.0f};   // FP32 vectors: p.Hp summed in float-float (Sum2)
    struct Ops {
        Vec pj, h;
    };
    cols_of<PAIRED, V, Vec, Acc>(
        ptr, col, val, ap, n, sm, &st->stage_err,
        [&](int64_t j, bool has) {
            Ops o{Vec(0), Vec(0)};
            if (has) {
                o.pj = beta != Vec(0) ? z[j] + beta * p[j] : z[j];
                o.h = hd[j];
            }
            return o;
        },
        [&](int64_t j, Acc a, const Ops& o) {
            const Vec h = o.h * o.pj + a;
            p[j] = o.pj;
            hp[j] = h;
            if constexpr (sizeof(Vec) == 8) q[0] += o.pj * h;
            else sum2_add(qf, two_prod(o.pj, h));
        });
    if constexpr (sizeof(Vec) == 4) q[0] = ff_to_double(qf);
    block_reduce<kBlock, 1>(q, 0u, red);
    double tot[1];
    if (grid_reduce_last<kBlock, 1>(q, 0u, partials, &st->cnt[4], tot, red) && threadIdx.x == 0) {
        st->products += 2;
        st->cg_total += 1;
        if (tot[0] <= 0.0) {
            st->cg_done = 1;
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / tot[0];
        }
    }
}

// ---- C3: d += alpha p, res -= alpha Hp, z = M^{-1} res ---------------------------------
template <class CV>
__global__ void __launch_bounds__(kBlock) k_pd_cgupd(CV* __restrict__ d, typename CgRes<CV>::type* __restrict__ rcg,
                                                     const CV* p0, const CV* p1, const CV* __restrict__ hp,
                                                     const CV* __restrict__ minv, CV* __restrict__ z, int64_t n,
                                                     double* partials, PdState* st) {
    __shared__ double red[2 * 32];
    if (halted(st) || *(volatile int32_t*)&st->cg_done) return;
    // p1 non-NULL: the search direction alternates between p0 and p1 by the CG iteration's parity
    const CV* __restrict__ p = (p1 && (st->cg_it & 1)) ? p1 : p0;
    double q[2] = {0.0, 0.0};
    if constexpr (sizeof(CV) == 8) {
        const double alpha = st->alpha;
        for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
            const double pj = p[j];
            d[j] += alpha * pj;
            const double rc = rcg[j] - alpha * hp[j];
            rcg[j] = rc;
            const double zj = minv[j] * rc;
            z[j] = zj;
            q[1] += rc * zj;
        }
    } else {
        // alpha as float-float; res -= alpha Hp and res.z in float-float on the FP32 pipes
        const ff alpha = ff_from_double(st->alpha);
        ff rz = {0.0f, 0.0f};
        for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
            const float pj = p[j], hj = hp[j];
            d[j] = __fmaf_rn(alpha.hi, pj, d[j]);
            const float2 r2 = rcg[j];
            ff ah = two_prod(alpha.hi, hj);
            ah.lo = __fmaf_rn(alpha.lo, hj, ah.lo);
            const ff r = ff_sub(ff{r2.x, r2.y}, ah);
            rcg[j] = make_float2(r.hi, r.lo);
            const float zj = minv[j] * r.hi;
            z[j] = zj;
            ff t = two_prod(r.hi, zj);
            t.lo = __fmaf_rn(r.lo, zj, t.lo);
            sum2_add(rz, t);
        }
        q[1] = ff_to_double(rz);
    }
    block_reduce<kBlock, 2>(q, 0u, red);
    double tot[2];
    if (grid_reduce_last<kBlock, 2>(q, 0u, partials, &st->cnt[5], tot, red) && threadIdx.x == 0) {
        st->cg_it += 1;
        // relative residual in the preconditioner's norm: sqrt(res.M^-1 res) vs sqrt(grad.M^-1 grad)
        if (sqrt(tot[1]) <= st->pcg_rtol * sqrt(st->rz0) || st->cg_it >= st->pcg_max) {
            st->cg_done = 1;
        } else {
            st->beta = tot[1] / st->rz;
            st->rz = tot[1];
        }
    }
}

// ---- LT: Armijo trials on f_tau^mu of Eq. (prob2) -------------------------------------------------------------------
// NT trials per pass: the first pass tries the full step alone (most Newton steps take it),
// later passes four halvings each; every trial costs a square root and a division per entry
// on the FP64 pipe
template <class CV, int NT>
__global__ void __launch_bounds__(kBlock) k_pd_trial(const double* __restrict__ x, const CV* __restrict__ d,
                                                     const double* __restrict__ grad, int64_t n, double* partials,
                                                     PdState* st) {
    constexpr int kTrialsPerPass = NT;
    __shared__ double red[(kTrialsPerPass + 1) * 32];
    if (halted(st) || *(volatile int32_t*)&st->ls_done) return;
    const double mu = st->mu, step0 = st->step;
    double q[kTrialsPerPass + 1];
#pragma unroll
    for (int t = 0; t <= kTrialsPerPass; ++t) q[t] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
        const double xj = x[j], dj = (double)d[j];
        const double w0 = sqrt(mu * mu + xj * xj);
        double a = step0;
#pragma unroll
        for (int t = 0; t < kTrialsPerPass; ++t) {
            const double xt = xj + a * dj;
            q[t] += (a * dj) * (xj + xt) / (sqrt(mu * mu + xt * xt) + w0);
            a *= 0.5;
        }
        q[kTrialsPerPass] += grad[j] * dj;
    }
    block_reduce<kBlock, kTrialsPerPass + 1>(q, 0u, red);
    double tot[kTrialsPerPass + 1];
    if (grid_reduce_last<kBlock, kTrialsPerPass + 1>(q, 0u, partials, &st->cnt[6], tot, red) && threadIdx.x == 0) {
        const double slope = tot[kTrialsPerPass];
        double a = step0;
        for (int t = 0; t < kTrialsPerPass; ++t) {
            const int64_t trial = st->ls_trial + t;
            const double df = st->tau * tot[t] - a * st->rAd + 0.5 * a * a * st->AdAd;
            if (df <= st->armijo * a * slope || trial >= st->ls_max - 1) {
                st->step = a;
                st->ls_done = 1;
                st->ls_total += trial + 1;
                return;
            }
            a *= 0.5;
        }
        st->step = a;
        st->ls_trial += kTrialsPerPass;
    }
}

// The same trials for FP32 CG vectors, in float-float on the FP32 pipes: x as its (hi, lo)
// pair, each per-coordinate difference with Dekker's double-word square root and quotient
// (relative error a few units of 2^-46, against 2^-53 in FP64; the Armijo test compares sums of
// these terms with c a slope, far above that error), so a trial costs FP32 operations
// instead of an FP64 square root and division per entry.  The trial steps are powers of two,
// so a d_j is exact in FP32.  Entries beyond the FP32 range (|x| or |x + a d| >= 1e18) take the
// FP64 formula.  The slope grad.d is summed in the first pass only.
template <int NT>
__global__ void __launch_bounds__(kBlock) k_pd_trial_ff(const float* __restrict__ xh, const float* __restrict__ xl,
                                                        const float* __restrict__ d, const double* __restrict__ grad,
                                                        int64_t n, double* partials, PdState* st) {
    __shared__ double red[(NT + 1) * 32];
    if (halted(st) || *(volatile int32_t*)&st->ls_done) return;
    const double mu = st->mu, step0 = st->step;
    const bool first = st->ls_trial == 0;
    const ff mu2 = ff_from_double(mu * mu);
    ff q[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) q[t] = {0.0f, 0.0f};
    double slope = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
        const ff x = {xh[j], xl[j]};
        const float dj = d[j];
        if (first) slope += grad[j] * (double)dj;
        const ff w0 = ff_sqrt(ff_add(mu2, ff_mul(x, x)));
        float a = (float)step0;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const float ad = a * dj;
            const ff xt = ff_add(x, ff_from_float(ad));
            ff term;
            if (fabsf(x.hi) < 1e18f && fabsf(xt.hi) < 1e18f) {
                const ff den = ff_add(ff_sqrt(ff_add(mu2, ff_mul(xt, xt))), w0);
                const ff s2 = ff_add(x, xt);
                ff num = two_prod(s2.hi, ad);
                num.lo = __fmaf_rn(s2.lo, ad, num.lo);
                term = den.hi > 0.0f ? ff_div(num, den) : ff{0.0f, 0.0f};
            } else {
                const double xd = ff_to_double(x), xtd = xd + (double)ad;
                term = ff_from_double((double)ad * (xd + xtd) / (sqrt(mu * mu + xtd * xtd) + sqrt(mu * mu + xd * xd)));
            }
            sum2_add(q[t], term);
            a *= 0.5f;
        }
    }
    double p[NT + 1];
#pragma unroll
    for (int t = 0; t < NT; ++t) p[t] = ff_to_double(q[t]);
    p[NT] = slope;
    block_reduce<kBlock, NT + 1>(p, 0u, red);
    double tot[NT + 1];
    if (grid_reduce_last<kBlock, NT + 1>(p, 0u, partials, &st->cnt[6], tot, red) && threadIdx.x == 0) {
        if (first) st->slope = tot[NT];
        const double sl = st->slope;
        double a = step0;
        for (int t = 0; t < NT; ++t) {
            const int64_t trial = st->ls_trial + t;
            const double df = st->tau * tot[t] - a * st->rAd + 0.5 * a * a * st->AdAd;
            if (df <= st->armijo * a * sl || trial >= st->ls_max - 1) {
                st->step = a;
                st->ls_done = 1;
                st->ls_total += trial + 1;
                return;
            }
            a *= 0.5;
        }
        st->step = a;
        st->ls_trial += NT;
    }
}

// ---- L3: x += step d (the dual estimate is recomputed from A^T r at the next N3) ----------
template <class CV>
__global__ void __launch_bounds__(kBlock) k_pd_apply(double* __restrict__ x, const CV* __restrict__ d, int64_t n,
                                                     float* __restrict__ xh, float* __restrict__ xl, PdState* st) {
    if (halted(st)) return;
    const double step = st->step;
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < n; j += (int64_t)gridDim.x * kBlock) {
        const double v = x[j] + step * (double)d[j];
        x[j] = v;
        if (xh) {   // the float-float copy that the compensated N1 gathers and the trials read
            const ff f = ff_from_double(v);
            xh[j] = f.hi;
            xl[j] = f.lo;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->prev_full = step == 1.0 ? 1 : 0;
        st->iter += 1;
    }
}

// ---- matrix-free pdNCG (instances generated with matrix_free = 1) ---------------------------
// A = L Sigma R^T with L orthogonal (the permutation and the left rotations, Eq. bd8), so
// A^T A = R Sigma^2 R^T: the Hessian's product needs the stages of R and Sigma only, and the
// left factor enters the gradient through c = A^T b alone, computed once per instance.  With
// u = Sigma R^T x:  A^T r = c - R Sigma u,  ||r||^2 = ||b||^2 - 2 c.x + ||u||^2,  b.r = ||b||^2
// - c.x (||A x|| = ||u||);  in the line search r.(A d) = (A^T r).d and ||A d|| = ||Sigma R^T d||.
// Every pass is a sweep over tiles of kMfTile entries with a halo of 2 kMfHalo (R^T then R,
// each widening the dependence by w <= kMfHalo entries); no m-vector is kept.  The gradient
// and the certificate run in FP64 once per Newton step; the PCG product and the line search's
// ||A d|| run in FP32 like the stored-matrix path with FP32 values.
constexpr int kPdHalo = 2 * kMfHalo;
constexpr int kPdLen = kMfTile + 2 * kPdHalo;
constexpr int kPdPer = (kPdLen + kMfThreads - 1) / kMfThreads;

struct MfPd {
    int64_t n;
    int w;
    float c, s;          // right angle (FP32: the PCG product)
    double c64, s64;     // (FP64: gradient, line search, diagonal, A^T b)
    const float* sigma32;
    const double* sigma;
};

// buf[p] = v[g0 + p] for the tile's buffer (0 outside [0, n))
template <class T, class S>
__device__ __forceinline__ void mfpd_load(T* buf, const S* __restrict__ v, int64_t g0, int64_t n) {
#pragma unroll
    for (int u = 0; u < kPdPer; ++u) {
        const int p = (int)threadIdx.x + u * kMfThreads;
        const int64_t i = g0 + p;
        if (p < kPdLen) buf[p] = (i >= 0 && i < n) ? (T)v[i] : T(0);
    }
    __syncthreads();
}

// buf[p] *= sigma[g0 + p]^POW
template <int POW, class T>
__device__ __forceinline__ void mfpd_scale(T* buf, const T* __restrict__ sigma, int64_t g0, int64_t n) {
#pragma unroll
    for (int u = 0; u < kPdPer; ++u) {
        const int p = (int)threadIdx.x + u * kMfThreads;
        const int64_t i = g0 + p;
        if (p < kPdLen && i >= 0 && i < n) {
            const T sg = sigma[i];
            buf[p] *= POW == 2 ? sg * sg : sg;
        }
    }
    __syncthreads();
}

// N1 + N2: A^T r at x (FP64), partials max |A^T r|, ||x||_1, c.x, ||u||^2; last CTA: the
// certificate (pd_certify) from ||r||^2 and b.r formed as above (st->bb = ||b||^2)
__global__ void __launch_bounds__(kMfThreads) k_mfpd_grad(MfPd P, const double* __restrict__ x,
                                                          const double* __restrict__ c, double* __restrict__ atr,
                                                          double* partials, PdState* st) {
    __shared__ double buf[kPdLen];
    __shared__ double red[4 * 32];
    if (halted(st)) return;
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t ntiles = (P.n + kMfTile - 1) / kMfTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t a0 = tile * kMfTile, g0 = a0 - kPdHalo;
        mfpd_load(buf, x, g0, P.n);
        mf_stages_t<true, double, kPdLen>(buf, g0, P.n, P.w, P.c64, P.s64);
#pragma unroll
        for (int u = 0; u < kPdPer; ++u) {   // u = Sigma R^T x; ||u||^2 over the tile's own entries
            const int p = (int)threadIdx.x + u * kMfThreads;
            const int64_t i = g0 + p;
            if (p < kPdLen && i >= 0 && i < P.n) {
                const double sg = P.sigma[i];
                const double uv = buf[p] * sg;
                if (p >= kPdHalo && p < kPdHalo + kMfTile) q[3] += uv * uv;
                buf[p] = uv * sg;
            }
        }
        __syncthreads();
        mf_stages_t<false, double, kPdLen>(buf, g0, P.n, P.w, P.c64, P.s64);
        for (int p = kPdHalo + (int)threadIdx.x; p < kPdHalo + kMfTile; p += kMfThreads) {
            const int64_t j = g0 + p;
            if (j >= P.n) break;
            const double cj = c[j], xj = x[j];
            const double a = cj - buf[p];
            atr[j] = a;
            q[0] = fmax(q[0], fabs(a));
            q[1] += fabs(xj);
            q[2] += cj * xj;
        }
        __syncthreads();   // the buffer is reloaded next
    }
    block_reduce<kMfThreads, 4>(q, 1u, red);
    double tot[4];
    if (grid_reduce_last<kMfThreads, 4>(q, 1u, partials, &st->cnt[1], tot, red) && threadIdx.x == 0) {
        st->k1[0] = st->bb - 2.0 * tot[2] + tot[3];   // ||b - A x||^2
        st->k1[1] = st->bb - tot[2];                  // b.(b - A x)
        const double t2[2] = {tot[0], tot[1]};
        pd_certify(st, t2);
    }
}

// C2 of the PCG iteration: p = z + beta p_old, Hp = h p + R Sigma^2 R^T p, alpha = rz / p.Hp
// (FP32; p alternates between two buffers by the parity of the CG iteration, since the tiles
// read their neighbours' p_old in the halo)
__global__ void __launch_bounds__(kMfThreads) k_mfpd_hp(MfPd P, const float* __restrict__ z, float* p0, float* p1,
                                                        const float* __restrict__ hd, float* __restrict__ hp,
                                                        double* partials, PdState* st) {
    __shared__ float buf[kPdLen];
    __shared__ double red[32];
    if (halted(st) || *(volatile int32_t*)&st->cg_done) return;
    const bool odd = (st->cg_it & 1) != 0;
    const float* pold = odd ? p0 : p1;
    float* pnew = odd ? p1 : p0;
    const float beta = (float)st->beta;
    ff qf = {0.0f, 0.0f};
    const int64_t ntiles = (P.n + kMfTile - 1) / kMfTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t a0 = tile * kMfTile, g0 = a0 - kPdHalo;
        float pv[kPdPer], hv[kPdPer];
#pragma unroll
        for (int u = 0; u < kPdPer; ++u) {
            const int p = (int)threadIdx.x + u * kMfThreads;
            const int64_t i = g0 + p;
            float v = 0.0f, h = 0.0f;
            if (p < kPdLen && i >= 0 && i < P.n) {
                v = z[i];
                if (beta != 0.0f) v = __fmaf_rn(beta, pold[i], v);
                if (p >= kPdHalo && p < kPdHalo + kMfTile) h = hd[i];
            }
            pv[u] = v;
            hv[u] = h;
            if (p < kPdLen) buf[p] = v;
        }
        __syncthreads();
        mf_stages_t<true, float, kPdLen>(buf, g0, P.n, P.w, P.c, P.s);
        mfpd_scale<2>(buf, P.sigma32, g0, P.n);
        mf_stages_t<false, float, kPdLen>(buf, g0, P.n, P.w, P.c, P.s);
#pragma unroll
        for (int u = 0; u < kPdPer; ++u) {
            const int p = (int)threadIdx.x + u * kMfThreads;
            const int64_t j = g0 + p;
            if (p < kPdHalo || p >= kPdHalo + kMfTile || j >= P.n) continue;
            const float h = __fmaf_rn(hv[u], pv[u], buf[p]);
            pnew[j] = pv[u];
            hp[j] = h;
            sum2_add(qf, two_prod(pv[u], h));
        }
        __syncthreads();
    }
    double q[1] = {ff_to_double(qf)};
    block_reduce<kMfThreads, 1>(q, 0u, red);
    double tot[1];
    if (grid_reduce_last<kMfThreads, 1>(q, 0u, partials, &st->cnt[4], tot, red) && threadIdx.x == 0) {
        st->products += 2;
        st->cg_total += 1;
        if (tot[0] <= 0.0) {
            st->cg_done = 1;
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / tot[0];
        }
    }
}

// L1: the line search's r.(A d) = (A^T r).d (FP64) and ||A d||^2 = ||Sigma R^T d||^2 (an FP32
// sweep like the stored path's FP32 A d, its squares summed in float-float: the Armijo test
// needs ||A d||^2 to a relative 1e-7 at most, since it weighs against armijo * slope)
__global__ void __launch_bounds__(kMfThreads) k_mfpd_ls(MfPd P, const float* __restrict__ d,
                                                        const double* __restrict__ atr, double* partials,
                                                        PdState* st) {
    __shared__ float buf[kPdLen];
    __shared__ double red[2 * 32];
    if (halted(st)) return;
    double q[2] = {0.0, 0.0};
    ff vv = {0.0f, 0.0f};
    const int64_t ntiles = (P.n + kMfTile - 1) / kMfTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t a0 = tile * kMfTile, g0 = a0 - kPdHalo;
        mfpd_load(buf, d, g0, P.n);
        mf_stages_t<true, float, kPdLen>(buf, g0, P.n, P.w, P.c, P.s);
        for (int p = kPdHalo + (int)threadIdx.x; p < kPdHalo + kMfTile; p += kMfThreads) {
            const int64_t j = g0 + p;
            if (j >= P.n) break;
            const float v = buf[p] * P.sigma32[j];
            q[0] += atr[j] * (double)d[j];
            sum2_add(vv, two_prod(v, v));
        }
        __syncthreads();
    }
    q[1] = ff_to_double(vv);
    block_reduce<kMfThreads, 2>(q, 0u, red);
    double tot[2];
    if (grid_reduce_last<kMfThreads, 2>(q, 0u, partials, &st->cnt[3], tot, red) && threadIdx.x == 0) {
        st->rAd = tot[0];
        st->AdAd = tot[1];
        st->products += 1;
        st->ls_done = 0;
        st->ls_trial = 0;
        st->step = 1.0;
    }
}

// diag(A^T A) = diag(R Sigma^2 R^T) by probing (FP64): R has half-bandwidth w, so R Sigma^2 R^T
// has at most 2w, and with K = 2w + 1 the product with the indicator of {i = q mod K} equals
// the diagonal on those i.  Once per instance.
__global__ void __launch_bounds__(kMfThreads) k_mfpd_diag(MfPd P, double* __restrict__ cn2) {
    __shared__ double buf[kPdLen];
    const int K = 2 * P.w + 1;
    const int64_t ntiles = (P.n + kMfTile - 1) / kMfTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t a0 = tile * kMfTile, g0 = a0 - kPdHalo;
        for (int q = 0; q < K; ++q) {
            for (int p = threadIdx.x; p < kPdLen; p += kMfThreads) {
                const int64_t i = g0 + p;
                buf[p] = (i >= 0 && i < P.n && (int)(i % K) == q) ? 1.0 : 0.0;
            }
            __syncthreads();
            mf_stages_t<true, double, kPdLen>(buf, g0, P.n, P.w, P.c64, P.s64);
            mfpd_scale<2>(buf, P.sigma, g0, P.n);
            mf_stages_t<false, double, kPdLen>(buf, g0, P.n, P.w, P.c64, P.s64);
            for (int p = kPdHalo + (int)threadIdx.x; p < kPdHalo + kMfTile; p += kMfThreads) {
                const int64_t j = g0 + p;
                if (j < P.n && (int)(j % K) == q) cn2[j] = buf[p];
            }
            __syncthreads();
        }
    }
}

// A^T b in FP64 (once per instance): zs = the first n entries of P2^T G~^T b (b in the stored
// row order), then c = R Sigma zs
__global__ void k_mfpd_scatter(MfLeft L, double ct, double stt, const double* __restrict__ b, double* __restrict__ zs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L.left == 0) {
        if (t < L.n) zs[t] = b[t];
        return;
    }
    if (t >= L.m / 2) return;
    const int32_t kx = L.perm[2 * t], ky = L.perm[2 * t + 1];
    const double y0 = b[2 * t], y1 = b[2 * t + 1];
    if (kx < L.n) zs[kx] = fma(ct, y0, stt * y1);
    if (ky < L.n) zs[ky] = fma(ct, y1, -stt * y0);
}

__global__ void __launch_bounds__(kMfThreads) k_mfpd_rsig(MfPd P, const double* __restrict__ zs, double* __restrict__ c) {
    __shared__ double buf[kPdLen];
    const int64_t ntiles = (P.n + kMfTile - 1) / kMfTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t a0 = tile * kMfTile, g0 = a0 - kPdHalo;
        mfpd_load(buf, zs, g0, P.n);
        mfpd_scale<1>(buf, P.sigma, g0, P.n);
        mf_stages_t<false, double, kPdLen>(buf, g0, P.n, P.w, P.c64, P.s64);
        for (int p = kPdHalo + (int)threadIdx.x; p < kPdHalo + kMfTile; p += kMfThreads) {
            const int64_t j = g0 + p;
            if (j < P.n) c[j] = buf[p];
        }
        __syncthreads();
    }
}

// ||b||^2 into the state (FP64; once per solve, after the state is uploaded)
__global__ void __launch_bounds__(kBlock) k_mfpd_bb(const double* __restrict__ b, int64_t m, double* partials,
                                                    PdState* st) {
    __shared__ double red[32];
    double q[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < m; i += (int64_t)gridDim.x * kBlock) q[0] += b[i] * b[i];
    block_reduce<kBlock, 1>(q, 0u, red);
    double tot[1];
    if (grid_reduce_last<kBlock, 1>(q, 0u, partials, &st->cnt[7], tot, red) && threadIdx.x == 0) st->bb = tot[0];
}

template <class K>
int grid_for(const Inst* I, K kernel, int64_t rows) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = (rows + 31) / 32 / (kBlock / 32) + 1;   // blocks with one warp tile per warp
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)I->ctx->num_sms * per_sm));
}

struct PdWork {
    double *X = nullptr, *atr = nullptr, *grad = nullptr;
    void *hd = nullptr, *minv = nullptr, *z = nullptr, *p = nullptr, *hp = nullptr, *d = nullptr;   // CG vectors
    void* rcg = nullptr;   // CG residual (CgRes)
    void *r = nullptr, *ap = nullptr, *ad = nullptr;
    float *xh = nullptr, *xl = nullptr, *rff = nullptr;   // compensated N1 / N2 (accum = 1)
    double *cn2 = nullptr, *atb = nullptr;   // matrix-free: diag(A^T A), A^T b
    void* p2 = nullptr;                      // matrix-free: the second search-direction buffer
    double* part = nullptr;
    PdState* st = nullptr;
    PdState* host = nullptr;
    int gm = 0, gn = 0, gv = 0, gmf = 0, gnf = 0;
    cudaGraphExec_t cg_exec = nullptr;
    int cg_chunk = 0;
    Ctx* pin_ctx = nullptr;   // host is a pinned slot of this context (else pageable)
    ~PdWork() {
        if (cg_exec) cudaGraphExecDestroy(cg_exec);
        if (pin_ctx) pin_ctx->pinned_put(host);
        else delete host;
    }
};

// the result of a solve (both loops): the iterate, the result record and the status
l1ls_status pd_finish(Inst* I, PdWork* w, l1ls_status final_status, double* x_out, l1ls_result* res,
                      std::chrono::steady_clock::time_point t0, cudaStream_t s) {
    const int64_t n = I->n;
    const PdState& f = *w->host;
    if (f.stage_err && final_status == L1LS_OK)
        final_status = set_error(L1LS_ECUDA, "a bulk-copy stage wait ran out of polls (sums read directly)");
    if (x_out) L1LS_CUDA(cudaMemcpyAsync(x_out, w->X, sizeof(double) * n, cudaMemcpyDefault, s));
    L1LS_CUDA(cudaStreamSynchronize(s));
    if (res) {
        memset(res, 0, sizeof(*res));
        res->iters = f.iter;
        res->products = f.products;
        res->cg_iters = f.cg_total;
        res->ls_trials = f.ls_total;
        res->f = f.P;
        res->dual = f.D;
        res->gap = f.gap;
        res->rel_gap = f.rel;
        res->mu = f.mu;
        res->status = final_status;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (final_status != L1LS_OK) {
        const char* why = final_status == L1LS_ENOCONV ? "Newton iteration limit reached"
                          : final_status == L1LS_ETIMEOUT ? "time limit reached"
                          : final_status == L1LS_ECANCELLED ? "cancelled"
                                                          : "NaN or Inf in the iteration";
        return set_error(final_status, "pdNCG: %s (rel_gap %.3e)", why, f.rel);
    }
    return L1LS_OK;
}

// row and column orientation of the stored matrix (plain or paired)
template <class V, bool PAIRED>
void views(const Inst* I, Csr<V>& rows, Csr<V>& cols) {
    if (PAIRED) {
        rows = {I->prow_ptr, I->prow_col, static_cast<const V*>(I->prow_val)};
        cols = {I->pcol_ptr, I->pcol_pair, static_cast<const V*>(I->pcol_val)};
    } else {
        rows = {I->csr_ptr, I->csr_col, static_cast<const V*>(I->csr_val)};
        cols = {I->csc_ptr, I->csc_row, static_cast<const V*>(I->csc_val)};
    }
}

template <class V, class Vec, bool PAIRED>
void enqueue_cg(Inst* I, PdWork* w, cudaStream_t s) {
    Csr<V> R, C;
    views<V, PAIRED>(I, R, C);
    k_pd_ax<V, Vec, Vec, false, PAIRED><<<w->gm, kBlock, 0, s>>>(R.ptr, R.idx, R.val, (const Vec*)w->z, (Vec*)w->ap,
                                                                 nullptr, I->m, w->part, w->st);
    k_pd_hp<V, Vec, PAIRED><<<w->gn, kBlock, 0, s>>>(C.ptr, C.idx, C.val, (const Vec*)w->ap, (const Vec*)w->hd,
                                                     (const Vec*)w->z, (Vec*)w->p, (Vec*)w->hp, I->n, w->part, w->st);
    k_pd_cgupd<Vec><<<w->gv, kBlock, 0, s>>>((Vec*)w->d, (typename CgRes<Vec>::type*)w->rcg, (const Vec*)w->p, nullptr,
                                             (const Vec*)w->hp,
                                             (const Vec*)w->minv, (Vec*)w->z, I->n, w->part, w->st);
}

template <class V, class Vec, bool PAIRED>
l1ls_status run(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res, cudaStream_t s) {
    Csr<V> R, C;
    views<V, PAIRED>(I, R, C);
    auto t0 = std::chrono::steady_clock::now();
    const int64_t m = I->m, n = I->n;
    PdWork* w = static_cast<PdWork*>(I->pd_work);
    if (!w) {
        // attached to the instance only once complete (a failed allocation leaves none behind)
        std::unique_ptr<PdWork> fresh(new PdWork());
        w = fresh.get();
        for (double** v : {&w->X, &w->atr, &w->grad}) L1LS_TRY(I->alloc_n(v, n));
        L1LS_TRY(I->alloc(&w->rcg, sizeof(typename CgRes<Vec>::type) * pad32(n)));
        for (void** v : {&w->hd, &w->minv, &w->z, &w->p, &w->hp, &w->d}) L1LS_TRY(I->alloc(v, sizeof(Vec) * pad32(n)));
        L1LS_TRY(I->alloc(&w->r, sizeof(Vec) * pad32(m)));
        L1LS_TRY(I->alloc(&w->ap, sizeof(Vec) * pad32(m)));
        L1LS_TRY(I->alloc(&w->ad, sizeof(Vec) * pad32(m)));
        // N1 gathers x in the product precision: the FP64 iterate, or with FP32 CG vectors
        // its FP32 rounding, the high word of the float-float copy (the same values the
        // FP32 sums would convert it to, at half the gathered bytes)
        w->gm = grid_for(I, k_pd_resid<V, Vec, Vec, PAIRED>, PAIRED ? m / 2 : m);
        w->gn = grid_for(I, k_pd_atr<V, Vec, PAIRED>, n);
        w->gv = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)I->ctx->num_sms * 8));
        int gmax = std::max(w->gm, std::max(w->gn, w->gv));
        if constexpr (sizeof(Vec) == 4) {
            w->gmf = grid_for(I, k_pd_resid_ff<V, PAIRED>, PAIRED ? m / 2 : m);
            w->gnf = grid_for(I, k_pd_atr_ff<V, PAIRED>, n);
            gmax = std::max(gmax, std::max(w->gmf, w->gnf));
        }
        L1LS_TRY(I->alloc_n(&w->part, (int64_t)gmax * (kTrialsPerPass + 1)));
        L1LS_TRY(I->alloc_n(&w->st, 1));
        // the state read back every Newton step: a pinned slot of the context, else pageable
        if (void* slot = I->ctx->pinned_get(sizeof(PdState))) {
            w->host = new (slot) PdState();
            w->pin_ctx = I->ctx;
        } else {
            w->host = new PdState();
        }
        I->pd_work = fresh.release();
        I->pd_work_free = [](void* q) { delete static_cast<PdWork*>(q); };
    }
    if (x0) L1LS_CUDA(cudaMemcpyAsync(w->X, x0, sizeof(double) * n, cudaMemcpyDefault, s));
    else L1LS_CUDA(cudaMemsetAsync(w->X, 0, sizeof(double) * n, s));
    // accum = 1 with FP32 / BF16 values: the gradient's products N1 / N2 in float-float.  With
    // FP32 CG vectors the iterate is also kept as a float-float pair for the line search.
    const bool comp = sizeof(Vec) == 4 && o->accum == 1;
    if constexpr (sizeof(Vec) == 4) {
        if (!w->xl) {   // xl last: set only when both exist
            if (!w->xh) L1LS_TRY(I->alloc_n(&w->xh, pad32(n)));
            L1LS_TRY(I->alloc_n(&w->xl, pad32(n)));
        }
        if (comp && !w->rff) L1LS_TRY(I->alloc_n(&w->rff, 2 * pad32(m)));
        k_pd_split<<<w->gv, kBlock, 0, s>>>(w->X, w->xh, w->xl, n);
        L1LS_CUDA(cudaGetLastError());
    }
    PdState h;
    memset(&h, 0, sizeof(h));
    h.tau = o->tau;
    h.tol = o->rel_gap_tol;
    h.f_target = o->f_target;
    h.mu = o->mu_start > o->mu ? o->mu_start : o->mu;
    h.mu_target = o->mu;
    h.mu_min = o->mu_min;
    h.pcg_rtol = o->pcg_rtol;
    h.armijo = o->armijo;
    h.stall = 0.5;
    h.max_newton = o->max_iter;
    h.pcg_max = o->pcg_max;
    h.ls_max = o->ls_max;
    h.prev_gap = INFINITY;
    *w->host = h;
    L1LS_CUDA(cudaMemcpyAsync(w->st, w->host, sizeof(PdState), cudaMemcpyHostToDevice, s));
    const Vec* bvec = sizeof(Vec) == 8 ? (const Vec*)I->bhat : (const Vec*)I->bhat32;
    l1ls_status final_status = L1LS_OK;
    int chunk = o->check_every > 0 ? std::min(o->check_every, 16) : 8;
    if (!w->cg_exec || w->cg_chunk != chunk) {
        if (w->cg_exec) {
            cudaGraphExecDestroy(w->cg_exec);
            w->cg_exec = nullptr;
        }
        cudaStream_t cap;
        L1LS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        L1LS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < chunk; ++i) enqueue_cg<V, Vec, PAIRED>(I, w, cap);
        cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        if (ce != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
        }
        L1LS_CUDA(cudaGraphInstantiate(&w->cg_exec, graph, 0));
        cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        w->cg_chunk = chunk;
    }
    const int ls_passes = (o->ls_max - 1 + kTrialsPerPass - 1) / kTrialsPerPass;   // after the full-step pass
    for (;;) {
        // N1 gathers the iterate (FP64, or its FP32 word with FP32 CG vectors), or its float-float copy
        if constexpr (sizeof(Vec) == 4) {
            if (comp) {
                k_pd_resid_ff<V, PAIRED><<<w->gmf, kBlock, 0, s>>>(R.ptr, R.idx, R.val, w->xh, w->xl, I->bhat32, w->rff,
                                                                   (float*)w->r, m, w->part, w->st);
                k_pd_atr_ff<V, PAIRED><<<w->gnf, kBlock, 0, s>>>(C.ptr, C.idx, C.val, w->rff, w->X, w->atr, n, w->part,
                                                                 w->st);
            }
        }
        if (!comp) {
            const Vec* xg = sizeof(Vec) == 8 ? (const Vec*)w->X : (const Vec*)w->xh;
            k_pd_resid<V, Vec, Vec, PAIRED><<<w->gm, kBlock, 0, s>>>(R.ptr, R.idx, R.val, xg, bvec, (Vec*)w->r, m,
                                                                     w->part, w->st);
            k_pd_atr<V, Vec, PAIRED><<<w->gn, kBlock, 0, s>>>(C.ptr, C.idx, C.val, (const Vec*)w->r, w->X, w->atr, n,
                                                              w->part, w->st);
        }
        L1LS_CUDA(cudaGetLastError());
        L1LS_CUDA(cudaMemcpyAsync(w->host, w->st, sizeof(PdState), cudaMemcpyDeviceToHost, s));
        L1LS_CUDA(cudaStreamSynchronize(s));
        if (w->host->stop) {
            final_status = (l1ls_status)w->host->status;
            break;
        }
        if (o->time_limit_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->time_limit_s) {
            final_status = L1LS_ETIMEOUT;
            break;
        }
        if (cancel_requested()) {
            final_status = L1LS_ECANCELLED;
            break;
        }
        k_pd_init<Vec><<<w->gv, kBlock, 0, s>>>(w->X, w->atr, I->colnorm2, w->grad, (Vec*)w->hd, (Vec*)w->minv,
                                                (typename CgRes<Vec>::type*)w->rcg, (Vec*)w->z, (Vec*)w->d, n,
                                                w->part, w->st);
        L1LS_CUDA(cudaGetLastError());
        const int64_t max_cg_launches = o->pcg_max / chunk + 3;
        for (int64_t launch = 0;; ++launch) {
            if (launch >= max_cg_launches) {
                final_status = set_error(L1LS_ECUDA, "internal: PCG did not raise its stop flag");
                break;
            }
            L1LS_CUDA(cudaGraphLaunch(w->cg_exec, s));
            L1LS_CUDA(cudaMemcpyAsync(&w->host->cg_done, &w->st->cg_done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            L1LS_CUDA(cudaStreamSynchronize(s));
            if (w->host->cg_done) break;
        }
        if (final_status != L1LS_OK) break;
        k_pd_ax<V, Vec, Vec, true, PAIRED><<<w->gm, kBlock, 0, s>>>(R.ptr, R.idx, R.val, (const Vec*)w->d,
                                                                    (Vec*)w->ad, (const Vec*)w->r, m, w->part, w->st);
        if constexpr (sizeof(Vec) == 4) {
            k_pd_trial_ff<1><<<w->gv, kBlock, 0, s>>>(w->xh, w->xl, (const float*)w->d, w->grad, n, w->part, w->st);
            for (int t = 0; t < ls_passes; ++t)
                k_pd_trial_ff<kTrialsPerPass><<<w->gv, kBlock, 0, s>>>(w->xh, w->xl, (const float*)w->d, w->grad, n,
                                                                       w->part, w->st);
        } else {
            k_pd_trial<Vec, 1><<<w->gv, kBlock, 0, s>>>(w->X, (const Vec*)w->d, w->grad, n, w->part, w->st);
            for (int t = 0; t < ls_passes; ++t)
                k_pd_trial<Vec, kTrialsPerPass><<<w->gv, kBlock, 0, s>>>(w->X, (const Vec*)w->d, w->grad, n,
                                                                         w->part, w->st);
        }
        k_pd_apply<Vec><<<w->gv, kBlock, 0, s>>>(w->X, (const Vec*)w->d, n, w->xh, w->xl, w->st);
        L1LS_CUDA(cudaGetLastError());
    }
    return pd_finish(I, w, final_status, x_out, res, t0, s);
}

MfPd mfpd_params(const Inst* I) {
    return MfPd{I->n, I->p.right_stages, I->mf_c, I->mf_s, I->mf_c64, I->mf_s64, I->sigma32, I->sigma};
}

int mfpd_grid(const Inst* I, const void* kernel) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kMfThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = (I->n + kMfTile - 1) / kMfTile;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)I->ctx->num_sms * per_sm));
}

void enqueue_cg_mf(Inst* I, PdWork* w, cudaStream_t s) {
    const MfPd P = mfpd_params(I);
    k_mfpd_hp<<<w->gn, kMfThreads, 0, s>>>(P, (const float*)w->z, (float*)w->p, (float*)w->p2, (const float*)w->hd,
                                           (float*)w->hp, w->part, w->st);
    k_pd_cgupd<float><<<w->gv, kBlock, 0, s>>>((float*)w->d, (float2*)w->rcg, (const float*)w->p, (const float*)w->p2,
                                               (const float*)w->hp, (const float*)w->minv, (float*)w->z, I->n, w->part,
                                               w->st);
}

// pdNCG on a matrix-free instance: the Newton loop of run() with the passes above
l1ls_status run_mf(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res,
                   cudaStream_t s) {
    auto t0 = std::chrono::steady_clock::now();
    const int64_t m = I->m, n = I->n;
    const MfPd P = mfpd_params(I);
    PdWork* w = static_cast<PdWork*>(I->pd_work);
    if (!w) {
        std::unique_ptr<PdWork> fresh(new PdWork());
        w = fresh.get();
        for (double** v : {&w->X, &w->atr, &w->grad, &w->cn2, &w->atb}) L1LS_TRY(I->alloc_n(v, n));
        L1LS_TRY(I->alloc(&w->rcg, sizeof(float2) * pad32(n)));
        for (void** v : {&w->hd, &w->minv, &w->z, &w->p, &w->p2, &w->hp, &w->d})
            L1LS_TRY(I->alloc(v, sizeof(float) * pad32(n)));
        L1LS_TRY(I->alloc_n(&w->xh, pad32(n)));
        L1LS_TRY(I->alloc_n(&w->xl, pad32(n)));
        w->gn = mfpd_grid(I, (const void*)k_mfpd_hp);
        w->gm = mfpd_grid(I, (const void*)k_mfpd_grad);
        w->gv = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)I->ctx->num_sms * 8));
        const int gmax = std::max(std::max(w->gm, w->gn), w->gv);
        L1LS_TRY(I->alloc_n(&w->part, (int64_t)gmax * (kTrialsPerPass + 1)));
        L1LS_TRY(I->alloc_n(&w->st, 1));
        if (void* slot = I->ctx->pinned_get(sizeof(PdState))) {
            w->host = new (slot) PdState();
            w->pin_ctx = I->ctx;
        } else {
            w->host = new PdState();
        }
        // once per instance: diag(A^T A) and A^T b (grad serves as the scatter's scratch)
        const MfLeft L{I->m, I->n, I->p.left_stages, I->mf_ct, I->mf_st, I->mf_pperm};
        const int64_t units = std::max<int64_t>(n, m / 2);
        k_mfpd_scatter<<<(unsigned)((units + 255) / 256), 256, 0, s>>>(L, I->mf_ct64, I->mf_st64, I->bhat, w->grad);
        k_mfpd_rsig<<<w->gm, kMfThreads, 0, s>>>(P, w->grad, w->atb);
        k_mfpd_diag<<<w->gm, kMfThreads, 0, s>>>(P, w->cn2);
        L1LS_CUDA(cudaGetLastError());
        I->pd_work = fresh.release();
        I->pd_work_free = [](void* q) { delete static_cast<PdWork*>(q); };
    }
    if (x0) L1LS_CUDA(cudaMemcpyAsync(w->X, x0, sizeof(double) * n, cudaMemcpyDefault, s));
    else L1LS_CUDA(cudaMemsetAsync(w->X, 0, sizeof(double) * n, s));
    k_pd_split<<<w->gv, kBlock, 0, s>>>(w->X, w->xh, w->xl, n);
    PdState h;
    memset(&h, 0, sizeof(h));
    h.tau = o->tau;
    h.tol = o->rel_gap_tol;
    h.f_target = o->f_target;
    h.mu = o->mu_start > o->mu ? o->mu_start : o->mu;
    h.mu_target = o->mu;
    h.mu_min = o->mu_min;
    h.pcg_rtol = o->pcg_rtol;
    h.armijo = o->armijo;
    h.stall = 0.5;
    h.max_newton = o->max_iter;
    h.pcg_max = o->pcg_max;
    h.ls_max = o->ls_max;
    h.prev_gap = INFINITY;
    *w->host = h;
    L1LS_CUDA(cudaMemcpyAsync(w->st, w->host, sizeof(PdState), cudaMemcpyHostToDevice, s));
    k_mfpd_bb<<<w->gv, kBlock, 0, s>>>(I->bhat, m, w->part, w->st);
    L1LS_CUDA(cudaGetLastError());
    l1ls_status final_status = L1LS_OK;
    // graphs of an even number of PCG iterations (the search direction alternates buffers)
    int chunk = o->check_every > 0 ? std::min(o->check_every, 16) : 8;
    chunk = std::max(2, chunk & ~1);
    if (!w->cg_exec || w->cg_chunk != chunk) {
        if (w->cg_exec) {
            cudaGraphExecDestroy(w->cg_exec);
            w->cg_exec = nullptr;
        }
        cudaStream_t cap;
        L1LS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        L1LS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < chunk; ++i) enqueue_cg_mf(I, w, cap);
        cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        if (ce != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
        }
        L1LS_CUDA(cudaGraphInstantiate(&w->cg_exec, graph, 0));
        cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        w->cg_chunk = chunk;
    }
    const int ls_passes = (o->ls_max - 1 + kTrialsPerPass - 1) / kTrialsPerPass;
    for (;;) {
        k_mfpd_grad<<<w->gm, kMfThreads, 0, s>>>(P, w->X, w->atb, w->atr, w->part, w->st);
        L1LS_CUDA(cudaGetLastError());
        L1LS_CUDA(cudaMemcpyAsync(w->host, w->st, sizeof(PdState), cudaMemcpyDeviceToHost, s));
        L1LS_CUDA(cudaStreamSynchronize(s));
        if (w->host->stop) {
            final_status = (l1ls_status)w->host->status;
            break;
        }
        if (o->time_limit_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->time_limit_s) {
            final_status = L1LS_ETIMEOUT;
            break;
        }
        if (cancel_requested()) {
            final_status = L1LS_ECANCELLED;
            break;
        }
        k_pd_init<float><<<w->gv, kBlock, 0, s>>>(w->X, w->atr, w->cn2, w->grad, (float*)w->hd, (float*)w->minv,
                                                  (float2*)w->rcg, (float*)w->z, (float*)w->d, n, w->part, w->st);
        L1LS_CUDA(cudaGetLastError());
        const int64_t max_cg_launches = o->pcg_max / chunk + 3;
        for (int64_t launch = 0;; ++launch) {
            if (launch >= max_cg_launches) {
                final_status = set_error(L1LS_ECUDA, "internal: PCG did not raise its stop flag");
                break;
            }
            L1LS_CUDA(cudaGraphLaunch(w->cg_exec, s));
            L1LS_CUDA(cudaMemcpyAsync(&w->host->cg_done, &w->st->cg_done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            L1LS_CUDA(cudaStreamSynchronize(s));
            if (w->host->cg_done) break;
        }
        if (final_status != L1LS_OK) break;
        k_mfpd_ls<<<w->gm, kMfThreads, 0, s>>>(P, (const float*)w->d, w->atr, w->part, w->st);
        k_pd_trial_ff<1><<<w->gv, kBlock, 0, s>>>(w->xh, w->xl, (const float*)w->d, w->grad, n, w->part, w->st);
        for (int t = 0; t < ls_passes; ++t)
            k_pd_trial_ff<kTrialsPerPass><<<w->gv, kBlock, 0, s>>>(w->xh, w->xl, (const float*)w->d, w->grad, n,
                                                                   w->part, w->st);
        k_pd_apply<float><<<w->gv, kBlock, 0, s>>>(w->X, (const float*)w->d, n, w->xh, w->xl, w->st);
        L1LS_CUDA(cudaGetLastError());
    }
    return pd_finish(I, w, final_status, x_out, res, t0, s);
}

}  // namespace

l1ls_status pdncg_solve(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res,
                        cudaStream_t st) {
    if (I->matrix_free) return run_mf(I, o, x0, x_out, res, st);
    if (I->paired) {
        switch (I->dtype) {
            case L1LS_F64: return run<double, double, true>(I, o, x0, x_out, res, st);
            case L1LS_F32: return run<float, float, true>(I, o, x0, x_out, res, st);
            default: return run<__nv_bfloat16, float, true>(I, o, x0, x_out, res, st);
        }
    }
    switch (I->dtype) {
        case L1LS_F64: return run<double, double, false>(I, o, x0, x_out, res, st);
        case L1LS_F32: return run<float, float, false>(I, o, x0, x_out, res, st);
        default: return run<__nv_bfloat16, float, false>(I, o, x0, x_out, res, st);
    }
}

}  // namespace l1ls

using namespace l1ls;

extern "C" l1ls_status l1ls_solve_pdncg(l1ls_inst* h, const l1ls_solve_opts* o, const double* x0, double* x_out,
                                        l1ls_result* res, void* stream) {
    if (!h || !o) return set_error(L1LS_EINVAL, "NULL argument");
    if (!(o->tau > 0.0) || !(o->rel_gap_tol >= 0.0) || o->max_iter < 0 || o->ls_max < 1 || o->pcg_max < 1 ||
        !(o->mu > 0.0))
        return set_error(L1LS_EINVAL, "bad solver options");
    Inst* I = reinterpret_cast<Inst*>(h);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    return pdncg_solve(I, o, x0, x_out, res, (cudaStream_t)stream);
}
