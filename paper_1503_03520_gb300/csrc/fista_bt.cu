// FISTA with backtracking on L (Beck & Teboulle 2009, Sec. 4 of their paper; the paper's FISTA
// runs through TFOCS, whose L is dynamic, Sec. 8.1).  Iteration k:
//   y_k = x_{k-1} + beta_k (x_{k-1} - x_{k-2}),  A y_k by linearity from A x_{k-1}, A x_{k-2},
//   r_k = b - A y_k,  g = A^T r_k  (one product),
//   trial: x = S_{tau/L}(y_k + g / L),  A x  (one product),  d = x - y_k,  A d = A x - A y_k;
//          accepted when ||A d||^2 <= L ||d||^2 (the sufficient-decrease test of the quadratic
//          smooth part 1/2 ||Ax - b||^2, free of the cancellation between its two objective
//          values), otherwise L <- eta L and the trial is repeated;
//   x_k = x, certified by P(x_k) = tau ||x_k||_1 + 1/2 ||A x_k - b||^2 against
//   max_{j<=k} D(theta(y_j)), D = s b.r - s^2/2 ||r||^2, s = min(1, tau / ||g||_inf).
// FP64 vectors in the stored row order; the products are the library's (FP64 sums for FP64
// values, FP32 sums otherwise).  The host reads seven reduced scalars per trial (the
// backtracking decision is data-dependent), so iterations are not graph-captured.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace l1ls {

namespace {

constexpr int kBtBlock = 256;

// FISTA with backtracking (Beck & Teboulle 2009), one iteration in four kernels.
// r = b - A y with A y = A x + beta (A x - A x_prev); writes A y and r; sums b.r, r.r
__global__ void __launch_bounds__(kBtBlock) k_bt_residual(const double* __restrict__ ax, const double* __restrict__ axp,
                                                        const double* __restrict__ b, double beta, int64_t m,
                                                        double* __restrict__ ay, double* __restrict__ r,
                                                        double* partials, unsigned* counter, double* out) {
    __shared__ double red[2 * 32];
    double v[2] = {0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const double u = ax[i];
        const double a = u + beta * (u - axp[i]);
        const double ri = b[i] - a;
        ay[i] = a;
        r[i] = ri;
        v[0] += b[i] * ri;
        v[1] += ri * ri;
    }
    block_reduce<kBtBlock, 2>(v, 0u, red);
    double tot[2];
    if (grid_reduce_last<kBtBlock, 2>(v, 0u, partials, counter, tot, red) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

// y = x + beta (x - x_prev)
__global__ void k_bt_y(const double* __restrict__ x, const double* __restrict__ xp, double beta, int64_t n,
                       double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] + beta * (x[i] - xp[i]);
}

// trial point x = S_{thr}(y + g / L); sums d.d, |x|, max |g|
__global__ void __launch_bounds__(kBtBlock) k_bt_prox(const double* __restrict__ y, const double* __restrict__ g,
                                                    double L, double thr, int64_t n, double* __restrict__ xn,
                                                    double* partials, unsigned* counter, double* out) {
    __shared__ double red[3 * 32];
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double gi = g[i];
        const double xi = soft_threshold(y[i] + gi / L, thr);
        const double di = xi - y[i];
        xn[i] = xi;
        v[0] += di * di;
        v[1] += fabs(xi);
        v[2] = fmax(v[2], fabs(gi));
    }
    block_reduce<kBtBlock, 3>(v, 4u, red);
    double tot[3];
    if (grid_reduce_last<kBtBlock, 3>(v, 4u, partials, counter, tot, red) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
        out[2] = tot[2];
    }
}

// A d = A x - A y and the fit A x - b; sums ||A d||^2, ||A x - b||^2
__global__ void __launch_bounds__(kBtBlock) k_bt_fit(const double* __restrict__ axn, const double* __restrict__ ay,
                                                   const double* __restrict__ b, int64_t m, double* partials,
                                                   unsigned* counter, double* out) {
    __shared__ double red[2 * 32];
    double v[2] = {0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const double u = axn[i];
        const double ad = u - ay[i];
        const double f = u - b[i];
        v[0] += ad * ad;
        v[1] += f * f;
    }
    block_reduce<kBtBlock, 2>(v, 0u, red);
    double tot[2];
    if (grid_reduce_last<kBtBlock, 2>(v, 0u, partials, counter, tot, red) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

inline unsigned blocks_of(int64_t count) { return (unsigned)std::max<int64_t>(1, (count + kBtBlock - 1) / kBtBlock); }

// Work space of one solve, released on every return path
struct BtWork {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit BtWork(cudaStream_t s) : st(s) {}
    template <class T> l1ls_status get(T** p, int64_t count) {
        cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1), st);
        if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(fista_bt)", __FILE__, __LINE__);
        ptrs.push_back(*p);
        return L1LS_OK;
    }
    ~BtWork() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    }
};

l1ls_status solve_bt(Inst* I, const l1ls_solve_opts* o, double L0, double eta, const double* x0, double* x_out,
                     l1ls_result* res, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t m = I->m, n = I->n;
    const double tau = o->tau;
    BtWork w(st);
    double *x, *xp, *xn, *y, *g, *ax, *axp, *axn, *ay, *r, *partials, *out;
    unsigned* counters;
    L1LS_TRY(w.get(&x, n));
    L1LS_TRY(w.get(&xp, n));
    L1LS_TRY(w.get(&xn, n));
    L1LS_TRY(w.get(&y, n));
    L1LS_TRY(w.get(&g, n));
    L1LS_TRY(w.get(&ax, m));
    L1LS_TRY(w.get(&axp, m));
    L1LS_TRY(w.get(&axn, m));
    L1LS_TRY(w.get(&ay, m));
    L1LS_TRY(w.get(&r, m));
    const unsigned gm = std::min<unsigned>(blocks_of(m), 8u * (unsigned)I->ctx->num_sms);
    const unsigned gn = std::min<unsigned>(blocks_of(n), 8u * (unsigned)I->ctx->num_sms);
    L1LS_TRY(w.get(&partials, 3 * (int64_t)std::max(gm, gn)));
    L1LS_TRY(w.get(&out, 8));
    L1LS_TRY(w.get(&counters, 3));
    L1LS_CUDA(cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned), st));
    if (x0) L1LS_CUDA(cudaMemcpyAsync(x, x0, sizeof(double) * n, cudaMemcpyDefault, st));
    else L1LS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    L1LS_CUDA(cudaMemcpyAsync(xp, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    L1LS_TRY(spmv_plain(I, false, x, L1LS_F64, ax, false, st));
    L1LS_CUDA(cudaMemcpyAsync(axp, ax, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    int64_t products = 1, backtracks = 0, k = 1;
    double t = 1.0, beta = 0.0, L = L0, best_d = -INFINITY;
    double P = NAN, gap = NAN, rel = NAN;
    l1ls_status status = L1LS_OK;
    double h[8];
    for (;;) {
        k_bt_y<<<blocks_of(n), kBtBlock, 0, st>>>(x, xp, beta, n, y);
        k_bt_residual<<<gm, kBtBlock, 0, st>>>(ax, axp, I->bhat, beta, m, ay, r, partials, counters + 0, out + 0);
        L1LS_CUDA(cudaGetLastError());
        L1LS_TRY(spmv_plain(I, true, r, L1LS_F64, g, false, st));
        products += 1;
        int trials = 0;
        bool accepted = false;
        for (;;) {
            k_bt_prox<<<gn, kBtBlock, 0, st>>>(y, g, L, tau / L, n, xn, partials, counters + 1, out + 2);
            L1LS_CUDA(cudaGetLastError());
            L1LS_TRY(spmv_plain(I, false, xn, L1LS_F64, axn, false, st));
            products += 1;
            k_bt_fit<<<gm, kBtBlock, 0, st>>>(axn, ay, I->bhat, m, partials, counters + 2, out + 5);
            L1LS_CUDA(cudaGetLastError());
            L1LS_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st));
            L1LS_CUDA(cudaStreamSynchronize(st));
            // h: [0] b.r [1] r.r [2] d.d [3] sum|x| [4] max|g| [5] ||A d||^2 [6] ||A x - b||^2
            if (!std::isfinite(h[5]) || !std::isfinite(h[2])) break;
            if (h[5] <= L * h[2]) {
                accepted = true;
                break;
            }
            if (++trials > o->ls_max) break;
            L *= eta;
            backtracks += 1;
        }
        if (!accepted) {
            status = set_error(L1LS_ENUMERIC, "FISTA backtracking: no step constant passed the test");
            k -= 1;   // x_{k-1} stays the returned iterate
            break;
        }
        const double s = h[4] <= tau ? 1.0 : tau / h[4];
        best_d = std::max(best_d, s * h[0] - 0.5 * s * s * h[1]);
        P = tau * h[3] + 0.5 * h[6];
        gap = P - best_d;
        rel = gap / std::max(std::fabs(P), 1e-300);
        if (!std::isfinite(P)) {
            status = set_error(L1LS_ENUMERIC, "FISTA backtracking: non-finite objective");
            k -= 1;
            break;
        }
        // x_k = the accepted trial; rotate the buffers
        std::swap(xp, x);
        std::swap(x, xn);
        std::swap(axp, ax);
        std::swap(ax, axn);
        if (rel <= o->rel_gap_tol || P <= o->f_target) break;
        if (k >= o->max_iter) {
            status = L1LS_ENOCONV;
            break;
        }
        if (cancel_requested()) {
            status = L1LS_ECANCELLED;
            break;
        }
        if (o->time_limit_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->time_limit_s) {
            status = L1LS_ETIMEOUT;
            break;
        }
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        beta = (t - 1.0) / tn;
        t = tn;
        k += 1;
    }
    if (x_out) L1LS_CUDA(cudaMemcpyAsync(x_out, x, sizeof(double) * n, cudaMemcpyDefault, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    if (res) {
        memset(res, 0, sizeof(*res));
        res->iters = k;
        res->products = products;
        res->ls_trials = backtracks;
        res->f = P;
        res->dual = best_d;
        res->gap = gap;
        res->rel_gap = rel;
        res->L = L;
        res->status = status;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

}  // namespace

}  // namespace l1ls

using namespace l1ls;

extern "C" l1ls_status l1ls_solve_fista_bt(l1ls_inst* h, const l1ls_solve_opts* o, double L0, double eta,
                                           const double* x0, double* x_out, l1ls_result* res, void* stream) {
    if (!h || !o) return set_error(L1LS_EINVAL, "NULL argument");
    if (!(o->tau > 0.0) || !(o->rel_gap_tol >= 0.0) || o->max_iter < 1 || o->ls_max < 0)
        return set_error(L1LS_EINVAL, "bad solver options");
    if (!(L0 > 0.0) || !std::isfinite(L0) || !(eta > 1.0) || !std::isfinite(eta))
        return set_error(L1LS_EINVAL, "FISTA backtracking needs L0 > 0 and eta > 1");
    Inst* I = reinterpret_cast<Inst*>(h);
    if (I->matrix_free) return set_error(L1LS_EINVAL, "FISTA backtracking needs the assembled matrix");
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    return solve_bt(I, o, L0, eta, x0, x_out, res, (cudaStream_t)stream);
}
