// Instance generator on the device: Procedure IGen (Sec. 3.1) on the matrix of Eq. (bd8),
// A = (P G~ P) Sigma R^T with the Givens stages of Sec. 4.1-4.2, x* from Procedure OsGen.
//
// The library stores Ahat = P1^T A = G~ P2 Sigma R^T, whose rows 2p and 2p+1 are the two
// rows mixed by one left rotation and share one column support.  Both CSR(Ahat) and
// CSR(Ahat^T) are produced directly from the structure:
//   column j of Sigma R^T  : rows I_j = supp(R^T e_j), a contiguous interval (each stage
//                            widens an interval by at most one on each side),
//   row k of R^T           : columns J_k = supp(R e_k), also an interval,
//   row q of P2 Sigma R^T  : row perm[q] of Sigma R^T (zero when perm[q] >= n),
//   row 2p / 2p+1 of Ahat  : c~ X_2p - s~ X_2p+1  /  s~ X_2p + c~ X_2p+1.
// Every entry value is computed once, column by column (R^T e_j by rotating a window, the
// MvPA order), and CSR(Ahat) copies it from CSR(Ahat^T), so the two are exact transposes.
// Products and sums use __dmul_rn / __dadd_rn so no contraction changes the rounding.
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "internal.h"
#include "spmv.cuh"

namespace l1ls {

l1ls_status exclusive_scan_i32(const int32_t* in, int64_t count, int32_t* out, int64_t* total, cudaStream_t st);
l1ls_status sum_i32(const int32_t* in, int64_t count, int64_t* total, cudaStream_t st);
l1ls_status radix_argsort_u64(const uint64_t* keys, int64_t count, uint32_t* order, cudaStream_t st);

namespace {

constexpr int kWMax = 8;                 // right stages supported
constexpr int kWin = 2 * kWMax + 1;      // window of R^T e_j

struct Geo {
    int64_t m, n;      // rows of A, size of the square Givens part
    int w;             // right stages
    int left;          // left stages (0 / 1)
    double c, s, ct, st;
};

__device__ __forceinline__ void expand(int64_t& lo, int64_t& hi, int first, int64_t n) {
    const int64_t d = lo - first;
    if (d >= 0 && (d & 1)) lo -= 1;                      // lo is the second of its plane
    const int64_t e = hi - first;
    if (e >= 0 && !(e & 1) && hi + 1 < n) hi += 1;       // hi is the first of its plane
}
// I_j = supp(R^T e_j): stages T_w^T first, T_1^T last
__device__ __forceinline__ void col_interval(int64_t j, const Geo& g, int64_t& lo, int64_t& hi) {
    lo = hi = j;
    for (int k = g.w; k >= 1; --k) expand(lo, hi, (k - 1) & 1, g.n);
}
// J_k = supp(R e_k): stages T_1 first, T_w last
__device__ __forceinline__ void row_interval(int64_t k, const Geo& g, int64_t& lo, int64_t& hi) {
    lo = hi = k;
    for (int q = 1; q <= g.w; ++q) expand(lo, hi, (q - 1) & 1, g.n);
}
// values of R^T e_j on the window [j - w, j + w]
__device__ void col_values(int64_t j, const Geo& g, double* v) {
    const int64_t base = j - g.w;
    for (int t = 0; t < kWin; ++t) v[t] = 0.0;
    v[g.w] = 1.0;
    for (int k = g.w; k >= 1; --k) {
        const int first = (k - 1) & 1;
        int64_t i = base < first ? first : base;
        if ((i - first) & 1) ++i;
        for (; i + 1 <= base + 2 * g.w && i + 1 < g.n; i += 2) {
            const double a = v[i - base], b = v[i + 1 - base];
            v[i - base] = __dadd_rn(__dmul_rn(g.c, a), __dmul_rn(g.s, b));
            v[i + 1 - base] = __dadd_rn(__dmul_rn(-g.s, a), __dmul_rn(g.c, b));
        }
    }
}

__global__ void k_keys(uint64_t seed, uint64_t tag, int64_t count, uint64_t* __restrict__ keys) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) keys[i] = sm_output(sm_stream(seed, tag), (uint64_t)i);
}

// Sigma of Sec. 4: sigma_i = kappa^(-rank_i/(n-1)) (kappa(A) = kappa, sigma_max = 1)
__global__ void k_sigma(const uint32_t* __restrict__ order, int64_t count, double logk, double* __restrict__ sigma) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    double v = 1.0;
    if (count > 1) v = exp(-((double)r / (double)(count - 1)) * logk);
    sigma[order[r]] = v;
}

__global__ void k_perm(const uint32_t* __restrict__ order, int64_t count, int32_t* __restrict__ perm,
                       int32_t* __restrict__ perm_inv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    perm[i] = (int32_t)order[i];
    perm_inv[order[i]] = (int32_t)i;
}

__global__ void k_identity_perm(int64_t count, int32_t* __restrict__ perm, int32_t* __restrict__ perm_inv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    perm[i] = (int32_t)i;
    perm_inv[i] = (int32_t)i;
}

// support S of x* (Procedure OsGen, Sec. 6): the s smallest keys
__global__ void k_support(const uint32_t* __restrict__ order, int64_t s, uint8_t* __restrict__ flag) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < s) flag[order[r]] = 1;
}

// OsGen with magnitudes U[lo, hi] and random signs; g of Eq. (bd6).
__global__ void k_xstar_g(uint64_t seed, int64_t n, int64_t nsup, const uint8_t* __restrict__ flag, double lo,
                          double hi, int goff_mode, double* __restrict__ xstar, double* __restrict__ g) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool on = i < nsup && flag[i];
    double x = 0.0, gi;
    if (on) {
        const double u = u01(sm_output(sm_stream(seed, kTagXVal), (uint64_t)i));
        const double mag = __dadd_rn(lo, __dmul_rn(hi - lo, u));
        const bool neg = (sm_output(sm_stream(seed, kTagXSign), (uint64_t)i) >> 63) != 0;
        x = neg ? -mag : mag;
        gi = neg ? -1.0 : 1.0;
    } else {
        gi = goff_mode == 0 ? __dadd_rn(2.0 * u01(sm_output(sm_stream(seed, kTagGOff), (uint64_t)i)), -1.0) : 0.0;
    }
    xstar[i] = x;
    if (i < nsup) g[i] = gi;
}

// Sec. 8.9's singular values: sigma_odd for odd i, sigma_even for even i (1-based i)
__global__ void k_sigma_alt(int64_t count, double s_odd, double s_even, double* __restrict__ sigma) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) sigma[j] = (j & 1) ? s_even : s_odd;
}

// support flags as int32 (for the exclusive scan that ranks the support in index order)
__global__ void k_flag_i32(const uint8_t* __restrict__ flag, int64_t count, int32_t* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) out[j] = flag[j];
}

// Sec. 8.9's x*: the first half of the support (index order) -hi, the rest +lo; g = sign(x*)
__global__ void k_xstar_alt(int64_t n, int64_t nsup, const uint8_t* __restrict__ flag,
                            const int32_t* __restrict__ rank, int64_t half, double lo, double hi, uint64_t seed,
                            int goff_mode, double* __restrict__ xstar, double* __restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool on = i < nsup && flag[i];
    double x = 0.0, gi;
    if (on) {
        x = rank[i] < half ? -hi : lo;
        gi = x < 0.0 ? -1.0 : 1.0;
    } else {
        gi = goff_mode == 0 ? __dadd_rn(2.0 * u01(sm_output(sm_stream(seed, kTagGOff), (uint64_t)i)), -1.0) : 0.0;
    }
    xstar[i] = x;
    if (i < nsup) g[i] = gi;
}

// Procedure OsGen3 (Sec. 6): the least-squares solution starts as gamma / sigma^2 (the stages of G follow)
__global__ void k_gamma_over_sigma2(const double* __restrict__ sigma, int64_t n, double gamma, double* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = __ddiv_rn(gamma, __dmul_rn(sigma[i], sigma[i]));
}
// sort keys: the bit pattern of |x| orders non-negative doubles; zeros counted
__global__ void k_abs_keys(const double* __restrict__ x, int64_t n, uint64_t* __restrict__ keys, int* __restrict__ zeros) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = fabs(x[i]);
    keys[i] = (uint64_t)__double_as_longlong(a);
    if (a == 0.0) atomicAdd(zeros, 1);
}
// OsGen3's selection (Sec. 6): keep ranks z .. z+s1-1 (the s1 smallest nonzero) and n-s2 .. n-1 (largest)
__global__ void k_osgen3_flags(const uint32_t* __restrict__ order, int64_t n, const int* __restrict__ zeros, int64_t s1,
                               int64_t s2, uint8_t* __restrict__ flag) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t z = *zeros;
    if (r >= z && (r < z + s1 || r >= n - s2)) flag[order[r]] = 1;
}
// x* = x on the kept entries (zero elsewhere); g = sign(x*) there, U(-1,1) elsewhere
__global__ void k_osgen3_xstar(const double* __restrict__ x, const uint8_t* __restrict__ flag, int64_t n, uint64_t seed,
                               int goff_mode, double* __restrict__ xstar, double* __restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi = 0.0, gi;
    if (flag[i]) {
        xi = x[i];
        gi = xi < 0.0 ? -1.0 : 1.0;
    } else {
        gi = goff_mode == 0 ? __dadd_rn(2.0 * u01(sm_output(sm_stream(seed, kTagGOff), (uint64_t)i)), -1.0) : 0.0;
    }
    xstar[i] = xi;
    g[i] = gi;
}

// one stage (Sec. 4.1-4.2) on a vector, in place: transpose ? T^T v : T v
__global__ void k_stage(double* __restrict__ v, int64_t n, int first, double c, double s, int transpose) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = first + 2 * t;
    if (i + 1 >= n) return;
    const double a = v[i], b = v[i + 1];
    if (transpose) {
        v[i] = __dadd_rn(__dmul_rn(c, a), __dmul_rn(s, b));
        v[i + 1] = __dadd_rn(__dmul_rn(-s, a), __dmul_rn(c, b));
    } else {
        v[i] = __dadd_rn(__dmul_rn(c, a), __dmul_rn(-s, b));
        v[i + 1] = __dadd_rn(__dmul_rn(s, a), __dmul_rn(c, b));
    }
}

// IGen's e and b (Sec. 3.1) by the route of Sec. 4, Sigma step: ze = tau vg / sigma, zb = sigma vx + tau vg / sigma (length n)
__global__ void k_scale(const double* __restrict__ vg, const double* __restrict__ vx, const double* __restrict__ sigma,
                        int64_t n, double tau, double* __restrict__ ze, double* __restrict__ zb,
                        double* __restrict__ u_lam) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double sg = sigma[k];
    const double e = __dmul_rn(tau, vg[k]) / sg;
    ze[k] = e;
    zb[k] = __dadd_rn(__dmul_rn(sg, vx[k]), e);
    // A^T b = R (Sigma^2 R^T x* + tau R^T g): the inner vector
    u_lam[k] = __dadd_rn(__dmul_rn(__dmul_rn(sg, sg), vx[k]), __dmul_rn(tau, vg[k]));
}

// left factor of Eq. (bd8) (Sec. 4.1): ehat = G~ P2 [ze; 0], bhat = G~ P2 [zb; 0] in the
// relabelled row order
__global__ void k_left(const double* __restrict__ ze, const double* __restrict__ zb, const int32_t* __restrict__ perm,
                       Geo g, double* __restrict__ ehat, double* __restrict__ bhat) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g.left == 0) {
        if (t >= g.m) return;
        ehat[t] = t < g.n ? ze[t] : 0.0;
        bhat[t] = t < g.n ? zb[t] : 0.0;
        return;
    }
    if (2 * t + 1 >= g.m) return;
    const int64_t ke = perm[2 * t], ko = perm[2 * t + 1];
    const double e0 = ke < g.n ? ze[ke] : 0.0, e1 = ko < g.n ? ze[ko] : 0.0;
    const double b0 = ke < g.n ? zb[ke] : 0.0, b1 = ko < g.n ? zb[ko] : 0.0;
    ehat[2 * t] = __dadd_rn(__dmul_rn(g.ct, e0), __dmul_rn(-g.st, e1));
    ehat[2 * t + 1] = __dadd_rn(__dmul_rn(g.st, e0), __dmul_rn(g.ct, e1));
    bhat[2 * t] = __dadd_rn(__dmul_rn(g.ct, b0), __dmul_rn(-g.st, b1));
    bhat[2 * t + 1] = __dadd_rn(__dmul_rn(g.st, b0), __dmul_rn(g.ct, b1));
}

// deterministic grid reduction: out[0] = sum |a|, out[1] = sum b^2, out[2] = max |c|
__global__ void k_reduce3(const double* __restrict__ a, int64_t na, const double* __restrict__ b, int64_t nb,
                          const double* __restrict__ c, int64_t nc, double* __restrict__ partials,
                          unsigned* __restrict__ counter, double* __restrict__ out) {
    __shared__ double smem[3 * 32];
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride) v[0] += fabs(a[i]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) v[1] += b[i] * b[i];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += stride) v[2] = fmax(v[2], fabs(c[i]));
    block_reduce<256, 3>(v, 4u, smem);
    double tot[3];
    if (grid_reduce_last<256, 3>(v, 4u, partials, counter, tot, smem) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
        out[2] = tot[2];
    }
}

// Eq. (bd12) sums: out[0] = sum x*_i^2, out[1] = sum over sigma_i^2 >= rho of (R^T x*)_i^2
__global__ void k_kappa_sums(const double* __restrict__ x, const double* __restrict__ z, const double* __restrict__ sigma,
                             int64_t n, double rho, double* __restrict__ partials, unsigned* __restrict__ counter,
                             double* __restrict__ out) {
    __shared__ double smem[2 * 32];
    double v[2] = {0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        v[0] += x[i] * x[i];
        if (sigma[i] * sigma[i] >= rho) v[1] += z[i] * z[i];
    }
    block_reduce<256, 2>(v, 4u, smem);
    double tot[2];
    if (grid_reduce_last<256, 2>(v, 4u, partials, counter, tot, smem) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

// number of distinct left planes touched by column j (x2 rows); L = I: |I_j|
__global__ void k_csc_count(Geo g, const int32_t* __restrict__ perm_inv, int32_t* __restrict__ cnt) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n) return;
    int64_t lo, hi;
    col_interval(j, g, lo, hi);
    if (g.left == 0) {
        cnt[j] = (int32_t)(hi - lo + 1);
        return;
    }
    int32_t pl[2 * kWMax];
    int np = 0;
    for (int64_t k = lo; k <= hi; ++k) {
        const int32_t p = perm_inv[k] >> 1;
        bool seen = false;
        for (int t = 0; t < np; ++t) seen |= (pl[t] == p);
        if (!seen) pl[np++] = p;
    }
    cnt[j] = 2 * np;
}

__global__ void k_csc_fill(Geo g, const int32_t* __restrict__ perm_inv, const double* __restrict__ sigma,
                           const int32_t* __restrict__ ptr, int32_t* __restrict__ rows, double* __restrict__ vals) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n) return;
    int64_t lo, hi;
    col_interval(j, g, lo, hi);
    double v[kWin];
    col_values(j, g, v);
    const int64_t base = j - g.w;
    int64_t o = ptr[j];
    if (g.left == 0) {
        for (int64_t k = lo; k <= hi; ++k) {
            rows[o] = (int32_t)k;
            vals[o] = __dmul_rn(sigma[k], v[k - base]);
            ++o;
        }
        return;
    }
    // entries (q, t_k) with q = perm_inv[k], sorted by q
    int32_t q[2 * kWMax];
    double tv[2 * kWMax];
    int ne = 0;
    for (int64_t k = lo; k <= hi; ++k) {
        const int32_t qq = perm_inv[k];
        const double tt = __dmul_rn(sigma[k], v[k - base]);
        int pos = ne++;
        while (pos > 0 && q[pos - 1] > qq) {
            q[pos] = q[pos - 1];
            tv[pos] = tv[pos - 1];
            --pos;
        }
        q[pos] = qq;
        tv[pos] = tt;
    }
    for (int a = 0; a < ne;) {
        const int32_t p = q[a] >> 1;
        bool he = false, ho = false;
        double te = 0.0, to = 0.0;
        while (a < ne && (q[a] >> 1) == p) {
            if (q[a] & 1) { ho = true; to = tv[a]; }
            else { he = true; te = tv[a]; }
            ++a;
        }
        double v0, v1;
        if (he && ho) {
            v0 = __dadd_rn(__dmul_rn(g.ct, te), __dmul_rn(-g.st, to));
            v1 = __dadd_rn(__dmul_rn(g.st, te), __dmul_rn(g.ct, to));
        } else if (he) {
            v0 = __dmul_rn(g.ct, te);
            v1 = __dmul_rn(g.st, te);
        } else {
            v0 = __dmul_rn(-g.st, to);
            v1 = __dmul_rn(g.ct, to);
        }
        rows[o] = 2 * p;
        vals[o] = v0;
        rows[o + 1] = 2 * p + 1;
        vals[o + 1] = v1;
        o += 2;
    }
}

// columns of row rho: J_{perm[2p]} U J_{perm[2p+1]} (those below n); L = I: J_rho
__device__ __forceinline__ int row_support(int64_t rho, const Geo& g, const int32_t* __restrict__ perm, int64_t& a1,
                                           int64_t& b1, int64_t& a2, int64_t& b2) {
    if (g.left == 0) {
        if (rho >= g.n) return 0;
        row_interval(rho, g, a1, b1);
        return 1;
    }
    const int64_t p = rho >> 1;
    const int64_t ke = perm[2 * p], ko = perm[2 * p + 1];
    int cnt = 0;
    if (ke < g.n) { row_interval(ke, g, a1, b1); cnt = 1; }
    if (ko < g.n) {
        if (cnt == 0) { row_interval(ko, g, a1, b1); cnt = 1; }
        else { row_interval(ko, g, a2, b2); cnt = 2; }
    }
    if (cnt == 2) {
        if (a2 < a1) { int64_t t = a1; a1 = a2; a2 = t; t = b1; b1 = b2; b2 = t; }
        if (a2 <= b1 + 1) {            // overlapping or touching: one interval
            b1 = b1 > b2 ? b1 : b2;
            cnt = 1;
        }
    }
    return cnt;
}

__global__ void k_csr_count(Geo g, const int32_t* __restrict__ perm, int32_t* __restrict__ cnt) {
    int64_t rho = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rho >= g.m) return;
    int64_t a1 = 0, b1 = -1, a2 = 0, b2 = -1;
    const int c = row_support(rho, g, perm, a1, b1, a2, b2);
    cnt[rho] = c == 0 ? 0 : (int32_t)((b1 - a1 + 1) + (c == 2 ? (b2 - a2 + 1) : 0));
}

__global__ void k_csr_fill(Geo g, const int32_t* __restrict__ perm, const int32_t* __restrict__ csc_ptr,
                           const int32_t* __restrict__ csc_row, const double* __restrict__ csc_val,
                           const int32_t* __restrict__ ptr, int32_t* __restrict__ cols, double* __restrict__ vals,
                           int* __restrict__ err) {
    int64_t rho = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rho >= g.m) return;
    int64_t a[2] = {0, 0}, b[2] = {-1, -1};
    const int c = row_support(rho, g, perm, a[0], b[0], a[1], b[1]);
    int64_t o = ptr[rho];
    for (int iv = 0; iv < c; ++iv) {
        for (int64_t j = a[iv]; j <= b[iv]; ++j) {
            int32_t lo = csc_ptr[j], hi = csc_ptr[j + 1];
            while (lo < hi) {                       // first position with row >= rho
                const int32_t mid = (lo + hi) >> 1;
                if (csc_row[mid] < rho) lo = mid + 1;
                else hi = mid;
            }
            double val = 0.0;
            if (lo < csc_ptr[j + 1] && csc_row[lo] == rho) val = csc_val[lo];
            else atomicExch(err, 1);
            cols[o] = (int32_t)j;
            vals[o] = val;
            ++o;
        }
    }
}

// most nonzeros in a tile of 32 rows
__global__ void k_tile_max(const int32_t* __restrict__ ptr, int64_t nrows, int* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t * 32 >= nrows) return;
    const int64_t r1 = min(t * 32 + 32, nrows);
    atomicMax(out, ptr[r1] - ptr[t * 32]);
}

template <class V>
__global__ void k_cast(const double* __restrict__ in, int64_t count, V* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = from_double<V>(in[i]);
}

__global__ void k_to_f32(const double* __restrict__ in, int64_t count, float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = __double2float_rn(in[i]);
}

// paired rows: pair p takes the columns of row 2p and the values of rows 2p and 2p+1
template <class V>
__global__ void k_pair_rows(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const V* __restrict__ val, int64_t npairs, int32_t* __restrict__ pptr,
                            int32_t* __restrict__ pcol, V* __restrict__ pval, int* __restrict__ err) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > npairs) return;
    const int32_t a = ptr[2 * p];
    pptr[p] = a / 2;
    if (p == npairs) return;
    const int32_t b = ptr[2 * p + 1], c = ptr[2 * p + 2];
    if ((a & 1) || b - a != c - b) {
        atomicExch(err, 2);
        return;
    }
    for (int32_t k = 0; k < b - a; ++k) {
        if (col[a + k] != col[b + k]) atomicExch(err, 2);
        const int32_t o = a / 2 + k;
        pcol[o] = col[a + k];
        pval[2 * (int64_t)o] = val[a + k];
        pval[2 * (int64_t)o + 1] = val[b + k];
    }
}

// paired columns: consecutive rows (2p, 2p+1) of a column become one entry
template <class V>
__global__ void k_pair_cols(const int32_t* __restrict__ ptr, const int32_t* __restrict__ row,
                            const V* __restrict__ val, int64_t n, int32_t* __restrict__ qptr,
                            int32_t* __restrict__ qpair, V* __restrict__ qval, int* __restrict__ err) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    const int32_t a = ptr[j];
    qptr[j] = a / 2;
    if (j == n) return;
    const int32_t b = ptr[j + 1];
    if ((a & 1) || ((b - a) & 1)) {
        atomicExch(err, 3);
        return;
    }
    for (int32_t e = a; e < b; e += 2) {
        if ((row[e] & 1) || row[e + 1] != row[e] + 1) atomicExch(err, 3);
        const int32_t o = e / 2;
        qpair[o] = row[e] >> 1;
        qval[2 * (int64_t)o] = val[e];
        qval[2 * (int64_t)o + 1] = val[e + 1];
    }
}

// ---- storage order of the row pairs ------------------------------------------------------
// Pair p holds the rows perm[2p], perm[2p+1] of Sigma R^T.  Pairs are stored in the order of
// the smaller of the two (pairs of two empty rows last), so consecutive stored pairs and the
// columns that touch them meet nearby entries of the gathered vectors for one of their two
// halves.  Any order of whole pairs describes the same problem (rows of A permuted).
__global__ void k_pair_keys(const int32_t* __restrict__ perm, int64_t npairs, int64_t n, uint64_t* __restrict__ keys) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int64_t a = perm[2 * p], b = perm[2 * p + 1];
    const int64_t k = a < b ? a : b;
    keys[p] = (uint64_t)(k < n ? k : n + p);
}

__global__ void k_qpos(const uint32_t* __restrict__ order, int64_t npairs, int32_t* __restrict__ qpos) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < npairs) qpos[order[r]] = (int32_t)r;
}

// entries per stored pair, in the new order
__global__ void k_pair_counts(const int32_t* __restrict__ pptr, const uint32_t* __restrict__ order, int64_t npairs,
                              int32_t* __restrict__ cnt) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < npairs) cnt[r] = pptr[order[r] + 1] - pptr[order[r]];
}

template <class V>
__global__ void k_move_pair_rows(const int32_t* __restrict__ optr, const int32_t* __restrict__ ocol,
                                 const V* __restrict__ oval, const uint32_t* __restrict__ order, int64_t npairs,
                                 const int32_t* __restrict__ nptr, int32_t* __restrict__ ncol, V* __restrict__ nval) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= npairs) return;
    const int64_t o = order[r];
    const int32_t a = optr[o], c = optr[o + 1] - a, d = nptr[r];
    for (int32_t k = 0; k < c; ++k) {
        ncol[d + k] = ocol[a + k];
        nval[2 * (int64_t)(d + k)] = oval[2 * (int64_t)(a + k)];
        nval[2 * (int64_t)(d + k) + 1] = oval[2 * (int64_t)(a + k) + 1];
    }
}

// plain rows 2r, 2r+1 <- 2 order[r], 2 order[r] + 1 (row pointers from the pair pointers)
template <class V>
__global__ void k_move_plain_rows(const int32_t* __restrict__ optr, const int32_t* __restrict__ ocol,
                                  const V* __restrict__ oval, const uint32_t* __restrict__ order, int64_t npairs,
                                  const int32_t* __restrict__ npptr, int32_t* __restrict__ nptr,
                                  int32_t* __restrict__ ncol, V* __restrict__ nval) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > npairs) return;
    nptr[2 * r] = 2 * npptr[r];
    if (r == npairs) return;
    const int64_t o = order[r];
    const int32_t c = optr[2 * o + 1] - optr[2 * o];
    nptr[2 * r + 1] = 2 * npptr[r] + c;
    for (int t = 0; t < 2; ++t) {
        const int32_t a = optr[2 * o + t], d = 2 * npptr[r] + t * c;
        for (int32_t k = 0; k < c; ++k) {
            ncol[d + k] = ocol[a + k];
            nval[d + k] = oval[a + k];
        }
    }
}

// paired columns: pair index -> stored position, entries re-sorted by it
template <class V>
__global__ void k_remap_pair_cols(const int32_t* __restrict__ ptr, int32_t* __restrict__ pair, V* __restrict__ val2,
                                  const int32_t* __restrict__ qpos, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t a = ptr[j], c = ptr[j + 1] - a;
    for (int32_t k = 0; k < c; ++k) pair[a + k] = qpos[pair[a + k]];
    for (int32_t k = 1; k < c; ++k) {               // insertion sort (a column holds <= 16 pairs)
        const int32_t key = pair[a + k];
        const V v0 = val2[2 * (int64_t)(a + k)], v1 = val2[2 * (int64_t)(a + k) + 1];
        int32_t q = k;
        while (q > 0 && pair[a + q - 1] > key) {
            pair[a + q] = pair[a + q - 1];
            val2[2 * (int64_t)(a + q)] = val2[2 * (int64_t)(a + q - 1)];
            val2[2 * (int64_t)(a + q) + 1] = val2[2 * (int64_t)(a + q - 1) + 1];
            --q;
        }
        pair[a + q] = key;
        val2[2 * (int64_t)(a + q)] = v0;
        val2[2 * (int64_t)(a + q) + 1] = v1;
    }
}

// plain columns: row q -> 2 qpos[q >> 1] + (q & 1), re-sorted (pairs stay adjacent)
template <class V>
__global__ void k_remap_plain_cols(const int32_t* __restrict__ ptr, int32_t* __restrict__ row, V* __restrict__ val,
                                   const int32_t* __restrict__ qpos, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t a = ptr[j], c = ptr[j + 1] - a;
    for (int32_t k = 0; k < c; ++k) {
        const int32_t q = row[a + k];
        row[a + k] = 2 * qpos[q >> 1] + (q & 1);
    }
    for (int32_t k = 1; k < c; ++k) {
        const int32_t key = row[a + k];
        const V v = val[a + k];
        int32_t q = k;
        while (q > 0 && row[a + q - 1] > key) {
            row[a + q] = row[a + q - 1];
            val[a + q] = val[a + q - 1];
            --q;
        }
        row[a + q] = key;
        val[a + q] = v;
    }
}

template <class T>
__global__ void k_move_pair_entries(const T* __restrict__ in, const uint32_t* __restrict__ order, int64_t npairs,
                                    T* __restrict__ out) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= npairs) return;
    out[2 * r] = in[2 * (int64_t)order[r]];
    out[2 * r + 1] = in[2 * (int64_t)order[r] + 1];
}

__global__ void k_store_maps(const int32_t* __restrict__ perm_inv, const uint32_t* __restrict__ order, int64_t m,
                             int32_t* __restrict__ row_of_store, int32_t* __restrict__ store_of_row) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m) return;
    const int64_t q = 2 * (int64_t)order[s >> 1] + (s & 1);
    const int32_t i = perm_inv[q];
    row_of_store[s] = i;
    store_of_row[i] = (int32_t)s;
}

template <class V>
__global__ void k_colnorm2(const int32_t* __restrict__ ptr, const V* __restrict__ vals, int64_t n,
                           double* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int32_t e = ptr[j]; e < ptr[j + 1]; ++e) {
        double v;
        if constexpr (sizeof(V) == 2) v = (double)__bfloat162float(vals[e]);
        else v = (double)vals[e];
        s += v * v;
    }
    out[j] = s;
}

// ---- IGen2 (Sec. 3.2, m < n): A = [B, N~] with B = L Sigma R^T square (m x m) ------------
constexpr int kNMax = 64;           // nonzeros per column of N
constexpr int kNTries = 4096;       // candidate rows drawn per column before giving up

// Column i of N~ (IGen2, Sec. 3.2): the first d distinct rows among draw(NROW, i*4096 + t) mod m
// (t = 0, 1, ...), the k-th accepted row with value 2 U(draw(NVAL, i*d + k)) - 1; then, in
// ascending row order, dot = N_i^T e and N~_i = xi_i tau / |dot| N_i (unscaled when dot = 0,
// where |N~_i^T e| <= tau holds anyway).  e and b are read in the stored row order
// (original row r is stored row perm[r]).  Writes rows (stored index) and values, the
// column's sum |N~_i| and |N~_i^T b| (for lambda_max).
__global__ void k_igen2_cols(uint64_t seed, int64_t m, int64_t ncols, int d, double tau,
                             const double* __restrict__ ehat, const double* __restrict__ bhat,
                             const int32_t* __restrict__ perm, int32_t* __restrict__ rows_out,
                             double* __restrict__ vals_out, double* __restrict__ col_abs, double* __restrict__ col_atb,
                             int* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncols) return;
    int64_t rows[kNMax];
    double v[kNMax];
    const uint64_t krow = sm_stream(seed, kTagNRow), kval = sm_stream(seed, kTagNVal);
    int cnt = 0;
    for (int64_t t = 0; cnt < d; ++t) {
        if (t >= kNTries) {
            atomicExch(err, 1);
            return;
        }
        const int64_t r = (int64_t)(sm_output(krow, (uint64_t)(i * kNTries + t)) % (uint64_t)m);
        bool seen = false;
        for (int k = 0; k < cnt; ++k) seen |= rows[k] == r;
        if (seen) continue;
        rows[cnt] = r;
        v[cnt] = __dadd_rn(2.0 * u01(sm_output(kval, (uint64_t)(i * d + cnt))), -1.0);
        ++cnt;
    }
    for (int a = 1; a < d; ++a) {                 // ascending rows (insertion sort)
        const int64_t r = rows[a];
        const double x = v[a];
        int k = a - 1;
        for (; k >= 0 && rows[k] > r; --k) {
            rows[k + 1] = rows[k];
            v[k + 1] = v[k];
        }
        rows[k + 1] = r;
        v[k + 1] = x;
    }
    double dot = 0.0;
    for (int k = 0; k < d; ++k) dot = __dadd_rn(dot, __dmul_rn(v[k], ehat[perm[rows[k]]]));
    if (dot != 0.0) {
        const double xi = __dadd_rn(2.0 * u01(sm_output(sm_stream(seed, kTagXi), (uint64_t)i)), -1.0);
        const double scale = __ddiv_rn(__dmul_rn(xi, tau), fabs(dot));
        for (int k = 0; k < d; ++k) v[k] = __dmul_rn(scale, v[k]);
    }
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < d; ++k) {
        rows_out[i * d + k] = perm[rows[k]];
        vals_out[i * d + k] = v[k];
        sa += fabs(v[k]);
        sb = __dadd_rn(sb, __dmul_rn(v[k], bhat[perm[rows[k]]]));
    }
    col_abs[i] = sa;
    col_atb[i] = fabs(sb);
}

__global__ void k_fill_i32(int32_t* __restrict__ out, int64_t count, int32_t v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = v;
}

// CSC -> CSR for IGen2 (any structure): per-row counts, scatter, then each row sorted by
// column so the result does not depend on the order of the atomic scatter.
__global__ void k_row_counts(const int32_t* __restrict__ row, int64_t nnz, int32_t* __restrict__ cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(cnt + row[e], 1);
}
__global__ void k_scatter_rows(const int32_t* __restrict__ cptr, const int32_t* __restrict__ row,
                               const double* __restrict__ cval, int64_t n, int32_t* __restrict__ fill,
                               int32_t* __restrict__ rcol, double* __restrict__ rval) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int32_t e = cptr[j]; e < cptr[j + 1]; ++e) {
        const int32_t pos = atomicAdd(fill + row[e], 1);
        rcol[pos] = (int32_t)j;
        rval[pos] = cval[e];
    }
}
__global__ void k_sort_rows(const int32_t* __restrict__ rptr, int64_t m, int32_t* __restrict__ rcol,
                            double* __restrict__ rval) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const int32_t b = rptr[r], e = rptr[r + 1];
    for (int32_t a = b + 1; a < e; ++a) {
        const int32_t c = rcol[a];
        const double x = rval[a];
        int32_t k = a - 1;
        for (; k >= b && rcol[k] > c; --k) {
            rcol[k + 1] = rcol[k];
            rval[k + 1] = rval[k];
        }
        rcol[k + 1] = c;
        rval[k + 1] = x;
    }
}
// per row: sum |a_rj| over the columns j >= m0 (the N~ part; sorted rows keep it last)
__global__ void k_row_abs_tail(const int32_t* __restrict__ rptr, const int32_t* __restrict__ rcol,
                               const double* __restrict__ rval, int64_t m, int64_t m0, double* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double s = 0.0;
    for (int32_t e = rptr[r]; e < rptr[r + 1]; ++e)
        if (rcol[e] >= m0) s += fabs(rval[e]);
    out[r] = s;
}

inline unsigned nblk(int64_t count, int b = 256) { return (unsigned)((count + b - 1) / b); }

struct TempList {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit TempList(cudaStream_t s) : st(s) {}
    template <class T> l1ls_status get(T** p, int64_t count) {
        cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (size_t)(count > 0 ? count : 1), st);
        if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(temp)", __FILE__, __LINE__);
        ptrs.push_back(*p);
        return L1LS_OK;
    }
    ~TempList() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

l1ls_status argsort_stream(uint64_t seed, uint64_t tag, int64_t count, uint32_t* order, TempList& tmp,
                           cudaStream_t st) {
    uint64_t* keys = nullptr;
    L1LS_TRY(tmp.get(&keys, count));
    k_keys<<<nblk(count), 256, 0, st>>>(seed, tag, count, keys);
    L1LS_CUDA(cudaGetLastError());
    return radix_argsort_u64(keys, count, order, st);
}

template <class V>
l1ls_status cast_and_norms(Inst* I, const double* csc64, const double* csr64, cudaStream_t st) {
    V* cv = nullptr;
    V* rv = nullptr;
    L1LS_TRY(I->alloc_n(&cv, I->nnz + kPad));
    L1LS_TRY(I->alloc_n(&rv, I->nnz + kPad));
    L1LS_CUDA(cudaMemsetAsync(cv + I->nnz, 0, sizeof(V) * kPad, st));
    L1LS_CUDA(cudaMemsetAsync(rv + I->nnz, 0, sizeof(V) * kPad, st));
    k_cast<V><<<nblk(I->nnz), 256, 0, st>>>(csc64, I->nnz, cv);
    k_cast<V><<<nblk(I->nnz), 256, 0, st>>>(csr64, I->nnz, rv);
    k_colnorm2<V><<<nblk(I->n), 256, 0, st>>>(I->csc_ptr, cv, I->n, I->colnorm2);
    L1LS_CUDA(cudaGetLastError());
    I->csc_val = cv;
    I->csr_val = rv;
    if (I->p.left_stages == 1 && I->m >= I->n) {   // paired storage (IGen only)
        const int64_t np = I->nnz / 2, npairs = I->m / 2;
        V* pv = nullptr;
        V* qv = nullptr;
        L1LS_TRY(I->alloc_n(&I->prow_ptr, npairs + 1));
        L1LS_TRY(I->alloc_n(&I->prow_col, np + kPad));
        L1LS_TRY(I->alloc_n(&pv, 2 * (np + kPad)));
        L1LS_TRY(I->alloc_n(&I->pcol_ptr, I->n + 1));
        L1LS_TRY(I->alloc_n(&I->pcol_pair, np + kPad));
        L1LS_TRY(I->alloc_n(&qv, 2 * (np + kPad)));
        L1LS_CUDA(cudaMemsetAsync(I->prow_col + np, 0, sizeof(int32_t) * kPad, st));
        L1LS_CUDA(cudaMemsetAsync(I->pcol_pair + np, 0, sizeof(int32_t) * kPad, st));
        L1LS_CUDA(cudaMemsetAsync(pv + 2 * np, 0, sizeof(V) * 2 * kPad, st));
        L1LS_CUDA(cudaMemsetAsync(qv + 2 * np, 0, sizeof(V) * 2 * kPad, st));
        k_pair_rows<V><<<nblk(npairs + 1), 256, 0, st>>>(I->csr_ptr, I->csr_col, rv, npairs, I->prow_ptr,
                                                          I->prow_col, pv, I->dev_err);
        k_pair_cols<V><<<nblk(I->n + 1), 256, 0, st>>>(I->csc_ptr, I->csc_row, cv, I->n, I->pcol_ptr, I->pcol_pair,
                                                        qv, I->dev_err);
        L1LS_CUDA(cudaGetLastError());
        I->prow_val = pv;
        I->pcol_val = qv;
        I->paired = true;
    }
    return L1LS_OK;
}

l1ls_status argsort_stream(uint64_t seed, uint64_t tag, int64_t count, uint32_t* order, TempList& tmp,
                           cudaStream_t st);

template <class V>
l1ls_status reorder_pairs(Inst* I, cudaStream_t st) {
    const int64_t m = I->m, n = I->n, npairs = m / 2, nnz = I->nnz, np = nnz / 2;
    TempList tmp(st);
    uint64_t* keys = nullptr;
    uint32_t* order = nullptr;
    int32_t *qpos = nullptr, *cnt = nullptr, *nptr = nullptr, *ncol = nullptr, *nrptr = nullptr, *nrcol = nullptr;
    V *nval = nullptr, *nrval = nullptr;
    L1LS_TRY(tmp.get(&keys, npairs));
    L1LS_TRY(tmp.get(&order, npairs));
    L1LS_TRY(tmp.get(&qpos, npairs));
    L1LS_TRY(tmp.get(&cnt, npairs));
    L1LS_TRY(tmp.get(&nptr, npairs + 1));
    L1LS_TRY(tmp.get(&ncol, np + kPad));
    L1LS_TRY(tmp.get(&nval, 2 * (np + kPad)));
    L1LS_TRY(tmp.get(&nrptr, m + 1));
    L1LS_TRY(tmp.get(&nrcol, nnz + kPad));
    L1LS_TRY(tmp.get(&nrval, nnz + kPad));
    k_pair_keys<<<nblk(npairs), 256, 0, st>>>(I->perm, npairs, n, keys);
    L1LS_CUDA(cudaGetLastError());
    L1LS_TRY(radix_argsort_u64(keys, npairs, order, st));
    k_qpos<<<nblk(npairs), 256, 0, st>>>(order, npairs, qpos);
    k_pair_counts<<<nblk(npairs), 256, 0, st>>>(I->prow_ptr, order, npairs, cnt);
    L1LS_CUDA(cudaGetLastError());
    int64_t tot = 0;
    L1LS_TRY(exclusive_scan_i32(cnt, npairs, nptr, &tot, st));
    if (tot != np) return set_error(L1LS_ECUDA, "internal: pair reorder lost entries");
    const V* pv = static_cast<const V*>(I->prow_val);
    const V* rv = static_cast<const V*>(I->csr_val);
    k_move_pair_rows<V><<<nblk(npairs), 256, 0, st>>>(I->prow_ptr, I->prow_col, pv, order, npairs, nptr, ncol, nval);
    k_move_plain_rows<V><<<nblk(npairs + 1), 256, 0, st>>>(I->csr_ptr, I->csr_col, rv, order, npairs, nptr, nrptr,
                                                            nrcol, nrval);
    k_remap_pair_cols<V><<<nblk(n), 256, 0, st>>>(I->pcol_ptr, I->pcol_pair, static_cast<V*>(I->pcol_val), qpos, n);
    k_remap_plain_cols<V><<<nblk(n), 256, 0, st>>>(I->csc_ptr, I->csc_row, static_cast<V*>(I->csc_val), qpos, n);
    L1LS_CUDA(cudaGetLastError());
    L1LS_CUDA(cudaMemcpyAsync(I->prow_ptr, nptr, sizeof(int32_t) * (npairs + 1), cudaMemcpyDeviceToDevice, st));
    L1LS_CUDA(cudaMemcpyAsync(I->prow_col, ncol, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, st));
    L1LS_CUDA(cudaMemcpyAsync(I->prow_val, nval, sizeof(V) * 2 * np, cudaMemcpyDeviceToDevice, st));
    L1LS_CUDA(cudaMemcpyAsync(I->csr_ptr, nrptr, sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToDevice, st));
    L1LS_CUDA(cudaMemcpyAsync(I->csr_col, nrcol, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st));
    L1LS_CUDA(cudaMemcpyAsync(I->csr_val, nrval, sizeof(V) * nnz, cudaMemcpyDeviceToDevice, st));
    // right-hand side in the stored order
    double* nb = nullptr;
    L1LS_TRY(tmp.get(&nb, m));
    k_move_pair_entries<double><<<nblk(npairs), 256, 0, st>>>(I->bhat, order, npairs, nb);
    L1LS_CUDA(cudaMemcpyAsync(I->bhat, nb, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    if (I->bhat32) {
        float* nb32 = nullptr;
        L1LS_TRY(tmp.get(&nb32, m));
        k_move_pair_entries<float><<<nblk(npairs), 256, 0, st>>>(I->bhat32, order, npairs, nb32);
        L1LS_CUDA(cudaMemcpyAsync(I->bhat32, nb32, sizeof(float) * m, cudaMemcpyDeviceToDevice, st));
    }
    k_store_maps<<<nblk(m), 256, 0, st>>>(I->perm_inv, order, m, I->row_of_store, I->store_of_row);
    L1LS_CUDA(cudaGetLastError());
    L1LS_CUDA(cudaStreamSynchronize(st));
    return L1LS_OK;
}

// sigma_max^2 of the square factor: 1 for the log-spaced values (kappa^0), else the larger of
// the two alternating values
double sigma_max2(const l1ls_gen_params* p) {
    if (p->sigma_mode != 1) return 1.0;
    const double s = std::min(p->m, p->n) > 1 ? std::max(p->sigma_odd, p->sigma_even) : p->sigma_odd;
    return s * s;
}

l1ls_status validate(const l1ls_gen_params* p) {
    if (!p) return set_error(L1LS_EINVAL, "params is NULL");
    if (p->m < 2 || p->n < 2) return set_error(L1LS_EINVAL, "m and n must be >= 2");
    if (p->m > (uint64_t)INT32_MAX - 2 || p->n > (uint64_t)INT32_MAX - 2)
        return set_error(L1LS_EINVAL, "m and n must be below 2^31 - 2");
    if (p->m < p->n && (p->n_nnz_per_col < 1 || p->n_nnz_per_col > kNMax || (uint64_t)p->n_nnz_per_col > p->m))
        return set_error(L1LS_EINVAL, "IGen2 (m < n): n_nnz_per_col must be in [1, min(%d, m)]", kNMax);
    if (!(p->kappa >= 1.0) || !std::isfinite(p->kappa)) return set_error(L1LS_EINVAL, "kappa must be >= 1");
    if (!(p->tau > 0.0)) return set_error(L1LS_EINVAL, "tau must be > 0");
    if (p->right_stages < 1 || p->right_stages > kWMax)
        return set_error(L1LS_EINVAL, "right_stages must be in [1, %d]", kWMax);
    if (p->left_stages != 0 && p->left_stages != 1) return set_error(L1LS_EINVAL, "left_stages must be 0 or 1");
    if (p->left_stages == 1 && (p->m & 1)) return set_error(L1LS_EINVAL, "m must be even with a left stage");
    if (p->value_dtype < L1LS_F64 || p->value_dtype > L1LS_BF16) return set_error(L1LS_EINVAL, "bad value_dtype");
    if (p->matrix_free != 0 && p->matrix_free != 1) return set_error(L1LS_EINVAL, "matrix_free must be 0 or 1");
    if ((p->sigma_mode != 0 && p->sigma_mode != 1) || p->xstar_mode < 0 || p->xstar_mode > 2)
        return set_error(L1LS_EINVAL, "sigma_mode must be 0 or 1, xstar_mode 0, 1 or 2");
    if (p->xstar_mode == 2 && (p->m < p->n || !(p->gamma > 0.0)))
        return set_error(L1LS_EINVAL, "OsGen3 (xstar_mode 2) needs m >= n and gamma > 0");
    if (p->sigma_mode == 1 && !(p->sigma_odd > 0.0 && p->sigma_even > 0.0))
        return set_error(L1LS_EINVAL, "sigma_odd and sigma_even must be > 0");
    if (p->matrix_free && (p->m < p->n || p->value_dtype != L1LS_F32))
        return set_error(L1LS_EINVAL, "matrix_free instances need m >= n and FP32 value_dtype");
    if (!(p->xstar_lo >= 0.0) || !(p->xstar_hi >= p->xstar_lo)) return set_error(L1LS_EINVAL, "bad x* magnitudes");
    if (!(p->xstar_frac >= 0.0) || !(p->xstar_frac <= 1.0)) return set_error(L1LS_EINVAL, "xstar_frac must be in [0, 1]");
    return L1LS_OK;
}

}  // namespace

l1ls_status generate_instance(Ctx* ctx, const l1ls_gen_params* p, cudaStream_t st, Inst** out,
                              bool stream_ordered) {
    L1LS_TRY(validate(p));
    Inst* I = new Inst();
    I->ctx = ctx;
    I->stream_ordered = stream_ordered;
    I->alloc_st = st;
    I->p = *p;
    I->m = (int64_t)p->m;
    I->n = (int64_t)p->n;
    const bool igen2 = p->m < p->n;             // Procedure IGen2 (Sec. 3.2): A = [B, N~]
    I->nsq = igen2 ? (int64_t)p->m : (int64_t)p->n;
    I->igen2 = igen2;
    I->matrix_free = p->matrix_free != 0;
    I->dtype = p->value_dtype;
    int64_t s = (int64_t)std::floor(p->xstar_frac * (double)p->n + 0.5);
    if (s < 1) s = 1;
    if (s > I->m) s = I->m;
    if (s > I->n) s = I->n;
    I->s = s;
    const int64_t m = I->m, n = I->n, nsq = I->nsq;
    const double vt = std::isnan(p->vartheta) ? p->theta : p->vartheta;
    Geo g{m, nsq, p->right_stages, p->left_stages, std::cos(p->theta), std::sin(p->theta), std::cos(vt), std::sin(vt)};

    auto fail = [&](l1ls_status e) {
        I->free_all();
        delete I;
        return e;
    };
#define GEN_TRY(x)                          \
    do {                                    \
        l1ls_status s__ = (x);              \
        if (s__ != L1LS_OK) return fail(s__); \
    } while (0)
#define GEN_CUDA(x)                                                              \
    do {                                                                         \
        cudaError_t e__ = (x);                                                   \
        if (e__ != cudaSuccess) return fail(cuda_error(e__, #x, __FILE__, __LINE__)); \
    } while (0)

    {
        TempList tmp(st);
        // persistent vectors
        GEN_TRY(I->alloc_n(&I->sigma, nsq));
        GEN_TRY(I->alloc_n(&I->xstar, n));
        GEN_TRY(I->alloc_n(&I->bhat, pad32(m)));
        GEN_CUDA(cudaMemsetAsync(I->bhat, 0, sizeof(double) * pad32(m), st));
        GEN_TRY(I->alloc_n(&I->perm, m));
        GEN_TRY(I->alloc_n(&I->perm_inv, m));
        GEN_TRY(I->alloc_n(&I->store_of_row, m));
        GEN_TRY(I->alloc_n(&I->row_of_store, m));
        GEN_TRY(I->alloc_n(&I->colnorm2, n));
        if (I->dtype != L1LS_F64) {
            GEN_TRY(I->alloc_n(&I->bhat32, pad32(m)));
            GEN_CUDA(cudaMemsetAsync(I->bhat32, 0, sizeof(float) * pad32(m), st));
        }
        GEN_TRY(I->alloc_n(&I->dev_err, 1));
        GEN_CUDA(cudaMemsetAsync(I->dev_err, 0, sizeof(int), st));

        // singular values: sigma_i = kappa^(-rank_i/(n-1))
        uint32_t* order_n = nullptr;
        GEN_TRY(tmp.get(&order_n, n));
        if (p->sigma_mode == 1) {
            k_sigma_alt<<<nblk(nsq), 256, 0, st>>>(nsq, p->sigma_odd, p->sigma_even, I->sigma);
        } else {
            GEN_TRY(argsort_stream(p->seed, kTagSigma, nsq, order_n, tmp, st));
            k_sigma<<<nblk(nsq), 256, 0, st>>>(order_n, nsq, std::log(p->kappa), I->sigma);
        }
        GEN_CUDA(cudaGetLastError());
        // row permutation P (P1 = P2 = P)
        if (p->left_stages == 1) {
            uint32_t* order_m = nullptr;
            GEN_TRY(tmp.get(&order_m, m));
            GEN_TRY(argsort_stream(p->seed, kTagPerm, m, order_m, tmp, st));
            k_perm<<<nblk(m), 256, 0, st>>>(order_m, m, I->perm, I->perm_inv);
        } else {
            k_identity_perm<<<nblk(m), 256, 0, st>>>(m, I->perm, I->perm_inv);
        }
        GEN_CUDA(cudaGetLastError());
        double *gvec = nullptr, *vg = nullptr, *vx = nullptr, *ze = nullptr, *zb = nullptr, *ul = nullptr,
               *ehat = nullptr;
        GEN_TRY(tmp.get(&gvec, n));
        GEN_TRY(tmp.get(&vg, n));
        GEN_TRY(tmp.get(&vx, n));
        GEN_TRY(tmp.get(&ze, n));
        GEN_TRY(tmp.get(&zb, n));
        GEN_TRY(tmp.get(&ul, n));
        GEN_TRY(tmp.get(&ehat, m));
        uint8_t* flag = nullptr;
        GEN_TRY(tmp.get(&flag, n));
        GEN_CUDA(cudaMemsetAsync(flag, 0, n, st));
        if (p->xstar_mode == 2) {
            // Procedure OsGen3 (Sec. 6): x = G gamma (Sigma^T Sigma)^{-1} 1 (G orthonormal), then
            // the s1 = s/2 smallest nonzero and s - s1 largest |x_i| kept (ties by index)
            double* xo = vg;   // free until IGen's e is formed
            uint64_t* keys = nullptr;
            int* zeros = nullptr;
            GEN_TRY(tmp.get(&keys, n));
            GEN_TRY(tmp.get(&zeros, 1));
            GEN_CUDA(cudaMemsetAsync(zeros, 0, sizeof(int), st));
            k_gamma_over_sigma2<<<nblk(n), 256, 0, st>>>(I->sigma, n, p->gamma, xo);
            for (int k = 1; k <= p->right_stages; ++k)
                k_stage<<<nblk(n / 2 + 1), 256, 0, st>>>(xo, n, (k - 1) & 1, g.c, g.s, 0);
            k_abs_keys<<<nblk(n), 256, 0, st>>>(xo, n, keys, zeros);
            GEN_CUDA(cudaGetLastError());
            GEN_TRY(radix_argsort_u64(keys, n, order_n, st));
            const int64_t s1 = s / 2, s2 = s - s1;
            k_osgen3_flags<<<nblk(n), 256, 0, st>>>(order_n, n, zeros, s1, s2, flag);
            k_osgen3_xstar<<<nblk(n), 256, 0, st>>>(xo, flag, n, p->seed, p->g_offsupport, I->xstar, gvec);
            GEN_CUDA(cudaGetLastError());
            // kept: ranks [z, z + s1) and [max(z, n - s2), n), i.e. min(s, n - z) entries
            int hz = 0;
            GEN_CUDA(cudaMemcpyAsync(&hz, zeros, sizeof(int), cudaMemcpyDeviceToHost, st));
            GEN_CUDA(cudaStreamSynchronize(st));
            I->s = std::min<int64_t>(s, n - (int64_t)hz);
        } else {
        // support of x*: the s smallest keys (among the first m columns for IGen2)
        GEN_TRY(argsort_stream(p->seed, kTagSupport, nsq, order_n, tmp, st));
        k_support<<<nblk(s), 256, 0, st>>>(order_n, s, flag);
        if (p->xstar_mode == 1) {
            int32_t *fi = nullptr, *rank = nullptr;
            GEN_TRY(tmp.get(&fi, nsq));
            GEN_TRY(tmp.get(&rank, nsq + 1));
            k_flag_i32<<<nblk(nsq), 256, 0, st>>>(flag, nsq, fi);
            GEN_CUDA(cudaGetLastError());
            int64_t scount = 0;
            GEN_TRY(exclusive_scan_i32(fi, nsq, rank, &scount, st));
            k_xstar_alt<<<nblk(n), 256, 0, st>>>(n, nsq, flag, rank, scount / 2, p->xstar_lo, p->xstar_hi, p->seed,
                                                 p->g_offsupport, I->xstar, gvec);
        } else {
            k_xstar_g<<<nblk(n), 256, 0, st>>>(p->seed, n, nsq, flag, p->xstar_lo, p->xstar_hi, p->g_offsupport, I->xstar,
                                            gvec);
        }
        GEN_CUDA(cudaGetLastError());
        }
        // IGen's e (Sec. 3.1) by the route of Sec. 4: R^T g and R^T x* (T_w^T first).  IGen2's e,
        // e = tau B^{-T} g = tau L Sigma^{-1} R^T g, and b = B x* + e are the same expressions
        // on the square part (x* is zero on the columns of N).
        GEN_CUDA(cudaMemcpyAsync(vg, gvec, sizeof(double) * nsq, cudaMemcpyDeviceToDevice, st));
        GEN_CUDA(cudaMemcpyAsync(vx, I->xstar, sizeof(double) * nsq, cudaMemcpyDeviceToDevice, st));
        for (int k = p->right_stages; k >= 1; --k) {
            k_stage<<<nblk(nsq / 2 + 1), 256, 0, st>>>(vg, nsq, (k - 1) & 1, g.c, g.s, 1);
            k_stage<<<nblk(nsq / 2 + 1), 256, 0, st>>>(vx, nsq, (k - 1) & 1, g.c, g.s, 1);
        }
        k_scale<<<nblk(nsq), 256, 0, st>>>(vg, vx, I->sigma, nsq, p->tau, ze, zb, ul);
        k_left<<<nblk(m), 256, 0, st>>>(ze, zb, I->perm, g, ehat, I->bhat);
        // B^T b = R u (T_1 first) for lambda_max
        for (int k = 1; k <= p->right_stages; ++k)
            k_stage<<<nblk(nsq / 2 + 1), 256, 0, st>>>(ul, nsq, (k - 1) & 1, g.c, g.s, 0);
        GEN_CUDA(cudaGetLastError());
        double* red = nullptr;
        double* partials = nullptr;
        unsigned* counter = nullptr;
        GEN_TRY(tmp.get(&red, 3));
        GEN_TRY(tmp.get(&partials, 3 * 512));
        GEN_TRY(tmp.get(&counter, 1));
        GEN_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
        k_reduce3<<<512, 256, 0, st>>>(I->xstar, n, ehat, m, ul, nsq, partials, counter, red);
        GEN_CUDA(cudaGetLastError());
        double hred[3];
        GEN_CUDA(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, st));

        if (I->matrix_free) {
            // A stays in factored form: FP32 copies of the factors for the products; the rows are
            // kept in the order of the left rotations (row i of A is row perm[i] of it)
            int32_t* cnt = nullptr;
            GEN_TRY(tmp.get(&cnt, n));
            k_csc_count<<<nblk(n), 256, 0, st>>>(g, I->perm_inv, cnt);
            GEN_CUDA(cudaGetLastError());
            int64_t nnz = 0;
            GEN_TRY(sum_i32(cnt, n, &nnz, st));
            I->nnz = nnz;                         // of the matrix the factors represent (may exceed 2^31)
            GEN_TRY(I->alloc_n(&I->sigma32, pad32(n)));
            GEN_CUDA(cudaMemsetAsync(I->sigma32, 0, sizeof(float) * pad32(n), st));
            k_to_f32<<<nblk(n), 256, 0, st>>>(I->sigma, n, I->sigma32);
            if (p->left_stages == 1) {
                // row pairs in the order of the smaller of their two entries of P (as for the
                // stored matrix): one of the two gathers of each pair then runs in order
                const int64_t npairs = m / 2;
                uint64_t* keys = nullptr;
                uint32_t* order = nullptr;
                double* nb = nullptr;
                GEN_TRY(tmp.get(&keys, npairs));
                GEN_TRY(tmp.get(&order, npairs));
                GEN_TRY(tmp.get(&nb, m));
                k_pair_keys<<<nblk(npairs), 256, 0, st>>>(I->perm, npairs, n, keys);
                GEN_CUDA(cudaGetLastError());
                GEN_TRY(radix_argsort_u64(keys, npairs, order, st));
                GEN_TRY(I->alloc_n(&I->mf_pperm, m));
                k_move_pair_entries<int32_t><<<nblk(npairs), 256, 0, st>>>(I->perm, order, npairs, I->mf_pperm);
                k_move_pair_entries<double><<<nblk(npairs), 256, 0, st>>>(I->bhat, order, npairs, nb);
                GEN_CUDA(cudaMemcpyAsync(I->bhat, nb, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
                k_store_maps<<<nblk(m), 256, 0, st>>>(I->perm_inv, order, m, I->row_of_store, I->store_of_row);
            } else {
                GEN_CUDA(cudaMemcpyAsync(I->store_of_row, I->perm, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
                GEN_CUDA(cudaMemcpyAsync(I->row_of_store, I->perm_inv, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice,
                                         st));
            }
            k_to_f32<<<nblk(m), 256, 0, st>>>(I->bhat, m, I->bhat32);
            GEN_CUDA(cudaGetLastError());
            GEN_CUDA(cudaStreamSynchronize(st));
            I->mf_c = (float)g.c;
            I->mf_s = (float)g.s;
            I->mf_ct = (float)g.ct;
            I->mf_st = (float)g.st;
            I->mf_c64 = g.c;
            I->mf_s64 = g.s;
            I->mf_ct64 = g.ct;
            I->mf_st64 = g.st;
            I->f_star = p->tau * hred[0] + 0.5 * hred[1];
            I->lam_max = hred[2];
            I->lipschitz = sigma_max2(p);
            *out = I;
            return L1LS_OK;
        }

        // CSR(Ahat^T): counts, scan, fill (FP64 values)
        int32_t* cnt = nullptr;
        GEN_TRY(tmp.get(&cnt, (m > n ? m : n)));
        GEN_TRY(I->alloc_n(&I->csc_ptr, n + 1));
        k_csc_count<<<nblk(nsq), 256, 0, st>>>(g, I->perm_inv, cnt);
        const int d = p->n_nnz_per_col;
        if (igen2) k_fill_i32<<<nblk(n - nsq), 256, 0, st>>>(cnt + nsq, n - nsq, d);
        GEN_CUDA(cudaGetLastError());
        int64_t nnz = 0;
        GEN_TRY(exclusive_scan_i32(cnt, n, I->csc_ptr, &nnz, st));
        if (nnz > (int64_t)INT32_MAX - 2 * kPad)
            return fail(set_error(L1LS_EINVAL, "nnz = %lld does not fit 32-bit offsets", (long long)nnz));
        I->nnz = nnz;
        const int64_t nnz_sq = nnz - (n - nsq) * (int64_t)d * (igen2 ? 1 : 0);
        double *csc64 = nullptr, *csr64 = nullptr;
        GEN_TRY(I->alloc_n(&I->csc_row, nnz + kPad));
        GEN_CUDA(cudaMemsetAsync(I->csc_row + nnz, 0, sizeof(int32_t) * kPad, st));
        GEN_TRY(tmp.get(&csc64, nnz));
        k_csc_fill<<<nblk(nsq), 256, 0, st>>>(g, I->perm_inv, I->sigma, I->csc_ptr, I->csc_row, csc64);
        GEN_CUDA(cudaGetLastError());
        double *col_abs = nullptr, *col_atb = nullptr, *row_abs = nullptr, *red2 = nullptr;
        int* err_n = nullptr;
        if (igen2) {
            // IGen2 (Sec. 3.2): the columns of N~ after those of B
            GEN_TRY(tmp.get(&col_abs, n - nsq));
            GEN_TRY(tmp.get(&col_atb, n - nsq));
            GEN_TRY(tmp.get(&err_n, 1));
            GEN_CUDA(cudaMemsetAsync(err_n, 0, sizeof(int), st));
            k_igen2_cols<<<nblk(n - nsq, 128), 128, 0, st>>>(p->seed, m, n - nsq, d, p->tau, ehat, I->bhat, I->perm,
                                                             I->csc_row + nnz_sq, csc64 + nnz_sq, col_abs, col_atb,
                                                             err_n);
            GEN_CUDA(cudaGetLastError());
        }
        // CSR(Ahat): counts, scan, fill by lookup in CSR(Ahat^T)
        GEN_TRY(I->alloc_n(&I->csr_ptr, m + 1));
        if (igen2) {
            GEN_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * m, st));
            k_row_counts<<<nblk(nnz), 256, 0, st>>>(I->csc_row, nnz, cnt);
        } else {
            k_csr_count<<<nblk(m), 256, 0, st>>>(g, I->perm, cnt);
        }
        GEN_CUDA(cudaGetLastError());
        int64_t nnz_r = 0;
        GEN_TRY(exclusive_scan_i32(cnt, m, I->csr_ptr, &nnz_r, st));
        if (nnz_r != nnz)
            return fail(set_error(L1LS_ECUDA, "internal: row and column structures disagree (%lld vs %lld)",
                                  (long long)nnz_r, (long long)nnz));
        int* err = nullptr;
        GEN_TRY(tmp.get(&err, 1));
        GEN_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        GEN_TRY(I->alloc_n(&I->csr_col, nnz + kPad));
        GEN_CUDA(cudaMemsetAsync(I->csr_col + nnz, 0, sizeof(int32_t) * kPad, st));
        GEN_TRY(tmp.get(&csr64, nnz));
        if (igen2) {
            int32_t* fill = nullptr;
            GEN_TRY(tmp.get(&fill, m));
            GEN_CUDA(cudaMemcpyAsync(fill, I->csr_ptr, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
            k_scatter_rows<<<nblk(n), 256, 0, st>>>(I->csc_ptr, I->csc_row, csc64, n, fill, I->csr_col, csr64);
            k_sort_rows<<<nblk(m), 256, 0, st>>>(I->csr_ptr, m, I->csr_col, csr64);
            // step size: sigma_max^2 + ||N~||_1 ||N~||_inf, and lambda_max over the columns of N~
            GEN_TRY(tmp.get(&row_abs, m));
            GEN_TRY(tmp.get(&red2, 9));
            k_row_abs_tail<<<nblk(m), 256, 0, st>>>(I->csr_ptr, I->csr_col, csr64, m, nsq, row_abs);
            GEN_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
            k_reduce3<<<512, 256, 0, st>>>(nullptr, 0, nullptr, 0, col_abs, n - nsq, partials, counter, red2);
            GEN_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
            k_reduce3<<<512, 256, 0, st>>>(nullptr, 0, nullptr, 0, row_abs, m, partials, counter, red2 + 3);
            GEN_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
            k_reduce3<<<512, 256, 0, st>>>(nullptr, 0, nullptr, 0, col_atb, n - nsq, partials, counter, red2 + 6);
        } else {
            k_csr_fill<<<nblk(m), 256, 0, st>>>(g, I->perm, I->csc_ptr, I->csc_row, csc64, I->csr_ptr, I->csr_col,
                                                 csr64, err);
        }
        GEN_CUDA(cudaGetLastError());
        switch (I->dtype) {
            case L1LS_F64: GEN_TRY(cast_and_norms<double>(I, csc64, csr64, st)); break;
            case L1LS_F32: GEN_TRY(cast_and_norms<float>(I, csc64, csr64, st)); break;
            default: GEN_TRY(cast_and_norms<__nv_bfloat16>(I, csc64, csr64, st)); break;
        }
        if (I->bhat32) k_to_f32<<<nblk(m), 256, 0, st>>>(I->bhat, m, I->bhat32);
        GEN_CUDA(cudaGetLastError());
        if (I->paired) {   // (never for IGen2: the columns of N~ do not keep row pairs together)
            switch (I->dtype) {
                case L1LS_F64: GEN_TRY(reorder_pairs<double>(I, st)); break;
                case L1LS_F32: GEN_TRY(reorder_pairs<float>(I, st)); break;
                default: GEN_TRY(reorder_pairs<__nv_bfloat16>(I, st)); break;
            }
        } else {
            GEN_CUDA(cudaMemcpyAsync(I->store_of_row, I->perm, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
            GEN_CUDA(cudaMemcpyAsync(I->row_of_store, I->perm_inv, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
        }
        GEN_CUDA(cudaGetLastError());
        int* tmax = nullptr;
        GEN_TRY(tmp.get(&tmax, 2));
        GEN_CUDA(cudaMemsetAsync(tmax, 0, 2 * sizeof(int), st));
        k_tile_max<<<nblk((m + 31) / 32), 256, 0, st>>>(I->csr_ptr, m, tmax);
        k_tile_max<<<nblk((n + 31) / 32), 256, 0, st>>>(I->csc_ptr, n, tmax + 1);
        GEN_CUDA(cudaGetLastError());
        int htmax[2] = {0, 0};
        GEN_CUDA(cudaMemcpyAsync(htmax, tmax, sizeof(htmax), cudaMemcpyDeviceToHost, st));
        int herr = 0, herr2 = 0, herr3 = 0;
        double hred2[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        GEN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        GEN_CUDA(cudaMemcpyAsync(&herr2, I->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (igen2) {
            GEN_CUDA(cudaMemcpyAsync(&herr3, err_n, sizeof(int), cudaMemcpyDeviceToHost, st));
            GEN_CUDA(cudaMemcpyAsync(hred2, red2, sizeof(hred2), cudaMemcpyDeviceToHost, st));
        }
        GEN_CUDA(cudaStreamSynchronize(st));
        if (herr3) return fail(set_error(L1LS_EINVAL, "IGen2: %d distinct rows of %lld not found in %d draws", d,
                                         (long long)m, kNTries));
        if (herr) return fail(set_error(L1LS_ECUDA, "internal: an entry of CSR(A) was not found in CSR(A^T)"));
        if (herr2) return fail(set_error(L1LS_ECUDA, "internal: the paired storage found unpaired rows (%d)", herr2));
        I->csr_tile_max = htmax[0];
        I->csc_tile_max = htmax[1];
        I->f_star = p->tau * hred[0] + 0.5 * hred[1];
        I->lam_max = hred[2];
        I->lipschitz = sigma_max2(p);   // lambda_max(A^T A) = sigma_max^2
        if (igen2) {
            // hred2: [2] max column sum |N~|, [5] max row sum |N~|, [8] max |N~^T b|
            I->lipschitz = sigma_max2(p) + hred2[2] * hred2[5];
            I->lam_max = std::max(I->lam_max, hred2[8]);
        }
    }
    GEN_CUDA(cudaStreamSynchronize(st));
#undef GEN_TRY
#undef GEN_CUDA
    *out = I;
    return L1LS_OK;
}

// kappa_rho(x*) of Eq. (bd12): R^T x* by the stages (T_w^T first), then the two sums
l1ls_status kappa_rho(const Inst* I, double rho, double* out) {
    if (I->igen2) return set_error(L1LS_EINVAL, "kappa_rho is defined for IGen instances (m >= n)");
    if (std::isnan(rho)) return set_error(L1LS_EINVAL, "rho is NaN");
    const int64_t n = I->n;
    const l1ls_gen_params& p = I->p;
    cudaStream_t st = nullptr;
    L1LS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    double hsum[2] = {0.0, 0.0};
    l1ls_status rc = L1LS_OK;
    {
        TempList tmp(st);
        double *z = nullptr, *partials = nullptr, *sums = nullptr;
        unsigned* counter = nullptr;
        rc = tmp.get(&z, n);
        if (rc == L1LS_OK) rc = tmp.get(&partials, 2 * 512);
        if (rc == L1LS_OK) rc = tmp.get(&sums, 2);
        if (rc == L1LS_OK) rc = tmp.get(&counter, 1);
        cudaError_t e = cudaSuccess;
        if (rc == L1LS_OK) {
            e = cudaMemcpyAsync(z, I->xstar, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
            const double c = std::cos(p.theta), s = std::sin(p.theta);
            for (int k = p.right_stages; k >= 1 && e == cudaSuccess; --k) {
                k_stage<<<nblk(n / 2 + 1), 256, 0, st>>>(z, n, (k - 1) & 1, c, s, 1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                k_kappa_sums<<<512, 256, 0, st>>>(I->xstar, z, I->sigma, n, rho, partials, counter, sums);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(hsum, sums, sizeof(hsum), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_error(e, "kappa_rho", __FILE__, __LINE__);
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc != L1LS_OK) return rc;
    if (e2 != cudaSuccess) return cuda_error(e2, "kappa_rho", __FILE__, __LINE__);
    *out = hsum[1] == 0.0 ? INFINITY : std::sqrt(hsum[0]) / std::sqrt(hsum[1]);
    return L1LS_OK;
}

}  // namespace l1ls
