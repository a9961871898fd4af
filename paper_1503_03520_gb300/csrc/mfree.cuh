// Matrix-free application of A = L Sigma R^T (Eq. bd8) by its factors, the device form of
// Algorithms MvPA / MvPAt (Sec. 4).  FP32 vectors; the rotations use FP32 cos / sin.
//
//   A x   : z = Sigma R^T x  (the stages T_w^T ... T_1^T, then Sigma), then per row pair t of
//           the left factor y_(2t, 2t+1) = G~ (z_perm[2t], z_perm[2t+1]) (entries >= n of the
//           padded [z; 0] are zero); without a left stage y = [z; 0].
//   A^T y : per row pair (u0, u1) = G~^T (y_2t, y_2t+1) scattered to z_perm[2t], z_perm[2t+1]
//           (those < n), then x = R Sigma z (Sigma, then T_1 ... T_w).
// Rows are stored in the row pairs of the left rotations (rows 2t, 2t+1 of stored pair t), the
// pairs in the order of the smaller of their two entries of P, so one of the two entries of z
// a pair reads (or writes) runs in order; L.perm lists both entries per stored pair.
//
// The stage sweeps work on tiles of kMfTile entries loaded with a halo of kMfHalo >= w entries
// on each side: each stage mixes neighbouring pairs, so after w stages the tile's own entries
// are exact (a pair straddling two tiles is computed identically by both).
#pragma once

#include "common.cuh"

namespace l1ls {

constexpr int kMfThreads = 256;
constexpr int kMfTile = 2048;
constexpr int kMfHalo = 8;
constexpr int kMfLen = kMfTile + 2 * kMfHalo;

struct MfRight {
    int64_t n;
    int w;
    float c, s;
};

struct MfLeft {
    int64_t m, n;
    int left;              // 0: L = I; 1: one stage of left rotations after the permutation
    float ct, st;
    const int32_t* perm;   // row pair t (stored order) of the left stage takes z_perm[2t], z_perm[2t+1]
};

// Every block that uses these helpers has kMfThreads threads: the loops below stride by the
// constant so that each thread's loads of a tile are unrolled and all in flight at once.
constexpr int kMfPerThread = (kMfLen + kMfThreads - 1) / kMfThreads;

// buf[p] = v[g0 + p] (0 outside [0, n)), scaled by sigma when SCALE; g0 = a - kMfHalo
template <bool SCALE>
__device__ __forceinline__ void mf_load(float* buf, const float* __restrict__ v, const float* __restrict__ sigma,
                                        int64_t g0, int64_t n) {
    float xv[kMfPerThread], sv[kMfPerThread];
#pragma unroll
    for (int u = 0; u < kMfPerThread; ++u) {
        const int p = (int)threadIdx.x + u * kMfThreads;
        const int64_t i = g0 + p;
        xv[u] = 0.0f;
        sv[u] = 1.0f;
        if (p < kMfLen && i >= 0 && i < n) {
            xv[u] = __ldcs(v + i);
            if (SCALE) sv[u] = __ldg(sigma + i);
        }
    }
#pragma unroll
    for (int u = 0; u < kMfPerThread; ++u) {
        const int p = (int)threadIdx.x + u * kMfThreads;
        if (p < kMfLen) buf[p] = SCALE ? xv[u] * sv[u] : xv[u];
    }
    __syncthreads();
}

// The stages of R on buf (buf[0] is entry g0): TRANS ? T_w^T ... T_1^T : T_1 ... T_w, stage k on
// the planes (i, i+1) with i = (k - 1) mod 2 + 2j (Sec. 4.2).
template <bool TRANS>
__device__ __forceinline__ void mf_stages(float* buf, int64_t g0, const MfRight& R) {
    for (int q = 0; q < R.w; ++q) {
        const int k = TRANS ? R.w - q : q + 1;
        const int first = (k - 1) & 1;
        const int p0 = (int)(((first - g0) % 2 + 2) % 2);   // first local index with i = first (mod 2)
        for (int p = p0 + 2 * (int)threadIdx.x; p + 1 < kMfLen; p += 2 * kMfThreads) {
            const int64_t i = g0 + p;
            if (i < 0 || i + 1 >= R.n) continue;
            const float a = buf[p], b = buf[p + 1];
            if (TRANS) {
                buf[p] = __fmaf_rn(R.c, a, R.s * b);
                buf[p + 1] = __fmaf_rn(R.c, b, -R.s * a);
            } else {
                buf[p] = __fmaf_rn(R.c, a, -R.s * b);
                buf[p + 1] = __fmaf_rn(R.c, b, R.s * a);
            }
        }
        __syncthreads();
    }
}

// The same stages on a buffer of LEN entries of type T (FP32 or FP64) with the rotation (c, s)
// given in that type: the tile kernels of matrix-free pdNCG, whose buffers carry a halo of
// 2 kMfHalo (R^T and R applied in one pass) and whose gradient sweep runs in FP64.
template <bool TRANS, class T, int LEN>
__device__ __forceinline__ void mf_stages_t(T* buf, int64_t g0, int64_t n, int w, T c, T s) {
    for (int q = 0; q < w; ++q) {
        const int k = TRANS ? w - q : q + 1;
        const int first = (k - 1) & 1;
        const int p0 = (int)(((first - g0) % 2 + 2) % 2);
        for (int p = p0 + 2 * (int)threadIdx.x; p + 1 < LEN; p += 2 * kMfThreads) {
            const int64_t i = g0 + p;
            if (i < 0 || i + 1 >= n) continue;
            const T a = buf[p], b = buf[p + 1];
            if (TRANS) {
                buf[p] = fma(c, a, s * b);
                buf[p + 1] = fma(c, b, -s * a);
            } else {
                buf[p] = fma(c, a, -s * b);
                buf[p + 1] = fma(c, b, s * a);
            }
        }
        __syncthreads();
    }
}

// y values of left row pair t (rows 2t, 2t+1) from z; L = I: row t alone (y1 unused)
__device__ __forceinline__ void mf_left_rows(const MfLeft& L, const float* __restrict__ z, int64_t t, float& y0,
                                             float& y1) {
    if (L.left == 0) {
        y0 = t < L.n ? __ldg(z + t) : 0.0f;
        y1 = 0.0f;
        return;
    }
    const int2 k = __ldcs(reinterpret_cast<const int2*>(L.perm) + t);
    const float z0 = k.x < L.n ? __ldg(z + k.x) : 0.0f;
    const float z1 = k.y < L.n ? __ldg(z + k.y) : 0.0f;
    y0 = __fmaf_rn(L.ct, z0, -L.st * z1);
    y1 = __fmaf_rn(L.ct, z1, L.st * z0);
}

// z entries of left row pair t from y (rows 2t, 2t+1): the transpose of mf_left_rows
__device__ __forceinline__ void mf_left_scatter(const MfLeft& L, float* __restrict__ z, int64_t t, float y0, float y1) {
    if (L.left == 0) {
        if (t < L.n) z[t] = y0;
        return;
    }
    const int2 k = __ldcs(reinterpret_cast<const int2*>(L.perm) + t);
    if (k.x < L.n) z[k.x] = __fmaf_rn(L.ct, y0, L.st * y1);
    if (k.y < L.n) z[k.y] = __fmaf_rn(L.ct, y1, -L.st * y0);
}

}  // namespace l1ls
