// Matrix-free products y = A x and x = A^T y of instances generated with matrix_free = 1
// (Algorithms MvPA / MvPAt of Sec. 4; see mfree.cuh).  Each product is two launches: the
// stage sweep over the n-vector and the pass over the rows of the left factor.
#include "internal.h"
#include "mfree.cuh"

namespace l1ls {

namespace {

// Algorithms MvPA / MvPAt (Sec. 4): the stages of the right factor applied to a vector
__global__ void __launch_bounds__(kMfThreads) k_mf_rt(const float* __restrict__ x, const float* __restrict__ sigma,
                                                      MfRight R, float* __restrict__ z) {
    __shared__ float buf[kMfLen];
    constexpr int kPer = kMfTile / kMfThreads;
    const int64_t a = (int64_t)blockIdx.x * kMfTile;
    float sg[kPer];   // sigma of this thread's outputs, loaded before the sweep
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int64_t i = a + (int)threadIdx.x + u * kMfThreads;
        sg[u] = i < R.n ? __ldg(sigma + i) : 0.0f;
    }
    mf_load<false>(buf, x, sigma, a - kMfHalo, R.n);
    mf_stages<true>(buf, a - kMfHalo, R);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int p = (int)threadIdx.x + u * kMfThreads;
        const int64_t i = a + p;
        if (i < R.n) z[i] = buf[kMfHalo + p] * sg[u];
    }
}

__global__ void __launch_bounds__(kMfThreads) k_mf_r(const float* __restrict__ z, const float* __restrict__ sigma,
                                                     MfRight R, float* __restrict__ x) {
    __shared__ float buf[kMfLen];
    const int64_t a = (int64_t)blockIdx.x * kMfTile;
    mf_load<true>(buf, z, sigma, a - kMfHalo, R.n);
    mf_stages<false>(buf, a - kMfHalo, R);
    for (int p = threadIdx.x; p < kMfTile; p += kMfThreads) {
        const int64_t i = a + p;
        if (i < R.n) x[i] = buf[kMfHalo + p];
    }
}

// rows of A x (MvPA, Sec. 4: the left factor's rotations): row h (stored order) written to y[map[h]] (map NULL: y[h])
__global__ void k_mf_rows(MfLeft L, const float* __restrict__ z, const int32_t* __restrict__ map, float* __restrict__ y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t units = L.left ? L.m / 2 : L.m;
    if (t >= units) return;
    float y0, y1;
    mf_left_rows(L, z, t, y0, y1);
    if (L.left) {
        y[map ? map[2 * t] : 2 * t] = y0;
        y[map ? map[2 * t + 1] : 2 * t + 1] = y1;
    } else {
        y[map ? map[t] : t] = y0;
    }
}

// z = the first n entries of P2^T G~^T y; row h of the stored order read from y[map[h]]
__global__ void k_mf_scatter(MfLeft L, const float* __restrict__ y, const int32_t* __restrict__ map,
                             float* __restrict__ z) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t units = L.left ? L.m / 2 : L.m;
    if (t >= units) return;
    if (L.left) {
        const float y0 = y[map ? map[2 * t] : 2 * t], y1 = y[map ? map[2 * t + 1] : 2 * t + 1];
        mf_left_scatter(L, z, t, y0, y1);
    } else {
        mf_left_scatter(L, z, t, y[map ? map[t] : t], 0.0f);
    }
}

inline unsigned blocks_of(int64_t count, int per) { return (unsigned)((count + per - 1) / per); }

}  // namespace

MfRight mf_right(const Inst* I) { return MfRight{I->n, I->p.right_stages, I->mf_c, I->mf_s}; }
MfLeft mf_left(const Inst* I) { return MfLeft{I->m, I->n, I->p.left_stages, I->mf_ct, I->mf_st, I->mf_pperm}; }

// z = Sigma R^T x (the first launch of A x)
l1ls_status mf_apply_rt(const Inst* I, const float* x, float* z, cudaStream_t st) {
    k_mf_rt<<<blocks_of(I->n, kMfTile), kMfThreads, 0, st>>>(x, I->sigma32, mf_right(I), z);
    return L1LS_OK;
}

// transpose = false: out (m) = A in (n); true: out (n) = A^T in (m).  The m-vector's row h of
// the stored order is entry map[h] (map NULL: h).  z: n floats of scratch.
l1ls_status mf_product(const Inst* I, bool transpose, const float* in, float* out, const int32_t* map, float* z,
                       cudaStream_t st) {
    const MfRight R = mf_right(I);
    const MfLeft L = mf_left(I);
    const int64_t units = L.left ? I->m / 2 : I->m;
    if (!transpose) {
        k_mf_rt<<<blocks_of(I->n, kMfTile), kMfThreads, 0, st>>>(in, I->sigma32, R, z);
        k_mf_rows<<<blocks_of(units, 256), 256, 0, st>>>(L, z, map, out);
    } else {
        k_mf_scatter<<<blocks_of(units, 256), 256, 0, st>>>(L, in, map, z);
        k_mf_r<<<blocks_of(I->n, kMfTile), kMfThreads, 0, st>>>(z, I->sigma32, R, out);
    }
    L1LS_CUDA(cudaGetLastError());
    return L1LS_OK;
}

}  // namespace l1ls
