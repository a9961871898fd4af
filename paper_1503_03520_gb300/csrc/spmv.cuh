// CSR "stream" traversal shared by every product kernel.
//
// A CTA owns a tile of BLOCK consecutive rows.  It stages the tile's row pointers in
// shared memory, then streams the tile's nonzeros (values and column indices, read once
// with evict-first loads) in coalesced chunks of CAP entries, gathers the vector entry
// of each nonzero and stores the product in shared memory; thread t then sums the
// products of row t in nonzero order.  Rows of the generated matrices hold 0-16 entries,
// so a thread per row keeps the sums short while the loads stay fully coalesced.
// Persistent kernels walk tiles tile = blockIdx.x + k * gridDim.x, which fixes the order
// of every reduction for a given grid.
#pragma once

#include "common.cuh"

namespace l1ls {

template <class T> __device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ld_stream<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(u);
}

template <class Acc, class V> __device__ __forceinline__ Acc val_to_acc(V v);
template <> __device__ __forceinline__ double val_to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float val_to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float val_to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class Acc, class X> __device__ __forceinline__ Acc vec_to_acc(X v);
template <> __device__ __forceinline__ double vec_to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double vec_to_acc<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ float vec_to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float vec_to_acc<float, double>(double v) { return (float)v; }

template <int BLOCK, int CAP, class Acc>
struct CsrSmem {
    Acc prod[CAP];
    int32_t ptr[BLOCK + 1];
};

// Row sums of one tile [r0, r0 + nr); returns the sum of row r0 + threadIdx.x (0 if outside).
template <int BLOCK, int CAP, class V, class X, class Acc>
__device__ __forceinline__ Acc csr_tile(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                        const V* __restrict__ val, const X* __restrict__ x, int64_t r0, int nr,
                                        CsrSmem<BLOCK, CAP, Acc>& sm) {
    for (int i = threadIdx.x; i <= nr; i += BLOCK) sm.ptr[i] = __ldcs(ptr + r0 + i);
    __syncthreads();
    const int32_t e0 = sm.ptr[0], e1 = sm.ptr[nr];
    const int t = threadIdx.x;
    const int32_t rb = t < nr ? sm.ptr[t] : e1;
    const int32_t re = t < nr ? sm.ptr[t + 1] : e1;
    Acc acc = Acc(0);
    for (int32_t c = e0; c < e1; c += CAP) {
        const int32_t ce = min(c + CAP, e1);
#pragma unroll 4
        for (int32_t e = c + t; e < ce; e += BLOCK) {
            const int32_t j = ld_stream(col + e);
            sm.prod[e - c] = val_to_acc<Acc>(ld_stream(val + e)) * vec_to_acc<Acc>(__ldg(x + j));
        }
        __syncthreads();
        const int32_t lo = max(rb, c), hi = min(re, ce);
        for (int32_t e = lo; e < hi; ++e) acc += sm.prod[e - c];
        __syncthreads();
    }
    return acc;
}

}  // namespace l1ls
