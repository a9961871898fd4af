// CSR traversal shared by every product kernel: one warp per tile of 32 rows.
//
// Lane l owns row r0 + l.  The warp streams the tile's nonzeros (values and column indices,
// read once with 16-byte evict-first vector loads, kEPL = 8 consecutive entries per lane, so
// a chunk covers 256 entries) from the 16-byte-aligned position at or below the tile's first
// entry; entries outside the tile are masked before their vector entry is gathered.  The
// products go to a warp-private shared-memory buffer and lane l sums the entries of its own
// row in nonzero order, so every row sum has a fixed order.  Rows of the generated matrices
// hold 0-16 entries.  No block-wide barrier is involved: warps advance independently and
// the epilogue operands of a tile are loaded before its nonzeros, so the memory system sees
// the loads of many tiles at once.  Warps walk tiles tile = warp_id + k * total_warps.
//
// Nonzero arrays must be allocated with kPad entries of slack after nnz (vector tails).
#pragma once

#include "common.cuh"

namespace l1ls {

constexpr int kEPL = 8;       // nonzeros per lane per chunk
constexpr int kPad = kEPL;    // slack entries after the nonzero arrays
constexpr int kWarpChunk = 32 * kEPL;
// nonzeros per lane and chunk of the paired traversal (a build parameter, 4 or 8)
#ifndef L1LS_PAIRED_EPL
#define L1LS_PAIRED_EPL 8
#endif
constexpr int kPEPL = L1LS_PAIRED_EPL;
static_assert(kPEPL == 4 || kPEPL == 8, "paired traversal: 4 or 8 nonzeros per lane");

template <class Acc, class V> __device__ __forceinline__ Acc val_to_acc(V v);
template <> __device__ __forceinline__ double val_to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float val_to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float val_to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class Acc, class X> __device__ __forceinline__ Acc vec_to_acc(X v);
template <> __device__ __forceinline__ double vec_to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double vec_to_acc<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ float vec_to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float vec_to_acc<float, double>(double v) { return (float)v; }

// kEPL consecutive entries starting at a 16-byte-aligned address, streaming loads
template <class T>
__device__ __forceinline__ void load_run(const T* __restrict__ p, T (&out)[kEPL]) {
    constexpr int kVecs = (int)(kEPL * sizeof(T) / 16);
    static_assert(kVecs * 16 == kEPL * sizeof(T), "run must be a whole number of 16-byte vectors");
    const uint4* q = reinterpret_cast<const uint4*>(p);
    uint4 w[kVecs];
#pragma unroll
    for (int i = 0; i < kVecs; ++i) w[i] = __ldcs(q + i);
    memcpy(out, w, sizeof(w));
}

// Traverse all rows of a CSR matrix; `pre(row, valid)` returns the epilogue operands of a
// row (loaded before the nonzeros), `epi(row, sum, operands)` consumes the row sum.
// `wbuf` is this warp's shared buffer of kWarpChunk accumulators.
template <class V, class X, class Acc, class Pre, class Epi>
__device__ __forceinline__ void warp_csr(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                         const V* __restrict__ val, const X* __restrict__ x, int64_t nrows,
                                         Acc* __restrict__ wbuf, Pre pre, Epi epi) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ntiles = (nrows + 31) >> 5;
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles; t += nwarps) {
        const int64_t r = (t << 5) + lane;
        const bool has = r < nrows;
        int32_t rb = 0, re = 0;
        if (has) {
            rb = __ldcs(ptr + r);
            re = __ldcs(ptr + r + 1);
        }
        auto ops = pre(r, has);
        const int last = (int)min((int64_t)31, nrows - 1 - (t << 5));
        const int32_t e0 = __shfl_sync(0xffffffffu, rb, 0);
        const int32_t e1 = __shfl_sync(0xffffffffu, re, last);
        Acc acc = Acc(0);
        for (int32_t c = e0 & ~(kEPL - 1); c < e1; c += kWarpChunk) {
            const int32_t base = c + lane * kEPL;
            Acc p[kEPL];
            if (base < e1) {
                int32_t cj[kEPL];
                V vv[kEPL];
                load_run(col + base, cj);
                load_run(val + base, vv);
#pragma unroll
                for (int k = 0; k < kEPL; ++k) {
                    const int32_t e = base + k;
                    p[k] = (e >= e0 && e < e1) ? val_to_acc<Acc>(vv[k]) * vec_to_acc<Acc>(__ldg(x + cj[k])) : Acc(0);
                }
            } else {
#pragma unroll
                for (int k = 0; k < kEPL; ++k) p[k] = Acc(0);
            }
            // entry i of the chunk lives at wbuf[(i % kEPL) * 32 + i / kEPL]: conflict-free stores
#pragma unroll
            for (int k = 0; k < kEPL; ++k) wbuf[k * 32 + lane] = p[k];
            __syncwarp();
            const int32_t lo = max(rb, c), hi = min(re, c + kWarpChunk);
            for (int32_t e = lo; e < hi; ++e) {
                const int32_t i = e - c;
                acc += wbuf[(i & (kEPL - 1)) * 32 + (i / kEPL)];
            }
            __syncwarp();
        }
        if (has) epi(r, acc, ops);
    }
}

struct NoOps {};

}  // namespace l1ls

namespace l1ls {

// ---- paired storage ----------------------------------------------------------------------
// With one left rotation, rows 2p and 2p+1 of P1^T A share their column set and every column
// holds complete row pairs.  Both orientations are stored with one index per pair of
// entries and the two values side by side:
//   rows:    pair p -> entries (column j, value in row 2p, value in row 2p+1)
//   columns: column j -> entries (pair p, value in row 2p, value in row 2p+1)
// A row-pair traversal gathers x[j] once for two rows; a column traversal gathers the two
// entries (2p, 2p+1) of the input as one 8- or 16-byte load.

template <class T> struct Two;
template <> struct Two<float> { using type = float2; };
template <> struct Two<double> { using type = double2; };

template <class T, int N>
__device__ __forceinline__ void load_span(const T* __restrict__ p, T (&out)[N]) {
    constexpr int kVecs = (int)(N * sizeof(T) / 16);
    static_assert(kVecs * 16 == N * sizeof(T), "span must be a whole number of 16-byte vectors");
    const uint4* q = reinterpret_cast<const uint4*>(p);
    uint4 w[kVecs];
#pragma unroll
    for (int i = 0; i < kVecs; ++i) w[i] = __ldcs(q + i);
    memcpy(out, w, sizeof(w));
}

// ROWS = true : npairs row pairs; x gathered at the column index; pre / epi are called per
//               row (2p and 2p+1) exactly as for warp_csr.
// ROWS = false: nrows columns; x gathered at (2p, 2p+1); pre / epi per column.
// wbuf: this warp's 2 * kWarpChunk accumulators.
// One tile t (32 row pairs, or 32 columns) of the paired traversal whose row extents rb, re
// (this lane's row) are already loaded; see warp_pcsr.
template <bool ROWS, class V, class X, class Acc, class Pre, class Epi>
__device__ __forceinline__ void pcsr_tile_body(int64_t t, int32_t rb, int32_t re, const int32_t* __restrict__ idx,
                                               const V* __restrict__ val2, const X* __restrict__ x, int64_t nrows,
                                               Acc* __restrict__ wbuf, Pre& pre, Epi& epi) {
    const int lane = threadIdx.x & 31;
    Acc* w0 = wbuf;
    Acc* w1 = wbuf + kWarpChunk;
    const int64_t r = (t << 5) + lane;
    const bool has = r < nrows;
    auto ops0 = pre(ROWS ? 2 * r : r, has);
    auto ops1 = pre(ROWS ? 2 * r + 1 : r, ROWS && has);
    const int last = (int)min((int64_t)31, nrows - 1 - (t << 5));
    const int32_t e0 = __shfl_sync(0xffffffffu, rb, 0);
    const int32_t e1 = __shfl_sync(0xffffffffu, re, last);
    Acc a0 = Acc(0), a1 = Acc(0);
    for (int32_t c = e0 & ~(kPEPL - 1); c < e1; c += 32 * kPEPL) {
        const int32_t base = c + lane * kPEPL;
        Acc p0[kPEPL], p1[kPEPL];
        if (base < e1) {
            int32_t ij[kPEPL];
            V vv[2 * kPEPL];
            load_span<int32_t, kPEPL>(idx + base, ij);
            load_span<V, 2 * kPEPL>(val2 + 2 * (int64_t)base, vv);
#pragma unroll
            for (int k = 0; k < kPEPL; ++k) {
                const int32_t e = base + k;
                const bool in = e >= e0 && e < e1;
                const Acc v0 = val_to_acc<Acc>(vv[2 * k]), v1 = val_to_acc<Acc>(vv[2 * k + 1]);
                if (ROWS) {
                    const Acc xv = in ? vec_to_acc<Acc>(__ldg(x + ij[k])) : Acc(0);
                    p0[k] = v0 * xv;
                    p1[k] = v1 * xv;
                } else {
                    Acc g0 = Acc(0), g1 = Acc(0);
                    if (in) {
                        const typename Two<X>::type g = __ldg(reinterpret_cast<const typename Two<X>::type*>(x) + ij[k]);
                        g0 = vec_to_acc<Acc>(g.x);
                        g1 = vec_to_acc<Acc>(g.y);
                    }
                    p0[k] = v0 * g0 + v1 * g1;
                    p1[k] = Acc(0);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < kPEPL; ++k) p0[k] = p1[k] = Acc(0);
        }
#pragma unroll
        for (int k = 0; k < kPEPL; ++k) {
            w0[k * 32 + lane] = p0[k];
            if (ROWS) w1[k * 32 + lane] = p1[k];
        }
        __syncwarp();
        const int32_t lo = max(rb, c), hi = min(re, c + 32 * kPEPL);
        for (int32_t e = lo; e < hi; ++e) {
            const int32_t i = e - c;
            const int32_t q = (i & (kPEPL - 1)) * 32 + (i / kPEPL);
            a0 += w0[q];
            if (ROWS) a1 += w1[q];
        }
        __syncwarp();
    }
    if (has) {
        if (ROWS) {
            epi(2 * r, a0, ops0);
            epi(2 * r + 1, a1, ops1);
        } else {
            epi(r, a0, ops0);
        }
    }
}

template <bool ROWS, class V, class X, class Acc, class Pre, class Epi>
__device__ __forceinline__ void pcsr_tile(int64_t t, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const V* __restrict__ val2, const X* __restrict__ x, int64_t nrows,
                                          Acc* __restrict__ wbuf, Pre& pre, Epi& epi) {
    const int64_t r = (t << 5) + (threadIdx.x & 31);
    int32_t rb = 0, re = 0;
    if (r < nrows) {
        rb = __ldcs(ptr + r);
        re = __ldcs(ptr + r + 1);
    }
    pcsr_tile_body<ROWS, V, X, Acc>(t, rb, re, idx, val2, x, nrows, wbuf, pre, epi);
}

// ROWS = true : npairs row pairs; x gathered at the column index; pre / epi are called per
//               row (2p and 2p+1) exactly as for warp_csr.
// ROWS = false: nrows columns; x gathered at (2p, 2p+1); pre / epi per column.
// wbuf: this warp's 2 * kWarpChunk accumulators.
template <bool ROWS, class V, class X, class Acc, class Pre, class Epi>
__device__ __forceinline__ void warp_pcsr(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const V* __restrict__ val2, const X* __restrict__ x, int64_t nrows,
                                          Acc* __restrict__ wbuf, Pre pre, Epi epi) {
    // the row extents of the warp's next tile are loaded before the current tile is processed,
    // so the pointer round trip overlaps the previous tile's work
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ntiles = (nrows + 31) >> 5;
    const int lane = threadIdx.x & 31;
    int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int32_t nb = 0, ne = 0;
    if (t < ntiles && (t << 5) + lane < nrows) {
        nb = __ldcs(ptr + (t << 5) + lane);
        ne = __ldcs(ptr + (t << 5) + lane + 1);
    }
    for (; t < ntiles; t += nwarps) {
        const int32_t rb = nb, re = ne;
        const int64_t tn = t + nwarps;
        nb = ne = 0;
        if (tn < ntiles && (tn << 5) + lane < nrows) {
            nb = __ldcs(ptr + (tn << 5) + lane);
            ne = __ldcs(ptr + (tn << 5) + lane + 1);
        }
        pcsr_tile_body<ROWS, V, X, Acc>(t, rb, re, idx, val2, x, nrows, wbuf, pre, epi);
    }
}

// Row traversal of A (nrows rows) in plain or paired storage.
template <bool PAIRED, class V, class X, class Acc, class Pre, class Epi>
__device__ __forceinline__ void rows_of(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const X* __restrict__ x, int64_t nrows,
                                        Acc* __restrict__ wbuf, Pre pre, Epi epi) {
    if constexpr (PAIRED) warp_pcsr<true, V, X, Acc>(ptr, idx, val, x, nrows / 2, wbuf, pre, epi);
    else warp_csr<V, X, Acc>(ptr, idx, val, x, nrows, wbuf, pre, epi);
}

// Column traversal of A (rows of A^T, ncols of them) in plain or paired storage.
template <bool PAIRED, class V, class X, class Acc, class Pre, class Epi>
__device__ __forceinline__ void cols_of(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const X* __restrict__ x, int64_t ncols,
                                        Acc* __restrict__ wbuf, Pre pre, Epi epi) {
    if constexpr (PAIRED) warp_pcsr<false, V, X, Acc>(ptr, idx, val, x, ncols, wbuf, pre, epi);
    else warp_csr<V, X, Acc>(ptr, idx, val, x, ncols, wbuf, pre, epi);
}

// shared accumulators per block for either storage
template <class Acc, int BLOCK> struct TraversalSmem {
    Acc buf[(BLOCK / 32) * 2 * kWarpChunk];
    __device__ Acc* warp_buf() { return buf + (threadIdx.x >> 5) * 2 * kWarpChunk; }
};

// Matrix operands of one orientation
template <class V> struct Csr {
    const int32_t* ptr;
    const int32_t* idx;
    const V* val;
};

}  // namespace l1ls

namespace l1ls {

// ---- compensated traversals ---------------------------------------------------------------
// Products of the FP32 (or BF16) matrix with float-float vectors, accumulated in float-float:
// each term a * (h + l) is TwoProduct(a, h) with a * l added to its low word, and the sums are
// float-float additions (Dekker 1971; Bailey's double-single arithmetic).  The result carries
// about 44 bits, enough for the residual b - A y of a nearly fitted row (a small difference of
// large terms) and for A^T r at a small tau, where plain FP32 holds the duality-gap
// certificate above 1e-6 (the floor grows as tau, and with it the objective, shrinks along a
// path).  The tile structure is that of pcsr_tile; the warp buffer holds high and low words.
//
// Inputs: the row traversal gathers a float-float vector kept as two FP32 arrays (high and low
// words).  The column traversal gathers the residual: in paired storage the residual of row
// pair p is one float4 {hi(2p), hi(2p+1), lo(2p), lo(2p+1)} (both rows with one 16-byte load),
// in plain storage one float2 {hi, lo} per row.

template <bool ROWS, bool PAIRED, class V, int EPL = kEPL, class Pre, class Epi>
__device__ __forceinline__ void tile_ff_body(int64_t t, int32_t rb, int32_t re, const int32_t* __restrict__ idx,
                                             const V* __restrict__ val, const float* __restrict__ xh,
                                             const float* __restrict__ xl, const void* __restrict__ rin, int64_t nrows,
                                             float* __restrict__ wbuf, Pre& pre, Epi& epi) {
    // ROWS: nrows rows (PAIRED: row pairs; pre / epi per row, 2p and 2p+1), (xh, xl) gathered
    // at the column index; otherwise nrows columns, the residual rin gathered at the pair (or
    // row) index.  EPL entries per lane and chunk (4 or 8): fewer registers with 4, more loads
    // in flight with 8 (plain BF16 storage needs 8 for whole 16-byte value loads).
    static_assert(EPL == 4 || EPL == 8, "EPL must be 4 or 8");
    constexpr int kVals = PAIRED ? 2 : 1;
    static_assert((kVals * EPL * sizeof(V)) % 16 == 0, "value spans must be whole 16-byte vectors");
    constexpr int kChunk = 32 * EPL;
    const int lane = threadIdx.x & 31;
    float* w0h = wbuf;
    float* w0l = wbuf + kChunk;
    float* w1h = wbuf + 2 * kChunk;
    float* w1l = wbuf + 3 * kChunk;
    constexpr bool kTwoRows = ROWS && PAIRED;
    const int64_t r = (t << 5) + lane;
    const bool has = r < nrows;
    auto ops0 = pre(kTwoRows ? 2 * r : r, has);
    auto ops1 = pre(kTwoRows ? 2 * r + 1 : r, kTwoRows && has);
    const int last = (int)min((int64_t)31, nrows - 1 - (t << 5));
    const int32_t e0 = __shfl_sync(0xffffffffu, rb, 0);
    const int32_t e1 = __shfl_sync(0xffffffffu, re, last);
    ff a0 = {0.f, 0.f}, a1 = {0.f, 0.f};
    for (int32_t c = e0 & ~(EPL - 1); c < e1; c += kChunk) {
        const int32_t base = c + lane * EPL;
        ff p0[EPL], p1[EPL];
        if (base < e1) {
            int32_t ij[EPL];
            V vv[kVals * EPL];
            load_span<int32_t, EPL>(idx + base, ij);
            load_span<V, kVals * EPL>(val + kVals * (int64_t)base, vv);
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int32_t e = base + k;
                const bool in = e >= e0 && e < e1;
                const float v0 = val_to_acc<float>(vv[kVals * k]);
                const float v1 = PAIRED ? val_to_acc<float>(vv[kVals * k + kVals - 1]) : 0.f;
                if (ROWS) {
                    const float hx = in ? __ldg(xh + ij[k]) : 0.f;
                    const float lx = in ? __ldg(xl + ij[k]) : 0.f;
                    p0[k] = two_prod(v0, hx);
                    p0[k].lo = __fmaf_rn(v0, lx, p0[k].lo);
                    if (PAIRED) {
                        p1[k] = two_prod(v1, hx);
                        p1[k].lo = __fmaf_rn(v1, lx, p1[k].lo);
                    } else {
                        p1[k] = {0.f, 0.f};
                    }
                } else if (PAIRED) {
                    const float4 g = in ? __ldg(static_cast<const float4*>(rin) + ij[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
                    ff q0 = two_prod(v0, g.x);
                    q0.lo = __fmaf_rn(v0, g.z, q0.lo);
                    ff q1 = two_prod(v1, g.y);
                    q1.lo = __fmaf_rn(v1, g.w, q1.lo);
                    p0[k] = ff_add(q0, q1);
                    p1[k] = {0.f, 0.f};
                } else {
                    const float2 g = in ? __ldg(static_cast<const float2*>(rin) + ij[k]) : make_float2(0.f, 0.f);
                    p0[k] = two_prod(v0, g.x);
                    p0[k].lo = __fmaf_rn(v0, g.y, p0[k].lo);
                    p1[k] = {0.f, 0.f};
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < EPL; ++k) p0[k] = p1[k] = {0.f, 0.f};
        }
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            w0h[k * 32 + lane] = p0[k].hi;
            w0l[k * 32 + lane] = p0[k].lo;
            if (kTwoRows) {
                w1h[k * 32 + lane] = p1[k].hi;
                w1l[k * 32 + lane] = p1[k].lo;
            }
        }
        __syncwarp();
        const int32_t lo = max(rb, c), hi = min(re, c + kChunk);
        for (int32_t e = lo; e < hi; ++e) {
            const int32_t i = e - c;
            const int32_t q = (i & (EPL - 1)) * 32 + (i / EPL);
            a0 = ff_add(a0, {w0h[q], w0l[q]});
            if (kTwoRows) a1 = ff_add(a1, {w1h[q], w1l[q]});
        }
        __syncwarp();
    }
    if (has) {
        if (kTwoRows) {
            epi(2 * r, a0, ops0);
            epi(2 * r + 1, a1, ops1);
        } else {
            epi(r, a0, ops0);
        }
    }
}

// row extents of this lane's row of tile t (0, 0 past the end)
__device__ __forceinline__ void tile_extents(const int32_t* __restrict__ ptr, int64_t t, int64_t nrows, int32_t& rb,
                                             int32_t& re) {
    const int64_t r = (t << 5) + (threadIdx.x & 31);
    rb = re = 0;
    if (r < nrows) {
        rb = __ldcs(ptr + r);
        re = __ldcs(ptr + r + 1);
    }
}

template <bool ROWS, bool PAIRED, class V, int EPL = kEPL, class Pre, class Epi>
__device__ __forceinline__ void tile_ff(int64_t t, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const float* __restrict__ xh,
                                        const float* __restrict__ xl, const void* __restrict__ rin, int64_t nrows,
                                        float* __restrict__ wbuf, Pre& pre, Epi& epi) {
    int32_t rb, re;
    tile_extents(ptr, t, nrows, rb, re);
    tile_ff_body<ROWS, PAIRED, V, EPL>(t, rb, re, idx, val, xh, xl, rin, nrows, wbuf, pre, epi);
}

// tiles t0 .. t1-1 in order, each tile's row extents loaded before the previous tile's work
template <bool ROWS, bool PAIRED, class V, int EPL = kEPL, class Pre, class Epi>
__device__ __forceinline__ void tiles_ff(int64_t t0, int64_t t1, const int32_t* __restrict__ ptr,
                                         const int32_t* __restrict__ idx, const V* __restrict__ val,
                                         const float* __restrict__ xh, const float* __restrict__ xl,
                                         const void* __restrict__ rin, int64_t nrows, float* __restrict__ wbuf,
                                         Pre& pre, Epi& epi) {
    int32_t nb, ne;
    tile_extents(ptr, t0, nrows, nb, ne);
#pragma unroll 1
    for (int64_t t = t0; t < t1; ++t) {
        const int32_t rb = nb, re = ne;
        if (t + 1 < t1) tile_extents(ptr, t + 1, nrows, nb, ne);
        tile_ff_body<ROWS, PAIRED, V, EPL>(t, rb, re, idx, val, xh, xl, rin, nrows, wbuf, pre, epi);
    }
}

// paired storage (the form the batched kernel uses)
template <bool ROWS, class V, int EPL = kEPL, class Pre, class Epi>
__device__ __forceinline__ void pcsr_tile_ff(int64_t t, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                             const V* __restrict__ val2, const float* __restrict__ xh,
                                             const float* __restrict__ xl, const float4* __restrict__ r4, int64_t nrows,
                                             float* __restrict__ wbuf, Pre& pre, Epi& epi) {
    tile_ff<ROWS, true, V, EPL>(t, ptr, idx, val2, xh, xl, r4, nrows, wbuf, pre, epi);
}

template <int BLOCK> struct CompSmem {
    float buf[(BLOCK / 32) * 4 * kWarpChunk];
    __device__ float* warp_buf() { return buf + (threadIdx.x >> 5) * 4 * kWarpChunk; }
};

}  // namespace l1ls
