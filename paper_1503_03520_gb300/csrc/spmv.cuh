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

#include <type_traits>

#include "common.cuh"

namespace l1ls {

constexpr int kEPL = 8;       // nonzeros per lane per chunk
constexpr int kPad = kEPL;    // slack entries after the nonzero arrays
constexpr int kWarpChunk = 32 * kEPL;

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

// Gather of a vector entry: the read-only non-coherent path (__ldg) where the vector is not
// written during the kernel, an L2 load (__ldcg) in persistent kernels whose later phases gather
// what earlier phases of the same launch wrote (the non-coherent path may return stale lines).
template <bool COH, class T> __device__ __forceinline__ T gather_load(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// Traverse all rows of a CSR matrix; `pre(row, valid)` returns the epilogue operands of a
// row (loaded before the nonzeros), `epi(row, sum, operands)` consumes the row sum.
// `wbuf` is this warp's shared buffer of kWarpChunk accumulators.
template <class V, class X, class Acc, bool COH = false, class Pre, class Epi>
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
                    p[k] = (e >= e0 && e < e1) ? val_to_acc<Acc>(vv[k]) * vec_to_acc<Acc>(gather_load<COH>(x + cj[k])) : Acc(0);
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

// the two values of one paired entry as one load
template <class V> struct ValPair;
template <> struct ValPair<float> { using type = float2; };
template <> struct ValPair<double> { using type = double2; };
template <> struct ValPair<__nv_bfloat16> { using type = __nv_bfloat162; };
template <class Acc> __device__ __forceinline__ void pair_to_acc(float2 v, Acc& a, Acc& b) { a = v.x; b = v.y; }
template <class Acc> __device__ __forceinline__ void pair_to_acc(double2 v, Acc& a, Acc& b) { a = v.x; b = v.y; }
template <class Acc> __device__ __forceinline__ void pair_to_acc(__nv_bfloat162 v, Acc& a, Acc& b) {
    a = __bfloat162float(v.x);
    b = __bfloat162float(v.y);
}

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

// ---- bulk-copy staging of the nonzero stream -----------------------------------------------
// Each warp owns two stages in shared memory.  While it works on tile t, one lane has already
// issued the bulk copies (cp.async.bulk, completion counted in bytes on the stage's mbarrier)
// of the index and value spans of its next tile t + nwarps into the other stage, so the
// stream of A arrives while the current tile's gathers are in flight: a tile costs one memory
// round trip (the gathers) instead of two (stream, then gathers).  A span starts at the
// 16-byte boundary at or below the tile's first entry and ends at the one at or above its
// last; a tile longer than one stage is staged in consecutive pieces.  The copies carry an
// L2 evict-first policy (A is read once per product).  Each wait polls at most kStagePolls
// times; if one runs out the warp records kStageTimeout in *err and reads the rest of its
// tiles directly from global memory (same sums, same order).

constexpr uint32_t kStagePolls = 1u << 20;
// build parameters of the stage wait: a sleep between unsuccessful polls (32 ns measured 1.7%
// faster in K2 than none: polling warps stop taking issue slots), and the suspend-time hint of
// mbarrier.try_wait (0: none; 1000 ns measured no different)
#ifndef L1LS_STAGE_SLEEP_NS
#define L1LS_STAGE_SLEEP_NS 32
#endif
#ifndef L1LS_STAGE_HINT_NS
#define L1LS_STAGE_HINT_NS 0
#endif
constexpr int kStageTimeout = 1 << 30;
constexpr int kStageBytes = 2880;   // per stage and warp (two stages x 8 warps fit 48 KB)

template <class V> struct StageGeom {
    static constexpr int kCap = (kStageBytes / (4 + 2 * (int)sizeof(V))) & ~3;   // entries per stage
};

template <class V, int BLOCK> struct PairedSmem {
    static constexpr int kWarps = BLOCK / 32;
    static constexpr int kCap = StageGeom<V>::kCap;
    alignas(16) int32_t idx[kWarps][2][kCap];
    alignas(16) V val[kWarps][2][2 * kCap];
    alignas(8) uint64_t bar[kWarps][2];
};
static_assert(StageGeom<float>::kCap % 4 == 0 && StageGeom<double>::kCap % 4 == 0, "stage spans of 16 bytes");

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
#if L1LS_STAGE_HINT_NS > 0
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"((uint32_t)L1LS_STAGE_HINT_NS)
        : "memory");
#else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
#endif
    return done != 0;
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// the stage of entries [lo, hi) (lo, hi multiples of 4): lane 0 arms the barrier and issues
template <class V>
__device__ __forceinline__ void stage_issue(int32_t* sidx, V* sval, uint64_t* bar, const int32_t* __restrict__ idx,
                                            const V* __restrict__ val2, int32_t lo, int32_t hi, uint64_t policy) {
    if ((threadIdx.x & 31) == 0) {
        const uint32_t cnt = (uint32_t)(hi - lo);
        const uint32_t bi = 4u * cnt, bv = 2u * (uint32_t)sizeof(V) * cnt;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of this stage
        mbar_expect_tx(bar, bi + bv);
        bulk_load(sidx, idx + lo, bi, bar, policy);
        bulk_load(sval, val2 + 2 * (int64_t)lo, bv, bar, policy);
    }
}

// bounded wait for a stage; false (warp-uniform) if some lane ran out of polls
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity) {
    bool done = false;
    for (uint32_t k = 0; k < kStagePolls && !done; ++k) {
        done = mbar_try_wait(bar, parity);
#if L1LS_STAGE_SLEEP_NS > 0
        if (!done) __nanosleep(L1LS_STAGE_SLEEP_NS);
#endif
    }
    return __all_sync(0xffffffffu, done);
}

// this lane's entries [eb, ee) of its row (ROWS: row pair, a0 / a1 for rows 2p / 2p+1) or
// column (a0), read from ib[e - off], vb[e - off] (shared stage or global arrays), in entry
// order, four entries' loads at a time
template <bool ROWS, class V, class X, class Acc, bool COH = false>
__device__ __forceinline__ void lane_entries(const int32_t* ib, const typename ValPair<V>::type* vb, int32_t off,
                                             int32_t eb, int32_t ee, const X* __restrict__ x, Acc& a0, Acc& a1) {
    for (int32_t e = eb; e < ee; e += 4) {
        Acc v0[4], v1[4], g0[4], g1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v0[k] = v1[k] = g0[k] = g1[k] = Acc(0);
            if (e + k < ee) {
                const int32_t j = ib[e + k - off];
                pair_to_acc<Acc>(vb[e + k - off], v0[k], v1[k]);
                if (ROWS) {
                    g0[k] = vec_to_acc<Acc>(gather_load<COH>(x + j));
                } else {
                    const typename Two<X>::type g =
                        gather_load<COH>(reinterpret_cast<const typename Two<X>::type*>(x) + j);
                    g0[k] = vec_to_acc<Acc>(g.x);
                    g1[k] = vec_to_acc<Acc>(g.y);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (e + k < ee) {
                if (ROWS) {
                    a0 += v0[k] * g0[k];
                    a1 += v1[k] * g0[k];
                } else {
                    a0 += v0[k] * g0[k] + v1[k] * g1[k];
                }
            }
        }
    }
}

// Summation policies of the staged traversal: how a lane gathers the vector for its entries
// and accumulates its row (column).
//   PlainSum: products and sums in Acc (FP64 for FP64 values, FP32 otherwise).
template <bool ROWS, class V, class X, class Acc, bool COH = false> struct PlainSum {
    using acc_t = Acc;
    const X* x;
    __device__ __forceinline__ Acc zero() const { return Acc(0); }
    __device__ __forceinline__ void entries(const int32_t* ib, const typename ValPair<V>::type* vb, int32_t off,
                                            int32_t eb, int32_t ee, Acc& a0, Acc& a1) const {
        lane_entries<ROWS, V, X, Acc, COH>(ib, vb, off, eb, ee, x, a0, a1);
    }
    __device__ __forceinline__ Acc finish(Acc a) const { return a; }
};

// Forward declaration: the float-float policy (FFSum) is defined with the float-float kernels.
template <bool ROWS, class V, bool COH = false> struct FFSum;

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

// first entry, end and the first stage piece [lo, hi) of the tile whose lane extents are (rb, re)
__device__ __forceinline__ void tile_span(int64_t t, int64_t nrows, int32_t rb, int32_t re, int cap, int32_t& e1,
                                          int32_t& lo, int32_t& hi) {
    const int last = (int)min((int64_t)31, nrows - 1 - (t << 5));
    const int32_t e0 = __shfl_sync(0xffffffffu, rb, 0);
    e1 = __shfl_sync(0xffffffffu, re, last);
    if (e1 <= e0) {
        lo = hi = e1;   // no entries
        return;
    }
    lo = e0 & ~3;
    hi = min(lo + cap, (e1 + 3) & ~3);
}

// A warp's staging state across calls: the L2 policy of its copies, the parity of each
// stage's next mbarrier phase, and whether staging is on (off after a wait ran out).
struct StageState {
    uint64_t policy;
    uint32_t parity;
    bool staging;
};

// Once per kernel and warp, before the warp's first staged_tiles (warp-uniform).
template <class V, int BLOCK>
__device__ __forceinline__ void stage_init(PairedSmem<V, BLOCK>& sm, StageState& ss) {
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        mbar_init(&sm.bar[wid][0], 1);
        mbar_init(&sm.bar[wid][1], 1);
        mbar_init_fence();
    }
    __syncwarp();
    ss.policy = l2_evict_first_policy();
    ss.parity = 0;
    ss.staging = true;
}

// Tiles t, t + step, ... (< tend) of one matrix in paired storage: lane l owns row pair (ROWS)
// or column tile*32 + l and sums its own entries in nonzero order from the staged stream, so
// every sum has a fixed order.  ROWS = true: nrows row pairs, pre / epi called per row (2p and
// 2p+1); ROWS = false: nrows columns, pre / epi per column.  `sum` (PlainSum or FFSum) gathers
// and accumulates a lane's entries.  Every copy issued here is waited for here, so calls can
// follow each other on the same state.  Warp-uniform arguments.
template <bool ROWS, class V, int BLOCK, class Sum, class Pre, class Epi>
__device__ __forceinline__ void staged_tiles(int64_t t, int64_t step, int64_t tend, const int32_t* __restrict__ ptr,
                                             const int32_t* __restrict__ idx, const V* __restrict__ val2,
                                             int64_t nrows, PairedSmem<V, BLOCK>& sm, StageState& ss, int* err,
                                             const Sum& sum, Pre& pre, Epi& epi) {
    using VP = typename ValPair<V>::type;
    using Acc = typename Sum::acc_t;
    constexpr int kCap = PairedSmem<V, BLOCK>::kCap;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (t >= tend) return;
    uint64_t* bar = sm.bar[wid];
    // arrays off 16-byte boundaries never stage
    const bool aligned = ((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(val2)) & 15u) == 0;

    int32_t rb, re, nb, ne;
    tile_extents(ptr, t, nrows, rb, re);
    tile_extents(ptr, t + step, nrows, nb, ne);
    int s = 0;
    int32_t e1, lo, hi;
    tile_span(t, nrows, rb, re, kCap, e1, lo, hi);
    bool issued = aligned && ss.staging && hi > lo;
    if (issued) stage_issue<V>(sm.idx[wid][0], sm.val[wid][0], &bar[0], idx, val2, lo, hi, ss.policy);

    for (; t < tend; t += step) {
        // the next tile's first piece into the other stage, then the extents of the one after
        const int64_t tn = t + step;
        int32_t e1n = 0, lon = 0, hin = 0;
        bool issued_n = false;
        if (tn < tend) {
            tile_span(tn, nrows, nb, ne, kCap, e1n, lon, hin);
            issued_n = aligned && ss.staging && hin > lon;
            if (issued_n)
                stage_issue<V>(sm.idx[wid][s ^ 1], sm.val[wid][s ^ 1], &bar[s ^ 1], idx, val2, lon, hin, ss.policy);
        }
        int32_t nb2, ne2;
        tile_extents(ptr, tn + step, nrows, nb2, ne2);

        const int64_t r = (t << 5) + lane;
        const bool has = r < nrows;
        auto ops0 = pre(ROWS ? 2 * r : r, has);
        auto ops1 = pre(ROWS ? 2 * r + 1 : r, ROWS && has);
        Acc a0 = sum.zero(), a1 = sum.zero();
        const int32_t end = (e1 + 3) & ~3;
        bool staged = issued && ss.staging;
        for (;;) {
            if (staged) {
                const bool ok = stage_wait(&bar[s], (ss.parity >> s) & 1u);
                ss.parity ^= 1u << s;
                if (!ok) {   // record, wait once more (bounded) for the copies in flight, read directly
                    ss.staging = staged = false;
                    if (lane == 0 && err) atomicOr(err, kStageTimeout);
                    stage_wait(&bar[s], ((ss.parity >> s) & 1u) ^ 1u);
                    if (issued_n) stage_wait(&bar[s ^ 1], (ss.parity >> (s ^ 1)) & 1u);
                }
            }
            const int32_t eb = max(rb, lo), ee = min(re, hi);
            if (staged)
                sum.entries(sm.idx[wid][s], reinterpret_cast<const VP*>(sm.val[wid][s]), lo, eb, ee, a0, a1);
            else
                sum.entries(idx, reinterpret_cast<const VP*>(val2), 0, eb, ee, a0, a1);
            if (hi >= e1) break;
            // a tile longer than one stage: its next piece into the same stage
            __syncwarp();
            lo = hi;
            hi = min(lo + kCap, end);
            staged = aligned && ss.staging;
            if (staged) stage_issue<V>(sm.idx[wid][s], sm.val[wid][s], &bar[s], idx, val2, lo, hi, ss.policy);
        }
        __syncwarp();   // every lane is done with stage s before it is refilled
        if (has) {
            if (ROWS) {
                epi(2 * r, sum.finish(a0), ops0);
                epi(2 * r + 1, sum.finish(a1), ops1);
            } else {
                epi(r, sum.finish(a0), ops0);
            }
        }
        rb = nb;
        re = ne;
        nb = nb2;
        ne = ne2;
        e1 = e1n;
        lo = lon;
        hi = hin;
        issued = issued_n;
        s ^= 1;
    }
}

// The whole matrix, tiles dealt round-robin: warp w of the grid takes tiles w, w + W, ...
template <bool ROWS, class V, int BLOCK, class Sum, class Pre, class Epi>
__device__ __forceinline__ void warp_pcsr(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const V* __restrict__ val2, int64_t nrows, PairedSmem<V, BLOCK>& sm,
                                          int* err, const Sum& sum, Pre pre, Epi epi) {
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ntiles = (nrows + 31) >> 5;
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    StageState ss;
    stage_init(sm, ss);
    staged_tiles<ROWS, V, BLOCK>(t, nwarps, ntiles, ptr, idx, val2, nrows, sm, ss, err, sum, pre, epi);
}

// Row traversal of A (nrows rows) in plain or paired storage; `sm` is the kernel's
// TraversalSmem, `err` receives kStageTimeout if a stage wait ran out (may be NULL).
template <bool PAIRED, class V, class X, class Acc, class Smem, class Pre, class Epi>
__device__ __forceinline__ void rows_of(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const X* __restrict__ x, int64_t nrows, Smem& sm,
                                        int* err, Pre pre, Epi epi) {
    if constexpr (PAIRED) warp_pcsr<true, V>(ptr, idx, val, nrows / 2, sm, err, PlainSum<true, V, X, Acc>{x}, pre, epi);
    else warp_csr<V, X, Acc>(ptr, idx, val, x, nrows, sm.warp_buf(), pre, epi);
}

// Column traversal of A (rows of A^T, ncols of them) in plain or paired storage.
template <bool PAIRED, class V, class X, class Acc, class Smem, class Pre, class Epi>
__device__ __forceinline__ void cols_of(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const X* __restrict__ x, int64_t ncols, Smem& sm,
                                        int* err, Pre pre, Epi epi) {
    if constexpr (PAIRED) warp_pcsr<false, V>(ptr, idx, val, ncols, sm, err, PlainSum<false, V, X, Acc>{x}, pre, epi);
    else warp_csr<V, X, Acc>(ptr, idx, val, x, ncols, sm.warp_buf(), pre, epi);
}

// shared memory of one traversal kernel: the two stages per warp (paired storage) or the
// chunk accumulators per warp (plain CSR)
template <class Acc, int BLOCK> struct CsrSmem {
    Acc buf[(BLOCK / 32) * kWarpChunk];
    __device__ Acc* warp_buf() { return buf + (threadIdx.x >> 5) * kWarpChunk; }
};
template <class V, class Acc, int BLOCK, bool PAIRED>
using TraversalSmem = typename std::conditional<PAIRED, PairedSmem<V, BLOCK>, CsrSmem<Acc, BLOCK>>::type;

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
// path).  The tile structure is that of warp_csr (lane runs of EPL entries, sums through a
// warp buffer), which holds high and low words here.
//
// Inputs: the row traversal gathers a float-float vector kept as two FP32 arrays (high and low
// words), or, when the low-word array is NULL, as one array of interleaved {hi, lo} pairs.  The column traversal gathers the residual: in paired storage the residual of row
// pair p is one float4 {hi(2p), hi(2p+1), lo(2p), lo(2p+1)} (both rows with one 16-byte load),
// in plain storage one float2 {hi, lo} per row.

template <bool ROWS, bool PAIRED, class V, int EPL = kEPL, bool COH = false, class Pre, class Epi>
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
                    float hx = 0.f, lx = 0.f;
                    if (in) {
                        if (xl) {
                            hx = gather_load<COH>(xh + ij[k]);
                            lx = gather_load<COH>(xl + ij[k]);
                        } else {   // interleaved {hi, lo} pairs: one 8-byte gather
                            const float2 g = gather_load<COH>(reinterpret_cast<const float2*>(xh) + ij[k]);
                            hx = g.x;
                            lx = g.y;
                        }
                    }
                    p0[k] = two_prod(v0, hx);
                    p0[k].lo = __fmaf_rn(v0, lx, p0[k].lo);
                    if (PAIRED) {
                        p1[k] = two_prod(v1, hx);
                        p1[k].lo = __fmaf_rn(v1, lx, p1[k].lo);
                    } else {
                        p1[k] = {0.f, 0.f};
                    }
                } else if (PAIRED) {
                    // the two terms of a column entry, summed in turn below (as FFSum does)
                    const float4 g = in ? gather_load<COH>(static_cast<const float4*>(rin) + ij[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
                    p0[k] = two_prod(v0, g.x);
                    p0[k].lo = __fmaf_rn(v0, g.z, p0[k].lo);
                    p1[k] = two_prod(v1, g.y);
                    p1[k].lo = __fmaf_rn(v1, g.w, p1[k].lo);
                } else {
                    const float2 g = in ? gather_load<COH>(static_cast<const float2*>(rin) + ij[k]) : make_float2(0.f, 0.f);
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
            if (PAIRED) {
                w1h[k * 32 + lane] = p1[k].hi;
                w1l[k * 32 + lane] = p1[k].lo;
            }
        }
        __syncwarp();
        // running sums by Sum2 in entry order (for a paired column: term of row 2p, then 2p+1),
        // the same operations as the staged traversal's FFSum, so both give the same bits
        const int32_t lo = max(rb, c), hi = min(re, c + kChunk);
        for (int32_t e = lo; e < hi; ++e) {
            const int32_t i = e - c;
            const int32_t q = (i & (EPL - 1)) * 32 + (i / EPL);
            sum2_add(a0, {w0h[q], w0l[q]});
            if (kTwoRows) sum2_add(a1, {w1h[q], w1l[q]});
            else if (PAIRED) sum2_add(a0, {w1h[q], w1l[q]});
        }
        __syncwarp();
    }
    if (has) {
        if (kTwoRows) {
            epi(2 * r, two_sum(a0.hi, a0.lo), ops0);
            epi(2 * r + 1, two_sum(a1.hi, a1.lo), ops1);
        } else {
            epi(r, two_sum(a0.hi, a0.lo), ops0);
        }
    }
}


template <bool ROWS, bool PAIRED, class V, int EPL = kEPL, bool COH = false, class Pre, class Epi>
__device__ __forceinline__ void tile_ff(int64_t t, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const float* __restrict__ xh,
                                        const float* __restrict__ xl, const void* __restrict__ rin, int64_t nrows,
                                        float* __restrict__ wbuf, Pre& pre, Epi& epi) {
    int32_t rb, re;
    tile_extents(ptr, t, nrows, rb, re);
    tile_ff_body<ROWS, PAIRED, V, EPL, COH>(t, rb, re, idx, val, xh, xl, rin, nrows, wbuf, pre, epi);
}

// tiles t0 .. t1-1 in order, each tile's row extents loaded before the previous tile's work
template <bool ROWS, bool PAIRED, class V, int EPL = kEPL, bool COH = false, class Pre, class Epi>
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
        tile_ff_body<ROWS, PAIRED, V, EPL, COH>(t, rb, re, idx, val, xh, xl, rin, nrows, wbuf, pre, epi);
    }
}

// The float-float policy of the staged traversal (paired storage): each product is
// TwoProduct(a, hi) with a * lo added to its low word, and the lane's running sum is kept by
// Algorithm Sum2 of Ogita, Rump & Oishi (TwoSum on the high word, the errors and low words in
// one FP32 word), which is as accurate as a sum in twice the working precision; the row sum
// is renormalised by TwoSum at the end.  ROWS gathers the float-float vector (xh, xl) at the
// column index (xl NULL: xh holds interleaved {hi, lo} pairs); otherwise the residual float4 {hi(2p), hi(2p+1), lo(2p), lo(2p+1)} at the pair.
template <bool ROWS, class V, bool COH> struct FFSum {
    using acc_t = ff;
    const float* xh;
    const float* xl;
    const float4* r4;
    __device__ __forceinline__ ff zero() const { return {0.0f, 0.0f}; }
    __device__ __forceinline__ void entries(const int32_t* ib, const typename ValPair<V>::type* vb, int32_t off,
                                            int32_t eb, int32_t ee, ff& a0, ff& a1) const {
        for (int32_t e = eb; e < ee; e += 4) {
            float v0[4], v1[4], g0[4], g1[4], h0[4], h1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v0[k] = v1[k] = g0[k] = g1[k] = h0[k] = h1[k] = 0.0f;
                if (e + k < ee) {
                    const int32_t j = ib[e + k - off];
                    pair_to_acc<float>(vb[e + k - off], v0[k], v1[k]);
                    if (ROWS) {
                        if (xl) {
                            g0[k] = gather_load<COH>(xh + j);
                            h0[k] = gather_load<COH>(xl + j);
                        } else {   // interleaved {hi, lo} pairs: one 8-byte gather
                            const float2 g = gather_load<COH>(reinterpret_cast<const float2*>(xh) + j);
                            g0[k] = g.x;
                            h0[k] = g.y;
                        }
                    } else {
                        const float4 g = gather_load<COH>(r4 + j);
                        g0[k] = g.x;
                        g1[k] = g.y;
                        h0[k] = g.z;
                        h1[k] = g.w;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (e + k < ee) {
                    ff p0 = two_prod(v0[k], g0[k]);
                    p0.lo = __fmaf_rn(v0[k], h0[k], p0.lo);
                    if (ROWS) {
                        ff p1 = two_prod(v1[k], g0[k]);
                        p1.lo = __fmaf_rn(v1[k], h0[k], p1.lo);
                        sum2_add(a0, p0);
                        sum2_add(a1, p1);
                    } else {
                        ff p1 = two_prod(v1[k], g1[k]);
                        p1.lo = __fmaf_rn(v1[k], h1[k], p1.lo);
                        sum2_add(a0, p0);
                        sum2_add(a0, p1);
                    }
                }
            }
        }
    }
    __device__ __forceinline__ ff finish(ff a) const { return two_sum(a.hi, a.lo); }
};

template <int BLOCK> struct CompSmem {
    float buf[(BLOCK / 32) * 4 * kWarpChunk];
    __device__ float* warp_buf() { return buf + (threadIdx.x >> 5) * 4 * kWarpChunk; }
};

}  // namespace l1ls
