// Ragged batches of instances solved by FISTA along a tau path (warm-started), in one
// persistent cooperative kernel per chunk of FISTA steps.
//
// The instances keep their own paired matrices, right-hand sides and iterates; the batch adds
// a device table of descriptors and two global tile lists (row-pair tiles and column tiles
// of every instance).  The unit of work is a segment of 16 tiles (a tile: 32 row pairs or 32
// columns) of one instance; warps take segments in turn from an atomic counter per phase (so
// a warp that drew short or retired segments takes more).  One launch runs `steps` FISTA
// steps; each step has two phases separated by bounded grid barriers:
//   1. every warp takes row-pair segments of active instances: K1's product, its epilogue and
//      the segment's gap partials (each lane sums its rows in tile order, then the warp), one
//      write per segment;
//   2. column segments: K2's product, the momentum and shrinkage, per-segment partials.
// Per-instance sums need no phase of their own: the warp that completes the last segment of an
// instance (an atomic count per instance, after a memory fence) sums the segment partials in
// segment order.  That warp then holds the instance's totals: after phase 1 it
// stores the sums of K1; after phase 2 it takes the scalar step of FISTA (Sec. 8.1) with the
// certificate, and when the tolerance is met records the result and moves to the next tau of
// the path, warm-started from the last iterate computed (one prox-gradient step past the
// certified one), or retires the instance.
// Every sum has a fixed order that depends only on the instance, so an instance's results
// are identical whatever else is in the batch and whatever schedule the autotuner picks.
// Both products and all vectors are float-float (compensated traversals): along a path tau
// shrinks and so does the objective, and with FP32 residuals and FP32 sums of A^T r the
// certificate stalls above 1e-6 (measured on the path instances of the tests: relative gaps of
// 1e-5 to 1e-1 after 1e5 iterations at the smaller taus).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "spmv.cuh"

namespace l1ls {

namespace {

constexpr uint32_t kBarrierPolls = 1u << 24;

struct BDesc {
    const int32_t* rptr;
    const int32_t* rcol;
    const void* rval;
    const int32_t* cptr;
    const int32_t* cpair;
    const void* cval;
    const float* b;
    float2* ax;                // A x_{k-1}, float-float per row
    float4* res;               // b - A y_k per row pair {hi(2p), hi(2p+1), lo(2p), lo(2p+1)}
    float2* x[2];              // iterates x_{k-1}, x_{k-2} (alternating), float-float {hi, lo}
                               //   pairs: the row phase gathers both words with one load
    int64_t m, n;
    int64_t s1_begin, s2_begin;    // first segment of the instance in each segment list
    int64_t n1, n2;                // tiles of the instance: row-pair tiles, column tiles
    int64_t ns1, ns2;              // segments of the instance
};

struct BState {
    double tau, L, tol;
    int64_t max_iter;
    double t, beta, best_d, l1_cur;
    double k1[3];              // phase-1 sums: ||A x - b||^2, b.r, r.r
    int64_t iter;
    int32_t stop, status, tau_idx, ntau, final_buf, restart;
    float beta_ff[2], invL_ff[2], thr_ff[2];   // beta, 1/L, tau/L as float-float (set with them)
};

__host__ __device__ inline void split_ff(double d, float (&out)[2]) {
    out[0] = (float)d;
    out[1] = (float)(d - (double)out[0]);
}

static_assert(sizeof(BState) % 8 == 0, "state is read as 64-bit words");

// read a state written by other CTAs in an earlier phase (bypassing L1)
__device__ __forceinline__ BState load_state(const BState* p) {
    BState s;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(BState) / 8); ++k) dst[k] = __ldcg(src + k);
    return s;
}

struct BResult {
    double P, D, gap, rel;
    int64_t iters;
    int32_t status, done;      // done: written by the kernel (the tau was finished)
};

struct BArgs {
    const BDesc* desc;
    BState* state;
    BResult* results;
    const double* taus;        // [inst][ntau]
    const int32_t* sinst1;     // row-pair segment -> instance
    const int32_t* sinst2;     // column segment -> instance
    int64_t nseg1, nseg2;
    double* part1;             // [segment][3]
    double* part2;             // [segment][3]
    unsigned* fetch;           // [2] next segment of phase 1 / phase 2 (warps take segments in turn)
    unsigned* instcnt1;        // segments done per instance (reset by the instance's last warp)
    unsigned* instcnt2;
    int ninst, ntau_max;
    unsigned* bar_count;
    unsigned* bar_gen;
    int* err;
    int* active;
    int64_t step0;
    int steps;
    uint32_t max_polls;        // the barrier's poll limit (kBarrierPolls in solves)
    unsigned extra_arrivals;   // 0 in solves; the failure self-test sets 1 (a barrier that never fills)
};

__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

// tiles per segment (measured on a shortened C4 run: 8 tiles 0.665 ms per step, 12 0.643,
// 16 0.641, 24 0.655, 32 0.675: fewer fetches, fences and partials against the tail of a phase)
constexpr int kSegTiles = 16;

// Count this warp's segment (lane 0 already wrote its partials at part[K sg]) in its instance;
// see the file comment.  Returns true on the one warp that completed the instance, with the
// instance totals in tot (every lane).  Partial 0 is combined by max when MAX0, else summed.
template <int K, bool MAX0>
__device__ bool segment_done(int64_t s_begin, int64_t nseg, const double* part, unsigned* instcnt, double (&tot)[K]) {
    const int lane = threadIdx.x & 31;
    __threadfence();
    int last = 0;
    if (lane == 0) last = atomicAdd(instcnt, 1u) == (unsigned)(nseg - 1);
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    if (lane == 0) *instcnt = 0u;
    __threadfence();
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0;
    for (int64_t q = lane; q < nseg; q += 32)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double w = __ldcg(part + K * (s_begin + q) + k);
            v[k] = (MAX0 && k == 0) ? fmax(v[k], w) : v[k] + w;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double w = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = (MAX0 && k == 0) ? fmax(v[k], w) : v[k] + w;
        }
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = __shfl_sync(0xffffffffu, v[k], 0);
    return true;
}

// The scalar step of instance i after its phase 2 (lane 0 of the completing warp).
__device__ void finish_step(const BArgs& a, int64_t i, int cur, double gm, double l1n, double rtn) {
    BState st = load_state(&a.state[i]);
    const double tau = st.tau;
    const double P = __dadd_rn(__dmul_rn(tau, st.l1_cur), __dmul_rn(0.5, st.k1[0]));
    const double sc = gm <= tau ? 1.0 : tau / gm;
    const double D = __dadd_rn(__dmul_rn(sc, st.k1[1]), -__dmul_rn(__dmul_rn(__dmul_rn(0.5, sc), sc), st.k1[2]));
    st.best_d = fmax(st.best_d, D);
    const double gap = P - st.best_d;
    const double rel = gap / fmax(fabs(P), 1e-300);
    const bool bad = !isfinite(P) || !isfinite(D);
    if (bad || rel <= st.tol || st.iter - 1 >= st.max_iter) {
        BResult& R = a.results[i * a.ntau_max + st.tau_idx];
        R.P = P;
        R.D = st.best_d;
        R.gap = gap;
        R.rel = rel;
        R.iters = st.iter - 1;
        R.status = bad ? L1LS_ENUMERIC : (rel <= st.tol ? L1LS_OK : L1LS_ENOCONV);
        R.done = 1;
        if (!bad && st.tau_idx + 1 < st.ntau) {
            st.tau_idx += 1;
            st.tau = a.taus[i * a.ntau_max + st.tau_idx];
            st.t = 1.0;
            st.beta = 0.0;
            st.best_d = -INFINITY;
            st.iter = 1;
            st.l1_cur = l1n;          // warm start: the iterate just computed
        } else {
            st.stop = 1;
            st.final_buf = cur;      // the certified iterate x_{k-1}
            atomicSub(a.active, 1);
        }
    } else {
        if (st.restart && rtn > 0.0) {
            st.t = 1.0;
            st.beta = 0.0;
        } else {
            const double tk = st.t;
            const double tn = __dmul_rn(0.5, __dadd_rn(1.0, sqrt(__dadd_rn(1.0, __dmul_rn(__dmul_rn(4.0, tk), tk)))));
            st.beta = (tk - 1.0) / tn;
            st.t = tn;
        }
        st.l1_cur = l1n;
        st.iter += 1;
    }
    split_ff(st.beta, st.beta_ff);
    split_ff(1.0 / st.L, st.invL_ff);
    split_ff(st.tau / st.L, st.thr_ff);
    a.state[i] = st;
}

// One row-pair segment (tiles t0 .. t1-1) of instance d: K1's product and epilogue; returns
// the segment's partials ||A x - b||^2, b.r, r.r in out (lane 0).  Not inlined: the two phases
// then get their registers allocated separately.
template <class V, int EPL, int BLOCK, class Smem>
__device__ __noinline__ void row_segment(const BDesc* __restrict__ dp, int cur, ff beta, int64_t t0, int64_t t1,
                                         Smem& sm, StageState& ss, int* err, double* out) {
    const int32_t* rptr = dp->rptr;
    const int32_t* rcol = dp->rcol;
    const V* rval = static_cast<const V*>(dp->rval);
    const float* xh = reinterpret_cast<const float*>(dp->x[cur]);   // interleaved pairs
    const float* xl = nullptr;
    float2* ax = dp->ax;
    const float* bv = dp->b;
    float* resf = reinterpret_cast<float*>(dp->res);
    const int64_t npairs = dp->m / 2;
    ff q0 = {0.f, 0.f}, q1 = {0.f, 0.f}, q2 = {0.f, 0.f};
    struct Ops {
        ff axo;
        float bb;
    };
    auto pre = [ax, bv](int64_t r, bool has) {
        Ops o{{0.f, 0.f}, 0.f};
        if (has) {   // A x_{k-1} and b: last use in this step (evict-first, as in K1)
            const float2 v = __ldcs(ax + r);
            o.axo = {v.x, v.y};
            o.bb = __ldcs(bv + r);
        }
        return o;
    };
    auto epi = [&](int64_t r, ff u, const Ops& o) {
        // A y = A x_k + beta (A x_k - A x_{k-1}), r = b - A y (Sec. 8.1)
        const ff ay = ff_add(u, ff_mul(beta, ff_sub(u, o.axo)));
        const ff rr = ff_sub(ff_from_float(o.bb), ay);
        __stcs(ax + r, make_float2(u.hi, u.lo));
        resf[4 * (r >> 1) + (r & 1)] = rr.hi;
        resf[4 * (r >> 1) + 2 + (r & 1)] = rr.lo;
        const ff dd = ff_sub(u, ff_from_float(o.bb));
        sum2_add(q0, ff_mul(dd, dd));
        sum2_add(q1, ff_mul(ff_from_float(o.bb), rr));
        sum2_add(q2, ff_mul(rr, rr));
    };
    if constexpr (EPL == 0)
        staged_tiles<true, V, BLOCK>(t0, 1, t1, rptr, rcol, rval, npairs, sm, ss, err, FFSum<true, V, true>{xh, xl, nullptr},
                                     pre, epi);
    else
        tiles_ff<true, true, V, EPL, true>(t0, t1, rptr, rcol, rval, xh, xl, nullptr, npairs, sm.warp_buf(), pre, epi);
    q0 = warp_sum_ff(q0);
    q1 = warp_sum_ff(q1);
    q2 = warp_sum_ff(q2);
    out[0] = ff_to_double(q0);
    out[1] = ff_to_double(q1);
    out[2] = ff_to_double(q2);
}

// One column segment of instance d: K2's product, momentum and shrinkage into x[nxt];
// returns max |A^T r|, sum |x_{k+1}| and the restart test's partial in out (lane 0).
template <class V, int EPL, int BLOCK, class Smem>
__device__ __noinline__ void col_segment(const BDesc* __restrict__ dp, int cur, ff beta_f, ff invL_f, ff thr_f,
                                         bool rs, int64_t t0, int64_t t1, Smem& sm, StageState& ss, int* err,
                                         double* out) {
    const int32_t* cptr = dp->cptr;
    const int32_t* cpair = dp->cpair;
    const V* cval = static_cast<const V*>(dp->cval);
    const float4* res = dp->res;
    const float2* x1p = dp->x[cur];
    float2* x0p = dp->x[cur ^ 1];
    const int64_t n = dp->n;
    float gmax = 0.0f;
    ff l1 = {0.0f, 0.0f}, rt = {0.0f, 0.0f};
    struct Ops {
        ff x1, x0;
    };
    auto pre = [x1p, x0p](int64_t j, bool has) {
        Ops o{{0.f, 0.f}, {0.f, 0.f}};
        if (has) {   // both iterates: last use before x_{k-1} is overwritten (evict-first)
            const float2 a = __ldcs(x1p + j), b = __ldcs(x0p + j);
            o.x1 = {a.x, a.y};
            o.x0 = {b.x, b.y};
        }
        return o;
    };
    auto epi = [&](int64_t j, ff g, const Ops& o) {
        // y = x_k + beta (x_k - x_{k-1}); x_{k+1} = S_{tau/L}(y + A^T r / L) (Sec. 8.1)
        const FfStep f = ff_fista_step(o.x1, o.x0, g, beta_f, invL_f, thr_f);
        x0p[j] = make_float2(f.x.hi, f.x.lo);
        gmax = fmaxf(gmax, fabsf(g.hi));
        sum2_add(l1, f.mag);
        if (rs) sum2_add(rt, ff_mul(ff_sub(f.y, f.x), ff_sub(f.x, o.x1)));
    };
    if constexpr (EPL == 0)
        staged_tiles<false, V, BLOCK>(t0, 1, t1, cptr, cpair, cval, n, sm, ss, err, FFSum<false, V, true>{nullptr, nullptr, res},
                                      pre, epi);
    else
        tiles_ff<false, true, V, EPL, true>(t0, t1, cptr, cpair, cval, nullptr, nullptr, res, n, sm.warp_buf(), pre, epi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_down_sync(0xffffffffu, gmax, o));
    l1 = warp_sum_ff(l1);
    rt = warp_sum_ff(rt);
    out[0] = (double)gmax;
    out[1] = ff_to_double(l1);
    out[2] = ff_to_double(rt);
}

// EPL = 0: the staged stream (each lane sums its own row from shared memory); 4 or 8: lane
// runs of EPL entries summed through a warp buffer.  Registers are sized for
// L1LS_BATCH_WARPS_PER_SM resident warps (a build parameter; with 128-thread blocks 20 allows
// 96 registers with about 40 bytes of spills, 24 allows 80 with about 110 and 32 allows 64:
// on a shortened C4 run 0.610, 0.647 and 0.871 ms per step).
#ifndef L1LS_BATCH_WARPS_PER_SM
#define L1LS_BATCH_WARPS_PER_SM 20
#endif
// The tau path of Sec. 8.8 for a batch of instances: FISTA (Sec. 8.1) with warm starts along
// each path, all instances in one persistent kernel.
template <int BLOCK, int EPL, class V>
__global__ void __launch_bounds__(BLOCK, L1LS_BATCH_WARPS_PER_SM * 32 / BLOCK) k_batch(BArgs a) {
    using Smem = typename std::conditional<EPL == 0, PairedSmem<V, BLOCK>, CompSmem<BLOCK>>::type;
    __shared__ Smem sm;
    const int lane = threadIdx.x & 31;
    StageState ss{0, 0, false};
    if constexpr (EPL == 0) stage_init(sm, ss);
    for (int s = 0; s < a.steps; ++s) {
        if (*(volatile int*)a.active == 0) return;
        const int64_t step = a.step0 + s;
        const int cur = (int)(step & 1);
        // phase 2's segment counter is idle until after the next barrier
        if (blockIdx.x == 0 && threadIdx.x == 0) a.fetch[1] = 0u;
        // ---- phase 1: row-pair segments (A x, residual, gap partials), taken in turn
        for (;;) {
            unsigned got = 0;
            if (lane == 0) got = atomicAdd(a.fetch, 1u);
            const int64_t sg = __shfl_sync(0xffffffffu, got, 0);
            if (sg >= a.nseg1) break;
            const int i = a.sinst1[sg];
            if (__ldcg(&a.state[i].stop)) continue;
            const BDesc* dp = a.desc + i;
            const int64_t sb = dp->s1_begin, ns = dp->ns1;
            const int64_t t0 = (sg - sb) * kSegTiles, t1 = min(dp->n1, t0 + kSegTiles);
            double part[3];
            const ff beta = {__ldcg(&a.state[i].beta_ff[0]), __ldcg(&a.state[i].beta_ff[1])};
            row_segment<V, EPL, BLOCK>(dp, cur, beta, t0, t1, sm, ss, a.err, part);
            if (lane == 0)
                for (int k = 0; k < 3; ++k) a.part1[3 * sg + k] = part[k];
            double tot[3];
            if (segment_done<3, false>(sb, ns, a.part1, a.instcnt1 + i, tot) && lane == 0)
                for (int k = 0; k < 3; ++k) a.state[i].k1[k] = tot[k];
        }
        if (!grid_sync(a.bar_count, a.bar_gen, a.err, a.max_polls, a.extra_arrivals)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.fetch[0] = 0u;
        // ---- phase 2: column segments (A^T r, momentum, shrinkage), then the scalar step
        for (;;) {
            unsigned got = 0;
            if (lane == 0) got = atomicAdd(a.fetch + 1, 1u);
            const int64_t g2 = __shfl_sync(0xffffffffu, got, 0);
            if (g2 >= a.nseg2) break;
            // in the reverse order of phase 1: the phase starts on the residuals phase 1 wrote
            // last (still in L2), and the next phase 1 on the iterates this phase writes last
            const int64_t sg = a.nseg2 - 1 - g2;
            const int i = a.sinst2[sg];
            if (__ldcg(&a.state[i].stop)) continue;
            const BDesc* dp = a.desc + i;
            const int64_t sb = dp->s2_begin, ns = dp->ns2;
            const int64_t t0 = (sg - sb) * kSegTiles, t1 = min(dp->n2, t0 + kSegTiles);
            double part[3];
            const BState* sp = a.state + i;
            col_segment<V, EPL, BLOCK>(dp, cur, {__ldcg(&sp->beta_ff[0]), __ldcg(&sp->beta_ff[1])},
                                {__ldcg(&sp->invL_ff[0]), __ldcg(&sp->invL_ff[1])},
                                {__ldcg(&sp->thr_ff[0]), __ldcg(&sp->thr_ff[1])}, __ldcg(&sp->restart) != 0, t0, t1,
                                sm, ss, a.err, part);
            if (lane == 0)
                for (int k = 0; k < 3; ++k) a.part2[3 * sg + k] = part[k];
            double tot[3];
            if (segment_done<3, true>(sb, ns, a.part2, a.instcnt2 + i, tot) && lane == 0)
                finish_step(a, i, cur, tot[0], tot[1], tot[2]);
        }
        if (!grid_sync(a.bar_count, a.bar_gen, a.err, a.max_polls, a.extra_arrivals)) return;
    }
}

__global__ void k_ff2d_b(const float2* __restrict__ x, int64_t n, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ff_to_double({x[i].x, x[i].y});
}

}  // namespace

struct Batch {
    Ctx* ctx = nullptr;
    std::vector<Inst*> insts;
    int dtype = L1LS_F32;
    int64_t nseg1 = 0, nseg2 = 0;
    BDesc* d_desc = nullptr;
    BState* d_state = nullptr;
    int32_t* d_sinst1 = nullptr;
    int32_t* d_sinst2 = nullptr;
    double* d_part1 = nullptr;
    double* d_part2 = nullptr;
    unsigned* d_cnt = nullptr;    // instance counters of phase 1, then of phase 2
    unsigned* d_bar = nullptr;    // [count, gen]
    int* d_err = nullptr;
    int* d_active = nullptr;
    float* slab = nullptr;        // per-instance vectors
    size_t slab_bytes = 0;
    std::vector<BDesc> desc;
    int sched = -1;               // schedule chosen by the autotuner (-1: not yet)
    double tune_ms[4] = {0, 0, 0, 0};
    int64_t last_steps = 0;       // of the last solve
    double last_ms = 0.0;
    struct Alloc {
        void* p;
        size_t bytes;
    };
    std::vector<Alloc> allocs;
    template <class T> l1ls_status get(T** p, int64_t count) {
        size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
        L1LS_TRY(ctx->alloc(reinterpret_cast<void**>(p), bytes));
        allocs.push_back({*p, bytes});
        return L1LS_OK;
    }
    ~Batch() {
        for (auto& a : allocs) ctx->release(a.p, a.bytes);
    }
};

namespace {

// Schedules: (threads per block, entries per lane and chunk) of the persistent kernel; 0
// entries per lane = the staged stream.
constexpr int kSchedBlock[4] = {256, 128, 256, 128};
constexpr int kSchedEPL[4] = {0, 0, 8, 8};

template <int BLOCK, int EPL, class V>
l1ls_status launch_batch(Batch* B, BArgs& args, cudaStream_t st, int* grid_out) {
    auto kern = k_batch<BLOCK, EPL, V>;
    int per_sm = 0;
    L1LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, 0));
    if (per_sm < 1) return set_error(L1LS_ECUDA, "batched kernel does not fit on an SM");
    int grid = per_sm * B->ctx->num_sms;
    *grid_out = grid;
    void* params[] = {&args};
    L1LS_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(BLOCK), params, 0, st));
    return L1LS_OK;
}

template <class V>
l1ls_status launch_sched(Batch* B, int sched, BArgs& args, cudaStream_t st) {
    int grid = 0;
    switch (sched) {
        case 0: return launch_batch<256, 0, V>(B, args, st, &grid);
        case 1: return launch_batch<128, 0, V>(B, args, st, &grid);
        case 2: return launch_batch<256, 8, V>(B, args, st, &grid);
        default: return launch_batch<128, 8, V>(B, args, st, &grid);
    }
}

l1ls_status launch_any(Batch* B, int sched, BArgs& args, cudaStream_t st) {
    if (B->dtype == L1LS_F32) return launch_sched<float>(B, sched, args, st);
    return launch_sched<__nv_bfloat16>(B, sched, args, st);
}

}  // namespace

}  // namespace l1ls

using namespace l1ls;

extern "C" l1ls_status l1ls_batch_create(l1ls_ctx* hctx, int count, l1ls_inst* const* hinsts, l1ls_batch** out) {
    if (!hctx || !hinsts || !out || count < 1) return set_error(L1LS_EINVAL, "bad argument");
    Ctx* ctx = reinterpret_cast<Ctx*>(hctx);
    L1LS_CUDA(cudaSetDevice(ctx->device));
    Batch* B = new Batch();
    B->ctx = ctx;
    auto fail = [&](l1ls_status s) {
        delete B;
        return s;
    };
    for (int i = 0; i < count; ++i) {
        Inst* I = reinterpret_cast<Inst*>(hinsts[i]);
        if (!I || I->ctx != ctx) return fail(set_error(L1LS_EINVAL, "instance %d is NULL or from another context", i));
        if (!I->paired) return fail(set_error(L1LS_EINVAL, "instance %d: batches need one left stage (paired storage)", i));
        if (I->dtype == L1LS_F64) return fail(set_error(L1LS_EINVAL, "instance %d: batches take FP32 or BF16 values", i));
        if (i > 0 && I->dtype != B->insts[0]->dtype)
            return fail(set_error(L1LS_EINVAL, "instance %d: all instances of a batch share one value type", i));
        B->insts.push_back(I);
    }
    B->dtype = B->insts[0]->dtype;
    // per-instance float-float vectors in one slab: ax, res (m rows), x[2] (n), each padded to
    // whole tiles (offsets stay multiples of 256 bytes)
    size_t floats = 0;
    for (Inst* I : B->insts) floats += 4 * (size_t)pad32(I->m) + 4 * (size_t)pad32(I->n);
    float* slab = nullptr;
    l1ls_status s = B->get(&slab, (int64_t)floats);
    if (s != L1LS_OK) return fail(s);
    B->slab = slab;
    B->slab_bytes = floats * sizeof(float);
    std::vector<int32_t> t1, t2;
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        Inst* I = B->insts[i];
        BDesc d{};
        d.rptr = I->prow_ptr;
        d.rcol = I->prow_col;
        d.rval = I->prow_val;
        d.cptr = I->pcol_ptr;
        d.cpair = I->pcol_pair;
        d.cval = I->pcol_val;
        d.b = I->bhat32;
        d.ax = reinterpret_cast<float2*>(slab + off);
        off += 2 * (size_t)pad32(I->m);
        d.res = reinterpret_cast<float4*>(slab + off);
        off += 2 * (size_t)pad32(I->m);
        for (int k = 0; k < 2; ++k) {
            d.x[k] = reinterpret_cast<float2*>(slab + off);
            off += 2 * (size_t)pad32(I->n);
        }
        d.m = I->m;
        d.n = I->n;
        const int64_t n1 = (I->m / 2 + 31) / 32, n2 = (I->n + 31) / 32;
        d.n1 = n1;
        d.n2 = n2;
        d.ns1 = (n1 + kSegTiles - 1) / kSegTiles;
        d.ns2 = (n2 + kSegTiles - 1) / kSegTiles;
        d.s1_begin = (int64_t)t1.size();
        d.s2_begin = (int64_t)t2.size();
        t1.insert(t1.end(), (size_t)d.ns1, i);
        t2.insert(t2.end(), (size_t)d.ns2, i);
        B->desc.push_back(d);
    }
    B->nseg1 = (int64_t)t1.size();
    B->nseg2 = (int64_t)t2.size();
    if ((s = B->get(&B->d_desc, count)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_state, count)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_sinst1, B->nseg1)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_sinst2, B->nseg2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_part1, 3 * B->nseg1)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_part2, 3 * B->nseg2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_cnt, 2 * (int64_t)count + 2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_bar, 2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_err, 1)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_active, 1)) != L1LS_OK) return fail(s);
    cudaError_t e = cudaMemcpy(B->d_desc, B->desc.data(), sizeof(BDesc) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_sinst1, t1.data(), sizeof(int32_t) * t1.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_sinst2, t2.data(), sizeof(int32_t) * t2.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(batch tables)", __FILE__, __LINE__));
    *out = reinterpret_cast<l1ls_batch*>(B);
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_batch_free(l1ls_batch* h) {
    if (!h) return set_error(L1LS_EINVAL, "batch is NULL");
    Batch* B = reinterpret_cast<Batch*>(h);
    cudaSetDevice(B->ctx->device);
    cudaDeviceSynchronize();
    delete B;
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_batch_solve_path(l1ls_batch* h, const double* taus, int ntau, const l1ls_solve_opts* o,
                                             l1ls_result* results, double* const* x_out, void* stream) {
    if (!h || !taus || ntau < 1 || !o) return set_error(L1LS_EINVAL, "bad argument");
    if (!(o->rel_gap_tol >= 0.0) || o->max_iter < 0) return set_error(L1LS_EINVAL, "bad solver options");
    Batch* B = reinterpret_cast<Batch*>(h);
    L1LS_CUDA(cudaSetDevice(B->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const int count = (int)B->insts.size();
    for (int64_t i = 0; i < (int64_t)count * ntau; ++i)
        if (!(taus[i] > 0.0)) return set_error(L1LS_EINVAL, "tau values must be > 0");
    // device copies of the path and result slots (allocated per call)
    double* d_taus = nullptr;
    BResult* d_res = nullptr;
    L1LS_CUDA(cudaMallocAsync((void**)&d_taus, sizeof(double) * count * ntau, st));
    L1LS_CUDA(cudaMallocAsync((void**)&d_res, sizeof(BResult) * count * ntau, st));
    L1LS_CUDA(cudaMemcpyAsync(d_taus, taus, sizeof(double) * count * ntau, cudaMemcpyHostToDevice, st));
    L1LS_CUDA(cudaMemsetAsync(d_res, 0, sizeof(BResult) * count * ntau, st));
    std::vector<BState> hs(count);
    for (int i = 0; i < count; ++i) {
        BState& s = hs[i];
        memset(&s, 0, sizeof(s));
        s.tau = taus[(int64_t)i * ntau];
        s.L = B->insts[i]->lipschitz;
        s.tol = o->rel_gap_tol;
        s.max_iter = o->max_iter;
        s.t = 1.0;
        s.beta = 0.0;
        s.best_d = -INFINITY;
        s.l1_cur = 0.0;
        s.iter = 1;
        s.ntau = ntau;
        s.restart = o->restart;
        split_ff(0.0, s.beta_ff);
        split_ff(1.0 / s.L, s.invL_ff);
        split_ff(s.tau / s.L, s.thr_ff);
    }
    L1LS_CUDA(cudaMemcpyAsync(B->d_state, hs.data(), sizeof(BState) * count, cudaMemcpyHostToDevice, st));
    L1LS_CUDA(cudaMemsetAsync(B->slab, 0, B->slab_bytes, st));
    L1LS_CUDA(cudaMemsetAsync(B->d_bar, 0, 2 * sizeof(unsigned), st));
    L1LS_CUDA(cudaMemsetAsync(B->d_cnt, 0, sizeof(unsigned) * (2 * (size_t)count + 2), st));
    L1LS_CUDA(cudaMemsetAsync(B->d_err, 0, sizeof(int), st));
    L1LS_CUDA(cudaMemcpyAsync(B->d_active, &count, sizeof(int), cudaMemcpyHostToDevice, st));
    BArgs args{};
    args.desc = B->d_desc;
    args.state = B->d_state;
    args.results = d_res;
    args.taus = d_taus;
    args.sinst1 = B->d_sinst1;
    args.sinst2 = B->d_sinst2;
    args.nseg1 = B->nseg1;
    args.nseg2 = B->nseg2;
    args.part1 = B->d_part1;
    args.part2 = B->d_part2;
    args.instcnt1 = B->d_cnt;
    args.instcnt2 = B->d_cnt + count;
    args.fetch = B->d_cnt + 2 * count;
    args.max_polls = kBarrierPolls;
    args.extra_arrivals = 0;
    args.ninst = count;
    args.ntau_max = ntau;
    args.bar_count = B->d_bar;
    args.bar_gen = B->d_bar + 1;
    args.err = B->d_err;
    args.active = B->d_active;
    int64_t step = 0;
    const int chunk = o->check_every > 0 ? o->check_every : 32;
    cudaEvent_t ev[2];
    L1LS_CUDA(cudaEventCreate(&ev[0]));
    L1LS_CUDA(cudaEventCreate(&ev[1]));
    L1LS_CUDA(cudaEventRecord(ev[0], st));
    // autotuner: time four steps of each schedule on the live solve (results do not depend on
    // the schedule: every sum keeps its order), keep the fastest
    if (B->sched < 0) {
        cudaEvent_t e0, e1;
        L1LS_CUDA(cudaEventCreate(&e0));
        L1LS_CUDA(cudaEventCreate(&e1));
        for (int c = 0; c < 4; ++c) {
            args.step0 = step;
            args.steps = 4;
            L1LS_CUDA(cudaEventRecord(e0, st));
            L1LS_TRY(launch_any(B, c, args, st));
            L1LS_CUDA(cudaEventRecord(e1, st));
            L1LS_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            L1LS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            B->tune_ms[c] = ms;
            step += 4;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        B->sched = 0;
        for (int c = 1; c < 4; ++c)
            if (B->tune_ms[c] < B->tune_ms[B->sched]) B->sched = c;
    }
    l1ls_status final_status = L1LS_OK;
    const int64_t max_steps = (o->max_iter + 2) * (int64_t)ntau + 16;
    for (;;) {
        int active = 0, err = 0;
        L1LS_CUDA(cudaMemcpyAsync(&active, B->d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        L1LS_CUDA(cudaMemcpyAsync(&err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        L1LS_CUDA(cudaStreamSynchronize(st));
        if (err) {
            final_status = err == kStageTimeout
                               ? set_error(L1LS_ECUDA, "batched FISTA: a bulk-copy stage wait ran out of polls")
                               : set_error(L1LS_ECUDA, "batched FISTA: a bounded grid barrier expired");
            break;
        }
        if (active == 0) break;
        if (step > max_steps) {
            final_status = set_error(L1LS_ECUDA, "internal: batched FISTA did not retire its instances");
            break;
        }
        if (o->time_limit_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->time_limit_s) {
            final_status = L1LS_ETIMEOUT;
            break;
        }
        args.step0 = step;
        args.steps = chunk;
        L1LS_TRY(launch_any(B, B->sched, args, st));
        step += chunk;
    }
    L1LS_CUDA(cudaEventRecord(ev[1], st));
    L1LS_CUDA(cudaEventSynchronize(ev[1]));
    float loop_ms = 0.f;
    L1LS_CUDA(cudaEventElapsedTime(&loop_ms, ev[0], ev[1]));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    B->last_steps = step;
    B->last_ms = loop_ms;
    std::vector<BResult> hr((size_t)count * ntau);
    L1LS_CUDA(cudaMemcpyAsync(hr.data(), d_res, sizeof(BResult) * count * ntau, cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaMemcpyAsync(hs.data(), B->d_state, sizeof(BState) * count, cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (results) {
        for (int64_t k = 0; k < (int64_t)count * ntau; ++k) {
            l1ls_result& r = results[k];
            memset(&r, 0, sizeof(r));
            r.iters = hr[k].iters;
            r.products = 2 * hr[k].iters + 2;
            r.f = hr[k].P;
            r.dual = hr[k].D;
            r.gap = hr[k].gap;
            r.rel_gap = hr[k].rel;
            // taus finished before a time limit or an error keep their own status
            r.status = hr[k].done ? hr[k].status : (final_status == L1LS_OK ? L1LS_ECUDA : final_status);
            r.seconds = secs;
        }
    }
    if (x_out && final_status == L1LS_OK) {
        for (int i = 0; i < count; ++i) {
            if (!x_out[i]) continue;
            const BDesc& d = B->desc[i];
            const int fb = hs[i].final_buf;
            double* tmp = nullptr;
            L1LS_CUDA(cudaMallocAsync((void**)&tmp, sizeof(double) * d.n, st));
            k_ff2d_b<<<(unsigned)((d.n + 255) / 256), 256, 0, st>>>(d.x[fb], d.n, tmp);
            L1LS_CUDA(cudaGetLastError());
            L1LS_CUDA(cudaMemcpyAsync(x_out[i], tmp, sizeof(double) * d.n, cudaMemcpyDefault, st));
            L1LS_CUDA(cudaFreeAsync(tmp, st));
        }
    }
    L1LS_CUDA(cudaFreeAsync(d_taus, st));
    L1LS_CUDA(cudaFreeAsync(d_res, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    return final_status;
}

extern "C" l1ls_status l1ls_batch_get_schedule(const l1ls_batch* h, int* block, int* entries_per_lane,
                                               double* tune_ms) {
    if (!h) return set_error(L1LS_EINVAL, "batch is NULL");
    const Batch* B = reinterpret_cast<const Batch*>(h);
    if (block) *block = B->sched < 0 ? 0 : kSchedBlock[B->sched];
    if (entries_per_lane) *entries_per_lane = B->sched < 0 ? 0 : kSchedEPL[B->sched];
    if (tune_ms)
        for (int c = 0; c < 4; ++c) tune_ms[c] = B->tune_ms[c];
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_batch_get_stats(const l1ls_batch* h, int64_t* steps, double* device_ms) {
    if (!h) return set_error(L1LS_EINVAL, "batch is NULL");
    const Batch* B = reinterpret_cast<const Batch*>(h);
    if (steps) *steps = B->last_steps;
    if (device_ms) *device_ms = B->last_ms;
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_batch_barrier_selftest(l1ls_batch* h, uint32_t max_polls, double* seconds) {
    if (!h || max_polls < 1) return set_error(L1LS_EINVAL, "bad argument");
    Batch* B = reinterpret_cast<Batch*>(h);
    L1LS_CUDA(cudaSetDevice(B->ctx->device));
    const int count = (int)B->insts.size();
    cudaStream_t st = nullptr;
    L1LS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    // every instance stopped (phase 1 has no work), one active so the step starts
    std::vector<BState> hs(count);
    for (auto& x : hs) {
        memset(&x, 0, sizeof(x));
        x.stop = 1;
    }
    const int one = 1;
    L1LS_CUDA(cudaMemcpyAsync(B->d_state, hs.data(), sizeof(BState) * count, cudaMemcpyHostToDevice, st));
    L1LS_CUDA(cudaMemsetAsync(B->d_bar, 0, 2 * sizeof(unsigned), st));
    L1LS_CUDA(cudaMemsetAsync(B->d_err, 0, sizeof(int), st));
    L1LS_CUDA(cudaMemsetAsync(B->d_cnt, 0, sizeof(unsigned) * (2 * (size_t)count + 2), st));
    L1LS_CUDA(cudaMemcpyAsync(B->d_active, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    BArgs args{};
    args.desc = B->d_desc;
    args.state = B->d_state;
    args.sinst1 = B->d_sinst1;
    args.sinst2 = B->d_sinst2;
    args.nseg1 = B->nseg1;
    args.nseg2 = B->nseg2;
    args.part1 = B->d_part1;
    args.part2 = B->d_part2;
    args.instcnt1 = B->d_cnt;
    args.instcnt2 = B->d_cnt + count;
    args.fetch = B->d_cnt + 2 * count;
    args.ninst = count;
    args.ntau_max = 1;
    args.bar_count = B->d_bar;
    args.bar_gen = B->d_bar + 1;
    args.err = B->d_err;
    args.active = B->d_active;
    args.step0 = 0;
    args.steps = 1;
    args.max_polls = max_polls;
    args.extra_arrivals = 1;
    auto t0 = std::chrono::steady_clock::now();
    L1LS_TRY(launch_any(B, 1, args, st));
    int err = 0;
    L1LS_CUDA(cudaMemcpyAsync(&err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    L1LS_CUDA(cudaMemsetAsync(B->d_bar, 0, 2 * sizeof(unsigned), st));
    L1LS_CUDA(cudaMemsetAsync(B->d_err, 0, sizeof(int), st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    cudaStreamDestroy(st);
    if (err == 2) return set_error(L1LS_ECUDA, "batched FISTA: a bounded grid barrier expired (self-test)");
    return set_error(L1LS_ECUDA, "self-test: the barrier did not report its expiry (err %d)", err);
}
