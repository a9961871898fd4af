// Ragged batches of instances solved by FISTA along a tau path (warm-started), in one
// persistent cooperative kernel per chunk of FISTA steps.
//
// The instances keep their own paired matrices, right-hand sides and iterates; the batch adds
// a device table of descriptors and two global tile lists (row-pair tiles and column tiles
// of every instance).  One launch runs `steps` FISTA steps; each step has three phases
// separated by bounded grid barriers:
//   1. every warp takes row-pair tiles of active instances: K1's product, its epilogue and the
//      tile's gap partials, reduced in the warp and written per tile;
//   2. column tiles: K2's product, the momentum and shrinkage, per-tile partials;
//   3. one warp per instance reduces its tiles' partials in tile order (FP64) and takes the
//      scalar step of FISTA (Sec. 8.1) with the certificate; when the tolerance is met it
//      records the result and moves to the next tau of its path, warm-started from the last
//      iterate computed (one prox-gradient step past the certified one), or retires.
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
    float* xh[2];              // iterates x_{k-1}, x_{k-2} (alternating), float-float:
    float* xl[2];              //   high and low words
    int64_t m, n;
    int64_t t1_begin, t2_begin;
};

struct BState {
    double tau, L, tol;
    int64_t max_iter;
    double t, beta, best_d, l1_cur;
    int64_t iter;
    int32_t stop, status, tau_idx, ntau, final_buf, restart;
};

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
    int32_t status, pad;
};

struct BArgs {
    const BDesc* desc;
    BState* state;
    BResult* results;
    const double* taus;        // [inst][ntau]
    const int32_t* tinst1;     // row-pair tile -> instance
    const int32_t* tinst2;     // column tile -> instance
    int64_t ntiles1, ntiles2;
    double* part1;             // [tile][3]
    double* part2;             // [tile][3]
    int ninst, ntau_max;
    unsigned* bar_count;
    unsigned* bar_gen;
    int* err;
    int* active;
    int64_t step0;
    int steps;
};

__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned* gen, int* err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *(volatile unsigned*)gen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            uint32_t polls = 0;
            while (*(volatile unsigned*)gen == g) {
                if (++polls > kBarrierPolls) {
                    ok = 0;
                    atomicExch(err, 2);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

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

template <int BLOCK, class V>
__global__ void __launch_bounds__(BLOCK) k_batch(BArgs a) {
    __shared__ CompSmem<BLOCK> sm;   // 4 * kWarpChunk floats per warp; phase 2 uses half
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (BLOCK / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (BLOCK / 32);
    for (int s = 0; s < a.steps; ++s) {
        if (*(volatile int*)a.active == 0) return;
        const int64_t step = a.step0 + s;
        const int cur = (int)(step & 1), nxt = cur ^ 1;
        // ---- phase 1: row-pair tiles (A x, residual, gap partials)
        for (int64_t t = gw; t < a.ntiles1; t += nw) {
            const int i = a.tinst1[t];
            double* pp = a.part1 + 3 * t;
            if (__ldcg(&a.state[i].stop)) {
                if (lane == 0) pp[0] = pp[1] = pp[2] = 0.0;
                continue;
            }
            const BDesc d = a.desc[i];
            const ff beta = ff_from_double(__ldcg(&a.state[i].beta));
            float* resf = reinterpret_cast<float*>(d.res);
            ff q[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            struct Ops {
                ff axo;
                float bb;
            };
            auto pre = [&](int64_t r, bool has) {
                Ops o{{0.f, 0.f}, 0.f};
                if (has) {
                    const float2 v = d.ax[r];
                    o.axo = {v.x, v.y};
                    o.bb = d.b[r];
                }
                return o;
            };
            auto epi = [&](int64_t r, ff u, const Ops& o) {
                // A y = A x_k + beta (A x_k - A x_{k-1}), r = b - A y (Sec. 8.1)
                const ff ay = ff_add(u, ff_mul(beta, ff_sub(u, o.axo)));
                const ff rr = ff_sub(ff_from_float(o.bb), ay);
                d.ax[r] = make_float2(u.hi, u.lo);
                resf[4 * (r >> 1) + (r & 1)] = rr.hi;
                resf[4 * (r >> 1) + 2 + (r & 1)] = rr.lo;
                const ff dd = ff_sub(u, ff_from_float(o.bb));
                q[0] = ff_add(q[0], ff_mul(dd, dd));
                q[1] = ff_add(q[1], ff_mul(ff_from_float(o.bb), rr));
                q[2] = ff_add(q[2], ff_mul(rr, rr));
            };
            pcsr_tile_ff<true, V>(t - d.t1_begin, d.rptr, d.rcol, static_cast<const V*>(d.rval), d.xh[cur], d.xl[cur],
                                  nullptr, d.m / 2, sm.warp_buf(), pre, epi);
            for (int k = 0; k < 3; ++k) q[k] = warp_sum_ff(q[k]);
            if (lane == 0) {
                pp[0] = ff_to_double(q[0]);
                pp[1] = ff_to_double(q[1]);
                pp[2] = ff_to_double(q[2]);
            }
        }
        if (!grid_sync(a.bar_count, a.bar_gen, a.err)) return;
        // ---- phase 2: column tiles (A^T r, momentum, shrinkage)
        for (int64_t t = gw; t < a.ntiles2; t += nw) {
            const int i = a.tinst2[t];
            double* pp = a.part2 + 3 * t;
            if (__ldcg(&a.state[i].stop)) {
                if (lane == 0) pp[0] = pp[1] = pp[2] = 0.0;
                continue;
            }
            const bool rs = __ldcg(&a.state[i].restart) != 0;
            const BDesc d = a.desc[i];
            const double beta = __ldcg(&a.state[i].beta), L = __ldcg(&a.state[i].L), tau = __ldcg(&a.state[i].tau);
            const ff beta_f = ff_from_double(beta), invL_f = ff_from_double(1.0 / L), thr_f = ff_from_double(tau / L);
            float gmax = 0.0f;
            ff l1 = {0.0f, 0.0f}, rt = {0.0f, 0.0f};
            struct Ops {
                ff x1, x0;
            };
            auto pre = [&](int64_t j, bool has) {
                Ops o{{0.f, 0.f}, {0.f, 0.f}};
                if (has) {
                    o.x1 = {d.xh[cur][j], d.xl[cur][j]};
                    o.x0 = {d.xh[nxt][j], d.xl[nxt][j]};
                }
                return o;
            };
            auto epi = [&](int64_t j, ff g, const Ops& o) {
                // y = x_k + beta (x_k - x_{k-1}); x_{k+1} = S_{tau/L}(y + A^T r / L) (Sec. 8.1)
                const ff y = ff_add(o.x1, ff_mul(beta_f, ff_sub(o.x1, o.x0)));
                const ff v = ff_add(y, ff_mul(g, invL_f));
                const ff xn = ff_soft_threshold(v, thr_f);
                d.xh[nxt][j] = xn.hi;
                d.xl[nxt][j] = xn.lo;
                gmax = fmaxf(gmax, fabsf(g.hi));
                l1 = ff_add(l1, ff_abs(xn));
                if (rs) rt = ff_add(rt, ff_mul(ff_sub(y, xn), ff_sub(xn, o.x1)));
            };
            pcsr_tile_ff<false, V>(t - d.t2_begin, d.cptr, d.cpair, static_cast<const V*>(d.cval), nullptr, nullptr,
                                   d.res, d.n, sm.warp_buf(), pre, epi);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_down_sync(0xffffffffu, gmax, o));
            l1 = warp_sum_ff(l1);
            rt = warp_sum_ff(rt);
            if (lane == 0) {
                pp[0] = (double)gmax;
                pp[1] = ff_to_double(l1);
                pp[2] = ff_to_double(rt);
            }
        }
        if (!grid_sync(a.bar_count, a.bar_gen, a.err)) return;
        // ---- phase 3: one warp per instance, scalar step and tau path
        for (int64_t i = gw; i < a.ninst; i += nw) {
            if (__ldcg(&a.state[i].stop)) continue;
            const BDesc d = a.desc[i];
            const int64_t n1 = (d.m / 2 + 31) / 32, n2 = (d.n + 31) / 32;
            double s0 = 0, s1 = 0, s2 = 0, gm = 0, l1n = 0, rtn = 0;
            for (int64_t t = lane; t < n1; t += 32) {
                const double* pp = a.part1 + 3 * (d.t1_begin + t);
                s0 += __ldcg(pp);
                s1 += __ldcg(pp + 1);
                s2 += __ldcg(pp + 2);
            }
            for (int64_t t = lane; t < n2; t += 32) {
                const double* pp = a.part2 + 3 * (d.t2_begin + t);
                gm = fmax(gm, __ldcg(pp));
                l1n += __ldcg(pp + 1);
                rtn += __ldcg(pp + 2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_down_sync(0xffffffffu, s0, o);
                s1 += __shfl_down_sync(0xffffffffu, s1, o);
                s2 += __shfl_down_sync(0xffffffffu, s2, o);
                gm = fmax(gm, __shfl_down_sync(0xffffffffu, gm, o));
                l1n += __shfl_down_sync(0xffffffffu, l1n, o);
                rtn += __shfl_down_sync(0xffffffffu, rtn, o);
            }
            if (lane == 0) {
                BState st = load_state(&a.state[i]);
                const double tau = st.tau;
                const double P = __dadd_rn(__dmul_rn(tau, st.l1_cur), __dmul_rn(0.5, s0));
                const double sc = gm <= tau ? 1.0 : tau / gm;
                const double D = __dadd_rn(__dmul_rn(sc, s1), -__dmul_rn(__dmul_rn(__dmul_rn(0.5, sc), sc), s2));
                st.best_d = fmax(st.best_d, D);
                const double gap = P - st.best_d;
                const double rel = gap / fmax(fabs(P), 1e-300);
                const bool bad = !isfinite(P) || !isfinite(D);
                if (bad || rel <= st.tol || st.iter - 1 >= st.max_iter) {
                    BResult& R = a.results[(int64_t)i * a.ntau_max + st.tau_idx];
                    R.P = P;
                    R.D = st.best_d;
                    R.gap = gap;
                    R.rel = rel;
                    R.iters = st.iter - 1;
                    R.status = bad ? L1LS_ENUMERIC : (rel <= st.tol ? L1LS_OK : L1LS_ENOCONV);
                    if (!bad && st.tau_idx + 1 < st.ntau) {
                        st.tau_idx += 1;
                        st.tau = a.taus[(int64_t)i * a.ntau_max + st.tau_idx];
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
                        const double tn =
                            __dmul_rn(0.5, __dadd_rn(1.0, sqrt(__dadd_rn(1.0, __dmul_rn(__dmul_rn(4.0, tk), tk)))));
                        st.beta = (tk - 1.0) / tn;
                        st.t = tn;
                    }
                    st.l1_cur = l1n;
                    st.iter += 1;
                }
                a.state[i] = st;
            }
        }
        if (!grid_sync(a.bar_count, a.bar_gen, a.err)) return;
    }
}

__global__ void k_ff2d_b(const float* __restrict__ hi, const float* __restrict__ lo, int64_t n, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ff_to_double({hi[i], lo[i]});
}

}  // namespace

struct Batch {
    Ctx* ctx = nullptr;
    std::vector<Inst*> insts;
    int dtype = L1LS_F32;
    int64_t ntiles1 = 0, ntiles2 = 0;
    BDesc* d_desc = nullptr;
    BState* d_state = nullptr;
    int32_t* d_tinst1 = nullptr;
    int32_t* d_tinst2 = nullptr;
    double* d_part1 = nullptr;
    double* d_part2 = nullptr;
    unsigned* d_bar = nullptr;    // [count, gen]
    int* d_err = nullptr;
    int* d_active = nullptr;
    float* slab = nullptr;        // per-instance vectors
    size_t slab_bytes = 0;
    std::vector<BDesc> desc;
    int block = 0;                // chosen by the autotuner (0: not yet)
    int grid = 0;
    double tune_ms[2] = {0, 0};
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

template <int BLOCK, class V>
l1ls_status launch_batch(Batch* B, BArgs& args, cudaStream_t st, int* grid_out) {
    auto kern = k_batch<BLOCK, V>;
    int per_sm = 0;
    L1LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, 0));
    if (per_sm < 1) return set_error(L1LS_ECUDA, "batched kernel does not fit on an SM");
    int grid = per_sm * B->ctx->num_sms;
    *grid_out = grid;
    void* params[] = {&args};
    L1LS_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(BLOCK), params, 0, st));
    return L1LS_OK;
}

l1ls_status launch_any(Batch* B, int block, BArgs& args, cudaStream_t st) {
    int grid = 0;
    if (B->dtype == L1LS_F32) {
        if (block == 128) return launch_batch<128, float>(B, args, st, &grid);
        return launch_batch<256, float>(B, args, st, &grid);
    }
    if (block == 128) return launch_batch<128, __nv_bfloat16>(B, args, st, &grid);
    return launch_batch<256, __nv_bfloat16>(B, args, st, &grid);
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
            d.xh[k] = slab + off;
            off += pad32(I->n);
            d.xl[k] = slab + off;
            off += pad32(I->n);
        }
        d.m = I->m;
        d.n = I->n;
        d.t1_begin = (int64_t)t1.size();
        d.t2_begin = (int64_t)t2.size();
        const int64_t n1 = (I->m / 2 + 31) / 32, n2 = (I->n + 31) / 32;
        t1.insert(t1.end(), (size_t)n1, i);
        t2.insert(t2.end(), (size_t)n2, i);
        B->desc.push_back(d);
    }
    B->ntiles1 = (int64_t)t1.size();
    B->ntiles2 = (int64_t)t2.size();
    if ((s = B->get(&B->d_desc, count)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_state, count)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_tinst1, B->ntiles1)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_tinst2, B->ntiles2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_part1, 3 * B->ntiles1)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_part2, 3 * B->ntiles2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_bar, 2)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_err, 1)) != L1LS_OK) return fail(s);
    if ((s = B->get(&B->d_active, 1)) != L1LS_OK) return fail(s);
    cudaError_t e = cudaMemcpy(B->d_desc, B->desc.data(), sizeof(BDesc) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_tinst1, t1.data(), sizeof(int32_t) * t1.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_tinst2, t2.data(), sizeof(int32_t) * t2.size(), cudaMemcpyHostToDevice);
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
    }
    L1LS_CUDA(cudaMemcpyAsync(B->d_state, hs.data(), sizeof(BState) * count, cudaMemcpyHostToDevice, st));
    L1LS_CUDA(cudaMemsetAsync(B->slab, 0, B->slab_bytes, st));
    L1LS_CUDA(cudaMemsetAsync(B->d_bar, 0, 2 * sizeof(unsigned), st));
    L1LS_CUDA(cudaMemsetAsync(B->d_err, 0, sizeof(int), st));
    L1LS_CUDA(cudaMemcpyAsync(B->d_active, &count, sizeof(int), cudaMemcpyHostToDevice, st));
    BArgs args{};
    args.desc = B->d_desc;
    args.state = B->d_state;
    args.results = d_res;
    args.taus = d_taus;
    args.tinst1 = B->d_tinst1;
    args.tinst2 = B->d_tinst2;
    args.ntiles1 = B->ntiles1;
    args.ntiles2 = B->ntiles2;
    args.part1 = B->d_part1;
    args.part2 = B->d_part2;
    args.ninst = count;
    args.ntau_max = ntau;
    args.bar_count = B->d_bar;
    args.bar_gen = B->d_bar + 1;
    args.err = B->d_err;
    args.active = B->d_active;
    int64_t step = 0;
    const int chunk = o->check_every > 0 ? o->check_every : 32;
    // autotuner: time two steps with each block size on the live solve (results do not depend
    // on the schedule), keep the faster
    if (B->block == 0) {
        cudaEvent_t e0, e1;
        L1LS_CUDA(cudaEventCreate(&e0));
        L1LS_CUDA(cudaEventCreate(&e1));
        const int cands[2] = {256, 128};
        for (int c = 0; c < 2; ++c) {
            args.step0 = step;
            args.steps = 2;
            L1LS_CUDA(cudaEventRecord(e0, st));
            L1LS_TRY(launch_any(B, cands[c], args, st));
            L1LS_CUDA(cudaEventRecord(e1, st));
            L1LS_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            L1LS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            B->tune_ms[c] = ms;
            step += 2;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        B->block = B->tune_ms[1] < B->tune_ms[0] ? 128 : 256;
    }
    l1ls_status final_status = L1LS_OK;
    const int64_t max_steps = (o->max_iter + 2) * (int64_t)ntau + 16;
    for (;;) {
        int active = 0, err = 0;
        L1LS_CUDA(cudaMemcpyAsync(&active, B->d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        L1LS_CUDA(cudaMemcpyAsync(&err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        L1LS_CUDA(cudaStreamSynchronize(st));
        if (err) {
            final_status = set_error(L1LS_ECUDA, "batched FISTA: a bounded grid barrier expired");
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
        L1LS_TRY(launch_any(B, B->block, args, st));
        step += chunk;
    }
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
            r.status = final_status == L1LS_OK ? hr[k].status : final_status;
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
            k_ff2d_b<<<(unsigned)((d.n + 255) / 256), 256, 0, st>>>(d.xh[fb], d.xl[fb], d.n, tmp);
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

extern "C" l1ls_status l1ls_batch_get_schedule(const l1ls_batch* h, int* block, double* tune_ms_256,
                                               double* tune_ms_128) {
    if (!h) return set_error(L1LS_EINVAL, "batch is NULL");
    const Batch* B = reinterpret_cast<const Batch*>(h);
    if (block) *block = B->block;
    if (tune_ms_256) *tune_ms_256 = B->tune_ms[0];
    if (tune_ms_128) *tune_ms_128 = B->tune_ms[1];
    return L1LS_OK;
}
