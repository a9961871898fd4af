// Serving loop: solve requests (generate an instance, solve it to the gap tolerance, return
// x and the certificate) admitted by device-memory footprint and run concurrently.
//
// Each context owns a pool of worker threads ("slots"), each with its own CUDA stream.  A
// request moves queued -> running -> done; the head of the FIFO queue is admitted as soon as a
// slot is free and its footprint fits next to the requests already running (AdmissionQueue).
// Requests that arrive while others run are admitted as slots and memory free up, and their
// kernels overlap on the device through the slots' streams.  All device memory a request
// uses is allocated and freed stream-ordered on its slot's stream, so no worker forces a
// device-wide synchronisation on the others.  A request's arithmetic depends only on the
// request (grid sizes come from the instance, every reduction has a fixed order), so its
// result is the same alone and in any mix.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "serve_queue.h"

namespace l1ls {

thread_local const std::atomic<int>* tl_cancel = nullptr;

namespace {

struct Payload {
    l1ls_gen_params gp;
    l1ls_solve_opts so;
    int method;
};

struct Outcome {
    l1ls_status status = L1LS_OK;
    l1ls_result res{};
    std::vector<double> x;
    std::string message;
};

using Queue = AdmissionQueue<Payload, Outcome>;

struct Server {
    Ctx* ctx;
    Queue q;
    int slots;
    std::vector<std::thread> workers;
    Server(Ctx* c, size_t capacity, int s) : ctx(c), q(capacity), slots(s) {}
};

void worker_main(Server* S) {
    Ctx* ctx = S->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    while (Queue::Ptr r = S->q.acquire()) {
        Outcome out;
        if (!st) {
            out.status = set_error(L1LS_ECUDA, "serving slot has no CUDA stream");
            out.message = l1ls_last_error();
            out.res.status = out.status;
            S->q.complete(r, out);
            continue;
        }
        tl_cancel = &r->cancel_flag;
        const Payload& p = r->payload;
        Inst* I = nullptr;
        l1ls_status s = generate_instance(ctx, &p.gp, st, &I, true);
        if (s == L1LS_OK) {
            out.x.assign((size_t)I->n, 0.0);
            l1ls_solve_opts o = p.so;
            if (o.tau < 0.0) o.tau = -o.tau * I->lam_max;     // relative to lambda_max
            s = p.method == L1LS_PDNCG ? pdncg_solve(I, &o, nullptr, out.x.data(), &out.res, st)
                                       : fista_solve(I, &o, nullptr, out.x.data(), &out.res, st);
        } else {
            out.res.status = s;
        }
        out.status = s;
        if (s != L1LS_OK) out.message = l1ls_last_error();
        if (I) {
            cudaStreamSynchronize(st);
            I->free_all();                 // stream-ordered frees on this slot's stream
            delete I;
        }
        cudaStreamSynchronize(st);
        tl_cancel = nullptr;
        S->q.complete(r, out);
    }
    if (st) cudaStreamDestroy(st);
}

void stop_server(void* p) {
    Server* S = static_cast<Server*>(p);
    S->q.close();
    for (auto& t : S->workers) t.join();
    delete S;
}

// Device memory one request may hold at its peak: the instance (both orientations, the
// paired copies, vectors), the generator's temporaries or the solver's work space, whichever
// is larger.  An upper bound: every right stage widens the rows of R^T e_j by at most one
// entry on each side, a left stage doubles them, a column of N~ has d entries.
size_t footprint(const l1ls_gen_params& gp, int method) {
    const double m = (double)gp.m, n = (double)gp.n;
    const double nsq = std::min(m, n), extra = n > m ? n - m : 0.0;
    const double v = (double)dtype_size(gp.value_dtype);
    const double per_col = (2.0 * gp.right_stages + 1.0) * (gp.left_stages ? 2.0 : 1.0);
    const double nnz = nsq * per_col + extra * (double)gp.n_nnz_per_col + 64.0;
    const bool paired = gp.left_stages == 1 && m >= n;
    double inst = nnz * 2.0 * (v + 4.0) + (paired ? nnz * (2.0 * v + 4.0) : 0.0);
    inst += m * (8.0 + 4.0 + 4.0 * 4.0) + n * 8.0 * 3.0 + 64.0 * 1024.0;
    const double gen_tmp = nnz * 16.0 + (m + n) * 64.0 + nnz * 2.0 * (v + 4.0);
    const double solver = method == L1LS_PDNCG ? (n * 8.0 * 16.0 + m * 8.0 * 8.0) : (n * 8.0 * 8.0 + m * 8.0 * 6.0);
    const double bytes = inst + std::max(gen_tmp, solver) + 4.0 * 1024.0 * 1024.0;
    return (size_t)std::ceil(bytes * 1.25);
}

l1ls_status get_server(Ctx* ctx, Server** out, int slots, size_t capacity, bool create_only) {
    std::lock_guard<std::mutex> g(ctx->server_mu);
    if (ctx->server) {
        if (create_only) return set_error(L1LS_EBUSY, "the serving loop is already running");
        *out = static_cast<Server*>(ctx->server);
        return L1LS_OK;
    }
    if (slots < 1) slots = 8;
    if (capacity == 0) {
        std::lock_guard<std::mutex> m(ctx->mem_mu);
        capacity = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
    }
    // keep memory freed by finished requests in the stream-ordered pool for the next ones
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t thr = (uint64_t)capacity;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    Server* S = new Server(ctx, capacity, slots);
    for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_main, S);
    ctx->server = S;
    ctx->server_stop = stop_server;
    *out = S;
    return L1LS_OK;
}

}  // namespace

}  // namespace l1ls

using namespace l1ls;

extern "C" size_t l1ls_footprint(const l1ls_gen_params* p, int method) { return p ? footprint(*p, method) : 0; }

extern "C" l1ls_status l1ls_serve_config(l1ls_ctx* h, int slots, size_t capacity_bytes) {
    if (!h || slots < 1 || slots > 256) return set_error(L1LS_EINVAL, "bad argument");
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    L1LS_CUDA(cudaSetDevice(ctx->device));
    Server* S = nullptr;
    return get_server(ctx, &S, slots, capacity_bytes, true);
}

extern "C" l1ls_status l1ls_submit(l1ls_ctx* h, const l1ls_gen_params* p, const l1ls_solve_opts* o, int method,
                                   uint64_t* ticket) {
    if (!h || !p || !o || !ticket) return set_error(L1LS_EINVAL, "NULL argument");
    if (method != L1LS_FISTA && method != L1LS_PDNCG) return set_error(L1LS_EINVAL, "unknown method %d", method);
    if (!(o->tau != 0.0) || !std::isfinite(o->tau) || !(o->rel_gap_tol >= 0.0) || o->max_iter < 0)
        return set_error(L1LS_EINVAL, "bad solver options");
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    L1LS_CUDA(cudaSetDevice(ctx->device));
    Server* S = nullptr;
    L1LS_TRY(get_server(ctx, &S, 0, 0, false));
    const size_t fp = footprint(*p, method);
    const uint64_t t = S->q.submit(Payload{*p, *o, method}, fp);
    if (t == 0)
        return set_error(L1LS_EBUSY, "request footprint %zu bytes exceeds the serving capacity %zu bytes", fp,
                         S->q.capacity());
    *ticket = t;
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_poll(l1ls_ctx* h, uint64_t ticket, int wait_ms, l1ls_result* res, double* x_out) {
    if (!h) return set_error(L1LS_EINVAL, "ctx is NULL");
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    Server* S = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->server_mu);
        S = static_cast<Server*>(ctx->server);
    }
    if (!S) return set_error(L1LS_ENOTFOUND, "no request was submitted to this context");
    Queue::Ptr r = S->q.wait(ticket, wait_ms, true);
    if (!r) return set_error(L1LS_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    const double queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
    const double latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (r->state == Queue::kQueued && r->cancelled) {
        if (res) {
            memset(res, 0, sizeof(*res));
            res->status = L1LS_ECANCELLED;
        }
        return set_error(L1LS_ECANCELLED, "request %llu was cancelled before it ran", (unsigned long long)ticket);
    }
    if (r->state != Queue::kDone) return set_error(L1LS_EBUSY, "request %llu is not finished", (unsigned long long)ticket);
    const Outcome& out = r->outcome;
    if (res) {
        *res = out.res;
        res->status = out.status;
        res->queue_s = queue_s;
        res->latency_s = latency_s;
    }
    if (x_out && !out.x.empty()) memcpy(x_out, out.x.data(), sizeof(double) * out.x.size());
    if (out.status != L1LS_OK) return set_error(out.status, "%s", out.message.c_str());
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_cancel(l1ls_ctx* h, uint64_t ticket) {
    if (!h) return set_error(L1LS_EINVAL, "ctx is NULL");
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    Server* S = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->server_mu);
        S = static_cast<Server*>(ctx->server);
    }
    if (!S || !S->q.cancel(ticket)) return set_error(L1LS_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_serve_stats(l1ls_ctx* h, l1ls_serve_info* info) {
    if (!h || !info) return set_error(L1LS_EINVAL, "NULL argument");
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    memset(info, 0, sizeof(*info));
    std::lock_guard<std::mutex> g(ctx->server_mu);
    Server* S = static_cast<Server*>(ctx->server);
    if (!S) return L1LS_OK;
    const Queue::Stats s = S->q.stats();
    info->slots = S->slots;
    info->running = s.running;
    info->peak_running = s.peak_running;
    info->completed = s.completed;
    info->queued = s.queued;
    info->capacity_bytes = S->q.capacity();
    info->reserved_bytes = s.reserved;
    info->peak_reserved_bytes = s.peak_reserved;
    return L1LS_OK;
}
