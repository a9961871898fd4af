// C ABI: contexts, instances, errors, exports, defaults.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>

#include "internal.h"

namespace l1ls {

static thread_local std::string g_last_error;

l1ls_status set_error(l1ls_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

l1ls_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    base = base ? base + 1 : file;
    set_error(e == cudaErrorMemoryAllocation ? L1LS_ENOMEM : L1LS_ECUDA, "%s failed: %s (%s:%d)", what,
              cudaGetErrorString(e), base, line);
    return e == cudaErrorMemoryAllocation ? L1LS_ENOMEM : L1LS_ECUDA;
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

l1ls_status Ctx::alloc(void** p, size_t bytes, cudaStream_t st, bool stream_ordered) {
    {
        std::lock_guard<std::mutex> g(mem_mu);
        if (used + bytes > budget)
            return set_error(L1LS_ENOMEM, "device memory budget exceeded (%zu + %zu > %zu bytes)", used, bytes, budget);
        used += bytes;
    }
    cudaError_t e = stream_ordered ? cudaMallocAsync(p, bytes, st) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> g(mem_mu);
        used -= bytes;
        *p = nullptr;
        return cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
    }
    return L1LS_OK;
}

void Ctx::release(void* p, size_t bytes, cudaStream_t st, bool stream_ordered) {
    if (!p) return;
    if (stream_ordered) cudaFreeAsync(p, st);
    else cudaFree(p);
    std::lock_guard<std::mutex> g(mem_mu);
    used -= bytes;
}

l1ls_status Ctx::staging(int which, size_t bytes, void** out) {
    if (which < 0 || which >= kStages) return set_error(L1LS_EINVAL, "internal: bad staging slot");
    if (stage_bytes[which] < bytes) {
        if (stage[which]) {
            cudaFree(stage[which]);
            stage[which] = nullptr;
            stage_bytes[which] = 0;
        }
        cudaError_t e = cudaMalloc(&stage[which], bytes);
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(staging)", __FILE__, __LINE__);
        stage_bytes[which] = bytes;
    }
    *out = stage[which];
    return L1LS_OK;
}

l1ls_status Inst::alloc(void** p, size_t bytes) {
    L1LS_TRY(ctx->alloc(p, bytes, alloc_st, stream_ordered));
    allocs.push_back({*p, bytes});
    this->bytes += bytes;
    return L1LS_OK;
}

void Inst::free_all() {
    if (fista_work && fista_work_free) fista_work_free(fista_work);
    if (pd_work && pd_work_free) pd_work_free(pd_work);
    fista_work = pd_work = nullptr;
    for (auto& a : allocs) ctx->release(a.p, a.bytes, alloc_st, stream_ordered);
    allocs.clear();
    bytes = 0;
}

}  // namespace l1ls

using namespace l1ls;

extern "C" {

const char* l1ls_last_error(void) { return g_last_error.c_str(); }

const char* l1ls_version(void) { return "l1ls 0.1 (sm_103a)"; }

void l1ls_gen_params_default(l1ls_gen_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->m = 2048;
    p->n = 1024;
    p->seed = 0;
    p->kappa = 100.0;
    p->tau = 1.0;
    p->xstar_frac = 0.05;
    p->xstar_lo = 1.0;
    p->xstar_hi = 10.0;
    p->theta = 2.0 * M_PI / 10.0;
    p->vartheta = NAN;
    p->right_stages = 1;
    p->left_stages = 1;
    p->value_dtype = L1LS_F64;
    p->g_offsupport = 0;
    p->n_nnz_per_col = 8;
    p->sigma_odd = 0.1;
    p->sigma_even = 100.0;
    p->gamma = 100.0;
}

void l1ls_solve_opts_default(l1ls_solve_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tau = 1.0;
    o->rel_gap_tol = 1e-6;
    o->f_target = -INFINITY;
    o->max_iter = 100000;
    o->time_limit_s = 0.0;
    o->mu = 1e-5;
    o->mu_min = 1e-14;
    o->mu_start = 1.0;
    o->pcg_rtol = 0.1;
    o->armijo = 1e-4;
    o->ls_max = 50;
    o->pcg_max = 1000;
    o->check_every = 32;
}

l1ls_status l1ls_create(int device, size_t budget, l1ls_ctx** out) {
    if (!out) return set_error(L1LS_EINVAL, "out is NULL");
    int count = 0;
    L1LS_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return set_error(L1LS_EINVAL, "device %d out of range (%d devices)", device, count);
    L1LS_CUDA(cudaSetDevice(device));
    Ctx* c = new Ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_error(e, "cudaGetDeviceProperties", __FILE__, __LINE__);
    }
    c->num_sms = prop.multiProcessorCount;
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete c;
        return cuda_error(e, "cudaMemGetInfo", __FILE__, __LINE__);
    }
    c->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    if (cudaHostAlloc((void**)&c->pinned, Ctx::kPinnedSlots * Ctx::kPinnedSlotBytes, cudaHostAllocDefault) ==
        cudaSuccess) {
        for (int i = Ctx::kPinnedSlots - 1; i >= 0; --i) c->pinned_free.push_back(i);
    } else {
        cudaGetLastError();
        c->pinned = nullptr;   // read-backs use pageable memory
    }
    *out = reinterpret_cast<l1ls_ctx*>(c);
    return L1LS_OK;
}

void* Ctx::pinned_get(size_t bytes) {
    if (!pinned || bytes > kPinnedSlotBytes) return nullptr;
    std::lock_guard<std::mutex> g(pinned_mu);
    if (pinned_free.empty()) return nullptr;
    const int i = pinned_free.back();
    pinned_free.pop_back();
    return pinned + (size_t)i * kPinnedSlotBytes;
}

void Ctx::pinned_put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(pinned_mu);
    pinned_free.push_back((int)((static_cast<char*>(p) - pinned) / (ptrdiff_t)kPinnedSlotBytes));
}

l1ls_status l1ls_destroy(l1ls_ctx* h) {
    if (!h) return set_error(L1LS_EINVAL, "ctx is NULL");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    cudaSetDevice(c->device);
    if (c->server && c->server_stop) c->server_stop(c->server);   // cancels and joins the workers
    c->server = nullptr;
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> g(c->inst_mu);
        for (Inst* I : c->insts) {
            I->free_all();
            delete I;
        }
        c->insts.clear();
    }
    for (int i = 0; i < Ctx::kStages; ++i)
        if (c->stage[i]) cudaFree(c->stage[i]);
    if (c->pinned) cudaFreeHost(c->pinned);
    delete c;
    return L1LS_OK;
}

l1ls_status l1ls_generate(l1ls_ctx* h, const l1ls_gen_params* p, void* stream, l1ls_inst** out) {
    if (!h || !p || !out) return set_error(L1LS_EINVAL, "NULL argument");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    L1LS_CUDA(cudaSetDevice(c->device));
    Inst* I = nullptr;
    L1LS_TRY(generate_instance(c, p, (cudaStream_t)stream, &I));
    {
        std::lock_guard<std::mutex> g(c->inst_mu);
        c->insts.push_back(I);
    }
    *out = reinterpret_cast<l1ls_inst*>(I);
    return L1LS_OK;
}

l1ls_status l1ls_inst_free(l1ls_inst* h) {
    if (!h) return set_error(L1LS_EINVAL, "inst is NULL");
    Inst* I = reinterpret_cast<Inst*>(h);
    Ctx* c = I->ctx;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> g(c->inst_mu);
        auto it = std::find(c->insts.begin(), c->insts.end(), I);
        if (it == c->insts.end()) return set_error(L1LS_EINVAL, "instance does not belong to a live context");
        c->insts.erase(it);
    }
    I->free_all();
    delete I;
    return L1LS_OK;
}

l1ls_status l1ls_inst_get_info(const l1ls_inst* h, l1ls_inst_info* info) {
    if (!h || !info) return set_error(L1LS_EINVAL, "NULL argument");
    const Inst* I = reinterpret_cast<const Inst*>(h);
    memset(info, 0, sizeof(*info));
    info->m = I->m;
    info->n = I->n;
    info->nnz = I->nnz;
    info->s = I->s;
    info->f_star = I->f_star;
    info->lipschitz = I->lipschitz;
    info->lam_max = I->lam_max;
    info->tau_gen = I->p.tau;
    info->value_dtype = I->dtype;
    info->right_stages = I->p.right_stages;
    info->left_stages = I->p.left_stages;
    info->igen2 = I->igen2 ? 1 : 0;
    info->matrix_free = I->matrix_free ? 1 : 0;
    info->device_bytes = I->bytes;
    return L1LS_OK;
}

static l1ls_status values_to_host(const Inst* I, const void* dev, int64_t count, std::vector<double>& out) {
    out.resize((size_t)count);
    if (count == 0) return L1LS_OK;
    if (I->dtype == L1LS_F64) {
        L1LS_CUDA(cudaMemcpy(out.data(), dev, sizeof(double) * count, cudaMemcpyDeviceToHost));
    } else if (I->dtype == L1LS_F32) {
        std::vector<float> t((size_t)count);
        L1LS_CUDA(cudaMemcpy(t.data(), dev, sizeof(float) * count, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < count; ++i) out[i] = t[i];
    } else {
        std::vector<uint16_t> t((size_t)count);
        L1LS_CUDA(cudaMemcpy(t.data(), dev, sizeof(uint16_t) * count, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < count; ++i) {
            uint32_t u = (uint32_t)t[i] << 16;
            float f;
            memcpy(&f, &u, 4);
            out[i] = f;
        }
    }
    return L1LS_OK;
}

l1ls_status l1ls_inst_kappa_rho(const l1ls_inst* h, double rho, double* out) {
    if (!h || !out) return set_error(L1LS_EINVAL, "NULL argument");
    const Inst* I = reinterpret_cast<const Inst*>(h);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    return kappa_rho(I, rho, out);
}

l1ls_status l1ls_inst_export(const l1ls_inst* h, int64_t* row_ptr, int32_t* col_idx, double* vals, double* b,
                             double* xstar, double* sigma, int64_t* perm) {
    if (!h) return set_error(L1LS_EINVAL, "inst is NULL");
    const Inst* I = reinterpret_cast<const Inst*>(h);
    if (I->matrix_free && (row_ptr || col_idx || vals))
        return set_error(L1LS_EINVAL, "a matrix-free instance has no assembled A to export");
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    L1LS_CUDA(cudaDeviceSynchronize());
    const int64_t m = I->m, n = I->n, nnz = I->matrix_free ? 0 : I->nnz;
    std::vector<int32_t> pm((size_t)m), st((size_t)m), ptr((size_t)m + 1), col((size_t)nnz);
    L1LS_CUDA(cudaMemcpy(pm.data(), I->perm, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    L1LS_CUDA(cudaMemcpy(st.data(), I->store_of_row, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    if (row_ptr || col_idx || vals) {
        L1LS_CUDA(cudaMemcpy(ptr.data(), I->csr_ptr, sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToHost));
        L1LS_CUDA(cudaMemcpy(col.data(), I->csr_col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
        std::vector<double> v;
        L1LS_TRY(values_to_host(I, I->csr_val, nnz, v));
        int64_t o = 0;
        if (row_ptr) row_ptr[0] = 0;
        for (int64_t i = 0; i < m; ++i) {           // row i of A = stored row store_of_row[i]
            const int64_t r = st[i];
            for (int32_t e = ptr[r]; e < ptr[r + 1]; ++e, ++o) {
                if (col_idx) col_idx[o] = col[e];
                if (vals) vals[o] = v[e];
            }
            if (row_ptr) row_ptr[i + 1] = o;
        }
    }
    if (b) {
        std::vector<double> bh((size_t)m);
        L1LS_CUDA(cudaMemcpy(bh.data(), I->bhat, sizeof(double) * m, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < m; ++i) b[i] = bh[st[i]];
    }
    if (xstar) L1LS_CUDA(cudaMemcpy(xstar, I->xstar, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (sigma) L1LS_CUDA(cudaMemcpy(sigma, I->sigma, sizeof(double) * I->nsq, cudaMemcpyDeviceToHost));
    if (perm)
        for (int64_t i = 0; i < m; ++i) perm[i] = pm[i];
    return L1LS_OK;
}

l1ls_status l1ls_inst_export_t(const l1ls_inst* h, int64_t* col_ptr, int32_t* row_idx, double* vals) {
    if (!h) return set_error(L1LS_EINVAL, "inst is NULL");
    const Inst* I = reinterpret_cast<const Inst*>(h);
    if (I->matrix_free) return set_error(L1LS_EINVAL, "a matrix-free instance has no assembled A to export");
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    L1LS_CUDA(cudaDeviceSynchronize());
    const int64_t m = I->m, n = I->n, nnz = I->nnz;
    std::vector<int32_t> pinv((size_t)m), ptr((size_t)n + 1), row((size_t)nnz);
    L1LS_CUDA(cudaMemcpy(pinv.data(), I->row_of_store, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    L1LS_CUDA(cudaMemcpy(ptr.data(), I->csc_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
    L1LS_CUDA(cudaMemcpy(row.data(), I->csc_row, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
    std::vector<double> v;
    L1LS_TRY(values_to_host(I, I->csc_val, nnz, v));
    std::vector<std::pair<int32_t, double>> tmp;
    for (int64_t j = 0; j < n; ++j) {
        if (col_ptr) col_ptr[j] = ptr[j];
        tmp.clear();
        for (int32_t e = ptr[j]; e < ptr[j + 1]; ++e) tmp.push_back({pinv[row[e]], v[e]});   // original row
        std::sort(tmp.begin(), tmp.end(), [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
            return a.first < b.first;
        });
        for (size_t k = 0; k < tmp.size(); ++k) {
            if (row_idx) row_idx[ptr[j] + k] = tmp[k].first;
            if (vals) vals[ptr[j] + k] = tmp[k].second;
        }
    }
    if (col_ptr) col_ptr[n] = ptr[n];
    return L1LS_OK;
}

}  // extern "C"
