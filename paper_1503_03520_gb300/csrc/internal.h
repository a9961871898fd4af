// Internal structures of the l1ls library (host side).  Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/l1ls.h"

namespace l1ls {

// ---- error reporting -------------------------------------------------------------------
l1ls_status set_error(l1ls_status st, const char* fmt, ...);
l1ls_status cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define L1LS_CUDA(...)                                                           \
    do {                                                                         \
        cudaError_t e_ = (__VA_ARGS__);                                          \
        if (e_ != cudaSuccess) return ::l1ls::cuda_error(e_, #__VA_ARGS__, __FILE__, __LINE__); \
    } while (0)

#define L1LS_TRY(...)                                                            \
    do {                                                                         \
        l1ls_status s_ = (__VA_ARGS__);                                          \
        if (s_ != L1LS_OK) return s_;                                            \
    } while (0)

// ---- context ------------------------------------------------------------------------------
struct Inst;

struct Ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;          // bytes the context may hold
    size_t used = 0;            // bytes currently held
    std::mutex mem_mu;
    // staging buffers for host pointers passed to products / solvers, and scratch
    static constexpr int kStages = 4;
    void* stage[kStages] = {nullptr, nullptr, nullptr, nullptr};
    size_t stage_bytes[kStages] = {0, 0, 0, 0};
    std::vector<Inst*> insts;   // instances owned by the context
    std::mutex inst_mu;

    // stream_ordered: cudaMallocAsync / cudaFreeAsync on `st` (no device-wide synchronisation;
    // the serving workers allocate this way so that their work overlaps)
    l1ls_status alloc(void** p, size_t bytes, cudaStream_t st = nullptr, bool stream_ordered = false);
    void release(void* p, size_t bytes, cudaStream_t st = nullptr, bool stream_ordered = false);
    l1ls_status staging(int which, size_t bytes, void** out);
    // Pinned host slots for the solvers' per-step state read-backs.  A copy into pageable
    // memory is staged through a buffer the driver shares between host threads, which
    // serialised the serving loop's concurrent requests; pinned slots are allocated once with
    // the context.  pinned_get returns NULL when every slot is taken (callers then fall back
    // to pageable memory).
    static constexpr int kPinnedSlots = 512;
    static constexpr size_t kPinnedSlotBytes = 1024;
    char* pinned = nullptr;
    std::vector<int> pinned_free;
    std::mutex pinned_mu;
    void* pinned_get(size_t bytes);
    void pinned_put(void* p);
    // serving loop (created by the first l1ls_submit or l1ls_serve_config)
    void* server = nullptr;
    void (*server_stop)(void*) = nullptr;
    std::mutex server_mu;
};

// ---- instance -----------------------------------------------------------------------------
struct Inst {
    Ctx* ctx = nullptr;
    l1ls_gen_params p{};
    int64_t m = 0, n = 0, nnz = 0, s = 0;
    int64_t nsq = 0;            // size of the square Givens part (n for IGen, m for IGen2)
    bool igen2 = false;
    // matrix-free instances: no CSR; the products apply the factors (Algorithms MvPA / MvPAt)
    bool matrix_free = false;
    float* sigma32 = nullptr;   // Sigma in FP32 (padded to whole tiles)
    int32_t* mf_pperm = nullptr;   // per stored row pair, the two entries of P it rotates
    float mf_c = 0, mf_s = 0, mf_ct = 0, mf_st = 0;   // cos / sin of the right and left angles
    double mf_c64 = 0, mf_s64 = 0, mf_ct64 = 0, mf_st64 = 0;   // the same in FP64 (pdNCG's gradient sweep)
    int dtype = L1LS_F64;
    // CSR of P1^T A (rows relabelled), m rows
    int32_t* csr_ptr = nullptr;
    int32_t* csr_col = nullptr;
    void* csr_val = nullptr;
    // CSR of A^T P1 (CSC of the relabelled matrix), n rows
    int32_t* csc_ptr = nullptr;
    int32_t* csc_row = nullptr;
    void* csc_val = nullptr;
    // paired storage (left_stages == 1): one index per row pair, two values per entry
    bool paired = false;
    int32_t* prow_ptr = nullptr;   // m/2 + 1
    int32_t* prow_col = nullptr;   // nnz/2 (+pad)
    void* prow_val = nullptr;      // nnz values: (row 2p, row 2p+1) per entry
    int32_t* pcol_ptr = nullptr;   // n + 1
    int32_t* pcol_pair = nullptr;  // nnz/2 (+pad)
    void* pcol_val = nullptr;      // nnz values: (row 2p, row 2p+1) per entry
    double* bhat = nullptr;     // P1^T b in FP64
    float* bhat32 = nullptr;    // FP32 copy (products in FP32)
    double* xstar = nullptr;
    double* sigma = nullptr;
    double* colnorm2 = nullptr; // diag(A^T A) from the stored values
    int32_t* perm = nullptr;    // P: (P v)_i = v_{perm[i]}
    int32_t* perm_inv = nullptr;
    // storage order of the rows: row i of A is stored as row store_of_row[i]
    int32_t* store_of_row = nullptr;
    int32_t* row_of_store = nullptr;
    double f_star = 0, lipschitz = 1, lam_max = 0;
    int64_t csr_tile_max = 0, csc_tile_max = 0;   // most nonzeros in a 32-row tile
    int* dev_err = nullptr;                       // set by kernels whose bounded waits expired
    size_t bytes = 0;
    bool stream_ordered = false;    // allocations ordered on alloc_st (serving workers)
    cudaStream_t alloc_st = nullptr;
    // solver work spaces (allocated on first use, owned by the instance)
    void* fista_work = nullptr;
    void (*fista_work_free)(void*) = nullptr;
    void* pd_work = nullptr;
    void (*pd_work_free)(void*) = nullptr;
    struct Alloc { void* p; size_t bytes; };
    std::vector<Alloc> allocs;

    l1ls_status alloc(void** p, size_t bytes);
    template <class T> l1ls_status alloc_n(T** p, int64_t count) {
        return alloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
    }
    void free_all();
};

// entries to allocate for a vector read in whole 32-entry tiles
inline int64_t pad32(int64_t count) { return (count + 31) / 32 * 32 + 32; }

// value size of a stored dtype
inline size_t dtype_size(int dt) { return dt == L1LS_F64 ? 8 : dt == L1LS_F32 ? 4 : 2; }

// pointer classification: true when the pointer is device (or managed) memory
bool is_device_pointer(const void* p);

// ---- entry points implemented per file ------------------------------------------------
l1ls_status generate_instance(Ctx* ctx, const l1ls_gen_params* p, cudaStream_t st, Inst** out,
                              bool stream_ordered = false);
l1ls_status kappa_rho(const Inst* I, double rho, double* out);

// the serving worker's cancel flag (null elsewhere); solver loops poll it between launches
extern thread_local const std::atomic<int>* tl_cancel;
inline bool cancel_requested() { return tl_cancel && tl_cancel->load(std::memory_order_relaxed) != 0; }

// products on device buffers (relabelled row order), vec_dtype F64 or F32
l1ls_status spmv_plain(const Inst* I, bool transpose, const void* x, int vec_dtype, void* y,
                       bool unpermute_rows, cudaStream_t st);

// matrix-free products (csrc/mfree.cu), FP32 vectors: transpose = false: out (m) = A in (n);
// true: out (n) = A^T in (m); the m-vector's stored row h is entry map[h] (map NULL: h);
// z: n floats of scratch
l1ls_status mf_product(const Inst* I, bool transpose, const float* in, float* out, const int32_t* map, float* z,
                       cudaStream_t st);
// z = Sigma R^T x, the first launch of A x alone (FISTA fuses the second with its epilogues)
l1ls_status mf_apply_rt(const Inst* I, const float* x, float* z, cudaStream_t st);

l1ls_status fista_solve(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res,
                        cudaStream_t st);
l1ls_status pdncg_solve(Inst* I, const l1ls_solve_opts* o, const double* x0, double* x_out, l1ls_result* res,
                        cudaStream_t st);

}  // namespace l1ls
