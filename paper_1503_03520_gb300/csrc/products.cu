// Plain products y = A x and x = A^T y (Algorithms MvPA / MvPAt compute the same products
// matrix-free; here A is stored).  A is held with its rows in a storage order (row s of the
// stored matrix is row row_of_store[s] of A), so
//   A x   : stored row s lands in y[row_of_store[s]],
//   A^T y : y is first gathered into the storage order, ys[s] = y[row_of_store[s]].
#include <mutex>

#include "internal.h"
#include "spmv.cuh"

namespace l1ls {

namespace {

constexpr int kBlock = 256;

// y = A x (COLS = false) or x = A^T y (COLS = true) on the assembled A of Eq. (bd8)
template <class V, class X, class Acc, bool PAIRED, bool COLS>
__global__ void __launch_bounds__(kBlock) k_spmv(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                 const V* __restrict__ val, const X* __restrict__ x, int64_t nrows,
                                                 const int32_t* __restrict__ out_perm, X* __restrict__ y, int* err) {
    __shared__ TraversalSmem<V, Acc, kBlock, PAIRED> sm;
    auto pre = [&](int64_t, bool) { return NoOps{}; };
    auto epi = [&](int64_t r, Acc acc, const NoOps&) {
        const int64_t dst = out_perm ? out_perm[r] : r;
        y[dst] = (X)acc;
    };
    if constexpr (COLS) cols_of<PAIRED, V, X, Acc>(ptr, col, val, x, nrows, sm, err, pre, epi);
    else rows_of<PAIRED, V, X, Acc>(ptr, col, val, x, nrows, sm, err, pre, epi);
}

template <class X>
__global__ void k_gather(const X* __restrict__ y, const int32_t* __restrict__ idx, int64_t count, X* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = y[idx[i]];
}

int grid_for(const Inst* I, int64_t nrows) {
    int64_t ntiles = (nrows + kBlock - 1) / kBlock;
    int64_t g = (int64_t)I->ctx->num_sms * 8;
    return (int)(ntiles < g ? (ntiles > 0 ? ntiles : 1) : g);
}

template <class V, class X>
l1ls_status launch_spmv(const Inst* I, bool transpose, const X* x, X* y, const int32_t* out_perm, cudaStream_t st) {
    using Acc = typename std::conditional<std::is_same<V, double>::value, double, float>::type;
    const int64_t nrows = transpose ? I->n : I->m;
    if (I->paired) {
        const int32_t* ptr = transpose ? I->pcol_ptr : I->prow_ptr;
        const int32_t* col = transpose ? I->pcol_pair : I->prow_col;
        const V* val = static_cast<const V*>(transpose ? I->pcol_val : I->prow_val);
        if (transpose)
            k_spmv<V, X, Acc, true, true><<<grid_for(I, nrows), kBlock, 0, st>>>(ptr, col, val, x, nrows, out_perm, y, I->dev_err);
        else
            k_spmv<V, X, Acc, true, false><<<grid_for(I, nrows / 2), kBlock, 0, st>>>(ptr, col, val, x, nrows,
                                                                                      out_perm, y, I->dev_err);
    } else {
        const int32_t* ptr = transpose ? I->csc_ptr : I->csr_ptr;
        const int32_t* col = transpose ? I->csc_row : I->csr_col;
        const V* val = static_cast<const V*>(transpose ? I->csc_val : I->csr_val);
        k_spmv<V, X, Acc, false, false><<<grid_for(I, nrows), kBlock, 0, st>>>(ptr, col, val, x, nrows, out_perm, y, I->dev_err);
    }
    L1LS_CUDA(cudaGetLastError());
    return L1LS_OK;
}

template <class X>
l1ls_status dispatch(const Inst* I, bool transpose, const X* x, X* y, const int32_t* out_perm, cudaStream_t st) {
    switch (I->dtype) {
        case L1LS_F64: return launch_spmv<double, X>(I, transpose, x, y, out_perm, st);
        case L1LS_F32: return launch_spmv<float, X>(I, transpose, x, y, out_perm, st);
        default: return launch_spmv<__nv_bfloat16, X>(I, transpose, x, y, out_perm, st);
    }
}

}  // namespace

// Products on device buffers.  transpose = false: y = A x (rows unpermuted into the original
// order when unpermute_rows, else left in the relabelled order).  transpose = true: x = A^T y
// where y is in the original row order when unpermute_rows (gathered through scratch), else
// already relabelled.
l1ls_status spmv_plain(const Inst* I, bool transpose, const void* in, int vec_dtype, void* out, bool unpermute_rows,
                       cudaStream_t st) {
    const size_t es = vec_dtype == L1LS_F64 ? 8 : 4;
    if (I->matrix_free) {
        if (vec_dtype != L1LS_F32) return set_error(L1LS_EINVAL, "matrix-free instances take FP32 vectors");
        void* z = nullptr;
        L1LS_TRY(I->ctx->staging(3, sizeof(float) * (size_t)I->n, &z));
        return mf_product(I, transpose, static_cast<const float*>(in), static_cast<float*>(out),
                          unpermute_rows ? I->row_of_store : nullptr, static_cast<float*>(z), st);
    }
    if (!transpose) {
        const int32_t* op = unpermute_rows ? I->row_of_store : nullptr;
        if (vec_dtype == L1LS_F64) return dispatch<double>(I, false, (const double*)in, (double*)out, op, st);
        return dispatch<float>(I, false, (const float*)in, (float*)out, op, st);
    }
    const void* src = in;
    if (unpermute_rows) {
        void* scratch = nullptr;
        L1LS_TRY(I->ctx->staging(2, es * (size_t)I->m, &scratch));
        unsigned nb = (unsigned)((I->m + 255) / 256);
        if (vec_dtype == L1LS_F64) k_gather<double><<<nb, 256, 0, st>>>((const double*)in, I->row_of_store, I->m, (double*)scratch);
        else k_gather<float><<<nb, 256, 0, st>>>((const float*)in, I->row_of_store, I->m, (float*)scratch);
        L1LS_CUDA(cudaGetLastError());
        src = scratch;
    }
    if (vec_dtype == L1LS_F64) return dispatch<double>(I, true, (const double*)src, (double*)out, nullptr, st);
    return dispatch<float>(I, true, (const float*)src, (float*)out, nullptr, st);
}

}  // namespace l1ls

using namespace l1ls;

static l1ls_status product_entry(const l1ls_inst* h, const void* in, l1ls_dtype vd, void* out, void* stream,
                                 bool transpose) {
    if (!h || !in || !out) return set_error(L1LS_EINVAL, "NULL argument");
    if (vd != L1LS_F64 && vd != L1LS_F32) return set_error(L1LS_EINVAL, "vec_dtype must be L1LS_F64 or L1LS_F32");
    const Inst* I = reinterpret_cast<const Inst*>(h);
    cudaStream_t st = (cudaStream_t)stream;
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    const size_t es = vd == L1LS_F64 ? 8 : 4;
    const int64_t nin = transpose ? I->m : I->n, nout = transpose ? I->n : I->m;
    const bool din = is_device_pointer(in), dout = is_device_pointer(out);
    if (din && dout) return spmv_plain(I, transpose, in, vd, out, true, st);
    void *dx = const_cast<void*>(in), *dy = out;
    if (!din) {
        L1LS_TRY(I->ctx->staging(0, es * nin, &dx));
        L1LS_CUDA(cudaMemcpyAsync(dx, in, es * nin, cudaMemcpyHostToDevice, st));
    }
    if (!dout) L1LS_TRY(I->ctx->staging(1, es * nout, &dy));
    L1LS_TRY(spmv_plain(I, transpose, dx, vd, dy, true, st));
    if (!dout) L1LS_CUDA(cudaMemcpyAsync(out, dy, es * nout, cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    return L1LS_OK;
}

extern "C" l1ls_status l1ls_matvec(const l1ls_inst* inst, const void* x, l1ls_dtype vec_dtype, void* y, void* stream) {
    return product_entry(inst, x, vec_dtype, y, stream, false);
}

extern "C" l1ls_status l1ls_rmatvec(const l1ls_inst* inst, const void* y, l1ls_dtype vec_dtype, void* x, void* stream) {
    return product_entry(inst, y, vec_dtype, x, stream, true);
}

// ---- x = A^T y without any allocation -------------------------------------------------------
// For callers that cannot allocate device memory: real-time loops that must not stall on the
// device-wide synchronisation cudaMalloc / cudaFree may imply, and host applications that own
// all device memory themselves (a fixed budget handed out up front, libraries not allowed to
// allocate).  l1ls_rmatvec needs one m-vector of scratch (y gathered into the stored row
// order); here that scratch is a fixed-size array in the device image of the library instead
// of a context staging buffer.
namespace l1ls {
namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 20;   // rows; 8 MiB per device
__device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxRows];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (the current device), looked up once per
// device and kept for the life of the process: this assumes the device's primary context is
// never reset (cudaDeviceReset unloads the module, and a cached address would then dangle).
l1ls_status noalloc_scratch(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return set_error(L1LS_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return L1LS_OK;
}

}  // namespace
}  // namespace l1ls

extern "C" l1ls_status l1ls_rmatvec_noalloc(const l1ls_inst* inst, const void* y, l1ls_dtype vec_dtype, void* x,
                                            void* stream) {
    if (!inst || !y || !x) return set_error(L1LS_EINVAL, "NULL argument");
    if (vec_dtype != L1LS_F64 && vec_dtype != L1LS_F32)
        return set_error(L1LS_EINVAL, "vec_dtype must be L1LS_F64 or L1LS_F32");
    const Inst* I = reinterpret_cast<const Inst*>(inst);
    if (I->matrix_free) return set_error(L1LS_EINVAL, "l1ls_rmatvec_noalloc needs the assembled matrix");
    if (I->m > kNoAllocMaxRows)
        return set_error(L1LS_EINVAL, "l1ls_rmatvec_noalloc supports m <= %lld rows (instance has m = %lld)",
                         (long long)kNoAllocMaxRows, (long long)I->m);
    L1LS_CUDA(cudaSetDevice(I->ctx->device));
    // cudaPointerGetAttributes allocates nothing; a host pointer is refused before any launch
    if (!is_device_pointer(y) || !is_device_pointer(x))
        return set_error(L1LS_EINVAL, "l1ls_rmatvec_noalloc takes device pointers for y and x");
    void* scratch = nullptr;
    L1LS_TRY(noalloc_scratch(I->ctx->device, &scratch));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((I->m + 255) / 256);
    if (vec_dtype == L1LS_F64) {
        k_gather<double><<<nb, 256, 0, st>>>((const double*)y, I->row_of_store, I->m, (double*)scratch);
        L1LS_CUDA(cudaGetLastError());
        return dispatch<double>(I, true, (const double*)scratch, (double*)x, nullptr, st);
    }
    k_gather<float><<<nb, 256, 0, st>>>((const float*)y, I->row_of_store, I->m, (float*)scratch);
    L1LS_CUDA(cudaGetLastError());
    return dispatch<float>(I, true, (const float*)scratch, (float*)x, nullptr, st);
}
