// Device primitives for the generator: stable LSD radix argsort of 64-bit keys and an
// exclusive scan of 32-bit counts.  Written for this library (no CUB / Thrust).
#include "common.cuh"
#include "internal.h"

namespace l1ls {

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

// per-tile sums of the counts
__global__ void k_scan_tile_sums(const int32_t* __restrict__ in, int64_t count, int64_t* __restrict__ sums) {
    __shared__ int64_t sm[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanBlock + threadIdx.x;
        if (i < count) v += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) t += sm[w];
        sums[blockIdx.x] = t;
    }
}

// exclusive scan of the tile sums in one block; total written to sums[ntiles]
__global__ void k_scan_top(int64_t* __restrict__ sums, int64_t ntiles) {
    __shared__ int64_t sm[kScanBlock];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += kScanBlock) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? sums[i] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kScanBlock; o <<= 1) {
            int64_t add = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
            __syncthreads();
            sm[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < ntiles) sums[i] = carry + sm[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += sm[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[ntiles] = carry;
}

// scan inside each tile and add the tile offset
__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t count, const int64_t* __restrict__ offs,
                             int32_t* __restrict__ out) {
    __shared__ int64_t sm[kScanBlock];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        loc[k] = run;
        run += (i < count) ? in[i] : 0;
    }
    sm[threadIdx.x] = run;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        int64_t add = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
        __syncthreads();
        sm[threadIdx.x] += add;
        __syncthreads();
    }
    const int64_t pre = offs[blockIdx.x] + sm[threadIdx.x] - run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < count) out[i] = (int32_t)(pre + loc[k]);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = (int32_t)offs[gridDim.x];
}

// ---- radix argsort ----------------------------------------------------------------------
constexpr int kRsBlock = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsBlock * kRsItems;
constexpr int kRsWarps = kRsBlock / 32;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t count, int shift, int32_t* __restrict__ counts,
                          int64_t ntiles) {
    __shared__ int32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        int64_t i = base + (int64_t)r * kRsBlock + threadIdx.x;
        if (i < count) atomicAdd(&hist[(keys[i] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter: items of a tile are ranked in their original order (round, warp, lane).
__global__ void k_rs_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t count,
                             int shift, const int32_t* __restrict__ offs, int64_t ntiles,
                             uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    __shared__ int32_t base_off[256];
    __shared__ int32_t wcnt[kRsWarps][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    base_off[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = tile0 + (int64_t)r * kRsBlock + threadIdx.x;
        const bool valid = i < count;
        uint64_t key = valid ? keys[i] : 0ull;
        uint32_t val = valid ? vals[i] : 0u;
        const unsigned d = valid ? (unsigned)((key >> shift) & 0xFF) : 256u + (unsigned)lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank_w = __popc(peers & lt_mask);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int32_t pos = base_off[d] + rank_w;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][d];
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        {
            int32_t tot = 0;
            for (int w = 0; w < kRsWarps; ++w) {
                tot += wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = 0;
            }
            base_off[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

__global__ void k_iota(uint32_t* __restrict__ v, int64_t count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) v[i] = (uint32_t)i;
}

}  // namespace

// Exclusive scan of `count` int32 values into out[0..count] (out[count] = total).
// Fails with EINVAL when the total does not fit in int32.
// the 64-bit sum of count int32 values (no 32-bit limit: the counts of a matrix that is never
// assembled)
l1ls_status sum_i32(const int32_t* in, int64_t count, int64_t* total, cudaStream_t st) {
    const int64_t ntiles = (count + kScanTile - 1) / kScanTile;
    int64_t* sums = nullptr;
    L1LS_CUDA(cudaMallocAsync((void**)&sums, sizeof(int64_t) * (ntiles + 1), st));
    if (ntiles > 0) {
        k_scan_tile_sums<<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, count, sums);
        L1LS_CUDA(cudaGetLastError());
    }
    k_scan_top<<<1, kScanBlock, 0, st>>>(sums, ntiles);
    L1LS_CUDA(cudaGetLastError());
    int64_t tot = 0;
    L1LS_CUDA(cudaMemcpyAsync(&tot, sums + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaFreeAsync(sums, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    *total = tot;
    return L1LS_OK;
}

l1ls_status exclusive_scan_i32(const int32_t* in, int64_t count, int32_t* out, int64_t* total, cudaStream_t st) {
    const int64_t ntiles = (count + kScanTile - 1) / kScanTile;
    int64_t* sums = nullptr;
    L1LS_CUDA(cudaMallocAsync((void**)&sums, sizeof(int64_t) * (ntiles + 1), st));
    if (ntiles > 0) {
        k_scan_tile_sums<<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, count, sums);
        L1LS_CUDA(cudaGetLastError());
    }
    k_scan_top<<<1, kScanBlock, 0, st>>>(sums, ntiles);
    L1LS_CUDA(cudaGetLastError());
    int64_t tot = 0;
    L1LS_CUDA(cudaMemcpyAsync(&tot, sums + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    L1LS_CUDA(cudaStreamSynchronize(st));
    if (tot > INT32_MAX) {
        cudaFreeAsync(sums, st);
        return set_error(L1LS_EINVAL, "scan total %lld exceeds int32 (nnz >= 2^31 is not supported)", (long long)tot);
    }
    if (ntiles > 0) {
        k_scan_apply<<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, count, sums, out);
        L1LS_CUDA(cudaGetLastError());
    } else {
        L1LS_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    }
    L1LS_CUDA(cudaFreeAsync(sums, st));
    *total = tot;
    return L1LS_OK;
}

// order[r] = index of the r-th smallest key (stable: equal keys keep index order).
l1ls_status radix_argsort_u64(const uint64_t* keys, int64_t count, uint32_t* order, cudaStream_t st) {
    if (count <= 0) return L1LS_OK;
    if (count > (int64_t)INT32_MAX) return set_error(L1LS_EINVAL, "sort of %lld keys not supported", (long long)count);
    const int64_t ntiles = (count + kRsTile - 1) / kRsTile;
    uint64_t *ka = nullptr, *kb = nullptr;
    uint32_t *va = nullptr, *vb = nullptr;
    int32_t *counts = nullptr, *offs = nullptr;
    L1LS_CUDA(cudaMallocAsync((void**)&ka, sizeof(uint64_t) * count, st));
    L1LS_CUDA(cudaMallocAsync((void**)&kb, sizeof(uint64_t) * count, st));
    L1LS_CUDA(cudaMallocAsync((void**)&va, sizeof(uint32_t) * count, st));
    L1LS_CUDA(cudaMallocAsync((void**)&vb, sizeof(uint32_t) * count, st));
    L1LS_CUDA(cudaMallocAsync((void**)&counts, sizeof(int32_t) * 256 * ntiles, st));
    L1LS_CUDA(cudaMallocAsync((void**)&offs, sizeof(int32_t) * (256 * ntiles + 1), st));
    L1LS_CUDA(cudaMemcpyAsync(ka, keys, sizeof(uint64_t) * count, cudaMemcpyDeviceToDevice, st));
    k_iota<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(va, count);
    L1LS_CUDA(cudaGetLastError());
    for (int shift = 0; shift < 64; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, kRsBlock, 0, st>>>(ka, count, shift, counts, ntiles);
        L1LS_CUDA(cudaGetLastError());
        int64_t tot = 0;
        L1LS_TRY(exclusive_scan_i32(counts, 256 * ntiles, offs, &tot, st));
        k_rs_scatter<<<(unsigned)ntiles, kRsBlock, 0, st>>>(ka, va, count, shift, offs, ntiles, kb, vb);
        L1LS_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    L1LS_CUDA(cudaMemcpyAsync(order, va, sizeof(uint32_t) * count, cudaMemcpyDeviceToDevice, st));
    cudaFreeAsync(ka, st);
    cudaFreeAsync(kb, st);
    cudaFreeAsync(va, st);
    cudaFreeAsync(vb, st);
    cudaFreeAsync(counts, st);
    cudaFreeAsync(offs, st);
    L1LS_CUDA(cudaGetLastError());
    return L1LS_OK;
}

}  // namespace l1ls
