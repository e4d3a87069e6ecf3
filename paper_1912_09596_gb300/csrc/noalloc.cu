// noalloc.cu -- ess_compact_mask_noalloc: the brick compaction (mask ->
// ascending ids of the non-empty bricks) for callers that cannot allocate
// device memory.
//
// Some callers run under a fixed device-memory budget that another allocator
// already owns (for example a host application or framework whose caching
// allocator has reserved the GPU's memory), or inside a per-frame callback
// where a cudaMalloc would stall the device.  They can pass in their input and
// output buffers but cannot let the library allocate.  This entry point
// therefore takes all buffers from the caller and keeps its only scratch (one
// partial count per 4096-flag tile) in a file-scope device array of fixed size.
//
// The array lives for as long as the library is loaded, on every GPU that
// loads it (16 KiB each).  All calls share it and it keeps the last call's
// contents; every entry a call reads is first written by that same call, so
// nothing has to be cleared, but two calls whose kernels overlap on the GPU
// (for example on two streams) race on it and must be serialised by the
// caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ess.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 16;
constexpr int NA_TILE = NA_THREADS * NA_ITEMS;  // flags per tile
constexpr int NA_MAX_TILES = 4096;              // => at most 16,777,216 flags
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) uint32_t g_tile_sums[NA_MAX_TILES];

std::mutex g_mtx;
uint32_t *g_tile_sums_addr[NA_MAX_DEVICES] = {};

// Device address of g_tile_sums on the current device (looked up once per
// device; in host code the symbol itself is only a host-side stand-in).
cudaError_t tile_sums_address(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mtx);
    if (!g_tile_sums_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tile_sums);
        if (e != cudaSuccess) return e;
        g_tile_sums_addr[dev] = (uint32_t *)p;
    }
    *out = g_tile_sums_addr[dev];
    return cudaSuccess;
}

template <int NT> __device__ __forceinline__ int na_block_excl_scan(int v, int &total)
{
    __shared__ int wsum[NT / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = lane < NT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) wsum[lane] = s;
    }
    __syncthreads();
    total = wsum[NT / 32 - 1];
    int r = (w > 0 ? wsum[w - 1] : 0) + incl - v;
    __syncthreads();
    return r;
}

// Flags are read one byte at a time with a bounds check, so any mask length
// and alignment is accepted.
__device__ __forceinline__ int na_count16(const uint8_t *mask, int64_t first, int64_t nb,
                                          uint32_t &bits)
{
    bits = 0;
    int c = 0;
#pragma unroll
    for (int j = 0; j < NA_ITEMS; ++j) {
        int64_t b = first + j;
        if (b < nb && mask[b]) {
            bits |= 1u << j;
            ++c;
        }
    }
    return c;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_count(const uint8_t *__restrict__ mask,
                                                         int64_t nb, uint32_t *tile_sums)
{
    uint32_t bits;
    int64_t first = (int64_t)blockIdx.x * NA_TILE + (int64_t)threadIdx.x * NA_ITEMS;
    int c = na_count16(mask, first, nb, bits);
    int total;
    na_block_excl_scan<NA_THREADS>(c, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = (uint32_t)total;
}

__global__ void __launch_bounds__(1024) k_na_scan(uint32_t *tile_sums, int ntiles, int *count)
{
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < ntiles ? (int)tile_sums[i] : 0;
        int total;
        int ex = na_block_excl_scan<1024>(v, total);
        if (i < ntiles) tile_sums[i] = (uint32_t)(carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_scatter(const uint8_t *__restrict__ mask,
                                                           int64_t nb,
                                                           const uint32_t *__restrict__ tile_sums,
                                                           uint32_t *__restrict__ ids)
{
    uint32_t bits;
    int64_t first = (int64_t)blockIdx.x * NA_TILE + (int64_t)threadIdx.x * NA_ITEMS;
    int c = na_count16(mask, first, nb, bits);
    int total;
    int off = na_block_excl_scan<NA_THREADS>(c, total) + (int)tile_sums[blockIdx.x];
    for (int j = 0; j < NA_ITEMS; ++j)
        if (bits & (1u << j)) ids[off++] = (uint32_t)(first + j);
}

}  // namespace

extern "C" ess_status ess_compact_mask_noalloc(const uint8_t *mask, int64_t n_bricks,
                                               uint32_t *ids, int *count, void *cuda_stream)
{
    if (n_bricks < 0 || n_bricks > (int64_t)NA_MAX_TILES * NA_TILE) return ESS_ERR_ARG;
    if (n_bricks > 0 && (!mask || !ids)) return ESS_ERR_ARG;
    if (!count) return ESS_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (n_bricks == 0) {
        return cudaMemsetAsync(count, 0, sizeof(int), stream) == cudaSuccess ? ESS_OK : ESS_ERR_CUDA;
    }
    uint32_t *sums = nullptr;
    if (tile_sums_address(&sums) != cudaSuccess) return ESS_ERR_CUDA;
    unsigned ntiles = (unsigned)((n_bricks + NA_TILE - 1) / NA_TILE);
    k_na_count<<<ntiles, NA_THREADS, 0, stream>>>(mask, n_bricks, sums);
    k_na_scan<<<1, 1024, 0, stream>>>(sums, (int)ntiles, count);
    k_na_scatter<<<ntiles, NA_THREADS, 0, stream>>>(mask, n_bricks, sums, ids);
    return cudaGetLastError() == cudaSuccess ? ESS_OK : ESS_ERR_CUDA;
}
