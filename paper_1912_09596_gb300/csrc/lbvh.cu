// lbvh.cu -- LBVH over the non-empty bricks (Sec. 3.1): 30-bit Morton codes
// (computed in the compaction scatter), a onesweep LSD radix sort of
// (code, brick id) pairs, Karras' per-node hierarchy emission and a bottom-up
// pass that assembles the inner-node boxes and the traversal nodes.
//
// The non-empty count n lives in device memory; kernels read it there and
// grids are sized for the brick capacity, so a rebuild needs no host round
// trip.
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "ess_internal.h"

namespace ess {

// ------------------------------------------------------------ K5 onesweep
// LSD radix sort, 8-bit digits.  One kernel builds the digit histograms of
// all passes at once; one block scans them into global digit offsets; then
// one kernel per pass ranks a tile of RS_TILE items stably in shared memory,
// publishes the tile's per-digit counts and resolves its prefix by decoupled
// look-back over earlier tiles (tile ids come from an atomic counter, so every
// earlier tile has already started), and scatters.  Waits on earlier tiles are
// bounded: after RS_SPIN_LIMIT polls the kernel records DEV_ERR_TIMEOUT and
// carries on with what it has; scatter positions are bounds-checked, so a
// timed-out sort returns a wrong order (reported by ess_sync) but never
// writes outside the buffers.
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_RADIX = 256;
constexpr uint32_t RS_FLAG_AGG = 1u << 30, RS_FLAG_INC = 2u << 30, RS_MASK = (1u << 30) - 1;
constexpr long RS_SPIN_LIMIT = 1L << 22;

// The bounded wait of the look-back: polls *p until one of the bits of `mask`
// is set or `limit` polls have passed; on a timeout records DEV_ERR_TIMEOUT.
// Returns the last value read (none of the `mask` bits set after a timeout).
__device__ __forceinline__ uint32_t poll_flag(const volatile uint32_t *p, uint32_t mask, long limit,
                                              uint32_t *status)
{
    uint32_t v;
    long spins = 0;
    while (((v = *p) & mask) == 0u) {
        if (++spins > limit) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            break;
        }
    }
    return v;
}

size_t sort_tiles(int64_t cap) { return (size_t)((cap + RS_TILE - 1) / RS_TILE); }

size_t sort_scratch_words(int64_t cap)
{
    // histograms (4 x 256) + tile counters (4) + tile status (4 x tiles x 256)
    return 4 * RS_RADIX + 4 + 4 * sort_tiles(cap) * RS_RADIX;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *__restrict__ keys,
                                                        const int *__restrict__ count, int passes,
                                                        uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t h[4][RS_RADIX];
    for (int i = threadIdx.x; i < 4 * RS_RADIX; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    int n = *count;
    for (int i = blockIdx.x * RS_THREADS + threadIdx.x; i < n; i += gridDim.x * RS_THREADS) {
        uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_RADIX; i += RS_THREADS) {
        uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(ghist + i, v);
    }
}

// exclusive scan of each pass's 256 bins: 4 x 256 threads
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t wsum[32];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t v = ghist[t];
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    // 8 warps per pass
    int p0 = (w >> 3) << 3;
    uint32_t before = 0;
    for (int j = p0; j < w; ++j) before += wsum[j];
    ghist[t] = before + incl - v;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_pass(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const int *__restrict__ count, int shift,
    const uint32_t *__restrict__ offsets, uint32_t *tile_status, uint32_t *tile_counter,
    uint32_t *status)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_cnt[RS_RADIX];
    __shared__ uint32_t s_warp[RS_THREADS / 32][RS_RADIX];
    __shared__ uint32_t s_base[RS_RADIX];
    const int t = threadIdx.x, w = t >> 5;
    if (t == 0) s_tile = atomicAdd(tile_counter, 1u);
    s_cnt[t] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int n = *count;
    const int64_t base = (int64_t)tile * RS_TILE;
    if (base >= n) return;  // uniform per block

    uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + t;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0u;
        val[r] = ok ? vin[i] : 0u;
    }
    // stable ranking, one round of 256 consecutive items at a time
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        bool ok = base + r * RS_THREADS + t < n;
        uint32_t d = ok ? (key[r] >> shift) & 0xffu : RS_RADIX;  // invalid: own group
        for (int i = t; i < (RS_THREADS / 32) * RS_RADIX; i += RS_THREADS) (&s_warp[0][0])[i] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t below = peers & lanemask_lt();
        if (ok && below == 0) s_warp[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pre = 0;
            for (int j = 0; j < w; ++j) pre += s_warp[j][d];
            rank[r] = s_cnt[d] + pre + __popc(below);
        }
        __syncthreads();
        {
            uint32_t add = 0;
#pragma unroll
            for (int j = 0; j < RS_THREADS / 32; ++j) add += s_warp[j][t];
            s_cnt[t] += add;
        }
        __syncthreads();
    }
    // publish and look back (thread t owns digit t)
    {
        uint32_t cnt = s_cnt[t];
        volatile uint32_t *st = tile_status;
        uint32_t excl = 0;
        if (tile == 0) {
            st[t] = RS_FLAG_INC | cnt;
        } else {
            st[(size_t)tile * RS_RADIX + t] = RS_FLAG_AGG | cnt;
            int64_t j = (int64_t)tile - 1;
            while (j >= 0) {
                const uint32_t v = poll_flag(st + (size_t)j * RS_RADIX + t, ~RS_MASK, RS_SPIN_LIMIT,
                                             status);
                const uint32_t f = v & ~RS_MASK;
                if (f == 0u) break;  // timed out
                excl += v & RS_MASK;
                if (f == RS_FLAG_INC) break;
                --j;
            }
            st[(size_t)tile * RS_RADIX + t] = RS_FLAG_INC | (excl + cnt);
        }
        s_base[t] = offsets[t] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + t;
        if (i < n) {
            uint32_t d = (key[r] >> shift) & 0xffu;
            uint32_t pos = s_base[d] + rank[r];
            if (pos < (uint32_t)n) {
                kout[pos] = key[r];
                vout[pos] = val[r];
            }
        }
    }
}

// Sorts the pairs (keys, vals) of length *count (<= cap) by the low `bits`
// key bits.  The inputs are only read; passes ping-pong between pair A and
// pair B.  Returns 0 if the sorted pairs are in A, 1 if in B.
int launch_radix_sort(Ctx &c, const uint32_t *keys, const uint32_t *vals, uint32_t *keys_a,
                      uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, const int *count,
                      int64_t cap, int bits, uint32_t *scratch)
{
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    if (passes > 4) passes = 4;
    size_t tiles = sort_tiles(cap);
    uint32_t *ghist = scratch;
    uint32_t *counters = scratch + 4 * RS_RADIX;
    uint32_t *tstatus = counters + 4;
    ESS_CUDA(cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * sort_scratch_words(cap), c.stream));
    {
        Launch L(c, "sort_hist");
        unsigned blocks = (unsigned)(tiles < 1216 ? (tiles ? tiles : 1) : 1216);
        k_rs_hist<<<blocks, RS_THREADS, 0, c.stream>>>(keys, count, passes, ghist);
    }
    {
        Launch L(c, "sort_scan");
        k_rs_scan<<<1, 1024, 0, c.stream>>>(ghist);
    }
    const uint32_t *ki = keys, *vi = vals;
    for (int p = 0; p < passes; ++p) {
        uint32_t *ko = (p & 1) ? keys_b : keys_a, *vo = (p & 1) ? vals_b : vals_a;
        {
            Launch L(c, "sort_pass");
            k_rs_pass<<<(unsigned)(tiles ? tiles : 1), RS_THREADS, 0, c.stream>>>(
                ki, vi, ko, vo, count, 8 * p, ghist + p * RS_RADIX,
                tstatus + (size_t)p * tiles * RS_RADIX, counters + p, c.dev_status);
        }
        ki = ko;
        vi = vo;
    }
    return (passes & 1) ? 0 : 1;
}

// ----------------------------------------------------------- K6 Karras
// Internal node i (0 <= i < n-1) of the binary radix tree over sorted unique
// keys: direction from the longer common prefix with a neighbour, range end by
// exponential then binary search, split by binary search on the common prefix
// (Karras 2012).  Children: inner g as g, leaf g as -1-g.
__device__ __forceinline__ int rs_delta(const uint32_t *k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    return __clz(k[i] ^ k[j]);
}

__global__ void k_karras(const uint32_t *__restrict__ k, const int *__restrict__ count,
                         int32_t *__restrict__ left, int32_t *__restrict__ right,
                         int32_t *__restrict__ parent, int32_t *__restrict__ leaf_parent,
                         int32_t *__restrict__ range_end)
{
    int n = *count;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = rs_delta(k, n, i, i + 1) - rs_delta(k, n, i, i - 1) > 0 ? 1 : -1;
    int dmin = rs_delta(k, n, i, i - d);
    int lmax = 2;
    while (rs_delta(k, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
        if (rs_delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = rs_delta(k, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) / 2;
        if (rs_delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int g = i + s * d + (d < 0 ? d : 0);
    int lo = min(i, j), hi = max(i, j);
    int lc = (lo == g) ? -1 - g : g;
    int rc = (hi == g + 1) ? -1 - (g + 1) : g + 1;
    left[i] = lc;
    right[i] = rc;
    range_end[i] = j;
    if (lc >= 0) parent[lc] = i; else leaf_parent[g] = i;
    if (rc >= 0) parent[rc] = i; else leaf_parent[g + 1] = i;
    if (i == 0) parent[0] = -1;
}

// ------------------------------------------------------- K7 node boxes
// An inner node covers a contiguous range of the sorted leaves, so its box is
// the union of the leaf boxes in that range (the same values a bottom-up
// union gives).  The leaves are cut into chunks of 32, 1024 and 32768; a
// first pass stores every chunk's box, and each inner node then unions its
// two children's ranges from at most 31 + 31 leaves, 31 + 31 chunks of 32,
// 31 + 31 chunks of 1024 and the chunks of 32768 between them, one warp per
// node.  No step waits for
// another node, unlike a bottom-up pass whose threads climb one level per
// dependent atomic.
//
// Solid subtrees: an inner node whose leaf count equals the number of bricks
// in its box covers that box with non-empty bricks and nothing else, so the
// ray's interval through the box is exactly the union of the leaves'
// intervals.  Its parent's traversal node refers to it as a leaf (a negative
// reference), and the traversal yields the box's interval without
// descending.  The topology arrays (left, right, boxes) are unchanged.
__device__ __forceinline__ void brick_box(uint32_t b, int gx, int gy, int32_t box[6])
{
    int x = (int)(b % (uint32_t)gx), y = (int)((b / (uint32_t)gx) % (uint32_t)gy);
    int z = (int)(b / ((uint32_t)gx * (uint32_t)gy));
    box[0] = x; box[1] = y; box[2] = z;
    box[3] = x + 1; box[4] = y + 1; box[5] = z + 1;
}

// root record: ref, then the box in voxel units as float bits
// Leaf reference standing for a solid subtree: the brick at its low corner
// (any brick id marks a leaf for the traversal, which uses the box alone).
__device__ __forceinline__ int32_t solid_ref(const int32_t box[6], int gx, int gy)
{
    return -1 - (int32_t)(((int64_t)box[2] * gy + box[1]) * gx + box[0]);
}

__device__ __forceinline__ bool solid(int32_t cnt, const int32_t box[6])
{
    return (int64_t)cnt == (int64_t)(box[3] - box[0]) * (box[4] - box[1]) * (box[5] - box[2]);
}

__device__ __forceinline__ void write_root(int32_t *root, int32_t ref, const int32_t box[6], int B)
{
    root[0] = ref;
#pragma unroll
    for (int a = 0; a < 6; ++a) root[1 + a] = __float_as_int((float)(box[a] * B));
}

constexpr int32_t LB_BIAS = 65536;  // brick coordinates are below 2^16

size_t lbvh_chunk_boxes(size_t cap)
{
    return cap / 32 + cap / 1024 + cap / 32768 + 3;
}

__device__ __forceinline__ void box_empty(int32_t b[6])
{
    b[0] = b[1] = b[2] = INT_MAX;
    b[3] = b[4] = b[5] = INT_MIN;
}

__device__ __forceinline__ void box_add(int32_t acc[6], const int32_t b[6])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = min(acc[a], b[a]);
        acc[3 + a] = max(acc[3 + a], b[3 + a]);
    }
}

// Chunk boxes: one block of 1024 threads per chunk of 1024 sorted leaves.
// Chunk-of-32 boxes from warp reductions, chunk-of-1024 boxes from the
// block's warps, chunk-of-32768 boxes by integer atomics on (bias - lo, hi),
// zeroed before the launch.  A single leaf makes the root itself.
__global__ void __launch_bounds__(1024) k_lbvh_chunks(const uint32_t *__restrict__ sorted_ids,
                                                      const int *__restrict__ count,
                                                      int32_t *chunk_box, int32_t *root, int gx,
                                                      int gy, int B, int64_t cap)
{
    const int n = *count;
    const int j = blockIdx.x * 1024 + threadIdx.x;
    if ((int64_t)blockIdx.x * 1024 >= n) return;  // uniform per block
    int32_t *c32 = chunk_box, *c1k = c32 + 6 * (cap / 32 + 1), *c32k = c1k + 6 * (cap / 1024 + 1);
    int32_t b[6];
    if (j < n) brick_box(sorted_ids[j], gx, gy, b);
    else box_empty(b);
    if (n == 1 && j == 0) write_root(root, -1 - (int32_t)sorted_ids[0], b, B);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b[a] = __reduce_min_sync(0xffffffffu, b[a]);
        b[3 + a] = __reduce_max_sync(0xffffffffu, b[3 + a]);
    }
    __shared__ int32_t wb[32][6];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            if (j < n) c32[6 * (j >> 5) + a] = b[a];  // chunks that hold a leaf only
            wb[w][a] = b[a];
        }
    }
    __syncthreads();
    if (w == 0) {
        int32_t t[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) t[a] = wb[lane][a];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t[a] = __reduce_min_sync(0xffffffffu, t[a]);
            t[3 + a] = __reduce_max_sync(0xffffffffu, t[3 + a]);
        }
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < 6; ++a) c1k[6 * blockIdx.x + a] = t[a];
            int32_t *q = c32k + 6 * (blockIdx.x >> 5);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                atomicMax(q + a, LB_BIAS - t[a]);
                atomicMax(q + 3 + a, t[3 + a]);
            }
        }
    }
}

// Union of the boxes of sorted leaves [L, R) (L < R) from the chunk tables,
// taken by a whole warp: [L, R) splits into at most 31 leaves, 31 chunks of 32
// and 31 chunks of 1024 on each side and the chunks of 32768 between, and
// lane l takes item l of every part (the chunks of 32768 by a stride of 32),
// so every load of a node is issued at once.  All lanes receive the box.
__device__ __forceinline__ void warp_range_box(int L, int R, const uint32_t *__restrict__ sorted_ids,
                                               const int32_t *c32, const int32_t *c1k,
                                               const int32_t *c32k, int gx, int gy, int lane,
                                               int32_t acc[6])
{
    box_empty(acc);
    int32_t b[6];
    const int a1 = min((L + 31) & ~31, R), b1 = max(R & ~31, a1);
    if (L + lane < a1) {
        brick_box(sorted_ids[L + lane], gx, gy, b);
        box_add(acc, b);
    }
    if (b1 + lane < R) {
        brick_box(sorted_ids[b1 + lane], gx, gy, b);
        box_add(acc, b);
    }
    if (a1 < b1) {
        const int a2 = min((a1 + 1023) & ~1023, b1), b2 = max(b1 & ~1023, a2);
        if (a1 + 32 * lane < a2) box_add(acc, c32 + 6 * ((a1 >> 5) + lane));
        if (b2 + 32 * lane < b1) box_add(acc, c32 + 6 * ((b2 >> 5) + lane));
        if (a2 < b2) {
            const int a3 = min((a2 + 32767) & ~32767, b2), b3 = max(b2 & ~32767, a3);
            if (a2 + 1024 * lane < a3) box_add(acc, c1k + 6 * ((a2 >> 10) + lane));
            if (b3 + 1024 * lane < b2) box_add(acc, c1k + 6 * ((b3 >> 10) + lane));
            for (int x = a3 + 32768 * lane; x < b3; x += 32 * 32768) {
                const int32_t *q = c32k + 6 * (x >> 15);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc[a] = min(acc[a], LB_BIAS - q[a]);
                    acc[3 + a] = max(acc[3 + a], q[3 + a]);
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = __reduce_min_sync(0xffffffffu, acc[a]);
        acc[3 + a] = __reduce_max_sync(0xffffffffu, acc[3 + a]);
    }
}

// The boxes and traversal node of inner node i (a whole warp; lane 0 writes).
__device__ __forceinline__ void lbvh_node_box(int i, int lane, const uint32_t *__restrict__ sorted_ids,
                                              const int32_t *__restrict__ left,
                                              const int32_t *__restrict__ right,
                                              const int32_t *__restrict__ range_end,
                                              const int32_t *c32, const int32_t *c1k,
                                              const int32_t *c32k, int32_t *inner_box,
                                              BoxNode *nodes, int32_t *root, int gx, int gy, int B)
{
    const int j = range_end[i], lo = min(i, j), hi = max(i, j);
    const int lc = left[i], rc = right[i];
    const int g = lc >= 0 ? lc : -1 - lc;  // left child: leaves [lo, g], right: [g + 1, hi]
    int32_t lb[6], rb[6], box[6];
    warp_range_box(lo, g + 1, sorted_ids, c32, c1k, c32k, gx, gy, lane, lb);
    warp_range_box(g + 1, hi + 1, sorted_ids, c32, c1k, c32k, gx, gy, lane, rb);
    if (lane != 0) return;
    const int32_t lcnt = g - lo + 1, rcnt = hi - g;
    BoxNode nd;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        box[a] = min(lb[a], rb[a]);
        box[3 + a] = max(lb[3 + a], rb[3 + a]);
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        inner_box[6 * i + a] = box[a];
        nd.lbox[a] = (float)(lb[a] * B);
        nd.rbox[a] = (float)(rb[a] * B);
    }
    nd.left = lc < 0 ? -1 - (int32_t)sorted_ids[-1 - lc]
                     : (solid(lcnt, lb) ? solid_ref(lb, gx, gy) : lc);
    nd.right = rc < 0 ? -1 - (int32_t)sorted_ids[-1 - rc]
                      : (solid(rcnt, rb) ? solid_ref(rb, gx, gy) : rc);
    nd.pad0 = nd.pad1 = 0;
    nodes[i] = nd;
    if (i == 0) write_root(root, solid(lcnt + rcnt, box) ? solid_ref(box, gx, gy) : 0, box, B);
}

// One warp per inner node: its children's boxes from their leaf ranges, then
// the traversal node (child references, solid subtrees) and the root.
__global__ void k_lbvh_node_boxes(const uint32_t *__restrict__ sorted_ids,
                                  const int *__restrict__ count, const int32_t *__restrict__ left,
                                  const int32_t *__restrict__ right,
                                  const int32_t *__restrict__ range_end,
                                  const int32_t *__restrict__ chunk_box, int32_t *inner_box,
                                  BoxNode *nodes, int32_t *root, int gx, int gy, int B,
                                  int64_t cap)
{
    const int n = *count;
    const int lane = threadIdx.x & 31;
    const int32_t *c32 = chunk_box, *c1k = c32 + 6 * (cap / 32 + 1),
                  *c32k = c1k + 6 * (cap / 1024 + 1);
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < n - 1; i += warps)
        lbvh_node_box(i, lane, sorted_ids, left, right, range_end, c32, c1k, c32k, inner_box,
                      nodes, root, gx, gy, B);
}

// Height of the tree (levels including root and leaves): each leaf counts its
// ancestors.  Run on demand (structure info), not in the rebuild.
__global__ void k_lbvh_height(const int *__restrict__ count, const int32_t *__restrict__ parent,
                              const int32_t *__restrict__ leaf_parent, int *height)
{
    int n = *count;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int h = 1;
    if (n >= 2) {
        int p = leaf_parent[j];
        while (p >= 0 && h <= 64) {
            ++h;
            p = parent[p];
        }
    }
    atomicMax(height, h);
}

// Diagnostics: one warp waits on `flag` with the look-back's bounded wait.
__global__ void k_selftest_wait(const uint32_t *flag, long limit, uint32_t *status)
{
    if (threadIdx.x == 0) poll_flag(flag, 1u, limit, status);
}

void launch_selftest_wait(Ctx &c, uint32_t *flag, bool set, long limit)
{
    ESS_CUDA(cudaMemsetAsync(flag, set ? 0xff : 0, sizeof(uint32_t), c.stream));
    Launch L(c, "selftest_wait");
    k_selftest_wait<<<1, 32, 0, c.stream>>>(flag, limit, c.dev_status);
}

void launch_lbvh(Ctx &c, Structure &s)
{
    int64_t cap = s.nb;
    int maxbits = 0;
    for (int g : {s.gx, s.gy, s.gz}) {
        int b = 0;
        while ((1 << b) < g) ++b;
        maxbits = b > maxbits ? b : maxbits;
    }
    int which = launch_radix_sort(c, s.keys, s.ids, s.keys_sorted, s.ids_sorted, s.keys_alt,
                                  s.ids_alt, s.count, cap, 3 * maxbits, s.sort_scratch);
    if (which == 1) {
        // keep the invariant that keys_sorted / ids_sorted hold the result
        std::swap(s.keys_sorted, s.keys_alt);
        std::swap(s.ids_sorted, s.ids_alt);
    }
    unsigned blocks = (unsigned)((cap + 255) / 256);
    {
        Launch L(c, "lbvh_karras");
        k_karras<<<blocks, 256, 0, c.stream>>>(s.keys_sorted, s.count, s.left, s.right, s.parent,
                                               s.leaf_parent, s.range_end);
    }
    {
        Launch L(c, "lbvh_bounds");
        // the chunk-of-32768 boxes are atomic maxima over zero
        const size_t c32k = (size_t)cap / 32 + 1 + (size_t)cap / 1024 + 1;
        ESS_CUDA(cudaMemsetAsync(s.chunk_box + 6 * c32k, 0,
                                 sizeof(int32_t) * 6 * ((size_t)cap / 32768 + 1), c.stream));
        k_lbvh_chunks<<<(unsigned)((cap + 1023) / 1024), 1024, 0, c.stream>>>(
            s.ids_sorted, s.count, s.chunk_box, s.root, s.gx, s.gy, s.p.brick, cap);
        int sms = 0;
        ESS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
        const unsigned nb_warps =
            (unsigned)std::min<int64_t>((32 * (int64_t)cap + 255) / 256, 16 * (int64_t)sms);
        k_lbvh_node_boxes<<<nb_warps, 256, 0, c.stream>>>(
            s.ids_sorted, s.count, s.left, s.right,
                                                        s.range_end, s.chunk_box, s.inner_box,
                                                        s.nodes, s.root, s.gx, s.gy, s.p.brick,
                                                        cap);
    }
}

int lbvh_height(Ctx &c, Structure &s)
{
    int *d = (int *)c.alloc(sizeof(int));
    ESS_CUDA(cudaMemsetAsync(d, 0, sizeof(int), c.stream));
    {
        Launch L(c, "lbvh_height");
        k_lbvh_height<<<(unsigned)((s.nb + 255) / 256), 256, 0, c.stream>>>(s.count, s.parent,
                                                                            s.leaf_parent, d);
    }
    int h = 0;
    ESS_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    ESS_CUDA(cudaStreamSynchronize(c.stream));
    c.free(d);
    return h;
}

}  // namespace ess
