// kd.cu -- k-d tree over the non-empty bricks (Sec. 3.2; parameters of
// Sec. 4.3), built level by level on the device.
//
// Definition (the same as the oracle's): boxes are brick-coordinate boxes
// [lo, hi); V(box) counts the voxels inside (partial bricks clamped).  The root
// is the tight box of all non-empty bricks.  A node is split by the candidate
// plane of least V(L) + V(R), L and R being the tight boxes of its bricks
// below and above the plane; candidates on an axis of brick extent e >= 2 are
// all interior brick boundaries (nbins = 0) or lo + floor(j e / nbins),
// j = 1..nbins-1, distinct and interior (binning on the brick raster, Sec.
// 3.2.2).  Ties go to the lower axis, then the lower plane.  The split is
// taken iff halting allows it (shallow: V > 10 % of the root; deep: V > 8^3)
// and its cost is below V(node); otherwise, when halting allows splitting and
// V > mls^3, the node is split in the middle of its longest axis (Sec. 4.3,
// maximum leaf size).  Children are numbered breadth first, left first.
//
// GPU scheme: the planes of a node cut each axis into "slabs"; per level one
// kernel accumulates the tight box of the bricks of every slab with integer
// min/max atomics (order independent, hence deterministic), one kernel per
// node turns slab boxes into the prefix/suffix unions that are the candidate
// L and R boxes and picks the split, a scan numbers the children, and one
// kernel emits them.  With an even nbins the middle plane lo + floor(e/2) is
// candidate j = nbins/2, so a forced middle split also falls on a slab border.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include <algorithm>

#include "ess_internal.h"

namespace ess {

struct KdParams {
    int B, nx, ny, nz, gx, gy;
    int nbins;    // 0 = every brick boundary
    int halting;  // 0 shallow, 1 deep
    unsigned long long mls3;  // 0 = no maximum leaf size
    int S;        // slab slots per axis
};

struct KdDecision {
    int32_t split;  // 1 if the node splits
    int32_t axis, plane;
    int32_t L[6], R[6];
};

__device__ __forceinline__ unsigned long long kd_volume(const int32_t *box, const KdParams &P)
{
    const int n[3] = {P.nx, P.ny, P.nz};
    unsigned long long v = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int x1 = min(box[3 + a] * P.B, n[a]);
        v *= (unsigned long long)(x1 - box[a] * P.B);
    }
    return v;
}

// Slab of brick coordinate c on an axis [lo, hi): the number of distinct
// interior candidate planes p <= c.
__device__ __forceinline__ int kd_slab_of(int c, int lo, int hi, int nbins)
{
    if (nbins == 0) return c - lo;
    int e = hi - lo, s = 0, prev = -1;
    for (int j = 1; j < nbins; ++j) {
        int p = lo + (j * e) / nbins;
        if (p > lo && p < hi && p != prev) {
            if (c >= p) ++s;
            prev = p;
        }
    }
    return s;
}

// Number of slabs of an axis and, for slab border j (1..slabs-1), its plane.
__device__ __forceinline__ int kd_slabs(int lo, int hi, int nbins)
{
    int e = hi - lo;
    if (e < 2) return 1;
    return kd_slab_of(hi - 1, lo, hi, nbins) + 1;
}

__device__ __forceinline__ int kd_plane(int j, int lo, int hi, int nbins)
{
    if (nbins == 0) return lo + j;
    int e = hi - lo, s = 0, prev = -1;
    for (int k = 1; k < nbins; ++k) {
        int p = lo + (k * e) / nbins;
        if (p > lo && p < hi && p != prev) {
            if (++s == j) return p;
            prev = p;
        }
    }
    return hi;
}

__device__ __forceinline__ void brick_coords(uint32_t b, int gx, int gy, int c[3])
{
    c[0] = (int)(b % (uint32_t)gx);
    c[1] = (int)((b / (uint32_t)gx) % (uint32_t)gy);
    c[2] = (int)(b / ((uint32_t)gx * (uint32_t)gy));
}

__device__ __forceinline__ void slab_reset(int32_t *slot)
{
    slot[0] = slot[1] = slot[2] = INT_MAX;
    slot[3] = slot[4] = slot[5] = INT_MIN;
}

// -------------------------------------------------------------- root box
__global__ void k_kd_root_reduce(const uint32_t *__restrict__ ids, const int *__restrict__ count,
                                 int gx, int gy, int32_t *root_box)
{
    int n = *count;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int v[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    if (i < n) {
        int c[3];
        brick_coords(ids[i], gx, gy, c);
        for (int a = 0; a < 3; ++a) {
            v[a] = c[a];
            v[3 + a] = c[a] + 1;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = __reduce_min_sync(0xffffffffu, v[a]);
        v[3 + a] = __reduce_max_sync(0xffffffffu, v[3 + a]);
    }
    if ((threadIdx.x & 31) == 0 && v[0] != INT_MAX) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(root_box + a, v[a]);
            atomicMax(root_box + 3 + a, v[3 + a]);
        }
    }
}

// node 0 record and the slabs of level 0
__global__ void k_kd_init(const int32_t *__restrict__ root_box, int32_t *nodes9, int32_t *slabs,
                          int S)
{
    int t = threadIdx.x;
    if (t < 6) nodes9[t] = root_box[t];
    if (t == 0) {
        nodes9[6] = -1;
        nodes9[7] = 0;
        nodes9[8] = -1;
    }
    for (int s = t; s < 3 * S; s += blockDim.x) slab_reset(slabs + 6 * s);
}

// ------------------------------------------------------------ per level
// Moves each brick of a node split on the previous level into its child,
// then adds the brick to the slab boxes of its node if that node is on the
// current level.
__global__ void k_kd_accumulate(const uint32_t *__restrict__ ids, const int *__restrict__ count,
                                int *__restrict__ brick_node, const int32_t *__restrict__ nodes9,
                                int prev_begin, int lvl_begin, int lvl_size, int32_t *slabs,
                                KdParams P)
{
    int n = *count;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    brick_coords(ids[i], P.gx, P.gy, c);
    int node = lvl_begin == 0 ? 0 : brick_node[i];
    if (node >= prev_begin && node < lvl_begin) {
        const int32_t *rec = nodes9 + 9 * (size_t)node;
        int fc = rec[8];
        if (fc >= 0) {
            node = fc + (c[rec[6]] >= rec[7] ? 1 : 0);
            brick_node[i] = node;
        }
    } else if (lvl_begin == 0) {
        brick_node[i] = 0;
    }
    if (node < lvl_begin || node >= lvl_begin + lvl_size) return;
    const int32_t *box = nodes9 + 9 * (size_t)node;
    int local = node - lvl_begin;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (box[3 + a] - box[a] < 2) continue;
        int s = kd_slab_of(c[a], box[a], box[3 + a], P.nbins);
        int32_t *slot = slabs + 6 * (((size_t)local * 3 + a) * P.S + s);
        atomicMin(slot + 0, c[0]);
        atomicMin(slot + 1, c[1]);
        atomicMin(slot + 2, c[2]);
        atomicMax(slot + 3, c[0] + 1);
        atomicMax(slot + 4, c[1] + 1);
        atomicMax(slot + 5, c[2] + 1);
    }
}

__device__ __forceinline__ void box_union(int32_t *acc, const int32_t *s)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = min(acc[a], s[a]);
        acc[3 + a] = max(acc[3 + a], s[3 + a]);
    }
}

// One thread per node of the level: cost of every candidate from prefix and
// suffix unions of the slab boxes, then the split rule.  `vr` is scratch for
// suffix volumes.  Writes the decision and the block's split count.
__global__ void __launch_bounds__(256) k_kd_decide(const int32_t *__restrict__ nodes9,
                                                   int lvl_begin, int lvl_size,
                                                   const int32_t *__restrict__ slabs,
                                                   unsigned long long *vr, KdDecision *dec,
                                                   uint32_t *block_sums, KdParams P)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    int split = 0;
    if (l < lvl_size) {
        const int32_t *X = nodes9 + 9 * (size_t)(lvl_begin + l);
        unsigned long long V = kd_volume(X, P), Vroot = kd_volume(nodes9, P);
        bool allowed = P.halting == 0 ? (10ull * V > Vroot) : (V > 512ull);
        unsigned long long best = ~0ull;
        int bax = -1, bj = 0, bpl = 0;
        if (allowed) {
            for (int a = 0; a < 3; ++a) {
                int lo = X[a], hi = X[3 + a];
                if (hi - lo < 2) continue;
                int ns = kd_slabs(lo, hi, P.nbins);
                const int32_t *sl = slabs + 6 * ((size_t)l * 3 + a) * P.S;
                unsigned long long *v = vr + ((size_t)l * 3 + a) * P.S;
                int32_t acc[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
                for (int j = ns - 1; j >= 1; --j) {
                    box_union(acc, sl + 6 * j);
                    v[j] = acc[0] == INT_MAX ? ~0ull : kd_volume(acc, P);
                }
                int32_t pre[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
                for (int j = 1; j < ns; ++j) {
                    box_union(pre, sl + 6 * (j - 1));
                    // both sides are non-empty for a tight node box; the test
                    // only guards the definition
                    if (pre[0] == INT_MAX || v[j] == ~0ull) continue;
                    unsigned long long cost = kd_volume(pre, P) + v[j];
                    if (cost < best) {
                        best = cost;
                        bax = a;
                        bj = j;
                        bpl = kd_plane(j, lo, hi, P.nbins);
                    }
                }
            }
            if (!(bax >= 0 && best < V)) {
                bax = -1;
                if (P.mls3 > 0 && V > P.mls3) {
                    int bestext = -1;
                    const int n[3] = {P.nx, P.ny, P.nz};
                    for (int a = 0; a < 3; ++a) {
                        int e = X[3 + a] - X[a];
                        if (e < 2) continue;
                        int ext = min(X[3 + a] * P.B, n[a]) - X[a] * P.B;
                        if (ext > bestext) {
                            bestext = ext;
                            bax = a;
                            bpl = X[a] + e / 2;
                        }
                    }
                    if (bax >= 0) bj = kd_slab_of(bpl, X[bax], X[3 + bax], P.nbins);
                }
            }
        }
        KdDecision d;
        d.split = 0;
        d.axis = -1;
        d.plane = 0;
        if (bax >= 0) {
            int lo = X[bax], hi = X[3 + bax];
            int ns = kd_slabs(lo, hi, P.nbins);
            const int32_t *sl = slabs + 6 * ((size_t)l * 3 + bax) * P.S;
            int32_t L[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
            int32_t R[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
            for (int j = 0; j < ns; ++j) box_union(j < bj ? L : R, sl + 6 * j);
            if (L[0] != INT_MAX && R[0] != INT_MAX) {
                d.split = 1;
                d.axis = bax;
                d.plane = bpl;
                for (int k = 0; k < 6; ++k) {
                    d.L[k] = L[k];
                    d.R[k] = R[k];
                }
                split = 1;
            }
        }
        dec[l] = d;
    }
    int total = __syncthreads_count(split);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = (uint32_t)total;
}

// exclusive scan of the block split counts; total splits -> *splits
__global__ void __launch_bounds__(1024) k_kd_scan(uint32_t *block_sums, int nblk, int *splits)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        int i = base + t;
        uint32_t v = i < nblk ? block_sums[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            uint32_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        uint32_t ex = carry + (w > 0 ? wsum[w - 1] : 0u) + incl - v;
        if (i < nblk) block_sums[i] = ex;
        __syncthreads();
        if (t == 0) carry += wsum[31];
        __syncthreads();
    }
    if (t == 0) *splits = (int)carry;
}

// Writes split decisions into the node records, creates the children (BFS
// numbering: after all nodes of this level, in node order, left first) and
// resets their slabs for the next level.
__global__ void __launch_bounds__(256) k_kd_emit(int lvl_begin, int lvl_size,
                                                 const KdDecision *__restrict__ dec,
                                                 const uint32_t *__restrict__ block_off,
                                                 int32_t *nodes9, int32_t *next_slabs, int S,
                                                 int capacity, uint32_t *status)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    int split = l < lvl_size ? dec[l].split : 0;
    // block-local exclusive rank of the split flag
    __shared__ uint32_t wcount[8];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ball = __ballot_sync(0xffffffffu, split);
    if (lane == 0) wcount[w] = __popc(ball);
    __syncthreads();
    uint32_t before = 0;
    for (int j = 0; j < w; ++j) before += wcount[j];
    if (!split) return;
    uint32_t rank = block_off[blockIdx.x] + before + __popc(ball & ((1u << lane) - 1u));
    int lvl_end = lvl_begin + lvl_size;
    int fc = lvl_end + 2 * (int)rank;
    if (fc + 1 >= capacity) {
        atomicOr(status, DEV_ERR_OVERFLOW);
        return;
    }
    const KdDecision &d = dec[l];
    int32_t *rec = nodes9 + 9 * (size_t)(lvl_begin + l);
    rec[6] = d.axis;
    rec[7] = d.plane;
    rec[8] = fc;
    int32_t *cl = nodes9 + 9 * (size_t)fc;
    int32_t *cr = cl + 9;
    for (int k = 0; k < 6; ++k) {
        cl[k] = d.L[k];
        cr[k] = d.R[k];
    }
    cl[6] = cr[6] = -1;
    cl[7] = cr[7] = 0;
    cl[8] = cr[8] = -1;
    for (int s = 0; s < 3 * S; ++s) {
        slab_reset(next_slabs + 6 * ((size_t)(2 * rank) * 3 * S + s));
        slab_reset(next_slabs + 6 * ((size_t)(2 * rank + 1) * 3 * S + s));
    }
}

// Traversal layout: one BoxNode per node id (leaf entries unused), children
// referenced as node ids, leaves as -1 - id; the root record.
__global__ void k_kd_pack(const int32_t *__restrict__ nodes9, const int *__restrict__ m_dev,
                          BoxNode *nodes, int32_t *root)
{
    int m = *m_dev;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t *rec = nodes9 + 9 * (size_t)i;
    if (i == 0) {
        root[0] = rec[8] >= 0 ? 0 : -1;
        for (int a = 0; a < 6; ++a) root[1 + a] = rec[a];
    }
    int fc = rec[8];
    if (fc < 0) return;
    const int32_t *L = nodes9 + 9 * (size_t)fc, *R = L + 9;
    BoxNode nd;
    for (int a = 0; a < 6; ++a) {
        nd.lbox[a] = (uint16_t)L[a];
        nd.rbox[a] = (uint16_t)R[a];
    }
    nd.left = L[8] >= 0 ? fc : -1 - fc;
    nd.right = R[8] >= 0 ? fc + 1 : -1 - (fc + 1);
    nodes[i] = nd;
}

// ------------------------------------------------------------------ host
// Per-level buffers: the current level's slabs were reset by the previous
// level's emit and already fit; the next level (at most twice as many nodes)
// may need a larger buffer, whose old contents are not needed.
void kd_reserve(Ctx &c, Structure &s, int lvl_size, int S, int cur)
{
    size_t slab_words = (size_t)3 * S * 6;
    auto grow = [&](void *&p, size_t &cap, size_t need, size_t elem) {
        if (cap >= need) return;
        c.free(p);
        size_t n = std::max(need, cap * 2);
        p = c.alloc(n * elem);
        cap = n;
    };
    if (s.kd_slab_cap[cur] < (size_t)lvl_size)
        throw Error{ESS_ERR_ARG, "internal: k-d slab buffer of the current level too small"};
    void *nx = s.kd_slabs[cur ^ 1];
    grow(nx, s.kd_slab_cap[cur ^ 1], (size_t)2 * lvl_size, slab_words * sizeof(int32_t));
    s.kd_slabs[cur ^ 1] = (int32_t *)nx;
    void *vr = s.kd_vr;
    grow(vr, s.kd_vr_cap, (size_t)lvl_size * 3 * S, sizeof(unsigned long long));
    s.kd_vr = (unsigned long long *)vr;
    grow(s.kd_dec, s.kd_dec_cap, (size_t)lvl_size, sizeof(KdDecision));
    void *bs = s.kd_block_sums;
    grow(bs, s.kd_bs_cap, (size_t)(lvl_size + 255) / 256, sizeof(uint32_t));
    s.kd_block_sums = (uint32_t *)bs;
}

void kd_free(Ctx &c, Structure &s)
{
    void *ptrs[] = {s.kd_slabs[0], s.kd_slabs[1], s.kd_vr, s.kd_dec, s.kd_block_sums};
    for (void *p : ptrs) c.free(p);
    s.kd_slabs[0] = s.kd_slabs[1] = nullptr;
    s.kd_vr = nullptr;
    s.kd_dec = nullptr;
    s.kd_block_sums = nullptr;
    s.kd_slab_cap[0] = s.kd_slab_cap[1] = s.kd_vr_cap = s.kd_dec_cap = s.kd_bs_cap = 0;
}

static int kd_slots(const Structure &s)
{
    if (s.p.nbins != 0) return s.p.nbins;
    return std::max(s.gx, std::max(s.gy, s.gz));
}

void launch_kd(Ctx &c, Structure &s, int64_t n)
{
    KdParams P;
    Volume *v = s.volume;
    P.B = s.p.brick;
    P.nx = v->nx;
    P.ny = v->ny;
    P.nz = v->nz;
    P.gx = s.gx;
    P.gy = s.gy;
    P.nbins = s.p.nbins;
    P.halting = s.p.halting;
    P.mls3 = s.p.mls > 0 ? (unsigned long long)s.p.mls * s.p.mls * s.p.mls : 0ull;
    P.S = kd_slots(s);
    s.height = 0;
    s.kd_count = 0;
    if (n <= 0) {
        ESS_CUDA(cudaMemsetAsync(s.kd_count_dev, 0, sizeof(int), c.stream));
        return;
    }
    const int capacity = s.kd_capacity;
    const unsigned bricks_blocks = (unsigned)((n + 255) / 256);
    // root
    int32_t init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    int32_t *root_box = s.kd_scratch_i32;
    ESS_CUDA(cudaMemcpyAsync(root_box, init, sizeof(init), cudaMemcpyHostToDevice, c.stream));
    {
        Launch L(c, "kd_root");
        k_kd_root_reduce<<<bricks_blocks, 256, 0, c.stream>>>(s.ids, s.count, s.gx, s.gy,
                                                              root_box);
    }
    if (s.kd_slab_cap[0] < 1) {
        c.free(s.kd_slabs[0]);
        s.kd_slabs[0] = (int32_t *)c.alloc(sizeof(int32_t) * 3 * P.S * 6 * 16);
        s.kd_slab_cap[0] = 16;
    }
    {
        Launch L(c, "kd_init");
        k_kd_init<<<1, 256, 0, c.stream>>>(root_box, s.kd_nodes, s.kd_slabs[0], P.S);
    }
    int prev_begin = 0, lvl_begin = 0, lvl_size = 1, cur = 0;
    int levels = 0;
    while (lvl_size > 0) {
        ++levels;
        if (levels > KD_MAX_LEVELS)
            throw Error{ESS_ERR_ARG, "k-d tree deeper than " + std::to_string(KD_MAX_LEVELS) +
                                         " levels (renderer stack limit)"};
        kd_reserve(c, s, lvl_size, P.S, cur);  // slabs for this level and 2x for the next
        unsigned nblk = (unsigned)((lvl_size + 255) / 256);
        {
            Launch L(c, "kd_accumulate");
            k_kd_accumulate<<<bricks_blocks, 256, 0, c.stream>>>(
                s.ids, s.count, s.brick_node, s.kd_nodes, prev_begin, lvl_begin, lvl_size,
                s.kd_slabs[cur], P);
        }
        {
            Launch L(c, "kd_decide");
            k_kd_decide<<<nblk, 256, 0, c.stream>>>(s.kd_nodes, lvl_begin, lvl_size,
                                                    s.kd_slabs[cur], s.kd_vr,
                                                    (KdDecision *)s.kd_dec, s.kd_block_sums, P);
        }
        {
            Launch L(c, "kd_scan");
            k_kd_scan<<<1, 1024, 0, c.stream>>>(s.kd_block_sums, (int)nblk, s.kd_splits_dev);
        }
        {
            Launch L(c, "kd_emit");
            k_kd_emit<<<nblk, 256, 0, c.stream>>>(lvl_begin, lvl_size, (const KdDecision *)s.kd_dec,
                                                  s.kd_block_sums, s.kd_nodes, s.kd_slabs[cur ^ 1],
                                                  P.S, capacity, c.dev_status);
        }
        ESS_CUDA(cudaMemcpyAsync(s.kd_splits_host, s.kd_splits_dev, sizeof(int),
                                 cudaMemcpyDeviceToHost, c.stream));
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        int splits = *s.kd_splits_host;
        prev_begin = lvl_begin;
        lvl_begin += lvl_size;
        lvl_size = 2 * splits;
        if (lvl_begin + lvl_size > capacity) {
            ESS_CUDA(cudaMemsetAsync(s.kd_count_dev, 0, sizeof(int), c.stream));
            throw Error{ESS_ERR_ARG, "k-d node capacity exceeded"};
        }
        cur ^= 1;
    }
    s.kd_count = lvl_begin;
    s.height = levels;
    s.kd_count_i32 = (int)s.kd_count;
    ESS_CUDA(cudaMemcpyAsync(s.kd_count_dev, &s.kd_count_i32, sizeof(int), cudaMemcpyHostToDevice,
                             c.stream));
    {
        Launch L(c, "kd_pack");
        k_kd_pack<<<(unsigned)((s.kd_count + 255) / 256), 256, 0, c.stream>>>(
            s.kd_nodes, s.kd_count_dev, s.nodes, s.root);
    }
}

size_t kd_decision_bytes() { return sizeof(KdDecision); }

}  // namespace ess
