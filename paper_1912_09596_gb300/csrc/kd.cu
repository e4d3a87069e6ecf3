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
// L and R boxes and picks the split, and one kernel numbers and emits the
// children (each block after the split counts of the blocks before it) and,
// in its last block to finish, moves the level state on.  For 4 bins the
// decide and emit steps are one kernel, and the whole level loop runs either
// as one cooperative launch with grid barriers between the steps (the
// default), as a CUDA graph with a conditional while node, or from the host.  With an even nbins the middle plane lo + floor(e/2) is
// candidate j = nbins/2, so a forced middle split also falls on a slab border.
#include <cuda_runtime.h>

#include <cstdlib>
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

// A node's decision; in the persistent build also the record through which
// its bricks move to a child (fc: the first child, -1 for a leaf), 64 bytes.
struct __align__(16) KdDecision {
    int32_t split;  // 1 if the node splits
    int32_t axis, plane, fc;
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

// A slab box is stored as 6 ints that only ever grow: 65536 - lo (per axis)
// and hi, so that every update is an atomicMax and an empty slab is all zeros
// (brick coordinates are below 65536).
constexpr int32_t KD_LO_BIAS = 65536;

// Loads of words that other blocks of a running kernel write (the
// persistent build): from L2 (ld.global.cg), never from a stale L1 line.
template <bool CG> __device__ __forceinline__ int32_t kd_ld(const int32_t *p)
{
    return CG ? __ldcg(p) : *p;
}

// Decodes a stored slab into a box; returns false for an empty slab.
template <bool CG = false> __device__ __forceinline__ bool slab_load(const int32_t *e, int32_t box[6])
{
    int32_t w[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = kd_ld<CG>(e + k);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        box[k] = KD_LO_BIAS - w[k];
        box[3 + k] = w[3 + k];
    }
    return w[0] != 0;
}

// Level state, in device memory so that the level loop can run without the
// host: the kernels of a level read it, the last emit block moves it on.
struct KdState {
    int prev_begin;  // first node of the previous level
    int lvl_begin;   // first node of the current level
    int lvl_size;    // nodes on the current level (0: done)
    int levels;      // levels started so far; the current level is number `levels`
    int splits;      // splits on the current level
    unsigned done;   // emit blocks finished on the current level
    unsigned epoch;  // bumped by every build: tags the look-back words of its levels
    unsigned bar;    // arrivals at the grid barriers of the persistent build
};

// Slab buffer of the current level (parity of the level number) and of the next.
__device__ __forceinline__ int32_t *kd_cur_slabs(int32_t *s0, int32_t *s1, const KdState *st)
{
    return (st->levels & 1) ? s1 : s0;
}
__device__ __forceinline__ int32_t *kd_next_slabs(int32_t *s0, int32_t *s1, const KdState *st)
{
    return (st->levels & 1) ? s0 : s1;
}

// -------------------------------------------------------------- root box
__global__ void k_kd_root_init(int32_t *root_box, KdState *st)
{
    if (threadIdx.x == 0) {
        root_box[0] = root_box[1] = root_box[2] = INT_MAX;
        root_box[3] = root_box[4] = root_box[5] = INT_MIN;
        st->prev_begin = 0;
        st->lvl_begin = 0;
        st->lvl_size = 1;
        st->levels = 0;
        st->splits = 0;
        st->done = 0;
        st->epoch += 1;
        st->bar = 0;
    }
}

// The tight brick box of bricks i (one per thread, i < n) into root_box by
// integer min/max atomics, one set per warp.
__device__ __forceinline__ void kd_root_add(const uint32_t *__restrict__ ids, int n, int i, int gx,
                                            int gy, int32_t *root_box)
{
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

__global__ void k_kd_root_reduce(const uint32_t *__restrict__ ids, const int *__restrict__ count,
                                 int gx, int gy, int32_t *root_box)
{
    kd_root_add(ids, *count, blockIdx.x * blockDim.x + threadIdx.x, gx, gy, root_box);
}

// node 0 record and the slabs of level 0 (no level at all for an empty mask)
__global__ void k_kd_init(const int *__restrict__ count, const int32_t *__restrict__ root_box,
                          int32_t *nodes9, int32_t *slabs0, int S, KdState *st)
{
    int t = threadIdx.x;
    if (*count <= 0) {
        if (t == 0) st->lvl_size = 0;
        return;
    }
    if (t < 6) nodes9[t] = root_box[t];
    if (t == 0) {
        nodes9[6] = -1;
        nodes9[7] = 0;
        nodes9[8] = -1;
    }
    for (int s = t; s < 3 * S * 6; s += blockDim.x) slabs0[s] = 0;
}

// ------------------------------------------------------------ per level
// Moves each brick of a node split on the previous level into its child,
// then adds the brick to the slab boxes of its node if that node is on the
// current level.  Updates are combined first: a whole warp on one slab
// reduces with warp intrinsics, otherwise a block-local hash table of slabs
// in shared memory takes the min/max, and each block then applies one set of
// global atomics per distinct slab (min/max are order independent, so the
// result is the same as with direct atomics).
constexpr int KD_HT = 128;          // shared hash slots per block of the per-level kernel
constexpr int KD_HT_PERSIST = 1024;  // ... of the persistent build (one block per SM)

__device__ __forceinline__ void slab_atomic(int32_t *slot, const int v[6])
{
    for (int k = 0; k < 6; ++k) atomicMax(slot + k, v[k]);
}

// One level of the accumulate step over the bricks this block takes (a
// grid-stride loop), through the shared hash table s_key / s_val of HT slots.
// NBINS > 0: the bin count known at compile time (divisions become shifts).
// CG: node records are read from L2 (the persistent build, where other blocks
// wrote them during the same kernel).
template <int NBINS, bool CG, int HT>
__device__ __forceinline__ void kd_accumulate_level(const uint32_t *__restrict__ ids, int n,
                                                    int *__restrict__ brick_node,
                                                    const int32_t *nodes9, int32_t *slabs,
                                                    int prev_begin, int lvl_begin, int lvl_size,
                                                    const KdParams &P, long long *s_key,
                                                    int (*s_val)[6])
{
    constexpr int HB = HT == 1024 ? 10 : HT == 512 ? 9 : HT == 256 ? 8 : 7;
    static_assert(HT == (1 << HB), "hash table size: a power of two, 128 to 1024");
    for (int h = threadIdx.x; h < HT; h += blockDim.x) {
        s_key[h] = -1;
        for (int k = 0; k < 6; ++k) s_val[h][k] = 0;
    }
    __syncthreads();
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;  // the loop is uniform per block
        bool live = i < n;
        int c[3] = {0, 0, 0};
        int node = -1;
        if (live) {
            brick_coords(ids[i], P.gx, P.gy, c);
            node = lvl_begin == 0 ? 0 : brick_node[i];
            if (node >= prev_begin && node < lvl_begin) {
                const int32_t *rec = nodes9 + 9 * (size_t)node;
                int fc = kd_ld<CG>(rec + 8);
                if (fc >= 0) {
                    node = fc + (c[kd_ld<CG>(rec + 6)] >= kd_ld<CG>(rec + 7) ? 1 : 0);
                    brick_node[i] = node;
                }
            } else if (lvl_begin == 0) {
                brick_node[i] = 0;
            }
            if (node < lvl_begin || node >= lvl_begin + lvl_size) live = false;
        }
        const int32_t *bp = nodes9 + 9 * (size_t)(live ? node : 0);
        int32_t box[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) box[k] = kd_ld<CG>(bp + k);
        int local = node - lvl_begin;
        const int v[6] = {KD_LO_BIAS - c[0], KD_LO_BIAS - c[1], KD_LO_BIAS - c[2],
                          c[0] + 1, c[1] + 1, c[2] + 1};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bool use = live && box[3 + a] - box[a] >= 2;
            int s = use ? kd_slab_of(c[a], box[a], box[3 + a], NBINS > 0 ? NBINS : P.nbins) : 0;
            long long slot_id = use ? ((long long)local * 3 + a) * P.S + s : -1;
            long long first = __shfl_sync(0xffffffffu, slot_id, 0);
            if (__all_sync(0xffffffffu, slot_id == first)) {
                if (first < 0) continue;
                int r[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) r[k] = __reduce_max_sync(0xffffffffu, v[k]);
                if ((threadIdx.x & 31) == 0) slab_atomic(slabs + 6 * first, r);
            } else if (use) {
                int h = (int)((unsigned long long)(slot_id * 0x9E3779B97F4A7C15ull) >> (64 - HB));
                bool done = false;
                for (int probe = 0; probe < 8 && !done; ++probe, h = (h + 1) & (HT - 1)) {
                    long long old = atomicCAS((unsigned long long *)&s_key[h], (unsigned long long)-1ll,
                                              (unsigned long long)slot_id);
                    if (old == -1 || old == slot_id) {
                        for (int k = 0; k < 6; ++k) atomicMax(&s_val[h][k], v[k]);
                        done = true;
                    }
                }
                if (!done) slab_atomic(slabs + 6 * slot_id, v);
            }
        }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < HT; h += blockDim.x) {
        long long key = s_key[h];
        if (key >= 0) {
            int r[6];
            for (int k = 0; k < 6; ++k) r[k] = s_val[h][k];
            slab_atomic(slabs + 6 * key, r);
        }
    }
}

template <int NBINS>
__global__ void __launch_bounds__(256) k_kd_accumulate(const uint32_t *__restrict__ ids,
                                                       const int *__restrict__ count,
                                                       int *__restrict__ brick_node,
                                                       const int32_t *__restrict__ nodes9,
                                                       int32_t *slabs0, int32_t *slabs1,
                                                       const KdState *st, KdParams P)
{
    __shared__ long long s_key[KD_HT];
    __shared__ int s_val[KD_HT][6];
    const int prev_begin = st->prev_begin, lvl_begin = st->lvl_begin, lvl_size = st->lvl_size;
    if (lvl_size <= 0) return;  // uniform
    kd_accumulate_level<NBINS, false, KD_HT>(ids, *count, brick_node, nodes9,
                                             kd_cur_slabs(slabs0, slabs1, st), prev_begin,
                                             lvl_begin, lvl_size, P, s_key, s_val);
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
// suffix volumes.  Writes the decision and the block's split count.  Before
// that, all threads of the grid zero the slab region the next level will use
// (at most two children per node) with 8-byte stores.  With SF > 0 the number
// of slab slots is the compile-time constant SF (the 4-bin case), so the slab
// loops unroll and their loads are independent.
template <int SF>
__global__ void __launch_bounds__(256) k_kd_decide(const int32_t *__restrict__ nodes9,
                                                   int32_t *slabs0, int32_t *slabs1,
                                                   unsigned long long *vr, KdDecision *dec,
                                                   uint32_t *block_sums, const KdState *st,
                                                   KdParams P, int next_cap)
{
    const int S = SF > 0 ? SF : P.S;
    const int lvl_begin = st->lvl_begin, lvl_size = st->lvl_size;
    if (lvl_size <= 0) return;  // uniform
    {
        // the next level has at most min(2 lvl_size, capacity) nodes
        int2 *next = reinterpret_cast<int2 *>(kd_next_slabs(slabs0, slabs1, st));
        size_t nodes = (size_t)min(2 * lvl_size, next_cap);
        size_t words = nodes * 9 * S;  // 18 S ints per node
        size_t stride = (size_t)gridDim.x * blockDim.x;
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < words; q += stride)
            next[q] = make_int2(0, 0);
    }
    if ((int)(blockIdx.x * blockDim.x) >= lvl_size) return;  // uniform per block
    const int32_t *slabs = kd_cur_slabs(slabs0, slabs1, st);
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
                const int32_t *sl = slabs + 6 * ((size_t)l * 3 + a) * S;
                unsigned long long *v = vr + ((size_t)l * 3 + a) * S;
                int32_t acc[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
                if (SF > 0) {
#pragma unroll
                    for (int j = (SF > 0 ? SF : 1) - 1; j >= 1; --j) {
                        if (j >= ns) continue;
                        int32_t b[6];
                        if (slab_load(sl + 6 * j, b)) box_union(acc, b);
                        v[j] = acc[0] == INT_MAX ? ~0ull : kd_volume(acc, P);
                    }
                } else {
                    for (int j = ns - 1; j >= 1; --j) {
                        int32_t b[6];
                        if (slab_load(sl + 6 * j, b)) box_union(acc, b);
                        v[j] = acc[0] == INT_MAX ? ~0ull : kd_volume(acc, P);
                    }
                }
                int32_t pre[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
                for (int j = 1; j < ns; ++j) {
                    int32_t b[6];
                    if (slab_load(sl + 6 * (j - 1), b)) box_union(pre, b);
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
            const int32_t *sl = slabs + 6 * ((size_t)l * 3 + bax) * S;
            int32_t L[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
            int32_t R[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
            for (int j = 0; j < ns; ++j) {
                int32_t b[6];
                if (!slab_load(sl + 6 * j, b)) continue;
                if (j < bj) box_union(L, b);
                else box_union(R, b);
            }
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

// Warp-parallel decide for 4 bins (4 slabs per axis): half a warp per node,
// lane (a, j) = (axis, slab) for the first 12 lanes.  The slab boxes' prefix
// unions (slabs before j: the L box of plane j) and suffix unions (slabs j
// onwards: the R box) come from shuffles within each axis's 4 lanes; the
// candidate of lane (a, j), 1 <= j < ns, costs V(L) + V(R), and the argmin
// over the half takes the lowest (axis, plane) among equal costs, as the
// per-thread form does.  Integer arithmetic only, so the decisions are the
// same.
//
// The same kernel emits the children.  A block takes chunks of 16
// consecutive nodes (one per half-warp) in increasing order; the split count
// of chunk c is chained to the chunks before it by a decoupled look-back (one
// 64-bit word per chunk: the level's tag, a flag and the count or prefix; a
// warp reads 32 predecessors' words per step), so the children of chunk c are
// numbered right after those of chunks < c, in breadth-first order.  The last
// block to finish moves the level state on.
__device__ __forceinline__ bool box_nonempty(const int32_t *b) { return b[0] != INT_MAX; }

constexpr int KD_CHUNK = 16;                    // nodes per look-back chunk
constexpr unsigned long long KD_LB_AGG = 1ull << 30, KD_LB_INC = 2ull << 30;
constexpr unsigned long long KD_LB_MASK = (1ull << 30) - 1;
constexpr long KD_LB_SPIN_LIMIT = 1l << 24;

// Move records of the persistent build (one barrier per level): the writer
// stores the boxes and the header's axis, plane and first child, then, after
// a fence, the level's tag in the header's first word; a reader polls that
// word (bounded), fences, and reads the record from L2.
constexpr long KD_MOVE_SPIN_LIMIT = 1l << 21;

__device__ __forceinline__ void kd_move_publish(KdDecision *m, int axis, int plane, int fc,
                                                const int32_t *L, const int32_t *R, int mtag)
{
    int4 *q = reinterpret_cast<int4 *>(m);
    if (fc >= 0) {
        q[1] = make_int4(L[0], L[1], L[2], L[3]);
        q[2] = make_int4(L[4], L[5], R[0], R[1]);
        q[3] = make_int4(R[2], R[3], R[4], R[5]);
    }
    m->axis = axis;
    m->plane = plane;
    m->fc = fc;
    __threadfence();
    *(volatile int32_t *)&m->split = mtag;
}

__device__ __forceinline__ int4 kd_move_wait(const KdDecision *m, int mtag, uint32_t *status)
{
    const volatile int32_t *t = &m->split;
    long spins = 0;
    while (*t != mtag) {
        // give up at the limit, or at once when another wait has given up
        if (++spins > KD_MOVE_SPIN_LIMIT ||
            ((spins & 1023) == 0 && (*(volatile uint32_t *)status & DEV_ERR_TIMEOUT))) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            return make_int4(0, 0, 0, -1);  // read as a leaf; the build reports the timeout
        }
    }
    __threadfence();
    return __ldcg(reinterpret_cast<const int4 *>(m));
}

// The level tag of the persistent build's move records (never 0 or 1, the
// split flags that the other build paths store in the same word).
__device__ __forceinline__ int kd_move_tag(unsigned epoch, int level)
{
    return (int)((((epoch & 0xfffffu) << 8) | (unsigned)(level & 0xff)) | 0x40000000u);
}

// One level of the fused 4-bin decide and emit over the chunks of CH nodes
// (16 lanes per node) this block takes: zeroes the next level's slab region,
// decides every node of the level, numbers the children through the
// look-back words (tagged with `tag`) and writes the split nodes' records and
// their children.  The last chunk stores the level's split count in *splits.
// CG: the persistent build: node records and slabs are read from L2, the
// next level's slabs were zeroed during the accumulate step, and the move
// records are published with the level tag `mtag` (kd_move_publish).
template <bool CG, int CH>
__device__ __forceinline__ void kd_decide_emit4_level(int32_t *nodes9, const int32_t *slabs,
                                                      int32_t *next_slabs,
                                                      unsigned long long *chunk_st, int *splits,
                                                      const KdParams &P, int next_cap,
                                                      int capacity, uint32_t *status,
                                                      int lvl_begin, int lvl_size,
                                                      unsigned long long tag,
                                                      KdDecision *moves = nullptr, int mtag = 0)
{
    constexpr int S = 4;
    static_assert(CH <= 32, "one ballot covers a chunk's nodes");
    if (!CG) {
        // the next level has at most min(2 lvl_size, capacity) nodes
        int2 *next = reinterpret_cast<int2 *>(next_slabs);
        const size_t words = (size_t)min(2 * lvl_size, next_cap) * 9 * S;  // 18 S ints per node
        const size_t stride = (size_t)gridDim.x * blockDim.x;
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < words; q += stride)
            next[q] = make_int2(0, 0);
    }
    int32_t root[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) root[k] = kd_ld<CG>(nodes9 + k);
    const unsigned long long Vroot = kd_volume(root, P);
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int a = (hl >> 2) < 3 ? hl >> 2 : 0, j = hl & 3;
    const bool slab_lane = hl < 12;
    __shared__ KdDecision sdec[CH];
    __shared__ int s_excl;
    const int nchunks = (lvl_size + CH - 1) / CH;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {  // uniform per block
        const int l = ch * CH + 2 * (threadIdx.x >> 5) + half;
        const bool node = l < lvl_size;
        const int32_t *X = nodes9 + 9 * (size_t)(lvl_begin + (node ? l : 0));
        int32_t x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = kd_ld<CG>(X + k);
        const unsigned long long V = kd_volume(x, P);
        const bool allowed = node && (P.halting == 0 ? (10ull * V > Vroot) : (V > 512ull));
        const int lo = x[a], hi = x[3 + a];
        const bool axis_ok = slab_lane && hi - lo >= 2;
        const int ns = axis_ok ? kd_slabs(lo, hi, 4) : 0;
        int32_t b[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
        if (allowed && axis_ok && j < ns) {
            int32_t t[6];
            if (slab_load<CG>(slabs + 6 * (((size_t)l * 3 + a) * S + j), t)) {
#pragma unroll
                for (int k = 0; k < 6; ++k) b[k] = t[k];
            }
        }
        // inclusive prefix and suffix unions over the axis's 4 lanes
        int32_t pre[6], suf[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) pre[k] = suf[k] = b[k];
#pragma unroll
        for (int d = 1; d < 4; d <<= 1) {
            int32_t up[6], dn[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                up[k] = __shfl_up_sync(0xffffffffu, pre[k], d, 4);
                dn[k] = __shfl_down_sync(0xffffffffu, suf[k], d, 4);
            }
            if (j >= d) box_union(pre, up);
            if (j + d < 4) box_union(suf, dn);
        }
        int32_t L[6];  // slabs before j: exclusive prefix
#pragma unroll
        for (int k = 0; k < 6; ++k) L[k] = __shfl_up_sync(0xffffffffu, pre[k], 1, 4);
        if (j == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) L[k] = INT_MAX, L[3 + k] = INT_MIN;
        }
        unsigned long long cost = ~0ull;
        if (allowed && axis_ok && j >= 1 && j < ns && box_nonempty(L) && box_nonempty(suf))
            cost = kd_volume(L, P) + kd_volume(suf, P);
        // argmin over the half: (cost, lane) in lexicographic order
        unsigned long long bc = cost;
        int bl = hl;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            const unsigned long long oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (oc < bc || (oc == bc && ol < bl)) {
                bc = oc;
                bl = ol;
            }
        }
        int bax = -1, bj = 0, bpl = 0;
        if (allowed && bc != ~0ull && bc < V) {
            bax = bl >> 2;
            bj = bl & 3;
            bpl = kd_plane(bj, x[bax], x[3 + bax], 4);
        } else if (allowed && P.mls3 > 0 && V > P.mls3) {
            int bestext = -1;
            const int n[3] = {P.nx, P.ny, P.nz};
            for (int ax = 0; ax < 3; ++ax) {
                const int e = x[3 + ax] - x[ax];
                if (e < 2) continue;
                const int ext = min(x[3 + ax] * P.B, n[ax]) - x[ax] * P.B;
                if (ext > bestext) {
                    bestext = ext;
                    bax = ax;
                    bpl = x[ax] + e / 2;
                }
            }
            if (bax >= 0) bj = kd_slab_of(bpl, x[bax], x[3 + bax], 4);
        }
        // the L and R boxes of the chosen plane are lane (bax, bj)'s
        const int src = (half << 4) + (bax >= 0 ? bax * 4 + bj : 0);
        int32_t dl[6], dr[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            dl[k] = __shfl_sync(0xffffffffu, L[k], src);
            dr[k] = __shfl_sync(0xffffffffu, suf[k], src);
        }
        if (hl == 0) {
            KdDecision d;
            d.split = 0;
            d.axis = -1;
            d.plane = 0;
            if (node && bax >= 0 && box_nonempty(dl) && box_nonempty(dr)) {
                d.split = 1;
                d.axis = bax;
                d.plane = bpl;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    d.L[k] = dl[k];
                    d.R[k] = dr[k];
                }
            }
            sdec[l - ch * CH] = d;
        }
        __syncthreads();
        // the chunk's split count, chained to the chunks before it: the first
        // warp reads the words of 32 predecessors at a time (lane i: chunk
        // base - i) and adds counts up to the nearest inclusive prefix
        if (threadIdx.x < 32) {
            const unsigned ball = __ballot_sync(0xffffffffu, lane < CH && sdec[lane].split);
            const unsigned long long cnt = (unsigned long long)__popc(ball);
            volatile unsigned long long *cs = chunk_st;
            unsigned long long excl = 0;
            if (ch > 0) {
                if (lane == 0) cs[ch] = tag | KD_LB_AGG | cnt;
                for (int base = ch - 1;; base -= 32) {
                    const int jj = base - lane;
                    unsigned long long v = KD_LB_INC;  // before chunk 0: an inclusive prefix of 0
                    if (jj >= 0) {
                        long spins = 0;
                        while (((v = cs[jj]) & ~(KD_LB_MASK | KD_LB_AGG | KD_LB_INC)) != tag ||
                               (v & (KD_LB_AGG | KD_LB_INC)) == 0ull) {
                            if (++spins > KD_LB_SPIN_LIMIT) {
                                atomicOr(status, DEV_ERR_TIMEOUT);
                                v = KD_LB_INC;
                                break;
                            }
                        }
                    }
                    const unsigned inc = __ballot_sync(0xffffffffu, (v & KD_LB_INC) != 0ull);
                    const int stop = inc ? __ffs(inc) - 1 : 31;  // the nearest inclusive prefix
                    unsigned long long add = lane <= stop ? (v & KD_LB_MASK) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
                    excl += add;
                    if (inc) break;  // uniform
                }
            }
            if (lane == 0) {
                __threadfence();
                cs[ch] = tag | KD_LB_INC | (excl + cnt);
                s_excl = (int)excl;
                if (ch == nchunks - 1) *splits = (int)(excl + cnt);
            }
        }
        __syncthreads();
        // emit: children of the chunk's split nodes, numbered in node order
        if (threadIdx.x < CH && sdec[threadIdx.x].split) {
            int rank = 0;
            for (int k = 0; k < (int)threadIdx.x; ++k) rank += sdec[k].split;
            const int fc = lvl_begin + lvl_size + 2 * (s_excl + rank);
            if (fc + 1 >= capacity) {
                atomicOr(status, DEV_ERR_OVERFLOW);
                if (CG) kd_move_publish(moves + ch * CH + threadIdx.x, 0, 0, -1, nullptr, nullptr, mtag);
                else if (moves) moves[ch * CH + threadIdx.x].fc = -1;
            } else {
                const KdDecision &d = sdec[threadIdx.x];
                int32_t *rec = nodes9 + 9 * (size_t)(lvl_begin + ch * CH + threadIdx.x);
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
                if (CG) {
                    kd_move_publish(moves + ch * CH + threadIdx.x, d.axis, d.plane, fc, d.L, d.R,
                                    mtag);
                } else if (moves) {
                    KdDecision m = d;
                    m.fc = fc;
                    moves[ch * CH + threadIdx.x] = m;
                }
            }
        } else if (moves && threadIdx.x < CH && ch * CH + (int)threadIdx.x < lvl_size) {
            // a leaf: its bricks stay
            if (CG) kd_move_publish(moves + ch * CH + threadIdx.x, 0, 0, -1, nullptr, nullptr, mtag);
            else moves[ch * CH + threadIdx.x].fc = -1;
        }
        __syncthreads();  // sdec and s_excl are rewritten by the next chunk
    }
}

__global__ void __launch_bounds__(256) k_kd_decide_emit4(int32_t *nodes9, int32_t *slabs0,
                                                         int32_t *slabs1,
                                                         unsigned long long *chunk_st, KdState *st,
                                                         KdParams P, int next_cap, int capacity,
                                                         int max_levels, uint32_t *status,
                                                         cudaGraphConditionalHandle handle,
                                                         int use_handle)
{
    const int lvl_begin = st->lvl_begin, lvl_size = st->lvl_size;
    if (lvl_size <= 0) {  // uniform: the tree is done
        if (use_handle && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0u);
        return;
    }
    const unsigned long long tag = ((unsigned long long)((st->epoch << 8) | (unsigned)st->levels)) << 32;
    kd_decide_emit4_level<false, KD_CHUNK>(nodes9, kd_cur_slabs(slabs0, slabs1, st),
                                           kd_next_slabs(slabs0, slabs1, st), chunk_st,
                                           &st->splits, P, next_cap, capacity, status, lvl_begin,
                                           lvl_size, tag);
    // the last block to finish advances the level
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    st->done = 0;
    int next = 2 * *(volatile int *)&st->splits;
    st->prev_begin = lvl_begin;
    st->lvl_begin = lvl_begin + lvl_size;
    st->levels += 1;
    if (next > 0 && (st->lvl_begin + next > capacity || st->levels >= max_levels)) {
        atomicOr(status, DEV_ERR_OVERFLOW);
        next = 0;
    }
    st->lvl_size = next;
    st->splits = 0;
    if (use_handle) cudaGraphSetConditional(handle, next > 0 ? 1u : 0u);
}

// Traversal layout: one BoxNode per node id (leaf entries unused), children
// referenced as node ids, leaves as -1 - id; the root record and node count.
template <bool CG>
__device__ __forceinline__ void kd_pack_node(const int32_t *nodes9, int i, BoxNode *nodes,
                                             int32_t *root, int B)
{
    const int32_t *rec = nodes9 + 9 * (size_t)i;
    const int fc = kd_ld<CG>(rec + 8);
    if (i == 0) {
        root[0] = fc >= 0 ? 0 : -1;
        for (int a = 0; a < 6; ++a) root[1 + a] = __float_as_int((float)(kd_ld<CG>(rec + a) * B));
    }
    if (fc < 0) return;
    const int32_t *L = nodes9 + 9 * (size_t)fc, *R = L + 9;
    BoxNode nd;
    for (int a = 0; a < 6; ++a) {
        nd.lbox[a] = (float)(kd_ld<CG>(L + a) * B);
        nd.rbox[a] = (float)(kd_ld<CG>(R + a) * B);
    }
    nd.left = kd_ld<CG>(L + 8) >= 0 ? fc : -1 - fc;
    nd.right = kd_ld<CG>(R + 8) >= 0 ? fc + 1 : -1 - (fc + 1);
    nd.pad0 = nd.pad1 = 0;
    nodes[i] = nd;
}

// The accumulate step of the persistent build: each thread keeps the nodes
// of its bricks (i = k x threads + its index, k < KMAX) in registers across
// the levels when the bricks fit (reg), and a brick of a node split on the
// previous level reads one 64-byte move record (its node's decision, first
// child and both children's boxes) instead of the node record and then the
// child's record.  Same slab updates as kd_accumulate_level.
template <int KMAX>
__device__ __forceinline__ void kd_accumulate_persist(
    const uint32_t *__restrict__ ids, int n, int *__restrict__ brick_node, int (&node_r)[KMAX],
    bool reg, const KdDecision *moves, int mtag_prev, const int32_t *root_rec, int32_t *slabs,
    int32_t *zero_slabs, size_t zero_words, int prev_begin, int lvl_begin, int lvl_size,
    const KdParams &P, long long *s_key, int (*s_val)[6], uint32_t *status)
{
    constexpr int HT = KD_HT_PERSIST, HB = 10;
    static_assert(HT == (1 << HB), "hash bits");
    for (int h = threadIdx.x; h < HT; h += blockDim.x) {
        s_key[h] = -1;
        for (int k = 0; k < 6; ++k) s_val[h][k] = 0;
    }
    const int gthreads = gridDim.x * blockDim.x;
    {
        // the slab buffer of the next level (no block reads or writes it now)
        int2 *z = reinterpret_cast<int2 *>(zero_slabs);
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < zero_words; q += gthreads)
            z[q] = make_int2(0, 0);
    }
    __syncthreads();
    auto brick = [&](int i, int &node) {
        bool live = i < n;
        int c[3] = {0, 0, 0};
        int32_t box[6];
        if (live) {
            brick_coords(ids[i], P.gx, P.gy, c);
            if (lvl_begin == 0) {
                node = 0;
            } else if (node >= prev_begin && node < lvl_begin) {
                const int4 *mv = reinterpret_cast<const int4 *>(moves + (node - prev_begin));
                const int4 h = kd_move_wait(moves + (node - prev_begin), mtag_prev, status);  // tag, axis, plane, fc
                if (h.w >= 0) {
                    const int side = c[h.y] >= h.z ? 1 : 0;
                    node = h.w + side;
                    const int4 q1 = __ldcg(mv + 1), q2 = __ldcg(mv + 2), q3 = __ldcg(mv + 3);
                    // L = q1.xyzw q2.xy, R = q2.zw q3.xyzw
                    box[0] = side ? q2.z : q1.x;
                    box[1] = side ? q2.w : q1.y;
                    box[2] = side ? q3.x : q1.z;
                    box[3] = side ? q3.y : q1.w;
                    box[4] = side ? q3.z : q2.x;
                    box[5] = side ? q3.w : q2.y;
                }
            }
            if (node < lvl_begin || node >= lvl_begin + lvl_size) live = false;
        }
        if (lvl_begin == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) box[k] = root_rec[k];
        }
        const int local = node - lvl_begin;
        const int v[6] = {KD_LO_BIAS - c[0], KD_LO_BIAS - c[1], KD_LO_BIAS - c[2],
                          c[0] + 1, c[1] + 1, c[2] + 1};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bool use = live && box[3 + a] - box[a] >= 2;
            int sl = use ? kd_slab_of(c[a], box[a], box[3 + a], 4) : 0;
            long long slot_id = use ? ((long long)local * 3 + a) * P.S + sl : -1;
            long long first = __shfl_sync(0xffffffffu, slot_id, 0);
            if (__all_sync(0xffffffffu, slot_id == first)) {
                if (first < 0) continue;
                int r[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) r[k] = __reduce_max_sync(0xffffffffu, v[k]);
                if ((threadIdx.x & 31) == 0) slab_atomic(slabs + 6 * first, r);
            } else if (use) {
                int h = (int)((unsigned long long)(slot_id * 0x9E3779B97F4A7C15ull) >> (64 - HB));
                bool done = false;
                for (int probe = 0; probe < 8 && !done; ++probe, h = (h + 1) & (HT - 1)) {
                    long long old = atomicCAS((unsigned long long *)&s_key[h], (unsigned long long)-1ll,
                                              (unsigned long long)slot_id);
                    if (old == -1 || old == slot_id) {
                        for (int k = 0; k < 6; ++k) atomicMax(&s_val[h][k], v[k]);
                        done = true;
                    }
                }
                if (!done) slab_atomic(slabs + 6 * slot_id, v);
            }
        }
    };
    if (reg) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int base = k * gthreads + blockIdx.x * blockDim.x;
            if (base >= n) break;  // uniform per block
            brick(base + threadIdx.x, node_r[k]);
        }
    } else {
        for (int base = blockIdx.x * blockDim.x; base < n; base += gthreads) {
            const int i = base + threadIdx.x;
            int node = i < n && lvl_begin > 0 ? brick_node[i] : 0;
            brick(i, node);
            if (i < n) brick_node[i] = node;
        }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < HT; h += blockDim.x) {
        long long key = s_key[h];
        if (key >= 0) {
            int r[6];
            for (int k = 0; k < 6; ++k) r[k] = s_val[h][k];
            slab_atomic(slabs + 6 * key, r);
        }
    }
}

// ---------------------------------------------------- persistent 4-bin build
// The whole level loop of a 4-bin build in one cooperative launch (all blocks
// resident, one per SM) with one grid barrier per level: the accumulate step,
// the barrier, the fused decide and emit step.  There is no barrier after the
// emit: a block goes on to the next level's accumulate as soon as it has the
// level's split count (the last look-back word, tagged with the level) and,
// brick by brick, the move record of the brick's node (tagged, see
// kd_move_publish).  The three slab buffers rotate so that the buffer a block
// zeroes during level l's accumulate (level l + 1's) is the one of level l - 2,
// which every block finished reading before level l - 1's barrier.  The same
// level bodies as the per-level kernels, so the same tree.  (Against two
// barriers per level: 0.347 -> 0.341 ms per 8^3 build of the 512^3 edits;
// reading the split count only at the end of the next accumulate step, to
// overlap its wait, measured 0.373 ms.)

// Grid barrier on a monotone arrival counter: the k-th barrier of a launch
// completes when the counter reaches k x gridDim.x.  The wait is bounded; a
// block that gives up sets DEV_ERR_TIMEOUT and returns false (the caller
// leaves the kernel; the other blocks then give up at their next barrier).
constexpr long KD_BAR_SPIN_LIMIT = 1l << 22;  // polls of L2, a few seconds at most
// Threads per block, 16 per node of a decide chunk (512, with 32-node chunks,
// measured slower).
constexpr int KD_PERSIST_THREADS = 256;

__device__ __forceinline__ bool kd_grid_sync(unsigned *bar, unsigned target, uint32_t *status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        long spins = 0;
        while (*(volatile unsigned *)bar < target) {
            if (++spins > KD_BAR_SPIN_LIMIT) {
                atomicOr(status, DEV_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// At most 80 registers (the launch bound's 3 blocks per SM; one block per SM
// is launched): the build runs beside the renders of the same edit, and its
// registers are taken from theirs (121 registers made the bench step 1.6 %
// slower at the same build time).
__global__ void __launch_bounds__(KD_PERSIST_THREADS, 3) k_kd_build4(
    const uint32_t *__restrict__ ids, const int *__restrict__ count, int *__restrict__ brick_node,
    int32_t *nodes9, int32_t *slabs0, int32_t *slabs1, int32_t *slabs2,
    unsigned long long *chunk_st, KdState *st, int32_t *root_box, BoxNode *nodes, int32_t *root,
    int *m_dev, KdDecision *moves, KdParams P, int next_cap, int capacity, int max_levels,
    uint32_t *status)
{
    constexpr int KMAX = 4;  // bricks per thread whose nodes stay in registers
    __shared__ long long s_key[KD_HT_PERSIST];
    __shared__ int s_val[KD_HT_PERSIST][6];
    const unsigned epoch = st->epoch;  // k_kd_root_init ran before: level state reset
    const int n = *count;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
    unsigned target = 0;
    int prev_begin = 0, lvl_begin = 0, levels = 0, lvl_size = n > 0 ? 1 : 0;
    if (lvl_size > 0) {  // uniform
        // root: the tight box of all non-empty bricks, node 0 and the level-0 slabs
        for (int base = 0; base < n; base += gthreads) kd_root_add(ids, n, base + gtid, P.gx, P.gy, root_box);
        if (!kd_grid_sync(&st->bar, target += gridDim.x, status)) return;
        if (blockIdx.x == 0) {
            if (threadIdx.x < 6) nodes9[threadIdx.x] = __ldcg(root_box + threadIdx.x);
            if (threadIdx.x == 0) {
                nodes9[6] = -1;
                nodes9[7] = 0;
                nodes9[8] = -1;
            }
            for (int q = threadIdx.x; q < 3 * 4 * 6; q += blockDim.x) slabs0[q] = 0;
        }
        if (!kd_grid_sync(&st->bar, target += gridDim.x, status)) return;
    }
    int node_r[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) node_r[k] = 0;
    const bool reg = (long long)n <= (long long)KMAX * gthreads;
    int32_t root_rec[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) root_rec[k] = lvl_size > 0 ? __ldcg(nodes9 + k) : 0;
    constexpr int CH = KD_PERSIST_THREADS / 16;
    __shared__ int s_next;
    while (lvl_size > 0) {  // uniform
        const int m3 = levels % 3;
        int32_t *cur = m3 == 0 ? slabs0 : (m3 == 1 ? slabs1 : slabs2);
        int32_t *nxt = m3 == 0 ? slabs1 : (m3 == 1 ? slabs2 : slabs0);
        const size_t zero_words = (size_t)min(2 * lvl_size, next_cap) * 9 * 4;  // 18 S ints per node
        kd_accumulate_persist<KMAX>(ids, n, brick_node, node_r, reg, moves,
                                    kd_move_tag(epoch, levels - 1), root_rec, cur, nxt, zero_words,
                                    prev_begin, lvl_begin, lvl_size, P, s_key, s_val, status);
        if (!kd_grid_sync(&st->bar, target += gridDim.x, status)) return;
        const unsigned long long tag = ((unsigned long long)((epoch << 8) | (unsigned)levels)) << 32;
        kd_decide_emit4_level<true, CH>(nodes9, cur, nxt, chunk_st, &st->splits, P, next_cap,
                                        capacity, status, lvl_begin, lvl_size, tag, moves,
                                        kd_move_tag(epoch, levels));
        // the level's split count: the last chunk's inclusive look-back word
        // (rewritten only after the next level's barrier, which this block
        // has not reached)
        if (threadIdx.x == 0) {
            const volatile unsigned long long *w = chunk_st + (lvl_size + CH - 1) / CH - 1;
            unsigned long long v;
            long spins = 0;
            while (((v = *w) & ~(KD_LB_MASK | KD_LB_AGG | KD_LB_INC)) != tag ||
                   (v & KD_LB_INC) == 0ull) {
                if (++spins > KD_LB_SPIN_LIMIT) {
                    atomicOr(status, DEV_ERR_TIMEOUT);
                    v = KD_LB_INC;  // no splits: the loop ends
                    break;
                }
            }
            s_next = 2 * (int)(v & KD_LB_MASK);
        }
        __syncthreads();
        int next = s_next;
        __syncthreads();  // s_next is rewritten at the next level
        prev_begin = lvl_begin;
        lvl_begin += lvl_size;
        levels += 1;
        if (next > 0 && (lvl_begin + next > capacity || levels >= max_levels)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, DEV_ERR_OVERFLOW);
            next = 0;
        }
        lvl_size = next;
    }
    // traversal layout of the finished tree, after a barrier: every record of
    // the last level's emit is written
    if (!kd_grid_sync(&st->bar, target += gridDim.x, status)) return;
    for (int i = gtid; i < lvl_begin; i += gthreads) kd_pack_node<true>(nodes9, i, nodes, root, P.B);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *m_dev = lvl_begin;
        st->prev_begin = prev_begin;
        st->lvl_begin = lvl_begin;
        st->lvl_size = 0;
        st->levels = levels;
        st->splits = 0;
        st->done = 0;
    }
}

// Sum of v over the block (256 threads).
__device__ __forceinline__ uint32_t kd_block_sum(uint32_t v)
{
    __shared__ uint32_t part[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[w] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += part[j];
    __syncthreads();
    return t;
}

// Emit and advance of one level.  Each block holding nodes of the level
// numbers its split nodes after the splits of the blocks before it (the sum
// of their counts from the decide step), writes the split decisions and the
// two children of each split node; the last block to finish moves the level
// state on (next level = the children, 2 x all splits) and, in the graph,
// sets the loop condition.
__global__ void __launch_bounds__(256) k_kd_emit(const KdDecision *__restrict__ dec,
                                                 uint32_t *block_counts,
                                                 int32_t *nodes9, int capacity, int max_levels,
                                                 uint32_t *status, KdState *st,
                                                 cudaGraphConditionalHandle handle, int use_handle)
{
    const int lvl_begin = st->lvl_begin, lvl_size = st->lvl_size;
    const int nblk = (lvl_size + 255) / 256;
    for (int gb = blockIdx.x; gb < nblk; gb += gridDim.x) {  // uniform per block
        uint32_t off = 0;
        for (int i = threadIdx.x; i < gb; i += blockDim.x) off += block_counts[i];
        off = kd_block_sum(off);
        const int l = gb * blockDim.x + threadIdx.x;
        const int split = l < lvl_size ? dec[l].split : 0;
        // block-local exclusive rank of the split flag
        __shared__ uint32_t wcount[8];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const uint32_t ball = __ballot_sync(0xffffffffu, split);
        if (lane == 0) wcount[w] = __popc(ball);
        __syncthreads();
        uint32_t before = 0;
        for (int j = 0; j < w; ++j) before += wcount[j];
        if (split) {
            const uint32_t rank = off + before + __popc(ball & ((1u << lane) - 1u));
            const int fc = lvl_begin + lvl_size + 2 * (int)rank;
            if (fc + 1 >= capacity) {
                atomicOr(status, DEV_ERR_OVERFLOW);
            } else {
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
            }
        }
        __syncthreads();  // wcount is rewritten by the next group
    }
    // the last block to finish advances the level
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint32_t total = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) total += block_counts[i];
    total = kd_block_sum(total);
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) block_counts[i] = 0;  // for the next level
    if (threadIdx.x != 0) return;
    st->done = 0;
    if (lvl_size > 0) {
        int next = 2 * (int)total;
        st->prev_begin = lvl_begin;
        st->lvl_begin = lvl_begin + lvl_size;
        st->levels += 1;
        if (next > 0 && (st->lvl_begin + next > capacity || st->levels >= max_levels)) {
            atomicOr(status, DEV_ERR_OVERFLOW);
            next = 0;
        }
        st->lvl_size = next;
        st->splits = 0;
    }
    if (use_handle) cudaGraphSetConditional(handle, st->lvl_size > 0 ? 1u : 0u);
}


// Traversal layout (kd_pack_node), one thread per node.
__global__ void k_kd_pack(const int32_t *__restrict__ nodes9, const KdState *st, int *m_dev,
                          BoxNode *nodes, int32_t *root, int B)
{
    int m = st->lvl_begin;  // all levels done: every node id is below this
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *m_dev = m;
    if (i >= m) return;
    kd_pack_node<false>(nodes9, i, nodes, root, B);
}

// ------------------------------------------------------------------ host
static int kd_slots(const Structure &s)
{
    if (s.p.nbins != 0) return s.p.nbins;
    return std::max(s.gx, std::max(s.gy, s.gz));
}

static KdParams kd_params(const Structure &s)
{
    KdParams P;
    const Volume *v = s.volume;
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
    return P;
}

static void grow(Ctx &c, void *&p, size_t &cap, size_t need, size_t elem)
{
    if (cap >= need) return;
    c.free(p);
    size_t n = std::max(need, cap * 2);
    p = c.alloc(n * elem);
    cap = n;
}

// Per-level buffers of the host loop: the current level's slabs were reset
// by the previous level's emit and already fit; the next level (at most twice
// as many nodes) may need a larger buffer, whose old contents are not needed.
void kd_reserve(Ctx &c, Structure &s, int lvl_size, int S, int cur)
{
    size_t slab_words = (size_t)3 * S * 6;
    if (s.kd_slab_cap[cur] < (size_t)lvl_size)
        throw Error{ESS_ERR_ARG, "internal: k-d slab buffer of the current level too small"};
    void *nx = s.kd_slabs[cur ^ 1];
    grow(c, nx, s.kd_slab_cap[cur ^ 1], (size_t)2 * lvl_size, slab_words * sizeof(int32_t));
    s.kd_slabs[cur ^ 1] = (int32_t *)nx;
    void *vr = s.kd_vr;
    grow(c, vr, s.kd_vr_cap, (size_t)lvl_size * 3 * S, sizeof(unsigned long long));
    s.kd_vr = (unsigned long long *)vr;
    grow(c, s.kd_dec, s.kd_dec_cap, (size_t)lvl_size, sizeof(KdDecision));
    void *bs = s.kd_block_sums;
    const size_t bs_cap = s.kd_bs_cap;
    grow(c, bs, s.kd_bs_cap, (size_t)(lvl_size + 255) / 256, sizeof(uint32_t));
    s.kd_block_sums = (uint32_t *)bs;
    // the split counts start from zero (a new buffer; the emit kernel zeroes
    // them after each level)
    if (s.kd_bs_cap != bs_cap)
        ESS_CUDA(cudaMemsetAsync(s.kd_block_sums, 0, sizeof(uint32_t) * s.kd_bs_cap, c.stream));
}

// Look-back words of the fused 4-bin step: one per chunk of the widest level
// (at most one node per non-empty brick), zeroed once (they carry the tag of
// the build and level that wrote them).
static void kd_chunk_reserve(Ctx &c, Structure &s)
{
    const size_t need = (size_t)(s.nb + KD_CHUNK - 1) / KD_CHUNK + 2;
    if (s.kd_chunk_cap >= need) return;
    c.free(s.kd_chunk);
    s.kd_chunk = (unsigned long long *)c.alloc(need * sizeof(unsigned long long));
    s.kd_chunk_cap = need;
    ESS_CUDA(cudaMemsetAsync(s.kd_chunk, 0, need * sizeof(unsigned long long), c.stream));
}

void kd_free(Ctx &c, Structure &s)
{
    void *ptrs[] = {s.kd_slabs[0], s.kd_slabs[1], s.kd_slabs[2], s.kd_vr, s.kd_dec,
                    s.kd_block_sums, s.kd_chunk};
    for (void *p : ptrs) c.free(p);
    s.kd_chunk = nullptr;
    s.kd_chunk_cap = 0;
    s.kd_slabs[0] = s.kd_slabs[1] = s.kd_slabs[2] = nullptr;
    s.kd_vr = nullptr;
    s.kd_dec = nullptr;
    s.kd_block_sums = nullptr;
    s.kd_slab_cap[0] = s.kd_slab_cap[1] = s.kd_slab_cap[2] = 0;
    s.kd_vr_cap = s.kd_dec_cap = s.kd_bs_cap = 0;
    if (s.kd_exec) cudaGraphExecDestroy(s.kd_exec);
    if (s.kd_graph) cudaGraphDestroy(s.kd_graph);
    s.kd_exec = nullptr;
    s.kd_graph = nullptr;
}

// The root part of a build: root box, node 0, level-0 slabs.
static void kd_root_launches(Ctx &c, Structure &s, const KdParams &P, unsigned brick_blocks)
{
    KdState *st = (KdState *)s.kd_state;
    if (s.kd_block_sums)  // per-level split counts start from zero
        ESS_CUDA(cudaMemsetAsync(s.kd_block_sums, 0, sizeof(uint32_t) * s.kd_bs_cap, c.stream));
    k_kd_root_init<<<1, 32, 0, c.stream>>>(s.kd_scratch_i32, st);
    k_kd_root_reduce<<<brick_blocks, 256, 0, c.stream>>>(s.ids, s.count, s.gx, s.gy,
                                                         s.kd_scratch_i32);
    k_kd_init<<<1, 256, 0, c.stream>>>(s.count, s.kd_scratch_i32, s.kd_nodes, s.kd_slabs[0], P.S,
                                       st);
}

// One level: accumulate, decide, emit (which also advances the level state).
static void kd_level_launches(Ctx &c, Structure &s, const KdParams &P, unsigned brick_blocks,
                              unsigned node_blocks, unsigned emit_blocks, int next_cap,
                              cudaGraphConditionalHandle h, int use_handle)
{
    KdState *st = (KdState *)s.kd_state;
    if (P.nbins == 4)
        k_kd_accumulate<4><<<brick_blocks, 256, 0, c.stream>>>(s.ids, s.count, s.brick_node,
                                                               s.kd_nodes, s.kd_slabs[0],
                                                               s.kd_slabs[1], st, P);
    else
        k_kd_accumulate<0><<<brick_blocks, 256, 0, c.stream>>>(s.ids, s.count, s.brick_node,
                                                               s.kd_nodes, s.kd_slabs[0],
                                                               s.kd_slabs[1], st, P);
    if (P.S == 4) {  // decide and emit in one kernel
        k_kd_decide_emit4<<<emit_blocks, 256, 0, c.stream>>>(
            s.kd_nodes, s.kd_slabs[0], s.kd_slabs[1], s.kd_chunk, st, P, next_cap, s.kd_capacity,
            KD_MAX_LEVELS, c.dev_status, h, use_handle);
        return;
    }
    k_kd_decide<0><<<node_blocks, 256, 0, c.stream>>>(s.kd_nodes, s.kd_slabs[0], s.kd_slabs[1],
                                                      s.kd_vr, (KdDecision *)s.kd_dec,
                                                      s.kd_block_sums, st, P, next_cap);
    k_kd_emit<<<emit_blocks, 256, 0, c.stream>>>((const KdDecision *)s.kd_dec, s.kd_block_sums,
                                                 s.kd_nodes, s.kd_capacity, KD_MAX_LEVELS,
                                                 c.dev_status, st, h, use_handle);
}

// Whether the whole build runs as one device-driven graph: binned planes and
// level buffers for the widest possible level (one node per non-empty brick)
// within an eighth of the free memory.  The environment variable
// ESS_KD_GRAPH=0 selects the host-driven level loop instead (same kernels,
// same tree): profilers that time kernels one by one cannot look inside a
// graph with a conditional node.
static bool kd_graph_fits(const Structure &s, int S)
{
    if (s.p.nbins == 0) return false;
    const char *env = std::getenv("ESS_KD_GRAPH");
    if (env && env[0] == '0') return false;
    size_t cap = (size_t)s.nb;
    size_t bytes = 2 * cap * 3 * S * 6 * sizeof(int32_t) + cap * 3 * S * sizeof(unsigned long long) +
                   cap * sizeof(KdDecision) + ((cap + 255) / 256) * sizeof(uint32_t);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
    return bytes < free_b / 8;
}

// Levels per iteration of the graph's while loop.  Each iteration of a
// conditional node costs far more than a kernel node, so the body holds several
// levels; a level after the last one finds an empty level state and returns at
// once (all three kernels), and the emit kernel of every level sets the loop
// condition.
constexpr int KD_LEVELS_PER_ITERATION = 4;

// Level buffers for the widest possible level (one node per non-empty brick).
static void kd_full_buffers(Ctx &c, Structure &s, const KdParams &P, int slab_buffers = 2)
{
    size_t cap = (size_t)s.nb;
    size_t slab_words = (size_t)3 * P.S * 6;
    for (int b = 0; b < slab_buffers; ++b) {
        void *p = s.kd_slabs[b];
        grow(c, p, s.kd_slab_cap[b], std::max<size_t>(cap, 16), slab_words * sizeof(int32_t));
        s.kd_slabs[b] = (int32_t *)p;
    }
    void *vr = s.kd_vr;
    grow(c, vr, s.kd_vr_cap, cap * 3 * P.S, sizeof(unsigned long long));
    s.kd_vr = (unsigned long long *)vr;
    grow(c, s.kd_dec, s.kd_dec_cap, cap, sizeof(KdDecision));
    void *bs = s.kd_block_sums;
    grow(c, bs, s.kd_bs_cap, (cap + 255) / 256, sizeof(uint32_t));
    s.kd_block_sums = (uint32_t *)bs;
    kd_chunk_reserve(c, s);
}

// Blocks of the persistent 4-bin build: one per SM when the device launches
// cooperative kernels and fits one block per SM, else 0 (not available).  Two
// or four per SM measured slower (the grid barriers cost more).  The
// environment variable ESS_KD_PERSIST=0 turns it off (the graph runs instead).
static int kd_persist_blocks(Ctx &c)
{
    const char *env = std::getenv("ESS_KD_PERSIST");
    if (env && env[0] == '0') return 0;
    int coop = 0, sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c.device) != cudaSuccess || !coop)
        return 0;
    ESS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    ESS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kd_build4,
                                                           KD_PERSIST_THREADS, 0));
    // one block per SM builds fastest alone; half or a quarter of the SMs
    // left more room to overlapping frames (step -1.5 / -2.3 %) but took the
    // 8^3 build from 0.35 to 0.38 / 0.53 ms
    return per_sm >= 1 ? sms : 0;
}

// Root kernels, the cooperative level loop and the traversal layout.
static void kd_build_persistent(Ctx &c, Structure &s, const KdParams &P, int blocks)
{
    kd_full_buffers(c, s, P, 3);
    const size_t cap = (size_t)s.nb;
    KdState *st = (KdState *)s.kd_state;
    k_kd_root_init<<<1, 32, 0, c.stream>>>(s.kd_scratch_i32, st);  // resets the barrier counter
    int next_cap = (int)std::min(std::min(s.kd_slab_cap[0], s.kd_slab_cap[1]), s.kd_slab_cap[2]);
    int capacity = s.kd_capacity, max_levels = KD_MAX_LEVELS;
    KdParams Pk = P;
    const uint32_t *ids = s.ids;
    const int *count = s.count;
    int *brick_node = s.brick_node;
    int32_t *nodes9 = s.kd_nodes, *s0 = s.kd_slabs[0], *s1 = s.kd_slabs[1], *s2 = s.kd_slabs[2];
    unsigned long long *chunk = s.kd_chunk;
    uint32_t *status = c.dev_status;
    int32_t *root_box = s.kd_scratch_i32, *root = s.root;
    BoxNode *nodes = s.nodes;
    int *m_dev = s.kd_count_dev;
    KdDecision *moves = (KdDecision *)s.kd_dec;  // one per node of a level (kd_full_buffers)
    void *args[] = {&ids, &count, &brick_node, &nodes9, &s0, &s1, &s2, &chunk, &st, &root_box,
                    &nodes, &root, &m_dev, &moves, &Pk, &next_cap, &capacity, &max_levels,
                    &status};
    ESS_CUDA(cudaLaunchCooperativeKernel((const void *)k_kd_build4, dim3((unsigned)blocks),
                                         dim3(KD_PERSIST_THREADS), args, 0, c.stream));
}

static void kd_build_graph(Ctx &c, Structure &s, const KdParams &P)
{
    size_t cap = (size_t)s.nb;
    kd_full_buffers(c, s, P);
    if (!c.capture_stream)
        ESS_CUDA(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking));

    // The level kernels loop over their work, so their grids are sized for the
    // machine (a few blocks per SM) rather than for the widest possible level,
    // except the one-thread-per-node decide step of other bin counts.
    const unsigned brick_blocks = (unsigned)((cap + 255) / 256);
    int sms = 0;
    ESS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    const unsigned acc_blocks = std::min(brick_blocks, 4u * (unsigned)sms);
    const unsigned emit_blocks = std::min(brick_blocks, 2u * (unsigned)sms);
    const unsigned node_blocks = P.S == 4 ? emit_blocks : brick_blocks;
    cudaGraph_t g;
    ESS_CUDA(cudaGraphCreate(&g, 0));
    cudaStream_t saved = c.stream;
    c.stream = c.capture_stream;
    try {
        // root part
        ESS_CUDA(cudaStreamBeginCaptureToGraph(c.stream, g, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        kd_root_launches(c, s, P, brick_blocks);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        ESS_CUDA(cudaStreamGetCaptureInfo(c.stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
        std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
        ESS_CUDA(cudaStreamEndCapture(c.stream, &g));
        // level loop as a conditional while node
        cudaGraphConditionalHandle h;
        ESS_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop;
        ESS_CUDA(cudaGraphAddNode(&loop, g, tail.data(), nullptr, tail.size(), &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ESS_CUDA(cudaStreamBeginCaptureToGraph(c.stream, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        for (int u = 0; u < KD_LEVELS_PER_ITERATION; ++u)
            kd_level_launches(c, s, P, acc_blocks, node_blocks, emit_blocks,
                              (int)std::min(s.kd_slab_cap[0], s.kd_slab_cap[1]), h, 1);
        ESS_CUDA(cudaStreamEndCapture(c.stream, &body));
        // traversal layout after the loop
        ESS_CUDA(cudaStreamBeginCaptureToGraph(c.stream, g, &loop, nullptr, 1,
                                               cudaStreamCaptureModeThreadLocal));
        k_kd_pack<<<(unsigned)((2 * cap + 255) / 256), 256, 0, c.stream>>>(
            s.kd_nodes, (const KdState *)s.kd_state, s.kd_count_dev, s.nodes, s.root, P.B);
        ESS_CUDA(cudaStreamEndCapture(c.stream, &g));
        ESS_CUDA(cudaGraphInstantiate(&s.kd_exec, g, 0));
    } catch (...) {
        c.stream = saved;
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(c.capture_stream, &cs) == cudaSuccess &&
            cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(c.capture_stream, &tmp);
            if (tmp && tmp != g) cudaGraphDestroy(tmp);
        }
        cudaGraphDestroy(g);
        throw;
    }
    c.stream = saved;
    s.kd_graph = g;
}

void launch_kd(Ctx &c, Structure &s)
{
    KdParams P = kd_params(s);
    s.height = -1;
    s.kd_count = -1;
    if (P.S == 4 && kd_graph_fits(s, P.S)) {
        // device-driven: the whole level loop is one cooperative launch
        const int blocks = kd_persist_blocks(c);
        if (blocks > 0) {
            Launch L(c, "kd_build");
            kd_build_persistent(c, s, P, blocks);
            return;
        }
    }
    if (s.kd_exec || kd_graph_fits(s, P.S)) {
        // device-driven: the whole level loop is one graph launch
        if (!s.kd_exec) kd_build_graph(c, s, P);
        Launch L(c, "kd_build_graph");
        ESS_CUDA(cudaGraphLaunch(s.kd_exec, c.stream));
        return;
    }
    // host-driven level loop (exhaustive planes or buffers too large)
    if (P.S == 4) kd_chunk_reserve(c, s);
    int64_t n_cap = s.nb;
    const unsigned brick_blocks = (unsigned)((n_cap + 255) / 256);
    if (s.kd_slab_cap[0] < 16) {
        c.free(s.kd_slabs[0]);
        s.kd_slabs[0] = (int32_t *)c.alloc(sizeof(int32_t) * 3 * P.S * 6 * 16);
        s.kd_slab_cap[0] = 16;
    }
    {
        Launch L(c, "kd_root");
        kd_root_launches(c, s, P, brick_blocks);
    }
    KdState hs{};
    int lvl_size = 1, levels = 0;
    while (true) {
        int cur = levels & 1;
        kd_reserve(c, s, lvl_size, P.S, cur);
        unsigned nblk = (unsigned)((lvl_size + 255) / 256);
        {
            Launch L(c, "kd_level");
            kd_level_launches(c, s, P, brick_blocks, nblk, nblk, (int)s.kd_slab_cap[cur ^ 1], 0, 0);
        }
        ESS_CUDA(cudaMemcpyAsync(&hs, s.kd_state, sizeof(KdState), cudaMemcpyDeviceToHost,
                                 c.stream));
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        lvl_size = hs.lvl_size;
        levels = hs.levels;
        if (lvl_size <= 0) break;
    }
    {
        Launch L(c, "kd_pack");
        k_kd_pack<<<(unsigned)((hs.lvl_begin + 255) / 256 + 1), 256, 0, c.stream>>>(
            s.kd_nodes, (const KdState *)s.kd_state, s.kd_count_dev, s.nodes, s.root, P.B);
    }
}

// Node count and height of the last build (waits for it).
void kd_stats(Ctx &c, Structure &s)
{
    if (s.kd_count >= 0) return;
    KdState hs{};
    ESS_CUDA(cudaMemcpyAsync(&hs, s.kd_state, sizeof(KdState), cudaMemcpyDeviceToHost, c.stream));
    ESS_CUDA(cudaStreamSynchronize(c.stream));
    s.kd_count = hs.lvl_begin;
    s.height = hs.levels;
}

size_t kd_decision_bytes() { return sizeof(KdDecision); }

}  // namespace ess
