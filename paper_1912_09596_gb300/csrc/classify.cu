// classify.cu -- the empty test: per-brick apron min/max (once per volume and
// brick size), TF prefix counts, the min/max range test that yields the brick
// mask, the per-cell vote variant, and stream compaction of the non-empty
// bricks (Sec. 3.1 compacts the brick list to the non-empty bricks before
// assigning Morton codes).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "ess_internal.h"

namespace ess {

// ------------------------------------------------------------------ helpers
template <typename T> __device__ __forceinline__ float to_f(T v) { return (float)v; }

__device__ __forceinline__ float tf_coord(float v, float value_lo, float s, float xmax)
{
    float x = (v - value_lo) * s;
    x = x < 0.0f ? 0.0f : x;
    x = x > xmax ? xmax : x;
    return x;
}

// ------------------------------------------------------------ finite check
__global__ void k_check_finite(const float *__restrict__ v, size_t n, uint32_t *status)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) bad |= !isfinite(v[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, DEV_ERR_NONFINITE);
}

void launch_check_finite(Ctx &c, const float *v, size_t n)
{
    Launch L(c, "check_finite");
    k_check_finite<<<152 * 8, 256, 0, c.stream>>>(v, n, c.dev_status);
}

// ------------------------------------------------------- trilinear cells
// Cell (cx, cy, cz), 0 <= c <= n, holds the 8 corner values that a sample with
// floor(p - 0.5) = (cx-1, cy-1, cz-1) interpolates, neighbours clamped to the
// volume, in the order 000 100 010 110 001 101 011 111 (x fastest): one
// vector load per sample instead of eight scalar ones, same values.
size_t cell_array_bytes(const Volume &v)
{
    size_t el = v.dtype == ESS_U8 ? 1 : (v.dtype == ESS_U16 ? 2 : 4);
    return (size_t)(v.nx + 1) * (v.ny + 1) * (v.nz + 1) * 8 * el;
}

template <typename T> struct CellStore;
template <> struct CellStore<uint8_t> {
    static __device__ __forceinline__ void put(void *cells, size_t i, const uint32_t v[8])
    {
        uint2 w = make_uint2(v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24),
                             v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24));
        reinterpret_cast<uint2 *>(cells)[i] = w;
    }
};
template <> struct CellStore<uint16_t> {
    static __device__ __forceinline__ void put(void *cells, size_t i, const uint32_t v[8])
    {
        uint4 w = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16),
                             v[6] | (v[7] << 16));
        reinterpret_cast<uint4 *>(cells)[i] = w;
    }
};
template <> struct CellStore<float> {
    static __device__ __forceinline__ void put(void *cells, size_t i, const uint32_t v[8])
    {
        uint4 *p = reinterpret_cast<uint4 *>(cells) + 2 * i;
        p[0] = make_uint4(v[0], v[1], v[2], v[3]);
        p[1] = make_uint4(v[4], v[5], v[6], v[7]);
    }
};

template <typename T> __device__ __forceinline__ uint32_t raw_bits(T x) { return (uint32_t)x; }
template <> __device__ __forceinline__ uint32_t raw_bits<float>(float x) { return __float_as_uint(x); }

template <typename T>
__global__ void k_build_cells(const T *__restrict__ vol, int nx, int ny, int nz, void *cells)
{
    size_t sx = (size_t)nx + 1, sy = (size_t)ny + 1;
    size_t ncell = sx * sy * ((size_t)nz + 1);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
         i += (size_t)gridDim.x * blockDim.x) {
        int cx = (int)(i % sx), cy = (int)((i / sx) % sy), cz = (int)(i / (sx * sy));
        int x0 = max(cx - 1, 0), x1 = min(cx, nx - 1);
        int y0 = max(cy - 1, 0), y1 = min(cy, ny - 1);
        int z0 = max(cz - 1, 0), z1 = min(cz, nz - 1);
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int x = (k & 1) ? x1 : x0, y = (k & 2) ? y1 : y0, z = (k & 4) ? z1 : z0;
            v[k] = raw_bits(__ldg(vol + ((size_t)z * ny + y) * (size_t)nx + x));
        }
        CellStore<T>::put(cells, i, v);
    }
}

void launch_build_cells(Ctx &c, const Volume &v, void *cells)
{
    Launch L(c, "build_cells");
    switch (v.dtype) {
    case ESS_U8:
        k_build_cells<uint8_t><<<152 * 16, 256, 0, c.stream>>>((const uint8_t *)v.data, v.nx, v.ny,
                                                               v.nz, cells);
        break;
    case ESS_U16:
        k_build_cells<uint16_t><<<152 * 16, 256, 0, c.stream>>>((const uint16_t *)v.data, v.nx, v.ny,
                                                                v.nz, cells);
        break;
    default:
        k_build_cells<float><<<152 * 16, 256, 0, c.stream>>>((const float *)v.data, v.nx, v.ny, v.nz,
                                                             cells);
    }
}

// ------------------------------------------------------------ K1 min/max
// Brick b covers voxels [bB, (b+1)B) and its samples read the apron range
// [bB-1, (b+1)B] (clamped to the volume), so min/max run over that range.
// One warp per (by, bz) and run of 32 bricks along x: lane l owns brick
// bx = 32*seg + l and walks its (B+2)^2 apron rows; the 32 lanes of a warp
// read one contiguous stretch of each row, so the loads coalesce and the
// apron overlap between neighbours is served by L1.
template <typename T>
__global__ void __launch_bounds__(256) k_brick_minmax(const T *__restrict__ vol, int nx,
                                                      int ny, int nz, int B, int gx, int gy,
                                                      int gz, float2 *__restrict__ out)
{
    int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    int nseg = (gx + 31) >> 5;
    int total = nseg * gy * gz;
    if (warp >= total) return;
    int seg = warp % nseg;
    int rest = warp / nseg;
    int by = rest % gy, bz = rest / gy;
    int bx = seg * 32 + lane;
    if (bx >= gx) return;
    int x0 = max(bx * B - 1, 0), x1 = min((bx + 1) * B, nx - 1);
    int y0 = max(by * B - 1, 0), y1 = min((by + 1) * B, ny - 1);
    int z0 = max(bz * B - 1, 0), z1 = min((bz + 1) * B, nz - 1);
    float mn = INFINITY, mx = -INFINITY;
    for (int z = z0; z <= z1; ++z) {
        for (int y = y0; y <= y1; ++y) {
            const T *row = vol + ((size_t)z * ny + y) * (size_t)nx;
            for (int x = x0; x <= x1; ++x) {
                float v = to_f(__ldg(row + x));
                mn = v < mn ? v : mn;
                mx = v > mx ? v : mx;
            }
        }
    }
    out[((size_t)bz * gy + by) * gx + bx] = make_float2(mn, mx);
}

// Vectorised form for rows made of whole 16-byte vectors and power-of-two
// bricks.  One CTA per unit (brick row y, brick row z, chunk of 32 vectors in
// x); lane l of each warp owns the 16-byte vector l of the chunk, i.e.
// VPL = 16 / sizeof(T) consecutive voxel columns.  The unit's (B+2)^2 apron
// rows are cut into steps of up to R consecutive rows of one z plane, dealt
// round-robin to the CTA's warps; each warp keeps a few steps in flight with
// cp.async copies (one coalesced 512-byte row per copy instruction) into a
// per-warp ring in shared memory, and every lane reads back only the 16
// bytes it copied itself.  Moving R rows per step spreads the pipeline's
// bookkeeping (wait, commit, addressing) over R rows.  The brick region is a box,
// so its minimum is the minimum over its x range of the per-column minima
// over its rows: a lane accumulates column-wise minima/maxima (for 8-bit
// voxels two columns per f16x2 register, one min/max instruction serving
// both) and reduces across x once at the end, after the warps have
// merged their columns through shared memory.  The apron columns on both
// sides of a brick come from neighbouring lanes by shuffles; at a chunk
// boundary the edge lane also copies the neighbouring chunk's vector.  With
// B <= VPL a lane holds VPL / B whole bricks; with B > VPL a brick spans
// B / VPL lanes, reduced by shuffles.

// Two 16-bit lanes per register.  min/max.f16x2 and min/max.u16x2 measured
// the same throughput as a 32-bit min; the byte-wise __vminu4/__vmaxu4
// measured about a sixth of it, so bytes are widened to halves first.
__device__ __forceinline__ uint32_t min_h2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max_h2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min_u2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max_u2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Column-wise min/max over rows of one 16-byte vector per row (add), plus the
// min/max of one edge column taken from another vector per row (edge: its
// last voxel for the column left of the lane's vector, else its first).
template <typename T> struct ColMinMax;
template <> struct ColMinMax<uint8_t> {
    // A byte b placed under the high byte 0x64 is the half 1024 + b, a normal
    // f16 whose order is that of b: word i of the vector gives the half pairs
    // (b0, b1) and (b2, b3), i.e. columns (4i, 4i+1) and (4i+2, 4i+3).
    uint32_t mna[4], mnb[4], mxa[4], mxb[4];
    uint32_t emn, emx;  // one edge column (see ColMinMax::edge)
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) mna[i] = mnb[i] = 0x64ff64ffu, mxa[i] = mxb[i] = 0x64006400u;
        emn = 0xffu, emx = 0u;
    }
    __device__ __forceinline__ void edge(const uint4 &w, bool last)
    {
        const uint32_t v = last ? w.w >> 24 : w.x & 0xffu;
        emn = min(emn, v), emx = max(emx, v);
    }
    __device__ __forceinline__ float edge_min() const { return (float)emn; }
    __device__ __forceinline__ float edge_max() const { return (float)emx; }
    __device__ __forceinline__ void add(const uint4 &w)
    {
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t a = __byte_perm(q[i], 0x64646464u, 0x4140);
            const uint32_t b = __byte_perm(q[i], 0x64646464u, 0x4342);
            mna[i] = min_h2(mna[i], a);
            mnb[i] = min_h2(mnb[i], b);
            mxa[i] = max_h2(mxa[i], a);
            mxb[i] = max_h2(mxb[i], b);
        }
    }
    __device__ __forceinline__ void columns(float *mn, float *mx) const
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            mn[4 * i + 0] = (float)(mna[i] & 0xffu), mn[4 * i + 1] = (float)((mna[i] >> 16) & 0xffu);
            mn[4 * i + 2] = (float)(mnb[i] & 0xffu), mn[4 * i + 3] = (float)((mnb[i] >> 16) & 0xffu);
            mx[4 * i + 0] = (float)(mxa[i] & 0xffu), mx[4 * i + 1] = (float)((mxa[i] >> 16) & 0xffu);
            mx[4 * i + 2] = (float)(mxb[i] & 0xffu), mx[4 * i + 3] = (float)((mxb[i] >> 16) & 0xffu);
        }
    }
};
template <> struct ColMinMax<uint16_t> {
    // word i holds columns 2i (low half) and 2i+1 (high half): one
    // min.u16x2 and one max.u16x2 per two voxels
    uint32_t mn[4], mx[4];
    uint32_t emn, emx;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) mn[i] = 0xffffffffu, mx[i] = 0u;
        emn = 0xffffu, emx = 0u;
    }
    __device__ __forceinline__ void edge(const uint4 &w, bool last)
    {
        const uint32_t v = last ? w.w >> 16 : w.x & 0xffffu;
        emn = min(emn, v), emx = max(emx, v);
    }
    __device__ __forceinline__ float edge_min() const { return (float)emn; }
    __device__ __forceinline__ float edge_max() const { return (float)emx; }
    __device__ __forceinline__ void add(const uint4 &w)
    {
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) mn[i] = min_u2(mn[i], q[i]), mx[i] = max_u2(mx[i], q[i]);
    }
    __device__ __forceinline__ void columns(float *cmn, float *cmx) const
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cmn[2 * i] = (float)(mn[i] & 0xffffu), cmn[2 * i + 1] = (float)(mn[i] >> 16);
            cmx[2 * i] = (float)(mx[i] & 0xffffu), cmx[2 * i + 1] = (float)(mx[i] >> 16);
        }
    }
};
template <> struct ColMinMax<float> {
    float mnf[4], mxf[4];
    float emn, emx;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) mnf[i] = INFINITY, mxf[i] = -INFINITY;
        emn = INFINITY, emx = -INFINITY;
    }
    __device__ __forceinline__ void edge(const uint4 &w, bool last)
    {
        const float v = __uint_as_float(last ? w.w : w.x);
        emn = fminf(v, emn), emx = fmaxf(v, emx);
    }
    __device__ __forceinline__ float edge_min() const { return emn; }
    __device__ __forceinline__ float edge_max() const { return emx; }
    __device__ __forceinline__ void add(const uint4 &w)
    {
        const float q[4] = {__uint_as_float(w.x), __uint_as_float(w.y), __uint_as_float(w.z),
                            __uint_as_float(w.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            mnf[i] = fminf(q[i], mnf[i]);
            mxf[i] = fmaxf(q[i], mxf[i]);
        }
    }
    __device__ __forceinline__ void columns(float *mn, float *mx) const
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) mn[i] = mnf[i], mx[i] = mxf[i];
    }
};

constexpr int MM_SLOT = 34;  // 16-byte vectors per row slot: 32 lanes + 2 edge vectors

// Pipeline shape for brick size B: a step moves a block of R consecutive
// rows of one z plane, NB blocks cover the plane's B + 2 apron rows, and a
// warp keeps DEPTH steps (about 20 rows) in flight.  Larger bricks mean
// fewer units with more rows each, so a unit gets more warps: 2 up to 8^3,
// 4 at 16^3, 8 beyond.  The (B + 2) * NB steps of an interior unit divide
// evenly among them for B <= 32.
template <int B> struct MmShape {
    static constexpr int NB = (B + 2 + 9) / 10;
    static constexpr int R = (B + 2 + NB - 1) / NB;
    static constexpr int DEPTH = 20 / R > 2 ? 20 / R : 2;
    static constexpr int WARPS = B <= 8 ? 2 : (B <= 16 ? 4 : 8);
};

// Shared memory of one unit (dynamic: above 48 KiB for the 8-warp units).
// Per warp: the ring of DEPTH steps, later reused for the merge of its
// columns (2 VPL + 2 floats per lane).
template <typename T, int B> struct MmSmem {
    static constexpr int VPL = 16 / (int)sizeof(T);
    static constexpr int ROW_BYTES = MM_SLOT * 16;
    static constexpr int STEP_BYTES = MmShape<B>::R * ROW_BYTES;
    static constexpr int RING_BYTES = MmShape<B>::DEPTH * STEP_BYTES;
    static constexpr int MERGE_BYTES = (2 * VPL + 2) * 32 * 4;
    static constexpr int WARP_BYTES = RING_BYTES > MERGE_BYTES ? RING_BYTES : MERGE_BYTES;
    static constexpr int BYTES = MmShape<B>::WARPS * WARP_BYTES;
};

__device__ __forceinline__ void cp_async16(uint32_t smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint4 lds16(uint32_t smem)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem)
                 : "memory");
    return v;
}
template <typename T, int B>
__global__ void __launch_bounds__(MmShape<B>::WARPS * 32) k_brick_minmax_vec(const T *__restrict__ vol, int nx,
                                                                    int ny, int nz, int gx, int gy,
                                                                    int gz, float2 *__restrict__ out)
{
    constexpr int VPL = 16 / (int)sizeof(T);
    constexpr int R = MmShape<B>::R, NB = MmShape<B>::NB, DEPTH = MmShape<B>::DEPTH;
    constexpr int MM_WARPS = MmShape<B>::WARPS;
    constexpr int ROW_BYTES = MmSmem<T, B>::ROW_BYTES;
    constexpr int STEP_BYTES = MmSmem<T, B>::STEP_BYTES;
    constexpr int RING_BYTES = MmSmem<T, B>::RING_BYTES;
    constexpr int WARP_BYTES = MmSmem<T, B>::WARP_BYTES;
    static_assert(NB * R >= B + 2, "blocks must cover the apron rows");
    extern __shared__ __align__(16) unsigned char smem[];  // MmSmem<T, B>::BYTES
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int row_vecs = nx / VPL;
    const int nchunk = (row_vecs + 31) >> 5;
    const int chunk = blockIdx.x % nchunk;
    const int rest = blockIdx.x / nchunk;
    const int by = rest % gy, bz = rest / gy;
    const int vec = chunk * 32 + lane;
    const bool have = vec < row_vecs;
    const bool ledge = lane == 0 && chunk > 0;             // column x0 - 1 is another chunk's
    const bool redge = lane == 31 && vec + 1 < row_vecs;  // column x0 + VPL is another chunk's
    const bool edge = ledge || redge;
    const bool edges = nchunk > 1;  // uniform: some lane of the unit needs an edge column
    const int y0 = max(by * B - 1, 0), y1 = min((by + 1) * B, ny - 1);
    const int z0 = max(bz * B - 1, 0), z1 = min((bz + 1) * B, nz - 1);
    const int nyr = y1 - y0 + 1;
    // steps g = (plane g / NB, block g % NB), dealt round-robin to the warps
    const int nsteps = (z1 - z0 + 1) * NB;
    const int my_steps = nsteps > wid ? (nsteps - wid + MM_WARPS - 1) / MM_WARPS : 0;

    // shared addresses of the lane's vector and of its edge vector in row 0 of slot 0
    const uint32_t ring = (uint32_t)__cvta_generic_to_shared(smem + wid * WARP_BYTES);
    const uint32_t mine = ring + lane * 16, edge_at = ring + (ledge ? 32 : 33) * 16;
    const size_t rv = (size_t)row_vecs;
    // A lane past the row's end copies the row's last vector: its columns are
    // then copies of voxels that the last brick holds anyway.
    const uint4 *base = reinterpret_cast<const uint4 *>(vol) + min(vec, row_vecs - 1);
    const int edelta = ledge ? -1 : 1;
    auto rows_of = [&](int k) {  // valid rows of this warp's step k
        const int blk = (wid + MM_WARPS * k) % NB;
        return min(R, nyr - blk * R);
    };
    auto issue = [&](int k, uint32_t off) {
        if (k < my_steps) {
            const int g = wid + MM_WARPS * k;
            const int blk = g % NB;
            const int nv = min(R, nyr - blk * R);
            const uint4 *src = base + ((size_t)(z0 + g / NB) * ny + (y0 + blk * R)) * rv;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (j < nv) {
                    cp_async16(mine + off + j * ROW_BYTES, src + j * rv);
                    if (edge) cp_async16(edge_at + off + j * ROW_BYTES, src + j * rv + edelta);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < DEPTH; ++k) issue(k, k * STEP_BYTES);

    ColMinMax<T> acc;
    acc.init();
    uint32_t off = 0;
    for (int k = 0; k < my_steps; ++k) {
        cp_async_wait<DEPTH - 1>();  // step k has landed
        const int nv = rows_of(k);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (j < nv) {
                acc.add(lds16(mine + off + j * ROW_BYTES));
                // lanes without an edge column read a slot nobody wrote and
                // discard the result; no branch on the lane
                if (edges) acc.edge(lds16(edge_at + off + j * ROW_BYTES), ledge);
            }
        }
        issue(k + DEPTH, off);
        off = off + STEP_BYTES == RING_BYTES ? 0u : off + STEP_BYTES;
    }
    cp_async_wait<0>();
    const float emn = acc.edge_min(), emx = acc.edge_max();  // meaningful on edge lanes only

    // merge the warps' columns through shared memory (the rings are done)
    float cmn[VPL], cmx[VPL];
    acc.columns(cmn, cmx);
    float lmn = emn, lmx = emx;
    __syncthreads();
    float *mrg = reinterpret_cast<float *>(smem);
    if (wid > 0) {
        float *m = reinterpret_cast<float *>(smem + wid * WARP_BYTES);
#pragma unroll
        for (int j = 0; j < VPL; ++j) m[j * 32 + lane] = cmn[j], m[(VPL + j) * 32 + lane] = cmx[j];
        m[(2 * VPL) * 32 + lane] = lmn;
        m[(2 * VPL + 1) * 32 + lane] = lmx;
    }
    __syncthreads();
    if (wid > 0) return;
#pragma unroll
    for (int w = 1; w < MM_WARPS; ++w) {
        const float *m = mrg + w * (WARP_BYTES / 4);
#pragma unroll
        for (int j = 0; j < VPL; ++j) {
            const float a = m[j * 32 + lane], b = m[(VPL + j) * 32 + lane];
            cmn[j] = a < cmn[j] ? a : cmn[j];
            cmx[j] = b > cmx[j] ? b : cmx[j];
        }
        const float a0 = m[(2 * VPL) * 32 + lane], a1 = m[(2 * VPL + 1) * 32 + lane];
        lmn = fminf(a0, lmn);
        lmx = fmaxf(a1, lmx);
    }

    // apron columns left and right of the lane's VPL columns
    float amn = __shfl_up_sync(0xffffffffu, cmn[VPL - 1], 1);
    float amx = __shfl_up_sync(0xffffffffu, cmx[VPL - 1], 1);
    float bmn = __shfl_down_sync(0xffffffffu, cmn[0], 1);
    float bmx = __shfl_down_sync(0xffffffffu, cmx[0], 1);
    if (lane == 0) {
        amn = ledge ? lmn : cmn[0];  // x = 0 clamps to itself
        amx = ledge ? lmx : cmx[0];
    }
    if (vec + 1 >= row_vecs) {
        bmn = cmn[VPL - 1];  // x = nx - 1 clamps to itself
        bmx = cmx[VPL - 1];
    } else if (lane == 31) {
        bmn = lmn;
        bmx = lmx;
    }
    if constexpr (B <= VPL) {
        constexpr int PER = VPL / B;
        if (!have) return;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            float m0 = k == 0 ? amn : cmn[k * B - 1];
            float m1 = k == 0 ? amx : cmx[k * B - 1];
            const float e0 = k == PER - 1 ? bmn : cmn[(k + 1) * B];
            const float e1 = k == PER - 1 ? bmx : cmx[(k + 1) * B];
            m0 = e0 < m0 ? e0 : m0;
            m1 = e1 > m1 ? e1 : m1;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                m0 = cmn[k * B + j] < m0 ? cmn[k * B + j] : m0;
                m1 = cmx[k * B + j] > m1 ? cmx[k * B + j] : m1;
            }
            out[((size_t)bz * gy + by) * gx + vec * PER + k] = make_float2(m0, m1);
        }
    } else {
        constexpr int LANES = B / VPL;  // divides 32
        float m0 = cmn[0], m1 = cmx[0];
#pragma unroll
        for (int j = 1; j < VPL; ++j) {
            m0 = cmn[j] < m0 ? cmn[j] : m0;
            m1 = cmx[j] > m1 ? cmx[j] : m1;
        }
        if (vec % LANES == 0) {
            m0 = amn < m0 ? amn : m0;
            m1 = amx > m1 ? amx : m1;
        }
        if (vec % LANES == LANES - 1 || vec + 1 >= row_vecs) {
            m0 = bmn < m0 ? bmn : m0;
            m1 = bmx > m1 ? bmx : m1;
        }
#pragma unroll
        for (int o = 1; o < LANES; o <<= 1) {
            const float a0 = __shfl_xor_sync(0xffffffffu, m0, o);
            const float a1 = __shfl_xor_sync(0xffffffffu, m1, o);
            m0 = a0 < m0 ? a0 : m0;
            m1 = a1 > m1 ? a1 : m1;
        }
        if (have && vec % LANES == 0) out[((size_t)bz * gy + by) * gx + vec / LANES] = make_float2(m0, m1);
    }
}

template <typename T>
bool launch_minmax_vec(Ctx &c, const T *data, int nx, int ny, int nz, int B, int gx, int gy, int gz,
                       float2 *out)
{
    constexpr int VPL = 16 / (int)sizeof(T);
    if ((nx % VPL) != 0 || ((uintptr_t)data & 15u) != 0) return false;
    size_t units = (size_t)((nx / VPL + 31) / 32) * gy * gz;
    if (units > (size_t)INT32_MAX) return false;
    unsigned blocks = (unsigned)units;
    Launch L(c, "brick_minmax");
#define ESS_MMV(BB)                                                                           \
    case BB:                                                                                  \
        if (MmSmem<T, BB>::BYTES > 48 * 1024)                                                 \
            ESS_CUDA(cudaFuncSetAttribute(k_brick_minmax_vec<T, BB>,                          \
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                          MmSmem<T, BB>::BYTES));                             \
        k_brick_minmax_vec<T, BB><<<blocks, MmShape<BB>::WARPS * 32, MmSmem<T, BB>::BYTES,      \
                                    c.stream>>>(data, nx, ny, nz, gx, gy, gz, out);           \
        return true;
    switch (B) {
        ESS_MMV(2)
        ESS_MMV(4)
        ESS_MMV(8)
        ESS_MMV(16)
        ESS_MMV(32)
        ESS_MMV(64)
    }
#undef ESS_MMV
    return false;
}

void launch_brick_minmax(Ctx &c, const Volume &v, int B, float2 *out)
{
    int gx = (v.nx + B - 1) / B, gy = (v.ny + B - 1) / B, gz = (v.nz + B - 1) / B;
    // rows of whole 16-byte blocks and bricks up to 8^3: staged by the tensor
    // copy engine (minmax_tma.cu); measured on a GB300 it moves 8^3-brick
    // tiles faster than the cp.async pipeline below, which is faster for the
    // larger bricks (their tiles hold more rows per thread)
    if (B <= 8 && launch_brick_minmax_tma(c, v, B, out)) return;
    bool done = false;
    switch (v.dtype) {
    case ESS_U8:
        done = launch_minmax_vec(c, (const uint8_t *)v.data, v.nx, v.ny, v.nz, B, gx, gy, gz, out);
        break;
    case ESS_U16:
        done = launch_minmax_vec(c, (const uint16_t *)v.data, v.nx, v.ny, v.nz, B, gx, gy, gz, out);
        break;
    default:
        done = launch_minmax_vec(c, (const float *)v.data, v.nx, v.ny, v.nz, B, gx, gy, gz, out);
    }
    if (done) return;
    // any other row length or brick size: one thread per brick
    size_t warps = (size_t)((gx + 31) / 32) * gy * gz;
    unsigned blocks = (unsigned)((warps + 7) / 8);
    Launch L(c, "brick_minmax");
    switch (v.dtype) {
    case ESS_U8:
        k_brick_minmax<uint8_t><<<blocks, 256, 0, c.stream>>>((const uint8_t *)v.data, v.nx, v.ny,
                                                              v.nz, B, gx, gy, gz, out);
        break;
    case ESS_U16:
        k_brick_minmax<uint16_t><<<blocks, 256, 0, c.stream>>>((const uint16_t *)v.data, v.nx,
                                                               v.ny, v.nz, B, gx, gy, gz, out);
        break;
    default:
        k_brick_minmax<float><<<blocks, 256, 0, c.stream>>>((const float *)v.data, v.nx, v.ny,
                                                            v.nz, B, gx, gy, gz, out);
    }
}

// --------------------------------------------------------- K2 TF prefix
// prefix[i] = #{j < i : alpha_j > 0}, i = 0..nt (one block).  With
// `validate`, a table that holds a non-finite value or an alpha outside
// [0, 1] sets DEV_ERR_BAD_TF (tables uploaded from device memory are checked
// here so that a TF edit never waits for the host).
__global__ void __launch_bounds__(1024) k_tf_prefix(const float4 *__restrict__ table, int nt,
                                                    int *__restrict__ prefix,
                                                    float4 *__restrict__ lut, int validate,
                                                    uint32_t *status)
{
    // the renderer's interpolation table: entry i and the difference to entry
    // i + 1 (the table's entry nt repeats nt - 1), rounded to float32 exactly
    // as the lerp fmaf(w, c1 - c0, c0) of R5 rounds it
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const float4 c0 = table[i], c1 = table[i + 1];
        lut[2 * i] = c0;
        lut[2 * i + 1] = make_float4(c1.x - c0.x, c1.y - c0.y, c1.z - c0.z, c1.w - c0.w);
    }
    __shared__ int warp_tot[32];
    int t = threadIdx.x;
    int per = (nt + 1023) / 1024;
    int b0 = t * per, b1 = min(nt, b0 + per);
    int cnt = 0;
    bool bad = false;
    for (int i = b0; i < b1; ++i) {
        float4 e = table[i];
        cnt += e.w > 0.0f ? 1 : 0;
        bad |= !(isfinite(e.x) && isfinite(e.y) && isfinite(e.z) && e.w >= 0.0f && e.w <= 1.0f);
    }
    if (validate && __syncthreads_or(bad) && t == 0) atomicOr(status, DEV_ERR_BAD_TF);
    // block-wide exclusive scan of cnt
    int lane = t & 31, w = t >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    int base = (w > 0 ? warp_tot[w - 1] : 0) + incl - cnt;
    for (int i = b0; i < b1; ++i) {
        prefix[i] = base;
        base += table[i].w > 0.0f ? 1 : 0;
    }
    if (t == 1023) prefix[nt] = warp_tot[31];
}

void launch_tf_prefix(Ctx &c, const float4 *table, int nt, int *prefix, float4 *lut,
                      int validate)
{
    Launch L(c, "tf_prefix");
    k_tf_prefix<<<1, 1024, 0, c.stream>>>(table, nt, prefix, lut, validate, c.dev_status);
}

// ---------------------------------------------------- K2 range test (mask)
// Every sample of a brick has a value in [min, max] of its apron (a lerp
// fmaf(f, b - a, a) with f in [0, 1) never leaves [a, b]); with x() monotone
// it reads TF entries floor(x(min)) .. floor(x(max)) + 1 only, so the brick is
// non-empty iff one of those entries has alpha > 0 (prefix-count difference).
__global__ void k_brick_mask(const float2 *__restrict__ minmax, int64_t nb,
                             const int *__restrict__ prefix, int nt, float value_lo, float s,
                             uint8_t *__restrict__ mask)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    float2 m = minmax[b];
    float xmax = (float)(nt - 1);
    int lo = (int)tf_coord(m.x, value_lo, s, xmax);
    int hi = (int)tf_coord(m.y, value_lo, s, xmax) + 1;
    hi = hi > nt - 1 ? nt - 1 : hi;
    mask[b] = (__ldg(prefix + hi + 1) - __ldg(prefix + lo)) > 0 ? 1 : 0;
}

void launch_brick_mask(Ctx &c, const float2 *minmax, int64_t nb, const TF &tf, float value_lo,
                       float s, uint8_t *mask)
{
    Launch L(c, "brick_mask");
    unsigned blocks = (unsigned)((nb + 255) / 256);
    k_brick_mask<<<blocks, 256, 0, c.stream>>>(minmax, nb, tf.prefix, tf.nt, value_lo, s, mask);
}

// ------------------------------------------------ per-cell vote variant
// The paper's LBVH classifier decides visibility per voxel and lets the
// threads of a brick vote (Sec. 3.1).  The exact form of that vote for
// interpolated samples: brick b is non-empty iff some trilinear cell c whose
// sample region [c+0.5, c+1.5) touches the brick's closed region (per axis
// c = bB-1 .. min((b+1)B, n)-1, corner voxels c and c+1 clamped) passes the
// range test of its own 8 corner values.  Those corners all lie in the
// brick's apron, so a cell's range lies inside the brick's min/max range and
// the vote can only clear bricks that the range test marked: the mask is
// first the range test's (K2, from the min/max of the volume pass K1), then
// one warp per marked brick tests its cells 32 at a time and stops at the
// first positive one; a brick without one is cleared.  Bricks the range test
// passes are nearly always truly visible, so the typical brick costs one
// round of 32 cells.
template <typename T>
__global__ void __launch_bounds__(256) k_vote_bricks(const T *__restrict__ vol, int nx, int ny,
                                                     int nz, int B, int gx, int gy, int64_t nb,
                                                     const int *__restrict__ prefix, int nt,
                                                     float value_lo, float s,
                                                     uint8_t *__restrict__ mask)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float xmax = (float)(nt - 1);
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += warps) {
        if (mask[b] == 0) continue;  // uniform: the range test already cleared it
        const int bx = (int)(b % gx), by = (int)((b / gx) % gy), bz = (int)(b / ((int64_t)gx * gy));
        // cells touching the brick, per axis: lo .. hi (lo >= -1, hi <= n - 1)
        const int lx = bx * B - 1, ly = by * B - 1, lz = bz * B - 1;
        const int ex = min((bx + 1) * B, nx) - 1 - lx + 1;
        const int ey = min((by + 1) * B, ny) - 1 - ly + 1;
        const int ez = min((bz + 1) * B, nz) - 1 - lz + 1;
        const int ncell = ex * ey * ez;
        bool found = false;
        for (int base = 0; base < ncell && !found; base += 32) {  // uniform
            const int i = base + lane;
            bool pos = false;
            if (i < ncell) {
                const int cx = lx + i % ex, cy = ly + (i / ex) % ey, cz = lz + i / (ex * ey);
                const int x0 = max(cx, 0), x1 = min(cx + 1, nx - 1);
                const int y0 = max(cy, 0), y1 = min(cy + 1, ny - 1);
                const int z0 = max(cz, 0), z1 = min(cz + 1, nz - 1);
                float mn = INFINITY, mx = -INFINITY;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const size_t idx = ((size_t)((k & 4) ? z1 : z0) * ny + ((k & 2) ? y1 : y0)) *
                                           (size_t)nx + ((k & 1) ? x1 : x0);
                    const float v = to_f(__ldg(vol + idx));
                    mn = v < mn ? v : mn;
                    mx = v > mx ? v : mx;
                }
                const int lo = (int)tf_coord(mn, value_lo, s, xmax);
                int hi = (int)tf_coord(mx, value_lo, s, xmax) + 1;
                hi = hi > nt - 1 ? nt - 1 : hi;
                pos = (__ldg(prefix + hi + 1) - __ldg(prefix + lo)) > 0;
            }
            found = __any_sync(0xffffffffu, pos);
        }
        if (!found && lane == 0) mask[b] = 0;
    }
}

// the k-th element of type T packed in 32-bit words
template <typename T> __device__ __forceinline__ T unpack(const uint32_t *w, int k)
{
    if constexpr (sizeof(T) == 1) return (T)((w[k >> 2] >> (8 * (k & 3))) & 0xffu);
    else if constexpr (sizeof(T) == 2) return (T)((w[k >> 1] >> (16 * (k & 1))) & 0xffffu);
    else return __uint_as_float(w[k]);
}

// the B elements of a brick row from an aligned address, as 32-bit words
template <typename T, int B>
__device__ __forceinline__ void vote_core(const T *p, T *v)
{
    constexpr int WORDS = B * (int)sizeof(T) / 4;
    uint32_t w[WORDS];
    if constexpr (WORDS == 1) {
        w[0] = __ldg(reinterpret_cast<const uint32_t *>(p));
    } else if constexpr (WORDS == 2) {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = a.x, w[1] = a.y;
    } else {
#pragma unroll
        for (int j = 0; j < WORDS / 4; ++j) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p) + j);
            w[4 * j] = a.x, w[4 * j + 1] = a.y, w[4 * j + 2] = a.z, w[4 * j + 3] = a.w;
        }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = unpack<T>(w, k);
}

template <typename T> __device__ __forceinline__ T vmin(T a, T b) { return b < a ? b : a; }
template <typename T> __device__ __forceinline__ T vmax(T a, T b) { return b > a ? b : a; }

__device__ __forceinline__ bool range_visible(float mn, float mx, const int *__restrict__ prefix,
                                              int nt, float value_lo, float s, float xmax)
{
    const int lo = (int)tf_coord(mn, value_lo, s, xmax);
    int hi = (int)tf_coord(mx, value_lo, s, xmax) + 1;
    hi = hi > nt - 1 ? nt - 1 : hi;
    return (__ldg(prefix + hi + 1) - __ldg(prefix + lo)) > 0;
}

// Staged form of the same vote for bricks of B = 4 or 8 voxels in rows of
// whole bricks (nx a multiple of B), one warp per marked brick: the warp
// first copies the brick's (B+2)^2 voxel rows x = bB-1 .. (b+1)B (clamped as
// above; the brick's B voxels as one aligned vector load, the two apron voxels
// singly) into its shared-memory stage, one row per lane, so that every row
// crosses the memory hierarchy once; then lane r takes cell row r (cells cy,
// cz fixed, cx = bB-1 .. (b+1)B-1), keeps the column minima and maxima of
// its four corner rows, and cell cx ranges over columns cx and cx+1.  The
// range test of the row's whole range runs first: every cell range lies
// inside it, so a row that fails has no positive cell; the cells of a row
// that passes are tested in order up to the first positive one.  A brick's
// (B+1)^2 cell rows take at most three rounds of 32.  (Two earlier forms,
// cells 32 at a time straight from global memory and cell rows straight from
// global memory, both took about 0.10 ms per 512^3 edit; the stage and the
// cheaper index arithmetic below take about 0.094 ms, and 0.079 ms with the
// two-block row loads of 8-bit voxels.)
// A warp's stage: the brick's (B+2)^2 voxel rows of B+2 values, each row
// padded to whole 16-byte words.
template <typename T, int B> struct VoteStage {
    static constexpr int NV = B + 2;
    static constexpr int VEC = (NV * (int)sizeof(T) + 15) / 16;  // 16-byte words per row
    static constexpr int RSB = 16 * VEC;
    static constexpr int ROWS = NV * NV;
    static constexpr int ITER = (ROWS + 31) / 32;
    static constexpr int WARP_BYTES = ROWS * RSB;
};

template <typename T> __device__ __forceinline__ uint32_t bits_of(T v)
{
    if constexpr (sizeof(T) == 4) return __float_as_uint(v);
    else return (uint32_t)v;
}

template <typename T, int B>
__device__ __forceinline__ void sts_row(unsigned char *p, const T *v)
{
    using S = VoteStage<T, B>;
    uint32_t w[4 * S::VEC];
#pragma unroll
    for (int j = 0; j < 4 * S::VEC; ++j) w[j] = 0;
#pragma unroll
    for (int k = 0; k < S::NV; ++k) {
        const int byte = k * (int)sizeof(T);
        w[byte >> 2] |= bits_of(v[k]) << (8 * (byte & 3));
    }
#pragma unroll
    for (int j = 0; j < S::VEC; ++j)
        *reinterpret_cast<uint4 *>(p + 16 * j) = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2],
                                                            w[4 * j + 3]);
}

template <typename T, int B>
__device__ __forceinline__ void lds_row(const unsigned char *p, T *v)
{
    using S = VoteStage<T, B>;
    uint32_t w[4 * S::VEC];
#pragma unroll
    for (int j = 0; j < S::VEC; ++j) {
        const uint4 a = *reinterpret_cast<const uint4 *>(p + 16 * j);
        w[4 * j] = a.x, w[4 * j + 1] = a.y, w[4 * j + 2] = a.z, w[4 * j + 3] = a.w;
    }
#pragma unroll
    for (int k = 0; k < S::NV; ++k) v[k] = unpack<T>(w, k);
}

template <typename T, int B>
__global__ void __launch_bounds__(256, 2) k_vote_staged(const T *__restrict__ vol, int nx, int ny,
                                                   int nz, int gx, int gy, int64_t nb,
                                                   const int *__restrict__ prefix, int nt,
                                                   float value_lo, float s,
                                                   uint8_t *__restrict__ mask, bool rows16)
{
    using S = VoteStage<T, B>;
    constexpr int NV = S::NV, RSB = S::RSB;
    __shared__ __align__(16) unsigned char stage[8][S::WARP_BYTES];
    const int lane = threadIdx.x & 31;
    unsigned char *sw = stage[threadIdx.x >> 5];
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float xmax = (float)(nt - 1);
    // the warp's bricks are w, w + W, w + 2W, ...: 32 mask bytes per ballot
    for (int64_t k0 = 0; w + k0 * W < nb; k0 += 32) {
        const int64_t bl = w + (k0 + lane) * W;
        unsigned marked = __ballot_sync(0xffffffffu, bl < nb && mask[bl] != 0);
        while (marked) {  // uniform
            const int k = __ffs(marked) - 1;
            marked &= marked - 1;
            const int64_t b = w + (k0 + k) * W;
            // nb < 2^31 (the launcher checks it): 32-bit index arithmetic
            const unsigned ub = (unsigned)b, urow = ub / (unsigned)gx;
            const int bx = (int)(ub - urow * (unsigned)gx);
            const int bz = (int)(urow / (unsigned)gy), by = (int)(urow - (unsigned)bz * (unsigned)gy);
            const int x0 = bx * B;  // the brick's first voxel; x0 + B <= nx
            const int ly = by * B - 1, lz = bz * B - 1;
            const int ey = min((by + 1) * B, ny) - ly, ez = min((bz + 1) * B, nz) - lz;
            const int ry = ey + 1, nvr = ry * (ez + 1);  // voxel rows ly .. ly + ey, lz .. lz + ez
            // q / ry and r / ey for q, r < 128 and divisors up to B + 2 <= 10:
            // (q + 0.5) / d lies at least 0.5 / d from an integer, far above the
            // rounding error of the float product
            const float inv_ry = 1.0f / (float)ry, inv_ey = 1.0f / (float)ey;
            const bool has_l = x0 > 0, has_r = x0 + B < nx;
            // stage the brick's voxel rows (clamped to the volume), one per lane
#pragma unroll
            for (int it = 0; it < S::ITER; ++it) {
                const int q = lane + 32 * it;
                if (q < nvr) {
                    const int qz = (int)(((float)q + 0.5f) * inv_ry), qy = q - qz * ry;
                    const int y = min(max(ly + qy, 0), ny - 1);
                    const int z = min(max(lz + qz, 0), nz - 1);
                    const T *row = vol + ((size_t)z * ny + y) * (size_t)nx + x0;
                    if constexpr (sizeof(T) == 1 && B == 8) {
                        if (rows16) {
                            // x0 - 1 .. x0 + 8 lie in two aligned 16-byte blocks of
                            // the row: [x0 - 8, x0 + 8) and [x0 + 8, x0 + 24) when x0
                            // is 8 mod 16, else [x0 - 16, x0) and [x0, x0 + 16)
                            const bool odd = (x0 & 8) != 0;  // odd implies x0 >= 8
                            uint4 A = make_uint4(0u, 0u, 0u, 0u), C = A;
                            if (has_l) A = __ldg(reinterpret_cast<const uint4 *>(row - (odd ? 8 : 16)));
                            if (!odd || has_r) C = __ldg(reinterpret_cast<const uint4 *>(row + (odd ? 8 : 0)));
                            const uint32_t c0 = odd ? A.z : C.x, c1 = odd ? A.w : C.y;
                            const uint32_t left = has_l ? ((odd ? A.y : A.w) >> 24) : (c0 & 0xffu);
                            const uint32_t right = has_r ? ((odd ? C.x : C.z) & 0xffu) : (c1 >> 24);
                            // the stage row: left, the 8 brick voxels, right
                            *reinterpret_cast<uint4 *>(sw + q * RSB) =
                                make_uint4((c0 << 8) | left, __funnelshift_l(c0, c1, 8),
                                           (c1 >> 24) | (right << 8), 0u);
                            continue;
                        }
                    }
                    T core[B], v[NV];
                    vote_core<T, B>(row, core);
#pragma unroll
                    for (int i = 0; i < B; ++i) v[i + 1] = core[i];
                    v[0] = has_l ? __ldg(row - 1) : v[1];
                    v[NV - 1] = has_r ? __ldg(row + B) : v[NV - 2];
                    sts_row<T, B>(sw + q * RSB, v);
                }
            }
            __syncwarp();
            const int nrow = ey * ez;
            bool found = false;
            for (int base = 0; base < nrow && !found; base += 32) {  // uniform
                const int r = base + lane;
                bool pos = false;
                if (r < nrow) {
                    // cell row (ly + a, lz + c): voxel rows a, a + 1 of planes c, c + 1
                    const int c = (int)(((float)r + 0.5f) * inv_ey), a = r - c * ey;
                    const unsigned char *p0 = sw + (c * ry + a) * RSB;
                    T cmn[NV], cmx[NV];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        T v[NV];
                        lds_row<T, B>(p0 + ((q & 1) + (q >> 1) * ry) * RSB, v);
#pragma unroll
                        for (int i = 0; i < NV; ++i) {
                            cmn[i] = q == 0 ? v[i] : vmin(cmn[i], v[i]);
                            cmx[i] = q == 0 ? v[i] : vmax(cmx[i], v[i]);
                        }
                    }
                    T rmn = cmn[0], rmx = cmx[0];
#pragma unroll
                    for (int i = 1; i < NV; ++i) rmn = vmin(rmn, cmn[i]), rmx = vmax(rmx, cmx[i]);
                    if (range_visible(to_f(rmn), to_f(rmx), prefix, nt, value_lo, s, xmax)) {
#pragma unroll
                        for (int i = 0; i < NV - 1; ++i)
                            if (!pos)
                                pos = range_visible(to_f(vmin(cmn[i], cmn[i + 1])),
                                                    to_f(vmax(cmx[i], cmx[i + 1])), prefix, nt,
                                                    value_lo, s, xmax);
                    }
                }
                found = __any_sync(0xffffffffu, pos);
            }
            __syncwarp();  // the stage is read before the next brick overwrites it
            if (!found && lane == 0) mask[b] = 0;
        }
    }
}

void launch_vote_bricks(Ctx &c, const Volume &v, int B, const TF &tf, float s, uint8_t *mask,
                        int gx, int gy, int gz)
{
    int sms = 0;
    ESS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    const int64_t nb = (int64_t)gx * gy * gz;
    const int blocks = (int)std::min<int64_t>((int64_t)sms * 8, (nb + 7) / 8);
    Launch L(c, "vote_bricks");
    // rows of whole bricks whose brick part is an aligned vector: the staged
    // kernel (32-bit brick indices)
    const size_t es = v.dtype == ESS_U8 ? 1 : (v.dtype == ESS_U16 ? 2 : 4);
    const size_t core = (size_t)B * es, al = core < 16 ? core : 16;
    if ((B == 4 || B == 8) && v.nx % B == 0 && ((uintptr_t)v.data % al) == 0 &&
        nb < ((int64_t)1 << 31)) {
#define ESS_VOTE_STAGED(T, BB)                                                                 \
    k_vote_staged<T, BB><<<blocks, 256, 0, c.stream>>>((const T *)v.data, v.nx, v.ny, v.nz, gx, \
                                                       gy, nb, tf.prefix, tf.nt, v.value_lo, s, \
                                                       mask, v.nx % 16 == 0)
        if (B == 8) {
            if (v.dtype == ESS_U8) ESS_VOTE_STAGED(uint8_t, 8);
            else if (v.dtype == ESS_U16) ESS_VOTE_STAGED(uint16_t, 8);
            else ESS_VOTE_STAGED(float, 8);
        } else {
            if (v.dtype == ESS_U8) ESS_VOTE_STAGED(uint8_t, 4);
            else if (v.dtype == ESS_U16) ESS_VOTE_STAGED(uint16_t, 4);
            else ESS_VOTE_STAGED(float, 4);
        }
#undef ESS_VOTE_STAGED
        return;
    }
    switch (v.dtype) {
    case ESS_U8:
        k_vote_bricks<uint8_t><<<blocks, 256, 0, c.stream>>>((const uint8_t *)v.data, v.nx, v.ny,
                                                             v.nz, B, gx, gy, nb, tf.prefix,
                                                             tf.nt, v.value_lo, s, mask);
        break;
    case ESS_U16:
        k_vote_bricks<uint16_t><<<blocks, 256, 0, c.stream>>>((const uint16_t *)v.data, v.nx, v.ny,
                                                              v.nz, B, gx, gy, nb, tf.prefix,
                                                              tf.nt, v.value_lo, s, mask);
        break;
    default:
        k_vote_bricks<float><<<blocks, 256, 0, c.stream>>>((const float *)v.data, v.nx, v.ny, v.nz,
                                                           B, gx, gy, nb, tf.prefix, tf.nt,
                                                           v.value_lo, s, mask);
    }
}

// ------------------------------------------------------------ K3 compaction
// Three passes over the byte mask: per-tile counts, one-block scan of the
// tile counts (also the total), per-tile scatter with a block-local scan, so
// the ids come out in ascending order.  A tile is 256 threads x 16 flags,
// each thread reading its flags as one 16-byte vector (the mask buffer is
// padded to whole tiles and zero-filled).
constexpr int CT_THREADS = 256;
constexpr int CT_ITEMS = 16;
constexpr int CT_TILE = CT_THREADS * CT_ITEMS;

size_t compact_block_count(int64_t nb) { return (size_t)((nb + CT_TILE - 1) / CT_TILE); }

__device__ __forceinline__ int popc_bytes(uint4 v)
{
    // each byte is 0 or 1
    uint32_t s = v.x + v.y + v.z + v.w;  // per-byte sums stay < 256
    return (int)((s & 0xffu) + ((s >> 8) & 0xffu) + ((s >> 16) & 0xffu) + (s >> 24));
}

template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int &total)
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

__global__ void __launch_bounds__(CT_THREADS) k_compact_count(const uint8_t *__restrict__ mask,
                                                              uint32_t *__restrict__ block_sums)
{
    const uint4 *m = reinterpret_cast<const uint4 *>(mask) + (size_t)blockIdx.x * CT_THREADS;
    int c = popc_bytes(m[threadIdx.x]);
    int total;
    block_excl_scan<CT_THREADS>(c, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = (uint32_t)total;
}

// exclusive scan of nblk tile counts in one block of 1024 threads
__global__ void __launch_bounds__(1024) k_compact_scan(uint32_t *__restrict__ block_sums,
                                                       int nblk, int *__restrict__ count)
{
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < nblk ? (int)block_sums[i] : 0;
        int total;
        int ex = block_excl_scan<1024>(v, total);
        if (i < nblk) block_sums[i] = (uint32_t)(carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

// 30-bit Morton code (Sec. 3.1), bit i of x/y/z at bit 3i/3i+1/3i+2: each
// 10-bit coordinate is spread to every third bit by shift-and-mask steps.
__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(CT_THREADS) k_compact_scatter(const uint8_t *__restrict__ mask,
                                                                const uint32_t *__restrict__ block_sums,
                                                                int64_t nb, uint32_t *__restrict__ ids,
                                                                uint32_t *__restrict__ keys, int gx,
                                                                int gy)
{
    const uint4 *m = reinterpret_cast<const uint4 *>(mask) + (size_t)blockIdx.x * CT_THREADS;
    uint4 v = m[threadIdx.x];
    int c = popc_bytes(v);
    int total;
    int off = block_excl_scan<CT_THREADS>(c, total) + (int)block_sums[blockIdx.x];
    if (c == 0) return;
    int64_t first = (int64_t)blockIdx.x * CT_TILE + (int64_t)threadIdx.x * CT_ITEMS;
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < CT_ITEMS; ++j) {
        if ((w[j >> 2] >> (8 * (j & 3))) & 0xffu) {
            int64_t b = first + j;
            if (b < nb) {
                ids[off] = (uint32_t)b;
                if (keys) {
                    uint32_t bx = (uint32_t)(b % gx), by = (uint32_t)((b / gx) % gy);
                    uint32_t bz = (uint32_t)(b / ((int64_t)gx * gy));
                    keys[off] = spread3(bx) | (spread3(by) << 1) | (spread3(bz) << 2);
                }
            }
            ++off;
        }
    }
}

void launch_compact(Ctx &c, const uint8_t *mask, int64_t nb, uint32_t *ids, int *count,
                    uint32_t *block_sums, uint32_t *morton_keys, int gx, int gy)
{
    unsigned nblk = (unsigned)compact_block_count(nb);
    {
        Launch L(c, "compact_count");
        k_compact_count<<<nblk, CT_THREADS, 0, c.stream>>>(mask, block_sums);
    }
    {
        Launch L(c, "compact_scan");
        k_compact_scan<<<1, 1024, 0, c.stream>>>(block_sums, (int)nblk, count);
    }
    {
        Launch L(c, "compact_scatter");
        k_compact_scatter<<<nblk, CT_THREADS, 0, c.stream>>>(mask, block_sums, nb, ids,
                                                             morton_keys, gx, gy);
    }
}

}  // namespace ess
