// minmax_tma.cu -- K1, the per-brick apron min/max (R3: brick b of edge B
// reads voxels bB-1 .. (b+1)B per axis, clamped to the volume), with the
// voxels staged by the Tensor Memory Accelerator.
//
// The paper classifies every brick from its voxels after each TF edit
// (Sec. 3.1), so this is the one pass over the whole volume per edit; it is
// bound by HBM bandwidth.  Design:
//
// * A tile is (x chunk of XC voxels = 256 bytes of a row, BR consecutive
//   brick rows in y, one brick slab in z).  Its voxels are the box
//   x0 .. x0+XC-1, rows by0*B-1 .. (by0+BR)*B, planes bz*B-1 .. (bz+1)*B: the
//   B+2 planes are loaded ZS planes per stage by three bulk tensor copies
//   (cp.async.bulk.tensor.3d) into a ring of shared-memory stages completed
//   by mbarriers: the chunk's rows, and the 16-byte column blocks just left
//   and right of the chunk (the x apron).  Out-of-volume parts of a box
//   arrive as zeros and are never read: rows, planes and columns are clamped
//   exactly as R3 clamps them.
// * Warp g of the CTA takes brick row g; its lane (h, c) owns the 16 bytes c
//   of the brick row's rows of parity h: it keeps column-wise minima and
//   maxima over them for every plane of the tile (8-bit voxels as f16x2
//   pairs, two columns per instruction), and the two parities merge by one
//   shuffle at the tile's end, so a tile's rows are read from shared memory
//   once.
// * At the tile's end the x reduction runs once per brick: neighbouring
//   column blocks come from the neighbouring lanes by shuffles, the chunk's
//   apron columns from the apron copies.
// * CTAs are persistent (as many as fit on the machine) and take tiles from
//   a device counter, x-fastest, so that the work stays balanced and the
//   neighbouring chunks, rows and slabs whose apron voxels a tile re-reads
//   are loaded by other CTAs at about the same time and come from L2: the
//   volume crosses HBM about once.
// * Every wait on an mbarrier is bounded in time; a wait that gives up sets
//   DEV_ERR_TIMEOUT in the status word, waits (bounded) for the CTA's copies
//   still in flight and leaves its tiles unwritten.
#include <cuda.h>  // CUtensorMap and its enums (types only)
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "ess_internal.h"

namespace ess {

namespace {

__device__ __forceinline__ uint32_t tma_min_h2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t tma_max_h2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// two 16-bit unsigned lanes per word
__device__ __forceinline__ uint32_t tma_min_u2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t tma_max_u2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Column-wise min/max of the 16-byte blocks of one column block over rows.
template <typename T> struct Cols;
template <> struct Cols<uint8_t> {
    // byte b under the high byte 0x64 is the half 1024 + b, ordered as b:
    // word i gives the pairs (b0, b1) and (b2, b3) = columns 4i.. 4i+3
    uint32_t mna[4], mnb[4], mxa[4], mxb[4];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) mna[i] = mnb[i] = 0x64ff64ffu, mxa[i] = mxb[i] = 0x64006400u;
    }
    __device__ __forceinline__ void add(const uint4 &w)
    {
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t a = __byte_perm(q[i], 0x64646464u, 0x4140);
            const uint32_t b = __byte_perm(q[i], 0x64646464u, 0x4342);
            mna[i] = tma_min_h2(mna[i], a);
            mnb[i] = tma_min_h2(mnb[i], b);
            mxa[i] = tma_max_h2(mxa[i], a);
            mxb[i] = tma_max_h2(mxb[i], b);
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
    // merge with lane ^ o of the warp
    __device__ __forceinline__ void shfl_merge(int o)
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            mna[i] = tma_min_h2(mna[i], __shfl_xor_sync(0xffffffffu, mna[i], o));
            mnb[i] = tma_min_h2(mnb[i], __shfl_xor_sync(0xffffffffu, mnb[i], o));
            mxa[i] = tma_max_h2(mxa[i], __shfl_xor_sync(0xffffffffu, mxa[i], o));
            mxb[i] = tma_max_h2(mxb[i], __shfl_xor_sync(0xffffffffu, mxb[i], o));
        }
    }
};
template <> struct Cols<uint16_t> {
    // word i holds columns 2i (low half) and 2i+1 (high half), as the voxels
    // lie in the row: one min.u16x2 and one max.u16x2 per two voxels
    uint32_t mn[4], mx[4];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) mn[i] = 0xffffffffu, mx[i] = 0u;
    }
    __device__ __forceinline__ void add(const uint4 &w)
    {
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) mn[i] = tma_min_u2(mn[i], q[i]), mx[i] = tma_max_u2(mx[i], q[i]);
    }
    __device__ __forceinline__ void columns(float *cmn, float *cmx) const
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cmn[2 * i] = (float)(mn[i] & 0xffffu), cmn[2 * i + 1] = (float)(mn[i] >> 16);
            cmx[2 * i] = (float)(mx[i] & 0xffffu), cmx[2 * i + 1] = (float)(mx[i] >> 16);
        }
    }
    __device__ __forceinline__ void shfl_merge(int o)
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            mn[i] = tma_min_u2(mn[i], __shfl_xor_sync(0xffffffffu, mn[i], o));
            mx[i] = tma_max_u2(mx[i], __shfl_xor_sync(0xffffffffu, mx[i], o));
        }
    }
};
template <> struct Cols<float> {
    float mn[4], mx[4];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int j = 0; j < 4; ++j) mn[j] = INFINITY, mx[j] = -INFINITY;
    }
    __device__ __forceinline__ void add(const uint4 &w)
    {
        const float q[4] = {__uint_as_float(w.x), __uint_as_float(w.y), __uint_as_float(w.z),
                            __uint_as_float(w.w)};
#pragma unroll
        for (int j = 0; j < 4; ++j) mn[j] = fminf(q[j], mn[j]), mx[j] = fmaxf(q[j], mx[j]);
    }
    __device__ __forceinline__ void columns(float *cmn, float *cmx) const
    {
#pragma unroll
        for (int j = 0; j < 4; ++j) cmn[j] = mn[j], cmx[j] = mx[j];
    }
    __device__ __forceinline__ void shfl_merge(int o)
    {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            mn[j] = fminf(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
            mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
        }
    }
};

// Min/max of the apron columns: per lane one running value over the apron
// rows it reads, reduced at a tile's end within each half-warp (half 0: the
// column left of the chunk, half 1: right of it).  `last` picks the 16-byte
// block's last voxel (from the 32-bit word holding it) instead of its first.
template <typename T> struct Apron {
    float mn, mx;
    __device__ __forceinline__ void init() { mn = INFINITY, mx = -INFINITY; }
    __device__ __forceinline__ void add(uint32_t w, bool last)
    {
        float v;
        if (sizeof(T) == 1) v = (float)(last ? w >> 24 : w & 0xffu);
        else if (sizeof(T) == 2) v = (float)(last ? w >> 16 : w & 0xffffu);
        else v = __uint_as_float(w);
        mn = fminf(v, mn), mx = fmaxf(v, mx);
    }
    // all lanes receive both sides' values
    __device__ __forceinline__ void reduce(float &lmn, float &lmx, float &rmn, float &rmx) const
    {
        float a = mn, b = mx;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        lmn = __shfl_sync(0xffffffffu, a, 0), lmx = __shfl_sync(0xffffffffu, b, 0);
        rmn = __shfl_sync(0xffffffffu, a, 16), rmx = __shfl_sync(0xffffffffu, b, 16);
    }
};

// Tile and pipeline shape for element size ES and brick size B.
//   XC: chunk width in voxels (rows of 256 bytes); CPR = 16 column blocks
//   of 16 bytes per row; BR: brick rows per tile, one warp each (a power of
//   two, rows BR*B + 2 <= 256, the copy engine's box limit), plus one warp
//   that issues the copies; ZS: planes per stage (up to 40 KiB); NS: ring
//   stages (4 up to 24 KiB stages, else 2: two CTAs per SM).
template <int ES, int B> struct TmaShape {
    static constexpr int VPL = 16 / ES;
    static constexpr int XC = 256 / ES;
    static constexpr int RB = 256;  // bytes of a chunk row
    static constexpr int CPR = 16;
    static constexpr int BR = (254 / B) >= 8 ? 8 : ((254 / B) >= 4 ? 4 : ((254 / B) >= 2 ? 2 : 1));
    static constexpr int THREADS = (BR + 1) * 32;  // BR consumer warps + one producer warp
    static constexpr int ROWS = BR * B + 2;
    static constexpr int PLANE = ROWS * (RB + 32);
    static constexpr int ZS0 = 40960 / PLANE;
    static constexpr int ZS = ZS0 < 1 ? 1 : (ZS0 > B + 2 ? B + 2 : ZS0);
    static constexpr int SPT = (B + 2 + ZS - 1) / ZS;  // stages per tile
    static constexpr int MAIN = ZS * ROWS * RB;       // bytes of the chunk copy of a stage
    static constexpr int APRON = ZS * ROWS * 16;      // bytes of one apron copy
    static constexpr int MAIN_AL = (MAIN + 127) / 128 * 128;
    static constexpr int APRON_AL = (APRON + 127) / 128 * 128;
    static constexpr int STAGE = MAIN_AL + 2 * APRON_AL;
    static constexpr int NS = STAGE <= 24576 ? 4 : 2;
    static constexpr int SMEM = NS * STAGE;
    static constexpr uint32_t TX = MAIN + 2 * APRON;
    static_assert(ROWS <= 256, "a copy box has at most 256 rows");
};

// Waits are bounded in time (about 2 s at the GB300's clock), not in polls.
constexpr long long TMA_WAIT_CYCLES = 4000000000ll;

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > TMA_WAIT_CYCLES) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ uint32_t lds32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ uint4 lds128(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}

template <typename T, int B>
__global__ void __launch_bounds__(TmaShape<sizeof(T), B>::THREADS)
    k_brick_minmax_tma(const __grid_constant__ CUtensorMap chunk_map,
                       const __grid_constant__ CUtensorMap apron_map, int nx, int ny, int nz,
                       int gx, int gy, int nchunk, int nbrow, int ntiles, int *tile_counter,
                       float2 *__restrict__ out, uint32_t *status)
{
    using S = TmaShape<sizeof(T), B>;
    constexpr int VPL = S::VPL, XC = S::XC, CPR = S::CPR, BR = S::BR, ROWS = S::ROWS;
    constexpr int ZS = S::ZS, SPT = S::SPT, NS = S::NS, RB = S::RB;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[NS];   // copies of the slot landed (producer's arrival + bytes)
    __shared__ __align__(8) uint64_t empty[NS];  // every consumer warp is done with the slot
    __shared__ int s_tile[NS];                   // tile of the stage in each slot, -1: no more tiles

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t fbase = (uint32_t)__cvta_generic_to_shared(full);
    const uint32_t ebase = (uint32_t)__cvta_generic_to_shared(empty);

    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fbase + 8u * k) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ebase + 8u * k), "r"(BR)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();  // the only CTA-wide barrier

    if (warp == BR) {
        // ---- producer: lane 0 takes tiles from the counter and issues the
        // copies of each stage into the next free slot
        if (lane != 0) return;
        int cur = -1;
        bool ok = true;
        int q = 0;
        for (;; ++q) {
            const int slot = q % NS, s = q % SPT;
            if (q >= NS && !mbar_wait(ebase + 8u * slot, (uint32_t)((q / NS - 1) & 1))) {
                ok = false;
                break;
            }
            if (s == 0) {
                cur = atomicAdd(tile_counter, 1);
                if (cur >= ntiles) cur = -1;
            }
            s_tile[slot] = cur;
            const uint32_t bar = fbase + 8u * slot;
            if (cur < 0) {
                mbar_arrive(bar);  // releases the consumers, who read -1 and stop
                break;
            }
            const int chunk = cur % nchunk, rest = cur / nchunk;
            const int brow = rest % nbrow, bz = rest / nbrow;
            const uint32_t dst = sbase + (uint32_t)(slot * S::STAGE);
            const int x0 = chunk * XC, y = brow * BR * B - 1, z = bz * B - 1 + s * ZS;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(S::TX)
                         : "memory");
            tma_load3(dst, &chunk_map, x0, y, z, bar);
            tma_load3(dst + S::MAIN_AL, &apron_map, x0 - VPL, y, z, bar);
            tma_load3(dst + S::MAIN_AL + S::APRON_AL, &apron_map, x0 + XC, y, z, bar);
        }
        if (!ok) {
            // a consumer warp stopped: wait (bounded) for the copies still in
            // flight (stages q - NS .. q - 1) so that none lands after the CTA
            // has left
            atomicOr(status, DEV_ERR_TIMEOUT);
            for (int k = q - NS; k < q; ++k)
                if (k >= 0) mbar_wait(fbase + 8u * (k % NS), (uint32_t)((k / NS) & 1));
        }
        return;
    }

    // ---- consumer warp g = brick row g of the tile; lane (h, c) owns the
    // 16 bytes c of the rows of parity h.  The apron columns (x0 - 1 and
    // x0 + XC) go to separate accumulators, once per plane: half-warp h takes
    // side h (0 left, 1 right), lane c its rows c, c + 16, ...
    const int g = warp, c = lane & 15, h = lane >> 4;
    Cols<T> acc;
    acc.init();
    Apron<T> ap;
    ap.init();
    for (int q = 0;; ++q) {
        const int slot = q % NS;
        // (the warp leaves together: its shuffles need every lane)
        if (!__all_sync(0xffffffffu, mbar_wait(fbase + 8u * slot, (uint32_t)((q / NS) & 1)))) {
            if (lane == 0) atomicOr(status, DEV_ERR_TIMEOUT);
            break;  // the producer's wait on this warp gives up in turn
        }
        const int tile = s_tile[slot];
        if (tile < 0) break;  // uniform
        const int chunk = tile % nchunk, rest = tile / nchunk;
        const int brow = rest % nbrow, bz = rest / nbrow;
        const int s = q % SPT;
        const int x0 = chunk * XC;
        const int yb = (brow * BR + g) * B - 1;  // first row of this brick row
        const bool side_on = h == 0 ? chunk > 0 : x0 + XC < nx;
        const uint32_t st = sbase + (uint32_t)(slot * S::STAGE);
        // rows of this brick row inside the volume (y = yb + r)
        const int r0 = yb < 0 ? -yb : 0, r1 = min(B + 1, ny - 1 - yb);
        const bool all_rows = r0 == 0 && r1 == B + 1;  // uniform
#pragma unroll
        for (int p = 0; p < ZS; ++p) {
            const int zr = s * ZS + p;  // plane of the tile, 0 .. B+1
            const int z = bz * B - 1 + zr;
            if (zr <= B + 1 && z >= 0 && z < nz) {
                const uint32_t plane = st + (uint32_t)(p * ROWS + g * B) * RB + 16u * c;
                if (all_rows) {
#pragma unroll
                    for (int r = h; r < B + 2; r += 2) acc.add(lds128(plane + (uint32_t)r * RB));
                } else {
#pragma unroll
                    for (int r = h; r < B + 2; r += 2)
                        if (r >= r0 && r <= r1) acc.add(lds128(plane + (uint32_t)r * RB));
                }
                if (side_on) {
                    // the apron copy of side h: 16 bytes per row; left takes
                    // the block's last voxel, right its first
                    const uint32_t apl = st + S::MAIN_AL + (uint32_t)h * S::APRON_AL +
                                         (uint32_t)(p * ROWS + g * B) * 16u + (h == 0 ? 12u : 0u);
                    for (int r = c; r < B + 2; r += 16)
                        if (r >= r0 && r <= r1) ap.add(lds32(apl + 16u * r), h == 0);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(ebase + 8u * slot);  // this warp is done with the slot
        if (s != SPT - 1) continue;

        // ---- the tile's last stage: merge the row parities, x reduction and
        // output for brick row g (lanes of parity 1 hold the same values and
        // write nothing)
        float emn_l, emx_l, emn_r, emx_r;  // the apron columns left and right
        ap.reduce(emn_l, emx_l, emn_r, emx_r);
        ap.init();
        acc.shfl_merge(16);
        const int by = brow * BR + g;
        float cmn[VPL], cmx[VPL];
        acc.columns(cmn, cmx);

        acc.init();
        const int xb = x0 + c * VPL;            // first column of this block
        const bool have = xb < nx;              // nx is a multiple of VPL
        const bool has_right = xb + VPL < nx;   // the column right of the block exists
        // the columns left and right of the block (clamped to the volume)
        float amn = __shfl_up_sync(0xffffffffu, cmn[VPL - 1], 1, CPR);
        float amx = __shfl_up_sync(0xffffffffu, cmx[VPL - 1], 1, CPR);
        float bmn = __shfl_down_sync(0xffffffffu, cmn[0], 1, CPR);
        float bmx = __shfl_down_sync(0xffffffffu, cmx[0], 1, CPR);
        if (c == 0) {
            amn = chunk > 0 ? emn_l : cmn[0];  // x = 0 clamps to itself
            amx = chunk > 0 ? emx_l : cmx[0];
        }
        if (!has_right) {
            bmn = cmn[VPL - 1];  // x = nx - 1 clamps to itself
            bmx = cmx[VPL - 1];
        } else if (c == CPR - 1) {
            bmn = emn_r;
            bmx = emx_r;
        }
        const bool row_ok = by < gy && h == 0;
        float2 *orow = out + ((size_t)bz * gy + by) * gx;
        if constexpr (B <= VPL) {
            constexpr int PER = VPL / B;
            if (have && row_ok) {
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int bx = xb / B + k;
                    float m0 = k == 0 ? amn : cmn[k * B - 1];
                    float m1 = k == 0 ? amx : cmx[k * B - 1];
                    // right apron: the next block's first column, or the next
                    // brick's first column inside this block
                    const bool last_here = k == PER - 1;
                    const float e0 = last_here ? bmn : cmn[(k + 1) * B];
                    const float e1 = last_here ? bmx : cmx[(k + 1) * B];
                    m0 = e0 < m0 ? e0 : m0;
                    m1 = e1 > m1 ? e1 : m1;
#pragma unroll
                    for (int j = 0; j < B; ++j) {
                        m0 = cmn[k * B + j] < m0 ? cmn[k * B + j] : m0;
                        m1 = cmx[k * B + j] > m1 ? cmx[k * B + j] : m1;
                    }
                    orow[bx] = make_float2(m0, m1);
                }
            }
        } else {
            constexpr int LANES = B / VPL;  // column blocks per brick, divides CPR
            float m0 = cmn[0], m1 = cmx[0];
#pragma unroll
            for (int j = 1; j < VPL; ++j) {
                m0 = cmn[j] < m0 ? cmn[j] : m0;
                m1 = cmx[j] > m1 ? cmx[j] : m1;
            }
            if (!have) {  // past the volume's end: neutral for the brick's reduction
                m0 = INFINITY;
                m1 = -INFINITY;
            } else {
                if (c % LANES == 0) {
                    m0 = amn < m0 ? amn : m0;
                    m1 = amx > m1 ? amx : m1;
                }
                if (c % LANES == LANES - 1 || !has_right) {
                    m0 = bmn < m0 ? bmn : m0;
                    m1 = bmx > m1 ? bmx : m1;
                }
            }
#pragma unroll
            for (int o = 1; o < LANES; o <<= 1) {
                const float a0 = __shfl_xor_sync(0xffffffffu, m0, o, CPR);
                const float a1 = __shfl_xor_sync(0xffffffffu, m1, o, CPR);
                m0 = a0 < m0 ? a0 : m0;
                m1 = a1 > m1 ? a1 : m1;
            }
            if (have && row_ok && c % LANES == 0) orow[xb / B] = make_float2(m0, m1);
        }
    }
}

// cuTensorMapEncodeTiled, found through the runtime (no link to the driver
// library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

template <typename T> constexpr CUtensorMapDataType tma_dtype()
{
    return sizeof(T) == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                          : (sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
}

template <typename T>
bool encode(CUtensorMap *m, const T *data, int nx, int ny, int nz, int bx, int by, int bz)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(T), (cuuint64_t)nx * ny * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, tma_dtype<T>(), 3, (void *)data, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int B>
bool launch_tma_b(Ctx &c, const T *data, int nx, int ny, int nz, int gx, int gy, int gz, float2 *out)
{
    using S = TmaShape<sizeof(T), B>;
    CUtensorMap chunk_map, apron_map;
    if (!encode(&chunk_map, data, nx, ny, nz, S::XC, S::ROWS, S::ZS)) return false;
    if (!encode(&apron_map, data, nx, ny, nz, S::VPL, S::ROWS, S::ZS)) return false;
    const int nchunk = (nx + S::XC - 1) / S::XC, nbrow = (gy + S::BR - 1) / S::BR;
    const int64_t ntiles = (int64_t)nchunk * nbrow * gz;
    if (ntiles > (int64_t)INT32_MAX / 2) return false;
    static int per_sm[3][4] = {};  // occupancy by element size and log2 B, found once
    int &occ = per_sm[sizeof(T) / 2][__builtin_ctz(B)];
    if (occ == 0) {
        ESS_CUDA(cudaFuncSetAttribute(k_brick_minmax_tma<T, B>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
        ESS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_brick_minmax_tma<T, B>,
                                                               S::THREADS, S::SMEM));
        if (occ < 1) occ = -1;
    }
    if (occ < 0) return false;
    int sms = 0;
    ESS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms * occ);
    int *&counter = c.tile_counters[c.stream];
    if (!counter) counter = (int *)c.alloc(sizeof(int));
    ESS_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), c.stream));
    Launch L(c, "brick_minmax");
    k_brick_minmax_tma<T, B><<<grid, S::THREADS, S::SMEM, c.stream>>>(
        chunk_map, apron_map, nx, ny, nz, gx, gy, nchunk, nbrow, (int)ntiles, counter, out,
        c.dev_status);
    return true;
}

template <typename T>
bool launch_tma_t(Ctx &c, const T *data, int nx, int ny, int nz, int B, int gx, int gy, int gz,
                  float2 *out)
{
    // the copy engine needs 16-byte aligned rows and base
    if (((size_t)nx * sizeof(T)) % 16 != 0 || ((uintptr_t)data & 15u) != 0) return false;
    switch (B) {
    case 2: return launch_tma_b<T, 2>(c, data, nx, ny, nz, gx, gy, gz, out);
    case 4: return launch_tma_b<T, 4>(c, data, nx, ny, nz, gx, gy, gz, out);
    case 8: return launch_tma_b<T, 8>(c, data, nx, ny, nz, gx, gy, gz, out);
    default: return false;
    }
}

}  // namespace

bool launch_brick_minmax_tma(Ctx &c, const Volume &v, int B, float2 *out)
{
    const int gx = (v.nx + B - 1) / B, gy = (v.ny + B - 1) / B, gz = (v.nz + B - 1) / B;
    switch (v.dtype) {
    case ESS_U8:
        return launch_tma_t(c, (const uint8_t *)v.data, v.nx, v.ny, v.nz, B, gx, gy, gz, out);
    case ESS_U16:
        return launch_tma_t(c, (const uint16_t *)v.data, v.nx, v.ny, v.nz, B, gx, gy, gz, out);
    default:
        return launch_tma_t(c, (const float *)v.data, v.nx, v.ny, v.nz, B, gx, gy, gz, out);
    }
}

}  // namespace ess
