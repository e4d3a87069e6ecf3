// render_kernels.h -- device code of the ray marchers (render.cu holds the
// rest of the description and the host side).  Included by render.cu and
// render_shaded.cu, which instantiate the plain and the shaded kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ess_internal.h"

namespace ess {

struct RArgs {
    const void *vol;
    const void *cells;   // corner-replicated cells (nullptr: dense sampling only)
    int nx, ny, nz;
    uint32_t cell_last;  // index of the last cell ((nx+1)(ny+1)(nz+1) - 1 < 2^32)
    // cell strides (y: nx+1, z: (nx+1)(ny+1)) and the index of cell (1, 1, 1),
    // so that the cell of voxel (ix, iy, iz) is iz cs_z + iy cs_y + ix + c_base
    uint32_t cs_y, cs_z, c_base;
    uint32_t c_base_m;  // c_base - 0x4b400000 (cs_z + cs_y + 1), modulo 2^32
    int dda_inc;        // host side: the grid may advance its crossings (GridWalkT<true>)
    float value_lo, s;   // TF coordinate x = (v - value_lo) * s
    const float4 *tf;    // 2 nt entries: entry i, then entry i+1 minus entry i
    int nt;
    float eye[3], u[3], v[3], w[3];
    int ortho;
    float dt, ert;
    float bg[4];
    int W, H;
    float4 *out;
    // macrocell grid / brick raster
    const uint8_t *mask;
    int B, gx, gy, gz;
    // box trees (LBVH, k-d)
    const BoxNode *nodes;
    const int32_t *root;      // ref, then the root box as 6 floats (voxels)
    const int *count;         // > 0 iff the tree is non-empty
    unsigned long long *samples;
    // second workload: gradient shading (R13) and opacity correction (R14)
    int shade, shin;          // shading on; specular exponent
    float ka, kd, ks;         // ambient, diffuse, specular weights
    float op_r;               // dt / dt_ref, or 0 (no correction)
};

struct Ray {
    float o[3], d[3], inv[3];
    bool zero[3];
    // box-tree slab tests: a finite inverse (1e30 on zero axes) and -o * sinv
    float sinv[3], noi[3];
};

struct Acc {
    float r, g, b, a;
};

// ---------------------------------------------------------------- rays (R1)
__device__ __forceinline__ void gen_ray(const RArgs &a, int x, int y, Ray &r)
{
    float sx = (float)(2 * x + 1) / (float)a.W - 1.0f;
    float sy = 1.0f - (float)(2 * y + 1) / (float)a.H;
    float dir[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (a.ortho) {
            r.o[i] = fmaf(sy, a.v[i], fmaf(sx, a.u[i], a.eye[i]));
            dir[i] = a.w[i];
        } else {
            r.o[i] = a.eye[i];
            dir[i] = fmaf(sy, a.v[i], fmaf(sx, a.u[i], a.w[i]));
        }
    }
    float len = sqrtf(fmaf(dir[2], dir[2], fmaf(dir[1], dir[1], dir[0] * dir[0])));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r.d[i] = dir[i] / len;
        r.zero[i] = !(fabsf(r.d[i]) >= 1e-30f);
        r.inv[i] = r.zero[i] ? 0.0f : 1.0f / r.d[i];
        r.sinv[i] = r.zero[i] ? 1e30f : r.inv[i];
        r.noi[i] = -(r.o[i] * r.sinv[i]);
    }
}

// Slab test against the closed box [lo, hi]; narrows [tmin, tmax].  A zero
// direction component keeps the interval iff lo <= o <= hi.
__device__ __forceinline__ void slab(const Ray &r, const float lo[3], const float hi[3],
                                     float &tmin, float &tmax)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (r.zero[a]) {
            if (r.o[a] < lo[a] || r.o[a] > hi[a]) {
                tmin = INFINITY;
                tmax = -INFINITY;
            }
            continue;
        }
        float t0 = (lo[a] - r.o[a]) * r.inv[a], t1 = (hi[a] - r.o[a]) * r.inv[a];
        float tn = t0 < t1 ? t0 : t1, tx = t0 < t1 ? t1 : t0;
        if (tn > tmin) tmin = tn;
        if (tx < tmax) tmax = tx;
    }
}

__device__ __forceinline__ float fmax3f(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmin3f(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Slab test of the box-tree traversals: plane crossings as fmaf(p, sinv,
// -o * sinv), branch-free (a zero axis has the finite inverse 1e30, so a box
// keeps the ray iff its slab contains o, up to one rounding of o * 1e30 that
// two boxes sharing the plane see alike, so at least one of them keeps it).
// It may differ from the exact test by rounding; a crossing misplaced along
// an axis moves the ray's position by a tiny fraction of a voxel, which the
// one-voxel apron of the brick min/max absorbs (a sample just outside a box
// reads only voxels that the box's range test covered), and rule S adds a
// sample at both ends of every interval.
__device__ __forceinline__ void slab_tree(const Ray &r, const float lo[3], const float hi[3],
                                          float &tmin, float &tmax)
{
    float n[3], f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t0 = fmaf(lo[a], r.sinv[a], r.noi[a]), t1 = fmaf(hi[a], r.sinv[a], r.noi[a]);
        n[a] = fminf(t0, t1);
        f[a] = fmaxf(t0, t1);
    }
    tmin = fmax3f(n[0], n[1], fmaxf(n[2], tmin));
    tmax = fmin3f(f[0], f[1], fminf(f[2], tmax));
}

// -------------------------------------------------------- sampling (R2, R5)
template <typename T> __device__ __forceinline__ float ldv(const T *p) { return (float)__ldg(p); }

__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// The 8 corner values of trilinear cell (ix, iy, iz) (i0 = floor(p - 0.5)),
// neighbours clamped to the volume, in the order 000 100 010 110 001 101 011 111.
// Dense sampling reads them from the volume (8 loads); cell sampling reads
// the copy that the cell array keeps of exactly those values (one vector
// load): cell (cx, cy, cz) = (ix + 1, iy + 1, iz + 1), 0 <= c <= n.
template <typename T, int SAMPLER> struct Corners;

template <typename T> struct Corners<T, 0> {
    static __device__ __forceinline__ void get(const RArgs &a, int ix, int iy, int iz, float v[8])
    {
        const T *vol = (const T *)a.vol;
        int x0 = min(max(ix, 0), a.nx - 1), x1 = min(max(ix + 1, 0), a.nx - 1);
        int y0 = min(max(iy, 0), a.ny - 1), y1 = min(max(iy + 1, 0), a.ny - 1);
        int z0 = min(max(iz, 0), a.nz - 1), z1 = min(max(iz + 1, 0), a.nz - 1);
        size_t r00 = (size_t)(z0 * a.ny + y0) * (size_t)a.nx, r10 = (size_t)(z0 * a.ny + y1) * (size_t)a.nx;
        size_t r01 = (size_t)(z1 * a.ny + y0) * (size_t)a.nx, r11 = (size_t)(z1 * a.ny + y1) * (size_t)a.nx;
        v[0] = ldv(vol + r00 + x0);
        v[1] = ldv(vol + r00 + x1);
        v[2] = ldv(vol + r10 + x0);
        v[3] = ldv(vol + r10 + x1);
        v[4] = ldv(vol + r01 + x0);
        v[5] = ldv(vol + r01 + x1);
        v[6] = ldv(vol + r11 + x0);
        v[7] = ldv(vol + r11 + x1);
    }
};

// Cell (ix + 1, iy + 1, iz + 1) with each coordinate clamped to [0, n], as
// the clamp-to-edge reconstruction of R2 reads it.
__device__ __forceinline__ uint32_t cell_index(const RArgs &a, int ix, int iy, int iz)
{
    int cx = min(max(ix + 1, 0), a.nx), cy = min(max(iy + 1, 0), a.ny), cz = min(max(iz + 1, 0), a.nz);
    return (uint32_t)((cz * (a.ny + 1) + cy) * (a.nx + 1) + cx);
}

// The same cell for a sample of the march, whose position lies in the volume
// box [0, n] up to rounding: t is in [t_near, t_far) of the exact slab test,
// and with camera coordinates bounded by 2^16 voxels (checked on the host)
// the rounding of t and of o + t d stays far below half a voxel, so q = p -
// 1/2 floors to -1 .. n-1 on every axis and no per-axis clamp can act.  The
// linear index is still clamped to the array, so no input can read outside
// it.
__device__ __forceinline__ uint32_t cell_index_inside(const RArgs &a, int ix, int iy, int iz)
{
    const uint32_t i = (uint32_t)iz * a.cs_z + (uint32_t)iy * a.cs_y + (uint32_t)ix + a.c_base;
    return min(i, a.cell_last);
}

// One trilinear sample (R2) in two steps: fetch() computes the position, the
// cell and the weights and loads the cell; value() unpacks the corners and
// interpolates.
template <typename T, int SAMPLER> struct CellRaw;
template <typename T> struct CellRaw<T, 0> {
    float v[8];
    template <bool INSIDE = false>
    __device__ __forceinline__ void load(const RArgs &a, int ix, int iy, int iz)
    {
        Corners<T, 0>::get(a, ix, iy, iz, v);
    }
    __device__ __forceinline__ void load_index(const RArgs &, uint32_t) {}
    __device__ __forceinline__ void corners(const RArgs &, float out[8]) const
    {
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = v[k];
    }
    // the four interpolations along x (R2: x first)
    __device__ __forceinline__ void xlerp(const RArgs &, float fx, float &c00, float &c10,
                                          float &c01, float &c11) const
    {
        c00 = lerpf(v[0], v[1], fx), c10 = lerpf(v[2], v[3], fx);
        c01 = lerpf(v[4], v[5], fx), c11 = lerpf(v[6], v[7], fx);
    }
};
template <bool INSIDE>
__device__ __forceinline__ uint32_t cell_of(const RArgs &a, int ix, int iy, int iz)
{
    return INSIDE ? cell_index_inside(a, ix, iy, iz) : cell_index(a, ix, iy, iz);
}

template <> struct CellRaw<uint8_t, 1> {
    uint2 c;
    template <bool INSIDE = false>
    __device__ __forceinline__ void load(const RArgs &a, int ix, int iy, int iz)
    {
        c = __ldg(reinterpret_cast<const uint2 *>(a.cells) + cell_of<INSIDE>(a, ix, iy, iz));
    }
    __device__ __forceinline__ void load_index(const RArgs &a, uint32_t i)
    {
        c = __ldg(reinterpret_cast<const uint2 *>(a.cells) + i);
    }
    __device__ __forceinline__ void corners(const RArgs &, float v[8]) const
    {
        // byte b under the exponent of 2^23 is the float 2^23 + b: exact
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = __int_as_float(__byte_perm(c.x, 0x4b000000u, 0x7650 | k)) - 8388608.0f;
            v[4 + k] = __int_as_float(__byte_perm(c.y, 0x4b000000u, 0x7650 | k)) - 8388608.0f;
        }
    }
    __device__ __forceinline__ void xlerp(const RArgs &a, float fx, float &c00, float &c10,
                                          float &c01, float &c11) const
    {
        float v[8];
        corners(a, v);
        c00 = lerpf(v[0], v[1], fx), c10 = lerpf(v[2], v[3], fx);
        c01 = lerpf(v[4], v[5], fx), c11 = lerpf(v[6], v[7], fx);
    }
};
template <> struct CellRaw<uint16_t, 1> {
    uint4 c;
    template <bool INSIDE = false>
    __device__ __forceinline__ void load(const RArgs &a, int ix, int iy, int iz)
    {
        c = __ldg(reinterpret_cast<const uint4 *>(a.cells) + cell_of<INSIDE>(a, ix, iy, iz));
    }
    __device__ __forceinline__ void load_index(const RArgs &a, uint32_t i)
    {
        c = __ldg(reinterpret_cast<const uint4 *>(a.cells) + i);
    }
    __device__ __forceinline__ void corners(const RArgs &, float v[8]) const
    {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __int_as_float(__byte_perm(w[k], 0x4b000000u, 0x7610)) - 8388608.0f;
            v[2 * k + 1] = __int_as_float(__byte_perm(w[k], 0x4b000000u, 0x7632)) - 8388608.0f;
        }
    }
    __device__ __forceinline__ void xlerp(const RArgs &a, float fx, float &c00, float &c10,
                                          float &c01, float &c11) const
    {
        float v[8];
        corners(a, v);
        c00 = lerpf(v[0], v[1], fx), c10 = lerpf(v[2], v[3], fx);
        c01 = lerpf(v[4], v[5], fx), c11 = lerpf(v[6], v[7], fx);
    }
};
template <> struct CellRaw<float, 1> {
    float4 c0, c1;
    template <bool INSIDE = false>
    __device__ __forceinline__ void load(const RArgs &a, int ix, int iy, int iz)
    {
        const float4 *p = reinterpret_cast<const float4 *>(a.cells) +
                          2 * (size_t)cell_of<INSIDE>(a, ix, iy, iz);
        c0 = __ldg(p);
        c1 = __ldg(p + 1);
    }
    __device__ __forceinline__ void load_index(const RArgs &a, uint32_t i)
    {
        const float4 *p = reinterpret_cast<const float4 *>(a.cells) + 2 * (size_t)i;
        c0 = __ldg(p);
        c1 = __ldg(p + 1);
    }
    __device__ __forceinline__ void corners(const RArgs &, float v[8]) const
    {
        v[0] = c0.x; v[1] = c0.y; v[2] = c0.z; v[3] = c0.w;
        v[4] = c1.x; v[5] = c1.y; v[6] = c1.z; v[7] = c1.w;
    }
    __device__ __forceinline__ void xlerp(const RArgs &a, float fx, float &c00, float &c10,
                                          float &c01, float &c11) const
    {
        float v[8];
        corners(a, v);
        c00 = lerpf(v[0], v[1], fx), c10 = lerpf(v[2], v[3], fx);
        c01 = lerpf(v[4], v[5], fx), c11 = lerpf(v[6], v[7], fx);
    }
};


template <typename T, int SAMPLER> struct SampleFetch {
    CellRaw<T, SAMPLER> raw;
    float fx, fy, fz;
    // a sample of the march (inside the volume box up to rounding)
    __device__ __forceinline__ void fetch(const RArgs &a, const Ray &r, float t)
    {
        at<true>(a, fmaf(t, r.d[0], r.o[0]), fmaf(t, r.d[1], r.o[1]), fmaf(t, r.d[2], r.o[2]));
    }
    // any position (the gradient's neighbours may lie a voxel outside)
    template <bool INSIDE = false>
    __device__ __forceinline__ void at(const RArgs &a, float px, float py, float pz)
    {
        const float qx = px - 0.5f, qy = py - 0.5f, qz = pz - 0.5f;
        if (INSIDE && SAMPLER == 1) {
            // floor by adding 1.5 * 2^23 rounded down: |q| < 2^22, so the sum
            // lies in [2^23, 2^24), where floats are the integers, and its
            // bits are 0x4b400000 + floor(q)
            const float M = 12582912.0f;
            const float sx = __fadd_rd(qx, M), sy = __fadd_rd(qy, M), sz = __fadd_rd(qz, M);
            fx = qx - (sx - M);
            fy = qy - (sy - M);
            fz = qz - (sz - M);
            const uint32_t i = (uint32_t)__float_as_int(sz) * a.cs_z +
                               (uint32_t)__float_as_int(sy) * a.cs_y +
                               (uint32_t)__float_as_int(sx) + a.c_base_m;
            raw.load_index(a, min(i, a.cell_last));
            return;
        }
        const float gxf = floorf(qx), gyf = floorf(qy), gzf = floorf(qz);
        fx = qx - gxf;
        fy = qy - gyf;
        fz = qz - gzf;
        raw.template load<INSIDE>(a, (int)gxf, (int)gyf, (int)gzf);
    }
    __device__ __forceinline__ float value(const RArgs &a) const
    {
        float c00, c10, c01, c11;
        raw.xlerp(a, fx, c00, c10, c01, c11);
        const float c0 = lerpf(c00, c10, fy), c1 = lerpf(c01, c11, fy);
        return lerpf(c0, c1, fz);
    }
};

// The lerp of R5, fmaf(w, c1 - c0, c0) per channel, with the float32
// difference c1 - c0 read from the table (entry 2 i0 + 1, computed when the TF
// was uploaded, rounded as the lerp rounds it); the last entry's difference is
// 0 (entry i1 = min(i0 + 1, nt - 1)).
__device__ __forceinline__ float4 classify(const RArgs &a, float v)
{
    float x = (v - a.value_lo) * a.s;
    float xmax = (float)(a.nt - 1);
    x = fminf(fmaxf(x, 0.0f), xmax);  // x is finite
    int i0 = (int)x;
    float w = x - (float)i0;
    float4 c0 = __ldg(a.tf + 2 * i0), d = __ldg(a.tf + 2 * i0 + 1);
    return make_float4(fmaf(w, d.x, c0.x), fmaf(w, d.y, c0.y), fmaf(w, d.z, c0.z),
                       fmaf(w, d.w, c0.w));
}

// ------------------------------------------- second workload (R13, R14)
// log2 of x in (0, 1] (normal) from ln m = 2 atanh(u) = 2 (u + u^3/3 + ...),
// u = (m - 1)/(m + 1), after splitting x = m 2^e with m in [sqrt(1/2),
// sqrt(2)]; terms to u^11.
__device__ __forceinline__ float own_log2(float x)
{
    const unsigned b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) {  // sqrt(2)
        m = m * 0.5f;
        e = e + 1;
    }
    const float u = (m - 1.0f) / (m + 1.0f);
    const float u2 = u * u;
    float q = fmaf(u2, 0x1.745d18p-3f, 0x1.c71c72p-3f);  // 2/11, 2/9
    q = fmaf(u2, q, 0x1.24924ap-2f);                      // 2/7
    q = fmaf(u2, q, 0x1.99999ap-2f);                      // 2/5
    q = fmaf(u2, q, 0x1.555556p-1f);                      // 2/3
    q = fmaf(u2, q, 2.0f);
    return fmaf(u * q, 0x1.715476p+0f, (float)e);         // log2(e)
}

// 2^y for y <= 0: 2^f = e^(f ln 2) by its Taylor series to the 10th power
// for the fraction f = y - floor(y), times 2^floor(y); 0 below 2^-126.
__device__ __forceinline__ float own_exp2(float y)
{
    if (y < -126.0f) return 0.0f;
    const float n = floorf(y);
    const float t = (y - n) * 0x1.62e430p-1f;  // ln 2
    float p = 0x1.27e4fcp-22f;                  // 1/10!
    p = fmaf(p, t, 0x1.71de3ap-19f);
    p = fmaf(p, t, 0x1.a01a02p-16f);
    p = fmaf(p, t, 0x1.a01a02p-13f);
    p = fmaf(p, t, 0x1.6c16c2p-10f);
    p = fmaf(p, t, 0x1.111112p-7f);
    p = fmaf(p, t, 0x1.555556p-5f);
    p = fmaf(p, t, 0x1.555556p-3f);
    p = fmaf(p, t, 0.5f);
    p = fmaf(p, t, 1.0f);
    p = fmaf(p, t, 1.0f);
    return p * __uint_as_float((unsigned)((int)n + 127) << 23);
}

// R14: 1 - (1 - alpha)^r for samples every dt voxels when the TF's alpha holds
// for dt_ref (r = dt / dt_ref); r = 0 or 1 leaves alpha, 0 and 1 stay fixed.
__device__ __forceinline__ float correct_alpha(float alpha, float r)
{
    // alpha 0 gives 1 - 2^(r log2 1) = 1 - 2^0 = 0 exactly: skip the series
    if (r == 0.0f || r == 1.0f || alpha == 0.0f) return alpha;
    const float om = 1.0f - alpha;
    if (om == 0.0f) return 1.0f;
    return 1.0f - own_exp2(r * own_log2(om));
}

// R13: gradient of the reconstruction by central differences one voxel apart,
// then two-sided Blinn-Phong under a headlight (light and eye along -d):
// c = min(|n . d|, 1), rgb' = rgb (ka + kd c) + ks c^shininess.  A zero
// gradient leaves the colour.
template <typename T, int SAMPLER, bool INSIDE>
__device__ __forceinline__ float value_at(const RArgs &a, float px, float py, float pz)
{
    SampleFetch<T, SAMPLER> f;
    f.template at<INSIDE>(a, px, py, pz);
    return f.value(a);
}

// Central differences one voxel apart (R13).  INSIDE: every neighbour lies in
// the volume box [0, n], so its cell needs no per-axis clamp.
template <typename T, int SAMPLER, bool INSIDE>
__device__ __forceinline__ void gradient(const RArgs &a, float px, float py, float pz, float &gx,
                                         float &gy, float &gz)
{
    gx = (value_at<T, SAMPLER, INSIDE>(a, px + 1.0f, py, pz) -
          value_at<T, SAMPLER, INSIDE>(a, px - 1.0f, py, pz)) * 0.5f;
    gy = (value_at<T, SAMPLER, INSIDE>(a, px, py + 1.0f, pz) -
          value_at<T, SAMPLER, INSIDE>(a, px, py - 1.0f, pz)) * 0.5f;
    gz = (value_at<T, SAMPLER, INSIDE>(a, px, py, pz + 1.0f) -
          value_at<T, SAMPLER, INSIDE>(a, px, py, pz - 1.0f)) * 0.5f;
}

template <typename T, int SAMPLER>
__device__ __forceinline__ void shade(const RArgs &a, const Ray &r, float t, float4 &c)
{
    const float px = fmaf(t, r.d[0], r.o[0]), py = fmaf(t, r.d[1], r.o[1]),
                pz = fmaf(t, r.d[2], r.o[2]);
    // a sample at least one voxel inside the box on every axis: p +- 1 stays
    // in [0, n] (float rounding is monotone), so the fast cell index applies
    const bool inside = px >= 1.0f && px <= (float)a.nx - 1.0f && py >= 1.0f &&
                        py <= (float)a.ny - 1.0f && pz >= 1.0f && pz <= (float)a.nz - 1.0f;
    float gx, gy, gz;
    if (inside) gradient<T, SAMPLER, true>(a, px, py, pz, gx, gy, gz);
    else gradient<T, SAMPLER, false>(a, px, py, pz, gx, gy, gz);
    const float len2 = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
    if (!(len2 > 0.0f)) return;
    const float len = sqrtf(len2);
    const float dotv = fmaf(gz, r.d[2], fmaf(gy, r.d[1], gx * r.d[0]));
    float cs = fabsf(dotv) / len;
    if (cs > 1.0f) cs = 1.0f;
    float spec = 1.0f, base = cs;
    for (int e = a.shin; e > 0; e >>= 1) {
        if (e & 1) spec = spec * base;
        if (e > 1) base = base * base;
    }
    const float lam = fmaf(a.kd, cs, a.ka), hs = a.ks * spec;
    c.x = fmaf(c.x, lam, hs);
    c.y = fmaf(c.y, lam, hs);
    c.z = fmaf(c.z, lam, hs);
}

// Classification and compositing of one sample value (R5, R6) and early
// termination (R7); true when A >= ert.  With SHADE the opacity is corrected
// (R14) and samples of non-zero opacity are shaded (R13) first.
template <typename T, int SAMPLER, int SHADE>
__device__ __forceinline__ bool composite(const RArgs &a, const Ray &r, float t, float value,
                                          Acc &acc)
{
    float4 c = classify(a, value);
    if (SHADE) {
        c.w = correct_alpha(c.w, a.op_r);
        if (a.shade && c.w > 0.0f) shade<T, SAMPLER>(a, r, t, c);
    }
    float tr = (1.0f - acc.a) * c.w;
    acc.r = fmaf(tr, c.x, acc.r);
    acc.g = fmaf(tr, c.y, acc.g);
    acc.b = fmaf(tr, c.z, acc.b);
    acc.a = acc.a + tr;
    return acc.a >= a.ert;
}

// ------------------------------------------------------------- traversals
template <typename T, int SAMPLER, int SHADE>
__device__ __forceinline__ void trace_naive(const RArgs &a, const Ray &r, float tn, float tf,
                                            Acc &acc, int &ns)
{
    float kf = 0.0f;
    for (int k = 0; k < 16777216; ++k, kf += 1.0f) {
        const float t = fmaf(kf, a.dt, tn);
        if (!(t < tf)) break;
        ++ns;
        SampleFetch<T, SAMPLER> f;
        f.fetch(a, r, t);
        if (composite<T, SAMPLER, SHADE>(a, r, t, f.value(a), acc)) break;
    }
}

// ---------------------------------------------------------- walkers
// A walker yields the hit intervals [ta, tb] of the non-empty regions of a
// ray in ray order: the DDA over the brick raster (macrocell grid) or the
// ordered traversal of a box tree.  Its step() takes one cell or node and
// reports an interval when that cell or leaf is non-empty, so that a lane
// that has found an interval goes on to the next one while the other lanes
// of its warp are still stepping.  The renderer alternates between a
// collection phase, in which the walker's next intervals become sample-index
// ranges (rule S, with the monotone cursor k_next; ranges that touch are
// merged), and a marching phase over the collected ranges.  Lanes of a warp
// therefore spend most of their time in the same phase, and samples are still
// taken in increasing k exactly as interval-by-interval marching would take
// them.

__device__ __forceinline__ void dda_axis(float o, float d, float inv, bool zero, float p, int B,
                                         int g, int &c, int &step, float &tnext)
{
    c = (int)floorf(p / (float)B);
    c = min(max(c, 0), g - 1);
    if (zero) {
        step = 0;
        tnext = INFINITY;
    } else if (d > 0.0f) {
        step = 1;
        tnext = ((float)((c + 1) * B) - o) * inv;
    } else {
        step = -1;
        tnext = ((float)(c * B) - o) * inv;
    }
}

// 3-D DDA over the brick raster.  Cells are visited in ray order and the
// boundary crossings of consecutive cells tile [t_near, t_far); a non-empty
// cell yields the span between its entry and exit crossing.  (A crossing
// rounded to the wrong side of a corner only moves a sample whose cell is in
// doubt, and such a sample is within half a voxel of both cells, so its
// opacity is zero unless both are non-empty.)  Every axis only moves one way,
// so at most gx+gy+gz steps.  A crossing is recomputed from its integer plane
// position, or, with INC (the kernel the host picks when the drift cannot
// reach a quarter of the sample step: (steps + 4) t_max 2^-24 <= dt / 4, every
// addition rounding by at most half an ulp of t_max), advanced by B |1/d|:
// rule S takes one sample beyond each end of an interval, so a crossing off by
// less than dt still covers every sample of a non-empty cell.
template <bool INC> struct GridWalkT {
    int cx, cy, cz, sx, sy, sz, left;
    float tx, ty, tz, tcur;
    bool done;

    __device__ __forceinline__ void init(const RArgs &a, const Ray &r, float tn)
    {
        dda_axis(r.o[0], r.d[0], r.inv[0], r.zero[0], fmaf(tn, r.d[0], r.o[0]), a.B, a.gx, cx, sx, tx);
        dda_axis(r.o[1], r.d[1], r.inv[1], r.zero[1], fmaf(tn, r.d[1], r.o[1]), a.B, a.gy, cy, sy, ty);
        dda_axis(r.o[2], r.d[2], r.inv[2], r.zero[2], fmaf(tn, r.d[2], r.o[2]), a.B, a.gz, cz, sz, tz);
        left = a.gx + a.gy + a.gz + 3;
        tcur = tn;
        done = false;
    }

    // One cell of the walk: true when the cell is non-empty ([ta, tb] its
    // span); sets `done` after the last cell.
    __device__ __forceinline__ bool step(const RArgs &a, const Ray &r, float, float tf, float &ta,
                                         float &tb)
    {
        if (--left < 0) {
            done = true;
            return false;
        }
        const int B = a.B;
        bool hit = false;
        float texit = fminf(tx, fminf(ty, tz));
        if (__ldg(a.mask + ((size_t)(cz * a.gy + cy) * a.gx + cx))) {
            ta = tcur;
            tb = fminf(texit, tf);
            hit = true;
        }
        if (!(texit <= tf)) done = true;
        if (tx <= ty && tx <= tz) {
            cx += sx;
            if (cx < 0 || cx >= a.gx) done = true;
            tx = INC ? fmaf((float)B, fabsf(r.inv[0]), tx)
                      : ((float)((cx + (sx > 0 ? 1 : 0)) * B) - r.o[0]) * r.inv[0];
        } else if (ty <= tz) {
            cy += sy;
            if (cy < 0 || cy >= a.gy) done = true;
            ty = INC ? fmaf((float)B, fabsf(r.inv[1]), ty)
                      : ((float)((cy + (sy > 0 ? 1 : 0)) * B) - r.o[1]) * r.inv[1];
        } else {
            cz += sz;
            if (cz < 0 || cz >= a.gz) done = true;
            tz = INC ? fmaf((float)B, fabsf(r.inv[2]), tz)
                      : ((float)((cz + (sz > 0 ? 1 : 0)) * B) - r.o[2]) * r.inv[2];
        }
        tcur = texit;
        return hit;
    }
};

using GridWalk = GridWalkT<false>;

// Ordered traversal of a binary box tree.  Each inner node carries both
// children's boxes (floats, voxel units); both are slab-tested, the child
// entered first is visited first and the other is pushed with its interval
// (LBVH children are separated by the Morton split plane and k-d children by
// the split plane, so entry order is front-to-back order).  A leaf yields the
// interval its parent computed for it, so leaves cost no further work.  The
// stack of STACK entries suffices because the build guarantees a height of at
// most STACK + 1 levels (30-bit Morton keys give LBVH heights <= 31).
// Reference and iteration bounds keep a corrupt structure from reading
// outside its buffers or looping; a valid tree never reaches them.
template <int KIND, int STACK> struct TreeWalk {
    float4 stk[STACK];  // pushed (ref bits, ta, tb, unused): one 16-byte store/load
    int sp, budget, n_inner;
    int64_t n_leaf;
    int32_t ref;
    float cta, ctb;  // interval of `ref` (used when it is a leaf)
    bool done;

    __device__ __forceinline__ void init(const RArgs &a, const Ray &r, float tn, float tf)
    {
        const int n = __ldg(a.count);
        done = true;
        if (n <= 0) return;
        n_inner = KIND == ESS_LBVH ? n - 1 : n;
        n_leaf = KIND == ESS_LBVH ? (int64_t)a.gx * a.gy * a.gz : n;
        budget = 2 * n + 1;
        ref = __ldg(a.root);
        sp = 0;
        float lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = __int_as_float(__ldg(a.root + 1 + k));
            hi[k] = __int_as_float(__ldg(a.root + 4 + k));
        }
        cta = tn;
        ctb = tf;
        slab_tree(r, lo, hi, cta, ctb);
        done = !(cta <= ctb);
    }

    __device__ __forceinline__ void pop()
    {
        if (sp == 0) {
            done = true;
        } else {
            --sp;
            const float4 e = stk[sp];
            ref = __float_as_int(e.x);
            cta = e.y;
            ctb = e.z;
        }
    }

    // One node of the traversal: true when it is a leaf ([ta, tb] its
    // interval); sets `done` when the stack runs out.
    __device__ __forceinline__ bool step(const RArgs &a, const Ray &r, float tn, float tf, float &ta,
                                         float &tb)
    {
        if (--budget < 0) {
            done = true;
            return false;
        }
        if (ref < 0) {
            if (-1 - (int64_t)ref < n_leaf) {
                ta = cta;
                tb = ctb;
                pop();
                return true;
            }
            done = true;
            return false;
        }
        if (ref >= n_inner) {
            done = true;
            return false;
        }
        const float4 *q = reinterpret_cast<const float4 *>(a.nodes + ref);
        float4 q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2);
        int4 q3 = __ldg(reinterpret_cast<const int4 *>(q + 3));
        const float llo[3] = {q0.x, q0.y, q0.z}, lhi[3] = {q0.w, q1.x, q1.y};
        const float rlo[3] = {q1.z, q1.w, q2.x}, rhi[3] = {q2.y, q2.z, q2.w};
        float la = tn, lb = tf, ra = tn, rb = tf;
        slab_tree(r, llo, lhi, la, lb);
        slab_tree(r, rlo, rhi, ra, rb);
        bool hl = la <= lb, hr = ra <= rb;
        if (hl && hr) {
            bool left_first = la <= ra;
            if (sp < STACK) {
                stk[sp] = left_first ? make_float4(__int_as_float(q3.y), ra, rb, 0.0f)
                                     : make_float4(__int_as_float(q3.x), la, lb, 0.0f);
                ++sp;
            }
            ref = left_first ? q3.x : q3.y;
            cta = left_first ? la : ra;
            ctb = left_first ? lb : rb;
        } else if (hl) {
            ref = q3.x;
            cta = la;
            ctb = lb;
        } else if (hr) {
            ref = q3.y;
            cta = ra;
            ctb = rb;
        } else {
            pop();
        }
        return false;
    }
};

// Hybrid grid (Sec. 3.3): ordered traversal of the k-d tree yields the
// leaves' intervals; inside each leaf interval the 3-D DDA over the brick
// raster (the macrocell grid) yields the intervals of the leaf's non-empty
// bricks.  Leaves are unions of bricks and come front to back, and the DDA
// runs front to back inside each, so the intervals come in ray order; they
// cover the same non-empty bricks as the grid's walk.
struct HybridWalk {
    TreeWalk<ESS_KD, 128> tree;
    GridWalk grid;
    float leaf_tb;
    bool in_leaf;
    bool done;

    __device__ __forceinline__ void init(const RArgs &a, const Ray &r, float tn, float tf)
    {
        tree.init(a, r, tn, tf);
        in_leaf = false;
        done = tree.done;
    }

    // One step of the walk: a brick of the current leaf, or a tree node
    // while no leaf is open; true for a non-empty brick ([ta, tb] its span).
    __device__ __forceinline__ bool step(const RArgs &a, const Ray &r, float tn, float tf, float &ta,
                                         float &tb)
    {
        if (in_leaf) {
            const bool hit = grid.step(a, r, tn, leaf_tb, ta, tb);
            if (grid.done) {
                in_leaf = false;
                done = tree.done;
            }
            return hit;
        }
        float la, lb;
        if (tree.step(a, r, tn, tf, la, lb)) {
            grid.init(a, r, la);
            leaf_tb = lb;
            in_leaf = true;
        }
        done = tree.done && !in_leaf;
        return false;
    }
};

// Collected sample ranges (at most RANGES = 4), kept in four named registers
// as a queue: appended at the back in collection order, consumed from the
// front (r0) by shifting.  A phase also stops once it holds LOOKAHEAD
// samples, so that early ray termination wastes little traversal.
constexpr int RANGES = 4;
constexpr int LOOKAHEAD = 64;

struct Ranges {
    int2 r0, r1, r2, r3;
    int n;
    __device__ __forceinline__ void clear()
    {
        r0 = r1 = r2 = r3 = make_int2(0, -1);
        n = 0;
    }
    __device__ __forceinline__ void append(int k0, int k1)
    {
        const int2 v = make_int2(k0, k1);
        if (n == 0) r0 = v;
        else if (n == 1) r1 = v;
        else if (n == 2) r2 = v;
        else r3 = v;
        ++n;
    }
    __device__ __forceinline__ void extend_last(int k1)
    {
        if (n == 1) r0.y = k1;
        else if (n == 2) r1.y = k1;
        else if (n == 3) r2.y = k1;
        else r3.y = k1;
    }
    __device__ __forceinline__ void pop_front()
    {
        r0 = r1;
        r1 = r2;
        r2 = r3;
        --n;
    }
};

// Interval-by-interval skipping in rounds.  Every lane keeps a queue of up to
// RANGES sample-index ranges (rule S, with the monotone cursor k_next; ranges
// that touch are merged) holding `held` samples.  A round first tops each
// queue up from the walker (lanes whose queue is full skip that), then every
// live lane of the warp marches the same number m of samples, m the smallest
// holding among them, so that no lane idles in the march unless its ray ends
// or terminates early; leftovers stay queued.  Samples are still taken in
// increasing k, exactly as interval-by-interval marching takes them.  The
// round loop is uniform over the lanes that entered together (m is a warp
// reduction) and its inner loops have single exits.
template <typename T, int SAMPLER, int SHADE, typename Walk>
__device__ __forceinline__ void trace_walk(const RArgs &a, const Ray &r, float tn, float tf,
                                           Walk &w, Acc &acc, int &ns)
{
    const unsigned lanes = __activemask();
    int k_next = 0;       // first sample index not queued yet
    int held = 0;         // samples queued
    int k = 0;            // next sample to march: the front range's cursor
    bool walking = true;  // the walker may still yield intervals
    bool alive = true;
    Ranges rg;
    rg.clear();
    while (true) {
        if (alive && walking) {
            float ta, tb;
            while (rg.n < RANGES && held < LOOKAHEAD) {
                if (w.done) {
                    walking = false;
                    break;
                }
                if (!w.step(a, r, tn, tf, ta, tb)) continue;
                float ka = ceilf((ta - tn) / a.dt) - 1.0f;
                float kb = floorf((tb - tn) / a.dt) + 1.0f;
                kb = kb < 16777216.0f ? kb : 16777216.0f;
                int k0 = ka > (float)k_next ? (int)ka : k_next;
                int k1 = (int)kb;
                if (k1 >= k0) {
                    if (rg.n > 0 && k0 == k_next) {
                        rg.extend_last(k1);  // touches the previous range
                    } else {
                        if (rg.n == 0) k = k0;
                        rg.append(k0, k1);
                    }
                    held += k1 - k0 + 1;
                    k_next = k1 + 1;
                }
            }
        }
        if (held == 0) alive = false;
        const int m = __reduce_min_sync(lanes, alive ? held : 0x7fffffff);
        if (m == 0x7fffffff) break;  // every lane's ray is done
        if (alive) {
            float kf = (float)k, kend = (float)rg.r0.y;
            int j = 0;
            for (; j < m; ++j) {
                const float t = fmaf(kf, a.dt, tn);
                if (!(t < tf)) {
                    alive = false;
                    break;
                }
                SampleFetch<T, SAMPLER> f;
                f.fetch(a, r, t);
                if (composite<T, SAMPLER, SHADE>(a, r, t, f.value(a), acc)) {
                    alive = false;
                    ++j;
                    break;
                }
                if (__builtin_expect(kf == kend, 0)) {
                    rg.pop_front();
                    kf = (float)rg.r0.x;  // meaningless once the queue is empty (held is 0 then)
                    kend = (float)rg.r0.y;
                } else {
                    kf += 1.0f;
                }
            }
            k = (int)kf;
            ns += j;
            held -= m;
        }
    }
}

// ------------------------------------------------------------------ kernels
// The grid walk with advanced crossings (GridWalkT<true>): a kernel variant,
// not a structure kind of the interface.
constexpr int KIND_GRID_INC = 8;

// One pixel: ray, volume interval, traversal of the structure, background.
// Shared by the plain and the batched kernels, so both give the same bits.
template <typename T, int SAMPLER, int KIND, int SHADE>
__device__ __forceinline__ void render_pixel(const RArgs &a, int x, int y, long long &ns_total)
{
    int ns = 0;  // samples of this ray (at most 2^24)
    Ray r;
    gen_ray(a, x, y, r);
    float lo[3] = {0.0f, 0.0f, 0.0f};
    float hi[3] = {(float)a.nx, (float)a.ny, (float)a.nz};
    float tn = 0.0f, tf = INFINITY;
    slab(r, lo, hi, tn, tf);
    Acc acc = {0.0f, 0.0f, 0.0f, 0.0f};
    if (tn < tf) {
        if (KIND == ESS_NONE) {
            trace_naive<T, SAMPLER, SHADE>(a, r, tn, tf, acc, ns);
        } else if (KIND == ESS_GRID || KIND == KIND_GRID_INC) {
            GridWalkT<KIND == KIND_GRID_INC> w;
            w.init(a, r, tn);
            trace_walk<T, SAMPLER, SHADE>(a, r, tn, tf, w, acc, ns);
        } else if (KIND == ESS_HYBRID) {
            HybridWalk w;
            w.init(a, r, tn, tf);
            trace_walk<T, SAMPLER, SHADE>(a, r, tn, tf, w, acc, ns);
        } else if (KIND == ESS_LBVH) {
            TreeWalk<ESS_LBVH, 32> w;
            w.init(a, r, tn, tf);
            trace_walk<T, SAMPLER, SHADE>(a, r, tn, tf, w, acc, ns);
        } else {
            TreeWalk<ESS_KD, 128> w;
            w.init(a, r, tn, tf);
            trace_walk<T, SAMPLER, SHADE>(a, r, tn, tf, w, acc, ns);
        }
    }
    ns_total += ns;
    float one_m = 1.0f - acc.a;
    a.out[(size_t)y * a.W + x] =
        make_float4(fmaf(one_m, a.bg[0], acc.r), fmaf(one_m, a.bg[1], acc.g),
                    fmaf(one_m, a.bg[2], acc.b), fmaf(one_m, a.bg[3], acc.a));
}

// A block is 4 warps arranged 2 x 2; a warp covers a tw x (32/tw) pixel tile
// (tw in {4, 8, 16, 32}) so that its rays stay close together.  The block
// covers (2 tw) x (64/tw) pixels.
__device__ __forceinline__ void block_pixel(int tw, int bx, int by, int &x, int &y)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int th = 32 / tw;
    x = bx * 2 * tw + (warp & 1) * tw + (lane % tw);
    y = by * 2 * th + (warp >> 1) * th + (lane / tw);
}

__device__ __forceinline__ void count_samples(unsigned long long *samples, long long ns)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
    if ((threadIdx.x & 31) == 0 && ns) atomicAdd(samples, (unsigned long long)ns);
}

template <typename T, int SAMPLER, int KIND, int SHADE>
__global__ void __launch_bounds__(128, SHADE ? 6 : 8) k_render(RArgs a, int tw)
{
    int x, y;
    block_pixel(tw, blockIdx.x, blockIdx.y, x, y);
    long long ns = 0;
    if (x < a.W && y < a.H) render_pixel<T, SAMPLER, KIND, SHADE>(a, x, y, ns);
    count_samples(a.samples, ns);
}

// Persistent batched render: every block repeatedly takes the next tile of
// the work list (an atomic counter), finds its image by binary search over the
// per-image tile prefix, and renders it.  Images of any size and count share
// one launch; the dynamic tile order balances uneven work.
struct BatchHeader {
    int nitems, total_tiles, tile_counter, tw;
};

template <typename T, int SAMPLER, int KIND, int SHADE>
__global__ void __launch_bounds__(128, SHADE ? 6 : 8) k_render_batch(const RArgs *__restrict__ items,
                                                      const int *__restrict__ tile_prefix,
                                                      BatchHeader *hdr)
{
    __shared__ RArgs sa;
    __shared__ int s_tile, s_item;
    const int nitems = hdr->nitems, total = hdr->total_tiles, tw = hdr->tw;
    const int bw = 2 * tw, bh = 64 / tw;
    long long ns = 0;
    while (true) {
        if (threadIdx.x == 0) {
            int t = atomicAdd(&hdr->tile_counter, 1);
            s_tile = t;
            int lo = 0, hi = nitems - 1;  // last item with prefix <= t
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (tile_prefix[mid] <= t) lo = mid; else hi = mid - 1;
            }
            s_item = lo;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= total) break;
        {
            const int *src = reinterpret_cast<const int *>(items + s_item);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int k = threadIdx.x; k < (int)(sizeof(RArgs) / 4); k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();
        int local = tile - tile_prefix[s_item];
        int tiles_x = (sa.W + bw - 1) / bw;
        int x, y;
        block_pixel(tw, local % tiles_x, local / tiles_x, x, y);
        (void)bh;
        if (x < sa.W && y < sa.H) render_pixel<T, SAMPLER, KIND, SHADE>(sa, x, y, ns);
        __syncthreads();
    }
    count_samples(items[0].samples, ns);
}

// ------------------------------------------------------- launchers (SHADE)
// Instantiated once per SHADE value, in render.cu (0) and render_shaded.cu (1),
// so that the two variants compile in parallel.
template <int KIND, int SHADE> static void launch_kind(Ctx &c, const RArgs &a, ess_dtype dt, int tw)
{
    dim3 grid((a.W + 2 * tw - 1) / (2 * tw), (a.H + 64 / tw - 1) / (64 / tw));
    bool cells = a.cells != nullptr;
    if constexpr (KIND == KIND_GRID_INC) {  // cell samplers only
        switch (dt) {
        case ESS_U8: k_render<uint8_t, 1, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw); break;
        case ESS_U16: k_render<uint16_t, 1, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw); break;
        default: k_render<float, 1, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw); break;
        }
        return;
    }
    switch (dt) {
    case ESS_U8:
        if (cells) k_render<uint8_t, 1, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw);
        else k_render<uint8_t, 0, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw);
        break;
    case ESS_U16:
        if (cells) k_render<uint16_t, 1, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw);
        else k_render<uint16_t, 0, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw);
        break;
    default:
        if (cells) k_render<float, 1, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw);
        else k_render<float, 0, KIND, SHADE><<<grid, 128, 0, c.stream>>>(a, tw);
        break;
    }
}

template <int SHADE> void launch_render_kernels(Ctx &c, const RArgs &a, int kind, ess_dtype dt, int tw)
{
    switch (kind) {
    case ESS_NONE: launch_kind<ESS_NONE, SHADE>(c, a, dt, tw); break;
    case ESS_GRID:
        if (a.dda_inc && a.cells != nullptr) launch_kind<KIND_GRID_INC, SHADE>(c, a, dt, tw);
        else launch_kind<ESS_GRID, SHADE>(c, a, dt, tw);
        break;
    case ESS_LBVH: launch_kind<ESS_LBVH, SHADE>(c, a, dt, tw); break;
    case ESS_HYBRID: launch_kind<ESS_HYBRID, SHADE>(c, a, dt, tw); break;
    default: launch_kind<ESS_KD, SHADE>(c, a, dt, tw); break;
    }
}

// Persistent launch over a packed batch: every SM filled to its occupancy.
template <int SHADE>
void launch_batch_kernels(Ctx &c, int kind, ess_dtype dt, bool cells, bool dda_inc,
                          const RArgs *args,
                          const int *prefix, BatchHeader *h)
{
    int sms = 0, per_sm = 0;
    ESS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
#define ESS_BATCH_S(T, S, K)                                                                  \
    do {                                                                                      \
        ESS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(                               \
            &per_sm, k_render_batch<T, S, K, SHADE>, 128, 0));                                \
        k_render_batch<T, S, K, SHADE><<<sms * (per_sm > 0 ? per_sm : 1), 128, 0, c.stream>>>( \
            args, prefix, h);                                                                 \
    } while (0)
#define ESS_BATCH(T, K)                        \
    do {                                       \
        if (cells) ESS_BATCH_S(T, 1, K);       \
        else ESS_BATCH_S(T, 0, K);             \
    } while (0)
#define ESS_BATCH_T(K)                                   \
    switch (dt) {                                        \
    case ESS_U8: ESS_BATCH(uint8_t, K); break;           \
    case ESS_U16: ESS_BATCH(uint16_t, K); break;         \
    default: ESS_BATCH(float, K); break;                 \
    }
    switch (kind) {
    case ESS_NONE: ESS_BATCH_T(ESS_NONE); break;
    case ESS_GRID:
        if (dda_inc && cells) {  // every item of the batch allows advanced crossings
            switch (dt) {
            case ESS_U8: ESS_BATCH_S(uint8_t, 1, KIND_GRID_INC); break;
            case ESS_U16: ESS_BATCH_S(uint16_t, 1, KIND_GRID_INC); break;
            default: ESS_BATCH_S(float, 1, KIND_GRID_INC); break;
            }
        } else {
            ESS_BATCH_T(ESS_GRID);
        }
        break;
    case ESS_LBVH: ESS_BATCH_T(ESS_LBVH); break;
    case ESS_HYBRID: ESS_BATCH_T(ESS_HYBRID); break;
    default: ESS_BATCH_T(ESS_KD); break;
    }
#undef ESS_BATCH_T
#undef ESS_BATCH
#undef ESS_BATCH_S
}

extern template void launch_render_kernels<0>(Ctx &, const RArgs &, int, ess_dtype, int);
extern template void launch_render_kernels<1>(Ctx &, const RArgs &, int, ess_dtype, int);
extern template void launch_batch_kernels<0>(Ctx &, int, ess_dtype, bool, bool, const RArgs *,
                                             const int *, BatchHeader *);
extern template void launch_batch_kernels<1>(Ctx &, int, ess_dtype, bool, bool, const RArgs *,
                                             const int *, BatchHeader *);

}  // namespace ess
