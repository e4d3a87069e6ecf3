// render.cu -- ray marching through the skipping structures (Sec. 4.1:
// absorption plus emission, post-classification TF lookups; Table 2 "Naive"
// is the no-skipping marcher).
//
// Every path evaluates the same samples t_k = fmaf(k, dt, t_near) with the
// same float32 operation sequence; a skipping path only leaves out samples
// whose opacity is exactly zero, which leave the accumulated colour and
// opacity bit-identical, so its image equals the naive image bit for bit.
// For a hit interval [ta, tb] of a non-empty region, samples are taken from
// k = max(k_next, ceil((ta - t_near)/dt) - 1) to floor((tb - t_near)/dt) + 1,
// one extra on each side to absorb rounding of the slab test; k_next only
// grows, so no sample is taken twice.
//
// Compiled with -fmad=false and IEEE division / square root: every fused
// multiply-add is an explicit fmaf().
#include <cuda_runtime.h>
#include <stdint.h>

#include "ess_internal.h"

namespace ess {

struct RArgs {
    const void *vol;
    int nx, ny, nz;
    float value_lo, s;   // TF coordinate x = (v - value_lo) * s
    const float4 *tf;
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
    const int32_t *root;      // ref, box lo xyz, hi xyz (brick coordinates)
    const int *count;         // > 0 iff the tree is non-empty
    const int32_t *kd_nodes;  // k-d: node records, 9 ints (box first)
    unsigned long long *samples;
};

struct Ray {
    float o[3], d[3], inv[3];
    bool zero[3];
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

// -------------------------------------------------------- sampling (R2, R5)
template <typename T> __device__ __forceinline__ float ldv(const T *p) { return (float)__ldg(p); }

__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

template <typename T>
__device__ __forceinline__ float sample_value(const RArgs &a, float px, float py, float pz)
{
    const T *vol = (const T *)a.vol;
    float qx = px - 0.5f, qy = py - 0.5f, qz = pz - 0.5f;
    float gxf = floorf(qx), gyf = floorf(qy), gzf = floorf(qz);
    int ix = (int)gxf, iy = (int)gyf, iz = (int)gzf;
    float fx = qx - gxf, fy = qy - gyf, fz = qz - gzf;
    int x0 = min(max(ix, 0), a.nx - 1), x1 = min(max(ix + 1, 0), a.nx - 1);
    int y0 = min(max(iy, 0), a.ny - 1), y1 = min(max(iy + 1, 0), a.ny - 1);
    int z0 = min(max(iz, 0), a.nz - 1), z1 = min(max(iz + 1, 0), a.nz - 1);
    size_t sy = (size_t)a.nx, sz = (size_t)a.nx * (size_t)a.ny;
    size_t r00 = z0 * sz + y0 * sy, r10 = z0 * sz + y1 * sy;
    size_t r01 = z1 * sz + y0 * sy, r11 = z1 * sz + y1 * sy;
    float v000 = ldv(vol + r00 + x0), v100 = ldv(vol + r00 + x1);
    float v010 = ldv(vol + r10 + x0), v110 = ldv(vol + r10 + x1);
    float v001 = ldv(vol + r01 + x0), v101 = ldv(vol + r01 + x1);
    float v011 = ldv(vol + r11 + x0), v111 = ldv(vol + r11 + x1);
    float c00 = lerpf(v000, v100, fx), c10 = lerpf(v010, v110, fx);
    float c01 = lerpf(v001, v101, fx), c11 = lerpf(v011, v111, fx);
    float c0 = lerpf(c00, c10, fy), c1 = lerpf(c01, c11, fy);
    return lerpf(c0, c1, fz);
}

__device__ __forceinline__ float4 classify(const RArgs &a, float v)
{
    float x = (v - a.value_lo) * a.s;
    float xmax = (float)(a.nt - 1);
    x = x < 0.0f ? 0.0f : x;
    x = x > xmax ? xmax : x;
    int i0 = (int)x;
    int i1 = i0 + 1 < a.nt ? i0 + 1 : a.nt - 1;
    float w = x - (float)i0;
    float4 c0 = __ldg(a.tf + i0), c1 = __ldg(a.tf + i1);
    return make_float4(fmaf(w, c1.x - c0.x, c0.x), fmaf(w, c1.y - c0.y, c0.y),
                       fmaf(w, c1.z - c0.z, c0.z), fmaf(w, c1.w - c0.w, c0.w));
}

// One sample (R6 compositing, R7 early termination); true when A >= ert.
template <typename T>
__device__ __forceinline__ bool sample_step(const RArgs &a, const Ray &r, float t, Acc &acc)
{
    float px = fmaf(t, r.d[0], r.o[0]), py = fmaf(t, r.d[1], r.o[1]), pz = fmaf(t, r.d[2], r.o[2]);
    float4 c = classify(a, sample_value<T>(a, px, py, pz));
    float tr = (1.0f - acc.a) * c.w;
    acc.r = fmaf(tr, c.x, acc.r);
    acc.g = fmaf(tr, c.y, acc.g);
    acc.b = fmaf(tr, c.z, acc.b);
    acc.a = acc.a + tr;
    return acc.a >= a.ert;
}

// Rule S over one hit interval; returns true when the ray is finished.
template <typename T>
__device__ __forceinline__ bool march(const RArgs &a, const Ray &r, float tn, float tf, float ta,
                                      float tb, int &k_next, Acc &acc, long long &ns)
{
    float ka = ceilf((ta - tn) / a.dt) - 1.0f;
    float kb = floorf((tb - tn) / a.dt) + 1.0f;
    kb = kb < 16777216.0f ? kb : 16777216.0f;
    int k0 = ka > (float)k_next ? (int)ka : k_next;
    int k1 = (int)kb;
    for (int k = k0; k <= k1; ++k) {
        float t = fmaf((float)k, a.dt, tn);
        if (!(t < tf)) return true;
        ++ns;
        if (sample_step<T>(a, r, t, acc)) return true;
    }
    if (k1 + 1 > k_next) k_next = k1 + 1;
    return false;
}

// ------------------------------------------------------------- traversals
template <typename T>
__device__ __forceinline__ void trace_naive(const RArgs &a, const Ray &r, float tn, float tf,
                                            Acc &acc, long long &ns)
{
    for (int k = 0;; ++k) {
        float t = fmaf((float)k, a.dt, tn);
        if (!(t < tf)) break;
        ++ns;
        if (sample_step<T>(a, r, t, acc)) break;
    }
}

// 3-D DDA over the brick raster (the macrocell grid).  Cells are visited in
// ray order; for a non-empty cell the exact slab interval of its box is
// marched.  Boundary crossings are recomputed from integer plane positions
// (no drift) and every axis only moves one way, so at most gx+gy+gz steps.
template <typename T>
__device__ __forceinline__ void trace_grid(const RArgs &a, const Ray &r, float tn, float tf,
                                           Acc &acc, long long &ns)
{
    const int g[3] = {a.gx, a.gy, a.gz};
    const int n[3] = {a.nx, a.ny, a.nz};
    const float Bf = (float)a.B;
    int cell[3], step[3];
    float tnext[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float p = fmaf(tn, r.d[ax], r.o[ax]);
        int c = (int)floorf(p / Bf);
        c = min(max(c, 0), g[ax] - 1);
        cell[ax] = c;
        if (r.zero[ax]) {
            step[ax] = 0;
            tnext[ax] = INFINITY;
        } else if (r.d[ax] > 0.0f) {
            step[ax] = 1;
            tnext[ax] = ((float)((c + 1) * a.B) - r.o[ax]) * r.inv[ax];
        } else {
            step[ax] = -1;
            tnext[ax] = ((float)(c * a.B) - r.o[ax]) * r.inv[ax];
        }
    }
    int k_next = 0;
    int maxit = g[0] + g[1] + g[2] + 3;
    for (int it = 0; it < maxit; ++it) {
        size_t id = ((size_t)cell[2] * a.gy + cell[1]) * a.gx + cell[0];
        if (__ldg(a.mask + id)) {
            float lo[3], hi[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                lo[ax] = (float)(cell[ax] * a.B);
                hi[ax] = (float)min((cell[ax] + 1) * a.B, n[ax]);
            }
            float ta = tn, tb = tf;
            slab(r, lo, hi, ta, tb);
            if (ta <= tb && march<T>(a, r, tn, tf, ta, tb, k_next, acc, ns)) return;
        }
        int ax = 0;
        if (tnext[1] < tnext[ax]) ax = 1;
        if (tnext[2] < tnext[ax]) ax = 2;
        if (!(tnext[ax] <= tf)) return;
        cell[ax] += step[ax];
        if (cell[ax] < 0 || cell[ax] >= g[ax]) return;
        tnext[ax] = ((float)((cell[ax] + (step[ax] > 0 ? 1 : 0)) * a.B) - r.o[ax]) * r.inv[ax];
    }
}

// Box in brick coordinates [lo, hi) -> closed voxel-space box, clamped at the
// volume's far faces (partial bricks).
__device__ __forceinline__ void brick_box_f(const RArgs &a, int lx, int ly, int lz, int hx, int hy,
                                            int hz, float lo[3], float hi[3])
{
    lo[0] = (float)(lx * a.B);
    lo[1] = (float)(ly * a.B);
    lo[2] = (float)(lz * a.B);
    hi[0] = (float)min(hx * a.B, a.nx);
    hi[1] = (float)min(hy * a.B, a.ny);
    hi[2] = (float)min(hz * a.B, a.nz);
}

__device__ __forceinline__ void leaf_box_f(const RArgs &a, int KIND, int32_t ref, float lo[3],
                                           float hi[3])
{
    int32_t id = -1 - ref;
    if (KIND == ESS_LBVH) {
        int x = id % a.gx, y = (id / a.gx) % a.gy, z = id / (a.gx * a.gy);
        brick_box_f(a, x, y, z, x + 1, y + 1, z + 1, lo, hi);
    } else {
        const int32_t *b = a.kd_nodes + 9 * (size_t)id;
        brick_box_f(a, __ldg(b), __ldg(b + 1), __ldg(b + 2), __ldg(b + 3), __ldg(b + 4),
                    __ldg(b + 5), lo, hi);
    }
}

// Ordered traversal of a binary box tree.  Each inner node carries both
// children's boxes; both are slab-tested, the child entered first is
// visited first and the other is pushed (LBVH children are separated by the
// Morton split plane and k-d children by the split plane, so entry order is
// front-to-back order).  A leaf's box interval is marched with rule S.  The
// stack of STACK entries suffices because the build guarantees a height of at
// most STACK + 1 levels (30-bit Morton keys give LBVH heights <= 31).
template <typename T, int KIND, int STACK>
__device__ __forceinline__ void trace_tree(const RArgs &a, const Ray &r, float tn, float tf,
                                           Acc &acc, long long &ns)
{
    const int n = __ldg(a.count);
    if (n <= 0) return;
    // reference bounds: a valid tree never leaves them and visits each node at
    // most once per ray; the checks keep a corrupt structure from reading
    // outside its buffers or looping
    const int n_inner = KIND == ESS_LBVH ? n - 1 : n;
    const int64_t n_leaf = KIND == ESS_LBVH ? (int64_t)a.gx * a.gy * a.gz : n;
    int budget = 2 * n + 1;
    int32_t ref = __ldg(a.root);
    {
        float lo[3], hi[3];
        brick_box_f(a, __ldg(a.root + 1), __ldg(a.root + 2), __ldg(a.root + 3), __ldg(a.root + 4),
                    __ldg(a.root + 5), __ldg(a.root + 6), lo, hi);
        float ta = tn, tb = tf;
        slab(r, lo, hi, ta, tb);
        if (!(ta <= tb)) return;
    }
    int32_t stack[STACK];
    int sp = 0;
    int k_next = 0;
    while (--budget >= 0) {
        if (ref < 0) {
            if (-1 - (int64_t)ref >= n_leaf) return;
            float lo[3], hi[3];
            leaf_box_f(a, KIND, ref, lo, hi);
            float ta = tn, tb = tf;
            slab(r, lo, hi, ta, tb);
            if (ta <= tb && march<T>(a, r, tn, tf, ta, tb, k_next, acc, ns)) return;
        } else {
            if (ref >= n_inner) return;
            const uint4 *q = reinterpret_cast<const uint4 *>(a.nodes + ref);
            uint4 q0 = __ldg(q), q1 = __ldg(q + 1);
            // lbox = q0.x..q0.z (6 x u16), rbox = q0.w, q1.x, q1.y; left = q1.z, right = q1.w
            float llo[3], lhi[3], rlo[3], rhi[3];
            brick_box_f(a, q0.x & 0xffff, q0.x >> 16, q0.y & 0xffff, q0.y >> 16, q0.z & 0xffff,
                        q0.z >> 16, llo, lhi);
            brick_box_f(a, q0.w & 0xffff, q0.w >> 16, q1.x & 0xffff, q1.x >> 16, q1.y & 0xffff,
                        q1.y >> 16, rlo, rhi);
            float la = tn, lb = tf, ra = tn, rb = tf;
            slab(r, llo, lhi, la, lb);
            slab(r, rlo, rhi, ra, rb);
            bool hl = la <= lb, hr = ra <= rb;
            int32_t lc = (int32_t)q1.z, rc = (int32_t)q1.w;
            if (hl && hr) {
                bool left_first = la <= ra;
                if (sp < STACK) stack[sp++] = left_first ? rc : lc;
                ref = left_first ? lc : rc;
                continue;
            }
            if (hl) {
                ref = lc;
                continue;
            }
            if (hr) {
                ref = rc;
                continue;
            }
        }
        if (sp == 0) return;
        ref = stack[--sp];
    }
}

// ------------------------------------------------------------------ kernel
// 128 threads per block, 16 x 8 pixels; each warp covers an 8 x 4 tile so
// that its rays stay close together.
template <typename T, int KIND>
__global__ void __launch_bounds__(128) k_render(RArgs a)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    int y = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    long long ns = 0;
    if (x < a.W && y < a.H) {
        Ray r;
        gen_ray(a, x, y, r);
        float lo[3] = {0.0f, 0.0f, 0.0f};
        float hi[3] = {(float)a.nx, (float)a.ny, (float)a.nz};
        float tn = 0.0f, tf = INFINITY;
        slab(r, lo, hi, tn, tf);
        Acc acc = {0.0f, 0.0f, 0.0f, 0.0f};
        if (tn < tf) {
            if (KIND == ESS_NONE)
                trace_naive<T>(a, r, tn, tf, acc, ns);
            else if (KIND == ESS_GRID)
                trace_grid<T>(a, r, tn, tf, acc, ns);
            else if (KIND == ESS_LBVH)
                trace_tree<T, ESS_LBVH, 32>(a, r, tn, tf, acc, ns);
            else
                trace_tree<T, ESS_KD, 128>(a, r, tn, tf, acc, ns);
        }
        float one_m = 1.0f - acc.a;
        a.out[(size_t)y * a.W + x] =
            make_float4(fmaf(one_m, a.bg[0], acc.r), fmaf(one_m, a.bg[1], acc.g),
                        fmaf(one_m, a.bg[2], acc.b), fmaf(one_m, a.bg[3], acc.a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
    if (lane == 0 && ns) atomicAdd(a.samples, (unsigned long long)ns);
}

template <int KIND> static void launch_kind(Ctx &c, const RArgs &a, ess_dtype dt)
{
    dim3 grid((a.W + 15) / 16, (a.H + 7) / 8);
    switch (dt) {
    case ESS_U8: k_render<uint8_t, KIND><<<grid, 128, 0, c.stream>>>(a); break;
    case ESS_U16: k_render<uint16_t, KIND><<<grid, 128, 0, c.stream>>>(a); break;
    default: k_render<float, KIND><<<grid, 128, 0, c.stream>>>(a); break;
    }
}

void launch_render(Ctx &c, const RenderJob &j)
{
    RArgs a;
    a.vol = j.vol->data;
    a.nx = j.vol->nx;
    a.ny = j.vol->ny;
    a.nz = j.vol->nz;
    a.value_lo = j.vol->value_lo;
    a.s = (float)(j.tf->nt - 1) / (j.vol->value_hi - j.vol->value_lo);
    a.tf = j.tf->table;
    a.nt = j.tf->nt;
    for (int i = 0; i < 3; ++i) {
        a.eye[i] = j.cam.eye[i];
        a.u[i] = j.cam.u[i];
        a.v[i] = j.cam.v[i];
        a.w[i] = j.cam.w[i];
    }
    a.ortho = j.cam.ortho;
    a.dt = j.rp.dt;
    a.ert = j.rp.ert;
    for (int i = 0; i < 4; ++i) a.bg[i] = j.rp.bg[i];
    a.W = j.W;
    a.H = j.H;
    a.out = reinterpret_cast<float4 *>(j.out);
    a.mask = j.st->mask;
    a.B = j.st->p.brick;
    a.gx = j.st->gx;
    a.gy = j.st->gy;
    a.gz = j.st->gz;
    a.nodes = j.st->nodes;
    a.root = j.st->root;
    a.count = j.st->kind == ESS_KD ? j.st->kd_count_dev : j.st->count;
    a.kd_nodes = j.st->kd_nodes;
    a.samples = c.samples;
    switch (j.st->kind) {
    case ESS_NONE: {
        Launch L(c, "render_naive");
        launch_kind<ESS_NONE>(c, a, j.vol->dtype);
        break;
    }
    case ESS_GRID: {
        Launch L(c, "render_grid");
        launch_kind<ESS_GRID>(c, a, j.vol->dtype);
        break;
    }
    case ESS_LBVH: {
        Launch L(c, "render_lbvh");
        launch_kind<ESS_LBVH>(c, a, j.vol->dtype);
        break;
    }
    case ESS_KD: {
        Launch L(c, "render_kd");
        launch_kind<ESS_KD>(c, a, j.vol->dtype);
        break;
    }
    default: throw Error{ESS_ERR_ARG, "render: structure kind not supported"};
    }
}

}  // namespace ess
