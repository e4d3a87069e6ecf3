/*
 * ess_oracle.c -- plain, slow, CPU oracle for the empty-space-skipping hot
 * path of Zellmann, "Comparing Hierarchical Data Structures for Sparse Volume
 * Rendering with Empty Space Skipping" (arXiv 1912.09596).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library product links, loads or
 * calls this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every function states the passage it follows.  Where the paper is silent the
 * reading used is named R1..R11 / S, the same readings the GPU path follows:
 *   R1  ray generation          R2  trilinear reconstruction, clamp-to-edge
 *   R3  brick region and apron  R4  conservative min/max range test
 *   R5  post-classification TF  R6  front-to-back absorption+emission
 *   R7  early ray termination   S   sample lattice t_k = t_near + k*dt
 *   R8  LBVH child order        R9  k-d cost, halting, binning, max leaf size
 *   R10 Morton bit order        R11 IEEE float32, explicit fma
 *   R13 gradient shading        R14 opacity correction
 * (R13 and R14 are the second render workload: the paper only mentions
 * gradient shading, which it switches off for its measurements, Sec. 4.1.)
 * Arithmetic: IEEE binary32 with every fused multiply-add written as fmaf()
 * and everything else single-rounded; build with -ffp-contract=off and
 * without fast-math.  The paper fixes no precision; the image oracle is float32
 * so that the GPU path can be compared on identical sample positions.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   naive marcher: closed form (constant slab), special cases (all-empty,
 *     voxel centres, constant volume, exact table entries);
 *   own log2/exp2: against float64 log2/exp2 over dense sweeps;
 *   opacity correction: special cases (0, 1, ratio 1), closed form of a
 *     constant slab and its independence of the step;
 *   gradient and shading: exact gradients of linear ramps, closed-form shading
 *     of ramp slabs, skipping invariance with both switched on;
 *   brick mask: brute-force point sampling on tiny volumes;
 *   Morton/sort: test vectors, library sort;
 *   LBVH: two independent constructions agree, 2n-1 nodes, Table 1 height
 *     bound, complete-tree case, containment and separation;
 *   k-d: invariants, per-node brute-force argmin, Table 1 "Menger sponge,
 *     shallow: 1 node, height 1".  The greedy topology itself has no printed
 *     value to compare with; hand-derived trees (two corner clusters; a full
 *     cube under the maximum leaf size) pin the choice, tie and MLS rules;
 *     beyond that, parity unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_U8 0
#define ORA_U16 1
#define ORA_F32 2

typedef struct {
    const void *data;   /* [nz][ny][nx], x fastest */
    int dtype;          /* ORA_U8 / ORA_U16 / ORA_F32 */
    int nx, ny, nz;
    float value_lo, value_hi;  /* value range mapped onto the TF (R5) */
} ora_volume;

typedef struct {
    const float *rgba;  /* nt x 4, alpha in [0,1] */
    int nt;
} ora_tf;

typedef struct {
    float eye[3], u[3], v[3], w[3];
    int ortho;
} ora_camera;

typedef struct {
    float dt;      /* step in voxels */
    float ert;     /* stop once accumulated alpha >= ert; > 1 disables */
    float bg[4];   /* background RGBA */
    int shade;     /* R13: 0 off, 1 gradient shading */
    float ka, kd, ks;
    int shininess; /* 1..128 */
    float dt_ref;  /* R14: 0 off, else the TF's alpha holds for this step */
} ora_render_params;

/* ------------------------------------------------------------------ R2 --- */
static int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

static float voxel(const ora_volume *V, int i, int j, int k)
{
    i = clampi(i, 0, V->nx - 1);
    j = clampi(j, 0, V->ny - 1);
    k = clampi(k, 0, V->nz - 1);
    size_t idx = ((size_t)k * (size_t)V->ny + (size_t)j) * (size_t)V->nx + (size_t)i;
    switch (V->dtype) {
    case ORA_U8: return (float)((const uint8_t *)V->data)[idx];
    case ORA_U16: return (float)((const uint16_t *)V->data)[idx];
    default: return ((const float *)V->data)[idx];
    }
}

static float lerp(float a, float b, float f) { return fmaf(f, b - a, a); }

/* R2: voxel i has its centre at i+0.5; q = p - 0.5; i0 = floor(q); f = q - i0;
 * neighbours clamped to the volume; seven lerps, x first, then y, then z. */
float ora_sample_value(const ora_volume *V, float px, float py, float pz)
{
    float qx = px - 0.5f, qy = py - 0.5f, qz = pz - 0.5f;
    float gx = floorf(qx), gy = floorf(qy), gz = floorf(qz);
    int ix = (int)gx, iy = (int)gy, iz = (int)gz;
    float fx = qx - gx, fy = qy - gy, fz = qz - gz;
    float v000 = voxel(V, ix, iy, iz), v100 = voxel(V, ix + 1, iy, iz);
    float v010 = voxel(V, ix, iy + 1, iz), v110 = voxel(V, ix + 1, iy + 1, iz);
    float v001 = voxel(V, ix, iy, iz + 1), v101 = voxel(V, ix + 1, iy, iz + 1);
    float v011 = voxel(V, ix, iy + 1, iz + 1), v111 = voxel(V, ix + 1, iy + 1, iz + 1);
    float c00 = lerp(v000, v100, fx), c10 = lerp(v010, v110, fx);
    float c01 = lerp(v001, v101, fx), c11 = lerp(v011, v111, fx);
    float c0 = lerp(c00, c10, fy), c1 = lerp(c01, c11, fy);
    return lerp(c0, c1, fz);
}

/* ------------------------------------------------------------------ R5 --- */
/* Post-classification (Sec. 4.1): TF coordinate of a value,
 *   s = (NT-1) / (value_hi - value_lo),  x = clamp((v - value_lo) * s, 0, NT-1). */
float ora_tf_scale(const ora_volume *V, int nt)
{
    return (float)(nt - 1) / (V->value_hi - V->value_lo);
}

float ora_tf_coord(float v, float value_lo, float s, int nt)
{
    float x = (v - value_lo) * s;
    float xmax = (float)(nt - 1);
    if (x < 0.0f) x = 0.0f;
    if (x > xmax) x = xmax;
    return x;
}

/* RGBA at coordinate x: linear interpolation between entries i0 and i0+1. */
void ora_classify(const ora_tf *T, float value_lo, float s, float v, float out[4])
{
    float x = ora_tf_coord(v, value_lo, s, T->nt);
    int i0 = (int)x;
    int i1 = i0 + 1 < T->nt ? i0 + 1 : T->nt - 1;
    float w = x - (float)i0;
    for (int c = 0; c < 4; ++c) {
        float a = T->rgba[4 * i0 + c], b = T->rgba[4 * i1 + c];
        out[c] = fmaf(w, b - a, a);
    }
}

/* ------------------------------------------------------------ R13, R14 --- */
static float f_of_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_of_f(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* log2 of x in (0, 1] (normal), from the series ln m = 2 atanh(u) =
 * 2 (u + u^3/3 + u^5/5 + ...), u = (m - 1)/(m + 1), after splitting x = m 2^e
 * with m in [sqrt(1/2), sqrt(2)]; terms to u^11 (|u| <= 0.1716). */
float ora_log2_own(float x)
{
    uint32_t b = bits_of_f(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = f_of_bits((b & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) {  /* sqrt(2) */
        m = m * 0.5f;
        e = e + 1;
    }
    float u = (m - 1.0f) / (m + 1.0f);
    float u2 = u * u;
    float q = fmaf(u2, 0x1.745d18p-3f, 0x1.c71c72p-3f);  /* 2/11, 2/9 */
    q = fmaf(u2, q, 0x1.24924ap-2f);                      /* 2/7 */
    q = fmaf(u2, q, 0x1.99999ap-2f);                      /* 2/5 */
    q = fmaf(u2, q, 0x1.555556p-1f);                      /* 2/3 */
    q = fmaf(u2, q, 2.0f);
    float ln_m = u * q;
    return fmaf(ln_m, 0x1.715476p+0f, (float)e);          /* log2(e) */
}

/* 2^y for y <= 0: y = n + f with n = floor(y), f in [0, 1); 2^f = e^(f ln 2)
 * by its Taylor series to the 10th power (Horner); then times 2^n.  Below
 * 2^-126 the result is 0. */
float ora_exp2_own(float y)
{
    if (y < -126.0f) return 0.0f;
    float n = floorf(y);
    float f = y - n;
    float t = f * 0x1.62e430p-1f;  /* ln 2 */
    float p = 0x1.27e4fcp-22f;     /* 1/10! */
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
    return p * f_of_bits((uint32_t)((int)n + 127) << 23);
}

/* R14: opacity of a sample taken every dt voxels when the TF's alpha holds
 * for dt_ref voxels: 1 - (1 - alpha)^r, r = dt / dt_ref.  r = 0 (no
 * correction) and r = 1 leave alpha as it is; alpha = 0 stays 0 and alpha = 1
 * stays 1 exactly. */
float ora_opacity_correct(float alpha, float r)
{
    if (r == 0.0f || r == 1.0f) return alpha;
    float om = 1.0f - alpha;
    if (om == 0.0f) return 1.0f;
    return 1.0f - ora_exp2_own(r * ora_log2_own(om));
}

/* R13: gradient of the R2 reconstruction by central differences one voxel
 * apart on each axis. */
void ora_gradient(const ora_volume *V, float px, float py, float pz, float g[3])
{
    g[0] = (ora_sample_value(V, px + 1.0f, py, pz) - ora_sample_value(V, px - 1.0f, py, pz)) * 0.5f;
    g[1] = (ora_sample_value(V, px, py + 1.0f, pz) - ora_sample_value(V, px, py - 1.0f, pz)) * 0.5f;
    g[2] = (ora_sample_value(V, px, py, pz + 1.0f) - ora_sample_value(V, px, py, pz - 1.0f)) * 0.5f;
}

/* R13: two-sided Blinn-Phong under a headlight (light and eye along -d, so the
 * half vector is the light): c = min(|n . d|, 1) with n = g / |g|;
 * rgb' = rgb (ka + kd c) + ks c^shininess (power by squaring).  A zero
 * gradient leaves rgb as it is. */
void ora_shade(const float g[3], const float d[3], float ka, float kd, float ks, int shininess,
               float rgb[3])
{
    float len2 = fmaf(g[2], g[2], fmaf(g[1], g[1], g[0] * g[0]));
    if (!(len2 > 0.0f)) return;
    float len = sqrtf(len2);
    float dotv = fmaf(g[2], d[2], fmaf(g[1], d[1], g[0] * d[0]));
    float c = fabsf(dotv) / len;
    if (c > 1.0f) c = 1.0f;
    float spec = 1.0f, base = c;
    for (int e = shininess; e > 0; e >>= 1) {
        if (e & 1) spec = spec * base;
        if (e > 1) base = base * base;
    }
    float lam = fmaf(kd, c, ka), hs = ks * spec;
    for (int i = 0; i < 3; ++i) rgb[i] = fmaf(rgb[i], lam, hs);
}

/* ------------------------------------------------------------------ R1 --- */
/* Pixel (x, y), y = 0 the top row.  sx = (2x+1)/W - 1, sy = 1 - (2y+1)/H.
 * Perspective: o = eye, d = normalize(w + sx u + sy v).
 * Orthographic: o = eye + sx u + sy v, d = normalize(w). */
void ora_ray(const ora_camera *C, int x, int y, int W, int H, float o[3], float d[3])
{
    float sx = (float)(2 * x + 1) / (float)W - 1.0f;
    float sy = 1.0f - (float)(2 * y + 1) / (float)H;
    float dir[3];
    for (int i = 0; i < 3; ++i) {
        if (C->ortho) {
            o[i] = fmaf(sy, C->v[i], fmaf(sx, C->u[i], C->eye[i]));
            dir[i] = C->w[i];
        } else {
            o[i] = C->eye[i];
            dir[i] = fmaf(sy, C->v[i], fmaf(sx, C->u[i], C->w[i]));
        }
    }
    float len = sqrtf(fmaf(dir[2], dir[2], fmaf(dir[1], dir[1], dir[0] * dir[0])));
    for (int i = 0; i < 3; ++i) d[i] = dir[i] / len;
}

/* Slab test of the ray against the closed box [lo, hi], starting from the
 * interval [tmin, tmax].  A direction component with |d| < 1e-30 counts as 0:
 * the ray then lies in the slab iff lo <= o <= hi.  No NaN can arise. */
void ora_slab(const float o[3], const float d[3], const float lo[3], const float hi[3],
              float tmin, float tmax, float *ta, float *tb)
{
    for (int a = 0; a < 3; ++a) {
        if (!(fabsf(d[a]) >= 1e-30f)) {
            if (o[a] < lo[a] || o[a] > hi[a]) { tmin = INFINITY; tmax = -INFINITY; }
            continue;
        }
        float inv = 1.0f / d[a];
        float t0 = (lo[a] - o[a]) * inv, t1 = (hi[a] - o[a]) * inv;
        float tn = t0 < t1 ? t0 : t1, tx = t0 < t1 ? t1 : t0;
        if (tn > tmin) tmin = tn;
        if (tx < tmax) tmax = tx;
    }
    *ta = tmin;
    *tb = tmax;
}

/* Volume box [0,nx]x[0,ny]x[0,nz]: t_near = max(0, entry), t_far = exit. */
static void volume_interval(const ora_volume *V, const float o[3], const float d[3],
                            float *tn, float *tf)
{
    float lo[3] = {0.0f, 0.0f, 0.0f};
    float hi[3] = {(float)V->nx, (float)V->ny, (float)V->nz};
    ora_slab(o, d, lo, hi, 0.0f, INFINITY, tn, tf);
}

/* ------------------------------------------------------- R6, R7, S ------- */
typedef struct { float C[3], A; } ora_acc;

/* One sample k of the ray (S: t_k = fmaf(k, dt, t_near)); classifies it,
 * corrects its opacity (R14) and shades it (R13, only if its opacity is not 0)
 * when asked, composites it front-to-back (R6) and returns 1 once A >= ert
 * (R7).  `r` is dt / dt_ref, or 0. */
static int composite_sample(const ora_volume *V, const ora_tf *T, float s,
                            const float o[3], const float d[3], float t,
                            const ora_render_params *P, float r, ora_acc *acc)
{
    float p0 = fmaf(t, d[0], o[0]), p1 = fmaf(t, d[1], o[1]), p2 = fmaf(t, d[2], o[2]);
    float val = ora_sample_value(V, p0, p1, p2);
    float rgba[4];
    ora_classify(T, V->value_lo, s, val, rgba);
    rgba[3] = ora_opacity_correct(rgba[3], r);
    if (P->shade && rgba[3] > 0.0f) {
        float g[3];
        ora_gradient(V, p0, p1, p2, g);
        ora_shade(g, d, P->ka, P->kd, P->ks, P->shininess, rgba);
    }
    float tr = (1.0f - acc->A) * rgba[3];
    acc->C[0] = fmaf(tr, rgba[0], acc->C[0]);
    acc->C[1] = fmaf(tr, rgba[1], acc->C[1]);
    acc->C[2] = fmaf(tr, rgba[2], acc->C[2]);
    acc->A = acc->A + tr;
    return acc->A >= P->ert;
}

static float step_ratio(const ora_render_params *P)
{
    return P->dt_ref > 0.0f ? P->dt / P->dt_ref : 0.0f;
}

static void finish_pixel(const ora_acc *acc, const float bg[4], float *px)
{
    float one_m = 1.0f - acc->A;
    px[0] = fmaf(one_m, bg[0], acc->C[0]);
    px[1] = fmaf(one_m, bg[1], acc->C[1]);
    px[2] = fmaf(one_m, bg[2], acc->C[2]);
    px[3] = fmaf(one_m, bg[3], acc->A);
}

/* Naive ray marching without skipping ("Naive" column of Table 2): every
 * sample t_k < t_far of the volume interval is evaluated.  Writes rows
 * [y0, y1) of a W x H RGBA float image (row-major, 4 floats per pixel).
 * Returns the number of samples evaluated. */
int64_t ora_render_naive(const ora_volume *V, const ora_tf *T, const ora_camera *C,
                         const ora_render_params *P, int W, int H, float *out,
                         int y0, int y1)
{
    float s = ora_tf_scale(V, T->nt), r = step_ratio(P);
    int64_t nsamp = 0;
    for (int y = y0; y < y1; ++y) {
        for (int x = 0; x < W; ++x) {
            float o[3], d[3], tn, tf;
            ora_acc acc = {{0.0f, 0.0f, 0.0f}, 0.0f};
            ora_ray(C, x, y, W, H, o, d);
            volume_interval(V, o, d, &tn, &tf);
            if (tn < tf) {
                for (int k = 0;; ++k) {
                    float t = fmaf((float)k, P->dt, tn);
                    if (!(t < tf)) break;
                    ++nsamp;
                    if (composite_sample(V, T, s, o, d, t, P, r, &acc)) break;
                }
            }
            finish_pixel(&acc, P->bg, out + 4 * ((size_t)y * W + x));
        }
    }
    return nsamp;
}

/* Naive marching of a list of pixels (x, y pairs): the same definition as
 * ora_render_naive, for spot checks of large images.  out: 4 floats per pixel. */
int64_t ora_render_pixels(const ora_volume *V, const ora_tf *T, const ora_camera *C,
                          const ora_render_params *P, int W, int H, const int32_t *xy, int n,
                          float *out)
{
    float s = ora_tf_scale(V, T->nt), r = step_ratio(P);
    int64_t nsamp = 0;
    for (int i = 0; i < n; ++i) {
        float o[3], d[3], tn, tf;
        ora_acc acc = {{0.0f, 0.0f, 0.0f}, 0.0f};
        ora_ray(C, xy[2 * i], xy[2 * i + 1], W, H, o, d);
        volume_interval(V, o, d, &tn, &tf);
        if (tn < tf) {
            for (int k = 0;; ++k) {
                float t = fmaf((float)k, P->dt, tn);
                if (!(t < tf)) break;
                ++nsamp;
                if (composite_sample(V, T, s, o, d, t, P, r, &acc)) break;
            }
        }
        finish_pixel(&acc, P->bg, out + 4 * (size_t)i);
    }
    return nsamp;
}

/* Rendering with skipping, by brute force (rule S).  `boxes` holds nbox
 * closed boxes [lo, hi] in voxel units (6 floats each) that together cover
 * every region whose samples may be non-zero (non-empty bricks or tree
 * leaves).  Per ray: intersect every box, order the hit intervals by entry,
 * then for each interval evaluate samples k from max(k_next, ceil((ta-t_near)
 * /dt) - 1) up to floor((tb-t_near)/dt) + 1, one extra sample at each end;
 * k_next only grows, so no sample is evaluated twice and samples are always
 * taken in increasing k.  This is the definition a GPU traversal has to match;
 * it must give the naive image bit for bit. */
typedef struct { float ta, tb; } ora_iv;

static int iv_cmp(const void *a, const void *b)
{
    const ora_iv *x = (const ora_iv *)a, *y = (const ora_iv *)b;
    if (x->ta < y->ta) return -1;
    if (x->ta > y->ta) return 1;
    if (x->tb < y->tb) return -1;
    if (x->tb > y->tb) return 1;
    return 0;
}

int64_t ora_render_boxes(const ora_volume *V, const ora_tf *T, const ora_camera *C,
                         const ora_render_params *P, int W, int H, const float *boxes,
                         int nbox, float *out, int y0, int y1)
{
    float s = ora_tf_scale(V, T->nt), r = step_ratio(P);
    ora_iv *iv = (ora_iv *)malloc(sizeof(ora_iv) * (size_t)(nbox > 0 ? nbox : 1));
    int64_t nsamp = 0;
    for (int y = y0; y < y1; ++y) {
        for (int x = 0; x < W; ++x) {
            float o[3], d[3], tn, tf;
            ora_acc acc = {{0.0f, 0.0f, 0.0f}, 0.0f};
            ora_ray(C, x, y, W, H, o, d);
            volume_interval(V, o, d, &tn, &tf);
            if (tn < tf) {
                int m = 0;
                for (int b = 0; b < nbox; ++b) {
                    float ta, tb;
                    ora_slab(o, d, boxes + 6 * b, boxes + 6 * b + 3, tn, tf, &ta, &tb);
                    if (ta <= tb) { iv[m].ta = ta; iv[m].tb = tb; ++m; }
                }
                qsort(iv, (size_t)m, sizeof(ora_iv), iv_cmp);
                int64_t k_next = 0;
                int done = 0;
                for (int i = 0; i < m && !done; ++i) {
                    double ka = ceil(((double)iv[i].ta - tn) / P->dt) - 1.0;
                    double kb = floor(((double)iv[i].tb - tn) / P->dt) + 1.0;
                    if (kb > 16777216.0) kb = 16777216.0;
                    int64_t k0 = ka > (double)k_next ? (int64_t)ka : k_next;
                    int64_t k1 = (int64_t)kb;
                    for (int64_t k = k0; k <= k1; ++k) {
                        float t = fmaf((float)k, P->dt, tn);
                        if (!(t < tf)) { done = 1; break; }
                        ++nsamp;
                        if (composite_sample(V, T, s, o, d, t, P, r, &acc)) { done = 1; break; }
                    }
                    if (k1 + 1 > k_next) k_next = k1 + 1;
                }
            }
            finish_pixel(&acc, P->bg, out + 4 * ((size_t)y * W + x));
        }
    }
    free(iv);
    return nsamp;
}

/* Classification of a single point (tests: brute-force occupancy). */
void ora_point_rgba(const ora_volume *V, const ora_tf *T, float px, float py, float pz,
                    float out[4])
{
    float s = ora_tf_scale(V, T->nt);
    ora_classify(T, V->value_lo, s, ora_sample_value(V, px, py, pz), out);
}

/* ------------------------------------------------------------------ R3 --- */
/* Brick b (size B, brick coordinates bx,by,bz) covers the closed region
 * [bB, min((b+1)B, n)] per axis; a sample there reads voxels bB-1 .. (b+1)B
 * (clamped), so min and max run over that apron range (Sec. 3.1 splits the
 * volume into bricks; the apron is reading R3).  Bricks: gx = ceil(nx/B) etc.,
 * linear id (bz*gy + by)*gx + bx. */
void ora_brick_minmax(const ora_volume *V, int B, float *bmin, float *bmax)
{
    int gx = (V->nx + B - 1) / B, gy = (V->ny + B - 1) / B, gz = (V->nz + B - 1) / B;
    for (int bz = 0; bz < gz; ++bz)
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) {
                float mn = INFINITY, mx = -INFINITY;
                for (int k = bz * B - 1; k <= (bz + 1) * B; ++k)
                    for (int j = by * B - 1; j <= (by + 1) * B; ++j)
                        for (int i = bx * B - 1; i <= (bx + 1) * B; ++i) {
                            float v = voxel(V, i, j, k);
                            if (v < mn) mn = v;
                            if (v > mx) mx = v;
                        }
                size_t b = ((size_t)bz * gy + by) * gx + bx;
                bmin[b] = mn;
                bmax[b] = mx;
            }
}

/* ------------------------------------------------------------------ R4 --- */
/* Min/max range query against the TF (Sec. 2 "min-max range queries"; the
 * empty test of the build).  A lerp fmaf(f, b - a, a) with f in [0, 1) never
 * leaves [min(a,b), max(a,b)]: the rounding error of b - a is at most
 * |b - a| 2^-24 and f <= 1 - 2^-24 absorbs it, so the exact fma result lies in
 * [a, b] and rounding keeps it there.  Every sample of a brick therefore has a
 * value in [min, max] of its apron, and since x() is monotone it reads TF
 * entries lo = floor(x(min)) .. hi = min(NT-1, floor(x(max)) + 1) only.
 * The brick is non-empty iff some alpha_j > 0 with lo <= j <= hi, counted with
 * prefix counts P[i] = #{j < i : alpha_j > 0}. */
void ora_brick_mask(const float *bmin, const float *bmax, int nb, const ora_tf *T,
                    float value_lo, float value_hi, uint8_t *mask)
{
    int nt = T->nt;
    float s = (float)(nt - 1) / (value_hi - value_lo);
    int *P = (int *)malloc(sizeof(int) * (size_t)(nt + 1));
    P[0] = 0;
    for (int i = 0; i < nt; ++i) P[i + 1] = P[i] + (T->rgba[4 * i + 3] > 0.0f ? 1 : 0);
    for (int b = 0; b < nb; ++b) {
        int lo = (int)ora_tf_coord(bmin[b], value_lo, s, nt);
        int hi = (int)ora_tf_coord(bmax[b], value_lo, s, nt) + 1;
        if (hi > nt - 1) hi = nt - 1;
        mask[b] = (P[hi + 1] - P[lo]) > 0 ? 1 : 0;
    }
    free(P);
}

/* Exact per-cell test (variant of the paper's per-voxel vote, Sec. 3.1): a
 * brick is non-empty iff some trilinear cell whose sample region touches the
 * brick's closed region passes the range test of its own 8 corner values.
 * Cell c (corner voxels c..c+1, clamped) is used by samples p with
 * floor(p - 0.5) = c, i.e. p in [c+0.5, c+1.5); it touches brick b on an axis
 * iff c+0.5 <= min((b+1)B, n) and c+1.5 >= bB, for c in [-1, n-1]. */
void ora_brick_mask_cells(const ora_volume *V, int B, const ora_tf *T, uint8_t *mask)
{
    int nt = T->nt;
    float s = (float)(nt - 1) / (V->value_hi - V->value_lo);
    int *P = (int *)malloc(sizeof(int) * (size_t)(nt + 1));
    P[0] = 0;
    for (int i = 0; i < nt; ++i) P[i + 1] = P[i] + (T->rgba[4 * i + 3] > 0.0f ? 1 : 0);
    int n[3] = {V->nx, V->ny, V->nz};
    int g[3] = {(V->nx + B - 1) / B, (V->ny + B - 1) / B, (V->nz + B - 1) / B};
    memset(mask, 0, (size_t)g[0] * g[1] * g[2]);
    for (int cz = -1; cz < n[2]; ++cz)
        for (int cy = -1; cy < n[1]; ++cy)
            for (int cx = -1; cx < n[0]; ++cx) {
                float mn = INFINITY, mx = -INFINITY;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            float v = voxel(V, cx + dx, cy + dy, cz + dz);
                            if (v < mn) mn = v;
                            if (v > mx) mx = v;
                        }
                int lo = (int)ora_tf_coord(mn, V->value_lo, s, nt);
                int hi = (int)ora_tf_coord(mx, V->value_lo, s, nt) + 1;
                if (hi > nt - 1) hi = nt - 1;
                if (P[hi + 1] - P[lo] <= 0) continue;
                int c[3] = {cx, cy, cz}, blo[3], bhi[3];
                for (int a = 0; a < 3; ++a) {
                    blo[a] = g[a];
                    bhi[a] = -1;
                    for (int b = 0; b < g[a]; ++b) {
                        int rlo = b * B, rhi = (b + 1) * B < n[a] ? (b + 1) * B : n[a];
                        /* 2c+1 <= 2 rhi  and  2c+3 >= 2 rlo  (halves kept exact) */
                        if (2 * c[a] + 1 <= 2 * rhi && 2 * c[a] + 3 >= 2 * rlo) {
                            if (b < blo[a]) blo[a] = b;
                            if (b > bhi[a]) bhi[a] = b;
                        }
                    }
                }
                for (int bz = blo[2]; bz <= bhi[2]; ++bz)
                    for (int by = blo[1]; by <= bhi[1]; ++by)
                        for (int bx = blo[0]; bx <= bhi[0]; ++bx)
                            mask[((size_t)bz * g[1] + by) * g[0] + bx] = 1;
            }
    free(P);
}

/* Compaction (Sec. 3.1): ids of the non-empty bricks in increasing order. */
int ora_compact(const uint8_t *mask, int nb, uint32_t *ids)
{
    int n = 0;
    for (int b = 0; b < nb; ++b)
        if (mask[b]) ids[n++] = (uint32_t)b;
    return n;
}

/* ----------------------------------------------------------------- R10 --- */
/* 30-bit 3-d Morton code (Sec. 3.1): bit i of x goes to bit 3i, of y to 3i+1,
 * of z to 3i+2, for i < 10. */
uint32_t ora_morton30(uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t code = 0;
    for (int i = 0; i < 10; ++i) {
        code |= ((x >> i) & 1u) << (3 * i);
        code |= ((y >> i) & 1u) << (3 * i + 1);
        code |= ((z >> i) & 1u) << (3 * i + 2);
    }
    return code;
}

void ora_morton_keys(const uint32_t *ids, int n, int gx, int gy, uint32_t *keys)
{
    for (int i = 0; i < n; ++i) {
        uint32_t b = ids[i];
        uint32_t bx = b % (uint32_t)gx, by = (b / (uint32_t)gx) % (uint32_t)gy;
        uint32_t bz = b / ((uint32_t)gx * (uint32_t)gy);
        keys[i] = ora_morton30(bx, by, bz);
    }
}

/* Sort by key (Sec. 3.1 sorts with a library O(n) sort; keys are unique, so the
 * sorted order is unique too).  The library sort qsort() stands in. */
typedef struct { uint32_t key, id; } ora_kv;

static int kv_cmp(const void *a, const void *b)
{
    uint32_t x = ((const ora_kv *)a)->key, y = ((const ora_kv *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void ora_sort_pairs(uint32_t *keys, uint32_t *ids, int n)
{
    ora_kv *kv = (ora_kv *)malloc(sizeof(ora_kv) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) { kv[i].key = keys[i]; kv[i].id = ids[i]; }
    qsort(kv, (size_t)n, sizeof(ora_kv), kv_cmp);
    for (int i = 0; i < n; ++i) { keys[i] = kv[i].key; ids[i] = kv[i].id; }
    free(kv);
}

/* ------------------------------------------------------------------ R8 --- */
/* LBVH over n sorted unique Morton keys (Sec. 3.1: the Morton order defines a
 * hierarchy that splits in the spatial middle; the split sits at the highest
 * bit in which the keys of a range differ).
 *
 * Node numbering is the one of Karras' radix tree: inner node 0 is the root
 * over [0, n-1]; a range [first, last] is split after index g, the last key
 * whose bit (31 - clz(k_first ^ k_last)) is 0; the left child covers
 * [first, g] and is leaf g if first == g, else inner node g; the right child
 * covers [g+1, last] and is leaf g+1 if g+1 == last, else inner node g+1.
 * Child references: inner i as i >= 0, leaf j as -1 - j.
 *
 * ora_lbvh_topdown is the definition, a recursion from the root;
 * ora_lbvh_karras computes each inner node independently from its index with
 * Karras' per-node search (a different algorithm); the tests require both to
 * agree exactly.  Returns 0, or -1 if keys are not strictly increasing. */
static int clz32(uint32_t x)
{
    int n = 0;
    if (x == 0) return 32;
    while (!(x & 0x80000000u)) { x <<= 1; ++n; }
    return n;
}

static void topdown_rec(const uint32_t *k, int first, int last, int node,
                        int32_t *left, int32_t *right, int32_t *rng)
{
    int bit = 31 - clz32(k[first] ^ k[last]);
    int g = first;
    while (g + 1 <= last && ((k[g + 1] >> bit) & 1u) == 0u) ++g;
    rng[2 * node] = first;
    rng[2 * node + 1] = last;
    if (first == g) {
        left[node] = -1 - g;
    } else {
        left[node] = g;
        topdown_rec(k, first, g, g, left, right, rng);
    }
    if (g + 1 == last) {
        right[node] = -1 - (g + 1);
    } else {
        right[node] = g + 1;
        topdown_rec(k, g + 1, last, g + 1, left, right, rng);
    }
}

int ora_lbvh_topdown(const uint32_t *keys, int n, int32_t *left, int32_t *right,
                     int32_t *ranges)
{
    for (int i = 0; i + 1 < n; ++i)
        if (!(keys[i] < keys[i + 1])) return -1;
    if (n >= 2) topdown_rec(keys, 0, n - 1, 0, left, right, ranges);
    return 0;
}

static int delta(const uint32_t *k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    return clz32(k[i] ^ k[j]);
}

int ora_lbvh_karras(const uint32_t *k, int n, int32_t *left, int32_t *right)
{
    for (int i = 0; i + 1 < n; ++i)
        if (!(k[i] < k[i + 1])) return -1;
    for (int i = 0; i + 1 < n; ++i) {
        int d = delta(k, n, i, i + 1) - delta(k, n, i, i - 1) > 0 ? 1 : -1;
        int dmin = delta(k, n, i, i - d);
        int lmax = 2;
        while (delta(k, n, i, i + lmax * d) > dmin) lmax *= 2;
        int l = 0;
        for (int t = lmax / 2; t >= 1; t /= 2)
            if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
        int j = i + l * d;
        int dnode = delta(k, n, i, j);
        int s = 0, t = l;
        do {
            t = (t + 1) / 2;
            if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        } while (t > 1);
        int g = i + s * d + (d < 0 ? d : 0);
        int lo = i < j ? i : j, hi = i < j ? j : i;
        left[i] = (lo == g) ? -1 - g : g;
        right[i] = (hi == g + 1) ? -1 - (g + 1) : g + 1;
    }
    return 0;
}

/* Inner-node boxes (Sec. 3.1 assembles each inner node's AABB from its
 * leaves): the union of the brick boxes [b, b+1) of the leaves in the node's
 * key range, in brick coordinates, as lo[3], hi[3] (exclusive).  Computed
 * directly from the ranges, not bottom-up. */
void ora_lbvh_boxes(const uint32_t *sorted_ids, int n, int gx, int gy,
                    const int32_t *ranges, int32_t *boxes)
{
    for (int i = 0; i + 1 < n; ++i) {
        int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
        for (int j = ranges[2 * i]; j <= ranges[2 * i + 1]; ++j) {
            uint32_t b = sorted_ids[j];
            int c[3] = {(int)(b % (uint32_t)gx), (int)((b / (uint32_t)gx) % (uint32_t)gy),
                        (int)(b / ((uint32_t)gx * (uint32_t)gy))};
            for (int a = 0; a < 3; ++a) {
                if (c[a] < lo[a]) lo[a] = c[a];
                if (c[a] + 1 > hi[a]) hi[a] = c[a] + 1;
            }
        }
        for (int a = 0; a < 3; ++a) { boxes[6 * i + a] = lo[a]; boxes[6 * i + 3 + a] = hi[a]; }
    }
}

/* ------------------------------------------------------------------ R9 --- */
/* k-d tree over the non-empty bricks (Sec. 3.2 and Sec. 4.3).
 *
 * Boxes are in brick coordinates [lo, hi).  V(box) is the number of voxels
 * inside it, the product over axes of min(hi*B, n) - lo*B.  The root is the
 * tight box of all non-empty bricks (Sec. 3.2.1 shrinks the volume box to
 * them).  A node X is split by the plane with the lowest cost V(L) + V(R),
 * L and R being the tight boxes of the non-empty bricks of X below and above
 * the plane (Sec. 3.2.1: plane sweep with the volume of the tight boxes).
 * Candidates on axis a with brick extent e >= 2: every interior brick boundary
 * (nbins == 0, the CPU builder), or lo + floor(j e / nbins), j = 1..nbins-1,
 * strictly inside and without repeats (binning on the brick raster, Sec.
 * 3.2.2, nbins = 4 in Sec. 4.3).  Ties go to the lower axis, then the lower
 * plane.  Halting (Sec. 4.3): shallow (halting 0) splits only while
 * V(X) > 10 % of V(root); deep (halting 1) while V(X) > 8^3.  A split is taken
 * iff halting allows it and its cost is below V(X).  Otherwise, when halting
 * allows splitting, mls > 0 and V(X) > mls^3, X is split in the middle of the
 * axis with the largest voxel extent among axes with e >= 2 (Sec. 4.3, maximum
 * leaf size; ties to the lower axis) at lo + floor(e/2).  Children are tight
 * boxes, numbered breadth first, left child first.
 *
 * Output: 9 ints per node: lo[3], hi[3], axis, plane, first_child; a leaf has
 * axis -1, plane 0, first_child -1.  Returns the node count (0 for an empty
 * mask) or -1 if max_nodes is too small. */
typedef struct { int lo[3], hi[3]; } ibox;

static uint64_t box_volume(const ibox *b, int B, const int n[3])
{
    uint64_t v = 1;
    for (int a = 0; a < 3; ++a) {
        int x1 = b->hi[a] * B < n[a] ? b->hi[a] * B : n[a];
        v *= (uint64_t)(x1 - b->lo[a] * B);
    }
    return v;
}

/* Tight box of the non-empty bricks of X with coordinate on `axis` in
 * [c0, c1).  Returns 0 if there is none. */
static int tight_box(const uint8_t *mask, const int g[3], const ibox *X, int axis,
                     int c0, int c1, ibox *out)
{
    int found = 0;
    ibox r = {{1 << 30, 1 << 30, 1 << 30}, {-1, -1, -1}};
    for (int z = X->lo[2]; z < X->hi[2]; ++z)
        for (int y = X->lo[1]; y < X->hi[1]; ++y)
            for (int x = X->lo[0]; x < X->hi[0]; ++x) {
                int c[3] = {x, y, z};
                if (axis >= 0 && (c[axis] < c0 || c[axis] >= c1)) continue;
                if (!mask[((size_t)z * g[1] + y) * g[0] + x]) continue;
                found = 1;
                for (int a = 0; a < 3; ++a) {
                    if (c[a] < r.lo[a]) r.lo[a] = c[a];
                    if (c[a] + 1 > r.hi[a]) r.hi[a] = c[a] + 1;
                }
            }
    if (found) *out = r;
    return found;
}

int ora_kd_build(const uint8_t *mask, int gx, int gy, int gz, int B, int nx, int ny,
                 int nz, int nbins, int halting, int mls, int32_t *out, int max_nodes)
{
    int g[3] = {gx, gy, gz}, n[3] = {nx, ny, nz};
    ibox full = {{0, 0, 0}, {gx, gy, gz}}, root;
    if (!tight_box(mask, g, &full, -1, 0, 0, &root)) return 0;
    if (max_nodes < 1) return -1;
    ibox *box = (ibox *)malloc(sizeof(ibox) * (size_t)max_nodes);
    box[0] = root;
    int count = 1;
    uint64_t vroot = box_volume(&root, B, n);
    uint64_t mls3 = (uint64_t)mls * (uint64_t)mls * (uint64_t)mls;
    for (int i = 0; i < count; ++i) {
        ibox X = box[i];
        int32_t *rec = out + 9 * (size_t)i;
        for (int a = 0; a < 3; ++a) { rec[a] = X.lo[a]; rec[3 + a] = X.hi[a]; }
        rec[6] = -1; rec[7] = 0; rec[8] = -1;
        uint64_t vx = box_volume(&X, B, n);
        int allowed = (halting == 0) ? (10 * vx > vroot) : (vx > 512);
        if (!allowed) continue;
        uint64_t best = UINT64_MAX;
        int bax = -1, bpl = 0;
        for (int a = 0; a < 3; ++a) {
            int e = X.hi[a] - X.lo[a];
            if (e < 2) continue;
            int prev = -1;
            int ncand = nbins == 0 ? e - 1 : nbins - 1;
            for (int j = 1; j <= ncand; ++j) {
                int p = nbins == 0 ? X.lo[a] + j : X.lo[a] + (j * e) / nbins;
                if (p <= X.lo[a] || p >= X.hi[a] || p == prev) continue;
                prev = p;
                ibox L, R;
                if (!tight_box(mask, g, &X, a, X.lo[a], p, &L)) continue;
                if (!tight_box(mask, g, &X, a, p, X.hi[a], &R)) continue;
                uint64_t cost = box_volume(&L, B, n) + box_volume(&R, B, n);
                if (cost < best) { best = cost; bax = a; bpl = p; }
            }
        }
        if (!(bax >= 0 && best < vx)) {
            bax = -1;
            if (mls > 0 && vx > mls3) {
                int bestext = -1;
                for (int a = 0; a < 3; ++a) {
                    int e = X.hi[a] - X.lo[a];
                    if (e < 2) continue;
                    int x1 = X.hi[a] * B < n[a] ? X.hi[a] * B : n[a];
                    int ext = x1 - X.lo[a] * B;
                    if (ext > bestext) { bestext = ext; bax = a; bpl = X.lo[a] + e / 2; }
                }
            }
        }
        if (bax < 0) continue;
        ibox L, R;
        tight_box(mask, g, &X, bax, X.lo[bax], bpl, &L);
        tight_box(mask, g, &X, bax, bpl, X.hi[bax], &R);
        if (count + 2 > max_nodes) { free(box); return -1; }
        rec[6] = bax; rec[7] = bpl; rec[8] = count;
        box[count++] = L;
        box[count++] = R;
    }
    free(box);
    return count;
}
