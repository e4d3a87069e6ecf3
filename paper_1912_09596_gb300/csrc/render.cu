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
//
// The device code lives in render_kernels.h; this file instantiates the plain
// kernels and render_shaded.cu the shaded ones (gradient shading, R13, and
// opacity correction, R14: the second render workload).
#include <algorithm>
#include <cmath>

#include "render_kernels.h"

namespace ess {

// Whether the grid walk may advance its crossings (GridWalkT<true>): the
// drift after every step it can take stays below a quarter of the sample step.
// t_max is the largest ray parameter of a sample: the farthest volume corner
// from the eye plus the image plane's extent (orthographic origins).
bool grid_dda_inc(const RenderJob &j)
{
    double tmax = 0.0;
    for (int k = 0; k < 8; ++k) {
        const double cx = (k & 1) ? j.vol->nx : 0, cy = (k & 2) ? j.vol->ny : 0,
                     cz = (k & 4) ? j.vol->nz : 0;
        const double dx = cx - j.cam.eye[0], dy = cy - j.cam.eye[1], dz = cz - j.cam.eye[2];
        tmax = std::max(tmax, std::sqrt(dx * dx + dy * dy + dz * dz));
    }
    double ext = 0.0;
    for (int i = 0; i < 3; ++i) ext += std::fabs(j.cam.u[i]) + std::fabs(j.cam.v[i]);
    tmax += ext;
    const double steps = (double)j.st->gx + j.st->gy + j.st->gz + 4.0;
    return steps * tmax * std::ldexp(1.0, -24) <= 0.25 * j.rp.dt;
}

static void fill_args(Ctx &c, const RenderJob &j, RArgs &a)
{
    a.vol = j.vol->data;
    a.cells = j.vol->use_cells ? j.vol->cells : nullptr;
    a.nx = j.vol->nx;
    a.ny = j.vol->ny;
    a.nz = j.vol->nz;
    a.value_lo = j.vol->value_lo;
    a.s = (float)(j.tf->nt - 1) / (j.vol->value_hi - j.vol->value_lo);
    a.cell_last = (uint32_t)((size_t)(j.vol->nx + 1) * (j.vol->ny + 1) * (j.vol->nz + 1) - 1);
    a.cs_y = (uint32_t)(j.vol->nx + 1);
    a.cs_z = (uint32_t)((j.vol->nx + 1) * (j.vol->ny + 1));
    a.c_base = a.cs_z + a.cs_y + 1;
    a.c_base_m = a.c_base - 0x4b400000u * (a.cs_z + a.cs_y + 1u);
    a.tf = j.tf->lut;
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
    a.dda_inc = grid_dda_inc(j) ? 1 : 0;
    a.nodes = j.st->nodes;
    a.root = j.st->root;
    a.count = (j.st->kind == ESS_KD || j.st->kind == ESS_HYBRID) ? j.st->kd_count_dev : j.st->count;
    a.samples = c.samples;
    a.shade = j.rp.shading;
    a.shin = j.rp.shininess;
    a.ka = j.rp.ka;
    a.kd = j.rp.kd;
    a.ks = j.rp.ks;
    a.op_r = j.rp.dt_ref > 0.0f ? j.rp.dt / j.rp.dt_ref : 0.0f;
}

// The shaded variant: shading on, or an opacity correction that changes alpha.
bool render_shaded(const ess_render_params &rp)
{
    return rp.shading != 0 || (rp.dt_ref > 0.0f && rp.dt / rp.dt_ref != 1.0f);
}

static const char *render_name(int kind, bool shaded)
{
    switch (kind) {
    case ESS_NONE: return shaded ? "render_shaded_naive" : "render_naive";
    case ESS_GRID: return shaded ? "render_shaded_grid" : "render_grid";
    case ESS_LBVH: return shaded ? "render_shaded_lbvh" : "render_lbvh";
    case ESS_HYBRID: return shaded ? "render_shaded_hybrid" : "render_hybrid";
    default: return shaded ? "render_shaded_kd" : "render_kd";
    }
}

static int tile_width(int w)
{
    return (w == 4 || w == 8 || w == 16 || w == 32) ? w : 8;
}

void launch_render(Ctx &c, const RenderJob &j)
{
    RArgs a;
    fill_args(c, j, a);
    int tw = tile_width(j.tile_w);
    Launch L(c, render_name(j.st->kind, render_shaded(j.rp)));
    if (render_shaded(j.rp)) launch_render_kernels<1>(c, a, j.st->kind, j.vol->dtype, tw);
    else launch_render_kernels<0>(c, a, j.st->kind, j.vol->dtype, tw);
}

// ------------------------------------------------------------ batched path
size_t batch_args_bytes() { return sizeof(RArgs); }

// Batch layout (fixed offsets, so that a captured launch stays valid for any
// item count): header, tile prefix (BATCH_MAX + 1 ints, 16-byte padded), then
// BATCH_MAX RArgs.
static size_t batch_prefix_bytes() { return ((sizeof(int) * (BATCH_MAX + 1)) + 15) & ~(size_t)15; }

size_t batch_bytes(int n) { return sizeof(BatchHeader) + batch_prefix_bytes() + sizeof(RArgs) * n; }

// Packs the jobs of one (dtype, kind) group into `host` (pinned).  Returns the
// number of bytes to copy to the device.
size_t pack_batch(Ctx &c, const RenderJob *jobs, int n, int tw, void *host, size_t cap)
{
    size_t prefix_bytes = batch_prefix_bytes();
    size_t need = batch_bytes(n);
    if (need > cap) throw Error{ESS_ERR_ARG, "render batch too large for the staging buffer"};
    char *p = (char *)host;
    BatchHeader *h = (BatchHeader *)p;
    int *prefix = (int *)(p + sizeof(BatchHeader));
    RArgs *args = (RArgs *)(p + sizeof(BatchHeader) + prefix_bytes);
    int bw = 2 * tw, bh = 64 / tw;
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        prefix[i] = acc;
        acc += ((jobs[i].W + bw - 1) / bw) * ((jobs[i].H + bh - 1) / bh);
        fill_args(c, jobs[i], args[i]);
    }
    prefix[n] = acc;
    h->nitems = n;
    h->total_tiles = acc;
    h->tile_counter = 0;
    h->tw = tw;
    return need;
}

// Persistent launch over a packed batch already copied to `dev` (same
// layout).
void launch_render_batch(Ctx &c, int kind, ess_dtype dt, bool cells, bool shaded, bool dda_inc,
                         void *dev)
{
    size_t prefix_bytes = batch_prefix_bytes();
    char *p = (char *)dev;
    BatchHeader *h = (BatchHeader *)p;
    const int *prefix = (const int *)(p + sizeof(BatchHeader));
    const RArgs *args = (const RArgs *)(p + sizeof(BatchHeader) + prefix_bytes);
    if (shaded) launch_batch_kernels<1>(c, kind, dt, cells, dda_inc, args, prefix, h);
    else launch_batch_kernels<0>(c, kind, dt, cells, dda_inc, args, prefix, h);
}

template void launch_render_kernels<0>(Ctx &, const RArgs &, int, ess_dtype, int);
template void launch_batch_kernels<0>(Ctx &, int, ess_dtype, bool, bool, const RArgs *, const int *,
                                      BatchHeader *);

}  // namespace ess
