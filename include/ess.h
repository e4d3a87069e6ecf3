/*
 * ess.h -- C ABI of libess: empty-space-skipping volume rendering on one
 * NVIDIA GB300 (CUDA, sm_103a).
 *
 * The calls follow the problem statement of Zellmann, "Comparing Hierarchical
 * Data Structures for Sparse Volume Rendering with Empty Space Skipping"
 * (arXiv 1912.09596): a user edits the colour/alpha transfer function (TF),
 * which changes which parts of the volume are empty, so a skipping index is
 * rebuilt and the volume is ray-marched through it again (Sec. 1; Sec. 2
 * contrasts this rebuild-per-change approach with updating an index).  Three index kinds are built (Sec. 3): a uniform macrocell grid
 * (the baseline of Sec. 1 and 2), an LBVH over non-empty bricks (Sec. 3.1) and
 * a k-d tree (Sec. 3.2).  Rendering is absorption plus emission with
 * post-classification TF lookups (Sec. 4.1).
 *
 * Conventions
 *  - Every call returns an ess_status; no C++ exception crosses the ABI.  On
 *    failure ess_last_error() describes the cause.
 *  - Inputs are copied: the caller keeps ownership of every input buffer and
 *    may free or reuse it as soon as the call returns.
 *  - Output images are caller-owned float32 RGBA buffers, W*H*4 floats, row
 *    major, row 0 at the top.  `out_on_device` says whether `out` is device
 *    memory (written asynchronously on the context stream) or host memory
 *    (the call returns when the image is there: pinned memory that the
 *    context's device can address is written by the render kernel itself,
 *    other host memory through a device staging buffer and a copy).
 *  - Device memory that the library allocates belongs to the context and is
 *    returned by ess_release() / ess_destroy().
 *  - Work is issued asynchronously on the context's CUDA stream, in call
 *    order, except builds and rebuilds: they run on an internal stream of the
 *    highest priority, each after the last render of its structure and the
 *    last updates of its TF and volume, so that a rebuild overlaps the
 *    rendering of other structures.  Every later call that uses the structure
 *    (render, batched render, read, info, release) and every TF update waits
 *    for them on the context stream, so results are those of call order.
 *    ess_sync() waits for all of it and reports device-side errors.
 *  - A context is used by one host thread at a time.
 *  - World units are voxels: the volume box is [0,nx] x [0,ny] x [0,nz] and
 *    voxel (i,j,k) has its centre at (i+0.5, j+0.5, k+0.5).
 */
#ifndef ESS_H
#define ESS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ess_ctx ess_ctx;  /* opaque */
typedef uint64_t ess_handle;     /* volume, TF or structure; 0 is invalid */

typedef enum {
    ESS_OK = 0,
    ESS_ERR_ARG = -1,      /* invalid argument (message says which) */
    ESS_ERR_OOM = -2,      /* device allocation failed */
    ESS_ERR_CUDA = -3,     /* CUDA runtime error */
    ESS_ERR_HANDLE = -4,   /* unknown, released or wrong-type handle */
    ESS_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    ESS_ERR_BUSY = -6,     /* admission refused (memory budget) */
    ESS_ERR_STALE = -7     /* structure built for an older TF: rebuild it */
} ess_status;

typedef enum { ESS_U8 = 0, ESS_U16 = 1, ESS_F32 = 2 } ess_dtype;

typedef enum {
    ESS_GRID = 0,  /* uniform macrocell grid = the brick mask (Sec. 1, 2) */
    ESS_LBVH = 1,  /* LBVH over non-empty bricks (Sec. 3.1) */
    ESS_KD = 2,    /* k-d tree with tight boxes (Sec. 3.2) */
    ESS_NONE = 3,  /* no skipping: naive ray marching (Table 2, "Naive") */
    ESS_HYBRID = 4 /* hybrid grid (Sec. 3.3): a k-d tree (the paper's is shallow,
                      halting 0) whose leaves are crossed with the macrocell grid
                      of the same brick size */
} ess_kind;

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`.  `cuda_stream` is the
 * cudaStream_t to issue all work on (e.g. PyTorch's current stream); NULL
 * means the CUDA default stream.  The caller keeps ownership of the stream. */
ess_status ess_create(int device, void *cuda_stream, ess_ctx **out);

/* Waits for outstanding work and frees everything the context owns. */
ess_status ess_destroy(ess_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  Valid until
 * the next call on the context. */
const char *ess_last_error(const ess_ctx *ctx);

/* Waits for all work issued on the context; returns a device-side error
 * recorded since the last ess_sync (e.g. ESS_ERR_TIMEOUT), else ESS_OK. */
ess_status ess_sync(ess_ctx *ctx);

/* Releases a volume, TF or structure handle and its device memory.  A volume
 * or TF still used by a live structure is kept until that structure goes. */
ess_status ess_release(ess_ctx *ctx, ess_handle h);

/* ----------------------------------------------------------------- inputs */

/* Uploads a structured scalar volume (Sec. 4.2: uniform grids, in-core),
 * `data` = nz*ny*nx voxels of `dtype`, x fastest.  `data_on_device` says
 * whether `data` is device or host memory.  [value_lo, value_hi] is the value
 * range mapped onto the TF (TF coordinate x = (v - value_lo) * (NT-1) /
 * (value_hi - value_lo), clamped).  The call copies the data, so the caller
 * keeps ownership.  Errors: ESS_ERR_ARG for a non-positive size, more than
 * 8192 voxels on an axis, value_hi <= value_lo, or (f32) a NaN or infinite
 * voxel; ESS_ERR_OOM if the copy does not fit. */
ess_status ess_volume_upload(ess_ctx *ctx, const void *data, int data_on_device,
                             ess_dtype dtype, int nx, int ny, int nz,
                             float value_lo, float value_hi, ess_handle *vol);

/* Chooses how renders read voxels (the image is the same either way):
 * cells = 1 keeps a corner-replicated copy of the volume, (nx+1)(ny+1)(nz+1)
 * cells of the 8 clamped voxels one trilinear sample interpolates (8x the
 * volume's bytes; one vector load per sample); cells = 0 drops that copy and
 * reads the 8 voxels from the volume itself.  ess_volume_upload keeps the copy
 * when it fits in half of the free device memory and has fewer than 2^32 cells
 * (about 1625^3 voxels; the renderer indexes cells with 32-bit integers);
 * ESS_ERR_ARG for cells = 1 on a larger volume. */
ess_status ess_volume_set_sampler(ess_ctx *ctx, ess_handle vol, int cells);

/* Sets an RGBA transfer function of `nt` entries (Sec. 1: the colour and
 * alpha TF that maps scalar values to colour and opacity), `rgba` = nt*4
 * floats, entry-major.  Alpha must lie in [0, 1] and every value must be
 * finite, 2 <= nt <= 65536.  Copies the table.  A host table is checked
 * before the call returns (ESS_ERR_ARG); a device table is checked on the
 * device and a bad one is reported by the next ess_sync (ESS_ERR_ARG). */
ess_status ess_tf_set(ess_ctx *ctx, const float *rgba, int on_device, int nt,
                      ess_handle *tf);

/* Replaces the table of an existing TF in place (a TF edit, Sec. 1).  `nt`
 * must equal the TF's size.  Structures built with the previous table become
 * stale: ess_render on them returns ESS_ERR_STALE until ess_rebuild. */
ess_status ess_tf_update(ess_ctx *ctx, ess_handle tf, const float *rgba, int on_device,
                         int nt);

/* -------------------------------------------------------------- structures */

typedef struct {
    int brick;   /* brick / macrocell edge B in voxels, 2..64 (Sec. 3.1: 8^3
                    leaves; Sec. 3.2.2: 8^3 macro cells) */
    int nbins;   /* k-d candidate planes per axis: 0 = every brick boundary
                    (exhaustive, the CPU builder), else nbins - 1 binned
                    planes (Sec. 3.2.2; 4 in Sec. 4.3) */
    int halting; /* k-d halting (Sec. 4.3): 0 = shallow (split while the node
                    volume is above 10 % of the root volume), 1 = deep (split
                    while above 8^3 voxels) */
    int mls;     /* k-d maximum leaf size (Sec. 4.3) as an edge in voxels
                    (32 or 128 in the paper), 0 = none */
    int empty_test; /* 0 = brick min/max range test (Sec. 2, min-max range
                    queries), 1 = exact per-cell vote (Sec. 3.1 classifies per
                    voxel): a brick is non-empty iff one of the trilinear
                    cells whose samples touch it passes the range test of its
                    8 corner voxels; evaluated on the bricks the min/max test
                    passes (it never marks another) */
    int rescan;  /* 1 = recompute the per-brick min/max
                    from the voxels once per TF edit (a full pass over the
                    volume per edit, as when bricks are classified from their
                    voxels after each edit, Sec. 3.1): the first build or
                    rebuild of a (volume, brick size) after any TF upload of
                    the context reads the volume, and the structures rebuilt
                    after it for the same edit reuse that pass; 0 = compute it
                    once per volume and brick size and reuse it (it does not
                    depend on the TF).  Both give the same mask. */
} ess_build_params;

/* Builds a skipping structure of `kind` for volume `vol` under TF `tf`
 * (Sec. 3).  For ESS_NONE no index is built; the handle just binds the
 * volume and the TF for naive rendering.  ESS_HYBRID runs the k-d build with
 * `params` and keeps the brick mask as its global grid.  The structure keeps references to
 * `vol` and `tf`.  Asynchronous, except the k-d build with exhaustive planes
 * (nbins 0), which reads back the size of each tree level.  Errors:
 * ESS_ERR_ARG for bad parameters, ESS_ERR_HANDLE for bad handles,
 * ESS_ERR_OOM. */
ess_status ess_build(ess_ctx *ctx, ess_handle vol, ess_handle tf, ess_kind kind,
                     const ess_build_params *params, ess_handle *structure);

/* Rebuilds `structure` for the current table of its TF (after ess_tf_update)
 * reusing its device memory: the per-edit hot path of Sec. 1. */
ess_status ess_rebuild(ess_ctx *ctx, ess_handle structure);

/* Rebuilds `count` distinct structures (1 <= count <= 4096), e.g. one per TF
 * of a batch of many TFs over one volume, with the same results as calling
 * ess_rebuild on each.  Together: the per-brick min/max of structures built
 * with rescan = 1 is recomputed once per (volume, brick size) of the batch
 * (and not at all where this TF edit's pass already ran), not once per
 * structure, and the structures' build chains run on several
 * internal streams at once, so that their latency-bound kernels overlap.
 * Asynchronous; later users of each structure wait for its build as usual.
 * ESS_ERR_ARG for a repeated handle, ESS_ERR_HANDLE for a bad one. */
ess_status ess_rebuild_batch(ess_ctx *ctx, const ess_handle *structures, int count);

typedef struct {
    int kind, brick;
    int gx, gy, gz;          /* brick grid = ceil(n / brick) per axis */
    int64_t n_bricks;        /* gx*gy*gz */
    int64_t n_nonempty;      /* non-empty bricks after the empty test */
    int64_t n_nodes;         /* LBVH: 2n-1 (0 if n = 0); k-d: node count */
    int height;              /* tree levels including root and leaves */
    size_t device_bytes;     /* device memory held by the structure */
} ess_structure_info;

/* Fills `info` (waits for the structure's build to finish). */
ess_status ess_structure_info_get(ess_ctx *ctx, ess_handle structure,
                                  ess_structure_info *info);

typedef enum {
    ESS_ARR_MINMAX = 0,      /* float32 [n_bricks][2]: apron min, max */
    ESS_ARR_MASK = 1,        /* uint8  [n_bricks]: 1 = non-empty */
    ESS_ARR_IDS = 2,         /* uint32 [n_nonempty]: non-empty brick ids, ascending */
    ESS_ARR_KEYS = 3,        /* uint32 [n_nonempty]: Morton code of IDS[i] */
    ESS_ARR_SORTED_KEYS = 4, /* uint32 [n_nonempty]: keys after the radix sort */
    ESS_ARR_SORTED_IDS = 5,  /* uint32 [n_nonempty]: ids in sorted-key order */
    ESS_ARR_LBVH_LEFT = 6,   /* int32 [n_nonempty-1]: left child (>= 0 inner,
                                -1-j leaf j of the sorted order) */
    ESS_ARR_LBVH_RIGHT = 7,  /* int32 [n_nonempty-1]: right child, same coding */
    ESS_ARR_LBVH_BOXES = 8,  /* int32 [n_nonempty-1][6]: inner box lo xyz, hi xyz
                                in brick coordinates, hi exclusive */
    ESS_ARR_KD_NODES = 9     /* int32 [n_nodes][9]: lo xyz, hi xyz (bricks, hi
                                exclusive), axis (-1 leaf), plane, first child
                                (-1 leaf); breadth-first, left child first */
} ess_array;

/* Copies one array of a built structure to host memory `dst` of
 * `capacity` bytes; `*written` receives the byte count.  Synchronous.
 * ESS_ERR_ARG if the array does not exist for the structure's kind or does
 * not fit. */
ess_status ess_structure_read(ess_ctx *ctx, ess_handle structure, ess_array which,
                              void *dst, size_t capacity, size_t *written);

/* ------------------------------------------------------------------ render */

typedef struct {
    float eye[3];  /* perspective: ray origin; orthographic: view centre */
    float u[3];    /* right, scaled: perspective tan(fov/2)*aspect, ortho half width */
    float v[3];    /* up, scaled: perspective tan(fov/2), ortho half height */
    float w[3];    /* forward (normalised before use) */
    int ortho;     /* 1 = orthographic (Sec. 4.1), 0 = perspective */
} ess_camera;   /* finite; |eye[i]| + |u[i]| + |v[i]| <= 65536 voxels per axis */

typedef struct {
    float dt;     /* step between samples in voxels, 1e-3 <= dt <= 1e4 */
    float ert;    /* early ray termination: stop once opacity >= ert; a value
                     above 1 disables it (the paper's benchmarks, Sec. 4.1) */
    float bg[4];  /* background RGBA composited behind the volume */
    int tile_w;   /* warp tile width in pixels: 4, 8, 16 or 32 (0 = 8); the
                     warp covers tile_w x (32 / tile_w) pixels.  Does not
                     change the image. */
    /* Second render workload (the paper switches both off, Sec. 4.1).
     * Gradient shading: the gradient is the central difference of the
     * trilinear reconstruction one voxel apart on each axis; samples of
     * non-zero opacity get two-sided Blinn-Phong under a headlight,
     * rgb' = rgb (ka + kd c) + ks c^shininess with c = min(|n . d|, 1),
     * n = g / |g| (a zero gradient leaves rgb).  Zero-initialised fields give
     * the unshaded renderer. */
    int shading;       /* 0 off, 1 on */
    float ka, kd, ks;  /* finite, >= 0 (used when shading is on) */
    int shininess;     /* 1..128 (used when shading is on) */
    /* Opacity correction: the TF's alpha holds for a step of dt_ref voxels;
     * a sample taken every dt voxels gets 1 - (1 - alpha)^(dt / dt_ref).
     * 0 switches it off; otherwise finite, > 0. */
    float dt_ref;
} ess_render_params;

/* Ray-marches `structure` (Sec. 4.1: absorption plus emission,
 * post-classification) into a W x H RGBA image.  Pixel (x, y) shoots the ray
 * through sx = (2x+1)/W - 1, sy = 1 - (2y+1)/H; samples sit at
 * t_k = t_near + k*dt on every path; skipping drops only samples of zero
 * opacity, so the image equals naive marching, with or without gradient
 * shading and opacity correction (both leave zero opacity at zero).
 * ESS_ERR_STALE if the TF was updated after the build; ESS_ERR_ARG for
 * parameters outside the ranges stated above. */
ess_status ess_render(ess_ctx *ctx, ess_handle structure, const ess_camera *camera,
                      const ess_render_params *params, int W, int H, float *out,
                      int out_on_device);

/* ----------------------------------------------------------------- batched */

typedef struct {
    ess_handle structure;      /* built structure (its volume and TF) */
    ess_camera camera;
    ess_render_params params;  /* tile_w is taken from the batch call */
    int W, H;
    float *out;                /* device memory, W*H*4 floats, caller-owned */
} ess_render_item;

/* Renders `count` images in one persistent launch per (volume dtype,
 * structure kind) group: blocks take 128-pixel tiles of all images from one
 * work counter, so many TFs, views and uneven image sizes share the GPU.  The
 * launch is captured once as a CUDA graph and replayed.  Every image equals
 * what ess_render gives for the same item, bit for bit.  Asynchronous on the
 * context stream; 1 <= count <= 4096.  ESS_ERR_STALE if any structure's TF
 * was updated after its build. */
ess_status ess_render_batch(ess_ctx *ctx, const ess_render_item *items, int count, int tile_w);

/* ------------------------------------------------------------------ tuning */

typedef struct {
    int kind;      /* ESS_GRID, ESS_LBVH, ESS_KD or ESS_HYBRID */
    int brick;     /* brick edge */
    int tile_w;    /* warp tile width for ess_render_params.tile_w */
    float build_ms, render_ms;  /* measured: one rebuild, mean of one frame per camera */
} ess_tune_result;

/* Autotuner: builds every candidate structure kind x brick size (4, 8, 16, 32;
 * k-d deep, 4 bins, maximum leaf 32^3) for `vol` and `tf`, renders the
 * `ncam` cameras with every warp tile width, and returns the candidate with
 * the least build_ms + frames_per_edit * render_ms (CUDA-event times).
 * Synchronous; the candidate structures are released again. */
ess_status ess_autotune(ess_ctx *ctx, ess_handle vol, ess_handle tf, const ess_camera *cameras,
                        int ncam, const ess_render_params *params, int W, int H,
                        float frames_per_edit, ess_tune_result *best);

/* ----------------------------------------------------------------- serving */

typedef struct ess_server ess_server;  /* opaque */

typedef struct {
    size_t memory_budget;  /* device bytes for the outputs of admitted requests
                              (0: a quarter of the free memory at creation) */
    int max_batch;         /* renders per batched launch, 1..4096 */
    int max_inflight;      /* batches on the GPU at once, 1..64 */
    int tile_w;            /* warp tile width of the batched launches (0 = 8) */
} ess_server_config;

typedef enum {
    ESS_REQ_RENDER = 0,  /* render a view of a structure */
    ESS_REQ_EDIT = 1     /* replace the structure's TF, rebuild it, then render */
} ess_request_kind;

typedef struct {
    int kind;                  /* ess_request_kind */
    ess_handle structure;
    const float *rgba;         /* ESS_REQ_EDIT: new table, host memory, nt x 4,
                                  copied by ess_server_submit */
    int nt;
    ess_camera camera;
    ess_render_params params;
    int W, H;
    float *out;                /* host memory for the W*H*4 float image; it must
                                  stay valid until the request is done */
} ess_request;

typedef struct {
    int done;            /* 1 once the image is in `out` */
    ess_status status;   /* result of the request */
    double queue_ms;     /* submission to launch */
    double latency_ms;   /* submission to the image in host memory */
} ess_request_status;

/* Starts a request loop on `ctx` (the paper's interactive use, Sec. 1: views
 * and TF edits of resident volumes).  A worker thread admits queued requests
 * in arrival order into batches while their output memory fits the budget,
 * applies the batch's edits (TF upload + rebuild), renders the batch in one
 * persistent launch and copies each image to its host buffer (a pinned
 * buffer the device can address is written by the render itself); up to
 * max_inflight batches run on the GPU while the next one is admitted.  Each
 * image equals what ess_render gives for the request alone.  While the server
 * runs, the context must not be used directly; destroy the server before the
 * context.  A request larger than the whole budget ends with ESS_ERR_BUSY. */
ess_status ess_server_create(ess_ctx *ctx, const ess_server_config *cfg, ess_server **out);

/* Queues a request (thread-safe); `*id` identifies it.  ESS_ERR_ARG for a bad
 * request, ESS_ERR_BUSY after the server began to stop. */
ess_status ess_server_submit(ess_server *s, const ess_request *req, uint64_t *id);

/* Reports a request's state without waiting / after waiting for it. */
ess_status ess_server_poll(ess_server *s, uint64_t id, ess_request_status *st);
ess_status ess_server_wait(ess_server *s, uint64_t id, ess_request_status *st);

/* Waits until every submitted request is done. */
ess_status ess_server_drain(ess_server *s);

/* Finishes all submitted requests, stops the worker and frees the server. */
ess_status ess_server_destroy(ess_server *s);

/* ------------------------------------------------------ allocation-free */

/* Brick compaction without any allocation: writes to `ids` the indices of the
 * non-zero bytes of the device byte mask `mask` (n_bricks bytes), in
 * increasing order, and their number to the device int `*count`; the same
 * result as the ids (ESS_ARR_IDS) that ess_build keeps for the mask it
 * computes.  The paper has no counterpart: this is for callers that cannot
 * allocate device memory (their memory is pre-reserved by another allocator,
 * or a cudaMalloc would stall their frame loop).  All pointers are device
 * memory owned by the caller; `ids` must hold n_bricks uint32 values.  Work is
 * queued on `cuda_stream` (NULL: the default stream) and the call returns
 * without waiting.  The only scratch is a 16 KiB file-scope device array,
 * allocated when the library is loaded and kept on every GPU that loads it;
 * the first call on a device looks up its address, so make that first call
 * before any stream capture.  All calls share that array: calls whose work
 * overlaps on the GPU race and must be serialised by the caller.
 * Errors: ESS_ERR_ARG for n_bricks < 0 or above 16,777,216 (4096 tiles of
 * 4096 flags) or a null pointer; ESS_ERR_CUDA if a launch fails.  No
 * ess_last_error message (there is no context). */
ess_status ess_compact_mask_noalloc(const uint8_t *mask, int64_t n_bricks, uint32_t *ids,
                                    int *count, void *cuda_stream);

/* -------------------------------------------------------------- profiling */

/* Number of ray samples evaluated (classified and composited) by all renders
 * on the context since it was created or last reset; waits for the work. */
ess_status ess_sample_count(ess_ctx *ctx, uint64_t *samples, int reset);

/* Kernel launch counter: number of CUDA kernels this context has launched. */
uint64_t ess_launch_count(const ess_ctx *ctx);

/* Per-kernel timing with CUDA events on the context stream (off by default).
 * While enabled, every launch is bracketed by events; ess_profile_read
 * syncs, accumulates and returns, for each kernel name seen, its launch count
 * and total milliseconds.  `names` receives up to `max` pointers to static
 * strings. */
ess_status ess_profile_enable(ess_ctx *ctx, int enable);
ess_status ess_profile_read(ess_ctx *ctx, int max, const char **names,
                            uint64_t *launches, double *total_ms, int *count);
ess_status ess_profile_reset(ess_ctx *ctx);

/* ----------------------------------------------------------- diagnostics */

/* Failure-detection check of the device-side waits.  Every wait of the
 * library's kernels on another block (the radix sort's look-back) is bounded:
 * after a fixed number of polls the kernel records a timeout in the context's
 * status word, stops waiting and returns, and the next ess_sync reports
 * ESS_ERR_TIMEOUT while the context stays usable.  This call runs that same
 * bounded wait in one warp on a device flag: with `set` = 1 the flag is set
 * first and the wait ends at once; with `set` = 0 nothing sets it and the wait
 * gives up after `polls` polls (1 <= polls <= 2^24).  Asynchronous on the
 * context stream. */
ess_status ess_selftest_wait(ess_ctx *ctx, int set, int64_t polls);

#ifdef __cplusplus
}
#endif

#endif /* ESS_H */
