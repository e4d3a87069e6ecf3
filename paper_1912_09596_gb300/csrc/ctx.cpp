// ctx.cpp -- host orchestration behind the C ABI of include/ess.h: context,
// handles, stream-ordered device memory, input validation, build dispatch,
// render dispatch, read-back and profiling.  All device work goes to the
// context stream; nothing here computes on the CPU what a kernel computes.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "ess_internal.h"

namespace ess {

// ------------------------------------------------------------ memory, events
void *Ctx::alloc(size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{ESS_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
    }
    return p;
}

void Ctx::free(void *p)
{
    if (p) cudaFreeAsync(p, stream);
}

cudaEvent_t Ctx::event()
{
    if (!free_events.empty()) {
        cudaEvent_t e = free_events.back();
        free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    ESS_CUDA(cudaEventCreate(&e));
    return e;
}

void Ctx::begin(const char *name)
{
    ++launches;
    current = name;
    if (profiling) {
        cur_a = event();
        cudaEventRecord(cur_a, stream);
    }
}

void Ctx::end()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        throw Error{ESS_ERR_CUDA, std::string("launch of ") + (current ? current : "?") + ": " +
                                      cudaGetErrorString(e)};
    if (profiling && current) {
        cudaEvent_t b = event();
        cudaEventRecord(b, stream);
        pending.push_back({current, cur_a, b});
    }
    current = nullptr;
}

void mark(Ctx &c, cudaEvent_t &e)
{
    if (!e) ESS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ESS_CUDA(cudaEventRecord(e, c.stream));
}

// The context stream waits for the structure's last build.
void join_build(Ctx &c, Structure &s)
{
    if (!s.build_pending) return;
    ESS_CUDA(cudaStreamWaitEvent(c.stream, s.built, 0));
    s.build_pending = false;
}

// The context stream waits for every build enqueued so far (before writing
// what builds read: TF tables, the cell copy; and before reading the status
// word or profiling events).
void join_all_builds(Ctx &c)
{
    if (!c.build_stream) return;
    ESS_CUDA(cudaEventRecord(c.fork_event, c.build_stream));
    ESS_CUDA(cudaStreamWaitEvent(c.stream, c.fork_event, 0));
    for (cudaStream_t st : c.batch_streams) {
        ESS_CUDA(cudaEventRecord(c.fork_event, st));
        ESS_CUDA(cudaStreamWaitEvent(c.stream, c.fork_event, 0));
    }
    for (auto &kv : c.structures) kv.second->build_pending = false;
}

}  // namespace ess

using namespace ess;

namespace {

enum : uint64_t { TAG_VOL = 1, TAG_TF = 2, TAG_ST = 3 };

ess_handle new_handle(Ctx &c, uint64_t tag) { return (tag << 56) | (c.next_handle++); }

template <typename F> ess_status guard(ess_ctx *ctx, F &&f)
{
    if (!ctx) return ESS_ERR_ARG;
    Ctx &c = ctx->c;
    c.last_error.clear();
    try {
        ESS_CUDA(cudaSetDevice(c.device));
        f(c);
        return ESS_OK;
    } catch (const Error &e) {
        c.last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        c.last_error = "host allocation failed";
        return ESS_ERR_OOM;
    } catch (...) {
        c.last_error = "unexpected internal error";
        return ESS_ERR_CUDA;
    }
}

Volume &get_vol(Ctx &c, ess_handle h)
{
    auto it = c.volumes.find(h);
    if (it == c.volumes.end() || it->second->released)
        throw Error{ESS_ERR_HANDLE, "unknown volume handle"};
    return *it->second;
}

TF &get_tf(Ctx &c, ess_handle h)
{
    auto it = c.tfs.find(h);
    if (it == c.tfs.end() || it->second->released) throw Error{ESS_ERR_HANDLE, "unknown TF handle"};
    return *it->second;
}

Structure &get_st(Ctx &c, ess_handle h)
{
    auto it = c.structures.find(h);
    if (it == c.structures.end() || it->second->released)
        throw Error{ESS_ERR_HANDLE, "unknown structure handle"};
    return *it->second;
}

size_t dtype_size(ess_dtype d) { return d == ESS_U8 ? 1 : (d == ESS_U16 ? 2 : 4); }

// Reads and clears the device status word (synchronises the stream).
ess_status take_status(Ctx &c, std::string &msg)
{
    join_all_builds(c);
    ESS_CUDA(cudaMemcpyAsync(c.host_status, c.dev_status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             c.stream));
    ESS_CUDA(cudaStreamSynchronize(c.stream));
    uint32_t s = *c.host_status;
    if (!s) return ESS_OK;
    ESS_CUDA(cudaMemsetAsync(c.dev_status, 0, sizeof(uint32_t), c.stream));
    if (s & DEV_ERR_TIMEOUT) {
        msg = "a bounded device-side wait gave up";
        return ESS_ERR_TIMEOUT;
    }
    if (s & DEV_ERR_OVERFLOW) {
        msg = "a device buffer reached its capacity";
        return ESS_ERR_ARG;
    }
    if (s & DEV_ERR_BAD_TF) {
        msg = "a TF table from device memory held a non-finite value or an alpha outside [0, 1]";
        return ESS_ERR_ARG;
    }
    msg = "volume holds a NaN or infinite value";
    return ESS_ERR_ARG;
}

void check_tf_host(const float *rgba, int nt)
{
    for (int i = 0; i < 4 * nt; ++i) {
        float v = rgba[i];
        if (!std::isfinite(v)) throw Error{ESS_ERR_ARG, "TF holds a NaN or infinite value"};
        if ((i & 3) == 3 && (v < 0.0f || v > 1.0f))
            throw Error{ESS_ERR_ARG, "TF alpha outside [0, 1]"};
    }
}

// Copies a TF table into `t` and recomputes its prefix counts.  A host table
// is validated on the host and staged through pinned memory (the caller's
// buffer is free on return and the copy stays asynchronous); a device table is
// copied device to device and validated by the prefix kernel, which reports a
// bad table at the next ess_sync.
void load_tf(Ctx &c, TF &t, const float *rgba, int on_device)
{
    size_t bytes = (size_t)t.nt * 4 * sizeof(float);
    if (on_device) {
        ESS_CUDA(cudaMemcpyAsync(t.table, rgba, bytes, cudaMemcpyDeviceToDevice, c.stream));
    } else {
        check_tf_host(rgba, t.nt);
        const int k = t.stage_next;
        if (!t.staging[k]) ESS_CUDA(cudaMallocHost(&t.staging[k], bytes));
        if (t.staged[k]) ESS_CUDA(cudaEventSynchronize(t.staged[k]));
        std::memcpy(t.staging[k], rgba, bytes);
        ESS_CUDA(cudaMemcpyAsync(t.table, t.staging[k], bytes, cudaMemcpyHostToDevice, c.stream));
        if (!t.staged[k]) ESS_CUDA(cudaEventCreateWithFlags(&t.staged[k], cudaEventDisableTiming));
        ESS_CUDA(cudaEventRecord(t.staged[k], c.stream));
        t.stage_next = (k + 1) % STAGE_RING;
    }
    // entry nt repeats entry nt-1 so that the renderer's upper neighbour needs no clamp
    ESS_CUDA(cudaMemcpyAsync(t.table + t.nt, t.table + (t.nt - 1), sizeof(float4),
                             cudaMemcpyDeviceToDevice, c.stream));
    launch_tf_prefix(c, t.table, t.nt, t.prefix, t.lut, on_device);
    mark(c, t.updated);
    ++t.version;
    ++c.edit_epoch;
}

// Builds (mode 1) or drops (mode 0) the corner-replicated cell copy.
// The renderer indexes cells with 32-bit integers.
bool cells_indexable(const Volume &v)
{
    return (uint64_t)(v.nx + 1) * (uint64_t)(v.ny + 1) * (uint64_t)(v.nz + 1) <= 0xffffffffull;
}

void set_sampler(Ctx &c, Volume &v, int mode)
{
    if (mode == 1) {
        ESS_REQUIRE(cells_indexable(v),
                    "the cell sampler needs (nx+1)(ny+1)(nz+1) < 2^32 (about 1625^3 voxels)");
        if (!v.cells) {
            v.cell_bytes = cell_array_bytes(v);
            v.cells = c.alloc(v.cell_bytes);
            launch_build_cells(c, v, v.cells);
        }
        v.use_cells = true;
    } else {
        c.free(v.cells);
        v.cells = nullptr;
        v.cell_bytes = 0;
        v.use_cells = false;
    }
}

// Per-brick min/max of volume v for brick size B, computed on first use and
// kept with the volume.  `rescan` recomputes a kept one, as the paper's
// classification reads the volume on every TF edit (Sec. 3.1), but only once
// per edit: the structures rebuilt for the same edit share the pass (the
// values are TF-independent, so any pass gives the same bits).
float2 *minmax_for(Ctx &c, Volume &v, int B, bool rescan)
{
    auto it = v.minmax.find(B);
    if (it != v.minmax.end()) {
        if (rescan && v.scan_epoch[B] != c.edit_epoch) {
            launch_brick_minmax(c, v, B, it->second);
            v.scan_epoch[B] = c.edit_epoch;
        }
        return it->second;
    }
    int gx = (v.nx + B - 1) / B, gy = (v.ny + B - 1) / B, gz = (v.nz + B - 1) / B;
    float2 *mm = (float2 *)c.alloc(sizeof(float2) * (size_t)gx * gy * gz);
    launch_brick_minmax(c, v, B, mm);
    v.minmax[B] = mm;
    v.scan_epoch[B] = c.edit_epoch;
    return mm;
}

void free_structure(Ctx &c, Structure &s)
{
    join_build(c, s);
    void *ptrs[] = {s.mask, s.ids, s.count, s.block_sums, s.keys, s.keys_sorted, s.ids_sorted,
                    s.keys_alt, s.ids_alt, s.sort_scratch, s.left, s.right, s.parent,
                    s.leaf_parent, s.inner_box, s.range_end, s.chunk_box, s.nodes, s.root, s.kd_nodes,
                    s.kd_count_dev, s.brick_node, s.kd_scratch_i32, s.kd_state};
    for (void *p : ptrs) c.free(p);
    kd_free(c, s);
    if (s.built) cudaEventDestroy(s.built);
    if (s.used) cudaEventDestroy(s.used);
    s.built = s.used = nullptr;
}

template <typename P> P *alloc_n(Ctx &c, Structure &s, size_t n)
{
    size_t bytes = sizeof(P) * (n ? n : 1);
    s.device_bytes += bytes;
    return (P *)c.alloc(bytes);
}

// Device buffers of an LBVH over up to nb bricks (Sec. 3.1).
void alloc_lbvh(Ctx &c, Structure &s)
{
    size_t cap = (size_t)s.nb, inner = cap > 1 ? cap - 1 : 1;
    s.keys = alloc_n<uint32_t>(c, s, cap);
    s.keys_sorted = alloc_n<uint32_t>(c, s, cap);
    s.ids_sorted = alloc_n<uint32_t>(c, s, cap);
    s.keys_alt = alloc_n<uint32_t>(c, s, cap);
    s.ids_alt = alloc_n<uint32_t>(c, s, cap);
    s.sort_scratch = alloc_n<uint32_t>(c, s, sort_scratch_words(s.nb));
    s.left = alloc_n<int32_t>(c, s, inner);
    s.right = alloc_n<int32_t>(c, s, inner);
    s.parent = alloc_n<int32_t>(c, s, inner);
    s.leaf_parent = alloc_n<int32_t>(c, s, cap);
    s.inner_box = alloc_n<int32_t>(c, s, 6 * inner);
    s.range_end = alloc_n<int32_t>(c, s, inner);
    s.chunk_box = alloc_n<int32_t>(c, s, 6 * lbvh_chunk_boxes(cap));
    s.nodes = alloc_n<BoxNode>(c, s, inner);
    s.root = alloc_n<int32_t>(c, s, 8);
}

// Device buffers of a k-d tree over up to nb bricks (Sec. 3.2): a full binary
// tree whose leaves hold at least one brick has at most 2 nb - 1 nodes.
void alloc_kd(Ctx &c, Structure &s)
{
    size_t cap = (size_t)s.nb;
    s.kd_capacity = (int)std::min<size_t>(2 * cap, (size_t)INT32_MAX / 16);
    s.kd_nodes = alloc_n<int32_t>(c, s, 9 * (size_t)s.kd_capacity);
    s.nodes = alloc_n<BoxNode>(c, s, (size_t)s.kd_capacity);
    s.root = alloc_n<int32_t>(c, s, 8);
    s.kd_count_dev = alloc_n<int>(c, s, 1);
    s.brick_node = alloc_n<int>(c, s, cap);
    s.kd_scratch_i32 = alloc_n<int32_t>(c, s, 8);
    s.kd_state = alloc_n<int32_t>(c, s, 8);
}

// The empty test and compaction (Sec. 3.1), then the kind-specific build.
void run_build(Ctx &c, Structure &s)
{
    Volume &v = get_vol(c, s.vol);
    TF &t = get_tf(c, s.tf);
    int B = s.p.brick;
    float sc = (float)(t.nt - 1) / (v.value_hi - v.value_lo);
    float2 *mm = minmax_for(c, v, B, s.p.rescan == 1);
    launch_brick_mask(c, mm, s.nb, t, v.value_lo, sc, s.mask);
    // the exact per-cell vote clears the range test's bricks that no cell shows
    if (s.p.empty_test == 1) launch_vote_bricks(c, v, B, t, sc, s.mask, s.gx, s.gy, s.gz);
    launch_compact(c, s.mask, s.nb, s.ids, s.count, s.block_sums,
                   s.kind == ESS_LBVH ? s.keys : nullptr, s.gx, s.gy);
    s.n_host = -1;
    s.height = -1;
    if (s.kind == ESS_LBVH) launch_lbvh(c, s);
    if (s.kind == ESS_KD || s.kind == ESS_HYBRID) {
        s.volume = &v;
        launch_kd(c, s);
    }
    s.tf_version = t.version;
}

// Restores the context stream when a build on the build stream ends or throws.
struct OnStream {
    Ctx &c;
    cudaStream_t saved;
    OnStream(Ctx &ctx, cudaStream_t s) : c(ctx), saved(ctx.stream) { c.stream = s; }
    ~OnStream() { c.stream = saved; }
};

// run_build on the build stream, recording `built`; the structure's users
// join it.  A first build starts after everything enqueued on the context
// stream so far (its buffers were just allocated there); a rebuild only after
// the last render of the structure and the last updates of its TF and volume,
// so it can run while the context stream renders other structures.  The build
// stream has the highest priority: the blocks of a rebuild are scheduled ahead
// of those of a render running meanwhile.
void ensure_build_stream(Ctx &c)
{
    if (c.build_stream) return;
    int least = 0, greatest = 0;
    ESS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    ESS_CUDA(cudaStreamCreateWithPriority(&c.build_stream, cudaStreamNonBlocking, greatest));
    ESS_CUDA(cudaEventCreateWithFlags(&c.fork_event, cudaEventDisableTiming));
}

// `st` waits for what a rebuild of `s` must follow: its last render, the last
// updates of its TF and volume, and its previous build (on whichever stream).
void wait_rebuild_deps(Ctx &c, Structure &s, cudaStream_t st)
{
    const cudaEvent_t deps[3] = {s.used, get_tf(c, s.tf).updated, get_vol(c, s.vol).updated};
    for (cudaEvent_t e : deps)
        if (e) ESS_CUDA(cudaStreamWaitEvent(st, e, 0));
    if (s.build_pending) ESS_CUDA(cudaStreamWaitEvent(st, s.built, 0));
}

// run_build on stream `st`, recording `built`.
void build_on(Ctx &c, Structure &s, cudaStream_t st)
{
    if (!s.built) ESS_CUDA(cudaEventCreateWithFlags(&s.built, cudaEventDisableTiming));
    s.build_pending = true;
    try {
        OnStream on(c, st);
        run_build(c, s);
    } catch (...) {
        cudaEventRecord(s.built, st);
        throw;
    }
    ESS_CUDA(cudaEventRecord(s.built, st));
}

void run_build_async(Ctx &c, Structure &s, bool first)
{
    ensure_build_stream(c);
    if (c.batch_streams_pending) {
        // builds of an ess_rebuild_batch may still read (or rescan) the
        // volumes' min/max that this build reads or rescans
        for (cudaStream_t st : c.batch_streams) {
            ESS_CUDA(cudaEventRecord(c.fork_event, st));
            ESS_CUDA(cudaStreamWaitEvent(c.build_stream, c.fork_event, 0));
        }
        c.batch_streams_pending = false;
    }
    if (first) {
        ESS_CUDA(cudaEventRecord(c.fork_event, c.stream));
        ESS_CUDA(cudaStreamWaitEvent(c.build_stream, c.fork_event, 0));
    } else {
        wait_rebuild_deps(c, s, c.build_stream);
    }
    build_on(c, s, c.build_stream);
}

// Streams of ess_rebuild_batch: latency-bound build chains of different
// structures overlap on them.
constexpr int BATCH_BUILD_STREAMS = 8;

int64_t nonempty_count(Ctx &c, Structure &s)
{
    if (s.n_host < 0) {
        int n = 0;
        ESS_CUDA(cudaMemcpyAsync(&n, s.count, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        s.n_host = n;
    }
    return s.n_host;
}

void check_render_args(const ess_camera *camera, const ess_render_params *params, int W, int H)
{
    ESS_REQUIRE(W > 0 && H > 0 && W <= 16384 && H <= 16384, "image size must be in 1..16384");
    ESS_REQUIRE(params->dt >= 1e-3f && params->dt <= 1e4f, "dt must be in [1e-3, 1e4]");
    ESS_REQUIRE(std::isfinite(params->ert), "ert must be finite");
    ESS_REQUIRE(params->tile_w == 0 || params->tile_w == 4 || params->tile_w == 8 ||
                    params->tile_w == 16 || params->tile_w == 32,
                "tile_w must be 0, 4, 8, 16 or 32");
    for (int i = 0; i < 3; ++i)
        ESS_REQUIRE(std::isfinite(camera->eye[i]) && std::isfinite(camera->u[i]) &&
                        std::isfinite(camera->v[i]) && std::isfinite(camera->w[i]),
                    "camera must be finite");
    ESS_REQUIRE(camera->w[0] != 0.0f || camera->w[1] != 0.0f || camera->w[2] != 0.0f,
                "camera needs a non-zero forward vector");
    // ray origins within 2^16 voxels of the volume's corner keep the rounding
    // of sample positions far below half a voxel (the renderer relies on it)
    for (int i = 0; i < 3; ++i)
        ESS_REQUIRE(std::fabs(camera->eye[i]) + std::fabs(camera->u[i]) + std::fabs(camera->v[i]) <=
                        65536.0f,
                    "camera eye +- u +- v must lie within 65536 voxels of the origin");
    ESS_REQUIRE(params->shading == 0 || params->shading == 1, "shading must be 0 or 1");
    if (params->shading) {
        ESS_REQUIRE(std::isfinite(params->ka) && std::isfinite(params->kd) &&
                        std::isfinite(params->ks) && params->ka >= 0.0f && params->kd >= 0.0f &&
                        params->ks >= 0.0f,
                    "ka, kd, ks must be finite and >= 0");
        ESS_REQUIRE(params->shininess >= 1 && params->shininess <= 128,
                    "shininess must be in 1..128");
    }
    ESS_REQUIRE(std::isfinite(params->dt_ref) && params->dt_ref >= 0.0f,
                "dt_ref must be 0 (no opacity correction) or finite and > 0");
}

void copy_out(Ctx &c, void *dst, const void *src, size_t bytes, size_t cap, size_t *written)
{
    if (bytes > cap) throw Error{ESS_ERR_ARG, "destination buffer too small"};
    if (bytes) ESS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.stream));
    ESS_CUDA(cudaStreamSynchronize(c.stream));
    if (written) *written = bytes;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

ess_status ess_create(int device, void *cuda_stream, ess_ctx **out)
{
    if (!out) return ESS_ERR_ARG;
    *out = nullptr;
    ess_ctx *ctx = new (std::nothrow) ess_ctx();
    if (!ctx) return ESS_ERR_OOM;
    Ctx &c = ctx->c;
    c.device = device;
    ess_status st = guard(ctx, [&](Ctx &c) {
        c.stream = (cudaStream_t)cuda_stream;  // NULL: the CUDA default stream
        c.own_stream = false;
        ESS_CUDA(cudaMalloc(&c.dev_status, sizeof(uint32_t)));
        ESS_CUDA(cudaMemset(c.dev_status, 0, sizeof(uint32_t)));
        ESS_CUDA(cudaMalloc(&c.samples, sizeof(unsigned long long)));
        ESS_CUDA(cudaMemset(c.samples, 0, sizeof(unsigned long long)));
        ESS_CUDA(cudaMallocHost(&c.host_status, sizeof(uint32_t)));
    });
    if (st != ESS_OK) {
        delete ctx;
        return st;
    }
    *out = ctx;
    return ESS_OK;
}

ess_status ess_destroy(ess_ctx *ctx)
{
    if (!ctx) return ESS_ERR_ARG;
    ess_status st = guard(ctx, [&](Ctx &c) {
        for (auto &kv : c.structures) free_structure(c, *kv.second);
        for (auto &kv : c.volumes) {
            c.free(kv.second->data);
            c.free(kv.second->cells);
            for (auto &m : kv.second->minmax) c.free(m.second);
        }
        for (auto &kv : c.tfs) {
            c.free(kv.second->table);
            c.free(kv.second->prefix);
            c.free(kv.second->lut);
        }
        c.free(c.stage);
        c.free(c.selftest_flag);
        for (auto &kv : c.tile_counters) c.free(kv.second);
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        for (auto &kv : c.tfs) {
            for (int k = 0; k < STAGE_RING; ++k) {
                if (kv.second->staging[k]) cudaFreeHost(kv.second->staging[k]);
                if (kv.second->staged[k]) cudaEventDestroy(kv.second->staged[k]);
            }
            if (kv.second->updated) cudaEventDestroy(kv.second->updated);
        }
        for (auto &kv : c.volumes)
            if (kv.second->updated) cudaEventDestroy(kv.second->updated);
        for (auto &p : c.pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : c.free_events) cudaEventDestroy(e);
        for (auto &kv : c.batch) {
            Ctx::BatchGroup &g = kv.second;
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            for (int k = 0; k < STAGE_RING; ++k) {
                if (g.done[k]) cudaEventDestroy(g.done[k]);
                if (g.host[k]) cudaFreeHost(g.host[k]);
            }
            if (g.dev) cudaFree(g.dev);
        }
        if (c.capture_stream) cudaStreamDestroy(c.capture_stream);
        if (c.build_stream) cudaStreamDestroy(c.build_stream);
        for (cudaStream_t st : c.batch_streams) cudaStreamDestroy(st);
        if (c.fork_event) cudaEventDestroy(c.fork_event);
        if (c.rescan_event) cudaEventDestroy(c.rescan_event);
        cudaFree(c.dev_status);
        cudaFree(c.samples);
        cudaFreeHost(c.host_status);
        if (c.own_stream) cudaStreamDestroy(c.stream);
    });
    delete ctx;
    return st;
}

const char *ess_last_error(const ess_ctx *ctx)
{
    return ctx ? ctx->c.last_error.c_str() : "null context";
}

ess_status ess_sync(ess_ctx *ctx)
{
    ess_status dev = ESS_OK;
    std::string msg;
    ess_status st = guard(ctx, [&](Ctx &c) { dev = take_status(c, msg); });
    if (st != ESS_OK) return st;
    if (dev != ESS_OK) ctx->c.last_error = msg;
    return dev;
}

ess_status ess_release(ess_ctx *ctx, ess_handle h)
{
    return guard(ctx, [&](Ctx &c) {
        uint64_t tag = h >> 56;
        if (tag == TAG_ST) {
            Structure &s = get_st(c, h);
            free_structure(c, s);
            get_vol(c, s.vol).refs--;
            get_tf(c, s.tf).refs--;
            c.structures.erase(h);
        } else if (tag == TAG_VOL) {
            Volume &v = get_vol(c, h);
            if (v.refs > 0) throw Error{ESS_ERR_ARG, "volume still used by a structure"};
            c.free(v.data);
            c.free(v.cells);
            for (auto &m : v.minmax) c.free(m.second);
            if (v.updated) cudaEventDestroy(v.updated);
            c.volumes.erase(h);
        } else if (tag == TAG_TF) {
            TF &t = get_tf(c, h);
            if (t.refs > 0) throw Error{ESS_ERR_ARG, "TF still used by a structure"};
            c.free(t.table);
            c.free(t.prefix);
            c.free(t.lut);
            ESS_CUDA(cudaStreamSynchronize(c.stream));
            for (int k = 0; k < STAGE_RING; ++k) {
                if (t.staging[k]) cudaFreeHost(t.staging[k]);
                if (t.staged[k]) cudaEventDestroy(t.staged[k]);
            }
            if (t.updated) cudaEventDestroy(t.updated);
            c.tfs.erase(h);
        } else {
            throw Error{ESS_ERR_HANDLE, "unknown handle"};
        }
    });
}

ess_status ess_volume_upload(ess_ctx *ctx, const void *data, int data_on_device, ess_dtype dtype,
                             int nx, int ny, int nz, float value_lo, float value_hi,
                             ess_handle *vol)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(data && vol, "null pointer");
        ESS_REQUIRE(dtype == ESS_U8 || dtype == ESS_U16 || dtype == ESS_F32, "bad dtype");
        ESS_REQUIRE(nx > 0 && ny > 0 && nz > 0 && nx <= 8192 && ny <= 8192 && nz <= 8192,
                    "volume dimensions must be in 1..8192");
        ESS_REQUIRE(std::isfinite(value_lo) && std::isfinite(value_hi) && value_hi > value_lo,
                    "value range must be finite with value_hi > value_lo");
        auto v = std::make_unique<Volume>();
        v->nx = nx;
        v->ny = ny;
        v->nz = nz;
        v->dtype = dtype;
        v->value_lo = value_lo;
        v->value_hi = value_hi;
        v->bytes = (size_t)nx * ny * nz * dtype_size(dtype);
        v->data = c.alloc(v->bytes);
        cudaError_t e = cudaMemcpyAsync(v->data, data, v->bytes,
                                        data_on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                                        c.stream);
        if (e == cudaSuccess && !data_on_device) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) {
            c.free(v->data);
            throw Error{ESS_ERR_CUDA, std::string("volume copy: ") + cudaGetErrorString(e)};
        }
        if (dtype == ESS_F32) {
            launch_check_finite(c, (const float *)v->data, (size_t)nx * ny * nz);
            std::string msg;
            if (take_status(c, msg) != ESS_OK) {
                c.free(v->data);
                throw Error{ESS_ERR_ARG, msg};
            }
        }
        // the corner-replicated cells cost 8x the volume; keep them when they
        // fit in half of the free device memory
        size_t free_b = 0, total_b = 0;
        ESS_CUDA(cudaMemGetInfo(&free_b, &total_b));
        if (cells_indexable(*v) && cell_array_bytes(*v) < free_b / 2) set_sampler(c, *v, 1);
        ess_handle h = new_handle(c, TAG_VOL);
        c.volumes[h] = std::move(v);
        *vol = h;
    });
}

ess_status ess_volume_set_sampler(ess_ctx *ctx, ess_handle vol, int cells)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(cells == 0 || cells == 1, "sampler must be 0 (dense) or 1 (cells)");
        join_all_builds(c);
        Volume &v = get_vol(c, vol);
        set_sampler(c, v, cells);
        mark(c, v.updated);
    });
}

ess_status ess_tf_set(ess_ctx *ctx, const float *rgba, int on_device, int nt, ess_handle *tf)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(rgba && tf, "null pointer");
        ESS_REQUIRE(nt >= 2 && nt <= 65536, "nt must be in 2..65536");
        auto t = std::make_unique<TF>();
        t->nt = nt;
        t->table = (float4 *)c.alloc(sizeof(float4) * (nt + 1));
        t->prefix = (int *)c.alloc(sizeof(int) * (nt + 1));
        t->lut = (float4 *)c.alloc(sizeof(float4) * 2 * (size_t)nt);
        try {
            load_tf(c, *t, rgba, on_device);
        } catch (...) {
            c.free(t->table);
            c.free(t->prefix);
            c.free(t->lut);
            throw;
        }
        ess_handle h = new_handle(c, TAG_TF);
        c.tfs[h] = std::move(t);
        *tf = h;
    });
}

ess_status ess_tf_update(ess_ctx *ctx, ess_handle tf, const float *rgba, int on_device, int nt)
{
    return guard(ctx, [&](Ctx &c) {
        TF &t = get_tf(c, tf);
        ESS_REQUIRE(rgba, "null pointer");
        ESS_REQUIRE(nt == t.nt, "TF update must keep the table size");
        join_all_builds(c);  // builds enqueued so far read the old table
        load_tf(c, t, rgba, on_device);
    });
}

ess_status ess_build(ess_ctx *ctx, ess_handle vol, ess_handle tf, ess_kind kind,
                     const ess_build_params *params, ess_handle *structure)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(structure, "null pointer");
        Volume &v = get_vol(c, vol);
        TF &t = get_tf(c, tf);
        ESS_REQUIRE(kind == ESS_GRID || kind == ESS_LBVH || kind == ESS_KD || kind == ESS_NONE ||
                        kind == ESS_HYBRID,
                    "unknown structure kind");
        ess_build_params p = params ? *params : ess_build_params{8, 4, 1, 0, 0, 0};
        auto s = std::make_unique<Structure>();
        s->kind = kind;
        s->vol = vol;
        s->tf = tf;
        if (kind != ESS_NONE) {
            ESS_REQUIRE(p.brick >= 2 && p.brick <= 64, "brick must be in 2..64");
            ESS_REQUIRE(p.nbins == 0 || (p.nbins >= 2 && p.nbins <= 64 && p.nbins % 2 == 0),
                        "nbins must be 0 or even in 2..64");
            ESS_REQUIRE(p.halting == 0 || p.halting == 1, "halting must be 0 or 1");
            ESS_REQUIRE(p.mls >= 0, "mls must be >= 0");
            ESS_REQUIRE(p.empty_test == 0 || p.empty_test == 1, "empty_test must be 0 or 1");
            ESS_REQUIRE(p.rescan == 0 || p.rescan == 1, "rescan must be 0 or 1");
            int B = p.brick;
            s->gx = (v.nx + B - 1) / B;
            s->gy = (v.ny + B - 1) / B;
            s->gz = (v.nz + B - 1) / B;
            s->nb = (int64_t)s->gx * s->gy * s->gz;
            size_t nblk = compact_block_count(s->nb);
            size_t mask_bytes = nblk * 4096;
            s->mask = (uint8_t *)c.alloc(mask_bytes);
            ESS_CUDA(cudaMemsetAsync(s->mask, 0, mask_bytes, c.stream));
            s->ids = (uint32_t *)c.alloc(sizeof(uint32_t) * (size_t)s->nb);
            s->count = (int *)c.alloc(sizeof(int));
            s->block_sums = (uint32_t *)c.alloc(sizeof(uint32_t) * nblk);
            s->block_sums_n = nblk;
            s->device_bytes = mask_bytes + sizeof(uint32_t) * ((size_t)s->nb + nblk) + sizeof(int);
            if (kind == ESS_LBVH) {
                ESS_REQUIRE(s->gx <= 1024 && s->gy <= 1024 && s->gz <= 1024,
                            "LBVH: at most 1024 bricks per axis (30-bit Morton codes)");
            }
            try {
                if (kind == ESS_LBVH) alloc_lbvh(c, *s);
                if (kind == ESS_KD || kind == ESS_HYBRID) alloc_kd(c, *s);
            } catch (...) {
                free_structure(c, *s);
                throw;
            }
        }
        s->p = p;
        try {
            if (kind != ESS_NONE) run_build_async(c, *s, true);
            else s->tf_version = t.version;
        } catch (...) {
            free_structure(c, *s);
            throw;
        }
        v.refs++;
        t.refs++;
        ess_handle h = new_handle(c, TAG_ST);
        c.structures[h] = std::move(s);
        *structure = h;
    });
}

ess_status ess_rebuild_batch(ess_ctx *ctx, const ess_handle *structures, int count)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(structures, "null pointer");
        ESS_REQUIRE(count >= 1 && count <= 4096, "count must be in 1..4096");
        std::vector<Structure *> sts;
        for (int i = 0; i < count; ++i) {
            Structure &s = get_st(c, structures[i]);
            ESS_REQUIRE(std::find(sts.begin(), sts.end(), &s) == sts.end(),
                        "a structure appears twice in the batch");
            sts.push_back(&s);
        }
        ensure_build_stream(c);
        if (c.batch_streams.empty()) {
            int least = 0, greatest = 0;
            ESS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            for (int k = 0; k < BATCH_BUILD_STREAMS; ++k) {
                cudaStream_t st;
                ESS_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest));
                c.batch_streams.push_back(st);
            }
            ESS_CUDA(cudaEventCreateWithFlags(&c.rescan_event, cudaEventDisableTiming));
        }
        // one min/max rescan per (volume, brick size), on the first stream,
        // after every build enqueued so far (they may still read the old one);
        // none where this TF edit's pass has already run
        std::vector<std::pair<ess_handle, int>> rescans;
        for (Structure *s : sts) {
            if (s->kind == ESS_NONE || s->p.rescan != 1) continue;
            const std::pair<ess_handle, int> key(s->vol, s->p.brick);
            Volume &v = get_vol(c, s->vol);
            auto se = v.scan_epoch.find(s->p.brick);
            if (v.minmax.count(s->p.brick) && se != v.scan_epoch.end() && se->second == c.edit_epoch)
                continue;
            if (std::find(rescans.begin(), rescans.end(), key) == rescans.end()) rescans.push_back(key);
        }
        // every batch stream starts after the builds enqueued on the build
        // stream so far (they read, and a rescan there writes, Volume::minmax)
        ESS_CUDA(cudaEventRecord(c.fork_event, c.build_stream));
        for (cudaStream_t st : c.batch_streams) ESS_CUDA(cudaStreamWaitEvent(st, c.fork_event, 0));
        c.batch_streams_pending = true;
        cudaStream_t s0 = c.batch_streams[0];
        if (!rescans.empty()) {
            for (cudaStream_t st : c.batch_streams) {
                if (st == s0) continue;
                ESS_CUDA(cudaEventRecord(c.fork_event, st));
                ESS_CUDA(cudaStreamWaitEvent(s0, c.fork_event, 0));
            }
            OnStream on(c, s0);
            for (auto &r : rescans) {
                Volume &v = get_vol(c, r.first);
                if (v.updated) ESS_CUDA(cudaStreamWaitEvent(s0, v.updated, 0));
                minmax_for(c, v, r.second, true);
            }
            ESS_CUDA(cudaEventRecord(c.rescan_event, s0));
        }
        // the builds, spread over the streams; the rescanned min/max is reused
        for (size_t i = 0; i < sts.size(); ++i) {
            Structure &s = *sts[i];
            if (s.kind == ESS_NONE) {
                s.tf_version = get_tf(c, s.tf).version;
                continue;
            }
            cudaStream_t st = c.batch_streams[i % c.batch_streams.size()];
            if (!rescans.empty()) ESS_CUDA(cudaStreamWaitEvent(st, c.rescan_event, 0));
            wait_rebuild_deps(c, s, st);
            const int rescan = s.p.rescan;
            s.p.rescan = 0;
            try {
                build_on(c, s, st);
            } catch (...) {
                s.p.rescan = rescan;
                throw;
            }
            s.p.rescan = rescan;
        }
    });
}

ess_status ess_rebuild(ess_ctx *ctx, ess_handle structure)
{
    return guard(ctx, [&](Ctx &c) {
        Structure &s = get_st(c, structure);
        if (s.kind == ESS_NONE) {
            s.tf_version = get_tf(c, s.tf).version;
            return;
        }
        run_build_async(c, s, false);
    });
}

ess_status ess_structure_info_get(ess_ctx *ctx, ess_handle structure, ess_structure_info *info)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(info, "null pointer");
        Structure &s = get_st(c, structure);
        join_build(c, s);
        std::memset(info, 0, sizeof(*info));
        info->kind = s.kind;
        info->brick = s.p.brick;
        info->gx = s.gx;
        info->gy = s.gy;
        info->gz = s.gz;
        info->n_bricks = s.nb;
        if (s.kind != ESS_NONE) info->n_nonempty = nonempty_count(c, s);
        info->n_nodes = 0;
        info->height = s.kind == ESS_NONE ? 0 : 1;
        if (s.kind == ESS_LBVH) {
            int64_t n = info->n_nonempty;
            info->n_nodes = n > 0 ? 2 * n - 1 : 0;
            if (s.height < 0) s.height = n > 0 ? lbvh_height(c, s) : 0;
            info->height = s.height;
        }
        if (s.kind == ESS_KD || s.kind == ESS_HYBRID) {
            kd_stats(c, s);
            info->n_nodes = s.kd_count;
            info->height = s.height;
        }
        info->device_bytes = s.device_bytes;
    });
}

ess_status ess_structure_read(ess_ctx *ctx, ess_handle structure, ess_array which, void *dst,
                              size_t capacity, size_t *written)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(dst || capacity == 0, "null destination");
        Structure &s = get_st(c, structure);
        ESS_REQUIRE(s.kind != ESS_NONE, "an ESS_NONE structure holds no arrays");
        join_build(c, s);
        int64_t n = nonempty_count(c, s);
        switch (which) {
        case ESS_ARR_MINMAX: {
            ESS_REQUIRE(s.p.empty_test == 0, "min/max is only kept for the range test");
            Volume &v = get_vol(c, s.vol);
            copy_out(c, dst, minmax_for(c, v, s.p.brick, false), sizeof(float2) * s.nb, capacity, written);
            break;
        }
        case ESS_ARR_MASK: copy_out(c, dst, s.mask, (size_t)s.nb, capacity, written); break;
        case ESS_ARR_IDS: copy_out(c, dst, s.ids, sizeof(uint32_t) * n, capacity, written); break;
        case ESS_ARR_KEYS:
        case ESS_ARR_SORTED_KEYS:
        case ESS_ARR_SORTED_IDS:
        case ESS_ARR_LBVH_LEFT:
        case ESS_ARR_LBVH_RIGHT:
        case ESS_ARR_LBVH_BOXES: {
            ESS_REQUIRE(s.kind == ESS_LBVH, "array only exists for an LBVH");
            size_t inner = n > 1 ? (size_t)(n - 1) : 0;
            const void *src = which == ESS_ARR_KEYS          ? (const void *)s.keys
                              : which == ESS_ARR_SORTED_KEYS ? (const void *)s.keys_sorted
                              : which == ESS_ARR_SORTED_IDS  ? (const void *)s.ids_sorted
                              : which == ESS_ARR_LBVH_LEFT   ? (const void *)s.left
                              : which == ESS_ARR_LBVH_RIGHT  ? (const void *)s.right
                                                             : (const void *)s.inner_box;
            size_t bytes = which <= ESS_ARR_SORTED_IDS ? sizeof(uint32_t) * (size_t)n
                           : which == ESS_ARR_LBVH_BOXES ? sizeof(int32_t) * 6 * inner
                                                         : sizeof(int32_t) * inner;
            copy_out(c, dst, src, bytes, capacity, written);
            break;
        }
        case ESS_ARR_KD_NODES:
            ESS_REQUIRE(s.kind == ESS_KD || s.kind == ESS_HYBRID, "array only exists for a k-d tree");
            kd_stats(c, s);
            copy_out(c, dst, s.kd_nodes, sizeof(int32_t) * 9 * (size_t)s.kd_count, capacity, written);
            break;
        default: throw Error{ESS_ERR_ARG, "array not available for this structure kind"};
        }
    });
}

ess_status ess_render(ess_ctx *ctx, ess_handle structure, const ess_camera *camera,
                      const ess_render_params *params, int W, int H, float *out, int out_on_device)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(camera && params && out, "null pointer");
        check_render_args(camera, params, W, H);
        Structure &s = get_st(c, structure);
        join_build(c, s);
        Volume &v = get_vol(c, s.vol);
        TF &t = get_tf(c, s.tf);
        if (s.tf_version != t.version)
            throw Error{ESS_ERR_STALE, "structure was built for an older TF table: rebuild it"};
        RenderJob j;
        j.vol = &v;
        j.tf = &t;
        j.st = &s;
        j.cam = *camera;
        j.rp = *params;
        j.W = W;
        j.H = H;
        j.tile_w = params->tile_w;
        size_t bytes = (size_t)W * H * 4 * sizeof(float);
        // host memory the device can address (pinned: cudaMallocHost or
        // cudaHostRegister) is written by the render itself over the host
        // link, with no staging copy; other host memory takes the copy
        float *host_dev = nullptr;
        if (!out_on_device) {
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, out) == cudaSuccess) {
                if (pa.type == cudaMemoryTypeHost && pa.devicePointer)  // for this device
                    host_dev = (float *)pa.devicePointer;
            } else {
                cudaGetLastError();  // not a CUDA pointer: the copy path
            }
        }
        if (out_on_device) {
            j.out = out;
            launch_render(c, j);
            mark(c, s.used);
        } else if (host_dev) {
            j.out = host_dev;
            launch_render(c, j);
            ESS_CUDA(cudaStreamSynchronize(c.stream));
        } else {
            if (c.stage_bytes < bytes) {
                c.free(c.stage);
                c.stage = (float *)c.alloc(bytes);
                c.stage_bytes = bytes;
            }
            j.out = c.stage;
            launch_render(c, j);
            ESS_CUDA(cudaMemcpyAsync(out, c.stage, bytes, cudaMemcpyDeviceToHost, c.stream));
            ESS_CUDA(cudaStreamSynchronize(c.stream));
        }
    });
}

ess_status ess_render_batch(ess_ctx *ctx, const ess_render_item *items, int count, int tile_w)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(items, "null pointer");
        ESS_REQUIRE(count >= 1 && count <= BATCH_MAX, "batch count must be in 1..4096");
        ESS_REQUIRE(tile_w == 0 || tile_w == 4 || tile_w == 8 || tile_w == 16 || tile_w == 32,
                    "tile_w must be 0, 4, 8, 16 or 32");
        int tw = tile_w ? tile_w : 8;
        // validate everything before touching the GPU; group by (dtype, kind)
        std::map<int, std::vector<RenderJob>> groups;
        for (int i = 0; i < count; ++i) {
            const ess_render_item &it = items[i];
            ESS_REQUIRE(it.out, "null output in batch item");
            check_render_args(&it.camera, &it.params, it.W, it.H);
            Structure &s = get_st(c, it.structure);
            Volume &v = get_vol(c, s.vol);
            TF &t = get_tf(c, s.tf);
            if (s.tf_version != t.version)
                throw Error{ESS_ERR_STALE, "batch item structure was built for an older TF table"};
            RenderJob j;
            j.vol = &v;
            j.tf = &t;
            j.st = &s;
            j.cam = it.camera;
            j.rp = it.params;
            j.W = it.W;
            j.H = it.H;
            j.out = it.out;
            j.tile_w = tw;
            const int shaded = render_shaded(it.params) ? 1 : 0;
            groups[((((int)v.dtype * 16 + (int)s.kind) * 2 + (v.use_cells ? 1 : 0)) * 2 + shaded) *
                       2 + (s.kind == ESS_GRID && grid_dda_inc(j) ? 1 : 0)]
                .push_back(j);
        }
        for (int i = 0; i < count; ++i) join_build(c, get_st(c, items[i].structure));
        if (!c.capture_stream)
            ESS_CUDA(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking));
        for (auto &kv : groups) {
            Ctx::BatchGroup &g = c.batch[kv.first];
            std::vector<RenderJob> &jobs = kv.second;
            int n = (int)jobs.size();
            if (!g.dev) {
                g.cap = batch_bytes(BATCH_MAX);
                ESS_CUDA(cudaMalloc(&g.dev, g.cap));
            }
            const int k = g.next;
            if (!g.host[k]) {
                ESS_CUDA(cudaMallocHost(&g.host[k], g.cap));
                ESS_CUDA(cudaEventCreateWithFlags(&g.done[k], cudaEventDisableTiming));
                ESS_CUDA(cudaEventRecord(g.done[k], c.stream));
            }
            // the replay that last read this slot must have run
            ESS_CUDA(cudaEventSynchronize(g.done[k]));
            size_t bytes = pack_batch(c, jobs.data(), n, tw, g.host[k], g.cap);
            if (!g.exec) {
                // capture: copy of the packed batch + the persistent kernel
                ESS_CUDA(cudaStreamBeginCapture(c.capture_stream, cudaStreamCaptureModeThreadLocal));
                cudaStream_t saved = c.stream;
                c.stream = c.capture_stream;
                cudaError_t e1 = cudaMemcpyAsync(g.dev, g.host[k], bytes, cudaMemcpyHostToDevice, c.stream);
                try {
                    if (e1 == cudaSuccess)
                        launch_render_batch(c, jobs[0].st->kind, jobs[0].vol->dtype,
                                            jobs[0].vol->use_cells, render_shaded(jobs[0].rp),
                                            (kv.first & 1) != 0, g.dev);
                } catch (...) {
                    c.stream = saved;
                    cudaGraph_t tmp;
                    cudaStreamEndCapture(c.capture_stream, &tmp);
                    if (tmp) cudaGraphDestroy(tmp);
                    throw;
                }
                c.stream = saved;
                ESS_CUDA(cudaStreamEndCapture(c.capture_stream, &g.graph));
                ESS_CUDA(e1);
                size_t nn = 0;
                ESS_CUDA(cudaGraphGetNodes(g.graph, nullptr, &nn));
                std::vector<cudaGraphNode_t> nodes(nn);
                ESS_CUDA(cudaGraphGetNodes(g.graph, nodes.data(), &nn));
                for (auto nd : nodes) {
                    cudaGraphNodeType ty;
                    ESS_CUDA(cudaGraphNodeGetType(nd, &ty));
                    if (ty == cudaGraphNodeTypeMemcpy) g.copy_node = nd;
                }
                ESS_REQUIRE(g.copy_node, "internal: batch graph has no copy node");
                ESS_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
            } else {
                ESS_CUDA(cudaGraphExecMemcpyNodeSetParams1D(g.exec, g.copy_node, g.dev, g.host[k],
                                                            bytes, cudaMemcpyHostToDevice));
            }
            {
                Launch L(c, "render_batch");
                ESS_CUDA(cudaGraphLaunch(g.exec, c.stream));
            }
            ESS_CUDA(cudaEventRecord(g.done[k], c.stream));
            g.next = (k + 1) % STAGE_RING;
        }
        // later rebuilds of these structures wait for this batch
        std::vector<Structure *> used;
        for (int i = 0; i < count; ++i) {
            Structure *p = &get_st(c, items[i].structure);
            if (std::find(used.begin(), used.end(), p) == used.end()) used.push_back(p);
        }
        for (Structure *p : used) mark(c, p->used);
    });
}

ess_status ess_autotune(ess_ctx *ctx, ess_handle vol, ess_handle tf, const ess_camera *cameras,
                        int ncam, const ess_render_params *params, int W, int H,
                        float frames_per_edit, ess_tune_result *best)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(cameras && params && best && ncam >= 1, "null pointer or no camera");
        check_render_args(&cameras[0], params, W, H);
        ESS_REQUIRE(frames_per_edit >= 0.0f, "frames_per_edit must be >= 0");
        get_vol(c, vol);
        get_tf(c, tf);
        float *img = (float *)c.alloc((size_t)W * H * 4 * sizeof(float));
        cudaEvent_t e0, e1;
        ESS_CUDA(cudaEventCreate(&e0));
        ESS_CUDA(cudaEventCreate(&e1));
        const int kinds[4] = {ESS_GRID, ESS_LBVH, ESS_KD, ESS_HYBRID};
        const int bricks[4] = {4, 8, 16, 32};
        const int tiles[4] = {4, 8, 16, 32};
        double best_cost = 1e300;
        ess_tune_result res{};
        std::string err;
        for (int kind : kinds) {
            for (int B : bricks) {
                // the hybrid's tree is the paper's shallow one
                ess_build_params bp{B, 4, kind == ESS_HYBRID ? 0 : 1, kind == ESS_HYBRID ? 0 : 32, 0, 0};
                ess_handle h = 0;
                if (ess_build(ctx, vol, tf, (ess_kind)kind, &bp, &h) != ESS_OK) {
                    c.last_error.clear();
                    continue;  // e.g. LBVH beyond 1024 bricks per axis
                }
                Structure &s = get_st(c, h);
                join_build(c, s);
                // time one rebuild
                ESS_CUDA(cudaEventRecord(e0, c.stream));
                run_build(c, s);
                ESS_CUDA(cudaEventRecord(e1, c.stream));
                ESS_CUDA(cudaEventSynchronize(e1));
                float bms = 0.0f;
                ESS_CUDA(cudaEventElapsedTime(&bms, e0, e1));
                for (int tw : tiles) {
                    RenderJob j;
                    j.vol = &get_vol(c, vol);
                    j.tf = &get_tf(c, tf);
                    j.st = &s;
                    j.rp = *params;
                    j.W = W;
                    j.H = H;
                    j.out = img;
                    j.tile_w = tw;
                    j.cam = cameras[0];
                    launch_render(c, j);  // warm-up
                    ESS_CUDA(cudaEventRecord(e0, c.stream));
                    for (int k = 0; k < ncam; ++k) {
                        j.cam = cameras[k];
                        launch_render(c, j);
                    }
                    ESS_CUDA(cudaEventRecord(e1, c.stream));
                    ESS_CUDA(cudaEventSynchronize(e1));
                    float rms = 0.0f;
                    ESS_CUDA(cudaEventElapsedTime(&rms, e0, e1));
                    rms /= (float)ncam;
                    double cost = bms + (double)frames_per_edit * rms;
                    if (cost < best_cost) {
                        best_cost = cost;
                        res.kind = kind;
                        res.brick = B;
                        res.tile_w = tw;
                        res.build_ms = bms;
                        res.render_ms = rms;
                    }
                }
                ess_release(ctx, h);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c.free(img);
        ESS_REQUIRE(best_cost < 1e300, "autotune: no candidate could be built");
        *best = res;
    });
}

uint64_t ess_launch_count(const ess_ctx *ctx) { return ctx ? ctx->c.launches : 0; }

ess_status ess_sample_count(ess_ctx *ctx, uint64_t *samples, int reset)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(samples, "null pointer");
        unsigned long long v = 0;
        ESS_CUDA(cudaMemcpyAsync(&v, c.samples, sizeof(v), cudaMemcpyDeviceToHost, c.stream));
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        *samples = v;
        if (reset) ESS_CUDA(cudaMemsetAsync(c.samples, 0, sizeof(v), c.stream));
    });
}

ess_status ess_profile_enable(ess_ctx *ctx, int enable)
{
    return guard(ctx, [&](Ctx &c) { c.profiling = enable != 0; });
}

ess_status ess_profile_read(ess_ctx *ctx, int max, const char **names, uint64_t *launches,
                            double *total_ms, int *count)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(count, "null pointer");
        join_all_builds(c);
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        for (auto &p : c.pending) {
            float ms = 0.0f;
            ESS_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
            auto &e = c.prof[p.name];
            e.first += 1;
            e.second += ms;
            c.free_events.push_back(p.a);
            c.free_events.push_back(p.b);
        }
        c.pending.clear();
        int k = 0;
        for (auto &kv : c.prof) {
            if (k < max) {
                if (names) {
                    // names are the static literals given at launch sites
                    names[k] = kv.first.c_str();
                }
                if (launches) launches[k] = kv.second.first;
                if (total_ms) total_ms[k] = kv.second.second;
            }
            ++k;
        }
        *count = k;
    });
}

ess_status ess_selftest_wait(ess_ctx *ctx, int set, int64_t polls)
{
    return guard(ctx, [&](Ctx &c) {
        ESS_REQUIRE(set == 0 || set == 1, "set must be 0 or 1");
        ESS_REQUIRE(polls >= 1 && polls <= (int64_t)1 << 24, "polls must be in 1..2^24");
        if (!c.selftest_flag) c.selftest_flag = (uint32_t *)c.alloc(sizeof(uint32_t));
        launch_selftest_wait(c, c.selftest_flag, set == 1, (long)polls);
    });
}

ess_status ess_profile_reset(ess_ctx *ctx)
{
    return guard(ctx, [&](Ctx &c) {
        join_all_builds(c);
        ESS_CUDA(cudaStreamSynchronize(c.stream));
        for (auto &p : c.pending) {
            c.free_events.push_back(p.a);
            c.free_events.push_back(p.b);
        }
        c.pending.clear();
        c.prof.clear();
    });
}

}  // extern "C"
