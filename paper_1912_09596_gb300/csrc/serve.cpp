// serve.cpp -- request loop with continuous batching over resident volumes
// and structures.  The paper's interaction model (Sec. 1) is a user who edits
// the TF and looks at the result; a server keeps volumes and their skipping
// structures in device memory and turns a stream of such requests (render a
// view; edit a TF, rebuild, render) into batched GPU work.
//
// One worker thread owns the context.  It admits queued requests in arrival
// order into a batch while the output memory of the batch fits the budget,
// applies the batch's TF edits (upload + rebuild of the edited structure),
// issues all renders of the batch as one persistent launch, queues the copies
// of the images to the callers' host buffers and records an event.  Up to
// max_inflight batches are on the GPU at once; while they run, newly arrived
// requests form the next batch, so requests are admitted as memory and slots
// free up.  Rebuilds and renders stay on the context stream, so a rebuild can
// never overtake a render of the same structure issued before it; the image
// copies of a batch run on a separate copy stream after that batch's render,
// overlapping the next batch.  Within a batch a request is not admitted if an
// edit in the batch would change the TF a render already in the batch has to
// see (the batch is cut there).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ess_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id;
    ess_request r;
    std::vector<float> table;  // edit: copy of the new TF
    Clock::time_point t_submit, t_launch, t_done;
    int done = 0;
    ess_status status = ESS_OK;
    float *dev_out = nullptr;
    bool direct = false;  // dev_out is the device's address of the caller's pinned image
    size_t out_bytes = 0;
};

struct Inflight {
    std::vector<Req *> reqs;
    cudaEvent_t ev;
    size_t bytes;
};

}  // namespace

struct ess_server {
    ess_ctx *ctx;
    ess_server_config cfg;
    std::mutex mtx;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    size_t in_use = 0;
    std::deque<Inflight> inflight;
    std::vector<cudaEvent_t> free_events;
    cudaStream_t copy_stream = nullptr;  // image copies overlap the next batch
    // stream-ordered pool for the per-request output buffers; it keeps up to
    // the memory budget mapped, so allocations after a synchronisation do not
    // go back to the driver
    cudaMemPool_t pool = nullptr;
    std::string error;
};

namespace {

double ms(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

void finish_request(ess_server *s, Req *q, ess_status st)
{
    q->status = st;
    q->t_done = Clock::now();
    q->done = 1;
}

// Retires finished batches (caller holds no lock); returns true if any.
bool retire(ess_server *s, bool block)
{
    bool any = false;
    while (!s->inflight.empty()) {
        Inflight &f = s->inflight.front();
        cudaError_t e = block ? cudaEventSynchronize(f.ev) : cudaEventQuery(f.ev);
        if (e == cudaErrorNotReady) break;
        ess_status st = e == cudaSuccess ? ESS_OK : ESS_ERR_CUDA;
        {
            std::lock_guard<std::mutex> lk(s->mtx);
            for (Req *q : f.reqs) {
                q->dev_out = nullptr;  // freed on the copy stream after its copy
                finish_request(s, q, st);
            }
            s->in_use -= f.bytes;
        }
        s->free_events.push_back(f.ev);
        s->inflight.pop_front();
        any = true;
        block = false;
        s->cv_done.notify_all();
    }
    return any;
}

// Takes the next batch from the queue (caller holds the lock).
std::vector<Req *> admit(ess_server *s)
{
    std::vector<Req *> batch;
    std::unordered_set<ess_handle> rendered;
    size_t bytes = 0;
    while (!s->queue.empty() && (int)batch.size() < s->cfg.max_batch) {
        Req *q = s->queue.front();
        if (q->r.kind == ESS_REQ_EDIT && rendered.count(q->r.structure)) break;
        size_t need = q->out_bytes;
        if (s->in_use + bytes + need > s->cfg.memory_budget) {
            if (batch.empty() && s->inflight.empty() && s->in_use == 0) {
                // larger than the whole budget: refuse it instead of waiting forever
                s->queue.pop_front();
                finish_request(s, q, ESS_ERR_BUSY);
                s->cv_done.notify_all();
                continue;
            }
            break;
        }
        s->queue.pop_front();
        bytes += need;
        rendered.insert(q->r.structure);
        batch.push_back(q);
    }
    s->in_use += bytes;
    return batch;
}

void issue(ess_server *s, std::vector<Req *> &batch)
{
    ess_ctx *ctx = s->ctx;
    ess::Ctx &c = ctx->c;
    auto now = Clock::now();
    std::vector<ess_render_item> items;
    std::vector<Req *> ok;
    size_t bytes = 0;
    for (Req *q : batch) {
        q->t_launch = now;
        bytes += q->out_bytes;
        ess_status st = ESS_OK;
        if (q->r.kind == ESS_REQ_EDIT) {
            ess::Structure *sp = nullptr;
            auto it = c.structures.find(q->r.structure);
            if (it == c.structures.end()) st = ESS_ERR_HANDLE;
            else sp = it->second.get();
            if (st == ESS_OK) st = ess_tf_update(ctx, sp->tf, q->table.data(), 0, q->r.nt);
            if (st == ESS_OK) st = ess_rebuild(ctx, q->r.structure);
        }
        if (st == ESS_OK) {
            // a pinned image the device can address is written by the render
            // itself; any other image goes through a pool buffer and a copy
            cudaPointerAttributes pa{};
            q->direct = false;
            if (cudaPointerGetAttributes(&pa, q->r.out) == cudaSuccess) {
                if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
                    q->dev_out = (float *)pa.devicePointer;
                    q->direct = true;
                }
            } else {
                cudaGetLastError();
            }
            if (!q->direct &&
                cudaMallocFromPoolAsync((void **)&q->dev_out, q->out_bytes, s->pool, c.stream) !=
                    cudaSuccess) {
                cudaGetLastError();
                q->dev_out = nullptr;
                st = ESS_ERR_OOM;
            }
        }
        if (st != ESS_OK) {
            std::lock_guard<std::mutex> lk(s->mtx);
            finish_request(s, q, st);
            continue;
        }
        ess_render_item it{};
        it.structure = q->r.structure;
        it.camera = q->r.camera;
        it.params = q->r.params;
        it.W = q->r.W;
        it.H = q->r.H;
        it.out = q->dev_out;
        items.push_back(it);
        ok.push_back(q);
    }
    if (!items.empty()) {
        ess_status st = ess_render_batch(ctx, items.data(), (int)items.size(), s->cfg.tile_w);
        if (st != ESS_OK) {
            std::lock_guard<std::mutex> lk(s->mtx);
            for (Req *q : ok) {
                if (!q->direct) cudaFreeAsync(q->dev_out, c.stream);
                q->dev_out = nullptr;
                finish_request(s, q, st);
            }
            ok.clear();
        }
    }
    auto take_event = [&]() {
        cudaEvent_t e;
        if (!s->free_events.empty()) {
            e = s->free_events.back();
            s->free_events.pop_back();
        } else {
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        }
        return e;
    };
    // the copies wait for the batch's render on the copy stream, so the next
    // batch can start on the context stream while they run
    cudaEvent_t rendered = take_event();
    cudaEventRecord(rendered, c.stream);
    cudaStreamWaitEvent(s->copy_stream, rendered, 0);
    for (Req *q : ok) {
        if (q->direct) continue;  // already in the caller's image
        cudaMemcpyAsync(q->r.out, q->dev_out, q->out_bytes, cudaMemcpyDeviceToHost,
                        s->copy_stream);
        cudaFreeAsync(q->dev_out, s->copy_stream);
    }
    Inflight f;
    f.reqs = ok;
    f.bytes = bytes;
    f.ev = take_event();
    cudaEventRecord(f.ev, s->copy_stream);
    s->free_events.push_back(rendered);  // reusable once recorded again later
    s->inflight.push_back(f);
    s->cv_done.notify_all();
}

void worker_loop(ess_server *s)
{
    cudaSetDevice(s->ctx->c.device);
    while (true) {
        retire(s, false);
        std::vector<Req *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mtx);
            if (s->stop && s->queue.empty() && s->inflight.empty()) break;
            if ((int)s->inflight.size() < s->cfg.max_inflight) batch = admit(s);
            if (batch.empty()) {
                if (s->inflight.empty()) {
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                    continue;
                }
            }
        }
        if (!batch.empty()) {
            issue(s, batch);
            continue;
        }
        // GPU busy and nothing admissible: wait for the oldest batch briefly
        if (!retire(s, false)) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

ess_status ess_server_create(ess_ctx *ctx, const ess_server_config *cfg, ess_server **out)
{
    if (!ctx || !out) return ESS_ERR_ARG;
    ess_server_config c = cfg ? *cfg : ess_server_config{0, 256, 2, 0};
    if (c.max_batch <= 0 || c.max_batch > ess::BATCH_MAX) return ESS_ERR_ARG;
    if (c.max_inflight <= 0 || c.max_inflight > 64) return ESS_ERR_ARG;
    if (c.memory_budget == 0) {
        size_t f = 0, t = 0;
        cudaSetDevice(ctx->c.device);
        if (cudaMemGetInfo(&f, &t) != cudaSuccess) return ESS_ERR_CUDA;
        c.memory_budget = f / 4;
    }
    ess_server *s = new (std::nothrow) ess_server();
    if (!s) return ESS_ERR_OOM;
    s->ctx = ctx;
    s->cfg = c;
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return ESS_ERR_CUDA;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->c.device;
    uint64_t keep = c.memory_budget;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        if (s->pool) cudaMemPoolDestroy(s->pool);
        cudaStreamDestroy(s->copy_stream);
        delete s;
        return ESS_ERR_CUDA;
    }
    // Grow the pool once now (up to 1 GiB of the budget, kept by the release
    // threshold), so that the first batches do not wait for it to map memory.
    {
        const size_t warm = std::min<size_t>(c.memory_budget, (size_t)1 << 30);
        void *p = nullptr;
        if (cudaMallocFromPoolAsync(&p, warm, s->pool, s->copy_stream) == cudaSuccess) {
            cudaFreeAsync(p, s->copy_stream);
        } else {
            cudaGetLastError();
        }
        cudaStreamSynchronize(s->copy_stream);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return ESS_OK;
}

ess_status ess_server_submit(ess_server *s, const ess_request *r, uint64_t *id)
{
    if (!s || !r || !id) return ESS_ERR_ARG;
    if (r->kind != ESS_REQ_RENDER && r->kind != ESS_REQ_EDIT) return ESS_ERR_ARG;
    if (!r->out || r->W <= 0 || r->H <= 0 || r->W > 16384 || r->H > 16384) return ESS_ERR_ARG;
    if (r->kind == ESS_REQ_EDIT && (!r->rgba || r->nt < 2 || r->nt > 65536)) return ESS_ERR_ARG;
    auto q = std::make_unique<Req>();
    q->r = *r;
    if (r->kind == ESS_REQ_EDIT) q->table.assign(r->rgba, r->rgba + 4 * (size_t)r->nt);
    q->out_bytes = (size_t)r->W * r->H * 4 * sizeof(float);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mtx);
        if (s->stop) return ESS_ERR_BUSY;
        q->id = s->next_id++;
        *id = q->id;
        s->queue.push_back(q.get());
        s->reqs[q->id] = std::move(q);
    }
    s->cv_work.notify_one();
    return ESS_OK;
}

static void fill_status(const Req *q, ess_request_status *st)
{
    st->done = q->done;
    st->status = q->status;
    st->queue_ms = q->done || q->t_launch.time_since_epoch().count() ? ms(q->t_submit, q->t_launch) : 0.0;
    st->latency_ms = q->done ? ms(q->t_submit, q->t_done) : 0.0;
}

ess_status ess_server_poll(ess_server *s, uint64_t id, ess_request_status *st)
{
    if (!s || !st) return ESS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mtx);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ESS_ERR_HANDLE;
    fill_status(it->second.get(), st);
    return ESS_OK;
}

ess_status ess_server_wait(ess_server *s, uint64_t id, ess_request_status *st)
{
    if (!s || !st) return ESS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mtx);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ESS_ERR_HANDLE;
    Req *q = it->second.get();
    s->cv_done.wait(lk, [&] { return q->done != 0; });
    fill_status(q, st);
    return ESS_OK;
}

ess_status ess_server_drain(ess_server *s)
{
    if (!s) return ESS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mtx);
    s->cv_done.wait(lk, [&] {
        if (!s->queue.empty()) return false;
        for (auto &kv : s->reqs)
            if (!kv.second->done) return false;
        return true;
    });
    return ESS_OK;
}

ess_status ess_server_destroy(ess_server *s)
{
    if (!s) return ESS_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mtx);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->copy_stream);
    try {
        ess::join_all_builds(s->ctx->c);  // rebuilds of edits whose render failed
    } catch (...) {
    }
    cudaStreamSynchronize(s->ctx->c.stream);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    cudaStreamDestroy(s->copy_stream);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return ESS_OK;
}

}  // extern "C"
