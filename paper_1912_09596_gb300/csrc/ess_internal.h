// ess_internal.h -- objects, device layouts and kernel launchers shared by
// the translation units of libess.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "ess.h"

namespace ess {

// ---------------------------------------------------------------- errors
// Bits of the device status word that kernels set instead of trapping.
enum : uint32_t {
    DEV_ERR_NONFINITE = 1u,  // a float voxel was NaN or infinite
    DEV_ERR_TIMEOUT = 2u,    // a bounded spin-wait gave up
    DEV_ERR_OVERFLOW = 4u,   // a fixed-capacity device buffer would overflow
    DEV_ERR_BAD_TF = 8u      // a device TF table held a non-finite value or alpha outside [0,1]
};

struct Error {
    ess_status st;
    std::string msg;
};

#define ESS_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            throw ::ess::Error{e_ == cudaErrorMemoryAllocation ? ESS_ERR_OOM        \
                                                               : ESS_ERR_CUDA,      \
                               std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define ESS_REQUIRE(cond, msg)                                    \
    do {                                                          \
        if (!(cond)) throw ::ess::Error{ESS_ERR_ARG, (msg)};      \
    } while (0)

// ---------------------------------------------------- device-side layouts
// Traversal node of a binary box tree (LBVH and k-d share it): both
// children's boxes live in the parent, as floats in voxel units (brick
// coordinates times the brick size; the far faces are not clamped to the
// volume, which only makes the boxes larger), so that four 16-byte loads feed
// both slab tests with no decoding.  child >= 0: inner node; child < 0: leaf,
// payload -1 - child (LBVH: brick id; k-d: node id).
struct __align__(16) BoxNode {
    float lbox[6];  // lo xyz, hi xyz
    float rbox[6];
    int32_t left, right, pad0, pad1;
};
static_assert(sizeof(BoxNode) == 64, "BoxNode must be 64 bytes");

// ------------------------------------------------------------------ objects
struct Ctx;

struct Volume {
    int nx, ny, nz;
    ess_dtype dtype;
    float value_lo, value_hi;
    void *data = nullptr;   // device copy, x fastest
    size_t bytes = 0;
    void *cells = nullptr;  // corner-replicated trilinear cells, (n+1)^3 x 8 values
    size_t cell_bytes = 0;
    bool use_cells = false;
    std::map<int, float2 *> minmax;  // per brick size: apron min/max (cached)
    // per brick size: the context's TF-edit epoch at the last rescan (a rescan
    // is skipped while no TF has changed since: one volume pass per edit)
    std::map<int, uint64_t> scan_epoch;
    int refs = 0;           // structures using the volume
    bool released = false;
    cudaEvent_t updated = nullptr;  // after the last change of the cell copy
};

// Pinned staging slots per TF and per batch group: the host fills the next
// slot while earlier uploads may still be queued behind running kernels.
constexpr int STAGE_RING = 4;

struct TF {
    int nt;
    float4 *table = nullptr;  // device, nt entries
    int *prefix = nullptr;    // device, nt+1 counts of alpha > 0
    // device, 2 nt entries: entry i and the float32 difference entry i+1 - i
    // (0 for the last), the two operands of the renderer's TF lerp
    float4 *lut = nullptr;
    uint64_t version = 0;     // bumped by every update
    // pinned host copies for asynchronous uploads, used in turn; a slot is
    // rewritten only after the upload that last read it has run
    float *staging[STAGE_RING] = {};
    cudaEvent_t staged[STAGE_RING] = {};
    int stage_next = 0;
    int refs = 0;
    bool released = false;
    cudaEvent_t updated = nullptr;  // after the last table upload and prefix
};

struct Structure {
    ess_kind kind;
    ess_build_params p;
    ess_handle vol = 0, tf = 0;
    uint64_t tf_version = 0;
    int gx = 0, gy = 0, gz = 0;
    int64_t nb = 0;
    // grid / common
    uint8_t *mask = nullptr;     // nb (padded)
    uint32_t *ids = nullptr;     // nb capacity
    int *count = nullptr;        // device: number of non-empty bricks
    uint32_t *block_sums = nullptr;
    size_t block_sums_n = 0;
    int64_t n_host = -1;         // non-empty count once read back
    // LBVH
    uint32_t *keys = nullptr;                                 // Morton code of ids[i]
    uint32_t *keys_sorted = nullptr, *ids_sorted = nullptr;   // sort result
    uint32_t *keys_alt = nullptr, *ids_alt = nullptr;         // sort ping-pong
    uint32_t *sort_scratch = nullptr;
    int32_t *left = nullptr, *right = nullptr, *parent = nullptr, *leaf_parent = nullptr;
    int32_t *inner_box = nullptr;  // (n-1) x 6
    int32_t *range_end = nullptr;  // (n-1): the far end of each inner node's leaf range
    int32_t *chunk_box = nullptr;  // boxes of 32, 1024 and 32768 consecutive sorted leaves
    BoxNode *nodes = nullptr;      // traversal nodes (LBVH: n-1; k-d: inner nodes)
    int32_t *root = nullptr;       // device root record: ref, then the box as 6 floats (voxels)
    int height = 0;
    // k-d
    Volume *volume = nullptr;
    int32_t *kd_nodes = nullptr;     // capacity x 9: lo xyz, hi xyz, axis, plane, first child
    int kd_capacity = 0;
    int64_t kd_count = 0;
    int kd_count_i32 = 0;
    int *kd_count_dev = nullptr;     // device: k-d node count
    int *brick_node = nullptr;       // per non-empty brick: its node on the current level
    int32_t *kd_scratch_i32 = nullptr;  // root box reduction
    // per-level slab boxes: ping-pong, and a third buffer for the persistent
    // build (which zeroes the buffer of level l + 1 during level l)
    int32_t *kd_slabs[3] = {nullptr, nullptr, nullptr};
    size_t kd_slab_cap[3] = {0, 0, 0};          // in nodes
    unsigned long long *kd_vr = nullptr;        // suffix volumes
    size_t kd_vr_cap = 0;
    void *kd_dec = nullptr;                     // per-node decisions
    size_t kd_dec_cap = 0;
    uint32_t *kd_block_sums = nullptr;
    size_t kd_bs_cap = 0;
    void *kd_state = nullptr;                   // device level state (32 bytes)
    unsigned long long *kd_chunk = nullptr;     // look-back words of the 4-bin decide/emit
    size_t kd_chunk_cap = 0;
    cudaGraph_t kd_graph = nullptr;             // device-driven build (binned planes)
    cudaGraphExec_t kd_exec = nullptr;
    size_t device_bytes = 0;
    bool released = false;
    // Builds run on the context's build stream: `built` is recorded after the
    // last one, and users of the structure on the context stream wait for it
    // first (join_build) while `build_pending` is set.  `used` is recorded on
    // the context stream after each use of its buffers there (a render); a
    // rebuild waits only for that, and for its TF and volume updates.
    cudaEvent_t built = nullptr;
    bool build_pending = false;
    cudaEvent_t used = nullptr;
};

// The k-d renderer keeps a stack of 128 entries, enough for 129 levels.
constexpr int KD_MAX_LEVELS = 129;

// ---------------------------------------------------------------- context
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string last_error;
    uint64_t next_handle = 1;
    std::unordered_map<ess_handle, std::unique_ptr<Volume>> volumes;
    std::unordered_map<ess_handle, std::unique_ptr<TF>> tfs;
    std::unordered_map<ess_handle, std::unique_ptr<Structure>> structures;
    uint32_t *dev_status = nullptr;   // device status word
    uint32_t *host_status = nullptr;  // pinned mirror
    float *stage = nullptr;           // device image staging for host output
    size_t stage_bytes = 0;
    uint64_t launches = 0;
    unsigned long long *samples = nullptr;  // device: samples evaluated by renders
    // profiling
    bool profiling = false;
    struct Pending { const char *name; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    std::map<std::string, std::pair<uint64_t, double>> prof;
    // batched rendering: one captured graph per (dtype, kind) group
    struct BatchGroup {
        void *host[STAGE_RING] = {};        // pinned staging slots, used in turn
        cudaEvent_t done[STAGE_RING] = {};  // the replay that last read each slot has run
        int next = 0;
        void *dev = nullptr;  // device copy (replays are ordered on the stream)
        size_t cap = 0;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t copy_node = nullptr;
        int n_captured = -1;
    };
    std::map<int, BatchGroup> batch;
    cudaStream_t capture_stream = nullptr;
    // Builds and rebuilds run here (highest priority), forked from and joined
    // back into `stream` by events, so that a rebuild overlaps the rendering of
    // other structures.
    cudaStream_t build_stream = nullptr;
    cudaEvent_t fork_event = nullptr;
    // ess_rebuild_batch spreads its structures over these (highest priority
    // too), after one min/max rescan per volume and brick size on the first.
    std::vector<cudaStream_t> batch_streams;
    cudaEvent_t rescan_event = nullptr;
    // Bumped by every TF upload; a rebuild with `rescan` reads the volume
    // again only if a TF changed since the last rescan of its (volume, brick).
    uint64_t edit_epoch = 1;
    // Set by ess_rebuild_batch: the next build on build_stream first waits for
    // the batch streams (both read, and rescans write, Volume::minmax).
    bool batch_streams_pending = false;
    uint32_t *selftest_flag = nullptr;  // device word of ess_selftest_wait
    // device words: next tile of the streaming kernels, one per stream that
    // launches them (launches on one stream are ordered, on two they are not)
    std::map<cudaStream_t, int *> tile_counters;

    void *alloc(size_t bytes);
    void free(void *p);
    void begin(const char *name);   // before a kernel launch
    void end();                     // after a kernel launch (checks the launch)
    cudaEvent_t event();
    const char *current = nullptr;
    cudaEvent_t cur_a = nullptr;
};

// Builds run on Ctx::build_stream (ctx.cpp): the context stream waits for a
// structure's last build, or for every build enqueued so far.
void join_build(Ctx &c, Structure &s);
void join_all_builds(Ctx &c);
// Records `e` (created on first use, no timing) on the context stream.
void mark(Ctx &c, cudaEvent_t &e);

// Launch bracket: counts the launch, records profiling events and checks the
// launch error.
struct Launch {
    Ctx &c;
    Launch(Ctx &ctx, const char *name) : c(ctx) { c.begin(name); }
    ~Launch() noexcept(false) { c.end(); }
};

// ----------------------------------------------------------- launchers
// classify.cu
void launch_check_finite(Ctx &c, const float *v, size_t n);
size_t cell_array_bytes(const Volume &v);
void launch_build_cells(Ctx &c, const Volume &v, void *cells);
void launch_brick_minmax(Ctx &c, const Volume &v, int B, float2 *out);
// minmax_tma.cu (bricks of 2, 4, 8): false when the volume's layout or brick
// size does not suit it
bool launch_brick_minmax_tma(Ctx &c, const Volume &v, int B, float2 *out);
void launch_tf_prefix(Ctx &c, const float4 *table, int nt, int *prefix, float4 *lut,
                      int validate);
void launch_brick_mask(Ctx &c, const float2 *minmax, int64_t nb, const TF &tf,
                       float value_lo, float s, uint8_t *mask);
// clears the bricks of a range-test mask that no trilinear cell of theirs
// makes visible (the exact per-cell vote)
void launch_vote_bricks(Ctx &c, const Volume &v, int B, const TF &tf, float s, uint8_t *mask,
                        int gx, int gy, int gz);
size_t compact_block_count(int64_t nb);
void launch_compact(Ctx &c, const uint8_t *mask, int64_t nb, uint32_t *ids, int *count,
                    uint32_t *block_sums, uint32_t *morton_keys, int gx, int gy);

// lbvh.cu
size_t sort_scratch_words(int64_t cap);
// Boxes in the LBVH's chunk tables for up to cap leaves (6 ints each).
size_t lbvh_chunk_boxes(size_t cap);
int launch_radix_sort(Ctx &c, const uint32_t *keys, const uint32_t *vals, uint32_t *keys_a,
                      uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, const int *count,
                      int64_t cap, int bits, uint32_t *scratch);
void launch_lbvh(Ctx &c, Structure &s);
int lbvh_height(Ctx &c, Structure &s);
void launch_selftest_wait(Ctx &c, uint32_t *flag, bool set, long limit);

// kd.cu
void launch_kd(Ctx &c, Structure &s);
void kd_stats(Ctx &c, Structure &s);
void kd_reserve(Ctx &c, Structure &s, int lvl_size, int S, int cur);
void kd_free(Ctx &c, Structure &s);

// render.cu
struct RenderJob {
    const Volume *vol;
    const TF *tf;
    const Structure *st;
    ess_camera cam;
    ess_render_params rp;
    int W, H;
    float *out;  // device, W*H*4
    int tile_w = 8;  // warp tile width in pixels (4, 8, 16 or 32)
};
void launch_render(Ctx &c, const RenderJob &job);
constexpr int BATCH_MAX = 4096;
size_t batch_bytes(int n);
size_t pack_batch(Ctx &c, const RenderJob *jobs, int n, int tw, void *host, size_t cap);
// Whether a grid render job may use the walk that advances its crossings.
bool grid_dda_inc(const RenderJob &j);
void launch_render_batch(Ctx &c, int kind, ess_dtype dt, bool cells, bool shaded, bool dda_inc,
                         void *dev);
// Whether the render needs the shaded kernels (shading, or an opacity
// correction that changes alpha).
bool render_shaded(const ess_render_params &rp);

}  // namespace ess

struct ess_ctx {
    ess::Ctx c;
};
