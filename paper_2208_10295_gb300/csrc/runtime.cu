// C ABI implementation: context, scenes, sensors, materials, cast and adjoint
// entry points.  Host code validates arguments, owns device buffers and
// enqueues the kernels of build.cu, cast.cu and adjoint.cu on the context
// stream.
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace lidar {

static thread_local std::string g_last_error;

// LIDAR_LOG=1 prints every error message to stderr as it is set, 2 also one
// line per scene build and per cast entry (read once per process).
static int log_level()
{
    static const int level = [] {
        const char* v = getenv("LIDAR_LOG");
        return v ? atoi(v) : 0;
    }();
    return level;
}

void set_error(const std::string& msg)
{
    g_last_error = msg;
    if (log_level() >= 1) fprintf(stderr, "lidar: error: %s\n", msg.c_str());
}

static void log_info(const std::string& msg)
{
    if (log_level() >= 2) fprintf(stderr, "lidar: %s\n", msg.c_str());
}

// NVTX range over one entry point (a profiler's timeline; no cost without a tool)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Host-side allocation fault injection for tests: LIDAR_FAULT_ALLOC_AT=n makes
// the n-th device allocation of the process (1-based) fail with ENOMEM.
static std::mutex g_alloc_mu;
static long g_alloc_count = 0;

static cudaError_t dev_alloc(void** p, size_t bytes)
{
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        ++g_alloc_count;
        const char* f = getenv("LIDAR_FAULT_ALLOC_AT");
        if (f && atol(f) == g_alloc_count) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    if (bytes == 0) bytes = 16;
    return cudaMalloc(p, bytes);
}

struct SensorSlot {
    bool set = false;
    int64_t n_beams = 0;
    float* dirs_dev = nullptr;
    uint32_t* order_dev = nullptr;       // the order the cast kernel follows
    uint32_t* base_order_dev = nullptr;  // Morton order of the beam directions
    float* sweep_dev = nullptr;          // firing fraction of each beam in a sweep
    SensorDev dev{};
};

}  // namespace lidar

using namespace lidar;

struct lidar_scene {
    lidar_ctx* ctx = nullptr;
    float4* nodes = nullptr;
    float4* nodes4 = nullptr;
    float4* tris = nullptr;
    uint32_t* leaf_tri = nullptr;
    uint32_t* orig_to_leaf = nullptr;  // inverse of leaf_tri, made on the first raster cast
    int64_t n_tris = 0;
    int64_t n_nodes = 0;
    int64_t n_nodes4 = 0;
    int levels4 = 0;
    float4* nodes8 = nullptr;  // NULL when the 8-wide tree could need a deeper stack than the traversal has
    int64_t n_nodes8 = 0;
    int levels8 = 0;
    int max_depth = 0;
    double build_ms = 0.0;
    int64_t bytes = 0;
    int64_t treelets = 0;  // treelets the restructuring rewrote
};

static SceneDev scene_dev(const lidar_scene* scene)
{
    return SceneDev{scene->nodes, scene->tris, scene->n_tris, scene->n_nodes,
                    scene->nodes4, scene->n_nodes4, scene->nodes8, scene->n_nodes8};
}

struct lidar_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int* status_dev = nullptr;
    unsigned long long* work_counter = nullptr;
    int* aux_dev = nullptr;  // scratch ints (build height)
    unsigned long long* adj_arrivals = nullptr;  // the one-pass adjoint's grid-wait counter (only grows)
    unsigned long long adj_arrivals_base = 0;    // its value once every launch so far has run
    int coop = 0;                 // the device launches cooperative kernels
    SensorSlot slots[LIDAR_MAX_SENSORS];
    SensorDev* sensors_dev = nullptr;
    TableDev table{nullptr, 0};
    FrameDev* frames_dev = nullptr;      // frame table and tile prefix, one device block
    int64_t* tile_prefix_dev = nullptr;
    size_t frames_cap = 0;
    char* stage_host[2] = {nullptr, nullptr};  // pinned staging of that block, used alternately
    cudaEvent_t stage_done[2] = {nullptr, nullptr};
    int stage_next = 0;
    SweepDev* sweeps_dev = nullptr;
    size_t sweeps_cap = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // three counter regions of direct casts, used in turn: a cast clears the
    // next one, so the next cast needs no memset (cnt_clean); with overlapped
    // casts the region a cast clears was last used by a completed cast
    unsigned* cnt_dev = nullptr;
    int64_t cnt_words = 0;  // per region
    bool cnt_clean[3] = {false, false, false};
    int cnt_cur = 0;
    int overlap = 1;         // consecutive direct casts may overlap (programmatic dependent launch)
    int dense_cur = 0;       // which half of the scratch the next direct cast's dense records use
    std::vector<std::pair<uintptr_t, uintptr_t>> last_out;  // output byte ranges of the last direct cast
    LaunchCfg cfg{128, 4, 32, 1, 2, 1};
    int build_method = 1;     // 0 Karras LBVH, 1 PLOC clustering (fewer node fetches per ray)
    int ploc_radius = 16;
    int collapse = 0;         // wide nodes: 0 open the largest child, 1 SAH dynamic program
    float tri_cost = 1.0f;    // a triangle test's cost relative to a node visit (collapse 1, treelets)
    int treelet_rounds = 0;   // rounds of treelet restructuring of the binary tree
    AreaW area_w{1.0f, 1.0f, 1.0f};  // face weights of the builders' area measure
    std::set<lidar_scene*> scenes;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

lidar_status ensure_scratch(lidar_ctx* c, size_t bytes)
{
    if (c->scratch_bytes >= bytes) return LIDAR_OK;
    if (c->scratch) {
        LIDAR_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    LIDAR_CUDA(dev_alloc(&c->scratch, want));
    c->scratch_bytes = want;
    return LIDAR_OK;
}

lidar_status upload_sensor_slot(lidar_ctx* c, int slot)
{
    SensorDev d = c->slots[slot].dev;
    if (c->cfg.ray_order == 0) d.order = nullptr;
    LIDAR_CUDA(cudaMemcpyAsync(c->sensors_dev + slot, &d, sizeof(SensorDev), cudaMemcpyHostToDevice, c->stream));
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    return LIDAR_OK;
}

lidar_status status_from_word(int w)
{
    switch (w) {
    case ST_OK: return LIDAR_OK;
    case ST_CAPACITY: set_error("point output capacity exceeded"); return LIDAR_ECAPACITY;
    case ST_STACK: set_error("BVH traversal stack overflow"); return LIDAR_ESTACK;
    case ST_TIMEOUT: set_error("a bounded device wait timed out"); return LIDAR_ETIMEOUT;
    case ST_INDEX: set_error("triangle vertex index out of range"); return LIDAR_EINVAL;
    case ST_BOUNDS:
        set_error("an index outside its array (the bounds-checked traversal, or the treelet restructuring of a "
                  "broken tree): corrupt scene data");
        return LIDAR_EINVAL;
    default: set_error("unknown device status"); return LIDAR_ECUDA;
    }
}

BeamsOut to_beams_out(const lidar_beams* b)
{
    BeamsOut o{};
    if (!b) return o;
    o.valid = b->valid; o.tri = b->tri; o.t = b->t; o.range = b->range; o.intensity = b->intensity;
    o.normal = b->normal; o.mat = b->mat; o.inst = b->inst; o.sub = b->sub; o.theta_deg = b->theta_deg;
    o.rf = b->rf;
    return o;
}

}  // namespace

extern "C" {

const char* lidar_last_error(void) { return g_last_error.c_str(); }

lidar_status lidar_create(int device, void* cuda_stream, lidar_ctx** out)
{
    LIDAR_CHECK_ARG(out != nullptr, "lidar_create: out is NULL");
    *out = nullptr;
    int n_dev = 0;
    LIDAR_CUDA(cudaGetDeviceCount(&n_dev));
    LIDAR_CHECK_ARG(device >= 0 && device < n_dev, "lidar_create: no such device");
    DeviceGuard g(device);
    lidar_ctx* c = new lidar_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (!coop) c->cfg.fused_scatter = 0;
    void* p = nullptr;
    cudaError_t e = dev_alloc(&p, 256);
    if (e != cudaSuccess) {
        delete c;
        set_error("lidar_create: device allocation failed");
        return LIDAR_ENOMEM;
    }
    c->status_dev = (int*)p;
    c->work_counter = (unsigned long long*)((char*)p + 64);
    c->aux_dev = (int*)((char*)p + 128);
    c->adj_arrivals = (unsigned long long*)((char*)p + 192);
    c->coop = coop;
    e = dev_alloc((void**)&c->sensors_dev, sizeof(SensorDev) * LIDAR_MAX_SENSORS);
    if (e != cudaSuccess) {
        cudaFree(p);
        delete c;
        set_error("lidar_create: device allocation failed");
        return LIDAR_ENOMEM;
    }
    cudaMemsetAsync(p, 0, 256, c->stream);
    cudaMemsetAsync(c->sensors_dev, 0, sizeof(SensorDev) * LIDAR_MAX_SENSORS, c->stream);
    for (int i = 0; i < 2; ++i) cudaEventCreateWithFlags(&c->stage_done[i], cudaEventDisableTiming);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaFree(p);
        cudaFree(c->sensors_dev);
        delete c;
        set_error("lidar_create: stream synchronisation failed");
        return LIDAR_ECUDA;
    }
    *out = c;
    return LIDAR_OK;
}

void lidar_scene_free(lidar_scene* s)
{
    if (!s) return;
    DeviceGuard g(s->ctx->device);
    cudaStreamSynchronize(s->ctx->stream);
    cudaFree(s->nodes);
    cudaFree(s->nodes4);
    cudaFree(s->nodes8);
    cudaFree(s->tris);
    cudaFree(s->leaf_tri);
    cudaFree(s->orig_to_leaf);
    s->ctx->scenes.erase(s);
    delete s;
}

void lidar_destroy(lidar_ctx* c)
{
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    std::set<lidar_scene*> sc = c->scenes;
    for (lidar_scene* s : sc) lidar_scene_free(s);
    for (auto& sl : c->slots) {
        cudaFree(sl.dirs_dev);
        cudaFree(sl.order_dev);
        cudaFree(sl.base_order_dev);
        cudaFree(sl.sweep_dev);
    }
    cudaFree(c->sensors_dev);
    cudaFree(c->sweeps_dev);
    cudaFree(c->frames_dev);
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(c->stage_host[i]);
        if (c->stage_done[i]) cudaEventDestroy(c->stage_done[i]);
    }
    cudaFree(c->scratch);
    cudaFree(c->cnt_dev);
    cudaFree(c->status_dev);
    delete c;
}

lidar_status lidar_sync_status(lidar_ctx* c)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_sync_status: ctx is NULL");
    DeviceGuard g(c->device);
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    int w = 0;
    LIDAR_CUDA(cudaMemcpy(&w, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost));
    LIDAR_CUDA(cudaMemset(c->status_dev, 0, sizeof(int)));
    return status_from_word(w);
}

lidar_status lidar_scene_build(lidar_ctx* c, const float* verts, int64_t n_verts, const uint32_t* tris,
                               int64_t n_tris, const uint16_t* mat, const uint32_t* inst, lidar_scene** out)
{
    NvtxRange nvtx_("lidar_scene_build");
    LIDAR_CHECK_ARG(c != nullptr && out != nullptr, "lidar_scene_build: ctx/out is NULL");
    *out = nullptr;
    LIDAR_CHECK_ARG(n_tris >= 0 && n_verts >= 0, "lidar_scene_build: negative size");
    LIDAR_CHECK_ARG(n_tris < (int64_t)1 << 31, "lidar_scene_build: more than 2^31 - 1 triangles");
    LIDAR_CHECK_ARG(n_tris == 0 || (verts && tris && n_verts > 0),
                    "lidar_scene_build: verts/tris must be non-NULL for a non-empty mesh");
    DeviceGuard g(c->device);
    lidar_scene* s = new lidar_scene();
    s->ctx = c;
    s->n_tris = n_tris;
    s->n_nodes = n_tris == 0 ? 0 : (n_tris == 1 ? 1 : n_tris - 1);
    auto fail = [&](lidar_status st) {
        cudaFree(s->nodes);
        cudaFree(s->nodes4);
        cudaFree(s->nodes8);
        cudaFree(s->tris);
        cudaFree(s->leaf_tri);
        delete s;
        return st;
    };
    if (n_tris > 0) {
        if (dev_alloc((void**)&s->nodes, (size_t)s->n_nodes * 4 * sizeof(float4)) != cudaSuccess ||
            dev_alloc((void**)&s->nodes4, (size_t)s->n_nodes * 8 * sizeof(float4)) != cudaSuccess ||
            dev_alloc((void**)&s->tris, (size_t)n_tris * 3 * sizeof(float4)) != cudaSuccess ||
            dev_alloc((void**)&s->leaf_tri, (size_t)n_tris * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            set_error("lidar_scene_build: device allocation failed");
            return fail(LIDAR_ENOMEM);
        }
        s->bytes = s->n_nodes * 64 + s->n_nodes * 128 + n_tris * 48 + n_tris * 4;
        lidar_status st = ensure_scratch(c, std::max({build_scratch_bytes(n_tris), collapse_scratch_bytes(s->n_nodes),
                                                      c->build_method == 1 ? ploc_scratch_bytes(n_tris) : (size_t)0,
                                                      c->treelet_rounds > 0 ? treelet_scratch_bytes(n_tris) : (size_t)0}));
        if (st != LIDAR_OK) return fail(st);
        struct Events {
            cudaEvent_t a = nullptr, b = nullptr;
            Events() { cudaEventCreate(&a); cudaEventCreate(&b); }
            ~Events() { cudaEventDestroy(a); cudaEventDestroy(b); }
        } ev;
        cudaEvent_t e0 = ev.a, e1 = ev.b;
        cudaEventRecord(e0, c->stream);
        cudaError_t e = build_lbvh(c->stream, verts, n_verts, tris, mat, inst, n_tris, s->nodes, s->tris,
                                   s->leaf_tri, c->status_dev, c->aux_dev, c->scratch, c->scratch_bytes,
                                   n_tris >= 2 ? c->build_method : 0, c->ploc_radius, c->area_w);
        unsigned long long treelets = 0;
        if (e == cudaSuccess && c->treelet_rounds > 0)
            e = restructure_treelets(c->stream, s->tris, n_tris, s->nodes, c->aux_dev, c->treelet_rounds, c->tri_cost,
                                     c->scratch, c->scratch_bytes, &treelets, c->status_dev, c->area_w);
        cudaEventRecord(e1, c->stream);
        if (e != cudaSuccess) {
            set_error(std::string("lidar_scene_build: ") + cudaGetErrorString(e));
            return fail(LIDAR_ECUDA);
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_error("lidar_scene_build: stream synchronisation failed");
            return fail(LIDAR_ECUDA);
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        s->build_ms = ms;
        s->treelets = (int64_t)treelets;
        int w = 0, h = 0;
        cudaMemcpy(&w, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemcpy(&h, c->aux_dev, sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemset(c->status_dev, 0, sizeof(int));
        s->max_depth = h;
        if (w != ST_OK) return fail(status_from_word(w));
        if (h > kTraversalStack) {
            set_error("lidar_scene_build: BVH height " + std::to_string(h) + " exceeds the traversal stack (" +
                      std::to_string(kTraversalStack) + ")");
            return fail(LIDAR_ESTACK);
        }
        cudaEventRecord(e0, c->stream);
        int need4 = 0;
        cudaError_t e4 = collapse_bvh(c->stream, 4, s->nodes, s->n_nodes, s->nodes4, &s->n_nodes4, &s->levels4,
                                      &need4, c->scratch, c->scratch_bytes, c->collapse, c->tri_cost, c->area_w);
        // the 8-wide tree: count its nodes and the stack it could need, then
        // write it into an exact allocation; a tree that could need more than
        // the traversal stack is not kept (the 4-wide and binary ones serve)
        int64_t n8 = 0;
        int levels8 = 0, need8 = 0;
        if (e4 == cudaSuccess)
            e4 = collapse_bvh(c->stream, 8, s->nodes, s->n_nodes, nullptr, &n8, &levels8, &need8, c->scratch,
                              c->scratch_bytes, c->collapse, c->tri_cost, c->area_w);
        if (e4 == cudaSuccess && need8 <= kTraversalStack && n8 > 0) {
            if (dev_alloc((void**)&s->nodes8, (size_t)n8 * 16 * sizeof(float4)) != cudaSuccess) {
                cudaGetLastError();
                set_error("lidar_scene_build: device allocation failed (8-wide tree)");
                return fail(LIDAR_ENOMEM);
            }
            e4 = collapse_bvh(c->stream, 8, s->nodes, s->n_nodes, s->nodes8, &s->n_nodes8, &s->levels8, &need8,
                              c->scratch, c->scratch_bytes, c->collapse, c->tri_cost, c->area_w);
            s->bytes += s->n_nodes8 * 256;
        }
        cudaEventRecord(e1, c->stream);
        if (e4 != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_error(std::string("lidar_scene_build: wide collapse: ") + cudaGetErrorString(e4));
            return fail(LIDAR_ECUDA);
        }
        cudaEventElapsedTime(&ms, e0, e1);
        s->build_ms += ms;
        if (need4 > kTraversalStack) {
            set_error("lidar_scene_build: 4-wide BVH could need " + std::to_string(need4) +
                      " stack entries, more than the traversal stack (" + std::to_string(kTraversalStack) + ")");
            return fail(LIDAR_ESTACK);
        }
    }
    c->scenes.insert(s);
    *out = s;
    log_info("scene built: " + std::to_string(n_tris) + " triangles, " + std::to_string(s->n_nodes4) +
             " 4-wide and " + std::to_string(s->n_nodes8) + " 8-wide nodes, " + std::to_string(s->build_ms) + " ms");
    return LIDAR_OK;
}

lidar_status lidar_get_scene_info(const lidar_scene* s, lidar_scene_info* out)
{
    LIDAR_CHECK_ARG(s != nullptr && out != nullptr, "lidar_get_scene_info: NULL argument");
    out->n_tris = s->n_tris;
    out->n_nodes = s->n_nodes;
    out->max_depth = s->max_depth;
    out->device_bytes = s->bytes;
    out->build_ms = s->build_ms;
    out->n_nodes4 = s->n_nodes4;
    out->levels4 = s->levels4;
    out->n_nodes8 = s->n_nodes8;
    out->levels8 = s->levels8;
    out->treelets = s->treelets;
    return LIDAR_OK;
}

lidar_status lidar_scene_export(const lidar_scene* s, float* nodes_host, uint32_t* leaf_tri_host)
{
    LIDAR_CHECK_ARG(s != nullptr, "lidar_scene_export: scene is NULL");
    DeviceGuard g(s->ctx->device);
    LIDAR_CUDA(cudaStreamSynchronize(s->ctx->stream));
    if (nodes_host && s->n_nodes)
        LIDAR_CUDA(cudaMemcpy(nodes_host, s->nodes, (size_t)s->n_nodes * 64, cudaMemcpyDeviceToHost));
    if (leaf_tri_host && s->n_tris)
        LIDAR_CUDA(cudaMemcpy(leaf_tri_host, s->leaf_tri, (size_t)s->n_tris * 4, cudaMemcpyDeviceToHost));
    return LIDAR_OK;
}

lidar_status lidar_scene_export_wide(const lidar_scene* s, int32_t width, float* nodes_host)
{
    LIDAR_CHECK_ARG(s != nullptr && nodes_host != nullptr, "lidar_scene_export_wide: NULL argument");
    LIDAR_CHECK_ARG(width == 4 || width == 8, "lidar_scene_export_wide: width is 4 or 8");
    LIDAR_CHECK_ARG(width == 4 || s->nodes8 != nullptr || s->n_tris == 0,
                    "lidar_scene_export_wide: the scene has no 8-wide tree");
    DeviceGuard g(s->ctx->device);
    LIDAR_CUDA(cudaStreamSynchronize(s->ctx->stream));
    const int64_t n = width == 4 ? s->n_nodes4 : s->n_nodes8;
    if (n)
        LIDAR_CUDA(cudaMemcpy(nodes_host, width == 4 ? s->nodes4 : s->nodes8, (size_t)n * 32 * width,
                              cudaMemcpyDeviceToHost));
    return LIDAR_OK;
}

lidar_status lidar_set_sensor(lidar_ctx* c, int32_t slot, const lidar_sensor_desc* d)
{
    LIDAR_CHECK_ARG(c != nullptr && d != nullptr, "lidar_set_sensor: NULL argument");
    LIDAR_CHECK_ARG(slot >= 0 && slot < LIDAR_MAX_SENSORS, "lidar_set_sensor: slot out of range");
    LIDAR_CHECK_ARG(d->n_beams > 0 && d->n_beams < (int64_t)1 << 31, "lidar_set_sensor: n_beams out of range");
    LIDAR_CHECK_ARG(d->az_rad && d->el_rad, "lidar_set_sensor: az_rad/el_rad are NULL");
    LIDAR_CHECK_ARG(d->n_subrays >= 1 && d->n_subrays <= LIDAR_MAX_SUBRAYS, "lidar_set_sensor: n_subrays out of range");
    LIDAR_CHECK_ARG(d->r_min >= 0.0f && d->r_max > d->r_min, "lidar_set_sensor: need 0 <= r_min < r_max");
    LIDAR_CHECK_ARG(d->d_max > 0.0f && d->RL_max >= 0.0f, "lidar_set_sensor: need d_max > 0, RL_max >= 0");
    LIDAR_CHECK_ARG(d->sigma >= 0.0f && isfinite(d->sigma), "lidar_set_sensor: sigma must be finite, >= 0");
    LIDAR_CHECK_ARG(d->sigma_k >= 0.0f && d->sigma_k < 0.1f, "lidar_set_sensor: sigma_k must be in [0, 0.1)");
    LIDAR_CHECK_ARG(d->divergence_rad >= 0.0f && d->divergence_rad < 0.1f, "lidar_set_sensor: divergence out of range");
    DeviceGuard g(c->device);
    const int64_t n = d->n_beams;
    // FP32 unit directions from the FP64 spherical coordinates
    std::vector<float> dirs((size_t)n * 3);
    for (int64_t b = 0; b < n; ++b) {
        const double ce = cos(d->el_rad[b]);
        dirs[3 * b + 0] = (float)(ce * cos(d->az_rad[b]));
        dirs[3 * b + 1] = (float)(ce * sin(d->az_rad[b]));
        dirs[3 * b + 2] = (float)sin(d->el_rad[b]);
    }
    SensorSlot& sl = c->slots[slot];
    if (sl.set) {
        LIDAR_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(sl.dirs_dev);
        cudaFree(sl.order_dev);
        cudaFree(sl.base_order_dev);
        cudaFree(sl.sweep_dev);
        sl = SensorSlot();
    }
    if (dev_alloc((void**)&sl.dirs_dev, n * 3 * sizeof(float)) != cudaSuccess ||
        dev_alloc((void**)&sl.order_dev, n * sizeof(uint32_t)) != cudaSuccess ||
        dev_alloc((void**)&sl.base_order_dev, n * sizeof(uint32_t)) != cudaSuccess ||
        dev_alloc((void**)&sl.sweep_dev, n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sl.dirs_dev);
        cudaFree(sl.order_dev);
        cudaFree(sl.base_order_dev);
        sl = SensorSlot();
        set_error("lidar_set_sensor: device allocation failed");
        return LIDAR_ENOMEM;
    }
    LIDAR_CUDA(cudaMemcpyAsync(sl.dirs_dev, dirs.data(), n * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    // firing fraction in a sweep: azimuth over 2 pi in [0, 1) (the sweep starts at azimuth 0, towards +y)
    std::vector<float> frac((size_t)n);
    for (int64_t b = 0; b < n; ++b) {
        double s = fmod(d->az_rad[b], 2.0 * M_PI) / (2.0 * M_PI);
        if (s < 0.0) s += 1.0;
        if (s >= 1.0) s = 0.0;
        frac[(size_t)b] = (float)s;
    }
    LIDAR_CUDA(cudaMemcpyAsync(sl.sweep_dev, frac.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    lidar_status st = ensure_scratch(c, ray_order_scratch_bytes(n));
    if (st != LIDAR_OK) return st;
    LIDAR_CUDA(launch_ray_order(c->stream, sl.dirs_dev, (int)n, sl.base_order_dev, c->scratch, c->scratch_bytes));
    LIDAR_CUDA(cudaMemcpyAsync(sl.order_dev, sl.base_order_dev, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                               c->stream));
    SensorDev& sd = sl.dev;
    sd.dirs = sl.dirs_dev;
    sd.sweep = sl.sweep_dev;
    sd.order = sl.order_dev;
    sd.n_beams = (int32_t)n;
    sd.n_sub = d->n_subrays;
    sd.r_min = d->r_min; sd.r_max = d->r_max; sd.d_max = d->d_max; sd.RL_max = d->RL_max;
    sd.sigma = d->sigma; sd.gain = d->gain; sd.range_exp = d->range_exp; sd.r_ref = d->r_ref;
    sd.sigma_k = d->sigma_k;
    // |z| <= 8.6 for the 53-bit uniforms: t (1 - 9 sigma_k) - 9 sigma > d_lim for any t beyond this
    sd.t_max = (fminf(d->r_max, d->d_max) + 9.0f * d->sigma) / (1.0f - 9.0f * d->sigma_k);
    // sub-ray offsets: ray 0 is the beam, rays 1..n-1 on the cone of half-angle divergence/2
    const double rad = tan(0.5 * (double)d->divergence_rad);
    for (int k = 0; k < LIDAR_MAX_SUBRAYS; ++k) {
        sd.alpha[k] = 0.0f;
        sd.beta[k] = 0.0f;
    }
    for (int k = 1; k < d->n_subrays; ++k) {
        const double a = 2.0 * M_PI * (double)(k - 1) / (double)(d->n_subrays - 1);
        sd.alpha[k] = (float)(rad * cos(a));
        sd.beta[k] = (float)(rad * sin(a));
    }
    sl.n_beams = n;
    sl.set = true;
    return upload_sensor_slot(c, slot);
}

lidar_status lidar_set_sensor_gain(lidar_ctx* c, int32_t slot, float gain)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_set_sensor_gain: ctx is NULL");
    LIDAR_CHECK_ARG(slot >= 0 && slot < LIDAR_MAX_SENSORS, "lidar_set_sensor_gain: slot out of range");
    LIDAR_CHECK_ARG(isfinite(gain), "lidar_set_sensor_gain: gain must be finite");
    if (!c->slots[slot].set) {
        set_error("lidar_set_sensor_gain: no sensor in this slot");
        return LIDAR_ESTATE;
    }
    DeviceGuard g(c->device);
    c->slots[slot].dev.gain = gain;
    return upload_sensor_slot(c, slot);
}

lidar_status lidar_get_beam_dirs(lidar_ctx* c, int32_t slot, float* host_out)
{
    LIDAR_CHECK_ARG(c != nullptr && host_out != nullptr, "lidar_get_beam_dirs: NULL argument");
    LIDAR_CHECK_ARG(slot >= 0 && slot < LIDAR_MAX_SENSORS, "lidar_get_beam_dirs: slot out of range");
    if (!c->slots[slot].set) {
        set_error("lidar_get_beam_dirs: no sensor in this slot");
        return LIDAR_ESTATE;
    }
    DeviceGuard g(c->device);
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    LIDAR_CUDA(cudaMemcpy(host_out, c->slots[slot].dirs_dev, c->slots[slot].n_beams * 3 * sizeof(float),
                          cudaMemcpyDeviceToHost));
    return LIDAR_OK;
}

lidar_status lidar_build_tables(lidar_ctx* c, const float* params, int32_t M, float* table)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_build_tables: ctx is NULL");
    LIDAR_CHECK_ARG(M >= 0 && (M == 0 || (params && table)), "lidar_build_tables: bad arguments");
    DeviceGuard g(c->device);
    LIDAR_CUDA(launch_build_tables(c->stream, params, M, table));
    return LIDAR_OK;
}

lidar_status lidar_build_tables_backward(lidar_ctx* c, const float* params, const float* grad_table, int32_t M,
                                         float* grad_params)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_build_tables_backward: ctx is NULL");
    LIDAR_CHECK_ARG(M >= 0 && (M == 0 || (params && grad_table && grad_params)),
                    "lidar_build_tables_backward: bad arguments");
    DeviceGuard g(c->device);
    LIDAR_CUDA(launch_build_tables_backward(c->stream, params, grad_table, M, grad_params));
    return LIDAR_OK;
}

lidar_status lidar_set_materials(lidar_ctx* c, const float* table, int32_t M)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_set_materials: ctx is NULL");
    LIDAR_CHECK_ARG(table != nullptr && M > 0 && M <= 65536, "lidar_set_materials: need a table with 1..65536 rows");
    c->table.table = table;
    c->table.n_mat = M;
    return LIDAR_OK;
}

// shared front half of the cast entry points
// Frame records and tile prefix of a cast.  With `inl` and at most
// kInlineFrames frames they go into *inl (the launch parameters) and nothing
// is copied to the device; otherwise into the device table.
static lidar_status prepare_frames(lidar_ctx* c, const lidar_frame* frames, int32_t n_frames, int64_t* n_beams_total,
                                   int64_t* n_tiles, InlineFrames* inl = nullptr)
{
    LIDAR_CHECK_ARG(frames != nullptr && n_frames > 0, "lidar_cast: need at least one frame");
    std::vector<FrameDev> fd((size_t)n_frames);
    std::vector<int64_t> prefix((size_t)n_frames);
    int64_t off = 0, tiles = 0;
    const int tr = c->cfg.tile_rays;
    for (int32_t k = 0; k < n_frames; ++k) {
        const int s = frames[k].sensor;
        if (s < 0 || s >= LIDAR_MAX_SENSORS || !c->slots[s].set) {
            set_error("lidar_cast: frame " + std::to_string(k) + " names an empty sensor slot");
            return LIDAR_ESTATE;
        }
        for (int j = 0; j < 12; ++j)
            LIDAR_CHECK_ARG(isfinite(frames[k].pose[j]), "lidar_cast: non-finite pose");
        fd[k].sensor = s;
        fd[k].frame = frames[k].frame;
        fd[k].beam_offset = off;
        memcpy(fd[k].pose, frames[k].pose, sizeof(fd[k].pose));
        prefix[k] = tiles;
        off += c->slots[s].n_beams;
        tiles += (c->slots[s].n_beams + tr - 1) / tr;
    }
    if (inl) inl->n = 0;
    if (inl && n_frames <= kInlineFrames) {
        for (int32_t k = 0; k < n_frames; ++k) {
            inl->f[k] = fd[k];
            inl->prefix[k] = prefix[k];
        }
        inl->n = n_frames;
        *n_beams_total = off;
        *n_tiles = tiles;
        return LIDAR_OK;
    }
    // frame table and tile prefix travel as one block: frames, then the prefix at a 256-byte boundary
    const size_t prefix_at = ((size_t)n_frames * sizeof(FrameDev) + 255) / 256 * 256;
    const size_t block = prefix_at + (size_t)n_frames * sizeof(int64_t);
    if ((size_t)n_frames > c->frames_cap) {
        LIDAR_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->frames_dev);
        for (int i = 0; i < 2; ++i) {
            cudaFreeHost(c->stage_host[i]);
            c->stage_host[i] = nullptr;
        }
        c->frames_dev = nullptr;
        c->tile_prefix_dev = nullptr;
        c->frames_cap = 0;
        if (dev_alloc((void**)&c->frames_dev, block) != cudaSuccess) {
            cudaGetLastError();
            set_error("lidar_cast: device allocation failed");
            return LIDAR_ENOMEM;
        }
        for (int i = 0; i < 2; ++i)
            if (cudaHostAlloc((void**)&c->stage_host[i], block, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                set_error("lidar_cast: pinned host allocation failed");
                return LIDAR_ENOMEM;
            }
        c->tile_prefix_dev = (int64_t*)((char*)c->frames_dev + prefix_at);
        c->frames_cap = n_frames;
    }
    // the block's device layout depends on n_frames: keep the prefix pointer in step
    c->tile_prefix_dev = (int64_t*)((char*)c->frames_dev + prefix_at);
    // pinned staging used alternately: wait until the copy made from this buffer two calls ago is done
    const int slot = c->stage_next;
    c->stage_next ^= 1;
    LIDAR_CUDA(cudaEventSynchronize(c->stage_done[slot]));
    memcpy(c->stage_host[slot], fd.data(), (size_t)n_frames * sizeof(FrameDev));
    memcpy(c->stage_host[slot] + prefix_at, prefix.data(), (size_t)n_frames * sizeof(int64_t));
    LIDAR_CUDA(cudaMemcpyAsync(c->frames_dev, c->stage_host[slot], block, cudaMemcpyHostToDevice, c->stream));
    LIDAR_CUDA(cudaEventRecord(c->stage_done[slot], c->stream));
    *n_beams_total = off;
    *n_tiles = tiles;
    return LIDAR_OK;
}

// scratch bytes a cast of n_total beams needs (all dense intermediates of the
// compaction plus its own scratch): used to pre-size scratch for batches
static size_t cast_scratch_upper_bound(int64_t n_total)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(n_total) + 2 * al(4 * n_total) + al(12 * n_total) + al(2 * n_total) + al(4 * n_total) +
           fused_compact_scratch_bytes(n_total);
}

// The 8-wide traversal needs the scene's 8-wide tree (not kept for trees that
// could need a deeper stack than the traversal has).
static lidar_status traversal_available(const lidar_ctx* c, const lidar_scene* scene, const char* who)
{
    if (c->cfg.traversal == 3 && scene->n_tris > 0 && scene->nodes8 == nullptr) {
        set_error(std::string(who) + ": traversal 3 needs the scene's 8-wide tree, which this scene does not have");
        return LIDAR_EINVAL;
    }
    return LIDAR_OK;
}

// Cast over frames already on the device.  `may_alloc` false: fail instead of
// growing the scratch (stream capture, batches).
// The counter region of a direct cast (`direct`: not captured, not a batch):
// the region the previous cast did not use, which that cast cleared.
static lidar_status counter_region(lidar_ctx* c, int64_t n_total, bool compact, CounterRegion* R)
{
    const int64_t need = ((int64_t)cast_counter_bytes(n_total, compact) + 3) / 4;
    if (c->cnt_words < need) {
        LIDAR_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->cnt_dev);
        c->cnt_dev = nullptr;
        c->cnt_words = 0;
        const int64_t words = (std::max<int64_t>(need, 256) + 63) / 64 * 64;
        if (dev_alloc((void**)&c->cnt_dev, (size_t)(3 * words) * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cast: device allocation failed (counters)");
            return LIDAR_ENOMEM;
        }
        c->cnt_words = words;
        c->cnt_clean[0] = c->cnt_clean[1] = c->cnt_clean[2] = false;
    }
    const int r = (c->cnt_cur + 1) % 3;
    R->base = c->cnt_dev + (int64_t)r * c->cnt_words;
    R->clean = c->cnt_clean[r];
    R->zero_next = c->cnt_dev + (int64_t)((r + 1) % 3) * c->cnt_words;
    R->zero_words = c->cnt_words;
    R->overlap = c->overlap != 0;
    return LIDAR_OK;
}

static lidar_status cast_impl(lidar_ctx* c, const lidar_scene* scene, const FrameDev* frames_dev,
                              const int64_t* prefix_dev, int32_t n_frames, int64_t n_total, int64_t n_tiles,
                              uint64_t seed, const lidar_beams* beams, const lidar_points* points,
                              int64_t* n_points_dev, bool may_alloc, const InlineFrames* inl = nullptr,
                              bool direct = false)
{
    lidar_status tst = traversal_available(c, scene, "cast");
    if (tst != LIDAR_OK) return tst;
    BeamsOut out = to_beams_out(beams);
    // a direct cast outside a stream capture counts in its own counter region
    // and may overlap the direct cast before it
    bool use_region = false;
    if (direct) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        LIDAR_CUDA(cudaStreamIsCapturing(c->stream, &cs));
        use_region = cs == cudaStreamCaptureStatusNone;
    }
    const bool overlapped = use_region && c->overlap != 0;
    // compaction reads the dense records: provide the ones the points need
    char* dense_base = nullptr;
    size_t dense_bytes = 0;
    if (points) {
        const bool need_valid = out.valid == nullptr, need_range = out.range == nullptr;
        const bool need_int = out.intensity == nullptr, need_norm = points->normal && out.normal == nullptr;
        const bool need_mat = points->material && out.mat == nullptr, need_inst = points->instance && out.inst == nullptr;
        auto al = [](size_t b) { return (b + 255) / 256 * 256; };
        dense_bytes = (need_valid ? al(n_total) : 0) + (need_range ? al(4 * n_total) : 0) +
                      (need_int ? al(4 * n_total) : 0) + (need_norm ? al(12 * n_total) : 0) +
                      (need_mat ? al(2 * n_total) : 0) + (need_inst ? al(4 * n_total) : 0);
        const size_t need = dense_bytes + fused_compact_scratch_bytes(n_total);
        // overlapped casts use the two halves of the scratch in turn, so a cast
        // does not overwrite the records the cast before it still compacts
        const size_t half = (need + 255) / 256 * 256;
        const size_t total = overlapped ? 2 * half : need;
        if (c->scratch_bytes < total) {
            if (!may_alloc) {
                set_error("cast: scratch too small for this batch (recreate the batch)");
                return LIDAR_ESTATE;
            }
            lidar_status st = ensure_scratch(c, total);
            if (st != LIDAR_OK) return st;
        }
        char* p = (char*)c->scratch;
        if (overlapped) {
            // the halves split the scratch at a fixed point, whatever each cast needs
            p += (size_t)c->dense_cur * (c->scratch_bytes / 2 / 256 * 256);
            c->dense_cur ^= 1;
        }
        dense_base = p;
        if (need_valid) { out.valid = (uint8_t*)p; p += al(n_total); }
        if (need_range) { out.range = (float*)p; p += al(4 * n_total); }
        if (need_int) { out.intensity = (float*)p; p += al(4 * n_total); }
        if (need_norm) { out.normal = (float*)p; p += al(12 * n_total); }
        if (need_mat) { out.mat = (uint16_t*)p; p += al(2 * n_total); }
        if (need_inst) { out.inst = (uint32_t*)p; p += al(4 * n_total); }
    }
    SceneDev S = scene_dev(scene);
    char* comp = points ? dense_base + dense_bytes : nullptr;
    bool scattered = false;
    CounterRegion R{};
    if (use_region) {
        lidar_status rs = counter_region(c, n_total, points != nullptr, &R);
        if (rs != LIDAR_OK) return rs;
        // overlap the previous direct cast only when no output of this cast
        // shares memory with one of its outputs (else plain stream order)
        std::vector<std::pair<uintptr_t, uintptr_t>> mine;
        auto add = [&](const void* p, size_t bytes) {
            if (p && bytes) mine.emplace_back((uintptr_t)p, (uintptr_t)p + bytes);
        };
        if (beams) {
            const size_t n = (size_t)n_total;
            add(beams->valid, n); add(beams->tri, 4 * n); add(beams->t, 4 * n); add(beams->range, 4 * n);
            add(beams->intensity, 4 * n); add(beams->normal, 12 * n); add(beams->mat, 2 * n); add(beams->inst, 4 * n);
            add(beams->sub, n); add(beams->theta_deg, 4 * n); add(beams->rf, 4 * n);
        }
        if (points) {
            const size_t m = (size_t)points->capacity;
            add(points->xyz, 12 * m); add(points->range, 4 * m); add(points->intensity, 4 * m);
            add(points->normal, 12 * m); add(points->material, 2 * m); add(points->instance, 4 * m);
            add(points->beam, 4 * m); add(points->frame, 4 * m);
        }
        add(n_points_dev, sizeof(int64_t));
        bool shared = false;
        for (const auto& a : mine)
            for (const auto& b : c->last_out)
                if (a.first < b.second && b.first < a.second) shared = true;
        R.overlap = R.overlap && !shared;
        c->last_out.swap(mine);
    }
    cudaError_t refused = cudaSuccess;
    R.overlap_refused = &refused;
    const cudaError_t le = launch_cast(c->stream, S, c->sensors_dev, frames_dev, n_frames, prefix_dev, n_tiles,
                                       c->table, seed, out, c->status_dev, c->work_counter, c->cfg, c->num_sms,
                                       n_total, nullptr, comp, n_points_dev, points, &scattered, inl,
                                       use_region ? &R : nullptr);
    if (refused != cudaSuccess)
        log_info(std::string("cast: overlapped launch refused (") + cudaGetErrorString(refused) +
                 "), launched after the previous cast instead");
    if (use_region) {
        // this cast dirtied its region and clears the next one
        const int r = (c->cnt_cur + 1) % 3;
        c->cnt_clean[r] = false;
        c->cnt_clean[(r + 1) % 3] = le == cudaSuccess;
        c->cnt_cur = r;
    }
    LIDAR_CUDA(le);
    if (points && !scattered)
        LIDAR_CUDA(launch_scatter(c->stream, c->sensors_dev, frames_dev, n_frames, n_total, out, *points, comp,
                                  c->status_dev, inl, c->num_sms, use_region && R.overlap && refused == cudaSuccess));
    return LIDAR_OK;
}

static lidar_status cast_checks(lidar_ctx* c, const lidar_scene* scene, const lidar_beams* beams,
                                const lidar_points* points)
{
    LIDAR_CHECK_ARG(c != nullptr && scene != nullptr, "lidar_cast: ctx/scene is NULL");
    LIDAR_CHECK_ARG(scene->ctx == c, "lidar_cast: scene belongs to another context");
    if (c->table.table == nullptr) {
        set_error("lidar_cast: no material table (lidar_set_materials)");
        return LIDAR_ESTATE;
    }
    LIDAR_CHECK_ARG(beams != nullptr || points != nullptr, "lidar_cast: nothing to write (beams and points NULL)");
    LIDAR_CHECK_ARG(points == nullptr || points->capacity >= 0, "lidar_cast: negative capacity");
    return LIDAR_OK;
}

lidar_status lidar_points_download(lidar_ctx* c, const lidar_points* dev, const lidar_points* host, int64_t count,
                                   void* stream)
{
    NvtxRange nvtx_("lidar_points_download");
    LIDAR_CHECK_ARG(c != nullptr && dev != nullptr && host != nullptr, "lidar_points_download: NULL argument");
    LIDAR_CHECK_ARG(count >= 0 && count <= dev->capacity && count <= host->capacity,
                    "lidar_points_download: count must be in [0, both capacities]");
    if (count == 0) return LIDAR_OK;
    DeviceGuard g(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const size_t n = (size_t)count;
    auto copy = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        if (dst == nullptr || src == nullptr) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    };
    LIDAR_CUDA(copy(host->xyz, dev->xyz, 3 * n * sizeof(float)));
    LIDAR_CUDA(copy(host->range, dev->range, n * sizeof(float)));
    LIDAR_CUDA(copy(host->intensity, dev->intensity, n * sizeof(float)));
    LIDAR_CUDA(copy(host->normal, dev->normal, 3 * n * sizeof(float)));
    LIDAR_CUDA(copy(host->material, dev->material, n * sizeof(uint16_t)));
    LIDAR_CUDA(copy(host->instance, dev->instance, n * sizeof(uint32_t)));
    LIDAR_CUDA(copy(host->beam, dev->beam, n * sizeof(uint32_t)));
    LIDAR_CUDA(copy(host->frame, dev->frame, n * sizeof(uint32_t)));
    return LIDAR_OK;
}

lidar_status lidar_cast(lidar_ctx* c, const lidar_scene* scene, const lidar_frame* frames, int32_t n_frames,
                        uint64_t seed, const lidar_beams* beams, const lidar_points* points, int64_t* n_points_dev)
{
    NvtxRange nvtx_("lidar_cast");
    lidar_status st = cast_checks(c, scene, beams, points);
    if (st != LIDAR_OK) return st;
    DeviceGuard g(c->device);
    int64_t n_total = 0, n_tiles = 0;
    InlineFrames inl;
    st = prepare_frames(c, frames, n_frames, &n_total, &n_tiles, &inl);
    if (st != LIDAR_OK) return st;
    if (log_level() >= 2)
        log_info("cast: " + std::to_string(n_frames) + " frames, " + std::to_string(n_total) + " beams, traversal " +
                 std::to_string(c->cfg.traversal) + (points ? ", point cloud" : ""));
    return cast_impl(c, scene, c->frames_dev, c->tile_prefix_dev, n_frames, n_total, n_tiles, seed, beams, points,
                     n_points_dev, true, &inl, true);
}

}  // extern "C"

// ------------------------------------------------------------ raster path

static lidar_status raster_setup(lidar_ctx* c, const lidar_scene* scene, const lidar_raster_config* cfg,
                                 bool with_tri, RasterCams& C)
{
    LIDAR_CHECK_ARG(c != nullptr && scene != nullptr && cfg != nullptr, "raster: NULL argument");
    LIDAR_CHECK_ARG(scene->ctx == c, "raster: scene belongs to another context");
    LIDAR_CHECK_ARG(cfg->width >= 1 && cfg->width <= 16384, "raster: width must be in [1, 16384]");
    LIDAR_CHECK_ARG(cfg->n_cameras >= 3 && cfg->n_cameras <= kMaxCameras, "raster: n_cameras must be in [3, 64]");
    LIDAR_CHECK_ARG(scene->n_tris < ((int64_t)1 << 26), "raster: at most 2^26 triangles");
    C.W = cfg->width;
    C.K = cfg->n_cameras;
    const double fov = 2.0 * M_PI / (double)C.K;
    C.f = (float)((double)C.W / (2.0 * tan(0.5 * fov)));
    C.c = (float)(0.5 * (double)C.W);
    for (int k = 0; k < kMaxCameras; ++k) {
        const double az = -M_PI + ((double)k + 0.5) * fov;
        C.ck[k] = k < C.K ? (float)cos(az) : 0.0f;
        C.sk[k] = k < C.K ? (float)sin(az) : 0.0f;
    }
    lidar_scene* sc = const_cast<lidar_scene*>(scene);
    if (!sc->orig_to_leaf && sc->n_tris > 0) {
        if (dev_alloc((void**)&sc->orig_to_leaf, (size_t)sc->n_tris * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            sc->orig_to_leaf = nullptr;
            set_error("raster: device allocation failed");
            return LIDAR_ENOMEM;
        }
        LIDAR_CUDA(launch_invert_leaf_order(c->stream, sc->leaf_tri, sc->n_tris, sc->orig_to_leaf));
    }
    return ensure_scratch(c, raster_scratch_bytes(C.W, C.K, scene->n_tris, with_tri));
}

static RasterFrame raster_frame(const RasterCams& C, const lidar_frame& fr, float t_max)
{
    RasterFrame F;
    memcpy(F.pose, fr.pose, sizeof(F.pose));
    F.t_max = t_max;
    for (int k = 0; k < kMaxCameras; ++k) {
        // sensor-frame axes L = (-s, c, 0), U = (0, 0, 1), F = (c, s, 0), rotated by the pose
        const double ax[3][3] = {{-(double)C.sk[k], (double)C.ck[k], 0.0}, {0.0, 0.0, 1.0},
                                 {(double)C.ck[k], (double)C.sk[k], 0.0}};
        for (int a = 0; a < 3; ++a)
            for (int r = 0; r < 3; ++r)
                F.axes[9 * k + 3 * a + r] =
                    (float)((double)fr.pose[4 * r] * ax[a][0] + (double)fr.pose[4 * r + 1] * ax[a][1] +
                            (double)fr.pose[4 * r + 2] * ax[a][2]);
    }
    return F;
}


extern "C" {

lidar_status lidar_raster_cast(lidar_ctx* c, const lidar_scene* scene, const lidar_frame* frames, int32_t n_frames,
                               uint64_t seed, const lidar_raster_config* cfg, const lidar_beams* beams)
{
    NvtxRange nvtx_("lidar_raster_cast");
    LIDAR_CHECK_ARG(beams != nullptr, "lidar_raster_cast: beams is NULL");
    LIDAR_CHECK_ARG(frames != nullptr && n_frames > 0, "lidar_raster_cast: need at least one frame");
    lidar_status st = cast_checks(c, scene, beams, nullptr);
    if (st != LIDAR_OK) return st;
    for (int32_t k = 0; k < n_frames; ++k) {
        const int s = frames[k].sensor;
        LIDAR_CHECK_ARG(s >= 0 && s < LIDAR_MAX_SENSORS, "lidar_raster_cast: sensor slot out of range");
        if (!c->slots[s].set) {
            set_error("lidar_raster_cast: frame " + std::to_string(k) + " names an empty sensor slot");
            return LIDAR_ESTATE;
        }
        for (int j = 0; j < 12; ++j)
            LIDAR_CHECK_ARG(isfinite(frames[k].pose[j]), "lidar_raster_cast: non-finite pose");
    }
    DeviceGuard g(c->device);
    RasterCams C;
    const BeamsOut out = to_beams_out(beams);
    st = raster_setup(c, scene, cfg, out.tri != nullptr, C);
    if (st != LIDAR_OK) return st;
    const SceneDev S = scene_dev(scene);
    int64_t offset = 0;
    for (int32_t k = 0; k < n_frames; ++k) {
        const SensorSlot& sl = c->slots[frames[k].sensor];
        const RasterFrame F = raster_frame(C, frames[k], sl.dev.t_max);
        GBuffer G{};
        LIDAR_CUDA(launch_rasterise(c->stream, S, C, F, scene->orig_to_leaf, c->scratch, out.tri != nullptr, &G,
                                    c->num_sms));
        LIDAR_CUDA(launch_resample(c->stream, C, F, c->sensors_dev, frames[k].sensor, (int)sl.n_beams, frames[k].frame,
                                   offset, c->table, seed, G, out));
        offset += sl.n_beams;
    }
    return LIDAR_OK;
}

// Unit quaternion (w, x, y, z) of a pose's rotation part, FP64: Shepperd's
// method (the largest of trace and diagonal entries picks the stable formula).
static void rotation_quaternion(const float* P, double q[4])
{
    const double r00 = P[0], r01 = P[1], r02 = P[2], r10 = P[4], r11 = P[5], r12 = P[6];
    const double r20 = P[8], r21 = P[9], r22 = P[10];
    const double tr = r00 + r11 + r22;
    if (tr >= r00 && tr >= r11 && tr >= r22) {
        const double r = sqrt(1.0 + tr), h = 0.5 / r;
        q[0] = 0.5 * r; q[1] = (r21 - r12) * h; q[2] = (r02 - r20) * h; q[3] = (r10 - r01) * h;
    } else if (r00 >= r11 && r00 >= r22) {
        const double r = sqrt(1.0 + r00 - r11 - r22), h = 0.5 / r;
        q[0] = (r21 - r12) * h; q[1] = 0.5 * r; q[2] = (r01 + r10) * h; q[3] = (r02 + r20) * h;
    } else if (r11 >= r22) {
        const double r = sqrt(1.0 + r11 - r00 - r22), h = 0.5 / r;
        q[0] = (r02 - r20) * h; q[1] = (r01 + r10) * h; q[2] = 0.5 * r; q[3] = (r12 + r21) * h;
    } else {
        const double r = sqrt(1.0 + r22 - r00 - r11), h = 0.5 / r;
        q[0] = (r10 - r01) * h; q[1] = (r02 + r20) * h; q[2] = (r12 + r21) * h; q[3] = 0.5 * r;
    }
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

lidar_status lidar_cast_sweep(lidar_ctx* c, const lidar_scene* scene, const lidar_sweep_frame* frames,
                              int32_t n_frames, uint64_t seed, const lidar_beams* beams, const lidar_echoes* echoes)
{
    NvtxRange nvtx_("lidar_cast_sweep");
    LIDAR_CHECK_ARG(c != nullptr && scene != nullptr, "lidar_cast_sweep: ctx/scene is NULL");
    LIDAR_CHECK_ARG(scene->ctx == c, "lidar_cast_sweep: scene belongs to another context");
    LIDAR_CHECK_ARG(frames != nullptr && n_frames > 0, "lidar_cast_sweep: need at least one frame");
    LIDAR_CHECK_ARG(beams != nullptr || echoes != nullptr, "lidar_cast_sweep: nothing to write");
    if (c->table.table == nullptr) {
        set_error("lidar_cast_sweep: no material table (lidar_set_materials)");
        return LIDAR_ESTATE;
    }
    EchoOut echo{0, 0, 0.0f, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (echoes) {
        LIDAR_CHECK_ARG(echoes->n_echoes >= 1 && echoes->n_echoes <= 4, "lidar_cast_sweep: n_echoes in [1, 4]");
        LIDAR_CHECK_ARG(echoes->mode == 0 || echoes->mode == 1, "lidar_cast_sweep: echo mode is 0 or 1");
        LIDAR_CHECK_ARG(isfinite(echoes->separation) && echoes->separation >= 0.0f,
                        "lidar_cast_sweep: separation must be finite, >= 0");
        LIDAR_CHECK_ARG(echoes->count != nullptr, "lidar_cast_sweep: echoes->count is NULL");
        echo = EchoOut{echoes->n_echoes, echoes->mode, echoes->separation, echoes->count, echoes->range,
                       echoes->intensity, echoes->tri, echoes->sub};
    }
    std::vector<SweepDev> fd((size_t)n_frames);
    std::vector<int64_t> prefix((size_t)n_frames);
    const int tr = c->cfg.tile_rays;
    int64_t off = 0, tiles = 0;
    for (int32_t k = 0; k < n_frames; ++k) {
        const int s = frames[k].sensor;
        LIDAR_CHECK_ARG(s >= 0 && s < LIDAR_MAX_SENSORS, "lidar_cast_sweep: sensor slot out of range");
        if (!c->slots[s].set) {
            set_error("lidar_cast_sweep: frame " + std::to_string(k) + " names an empty sensor slot");
            return LIDAR_ESTATE;
        }
        for (int j = 0; j < 12; ++j)
            LIDAR_CHECK_ARG(isfinite(frames[k].pose0[j]) && isfinite(frames[k].pose1[j]),
                            "lidar_cast_sweep: non-finite pose");
        double q0[4], q1[4];
        rotation_quaternion(frames[k].pose0, q0);
        rotation_quaternion(frames[k].pose1, q1);
        const double dq = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2] + q0[3] * q1[3];
        SweepDev& f = fd[(size_t)k];
        for (int i = 0; i < 4; ++i) {
            f.q0[i] = (float)q0[i];
            f.q1[i] = (float)(dq < 0.0 ? -q1[i] : q1[i]);
        }
        for (int r = 0; r < 3; ++r) {
            f.t0[r] = frames[k].pose0[4 * r + 3];
            f.t1[r] = frames[k].pose1[4 * r + 3];
        }
        f.sensor = s;
        f.frame = frames[k].frame;
        f.beam_offset = off;
        prefix[(size_t)k] = tiles;
        off += c->slots[s].n_beams;
        tiles += (c->slots[s].n_beams + tr - 1) / tr;
    }
    DeviceGuard g(c->device);
    // sweep records, then the tile prefix at a 256-byte boundary, in one block
    const size_t prefix_at = ((size_t)n_frames * sizeof(SweepDev) + 255) / 256 * 256;
    if ((size_t)n_frames > c->sweeps_cap) {
        LIDAR_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->sweeps_dev);
        c->sweeps_dev = nullptr;
        c->sweeps_cap = 0;
        if (dev_alloc((void**)&c->sweeps_dev, prefix_at + (size_t)n_frames * sizeof(int64_t)) != cudaSuccess) {
            cudaGetLastError();
            set_error("lidar_cast_sweep: device allocation failed");
            return LIDAR_ENOMEM;
        }
        c->sweeps_cap = n_frames;
    }
    // pageable source: the copy is staged before the call returns
    LIDAR_CUDA(cudaMemcpyAsync(c->sweeps_dev, fd.data(), (size_t)n_frames * sizeof(SweepDev), cudaMemcpyHostToDevice,
                               c->stream));
    int64_t* prefix_dev = (int64_t*)((char*)c->sweeps_dev + prefix_at);
    LIDAR_CUDA(cudaMemcpyAsync(prefix_dev, prefix.data(), (size_t)n_frames * sizeof(int64_t), cudaMemcpyHostToDevice,
                               c->stream));
    // persistent tiles that follow the slots' ray orders and schedules
    LIDAR_CUDA(launch_sweep_tiles(c->stream, scene_dev(scene), c->sensors_dev, c->sweeps_dev, n_frames, prefix_dev,
                                  tiles, c->table, seed, to_beams_out(beams), echo, c->status_dev, c->work_counter,
                                  c->cfg, c->num_sms));
    return LIDAR_OK;
}

lidar_status lidar_raster_gbuffer(lidar_ctx* c, const lidar_scene* scene, const lidar_frame* frame,
                                  const lidar_raster_config* cfg, uint32_t* depth_dev, uint32_t* angle_mat_dev,
                                  uint32_t* inst_dev, uint32_t* tri_dev)
{
    NvtxRange nvtx_("lidar_raster_gbuffer");
    LIDAR_CHECK_ARG(c != nullptr && frame != nullptr, "lidar_raster_gbuffer: NULL argument");
    const int s = frame->sensor;
    LIDAR_CHECK_ARG(s >= 0 && s < LIDAR_MAX_SENSORS, "lidar_raster_gbuffer: sensor slot out of range");
    if (!c->slots[s].set) {
        set_error("lidar_raster_gbuffer: the frame names an empty sensor slot");
        return LIDAR_ESTATE;
    }
    for (int j = 0; j < 12; ++j)
        LIDAR_CHECK_ARG(isfinite(frame->pose[j]), "lidar_raster_gbuffer: non-finite pose");
    DeviceGuard g(c->device);
    RasterCams C;
    lidar_status st = raster_setup(c, scene, cfg, tri_dev != nullptr, C);
    if (st != LIDAR_OK) return st;
    const RasterFrame F = raster_frame(C, *frame, c->slots[s].dev.t_max);
    GBuffer G{};
    LIDAR_CUDA(launch_rasterise(c->stream, scene_dev(scene), C, F, scene->orig_to_leaf, c->scratch, tri_dev != nullptr,
                                &G, c->num_sms));
    const size_t bytes = (size_t)C.K * C.W * C.W * sizeof(uint32_t);
    if (depth_dev) LIDAR_CUDA(cudaMemcpyAsync(depth_dev, G.depth, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (angle_mat_dev)
        LIDAR_CUDA(cudaMemcpyAsync(angle_mat_dev, G.angle_mat, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (inst_dev) LIDAR_CUDA(cudaMemcpyAsync(inst_dev, G.inst, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (tri_dev) LIDAR_CUDA(cudaMemcpyAsync(tri_dev, G.tri, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return LIDAR_OK;
}

}  // extern "C"

struct lidar_batch {
    lidar_ctx* ctx = nullptr;
    FrameDev* frames_dev = nullptr;
    int64_t* prefix_dev = nullptr;
    int32_t n_frames = 0;
    int64_t n_total = 0, n_tiles = 0;
    int tile_rays = 0;
    std::vector<int32_t> slot_beams;  // beams of each slot at creation (-1 = unused)
};

struct lidar_graph {
    lidar_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

lidar_status lidar_batch_create(lidar_ctx* c, const lidar_frame* frames, int32_t n_frames, lidar_batch** out)
{
    LIDAR_CHECK_ARG(c != nullptr && out != nullptr, "lidar_batch_create: NULL argument");
    LIDAR_CHECK_ARG(frames != nullptr && n_frames > 0, "lidar_batch_create: need at least one frame");
    *out = nullptr;
    DeviceGuard g(c->device);
    int64_t n_total = 0, n_tiles = 0;
    lidar_status st = prepare_frames(c, frames, n_frames, &n_total, &n_tiles);
    if (st != LIDAR_OK) return st;
    lidar_batch* b = new lidar_batch();
    b->ctx = c;
    b->n_frames = n_frames;
    b->n_total = n_total;
    b->n_tiles = n_tiles;
    b->tile_rays = c->cfg.tile_rays;
    b->slot_beams.assign(LIDAR_MAX_SENSORS, -1);
    for (int s = 0; s < LIDAR_MAX_SENSORS; ++s)
        if (c->slots[s].set) b->slot_beams[s] = (int32_t)c->slots[s].n_beams;
    if (dev_alloc((void**)&b->frames_dev, n_frames * sizeof(FrameDev)) != cudaSuccess ||
        dev_alloc((void**)&b->prefix_dev, n_frames * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->frames_dev);
        delete b;
        set_error("lidar_batch_create: device allocation failed");
        return LIDAR_ENOMEM;
    }
    // the context's staging copies were made by prepare_frames: copy them over
    cudaMemcpyAsync(b->frames_dev, c->frames_dev, n_frames * sizeof(FrameDev), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(b->prefix_dev, c->tile_prefix_dev, n_frames * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                    c->stream);
    st = ensure_scratch(c, cast_scratch_upper_bound(n_total));
    if (st == LIDAR_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
        set_error("lidar_batch_create: stream synchronisation failed");
        st = LIDAR_ECUDA;
    }
    if (st != LIDAR_OK) {
        cudaFree(b->frames_dev);
        cudaFree(b->prefix_dev);
        delete b;
        return st;
    }
    *out = b;
    return LIDAR_OK;
}

void lidar_batch_free(lidar_batch* b)
{
    if (!b) return;
    DeviceGuard g(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    cudaFree(b->frames_dev);
    cudaFree(b->prefix_dev);
    delete b;
}

lidar_status lidar_batch_set_poses(lidar_ctx* c, lidar_batch* b, const float* poses_dev)
{
    LIDAR_CHECK_ARG(c != nullptr && b != nullptr && poses_dev != nullptr, "lidar_batch_set_poses: NULL argument");
    LIDAR_CHECK_ARG(b->ctx == c, "lidar_batch_set_poses: batch belongs to another context");
    DeviceGuard g(c->device);
    LIDAR_CUDA(launch_set_poses(c->stream, b->frames_dev, b->n_frames, poses_dev));
    return LIDAR_OK;
}

static lidar_status batch_valid(lidar_ctx* c, const lidar_batch* b)
{
    LIDAR_CHECK_ARG(b != nullptr && b->ctx == c, "lidar_cast_batch: batch is NULL or belongs to another context");
    if (c->cfg.tile_rays != b->tile_rays) {
        set_error("lidar_cast_batch: launch tile size changed since the batch was created");
        return LIDAR_ESTATE;
    }
    for (int s = 0; s < LIDAR_MAX_SENSORS; ++s) {
        const int32_t now = c->slots[s].set ? (int32_t)c->slots[s].n_beams : -1;
        if (b->slot_beams[s] >= 0 && now != b->slot_beams[s]) {
            set_error("lidar_cast_batch: a sensor slot changed since the batch was created");
            return LIDAR_ESTATE;
        }
    }
    return LIDAR_OK;
}

lidar_status lidar_cast_batch(lidar_ctx* c, const lidar_scene* scene, const lidar_batch* b, uint64_t seed,
                              const lidar_beams* beams, const lidar_points* points, int64_t* n_points_dev)
{
    NvtxRange nvtx_("lidar_cast_batch");
    lidar_status st = cast_checks(c, scene, beams, points);
    if (st != LIDAR_OK) return st;
    st = batch_valid(c, b);
    if (st != LIDAR_OK) return st;
    DeviceGuard g(c->device);
    return cast_impl(c, scene, b->frames_dev, b->prefix_dev, b->n_frames, b->n_total, b->n_tiles, seed, beams, points,
                     n_points_dev, false);
}

lidar_status lidar_graph_create(lidar_ctx* c, const lidar_scene* scene, lidar_batch* b, const float* poses_dev,
                                uint64_t seed, const lidar_beams* beams, const lidar_points* points,
                                int64_t* n_points_dev, lidar_graph** out)
{
    LIDAR_CHECK_ARG(out != nullptr, "lidar_graph_create: out is NULL");
    *out = nullptr;
    lidar_status st = cast_checks(c, scene, beams, points);
    if (st != LIDAR_OK) return st;
    st = batch_valid(c, b);
    if (st != LIDAR_OK) return st;
    DeviceGuard g(c->device);
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    cudaStream_t cap = nullptr;
    LIDAR_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    c->stream = cap;
    lidar_graph* gr = new lidar_graph();
    gr->ctx = c;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (poses_dev) e = launch_set_poses(cap, b->frames_dev, b->n_frames, poses_dev);
        if (e == cudaSuccess)
            st = cast_impl(c, scene, b->frames_dev, b->prefix_dev, b->n_frames, b->n_total, b->n_tiles, seed, beams,
                           points, n_points_dev, false);
        cudaError_t e2 = cudaStreamEndCapture(cap, &gr->graph);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = saved;
    cudaStreamDestroy(cap);
    if (e == cudaSuccess && st == LIDAR_OK) e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
    if (e != cudaSuccess || st != LIDAR_OK) {
        if (gr->graph) cudaGraphDestroy(gr->graph);
        delete gr;
        if (st != LIDAR_OK) return st;
        set_error(std::string("lidar_graph_create: ") + cudaGetErrorString(e));
        return LIDAR_ECUDA;
    }
    *out = gr;
    return LIDAR_OK;
}

lidar_status lidar_graph_launch(lidar_graph* gr)
{
    NvtxRange nvtx_("lidar_graph_launch");
    LIDAR_CHECK_ARG(gr != nullptr, "lidar_graph_launch: graph is NULL");
    DeviceGuard g(gr->ctx->device);
    LIDAR_CUDA(cudaGraphLaunch(gr->exec, gr->ctx->stream));
    return LIDAR_OK;
}

void lidar_graph_free(lidar_graph* gr)
{
    if (!gr) return;
    DeviceGuard g(gr->ctx->device);
    cudaStreamSynchronize(gr->ctx->stream);
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
}

static lidar_status backward_common(lidar_ctx* c, int64_t n, const lidar_beams* tape, float gain,
                                    const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                    float* loss, float* grad_table, float* grad_gain,
                                    unsigned long long* n_used = nullptr)
{
    LIDAR_CHECK_ARG(c != nullptr && tape != nullptr, "lidar_cast_backward: ctx/tape is NULL");
    LIDAR_CHECK_ARG(n >= 0, "lidar_cast_backward: negative beam count");
    LIDAR_CHECK_ARG(n == 0 || (tape->valid && tape->mat && tape->theta_deg && tape->rf),
                    "lidar_cast_backward: tape needs valid, mat, theta_deg and rf");
    if (c->table.table == nullptr) {
        set_error("lidar_cast_backward: no material table (lidar_set_materials)");
        return LIDAR_ESTATE;
    }
    DeviceGuard g(c->device);
    lidar_status st = ensure_scratch(c, std::max(backward_scratch_bytes(c->table.n_mat),
                                                 onepass_scratch_bytes(c->table.n_mat, c->num_sms)));
    if (st != LIDAR_OK) return st;
    // one pass over the tape (cooperative launch) unless its accumulators do
    // not fit in shared memory or the device cannot launch cooperatively
    cudaError_t e = cudaErrorNotSupported;
    if (c->coop)
        e = launch_cast_backward_onepass(c->stream, n, tape->valid, tape->mat, tape->theta_deg, tape->rf, c->table,
                                         gain, grad_I, target_I, target_valid, loss, grad_table, grad_gain, c->scratch,
                                         c->scratch_bytes, c->adj_arrivals, &c->adj_arrivals_base, c->status_dev,
                                         c->cfg.wait_ns, c->num_sms, n_used);
    if (e == cudaErrorNotSupported)
        e = launch_cast_backward(c->stream, n, tape->valid, tape->mat, tape->theta_deg, tape->rf, c->table, gain,
                                 grad_I, target_I, target_valid, loss, grad_table, grad_gain, c->scratch,
                                 c->scratch_bytes, n_used);
    LIDAR_CUDA(e);
    return LIDAR_OK;
}

lidar_status lidar_cast_backward(lidar_ctx* c, int64_t n, const lidar_beams* tape, float gain, const float* grad_I,
                                 float* grad_table, float* grad_gain)
{
    NvtxRange nvtx_("lidar_cast_backward");
    LIDAR_CHECK_ARG(n == 0 || grad_I != nullptr, "lidar_cast_backward: grad_I is NULL");
    return backward_common(c, n, tape, gain, grad_I, nullptr, nullptr, nullptr, grad_table, grad_gain);
}

lidar_status lidar_cast_backward_mse(lidar_ctx* c, int64_t n, const lidar_beams* tape, float gain,
                                     const float* target_I, const uint8_t* target_valid, float* loss,
                                     float* grad_table, float* grad_gain)
{
    NvtxRange nvtx_("lidar_cast_backward_mse");
    LIDAR_CHECK_ARG(n == 0 || (target_I != nullptr && target_valid != nullptr),
                    "lidar_cast_backward_mse: targets are NULL");
    return backward_common(c, n, tape, gain, nullptr, target_I, target_valid, loss, grad_table, grad_gain);
}

lidar_status lidar_cast_backward_mse_count(lidar_ctx* c, int64_t n, const lidar_beams* tape, float gain,
                                           const float* target_I, const uint8_t* target_valid, float* loss,
                                           float* grad_table, float* grad_gain, uint64_t* n_used)
{
    NvtxRange nvtx_("lidar_cast_backward_mse_count");
    LIDAR_CHECK_ARG(n == 0 || (target_I != nullptr && target_valid != nullptr),
                    "lidar_cast_backward_mse_count: targets are NULL");
    LIDAR_CHECK_ARG(n_used != nullptr, "lidar_cast_backward_mse_count: n_used is NULL");
    static_assert(sizeof(uint64_t) == sizeof(unsigned long long), "64-bit count");
    return backward_common(c, n, tape, gain, nullptr, target_I, target_valid, loss, grad_table, grad_gain,
                           reinterpret_cast<unsigned long long*>(n_used));
}

// Device address of the allocation-free variant's scratch array, looked up once
// per device (with that device current) and cached.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256] = {};

lidar_status lidar_cast_backward_mse_noalloc(void* cuda_stream, int64_t n, const uint8_t* valid, const uint16_t* mat,
                                             const float* theta_deg, const float* rf, const float* table, int32_t M,
                                             float gain, const float* target_I, const uint8_t* target_valid,
                                             float* loss, float* grad_table, float* grad_gain)
{
    NvtxRange nvtx_("lidar_cast_backward_mse_noalloc");
    LIDAR_CHECK_ARG(n >= 0, "lidar_cast_backward_mse_noalloc: negative beam count");
    LIDAR_CHECK_ARG(table != nullptr && M >= 1, "lidar_cast_backward_mse_noalloc: need a reflectance table");
    if (M > LIDAR_NOALLOC_MAX_MATERIALS) {
        set_error("lidar_cast_backward_mse_noalloc: " + std::to_string(M) + " materials exceed the fixed scratch (" +
                  std::to_string(LIDAR_NOALLOC_MAX_MATERIALS) + " materials max); use lidar_cast_backward_mse");
        return LIDAR_EINVAL;
    }
    LIDAR_CHECK_ARG(n == 0 || (valid && mat && theta_deg && rf && target_I && target_valid),
                    "lidar_cast_backward_mse_noalloc: tape or target arrays are NULL");
    int dev = 0;
    LIDAR_CUDA(cudaGetDevice(&dev));
    LIDAR_CHECK_ARG(dev >= 0 && dev < 256, "lidar_cast_backward_mse_noalloc: device ordinal out of range");
    void* scratch = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (g_noalloc_ptr[dev] == nullptr) {
            void* p = nullptr;
            cudaError_t e = noalloc_scratch(&p, &bytes);
            if (e != cudaSuccess || p == nullptr) {
                set_error(std::string("lidar_cast_backward_mse_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
                return LIDAR_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    bytes = LIDAR_NOALLOC_SCRATCH_BYTES;
    TableDev T{table, M};
    LIDAR_CUDA(launch_cast_backward((cudaStream_t)cuda_stream, n, valid, mat, theta_deg, rf, T, gain, nullptr, target_I,
                                    target_valid, loss, grad_table, grad_gain, scratch, bytes));
    return LIDAR_OK;
}

// Instrumented cast: totals h[0..3] (node fetches, triangle tests, distinct
// nodes, distinct triangles); optionally the per-beam cost (dense layout) in
// scratch.  `tail_bytes` of scratch after the cost array are left free for the
// caller (returned through *tail).
static lidar_status counting_cast(lidar_ctx* c, const lidar_scene* scene, const lidar_frame* frames,
                                  int32_t n_frames, uint64_t seed, bool want_cost, size_t tail_bytes,
                                  unsigned long long h[4], uint32_t** cost, void** tail, int64_t* n_total_out)
{
    LIDAR_CHECK_ARG(c != nullptr && scene != nullptr, "counting cast: NULL argument");
    LIDAR_CHECK_ARG(scene->ctx == c, "counting cast: scene belongs to another context");
    if (c->table.table == nullptr) {
        set_error("counting cast: no material table (lidar_set_materials)");
        return LIDAR_ESTATE;
    }
    lidar_status st = traversal_available(c, scene, "counting cast");
    if (st != LIDAR_OK) return st;
    int64_t n_total = 0, n_tiles = 0;
    st = prepare_frames(c, frames, n_frames, &n_total, &n_tiles);
    if (st != LIDAR_OK) return st;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const int64_t node_words = (scene->n_nodes + 31) / 32 + 1, leaf_words = (scene->n_tris + 31) / 32 + 1;
    const size_t head = al(64 + (node_words + leaf_words) * 4);
    const size_t bytes = head + al(n_total) + (want_cost ? al(4 * n_total) : 0) + tail_bytes;
    st = ensure_scratch(c, bytes);
    if (st != LIDAR_OK) return st;
    char* p = (char*)c->scratch;
    unsigned long long* totals = (unsigned long long*)p;
    uint32_t* node_bits = (uint32_t*)(p + 64);
    uint32_t* leaf_bits = node_bits + node_words;
    uint8_t* valid = (uint8_t*)(p + head);
    uint32_t* cost_dev = want_cost ? (uint32_t*)(p + head + al(n_total)) : nullptr;
    if (tail) *tail = p + head + al(n_total) + (want_cost ? al(4 * n_total) : 0);
    if (cost) *cost = cost_dev;
    LIDAR_CUDA(cudaMemsetAsync(p, 0, 64 + (node_words + leaf_words) * 4, c->stream));
    WorkCount wc{totals, node_bits, leaf_bits, cost_dev};
    BeamsOut dense{};
    dense.valid = valid;
    SceneDev S = scene_dev(scene);
    LIDAR_CUDA(launch_cast(c->stream, S, c->sensors_dev, c->frames_dev, n_frames, c->tile_prefix_dev, n_tiles,
                           c->table, seed, dense, c->status_dev, c->work_counter, c->cfg, c->num_sms, n_total,
                           &wc));
    LIDAR_CUDA(launch_popcount(c->stream, node_bits, node_words, totals + 2));
    LIDAR_CUDA(launch_popcount(c->stream, leaf_bits, leaf_words, totals + 3));
    LIDAR_CUDA(cudaMemcpyAsync(h, totals, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    if (n_total_out) *n_total_out = n_total;
    return LIDAR_OK;
}

lidar_status lidar_count_work(lidar_ctx* c, const lidar_scene* scene, const lidar_frame* frames, int32_t n_frames,
                              uint64_t seed, lidar_work_counts* out, uint32_t* beam_cost_dev)
{
    NvtxRange nvtx_("lidar_count_work");
    LIDAR_CHECK_ARG(c != nullptr && scene != nullptr && out != nullptr, "lidar_count_work: NULL argument");
    DeviceGuard g(c->device);
    unsigned long long h[4];
    uint32_t* cost = nullptr;
    int64_t n_total = 0;
    lidar_status st = counting_cast(c, scene, frames, n_frames, seed, beam_cost_dev != nullptr, 0, h, &cost, nullptr,
                                    &n_total);
    if (st != LIDAR_OK) return st;
    if (beam_cost_dev) {
        LIDAR_CUDA(cudaMemcpyAsync(beam_cost_dev, cost, n_total * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                   c->stream));
        LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    }
    uint64_t rays = 0;
    for (int32_t k = 0; k < n_frames; ++k) {
        const SensorSlot& sl = c->slots[frames[k].sensor];
        rays += (uint64_t)sl.n_beams * (uint64_t)sl.dev.n_sub;
    }
    out->rays = rays;
    out->node_bytes = c->cfg.traversal == 3 ? 256 : (c->cfg.traversal == 2 ? 128 : 64);
    out->node_visits = h[0];
    out->tri_tests = h[1];
    out->unique_nodes = h[2];
    out->unique_tris = h[3];
    return LIDAR_OK;
}

lidar_status lidar_schedule_by_cost(lidar_ctx* c, const lidar_scene* scene, const lidar_frame* frame, uint64_t seed,
                                    int32_t mode)
{
    NvtxRange nvtx_("lidar_schedule_by_cost");
    LIDAR_CHECK_ARG(mode == 0 || mode == 1, "lidar_schedule_by_cost: mode is 0 or 1");
    LIDAR_CHECK_ARG(c != nullptr && scene != nullptr && frame != nullptr, "lidar_schedule_by_cost: NULL argument");
    const int slot = frame->sensor;
    LIDAR_CHECK_ARG(slot >= 0 && slot < LIDAR_MAX_SENSORS, "lidar_schedule_by_cost: slot out of range");
    if (!c->slots[slot].set) {
        set_error("lidar_schedule_by_cost: no sensor in this slot");
        return LIDAR_ESTATE;
    }
    DeviceGuard g(c->device);
    SensorSlot& sl = c->slots[slot];
    const int64_t n = sl.n_beams;
    unsigned long long h[4];
    uint32_t* cost = nullptr;
    void* tail = nullptr;
    const size_t need = std::max(cost_schedule_scratch_bytes(n), bucket_schedule_scratch_bytes(n));
    lidar_status st = counting_cast(c, scene, frame, 1, seed, true, need, h, &cost, &tail, nullptr);
    if (st != LIDAR_OK) return st;
    const size_t tail_bytes = c->scratch_bytes - (size_t)((char*)tail - (char*)c->scratch);
    if (mode == 0)
        LIDAR_CUDA(launch_cost_schedule(c->stream, cost, sl.base_order_dev, (int)n, sl.order_dev, tail, tail_bytes));
    else
        LIDAR_CUDA(launch_bucket_schedule(c->stream, cost, sl.base_order_dev, (int)n, sl.order_dev, tail,
                                          tail_bytes));
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    return LIDAR_OK;
}

lidar_status lidar_reset_schedule(lidar_ctx* c, int32_t slot)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_reset_schedule: ctx is NULL");
    LIDAR_CHECK_ARG(slot >= 0 && slot < LIDAR_MAX_SENSORS, "lidar_reset_schedule: slot out of range");
    if (!c->slots[slot].set) {
        set_error("lidar_reset_schedule: no sensor in this slot");
        return LIDAR_ESTATE;
    }
    DeviceGuard g(c->device);
    SensorSlot& sl = c->slots[slot];
    LIDAR_CUDA(cudaMemcpyAsync(sl.order_dev, sl.base_order_dev, sl.n_beams * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, c->stream));
    LIDAR_CUDA(cudaStreamSynchronize(c->stream));
    return LIDAR_OK;
}

lidar_status lidar_set_build_options(lidar_ctx* c, const lidar_build_options* o)
{
    LIDAR_CHECK_ARG(c != nullptr && o != nullptr, "lidar_set_build_options: NULL argument");
    LIDAR_CHECK_ARG(o->method == 0 || o->method == 1, "lidar_set_build_options: method is 0 or 1");
    LIDAR_CHECK_ARG(o->ploc_radius >= 1 && o->ploc_radius <= 64, "lidar_set_build_options: ploc_radius in [1, 64]");
    LIDAR_CHECK_ARG(o->collapse == 0 || o->collapse == 1, "lidar_set_build_options: collapse is 0 or 1");
    LIDAR_CHECK_ARG(o->tri_cost > 0.0f && o->tri_cost <= 100.0f, "lidar_set_build_options: tri_cost in (0, 100]");
    LIDAR_CHECK_ARG(o->treelet_rounds >= 0 && o->treelet_rounds <= 8,
                    "lidar_set_build_options: treelet_rounds in [0, 8]");
    for (int k = 0; k < 3; ++k)
        LIDAR_CHECK_ARG(o->area_weight[k] > 0.0f && o->area_weight[k] <= 100.0f,
                        "lidar_set_build_options: area_weight in (0, 100]");
    c->build_method = o->method;
    c->ploc_radius = o->ploc_radius;
    c->collapse = o->collapse;
    c->tri_cost = o->tri_cost;
    c->treelet_rounds = o->treelet_rounds;
    c->area_w = AreaW{o->area_weight[0], o->area_weight[1], o->area_weight[2]};
    return LIDAR_OK;
}

lidar_status lidar_get_build_options(lidar_ctx* c, lidar_build_options* o)
{
    LIDAR_CHECK_ARG(c != nullptr && o != nullptr, "lidar_get_build_options: NULL argument");
    o->method = c->build_method;
    o->ploc_radius = c->ploc_radius;
    o->collapse = c->collapse;
    o->tri_cost = c->tri_cost;
    o->treelet_rounds = c->treelet_rounds;
    o->area_weight[0] = c->area_w.x;
    o->area_weight[1] = c->area_w.y;
    o->area_weight[2] = c->area_w.z;
    return LIDAR_OK;
}

lidar_status lidar_get_launch_config(lidar_ctx* c, lidar_launch_config* out)
{
    LIDAR_CHECK_ARG(c != nullptr && out != nullptr, "lidar_get_launch_config: NULL argument");
    out->block_threads = c->cfg.block_threads;
    out->blocks_per_sm = c->cfg.blocks_per_sm;
    out->tile_rays = c->cfg.tile_rays;
    out->ray_order = c->cfg.ray_order;
    out->traversal = c->cfg.traversal;
    out->fused_scatter = c->cfg.fused_scatter;
    return LIDAR_OK;
}

lidar_status lidar_set_launch_config(lidar_ctx* c, const lidar_launch_config* cfg)
{
    LIDAR_CHECK_ARG(c != nullptr && cfg != nullptr, "lidar_set_launch_config: NULL argument");
    LIDAR_CHECK_ARG(cfg->block_threads >= 32 && cfg->block_threads <= 256 && cfg->block_threads % 32 == 0,
                    "lidar_set_launch_config: block_threads must be a multiple of 32 in [32, 256]");
    LIDAR_CHECK_ARG(cfg->blocks_per_sm >= 1 && cfg->blocks_per_sm <= 64, "lidar_set_launch_config: blocks_per_sm in [1, 64]");
    LIDAR_CHECK_ARG(cfg->tile_rays >= 32 && cfg->tile_rays <= (1 << 20) && cfg->tile_rays % 32 == 0,
                    "lidar_set_launch_config: tile_rays must be a multiple of 32 in [32, 2^20]");
    LIDAR_CHECK_ARG(cfg->ray_order == 0 || cfg->ray_order == 1, "lidar_set_launch_config: ray_order is 0 or 1");
    LIDAR_CHECK_ARG(cfg->traversal >= 0 && cfg->traversal <= 3, "lidar_set_launch_config: traversal is 0, 1, 2 or 3");
    LIDAR_CHECK_ARG(cfg->fused_scatter == 0 || cfg->fused_scatter == 1,
                    "lidar_set_launch_config: fused_scatter is 0 or 1");
    DeviceGuard g(c->device);
    c->cfg.block_threads = cfg->block_threads;
    c->cfg.blocks_per_sm = cfg->blocks_per_sm;
    c->cfg.tile_rays = cfg->tile_rays;
    c->cfg.ray_order = cfg->ray_order;
    c->cfg.traversal = cfg->traversal;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    c->cfg.fused_scatter = (cfg->fused_scatter && coop) ? 1 : 0;
    for (int s = 0; s < LIDAR_MAX_SENSORS; ++s)
        if (c->slots[s].set) {
            lidar_status st = upload_sensor_slot(c, s);
            if (st != LIDAR_OK) return st;
        }
    return LIDAR_OK;
}

lidar_status lidar_measure_fp32_rate(lidar_ctx* c, int64_t fma_per_thread, double* flops_per_s, double* kernel_ms,
                                     int32_t* packed)
{
    LIDAR_CHECK_ARG(c != nullptr && flops_per_s != nullptr && kernel_ms != nullptr && packed != nullptr,
                    "lidar_measure_fp32_rate: NULL argument");
    LIDAR_CHECK_ARG(fma_per_thread >= 64 && fma_per_thread <= ((int64_t)1 << 40),
                    "lidar_measure_fp32_rate: fma_per_thread in [64, 2^40]");
    DeviceGuard g(c->device);
    lidar_status st = ensure_scratch(c, (size_t)c->num_sms * 4 * sizeof(float));
    if (st != LIDAR_OK) return st;
    int form = 0;
    LIDAR_CUDA(measure_fp32_rate(c->stream, c->num_sms, fma_per_thread, c->scratch, flops_per_s, kernel_ms, &form));
    *packed = form;
    return LIDAR_OK;
}

lidar_status lidar_set_cast_overlap(lidar_ctx* c, int32_t enable)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_set_cast_overlap: NULL context");
    LIDAR_CHECK_ARG(enable == 0 || enable == 1, "lidar_set_cast_overlap: enable is 0 or 1");
    c->overlap = enable;
    return LIDAR_OK;
}

lidar_status lidar_get_cast_overlap(lidar_ctx* c, int32_t* enable)
{
    LIDAR_CHECK_ARG(c != nullptr && enable != nullptr, "lidar_get_cast_overlap: NULL argument");
    *enable = c->overlap;
    return LIDAR_OK;
}

lidar_status lidar_set_wait_limit(lidar_ctx* c, uint64_t ns)
{
    LIDAR_CHECK_ARG(c != nullptr, "lidar_set_wait_limit: NULL context");
    c->cfg.wait_ns = ns;
    return LIDAR_OK;
}

lidar_status lidar_get_wait_limit(lidar_ctx* c, uint64_t* ns)
{
    LIDAR_CHECK_ARG(c != nullptr && ns != nullptr, "lidar_get_wait_limit: NULL argument");
    *ns = c->cfg.wait_ns;
    return LIDAR_OK;
}

}  // extern "C"
