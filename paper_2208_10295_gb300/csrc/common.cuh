// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/lidar.h"

namespace lidar {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);

#define LIDAR_CHECK_ARG(cond, msg)              \
    do {                                        \
        if (!(cond)) {                          \
            ::lidar::set_error(msg);            \
            return LIDAR_EINVAL;                \
        }                                       \
    } while (0)

#define LIDAR_CUDA(call)                                                                      \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess) {                                                              \
            ::lidar::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));           \
            return _e == cudaErrorMemoryAllocation ? LIDAR_ENOMEM : LIDAR_ECUDA;              \
        }                                                                                     \
    } while (0)

// device status word codes (first error wins)
enum : int { ST_OK = 0, ST_CAPACITY = 1, ST_STACK = 2, ST_TIMEOUT = 3, ST_INDEX = 4, ST_BOUNDS = 5 };

__device__ __forceinline__ void raise_status(int* status, int code)
{
    atomicCAS(status, ST_OK, code);
}

// ------------------------------------------------------------------ scene layout
//
// BVH node (64 bytes, four 16-byte loads): both children's boxes live in the
// parent so one fetch decides both children.
//   n0 = (L.lo.x, L.hi.x, L.lo.y, L.hi.y)
//   n1 = (R.lo.x, R.hi.x, R.lo.y, R.hi.y)
//   n2 = (L.lo.z, L.hi.z, R.lo.z, R.hi.z)
//   n3 = (left, right, -, -) as int bits; child >= 0: internal node, child < 0:
//        leaf ~child = position in the leaf-ordered triangle array.
// Triangle (48 bytes, three 16-byte loads), leaf order:
//   v0.xyz, w = original triangle index (bits)
//   v1.xyz, w = material (bits)
//   v2.xyz, w = instance (bits)
constexpr int kTraversalStack = 96;

struct SceneDev {
    const float4* nodes;     // [n_nodes * 4] binary hierarchy
    const float4* tris;      // [n_tris * 3]
    int64_t n_tris;
    int64_t n_nodes;
    const float4* nodes4;    // [n_nodes4 * 8] 4-wide hierarchy (same leaves)
    int64_t n_nodes4;
    const float4* nodes8;    // [n_nodes8 * 16] 8-wide hierarchy (same leaves), NULL if not built
    int64_t n_nodes8;
};

// ------------------------------------------------------------------ sensors

struct SensorDev {
    const float* dirs;        // [n_beams][3], sensor frame
    const float* sweep;       // [n_beams] firing fraction of each beam in a sweep (azimuth / 2 pi in [0, 1))
    const uint32_t* order;    // ray order permutation [n_beams] (beam processed at position j)
    int32_t n_beams;
    int32_t n_sub;
    float r_min, r_max, d_max, RL_max, sigma, gain, range_exp, r_ref;
    float sigma_k;            // range-scaled noise: std = sigma + sigma_k t
    float t_max;              // search range end: (min(r_max, d_max) + 9 sigma) / (1 - 9 sigma_k)
    float alpha[LIDAR_MAX_SUBRAYS], beta[LIDAR_MAX_SUBRAYS];
};

struct FrameDev {
    int32_t sensor;
    int32_t frame;
    int64_t beam_offset;      // first dense index of this frame
    float pose[12];
};

// A few frames travel inside the kernel's launch parameters instead of a
// device table (no copy ahead of the launch); n == 0: use the device table.
constexpr int kInlineFrames = 4;
struct InlineFrames {
    FrameDev f[kInlineFrames];
    int64_t prefix[kInlineFrames];  // first tile of each frame
    int n;
};

// The counters of a direct cast (tile counts, finished-block word, work
// counter) in a region the caller keeps all zero between casts: the launch
// needs no memset when `clean`, and clears `zero_next` (the region of the cast
// after it, zero_words words) at its start.  Direct casts rotate through three
// regions, so that with overlapped casts the region being cleared was last
// used by a cast that has completed.
struct CounterRegion {
    unsigned* base;
    bool clean;
    unsigned* zero_next;
    int64_t zero_words;
    bool overlap;   // launch with programmatic dependent launch (consecutive direct casts overlap)
    cudaError_t* overlap_refused;  // nullable: the launch's answer when it refused the overlapped launch
};
// bytes of a CounterRegion a cast of n_total dense beams uses
size_t cast_counter_bytes(int64_t n_total, bool compact);

struct TableDev {
    const float* table;       // [n_mat][91]
    int32_t n_mat;
};

struct BeamsOut {
    uint8_t* valid;
    uint32_t* tri;
    float* t;
    float* range;
    float* intensity;
    float* normal;
    uint16_t* mat;
    uint32_t* inst;
    uint8_t* sub;
    float* theta_deg;
    float* rf;
};

struct LaunchCfg {
    int block_threads;
    int blocks_per_sm;
    int tile_rays;
    int ray_order;
    int traversal;
    int fused_scatter;   // compaction scatter inside the cast (cooperative launch)
    uint64_t wait_ns = 2000000000ull;  // limit of every bounded device-side wait
};

// ------------------------------------------------------------------ kernel launchers

// Weights of a box's faces in the area measure the builders compare: half the
// weighted surface of a box of extents (dx, dy, dz) is
//   z dx dy + x dy dz + y dz dx
// (x weights the faces normal to x, ...); 1, 1, 1 is half the surface area.
struct AreaW {
    float x, y, z;
};

// build.cu
struct BuildScratch;
cudaError_t build_lbvh(cudaStream_t s, const float* verts, int64_t n_verts, const uint32_t* tris,
                       const uint16_t* mat, const uint32_t* inst, int64_t n_tris, float4* nodes_out,
                       float4* tris_out, uint32_t* leaf_tri_out, int* status, int* max_depth_dev,
                       void* scratch, size_t scratch_bytes, int method = 0, int ploc_radius = 16,
                       AreaW area_w = AreaW{1.0f, 1.0f, 1.0f});
// scratch of the clustering build (method 1), on top of nothing: it reuses build_lbvh's scratch
size_t ploc_scratch_bytes(int64_t n_tris);
size_t build_scratch_bytes(int64_t n_tris);
// W-wide hierarchy (width 4 or 8) from the binary one (breadth-first,
// deterministic); synchronises once per level.  `nodes` may be NULL to count
// only.  *n_wide = wide nodes, *levels = height of the wide tree, *stack_need =
// deepest traversal stack the tree can require.
// sah_dp: children chosen by the SAH dynamic program (triangle test cost
// tri_cost relative to a wide-node visit) instead of opening the largest child
cudaError_t collapse_bvh(cudaStream_t s, int width, const float4* binary_nodes, int64_t n_binary, float4* nodes,
                         int64_t* n_wide, int* levels, int* stack_need, void* scratch, size_t scratch_bytes,
                         int sah_dp = 0, float tri_cost = 1.0f, AreaW area_w = AreaW{1.0f, 1.0f, 1.0f});
size_t collapse_scratch_bytes(int64_t n_binary);
// treelet restructuring of the binary hierarchy (rounds > 0, n_tris >= 3);
// recomputes the root height; *changed_host (valid after a stream
// synchronisation) receives the number of treelets rewritten; a broken input
// tree records ST_BOUNDS in *status
size_t treelet_scratch_bytes(int64_t n_tris);
cudaError_t restructure_treelets(cudaStream_t s, const float4* tris, int64_t n, float4* nodes, int* max_height_dev,
                                 int rounds, float tri_cost, void* scratch, size_t scratch_bytes,
                                 unsigned long long* changed_host, int* status,
                                 AreaW area_w = AreaW{1.0f, 1.0f, 1.0f});

// sort.cu: stable LSD radix sort of (key, value) pairs, keys of `key_bits` bits
size_t radix_sort_scratch_bytes(int64_t n);
cudaError_t radix_sort_pairs_u64(cudaStream_t s, uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                 void* scratch, size_t scratch_bytes);
cudaError_t radix_sort_pairs_u32(cudaStream_t s, uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                 void* scratch, size_t scratch_bytes);

// cast.cu
// Instrumentation of the traversal (work counted per launch, not timed).
struct WorkCount {
    unsigned long long* totals;   // [0] node visits, [1] triangle tests
    uint32_t* node_bits;          // one bit per internal node touched
    uint32_t* leaf_bits;          // one bit per triangle tested
    uint32_t* beam_cost;          // optional, dense per beam: node fetches + triangle tests
};
cudaError_t launch_cast(cudaStream_t s, const SceneDev& scene, const SensorDev* sensors_dev,
                        const FrameDev* frames_dev, int n_frames, const int64_t* tile_prefix_dev,
                        int64_t n_tiles, TableDev table, uint64_t seed, BeamsOut out, int* status,
                        unsigned long long* work_counter, const LaunchCfg& cfg, int num_sms,
                        int64_t n_beams_total, const WorkCount* count = nullptr, void* compact_scratch = nullptr,
                        int64_t* n_points_dev = nullptr, const lidar_points* points = nullptr,
                        bool* scattered = nullptr, const InlineFrames* inline_frames = nullptr,
                        const CounterRegion* region = nullptr);
// ordered compaction fused with the cast: the cast counts kept returns per
// 1024-beam tile and scans them (compact_scratch of fused_compact_scratch_bytes);
// with `points` and cfg.fused_scatter it also writes the points after a
// grid-wide wait (cooperative launch, *scattered = true), otherwise
// launch_scatter writes them
size_t fused_compact_scratch_bytes(int64_t n_beams_total);
cudaError_t launch_scatter(cudaStream_t s, const SensorDev* sensors_dev, const FrameDev* frames_dev, int n_frames,
                           int64_t n_beams_total, BeamsOut dense, const lidar_points& pts, void* compact_scratch,
                           int* status, const InlineFrames* inline_frames = nullptr, int num_sms = 0,
                           bool pdl = false);
cudaError_t launch_popcount(cudaStream_t s, const uint32_t* bits, int64_t n_words, unsigned long long* total);
// frames[i].pose = poses[12 i .. 12 i + 11]
cudaError_t launch_set_poses(cudaStream_t s, FrameDev* frames, int n_frames, const float* poses);
cudaError_t launch_ray_order(cudaStream_t s, const float* dirs, int n_beams, uint32_t* order,
                             void* scratch, size_t scratch_bytes);
size_t ray_order_scratch_bytes(int64_t n_beams);
// Reorders 32-ray groups of `base_order` by their largest measured beam cost,
// most expensive first (cost indexed by beam).
cudaError_t launch_cost_schedule(cudaStream_t s, const uint32_t* cost, const uint32_t* base_order, int n_beams,
                                 uint32_t* new_order, void* scratch, size_t scratch_bytes);
size_t cost_schedule_scratch_bytes(int64_t n_beams);
// Orders single beams by cost bucket (4 per octave, most expensive first),
// keeping the base order within a bucket, so each warp gets beams of similar cost.
cudaError_t launch_bucket_schedule(cudaStream_t s, const uint32_t* cost, const uint32_t* base_order, int n_beams,
                                   uint32_t* new_order, void* scratch, size_t scratch_bytes);
size_t bucket_schedule_scratch_bytes(int64_t n_beams);

// probe.cu: FP32 fused multiply-add rate over every SM (sink: 4 bytes per SM x 4)
cudaError_t measure_fp32_rate(cudaStream_t s, int num_sms, int64_t fma_per_thread, void* sink_dev,
                              double* flops_per_s, double* ms, int* form);

// adjoint.cu
cudaError_t launch_build_tables(cudaStream_t s, const float* params, int M, float* table);
cudaError_t launch_build_tables_backward(cudaStream_t s, const float* params, const float* grad_table, int M,
                                         float* grad_params);
cudaError_t launch_cast_backward(cudaStream_t s, int64_t n, const uint8_t* valid, const uint16_t* mat,
                                 const float* theta_deg, const float* rf, TableDev table, float gain,
                                 const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                 float* loss, float* grad_table, float* grad_gain, void* scratch,
                                 size_t scratch_bytes, unsigned long long* n_used = nullptr);
size_t backward_scratch_bytes(int M);
// One-pass variant (one cooperative launch, the tape read once); returns
// cudaErrorNotSupported when the table's accumulators do not fit in shared
// memory beside the copy stages (then launch_cast_backward applies).
// arrivals: the grid-wait counter, *arrivals_base its value before this
// launch (advanced by the launcher).  n_used (device, may be NULL) receives
// the number of beams the mean runs over.
size_t onepass_scratch_bytes(int M, int num_sms);
cudaError_t launch_cast_backward_onepass(cudaStream_t s, int64_t n, const uint8_t* valid, const uint16_t* mat,
                                         const float* theta_deg, const float* rf, TableDev table, float gain,
                                         const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                         float* loss, float* grad_table, float* grad_gain, void* scratch,
                                         size_t scratch_bytes, unsigned long long* arrivals,
                                         unsigned long long* arrivals_base, int* status, uint64_t wait_ns,
                                         int num_sms, unsigned long long* n_used = nullptr);
// address (on the current device) and size of the allocation-free variant's scratch array
cudaError_t noalloc_scratch(void** ptr, size_t* bytes);

// --------------------------------------------- rolling shutter, multi-echo

// One sweep: unit quaternions (w, x, y, z) and translations of the poses at
// its start and end (same hemisphere), the frame's ids and dense offset
struct SweepDev {
    float q0[4], q1[4], t0[3], t1[3];
    int32_t sensor, frame;
    int64_t beam_offset;
};

struct EchoOut {
    int n_echoes;     // 1..4 (0: no echo output)
    int mode;         // 0: strongest, 1: first and last
    float separation;
    uint8_t* count;
    float* range;     // [n][n_echoes]
    float* intensity;
    uint32_t* tri;
    uint8_t* sub;
};

// persistent sweep cast (dense records, no echoes), tiles as in launch_cast
// echo.n_echoes == 0: dense records only
cudaError_t launch_sweep_tiles(cudaStream_t s, const SceneDev& S, const SensorDev* sensors_dev,
                               const SweepDev* frames_dev, int n_frames, const int64_t* tile_prefix_dev,
                               int64_t n_tiles, TableDev T, uint64_t seed, BeamsOut out, EchoOut echo, int* status,
                               unsigned long long* work_counter, const LaunchCfg& cfg, int num_sms);

// ------------------------------------------------------------ raster path

constexpr int kMaxCameras = 64;

// K pin-hole cameras of W x W pixels around the sensor's vertical axis
// (Eq. 1-2): focal length f = W / (2 tan(pi / K)), principal point c = W / 2,
// camera k looking along sensor azimuth -pi + (k + 1/2) 2 pi / K.
struct RasterCams {
    int W, K;
    float f, c;
    float ck[kMaxCameras], sk[kMaxCameras];   // cos, sin of each camera's azimuth
};

// One frame: pose, search range, and each camera's L, U, F axes in the world
struct RasterFrame {
    float pose[12];
    float t_max;
    float axes[9 * kMaxCameras];
};

// G-buffer of K images (SoA, [K][W][W]): depth code (24 bits, 2^24 - 1 = no
// hit), angle code (24 bits) | material stencil << 24, instance colour
// (24 bits), and (optional) the triangle's original index
struct GBuffer {
    uint32_t* depth;
    uint32_t* angle_mat;
    uint32_t* inst;
    uint32_t* tri;
};

size_t raster_big_capacity(int n_cameras, int64_t n_tris);
size_t raster_scratch_bytes(int width, int n_cameras, int64_t n_tris, bool with_tri);
cudaError_t launch_invert_leaf_order(cudaStream_t s, const uint32_t* leaf_tri, int64_t n, uint32_t* orig_to_leaf);
// rasterises one frame's K images into scratch (raster_scratch_bytes); *G
// receives the G-buffer's location inside it (with_tri: also the triangles)
cudaError_t launch_rasterise(cudaStream_t s, const SceneDev& S, const RasterCams& C, const RasterFrame& F,
                             const uint32_t* orig_to_leaf, void* scratch, bool with_tri, GBuffer* G, int num_sms);
cudaError_t launch_resample(cudaStream_t s, const RasterCams& C, const RasterFrame& F, const SensorDev* sensors_dev,
                            int sensor, int n_beams, int frame_id, int64_t beam_offset, TableDev T, uint64_t seed,
                            const GBuffer& G, BeamsOut out);

}  // namespace lidar
