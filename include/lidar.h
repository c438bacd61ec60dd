/*
 * lidar.h — C ABI of the GB300 per-beam LiDAR return-generation library.
 *
 * The operation is the per-beam model of "Physical LiDAR Simulation in
 * Real-Time Engine" (Jansen, Huebel, Steckel, 2022), Sec. II:
 *   - beam pattern: spherical beam coordinates (azimuth theta_i, elevation
 *     phi_j) from the sensor's horizontal/vertical FOV (Sec. II-A);
 *   - range: distance to the first surface along the beam (Sec. II-A; found
 *     here by ray casting a triangle BVH instead of sampling a depth pass),
 *     with additive Gaussian range noise scaled by a noise factor (Sec. II-A);
 *   - labels: per-point instance ID (Sec. II-B) and material ID (Sec. II-C);
 *   - reflectance: Lambertian R(theta) = R(0) cos(theta) (Eq. 4), generalised
 *     to a per-material 91-entry table over incidence angle 0..90 degrees that
 *     is interpolated linearly (Sec. III); theta is the angle between the beam
 *     and the surface normal (Sec. II-C);
 *   - capability model: R_L(d) = R_L,max / d_max * d (Eq. 5); a point is kept
 *     iff R_L(d) <= R and d <= d_max, d including the noise (Sec. II-D).
 *
 * Conventions
 *   - Every pointer named *_dev is a device pointer on the context's device;
 *     every other pointer is host memory.  All device arrays passed in are
 *     owned by the caller and must stay valid until the work that uses them has
 *     completed on the context stream.  The library owns only what it returns
 *     through an opaque handle (context, scene) and its internal scratch.
 *   - Calls are asynchronous on the context's CUDA stream unless stated.
 *     Argument errors are detected on the host and returned immediately as
 *     LIDAR_EINVAL with a message in lidar_last_error().  Errors found by a
 *     kernel (capacity, traversal stack, bounded waits) are recorded in a
 *     device status word and returned by lidar_sync_status().
 *   - Floating point: all per-beam arithmetic is FP32.
 */
#ifndef LIDAR_H
#define LIDAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lidar_ctx lidar_ctx;
typedef struct lidar_scene lidar_scene;

typedef enum {
    LIDAR_OK = 0,
    LIDAR_EINVAL = -1,    /* bad argument (host-side check) */
    LIDAR_ENOMEM = -2,    /* device or host allocation failed */
    LIDAR_ECUDA = -3,     /* a CUDA runtime call failed */
    LIDAR_ESTATE = -4,    /* call not valid in the current state (e.g. no sensor in a slot) */
    LIDAR_ESTACK = -5,    /* BVH deeper than the traversal stack */
    LIDAR_ETIMEOUT = -6,  /* a bounded device-side wait gave up */
    LIDAR_ECAPACITY = -7  /* point output capacity exceeded; count holds the needed size */
} lidar_status;

#define LIDAR_NO_HIT 0xFFFFFFFFu
#define LIDAR_TABLE_SIZE 91      /* reflectance entries per material: 0..90 degrees, 1-degree grid */
#define LIDAR_MAX_SENSORS 16
#define LIDAR_MAX_SUBRAYS 8

/* ------------------------------------------------------------------ context */

/* Creates a context on `device` that enqueues all work on `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  The caller keeps
 * ownership of the stream.  *out receives the handle; free with lidar_destroy. */
lidar_status lidar_create(int device, void* cuda_stream, lidar_ctx** out);

/* Releases the context, its sensors, its scratch and every scene still alive
 * that it created.  Synchronises the context stream first. */
void lidar_destroy(lidar_ctx* ctx);

/* Thread-local, NUL-terminated message describing the last failed call on
 * this thread ("" if none).  Valid until the next call on this thread. */
const char* lidar_last_error(void);

/* Synchronises the context stream, then returns and clears the device status
 * word (LIDAR_OK, LIDAR_ECAPACITY, LIDAR_ESTACK or LIDAR_ETIMEOUT). */
lidar_status lidar_sync_status(lidar_ctx* ctx);

/* ------------------------------------------------------------------- scene */

/* Builds a linear BVH (Karras 2012: 63-bit Morton codes of triangle centroids,
 * radix sort, hierarchy from key prefixes, bottom-up exact FP32 box refit)
 * over a triangle mesh, collapses it into a 4-wide hierarchy over the same
 * leaves (each 4-wide node opens its largest-area children), and copies the
 * triangles, in leaf order, into a library-owned layout.
 *   verts_dev        float32 [n_verts][3], metres, world frame
 *   tris_dev         uint32  [n_tris][3], vertex indices (< n_verts)
 *   tri_material_dev uint16  [n_tris], material ID (row of the reflectance table;
 *                    IDs >= the table's row count use the last row)
 *   tri_instance_dev uint32  [n_tris], instance label reported per point
 * n_tris may be 0 (every beam misses).  The input arrays are only read during
 * the call.  This call synchronises the stream to report build errors
 * (LIDAR_EINVAL for an out-of-range vertex index, LIDAR_ESTACK if the tree is
 * deeper than the traversal stack). */
lidar_status lidar_scene_build(lidar_ctx* ctx, const float* verts_dev, int64_t n_verts,
                               const uint32_t* tris_dev, int64_t n_tris,
                               const uint16_t* tri_material_dev, const uint32_t* tri_instance_dev,
                               lidar_scene** out);

void lidar_scene_free(lidar_scene* scene);

typedef struct {
    int64_t n_tris;
    int64_t n_nodes;       /* internal nodes (n_tris - 1, or 1 for a single triangle) */
    int32_t max_depth;     /* longest root-to-leaf path, in internal nodes */
    int64_t device_bytes;  /* bytes held by the scene on the device */
    double build_ms;       /* device time of the last build, CUDA events */
    int64_t n_nodes4;      /* nodes of the 4-wide hierarchy collapsed from the binary one */
    int32_t levels4;       /* its height */
    int64_t n_nodes8;      /* nodes of the 8-wide hierarchy (same collapse), 0 when not kept because
                              its traversal could need a deeper stack than the kernel's 96 entries */
    int32_t levels8;       /* its height */
    int64_t treelets;      /* treelets the restructuring rewrote (lidar_build_options.treelet_rounds) */
} lidar_scene_info;

lidar_status lidar_get_scene_info(const lidar_scene* scene, lidar_scene_info* out);

/* How lidar_scene_build makes the binary hierarchy that is then collapsed
 * into the 4-wide tree the cast walks (any valid hierarchy gives the same
 * closest hits; they differ in how many nodes a ray visits):
 *   method 0: the Karras LBVH (split at the highest differing Morton bit);
 *   method 1: PLOC, parallel locally-ordered clustering (Meister and Bittner,
 *             IEEE TVCG 2018) over the same Morton-ordered triangles: each
 *             cluster's nearest neighbour by union-box surface area within
 *             ploc_radius positions, mutual pairs merged, repeated; one host
 *             synchronisation per round.
 * Applies to scenes built afterwards. */
typedef struct {
    int32_t method;        /* 0 LBVH, 1 PLOC (default: about a third fewer node fetches per ray) */
    int32_t ploc_radius;   /* 1..64, default 16 */
    int32_t collapse;      /* children of the wide nodes: 0 (default) each node opens its largest-area
                              child until it is full; 1 the surface-area-heuristic optimum over the
                              binary tree (a bottom-up dynamic program, Ylitie, Karras and Laine 2017) */
    float tri_cost;        /* a triangle test's cost relative to a node visit, (0, 100], default 1: the
                              collapse-1 program's and the treelet restructuring's */
    int32_t treelet_rounds;  /* 0..8, default 0: rounds of treelet restructuring of the binary tree before
                                the collapse (Karras and Aila, HPG 2013): bottom-up, each node's treelet
                                of up to 7 leaves (opened largest area first) is rewritten in the
                                shape of least surface-area cost, found by a dynamic program over the
                                subsets of its leaves */
    float area_weight[3];  /* (0, 100] each, default 1, 1, 1: weights of a box's faces normal to x, y and z
                              in the area that PLOC's nearest-neighbour distance, the collapse's
                              largest-area rule and both surface-area programs compare; half the
                              weighted surface of a box is z dx dy + x dy dz + y dz dx.  1, 1, 1 is
                              the surface area (rays of every direction alike); weights proportional
                              to the sensors' mean |direction| components (mostly level rays: a
                              smaller z) fit a LiDAR's beam pattern */
} lidar_build_options;

lidar_status lidar_set_build_options(lidar_ctx* ctx, const lidar_build_options* options);
lidar_status lidar_get_build_options(lidar_ctx* ctx, lidar_build_options* options);

/* Exports the built hierarchy for validation (host buffers, may be NULL):
 * nodes [n_nodes][16] float32 bit patterns in the device layout, and the
 * leaf-order -> original triangle index map [n_tris].  Synchronises. */
lidar_status lidar_scene_export(const lidar_scene* scene, float* nodes_host, uint32_t* leaf_tri_host);

/* Exports a wide hierarchy for validation: width 4 -> [n_nodes4][32] floats,
 * width 8 -> [n_nodes8][64] floats (host buffer), the device layout: for axis
 * a and group g of four children (G = width / 4 groups), lower planes at float4
 * (2a)G + g, upper planes at (2a + 1)G + g, child codes (int32 bit patterns:
 * >= 0 wide node, < 0 ~leaf position, empty slots an empty box and code 0) at
 * 6G + g.  LIDAR_EINVAL for another width or an 8-wide tree the scene does
 * not have.  Synchronises. */
lidar_status lidar_scene_export_wide(const lidar_scene* scene, int32_t width, float* nodes_host);

/* ----------------------------------------------------------------- sensors */

/* One sensor (Sec. II-A beam configuration, Sec. II-D capability model).
 * Beam b has azimuth az_rad[b] (from +x towards +y in the sensor frame) and
 * elevation el_rad[b] (from the x-y plane towards +z); its unit direction
 * (cos el cos az, cos el sin az, sin el) is evaluated in FP64 on the host and
 * rounded once to FP32.  Ranges in metres; reflectances as fractions. */
typedef struct {
    int64_t n_beams;
    const double* az_rad;      /* host, [n_beams] */
    const double* el_rad;      /* host, [n_beams] */
    float r_min, r_max;        /* returns outside [r_min, r_max] are dropped (nearer hits still occlude) */
    float d_max;               /* capability model maximum range (Eq. 5) */
    float RL_max;              /* reflectance needed at d_max (Eq. 5) */
    float sigma;               /* range-noise standard deviation (Sec. II-A noise factor) */
    float gain;                /* intensity gain g: I = g R (r_ref/d)^p */
    float range_exp;           /* p; 0 reproduces the paper's reflectance intensity */
    float r_ref;
    float divergence_rad;      /* full beam divergence; sampled by n_subrays rays, strongest return kept */
    int32_t n_subrays;         /* 1..LIDAR_MAX_SUBRAYS */
    float sigma_k;             /* range-scaled noise: the standard deviation at true range t is
                                  sigma + sigma_k t, in [0, 0.1); 0 = the paper's constant factor */
} lidar_sensor_desc;

/* Installs a sensor in slot [0, LIDAR_MAX_SENSORS).  Copies the beam
 * directions to the device (synchronously; the host arrays may be freed on
 * return) and computes the slot's ray-order permutation. */
lidar_status lidar_set_sensor(lidar_ctx* ctx, int32_t slot, const lidar_sensor_desc* desc);

/* Replaces the intensity gain g of an installed sensor (the differentiable
 * sensor constant of the adjoint); everything else in the slot is kept. */
lidar_status lidar_set_sensor_gain(lidar_ctx* ctx, int32_t slot, float gain);

/* Copies the slot's FP32 sensor-frame beam directions to host_out [n_beams][3]. */
lidar_status lidar_get_beam_dirs(lidar_ctx* ctx, int32_t slot, float* host_out);

/* --------------------------------------------------------------- materials */

/* Reflectance tables from per-material parameters (a, s, w) [M][3]:
 *   T[m][k] = a_m cos(k deg) + s_m exp(-k^2 / (2 w_m^2)),  k = 0..90,
 * i.e. Eq. 4's Lambertian term with R(0) = a_m plus a specular lobe of height
 * s_m and width w_m degrees.  table_dev: float32 [M][91]. */
lidar_status lidar_build_tables(lidar_ctx* ctx, const float* params_dev, int32_t n_materials,
                                float* table_dev);

/* Chain rule of lidar_build_tables: grad_params_dev [M][3] = dL/d(a, s, w)
 * given grad_table_dev [M][91] = dL/dT (overwrites grad_params_dev). */
lidar_status lidar_build_tables_backward(lidar_ctx* ctx, const float* params_dev,
                                         const float* grad_table_dev, int32_t n_materials,
                                         float* grad_params_dev);

/* Selects the reflectance table [n_materials][91] used by later casts and
 * backward passes.  The table is read in place (not copied). */
lidar_status lidar_set_materials(lidar_ctx* ctx, const float* table_dev, int32_t n_materials);

/* -------------------------------------------------------------------- cast */

/* One frame: sensor slot, frame number (part of the noise counter) and the
 * sensor-to-world pose as a row-major 3x4 [R | t] (56 bytes, no padding). */
typedef struct {
    int32_t sensor;
    int32_t frame;
    float pose[12];
} lidar_frame;

/* Dense per-beam results.  Frame k's beams occupy the index range
 * [off_k, off_k + n_beams(sensor_k)), off_k = sum of n_beams over frames < k.
 * Every array is optional (NULL = not written) and has one entry per beam
 * (normal: 3).  The tape used by lidar_cast_backward is {valid, mat,
 * theta_deg, rf}. */
typedef struct {
    uint8_t* valid;       /* 1 if the return is kept */
    uint32_t* tri;        /* original index of the hit triangle, LIDAR_NO_HIT on a miss */
    float* t;             /* hit distance along the beam before noise (+inf on a miss) */
    float* range;         /* noisy range d = t + sigma z */
    float* intensity;     /* I = g R (r_ref/d)^p (0 on a miss) */
    float* normal;        /* [3] face normal facing the sensor, sensor frame */
    uint16_t* mat;        /* material of the hit triangle */
    uint32_t* inst;       /* instance of the hit triangle */
    uint8_t* sub;         /* chosen sub-ray (strongest valid return) */
    float* theta_deg;     /* incidence angle in degrees */
    float* rf;            /* range factor (r_ref/d)^p */
} lidar_beams;

/* Compacted point cloud: kept returns in (frame, beam) order.  All arrays
 * optional; one entry per point (xyz, normal: 3). */
typedef struct {
    int64_t capacity;
    float* xyz;           /* [3] d * beam direction, sensor frame */
    float* range;
    float* intensity;
    float* normal;        /* [3] sensor frame */
    uint16_t* material;
    uint32_t* instance;
    uint32_t* beam;       /* beam index within its sensor pattern */
    uint32_t* frame;      /* index of the frame in the frames array */
} lidar_points;

/* Casts every beam of every frame against `scene`.
 *   frames_host  [n_frames] host array, copied during the call
 *   seed         noise key: the draw for (beam b, frame f, sensor s, sub-ray k)
 *                is Philox4x64-10 with key (seed, 0) and counter
 *                (b, f | s << 32, k, 0), Box-Muller on its first two words
 *   beams        dense output (may be NULL)
 *   points       compacted output (may be NULL); n_points_dev (device int64)
 *                receives the number of kept returns, which may exceed the
 *                capacity: then only `capacity` points are written and the
 *                status word records LIDAR_ECAPACITY.
 * Requires a material table (lidar_set_materials) and a sensor in every slot
 * the frames name. */
lidar_status lidar_cast(lidar_ctx* ctx, const lidar_scene* scene, const lidar_frame* frames_host,
                        int32_t n_frames, uint64_t seed, const lidar_beams* beams,
                        const lidar_points* points, int64_t* n_points_dev);

/* Copies the first `count` points of a cast's point cloud to the host: for
 * every field that both `dev` (device arrays, as passed to the cast) and
 * `host` (host arrays; pinned memory makes the copies asynchronous) have
 * non-NULL, one device-to-host copy queued on `stream` (a cudaStream_t; NULL:
 * the context's stream), in one call.  `count` is the number of kept returns
 * as read back from the cast's n_points_dev, already on the host (the copies
 * are ordered after the cast only by the stream).  Returns without copying
 * when count is 0.  LIDAR_EINVAL: a NULL ctx, dev or host, or count < 0 or
 * above either capacity; LIDAR_ECUDA: a copy could not be queued. */
lidar_status lidar_points_download(lidar_ctx* ctx, const lidar_points* dev, const lidar_points* host,
                                   int64_t count, void* stream);

/* -------------------------------------------------------- batches and graphs */

/* A device-resident list of frames for repeated casts (many frames along a
 * trajectory, several sensors): the frame records are uploaded once, so casts
 * of a batch make no host copy and can be captured into a CUDA graph.  The
 * batch keeps the sensor slots' beam counts and the launch configuration's
 * tile size of the moment it is created; changing either afterwards makes
 * lidar_cast_batch return LIDAR_ESTATE (create the batch again).  Creating a
 * batch also sizes the context's scratch for casts of it (dense records and
 * compaction), so casting it allocates nothing.  Synchronises. */
typedef struct lidar_batch lidar_batch;
lidar_status lidar_batch_create(lidar_ctx* ctx, const lidar_frame* frames_host, int32_t n_frames,
                                lidar_batch** out);
void lidar_batch_free(lidar_batch* batch);

/* Replaces every frame's pose from device memory poses_dev [n_frames][12]
 * (row-major 3x4 sensor-to-world), asynchronously on the context stream. */
lidar_status lidar_batch_set_poses(lidar_ctx* ctx, lidar_batch* batch, const float* poses_dev);

/* lidar_cast over the frames of a batch; same outputs and semantics. */
lidar_status lidar_cast_batch(lidar_ctx* ctx, const lidar_scene* scene, const lidar_batch* batch, uint64_t seed,
                              const lidar_beams* beams, const lidar_points* points, int64_t* n_points_dev);

/* Captures [pose update from poses_dev (if not NULL)] + lidar_cast_batch into
 * a CUDA graph (captured on a private stream) and instantiates it.  Every
 * lidar_graph_launch replays the whole batch with one launch on the context
 * stream, reading the poses currently in poses_dev.  All pointers are baked
 * into the graph and must stay valid while it is used. */
typedef struct lidar_graph lidar_graph;
lidar_status lidar_graph_create(lidar_ctx* ctx, const lidar_scene* scene, lidar_batch* batch,
                                const float* poses_dev, uint64_t seed, const lidar_beams* beams,
                                const lidar_points* points, int64_t* n_points_dev, lidar_graph** out);
lidar_status lidar_graph_launch(lidar_graph* graph);
void lidar_graph_free(lidar_graph* graph);

/* Adjoint of the intensity with the hits and masks of the forward pass held
 * fixed.  For every beam b with tape valid[b] = 1 and grad_I_dev[b] = dL/dI_b:
 *   dL/dT[m][i]   += g rf (1 - f) dL/dI,   dL/dT[m][i+1] += g rf f dL/dI,
 *   dL/dg         += rf R dL/dI,
 * with i = min(floor(theta), 89), f = theta - i, R the interpolated table
 * value and g = gain.  grad_table_dev [M][91] and grad_gain_dev [1] are
 * accumulated into (not overwritten).  Accumulation uses 64-bit fixed point,
 * so the result is bit-reproducible run to run.  The tape is read once by one
 * cooperative kernel whose device-side waits are bounded by the context's
 * wait limit (LIDAR_ETIMEOUT in the status word if one runs out); tables of
 * more than about 130 materials, and devices without cooperative launch, take
 * three kernels (two reads of the tape) instead.  Tape arrays that start on
 * a 16-byte boundary are streamed by the copy engine; others are read by the
 * threads, with the same result. */
lidar_status lidar_cast_backward(lidar_ctx* ctx, int64_t n_beams, const lidar_beams* tape, float gain,
                                 const float* grad_I_dev, float* grad_table_dev, float* grad_gain_dev);

/* Fused mean-squared-error variant: dL/dI_b = 2 (I_b - I*_b) / N over the
 * beams valid in both the tape and target_valid_dev, N their count.  Writes
 * loss_dev [1] (overwritten) and accumulates grad_table_dev, grad_gain_dev. */
lidar_status lidar_cast_backward_mse(lidar_ctx* ctx, int64_t n_beams, const lidar_beams* tape, float gain,
                                     const float* target_I_dev, const uint8_t* target_valid_dev,
                                     float* loss_dev, float* grad_table_dev, float* grad_gain_dev);

/* As lidar_cast_backward_mse, and writes N, the number of beams the mean
 * runs over, to n_used_dev (device, one uint64; LIDAR_EINVAL if NULL).  For a
 * batch whose beams are split over ranks (data-parallel fitting): rank r
 * computes its loss L_r and gradients G_r (into zeroed buffers) over its own
 * beams with its own N_r; the batch's loss and gradients are then
 * sum_r N_r L_r / sum_r N_r and sum_r N_r G_r / sum_r N_r, one all-reduce of
 * the (N_r x, N_r) vector. */
lidar_status lidar_cast_backward_mse_count(lidar_ctx* ctx, int64_t n_beams, const lidar_beams* tape, float gain,
                                           const float* target_I_dev, const uint8_t* target_valid_dev,
                                           float* loss_dev, float* grad_table_dev, float* grad_gain_dev,
                                           uint64_t* n_used_dev);

/* Allocation-free variant of lidar_cast_backward_mse (no counterpart in the
 * paper; it exists for callers that must not allocate device memory: sensor
 * loops with hard real-time deadlines that cannot afford cudaMalloc's implicit
 * device synchronisation, host applications or plugins whose own memory pool
 * already holds the device's memory, and code that may not create a context).
 * It needs no context either: the caller passes the stream, the tape arrays
 * and the reflectance table directly.
 *   cuda_stream    cudaStream_t to enqueue on (NULL = legacy default stream),
 *                  on the device that is current on the calling thread
 *   valid_dev, mat_dev, theta_deg_dev, rf_dev
 *                  the tape of lidar_beams, [n_beams] each
 *   table_dev      [n_materials][91] reflectance table used by the forward pass
 *   n_materials    1..LIDAR_NOALLOC_MAX_MATERIALS; larger tables are rejected
 *                  with LIDAR_EINVAL (use lidar_cast_backward_mse)
 *   gain, target_I_dev, target_valid_dev, loss_dev, grad_table_dev, grad_gain_dev
 *                  as for lidar_cast_backward_mse (loss overwritten, gradients
 *                  accumulated)
 * Scratch lives in a fixed device array inside the library
 * (LIDAR_NOALLOC_SCRATCH_BYTES, held by every device that loads the library
 * until the process exits).  The entry point calls no cudaMalloc, cudaFree or
 * allocating library routine.  Its first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, once per device, cached), so
 * make that first call before any stream capture.  The cached address belongs
 * to the device's primary context as it was then: after cudaDeviceReset on
 * that device the array may move, and this entry point must not be called
 * again in that process.  All calls share the one array: the accumulators are
 * cleared on the stream at the start of every call, and calls whose work
 * overlaps on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller. */
#define LIDAR_NOALLOC_MAX_MATERIALS 64
#define LIDAR_NOALLOC_SCRATCH_BYTES 55296
lidar_status lidar_cast_backward_mse_noalloc(void* cuda_stream, int64_t n_beams, const uint8_t* valid_dev,
                                             const uint16_t* mat_dev, const float* theta_deg_dev,
                                             const float* rf_dev, const float* table_dev, int32_t n_materials,
                                             float gain, const float* target_I_dev,
                                             const uint8_t* target_valid_dev, float* loss_dev,
                                             float* grad_table_dev, float* grad_gain_dev);

/* ----------------------------------------------------------- instrumentation */

/* Work of one cast, counted by an instrumented instantiation of the same
 * traversal kernel (not the timed one): BVH nodes fetched, triangles tested,
 * and how many distinct nodes and triangles were touched.  Used to state the
 * algorithmic bytes and flops behind the roofline. */
typedef struct {
    uint64_t rays;           /* traced rays (beams x sub-rays) */
    uint64_t node_bytes;     /* bytes per node fetch: 64 (binary tree), 128 (4-wide) or 256 (8-wide) */
    uint64_t node_visits;    /* node fetches */
    uint64_t tri_tests;      /* 48-byte triangle fetches + watertight tests */
    uint64_t unique_nodes;   /* distinct nodes fetched */
    uint64_t unique_tris;    /* distinct triangles fetched */
} lidar_work_counts;

/* Runs the cast of lidar_cast (dense valid flags only) with counting enabled
 * and returns the totals.  beam_cost_dev (may be NULL): uint32 per beam in the
 * dense layout, node fetches + triangle tests of that beam (all sub-rays).
 * Synchronises. */
lidar_status lidar_count_work(lidar_ctx* ctx, const lidar_scene* scene, const lidar_frame* frames_host,
                              int32_t n_frames, uint64_t seed, lidar_work_counts* out, uint32_t* beam_cost_dev);

/* Measured FP32 arithmetic rate of the context's device, the denominator of
 * the traversal's ALU fraction (its box and triangle tests are FP32 adds,
 * multiplies, fused multiply-adds and min/max).  Runs a kernel of independent
 * fused multiply-add chains on every SM (eight warps per scheduler, no memory
 * traffic), fma_per_thread FMAs per thread (>= 64; about 8e6 runs for tens of
 * milliseconds), once as scalar FMAs and once as packed FP32 pairs, and
 * returns the faster: *flops_per_s (2 FLOPs per FMA, CUDA-event time),
 * *kernel_ms and *packed (1 if the packed form was faster).  The rate follows
 * the SM clock of the moment, which the caller should sample alongside.
 * Synchronises. */
lidar_status lidar_measure_fp32_rate(lidar_ctx* ctx, int64_t fma_per_thread, double* flops_per_s,
                                     double* kernel_ms, int32_t* packed);

/* --------------------------------------------------------------- scheduling */

/* Ray schedule of a sensor slot.  The cast kernel's warps take groups of 32
 * consecutive positions of the slot's ray order; by default that order is the
 * Morton order of the beam directions (coherent warps).  This call measures
 * the traversal cost of every beam on `frame` (one frame of that slot, cast
 * with counting enabled), and reorders the 32-beam groups so that the most
 * expensive groups run first (longest-processing-time-first), which shortens
 * the tail of a cast where the last warps would otherwise run alone.
 * mode 0: whole 32-beam groups of the Morton order, by their largest cost;
 * mode 1: single beams by cost bucket (4 buckets per octave of cost, most
 *         expensive first, Morton order within a bucket), so that each warp
 *         gets beams of similar cost (fewer idle lanes).
 * The schedule never changes results, only their timing; use the costs of a
 * nearby pose (e.g. the previous frame).  Synchronises. */
lidar_status lidar_schedule_by_cost(lidar_ctx* ctx, const lidar_scene* scene, const lidar_frame* frame,
                                    uint64_t seed, int32_t mode);

/* Restores the Morton order of a slot. */
lidar_status lidar_reset_schedule(lidar_ctx* ctx, int32_t slot);

/* --------------------------------------------- rolling shutter, multi-echo */

/* One sweep of a spinning sensor: the sensor-to-world pose at its start and
 * at its end (row-major 3x4 each).  Beam b fires at the fraction s_b of the
 * sweep — its azimuth over 2 pi, in [0, 1): the sweep starts at azimuth 0 and
 * turns towards +y — and sees the blended pose (Sec. II-A turns the render
 * camera with the sensor's spin over each time step): translation
 * (1 - s) t0 + s t1, rotation of the normalised blend (1 - s) q0 + s q1 of the
 * poses' unit quaternions (found in FP64, rounded once, same hemisphere),
 * both in FP32 with every operation rounded as written. */
typedef struct {
    int32_t sensor;
    int32_t frame;
    float pose0[12];
    float pose1[12];
} lidar_sweep_frame;

/* Multiple returns per beam (Sec. IV: multiple echoes are future work), from
 * the returns of the beam's sub-rays (LIDAR_MAX_SUBRAYS at most):
 *   mode 0: the n_echoes strongest, strongest first (ties to the lower
 *           sub-ray), skipping a return closer than `separation` metres in
 *           range to one already kept;
 *   mode 1: the first (smallest range) and, if n_echoes >= 2 and it lies at
 *           least `separation` beyond it, the last (largest range) return.
 * Per beam (dense layout): count, and [n][n_echoes] range, intensity, tri
 * (original index), sub (sub-ray index); slots past count hold 0,
 * LIDAR_NO_HIT and 255.  count is required, the arrays optional. */
typedef struct {
    int32_t n_echoes;      /* 1..4 */
    int32_t mode;          /* 0 strongest, 1 first and last */
    float separation;      /* metres, >= 0 */
    uint8_t* count;
    float* range;
    float* intensity;
    uint32_t* tri;
    uint8_t* sub;
} lidar_echoes;

/* Casts every beam of every sweep (dense outputs as lidar_cast: the strongest
 * return in `beams`, normals rotated by the beam's own pose; no point cloud)
 * and, if `echoes` is given, the multi-echo outputs.  Persistent warp tiles
 * over each slot's ray order and cost schedule with the 4-wide traversal; the
 * sub-rays, noise draws and model are those of lidar_cast.  Asynchronous. */
lidar_status lidar_cast_sweep(lidar_ctx* ctx, const lidar_scene* scene, const lidar_sweep_frame* frames_host,
                              int32_t n_frames, uint64_t seed, const lidar_beams* beams, const lidar_echoes* echoes);

/* ------------------------------------------------- raster-and-resample path */

/* The paper's own sampling (Sec. II-A..II-C), as compute rasterisation: per
 * frame, n_cameras pin-hole cameras at the sensor pose share the 360-degree
 * horizontal field (camera k looks along sensor azimuth
 * -pi + (k + 1/2) 2 pi / n_cameras; square width x width image; Eq. 1-2:
 * f = width / (2 tan(pi / n_cameras)), c = width / 2).  Each camera renders,
 * through every pixel centre, the depth pass as z-depth in three bytes
 * (q = rn(z (2^24 - 1) / T_max), 2^24 - 1 = no hit), the incidence angle in
 * three bytes (theta / 90 degrees), the material stencil in one byte
 * (material & 255) and the instance colour in three bytes (instance & 2^24-1).
 * A beam reads the pixel its direction d projects to (Eq. 3, corrected:
 * camera = largest d . F_k, n_x = c + f x/z, n_y = c - f y/z with (x, y, z)
 * = d in camera axes, pixel = floor; a column outside the image is clamped —
 * a beam on the border of two cameras — and a row outside it leaves the beam
 * without a return), takes range = depth / (d . F_k) and the decoded angle
 * and stencil, and goes through the noise, Eq. 4 lookup, Eq. 5 and intensity
 * of lidar_cast (the draw of sub-ray 0; sensors' sub-rays are not used). */
typedef struct {
    int32_t width;       /* pixels per side of each camera image, 1..16384 */
    int32_t n_cameras;   /* cameras around the vertical axis, 3..64 (FOV_c = 360 / n_cameras degrees) */
} lidar_raster_config;

/* Dense per-beam outputs like lidar_cast (beams required; points are not
 * produced): tri = the triangle seen through the beam's pixel centre, t = the
 * range before noise, normal = 0 (the G-buffer has no normal), mat = the
 * 8-bit stencil, inst = the 24-bit colour, sub = 0.  Frames are rendered one
 * after another in the context's scratch (about 16 + 4 bytes per pixel per
 * camera plus 3 bytes per triangle and camera).  Asynchronous. */
lidar_status lidar_raster_cast(lidar_ctx* ctx, const lidar_scene* scene, const lidar_frame* frames_host,
                               int32_t n_frames, uint64_t seed, const lidar_raster_config* cfg,
                               const lidar_beams* beams);

/* The G-buffer of one frame, [n_cameras][width][width] uint32 each (any may be
 * NULL): depth code, angle code | stencil << 24, colour, and the original index
 * of the triangle seen (LIDAR_NO_HIT on a miss).  Asynchronous. */
lidar_status lidar_raster_gbuffer(lidar_ctx* ctx, const lidar_scene* scene, const lidar_frame* frame_host,
                                  const lidar_raster_config* cfg, uint32_t* depth_dev, uint32_t* angle_mat_dev,
                                  uint32_t* inst_dev, uint32_t* tri_dev);

/* --------------------------------------------------------------- launch tuning */

typedef struct {
    int32_t block_threads;   /* threads per block of the cast kernel (multiple of 32, <= 256) */
    int32_t blocks_per_sm;   /* persistent blocks per SM */
    int32_t tile_rays;       /* rays a warp takes from the work counter at a time (multiple of 32) */
    int32_t ray_order;       /* 0 = beam order, 1 = Morton order of beam directions */
    int32_t traversal;       /* binary tree: 0 = each lane tests its triangles as it meets them,
                                1 = warp-synchronous with postponed triangle tests;
                                2 = 4-wide tree, per lane, children visited near to far;
                                3 = 8-wide tree, per lane, children visited near to far (a cast on a
                                    scene without an 8-wide tree returns LIDAR_EINVAL) */
    int32_t fused_scatter;   /* 1: the point-cloud scatter runs inside the cast kernel after a grid-wide
                                wait (cooperative launch); 0: as a separate kernel */
} lidar_launch_config;

lidar_status lidar_get_launch_config(lidar_ctx* ctx, lidar_launch_config* out);
lidar_status lidar_set_launch_config(lidar_ctx* ctx, const lidar_launch_config* cfg);

/* Overlap of consecutive direct casts (lidar_cast calls on the context's
 * stream, outside a stream capture; enable 1 by default, 0 to cast one after
 * the other).  A cast then starts on the SMs the cast before it leaves idle
 * once that cast's work queue is empty (its last, longest traversals still
 * running), by programmatic dependent launch; the library orders everything
 * the two share (counter regions, dense scratch).  Results are bit-identical
 * either way.  Anything else on the stream between two casts (a copy, an event
 * wait, another kernel) lets the second start only when the first has
 * finished, as usual.  Callers must not let the point or dense buffers of one
 * cast be read by later stream work that does not follow that cast on the
 * stream. */
lidar_status lidar_set_cast_overlap(lidar_ctx* ctx, int32_t enable);
lidar_status lidar_get_cast_overlap(lidar_ctx* ctx, int32_t* enable);

/* Limit, in nanoseconds of GPU time (the device's global timer), of every
 * bounded device-side wait in the context's kernels: the grid-wide wait of a
 * cast whose point-cloud scatter runs inside the cast kernel, and the waits of
 * the one-pass adjoint.  A wait that runs out records LIDAR_ETIMEOUT in the
 * status word (read by lidar_sync_status) and its block leaves the kernel
 * without the work after the wait, so that call's outputs past the wait are
 * incomplete; nothing hangs and the context stays usable.  Default
 * 2,000,000,000 (2 s), far beyond any legitimate wait; 0 gives up at the first
 * check that finds the wait unfinished (exercises the timeout path).  Applies
 * to launches made afterwards. */
lidar_status lidar_set_wait_limit(lidar_ctx* ctx, uint64_t nanoseconds);
lidar_status lidar_get_wait_limit(lidar_ctx* ctx, uint64_t* nanoseconds);

#ifdef __cplusplus
}
#endif
#endif /* LIDAR_H */
