// Per-beam return generation: one persistent kernel takes tiles of beams from
// a global work counter (tiles ordered by frame, then by position in the
// sensor's ray order), and for every beam runs
//   ray generation -> closest-hit BVH traversal -> surface attributes ->
//   incidence angle -> reflectance lerp -> Philox range noise -> cut-offs ->
//   intensity -> strongest of the sub-rays
// writing a dense per-beam record (a beam's sub-rays on neighbouring lanes).
// The kept returns are then compacted in (frame, beam) order, in the same
// launch after one grid-wide wait, or by a second kernel.

#include "common.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include "philox.cuh"
#include "trace.cuh"
#include "shade.cuh"

namespace lidar {
namespace {

__device__ __forceinline__ int find_frame(const int64_t* __restrict__ prefix, int n_frames, int64_t tile)
{
    int lo = 0, hi = n_frames - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&prefix[mid]) <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent kernel, work taken per warp: lane 0 claims a tile of `tile_rays`
// consecutive ray-order positions of one frame (a multiple of 32) and the warp
// traces it 32 rays at a time; no block-wide barrier.
__device__ __forceinline__ int frame_of_index(const FrameDev* __restrict__ frames, int n_frames, int64_t idx)
{
    int lo = 0, hi = n_frames - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (frames[mid].beam_offset <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kCompactTileBeams = 1024;
constexpr int kScatterItems = 4;
constexpr int kPdlScatterThreads = 64;  // an overlapped cast's scatter blocks

// Ordered scatter of one compaction tile of kCompactTileBeams dense beams by
// the calling block (blockDim a multiple of 32, at most 256).  A chunk is
// kScatterItems rows of blockDim consecutive beams, row k read by thread t at
// beam chunk + k * blockDim + t, so the kept beams of one warp row land in
// consecutive output slots (coalesced stores); ballots rank them in the warp
// and one table of per-(row, warp) counts in shared memory orders the rows
// and warps.  `s_warp` holds kScatterItems * 8 words.
template <int kItems = kScatterItems>
__device__ void scatter_tile(const SensorDev* __restrict__ sensors, const FrameDev* __restrict__ frames,
                             int n_frames, int64_t n, const BeamsOut& dense, int64_t tile, int64_t tile_offset,
                             const lidar_points& pts, int* status, uint32_t* s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const int chunk_beams = blockDim.x * kItems;
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t running = tile_offset;
    for (int chunk = 0; chunk < kCompactTileBeams; chunk += chunk_beams) {
        const int64_t base = tile * kCompactTileBeams + chunk;
        // gather every field of the chunk's beams before the scan and the
        // first store: the point arrays could alias the dense ones as far as
        // the compiler knows, so loads after a store would wait for it
        bool v[kItems];
        float rg[kItems], it[kItems], nx[kItems], ny[kItems], nz[kItems];
        float dx[kItems], dy[kItems], dz[kItems];
        uint16_t mt[kItems];
        uint32_t in[kItems], bm[kItems], fk[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            rg[k] = it[k] = nx[k] = ny[k] = nz[k] = dx[k] = dy[k] = dz[k] = 0.0f;
            mt[k] = 0;
            in[k] = bm[k] = fk[k] = 0;
            v[k] = false;
            const int row = chunk + k * blockDim.x + threadIdx.x;
            const int64_t idx = base + k * blockDim.x + threadIdx.x;
            if (row >= kCompactTileBeams || idx >= n) continue;
            v[k] = __ldcg(&dense.valid[idx]) != 0;
            const int fi = frame_of_index(frames, n_frames, idx);
            const FrameDev& fr = frames[fi];
            bm[k] = (uint32_t)(idx - fr.beam_offset);
            fk[k] = (uint32_t)fi;
            rg[k] = __ldcg(&dense.range[idx]);
            if (pts.xyz) {
                const float* dir = sensors[fr.sensor].dirs + 3 * (int64_t)bm[k];
                dx[k] = __ldg(dir);
                dy[k] = __ldg(dir + 1);
                dz[k] = __ldg(dir + 2);
            }
            if (pts.intensity) it[k] = __ldcg(&dense.intensity[idx]);
            if (pts.normal) {
                nx[k] = __ldcg(&dense.normal[3 * idx + 0]);
                ny[k] = __ldcg(&dense.normal[3 * idx + 1]);
                nz[k] = __ldcg(&dense.normal[3 * idx + 2]);
            }
            if (pts.material) mt[k] = __ldcg(&dense.mat[idx]);
            if (pts.instance) in[k] = __ldcg(&dense.inst[idx]);
        }
        unsigned mask[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            mask[k] = __ballot_sync(0xffffffffu, v[k]);
            if (lane == 0) s_warp[k * 8 + warp] = (uint32_t)__popc(mask[k]);
        }
        __syncthreads();
        // slots before row k, warp w: all of rows < k, then warps < w of row k
        uint32_t before[kItems], total = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            for (int w = 0; w < n_warps; ++w) {
                const uint32_t c = s_warp[k * 8 + w];
                if (w == warp) before[k] = total;
                total += c;
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (!v[k]) continue;
            const int64_t pos = running + before[k] + (uint32_t)__popc(mask[k] & lt_mask);
            if (pos >= pts.capacity) {
                raise_status(status, ST_CAPACITY);
                continue;
            }
            if (pts.xyz) {
                pts.xyz[3 * pos + 0] = rg[k] * dx[k];
                pts.xyz[3 * pos + 1] = rg[k] * dy[k];
                pts.xyz[3 * pos + 2] = rg[k] * dz[k];
            }
            if (pts.range) pts.range[pos] = rg[k];
            if (pts.intensity) pts.intensity[pos] = it[k];
            if (pts.normal) {
                pts.normal[3 * pos + 0] = nx[k];
                pts.normal[3 * pos + 1] = ny[k];
                pts.normal[3 * pos + 2] = nz[k];
            }
            if (pts.material) pts.material[pos] = mt[k];
            if (pts.instance) pts.instance[pos] = in[k];
            if (pts.beam) pts.beam[pos] = bm[k];
            if (pts.frame) pts.frame[pos] = fk[k];
        }
        running += total;
        __syncthreads();
    }
}

// Counts of kept returns per compaction tile of kCompactTileBeams dense
// indices, gathered by the cast itself (warp-aggregated atomics).  With the
// scatter fused into the cast, every block waits once for all counts and
// scatters a run of tiles; otherwise the last block to finish turns them into
// exclusive offsets for one more kernel (k_scatter_points).
struct CompactCounts {
    unsigned* counts;     // [n_tiles], zeroed before the cast; NULL: not counting
    unsigned* done;       // finished-block counter, zeroed before the cast
    int64_t* offsets;     // [n_tiles] exclusive prefix of counts (written by the last block)
    int64_t* total;       // number of kept returns (may be NULL)
    int64_t n_tiles;
};

// byte offset, from the tile counts, of the cast's 64-bit work counter: after
// the counts and the finished-block word, 8-byte aligned
static size_t compact_counter_offset(int64_t n_tiles)
{
    return (size_t)(((n_tiles + 1) * 4 + 7) / 8 * 8);
}

__device__ __forceinline__ void count_kept_warp(const CompactCounts& cc, bool kept, int64_t dense_index, int lane)
{
    const unsigned vm = __ballot_sync(0xffffffffu, kept);
    if (!kept) return;
    const unsigned long long t = (unsigned long long)(dense_index / kCompactTileBeams);
    const unsigned peers = __match_any_sync(vm, t);
    if (lane == __ffs(peers) - 1) atomicAdd(&cc.counts[t], (unsigned)__popc(peers));
}

// exclusive scan of cc.counts by one block (runs in the last block only)
__device__ void scan_counts_block(const CompactCounts& cc)
{
    __shared__ long long s_part[256];
    const int nt = blockDim.x;
    const int64_t per = (cc.n_tiles + nt - 1) / nt;
    const int64_t lo = (int64_t)threadIdx.x * per, hi = min(lo + per, cc.n_tiles);
    long long sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += __ldcg(&cc.counts[i]);
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const long long v = threadIdx.x >= (unsigned)off ? s_part[threadIdx.x - off] : 0;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = threadIdx.x == 0 ? 0 : s_part[threadIdx.x - 1];
    for (int64_t i = lo; i < hi; ++i) {
        cc.offsets[i] = run;
        run += __ldcg(&cc.counts[i]);
    }
    if (threadIdx.x == nt - 1 && cc.total) *cc.total = s_part[nt - 1];
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier number `k` (1, 2, ...) over a counter zeroed before the
// launch, for cooperative launches only (all blocks co-resident).  The wait
// is bounded: after wait_ns nanoseconds (the context's wait limit, 2 s by
// default) it raises ST_TIMEOUT and returns false in every thread of the
// block, which then leaves the kernel.
__device__ bool grid_barrier(unsigned* counter, unsigned k, int* status, uint64_t wait_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        const unsigned target = k * gridDim.x;
        const uint64_t t0 = global_ns();
        int ok = 1;
        while (*(volatile unsigned*)counter < target) {
            if (global_ns() - t0 > wait_ns) {
                raise_status(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <bool kCount, int kMinBlocks, int kTrav>
__global__ void __launch_bounds__(256, kMinBlocks) k_cast(SceneDev S, const SensorDev* __restrict__ sensors,
                                              const FrameDev* __restrict__ frames, int n_frames,
                                              const int64_t* __restrict__ tile_prefix, int64_t n_tiles,
                                              TableDev T, uint64_t seed, BeamsOut out, int* status,
                                              unsigned long long* work_counter, int tile_rays, WorkCount wc,
                                              CompactCounts cc, lidar_points pts, int64_t n_beams_total, int fused,
                                              const __grid_constant__ InlineFrames inl, unsigned* zero_next,
                                              int64_t zero_words, uint64_t wait_ns, int pdl)
{
    const int lane = threadIdx.x & 31;
    // clear the counter region of the cast after this one
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < zero_words; i += (int64_t)gridDim.x * blockDim.x)
        zero_next[i] = 0u;
    // overlapped casts: the block's clearing is done before any of its warps
    // lets the next cast start
    if (pdl) __syncthreads();
    // frames and their first tiles: from the launch parameters when they came inline
    const FrameDev* fr_tab = inl.n ? inl.f : frames;
    const int64_t* tile_first = inl.n ? inl.prefix : tile_prefix;
    extern __shared__ int2 sh_stack[];  // [kSharedStack][blockDim.x]
    // closest hit of one ray with the instantiated traversal (the warp-synchronous
    // one needs every lane; the others run on the active lanes)
    auto trace = [&](const RayPre& p, float t_max, HitRec& h, bool active, unsigned* cost) -> bool {
        if (kTrav == 1) return trace_closest_warp<kCount>(S, p, t_max, h, active, &wc);
        if (!active) return true;
        if (kTrav == 3)
            return trace_closest8<kCount>(S, p, t_max, h, &wc, sh_stack + threadIdx.x, blockDim.x, cost);
        if (kTrav == 2)
            return trace_closest4<kCount>(S, p, t_max, h, &wc, sh_stack + threadIdx.x, blockDim.x, cost);
        return trace_closest<kCount>(S, p, t_max, h, &wc, sh_stack + threadIdx.x, blockDim.x, cost);
    };
    while (true) {
        unsigned long long claimed = 0;
        if (lane == 0) claimed = atomicAdd(work_counter, 1ull);
        const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, claimed, 0);
        if (tile >= n_tiles) {
            if (pdl && lane == 0) {
                // the work queue is empty: once the cast before this one has
                // completed (its counter region and dense records are then free
                // for the cast after this one), the next cast may start on the
                // SMs this cast's last tiles leave idle
                __threadfence();
                asm volatile("griddepcontrol.wait;" ::: "memory");
                asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
            }
            break;
        }
        const int fi = find_frame(tile_first, n_frames, tile);
        const FrameDev& fr = fr_tab[fi];
        const SensorDev& sd = sensors[fr.sensor];
        const int64_t base = (tile - tile_first[fi]) * tile_rays;
        if (!kCount && sd.n_sub > 1) {
            // a beam's sub-rays on neighbouring lanes (32 / n_sub beams per warp
            // step): they take nearly the same path through the tree, so the warp
            // stays converged and shares its node fetches; the strongest return
            // (ties to the lower sub-ray, sub-ray 0 when none is kept) is picked
            // across the beam's lanes and written by its lane
            const int ns = sd.n_sub;
            const int G = 32 / ns;
            const int g = lane / ns, k = lane - g * ns;
            for (int j0 = 0; j0 < tile_rays; j0 += G) {
                const int64_t pos = base + j0 + g;
                const bool active = g < G && j0 + g < tile_rays && pos < sd.n_beams;
                if (!__any_sync(0xffffffffu, active)) break;
                uint32_t beam = 0;
                float d0 = 0.0f, d1 = 0.0f, d2 = 1.0f;
                if (active) {
                    beam = sd.order ? __ldg(&sd.order[pos]) : (uint32_t)pos;
                    d0 = __ldg(&sd.dirs[3 * (int64_t)beam]);
                    d1 = __ldg(&sd.dirs[3 * (int64_t)beam + 1]);
                    d2 = __ldg(&sd.dirs[3 * (int64_t)beam + 2]);
                }
                RayW r = world_ray(fr.pose, d0, d1, d2);
                if (k > 0) subray_dir(r.dx, r.dy, r.dz, sd.alpha[k], sd.beta[k]);
                const RayPre p = prepare_ray(r);
                HitRec h;
                if (!trace(p, sd.t_max, h, active, nullptr))
                    raise_status(status, h.leaf == kBadIndex ? ST_BOUNDS : ST_STACK);
                BeamResult res;
                res.valid = 0;
                res.intensity = 0.0f;
                if (active)
                    shade(S, h, r, sd, T, seed, beam, (uint32_t)fr.frame, (uint32_t)fr.sensor, (uint32_t)k, res);
                const float score = active ? (res.valid ? res.intensity : -1.0f) : -2.0f;
                float top = -3.0f;
                int arg = 0;
                for (int m = 0; m < ns; ++m) {
                    const float sm = __shfl_sync(0xffffffffu, score, min(g * ns + m, 31));
                    if (sm > top) {
                        top = sm;
                        arg = m;
                    }
                }
                const bool winner = active && k == arg;
                if (cc.counts) count_kept_warp(cc, winner && res.valid, fr.beam_offset + beam, lane);
                if (winner) write_beam(out, fr.beam_offset + beam, res, fr.pose, k);
            }
            continue;
        }
        // one beam per lane, its sub-rays in turn (the counting launch: per-beam costs)
        for (int j0 = 0; j0 < tile_rays; j0 += 32) {
            const int64_t pos = base + j0 + lane;
            const bool active = pos < sd.n_beams;
            if (!__any_sync(0xffffffffu, active)) break;
            uint32_t beam = 0;
            float d0 = 0.0f, d1 = 0.0f, d2 = 1.0f;
            if (active) {
                beam = sd.order ? __ldg(&sd.order[pos]) : (uint32_t)pos;
                d0 = __ldg(&sd.dirs[3 * (int64_t)beam]);
                d1 = __ldg(&sd.dirs[3 * (int64_t)beam + 1]);
                d2 = __ldg(&sd.dirs[3 * (int64_t)beam + 2]);
            }
            const RayW beam_ray = world_ray(fr.pose, d0, d1, d2);
            BeamResult best;
            int best_sub = 0;
            float best_I = -1.0f;
            unsigned cost = 0;
            for (int k = 0; k < sd.n_sub; ++k) {
                RayW r = beam_ray;
                if (k > 0) subray_dir(r.dx, r.dy, r.dz, sd.alpha[k], sd.beta[k]);
                const RayPre p = prepare_ray(r);
                HitRec h;
                if (!trace(p, sd.t_max, h, active, &cost))
                    raise_status(status, h.leaf == kBadIndex ? ST_BOUNDS : ST_STACK);
                if (active) {
                    BeamResult res;
                    shade(S, h, r, sd, T, seed, beam, (uint32_t)fr.frame, (uint32_t)fr.sensor, (uint32_t)k, res);
                    if (k == 0) best = res;
                    if (res.valid && res.intensity > best_I) {
                        best_I = res.intensity;
                        best = res;
                        best_sub = k;
                    }
                }
            }
            if (cc.counts) count_kept_warp(cc, active && best.valid, fr.beam_offset + beam, lane);
            if (!active) continue;
            write_beam(out, fr.beam_offset + beam, best, fr.pose, best_sub);
            if (kCount && wc.beam_cost) wc.beam_cost[fr.beam_offset + beam] = cost;
        }
    }
    if (cc.counts && fused) {
        // cooperative launch: every block of the grid is resident, so the grid
        // can wait until every kept return is counted; then each block
        // scatters a contiguous run of tiles, whose first offset is the sum of
        // the (final) counts before the run — no scan and no second wait
        if (!grid_barrier(cc.done, 1, status, wait_ns)) return;
        __shared__ uint32_t s_warp[kScatterItems * 8];
        __shared__ long long s_red[8];
        const int64_t t0 = (int64_t)blockIdx.x * cc.n_tiles / gridDim.x;
        const int64_t t1 = ((int64_t)blockIdx.x + 1) * cc.n_tiles / gridDim.x;
        long long before = 0;
        for (int64_t i = threadIdx.x; i < t0; i += blockDim.x) before += __ldcg(&cc.counts[i]);
        for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
        if (lane == 0) s_red[threadIdx.x >> 5] = before;
        __syncthreads();
        long long run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) run += s_red[w];
        for (int64_t t = t0; t < t1; ++t) {
            scatter_tile(sensors, fr_tab, n_frames, n_beams_total, out, t, run, pts, status, s_warp);
            run += __ldcg(&cc.counts[t]);
        }
        // the block holding the last tile knows the total
        if (t1 == cc.n_tiles && threadIdx.x == 0 && cc.total) *cc.total = run;
    } else if (cc.counts) {
        __shared__ bool s_last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(cc.done, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            scan_counts_block(cc);
        }
    }
}

// ------------------------------------------------------------------ compaction

constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 4;
constexpr int kCompactTile = kCompactThreads * kCompactItems;
static_assert(kCompactTile == kCompactTileBeams, "the scatter tiles are the cast's counting tiles");

// Compaction tiles (kCompactTileBeams beams) blockIdx.x, blockIdx.x + gridDim.x, ...
// With `pdl` (an overlapped cast's scatter) the block first lets the next
// cast start, then waits for its own cast to complete.
template <int kItems>
__global__ void __launch_bounds__(kCompactThreads) k_scatter_points(
    const SensorDev* __restrict__ sensors, const FrameDev* __restrict__ frames, int n_frames, int64_t n,
    BeamsOut dense, const int64_t* __restrict__ tile_offsets, lidar_points pts, int* status,
    const __grid_constant__ InlineFrames inl, int pdl)
{
    if (pdl) {
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        asm volatile("griddepcontrol.wait;" ::: "memory");
    }
    __shared__ uint32_t s_warp[kItems * 8];
    const int64_t n_tiles = (n + kCompactTileBeams - 1) / kCompactTileBeams;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x)
        scatter_tile<kItems>(sensors, inl.n ? inl.f : frames, n_frames, n, dense, t, tile_offsets[t], pts, status,
                             s_warp);
}

// ------------------------------------------------------------------ ray order

// Octahedral map of a unit direction to [0,1]^2 (Praun & Hoppe 2003), then a
// 32-bit Morton code of the two 16-bit coordinates.
__device__ __forceinline__ uint32_t spread2(uint32_t x)
{
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__global__ void k_dir_keys(const float* __restrict__ dirs, int n, uint32_t* keys, uint32_t* vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = dirs[3 * i], y = dirs[3 * i + 1], z = dirs[3 * i + 2];
    const float s = fabsf(x) + fabsf(y) + fabsf(z);
    x /= s; y /= s; z /= s;
    float u = x, v = y;
    if (z < 0.0f) {
        u = (1.0f - fabsf(y)) * (x >= 0.0f ? 1.0f : -1.0f);
        v = (1.0f - fabsf(x)) * (y >= 0.0f ? 1.0f : -1.0f);
    }
    const uint32_t qu = (uint32_t)fminf(fmaxf((u * 0.5f + 0.5f) * 65535.0f, 0.0f), 65535.0f);
    const uint32_t qv = (uint32_t)fminf(fmaxf((v * 0.5f + 0.5f) * 65535.0f, 0.0f), 65535.0f);
    keys[i] = (spread2(qu) << 1) | spread2(qv);
    vals[i] = (uint32_t)i;
}

}  // namespace

namespace {

struct CastArgs {
    SceneDev scene;
    const SensorDev* sensors;
    const FrameDev* frames;
    int n_frames;
    const int64_t* prefix;
    int64_t n_tiles;
    TableDev table;
    uint64_t seed;
    BeamsOut out;
    int* status;
    unsigned long long* work_counter;
    int tile_rays;
    WorkCount wc;
    CompactCounts cc;
    lidar_points pts;
    int64_t n_total;
    int fused;
    InlineFrames inl;
    unsigned* zero_next;
    int64_t zero_words;
    uint64_t wait_ns;
    int pdl;
};

template <bool C, int V, int W>
cudaError_t launch_one(cudaStream_t s, CastArgs a, int64_t grid, int block, size_t smem, int num_sms,
                       cudaError_t* refused)
{
    auto fn = k_cast<C, V, W>;
    void* args[] = {&a.scene, &a.sensors, &a.frames, &a.n_frames, &a.prefix, &a.n_tiles, &a.table, &a.seed,
                    &a.out, &a.status, &a.work_counter, &a.tile_rays, &a.wc, &a.cc, &a.pts, &a.n_total,
                    &a.fused, &a.inl, &a.zero_next, &a.zero_words, &a.wait_ns, &a.pdl};
    if (a.fused) {
        // every block must be resident for the grid-wide waits; the occupancy
        // of this instantiation depends only on the block size and the shared
        // memory, so it is asked once per pair
        static std::mutex m;
        static std::map<std::pair<int, size_t>, int> cache;
        int per_sm = 0;
        {
            std::lock_guard<std::mutex> lock(m);
            auto it = cache.find({block, smem});
            if (it != cache.end()) {
                per_sm = it->second;
            } else {
                cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
                if (e != cudaSuccess) return e;
                cache[{block, smem}] = per_sm;
            }
        }
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        if (grid > (int64_t)per_sm * num_sms) grid = (int64_t)per_sm * num_sms;
    }
    if (a.pdl) {
        // programmatic dependent launch: this cast may start before the one
        // ahead of it in the stream has finished (the kernel orders what must be
        // ordered, see k_cast); refused combinations fall back to a plain launch
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)grid);
        lc.blockDim = dim3(block);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        attr[1].id = cudaLaunchAttributeCooperative;
        attr[1].val.cooperative = 1;
        lc.attrs = attr;
        lc.numAttrs = a.fused ? 2 : 1;
        const cudaError_t pe = cudaLaunchKernelExC(&lc, (const void*)fn, args);
        if (pe == cudaSuccess) return cudaSuccess;
        cudaGetLastError();
        if (refused) *refused = pe;
        a.pdl = 0;
    }
    if (a.fused) return cudaLaunchCooperativeKernel((const void*)fn, dim3((unsigned)grid), dim3(block), args, smem, s);
    fn<<<(unsigned)grid, block, smem, s>>>(a.scene, a.sensors, a.frames, a.n_frames, a.prefix, a.n_tiles, a.table,
                                            a.seed, a.out, a.status, a.work_counter, a.tile_rays, a.wc, a.cc, a.pts,
                                            a.n_total, a.fused, a.inl, a.zero_next, a.zero_words, a.wait_ns, a.pdl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cast(cudaStream_t s, const SceneDev& scene, const SensorDev* sensors_dev,
                        const FrameDev* frames_dev, int n_frames, const int64_t* tile_prefix_dev,
                        int64_t n_tiles, TableDev table, uint64_t seed, BeamsOut out, int* status,
                        unsigned long long* work_counter, const LaunchCfg& cfg, int num_sms,
                        int64_t n_beams_total, const WorkCount* count, void* compact_scratch,
                        int64_t* n_points_dev, const lidar_points* points, bool* scattered,
                        const InlineFrames* inline_frames, const CounterRegion* region)
{
    if (scattered) *scattered = false;
    if (n_tiles == 0) return cudaSuccess;
    const int64_t warps = cfg.block_threads / 32;
    int64_t grid = (int64_t)num_sms * cfg.blocks_per_sm;
    if (grid > (n_tiles + warps - 1) / warps) grid = (n_tiles + warps - 1) / warps;
    // register budget from the requested residency: threads per SM <= 512 ->
    // up to 128 registers, <= 768 -> 85, more -> 64
    const int resident = cfg.block_threads * cfg.blocks_per_sm;
    const int variant = resident <= 512 ? 2 : (resident <= 768 ? 3 : 4);
    CastArgs a{};
    a.scene = scene;
    a.sensors = sensors_dev;
    a.frames = frames_dev;
    a.n_frames = n_frames;
    a.prefix = tile_prefix_dev;
    a.n_tiles = n_tiles;
    a.table = table;
    a.seed = seed;
    a.out = out;
    a.status = status;
    a.work_counter = work_counter;
    a.tile_rays = cfg.tile_rays;
    a.wc = count ? *count : WorkCount{nullptr, nullptr, nullptr, nullptr};
    a.n_total = n_beams_total;
    a.wait_ns = cfg.wait_ns;
    if (inline_frames) a.inl = *inline_frames;  // else n == 0: the device table
    const bool clean = region && region->clean;
    cudaError_t* refused = region ? region->overlap_refused : nullptr;
    if (region) {
        a.zero_next = region->zero_next;
        a.zero_words = region->zero_next ? region->zero_words : 0;
        a.pdl = region->overlap ? 1 : 0;
    }
    if (compact_scratch) {
        const int64_t nt = (n_beams_total + kCompactTileBeams - 1) / kCompactTileBeams;
        a.cc.n_tiles = nt;
        a.cc.offsets = (int64_t*)compact_scratch;
        a.cc.counts = region ? region->base : (unsigned*)((char*)compact_scratch + ((nt * 8 + 255) / 256) * 256);
        a.cc.done = a.cc.counts + nt;
        a.cc.total = n_points_dev;
        // the work counter sits behind the tile counts: one memset clears all
        const size_t wc_off = compact_counter_offset(nt);
        a.work_counter = (unsigned long long*)((char*)a.cc.counts + wc_off);
        if (!clean) cudaMemsetAsync(a.cc.counts, 0, wc_off + sizeof(unsigned long long), s);
        // an overlapped cast compacts in the scatter kernel that follows it (a
        // cooperative grid could not start before the cast ahead of it ends)
        if (points && cfg.fused_scatter && !(region && region->overlap)) {
            a.pts = *points;
            a.fused = 1;
        }
    } else if (region) {
        a.work_counter = (unsigned long long*)region->base;
        if (!clean) cudaMemsetAsync(a.work_counter, 0, sizeof(unsigned long long), s);
    } else {
        cudaMemsetAsync(work_counter, 0, sizeof(unsigned long long), s);
    }
    // dynamic shared memory: the per-lane traversals keep kSharedStack stack
    // entries per thread there; the warp-synchronous one uses none.  It
    // follows the instantiated variant W, not the configuration, because the
    // counting launch always uses a per-lane traversal.
    const size_t stack_bytes = (size_t)kSharedStack * cfg.block_threads * sizeof(int2);
    const int bt = cfg.block_threads;
    cudaError_t e;
    if (count) {
        // the work counted depends on the tree the traversal walks, not on the launch shape
        a.fused = 0;
        e = cfg.traversal == 3   ? launch_one<true, 4, 3>(s, a, grid, bt, stack_bytes, num_sms, refused)
            : cfg.traversal == 2 ? launch_one<true, 4, 2>(s, a, grid, bt, stack_bytes, num_sms, refused)
                                 : launch_one<true, 4, 0>(s, a, grid, bt, stack_bytes, num_sms, refused);
    } else if (cfg.traversal == 1) {
        e = variant == 2   ? launch_one<false, 2, 1>(s, a, grid, bt, 0, num_sms, refused)
            : variant == 3 ? launch_one<false, 3, 1>(s, a, grid, bt, 0, num_sms, refused)
                           : launch_one<false, 4, 1>(s, a, grid, bt, 0, num_sms, refused);
    } else if (cfg.traversal == 2) {
        e = variant == 2   ? launch_one<false, 2, 2>(s, a, grid, bt, stack_bytes, num_sms, refused)
            : variant == 3 ? launch_one<false, 3, 2>(s, a, grid, bt, stack_bytes, num_sms, refused)
                           : launch_one<false, 4, 2>(s, a, grid, bt, stack_bytes, num_sms, refused);
    } else if (cfg.traversal == 3) {
        e = variant == 2   ? launch_one<false, 2, 3>(s, a, grid, bt, stack_bytes, num_sms, refused)
            : variant == 3 ? launch_one<false, 3, 3>(s, a, grid, bt, stack_bytes, num_sms, refused)
                           : launch_one<false, 4, 3>(s, a, grid, bt, stack_bytes, num_sms, refused);
    } else {
        e = variant == 2   ? launch_one<false, 2, 0>(s, a, grid, bt, stack_bytes, num_sms, refused)
            : variant == 3 ? launch_one<false, 3, 0>(s, a, grid, bt, stack_bytes, num_sms, refused)
                           : launch_one<false, 4, 0>(s, a, grid, bt, stack_bytes, num_sms, refused);
    }
    if (e == cudaSuccess && scattered) *scattered = a.fused != 0;
    return e;
}

namespace {
__global__ void k_popcount(const uint32_t* __restrict__ bits, int64_t n_words, unsigned long long* total)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += (int64_t)gridDim.x * blockDim.x)
        c += __popc(bits[i]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, c);
}
}  // namespace

namespace {
__global__ void k_set_poses(FrameDev* frames, int n_frames, const float* __restrict__ poses)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_frames * 12) return;
    frames[i / 12].pose[i % 12] = poses[i];
}
}  // namespace

cudaError_t launch_set_poses(cudaStream_t s, FrameDev* frames, int n_frames, const float* poses)
{
    if (n_frames <= 0) return cudaSuccess;
    k_set_poses<<<(n_frames * 12 + 255) / 256, 256, 0, s>>>(frames, n_frames, poses);
    return cudaGetLastError();
}

cudaError_t launch_popcount(cudaStream_t s, const uint32_t* bits, int64_t n_words, unsigned long long* total)
{
    if (n_words == 0) return cudaSuccess;
    k_popcount<<<256, 256, 0, s>>>(bits, n_words, total);
    return cudaGetLastError();
}

size_t cast_counter_bytes(int64_t n_total, bool compact)
{
    if (!compact) return sizeof(unsigned long long);
    return compact_counter_offset((n_total + kCompactTileBeams - 1) / kCompactTileBeams) + sizeof(unsigned long long);
}

size_t fused_compact_scratch_bytes(int64_t n)
{
    const int64_t nt = (n + kCompactTileBeams - 1) / kCompactTileBeams;
    return ((nt * 8 + 255) / 256) * 256 + ((compact_counter_offset(nt) + 8 + 255) / 256) * 256;
}

cudaError_t launch_scatter(cudaStream_t s, const SensorDev* sensors_dev, const FrameDev* frames_dev, int n_frames,
                           int64_t n, BeamsOut dense, const lidar_points& pts, void* compact_scratch, int* status,
                           const InlineFrames* inline_frames, int num_sms, bool pdl)
{
    const int64_t tiles = (n + kCompactTile - 1) / kCompactTile;
    if (tiles == 0) return cudaSuccess;
    InlineFrames inl{};
    if (inline_frames) inl = *inline_frames;
    const int64_t* offsets = (const int64_t*)compact_scratch;
    int flag = 0;
    if (pdl && num_sms > 0) {
        // an overlapped cast's scatter: a small grid that lets the next cast
        // start at once and then waits for its own cast.  Its blocks must become
        // resident beside the running cast's (two 256-thread blocks of ~112
        // registers leave 8,192 registers of an SM free), or the next cast
        // could not start before the cast's blocks exit: one 64-thread block
        // per SM at ~80 registers
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)std::min<int64_t>(tiles, num_sms));
        lc.blockDim = dim3(kPdlScatterThreads);
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        flag = 1;
        void* args[] = {&sensors_dev, &frames_dev, &n_frames, &n, &dense, &offsets, (void*)&pts, &status, &inl, &flag};
        if (cudaLaunchKernelExC(&lc, (const void*)k_scatter_points<kScatterItems>, args) == cudaSuccess)
            return cudaSuccess;
        cudaGetLastError();
        flag = 0;
    }
    k_scatter_points<kScatterItems><<<(unsigned)tiles, kCompactThreads, 0, s>>>(sensors_dev, frames_dev, n_frames, n,
                                                                                dense, offsets, pts, status, inl, flag);
    return cudaGetLastError();
}

namespace {
constexpr int kScheduleGroup = 32;

__global__ void k_group_cost(const uint32_t* __restrict__ cost, const uint32_t* __restrict__ order, int n,
                             uint32_t* keys, uint32_t* vals)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_groups = (n + kScheduleGroup - 1) / kScheduleGroup;
    if (g >= n_groups) return;
    const int lo = g * kScheduleGroup, hi = min(n, lo + kScheduleGroup);
    uint32_t mx = 0;
    for (int j = lo; j < hi; ++j) mx = max(mx, cost[order[j]]);
    // ascending sort of ~cost runs the most expensive group first (ties keep the
    // base order); a partial group sorts last so every other group stays whole
    keys[g] = (hi - lo < kScheduleGroup) ? 0xFFFFFFFFu : ~min(mx, 0xFFFFFFFEu);
    vals[g] = (uint32_t)g;
}

__global__ void k_permute_groups(const uint32_t* __restrict__ groups, const uint32_t* __restrict__ base, int n,
                                 uint32_t* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // output position
    if (i >= n) return;
    const int g = (int)groups[i / kScheduleGroup];
    out[i] = base[g * kScheduleGroup + (i % kScheduleGroup)];
}
}  // namespace

size_t cost_schedule_scratch_bytes(int64_t n)
{
    const int64_t g = (n + kScheduleGroup - 1) / kScheduleGroup;
    return ((g * 4 + 255) / 256) * 256 * 2 + radix_sort_scratch_bytes(g);
}

namespace {
// key of beam at base-order position p: cost bucket (4 per octave, most
// expensive first) above the base position, so equal buckets keep the
// base (Morton) order
__global__ void k_bucket_keys(const uint32_t* __restrict__ cost, const uint32_t* __restrict__ base, int n,
                              uint64_t* keys, uint32_t* vals)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t b = base[p];
    const uint32_t bucket = (uint32_t)(4.0f * log2f((float)cost[b] + 1.0f));
    keys[p] = ((uint64_t)(63u - min(bucket, 63u)) << 32) | (uint64_t)p;
    vals[p] = b;
}
}  // namespace

size_t bucket_schedule_scratch_bytes(int64_t n)
{
    return ((n * 8 + 255) / 256) * 256 + radix_sort_scratch_bytes(n);
}

cudaError_t launch_bucket_schedule(cudaStream_t s, const uint32_t* cost, const uint32_t* base_order, int n,
                                   uint32_t* new_order, void* scratch, size_t scratch_bytes)
{
    if (n == 0) return cudaSuccess;
    if (scratch_bytes < bucket_schedule_scratch_bytes(n)) return cudaErrorInvalidValue;
    uint64_t* keys = (uint64_t*)scratch;
    char* rest = (char*)scratch + ((n * 8 + 255) / 256) * 256;
    k_bucket_keys<<<(n + 255) / 256, 256, 0, s>>>(cost, base_order, n, keys, new_order);
    return radix_sort_pairs_u64(s, keys, new_order, n, 38, rest, scratch_bytes - (rest - (char*)scratch));
}

cudaError_t launch_cost_schedule(cudaStream_t s, const uint32_t* cost, const uint32_t* base_order, int n,
                                 uint32_t* new_order, void* scratch, size_t scratch_bytes)
{
    if (n == 0) return cudaSuccess;
    if (scratch_bytes < cost_schedule_scratch_bytes(n)) return cudaErrorInvalidValue;
    const int g = (n + kScheduleGroup - 1) / kScheduleGroup;
    uint32_t* keys = (uint32_t*)scratch;
    uint32_t* vals = (uint32_t*)((char*)scratch + ((g * 4 + 255) / 256) * 256);
    char* rest = (char*)scratch + ((g * 4 + 255) / 256) * 256 * 2;
    k_group_cost<<<(g + 255) / 256, 256, 0, s>>>(cost, base_order, n, keys, vals);
    cudaError_t e = radix_sort_pairs_u32(s, keys, vals, g, 32, rest, scratch_bytes - (rest - (char*)scratch));
    if (e != cudaSuccess) return e;
    k_permute_groups<<<(n + 255) / 256, 256, 0, s>>>(vals, base_order, n, new_order);
    return cudaGetLastError();
}

size_t ray_order_scratch_bytes(int64_t n)
{
    return ((n * sizeof(uint32_t) + 255) / 256) * 256 + radix_sort_scratch_bytes(n);
}

cudaError_t launch_ray_order(cudaStream_t s, const float* dirs, int n, uint32_t* order, void* scratch,
                             size_t scratch_bytes)
{
    if (n == 0) return cudaSuccess;
    uint32_t* keys = (uint32_t*)scratch;
    char* rest = (char*)scratch + ((n * sizeof(uint32_t) + 255) / 256) * 256;
    k_dir_keys<<<(n + 255) / 256, 256, 0, s>>>(dirs, n, keys, order);
    return radix_sort_pairs_u32(s, keys, order, n, 32, rest, scratch_bytes - (rest - (char*)scratch));
}

}  // namespace lidar
