// Rolling shutter and multi-echo returns.  A sweep carries the sensor pose at
// its start and at its end; beam b fires at the fraction s_b of the sweep (its
// azimuth over 2 pi) and sees the pose blended between the two (translation
// (1 - s) t0 + s t1; rotation of the normalised blend (1 - s) q0 + s q1 of the
// unit quaternions) — the camera turned with the sensor's spin over the time
// step of Sec. II-A, here per beam.  From the returns of a beam's sub-rays it
// also reports several echoes (Sec. IV: multiple returns are future work):
// mode 0 the n strongest apart by at least `separation` in range, mode 1 the
// first and the last.  Persistent warp tiles like the frame cast's (a beam's
// sub-rays on neighbouring lanes), 4-wide traversal.
#include "common.cuh"
#include "philox.cuh"
#include "trace.cuh"
#include "shade.cuh"

namespace lidar {
namespace {

// pose at fraction s of a sweep, FP32, every operation rounded as written
__device__ __forceinline__ void sweep_pose(const SweepDev& f, float s, float* P)
{
    const float ms = __fsub_rn(1.0f, s);
    float q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = __fmaf_rn(s, f.q1[i], __fmul_rn(ms, f.q0[i]));
    float n2 = __fmul_rn(q[0], q[0]);
    n2 = __fadd_rn(n2, __fmul_rn(q[1], q[1]));
    n2 = __fadd_rn(n2, __fmul_rn(q[2], q[2]));
    n2 = __fadd_rn(n2, __fmul_rn(q[3], q[3]));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    const float w = __fmul_rn(q[0], inv), x = __fmul_rn(q[1], inv), y = __fmul_rn(q[2], inv),
                z = __fmul_rn(q[3], inv);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    P[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    P[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    P[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    P[4] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    P[5] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    P[6] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    P[8] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    P[9] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    P[10] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
#pragma unroll
    for (int r = 0; r < 3; ++r) P[4 * r + 3] = __fmaf_rn(s, f.t1[r], __fmul_rn(ms, f.t0[r]));
}

// The echoes of one beam from its sub-rays' returns (sub_ok: kept), written at
// dense position g.
__device__ __forceinline__ void write_echoes(const EchoOut& echo, int64_t g, int n_sub, const float* sub_range,
                                             const float* sub_I, const uint32_t* sub_tri, const bool* sub_ok)
{
    int pick[4];
    int n = 0;
    if (echo.mode == 0) {
        // strongest first (ties to the lower sub-ray), skipping returns within
        // `separation` in range of one already kept
        bool used[LIDAR_MAX_SUBRAYS];
        for (int k = 0; k < n_sub; ++k) used[k] = false;
        while (n < echo.n_echoes) {
            int b = -1;
            for (int k = 0; k < n_sub; ++k)
                if (sub_ok[k] && !used[k] && (b < 0 || sub_I[k] > sub_I[b])) b = k;
            if (b < 0) break;
            used[b] = true;
            bool apart = true;
            for (int j = 0; j < n; ++j)
                if (fabsf(sub_range[b] - sub_range[pick[j]]) < echo.separation) apart = false;
            if (apart) pick[n++] = b;
        }
    } else {
        // first and last (ties to the lower sub-ray)
        int first = -1, last = -1;
        for (int k = 0; k < n_sub; ++k) {
            if (!sub_ok[k]) continue;
            if (first < 0 || sub_range[k] < sub_range[first]) first = k;
            if (last < 0 || sub_range[k] > sub_range[last]) last = k;
        }
        if (first >= 0) {
            pick[n++] = first;
            if (echo.n_echoes > 1 && sub_range[last] - sub_range[first] >= echo.separation) pick[n++] = last;
        }
    }
    echo.count[g] = (uint8_t)n;
    for (int j = 0; j < echo.n_echoes; ++j) {
        const int64_t e = g * echo.n_echoes + j;
        const bool have = j < n;
        if (echo.range) echo.range[e] = have ? sub_range[pick[j]] : 0.0f;
        if (echo.intensity) echo.intensity[e] = have ? sub_I[pick[j]] : 0.0f;
        if (echo.tri) echo.tri[e] = have ? sub_tri[pick[j]] : LIDAR_NO_HIT;
        if (echo.sub) echo.sub[e] = have ? (uint8_t)pick[j] : (uint8_t)0xFF;
    }
}

// Persistent sweep cast: warps take tiles of `tile_rays` positions of a
// sweep's ray order from the work counter, as the frame cast does, so the
// sensor's ray order and cost schedule apply.  Dense records (the strongest
// return) and, with kEcho, the echoes of each beam's sub-rays.
template <int kMinBlocks, bool kEcho>
__global__ void __launch_bounds__(256, kMinBlocks) k_sweep_tiles(SceneDev S, const SensorDev* __restrict__ sensors,
                                                                 const SweepDev* __restrict__ frames, int n_frames,
                                                                 const int64_t* __restrict__ tile_prefix,
                                                                 int64_t n_tiles, int tile_rays, TableDev T,
                                                                 uint64_t seed, BeamsOut out, EchoOut echo,
                                                                 int* status, unsigned long long* work_counter)
{
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long claimed = 0;
        if (lane == 0) claimed = atomicAdd(work_counter, 1ull);
        const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, claimed, 0);
        if (tile >= n_tiles) break;
        int lo = 0, hi = n_frames - 1;  // last sweep whose first tile is at or before `tile`
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_prefix[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        const SweepDev f = frames[lo];
        const SensorDev& sd = sensors[f.sensor];
        const int64_t base = (tile - tile_prefix[lo]) * tile_rays;
        if (sd.n_sub > 1) {
            // a beam's sub-rays on neighbouring lanes (as in the frame cast): the
            // strongest return is picked across the beam's lanes and written by its
            // lane; the beam's first lane gathers the returns for the echoes
            const int ns = sd.n_sub;
            const int G = 32 / ns;
            const int g = lane / ns, k = lane - g * ns;
            for (int j0 = 0; j0 < tile_rays; j0 += G) {
                const int64_t pos = base + j0 + g;
                const bool active = g < G && j0 + g < tile_rays && pos < sd.n_beams;
                if (!__any_sync(0xffffffffu, active)) break;
                uint32_t beam = 0;
                float P[12];
                float d0 = 0.0f, d1 = 0.0f, d2 = 1.0f, sfrac = 0.0f;
                if (active) {
                    beam = sd.order ? __ldg(&sd.order[pos]) : (uint32_t)pos;
                    sfrac = __ldg(&sd.sweep[beam]);
                    d0 = __ldg(&sd.dirs[3 * (int64_t)beam]);
                    d1 = __ldg(&sd.dirs[3 * (int64_t)beam + 1]);
                    d2 = __ldg(&sd.dirs[3 * (int64_t)beam + 2]);
                }
                sweep_pose(f, sfrac, P);
                RayW r = world_ray(P, d0, d1, d2);
                if (k > 0) subray_dir(r.dx, r.dy, r.dz, sd.alpha[k], sd.beta[k]);
                const RayPre p = prepare_ray(r);
                HitRec h;
                if (active && !trace_closest4<false>(S, p, sd.t_max, h, nullptr, nullptr, 0))
                    raise_status(status, h.leaf == kBadIndex ? ST_BOUNDS : ST_STACK);
                BeamResult res;
                res.valid = 0;
                res.intensity = 0.0f;
                res.range = 0.0f;
                res.tri = LIDAR_NO_HIT;
                if (active)
                    shade(S, h, r, sd, T, seed, beam, (uint32_t)f.frame, (uint32_t)f.sensor, (uint32_t)k, res);
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
                const int64_t gi = f.beam_offset + beam;
                if (active && k == arg) write_beam(out, gi, res, P, k);
                if (kEcho) {
                    float sub_range[LIDAR_MAX_SUBRAYS], sub_I[LIDAR_MAX_SUBRAYS];
                    uint32_t sub_tri[LIDAR_MAX_SUBRAYS];
                    bool sub_ok[LIDAR_MAX_SUBRAYS];
                    for (int m = 0; m < ns; ++m) {
                        const int src = min(g * ns + m, 31);
                        sub_range[m] = __shfl_sync(0xffffffffu, res.range, src);
                        sub_I[m] = __shfl_sync(0xffffffffu, res.intensity, src);
                        sub_tri[m] = __shfl_sync(0xffffffffu, res.tri, src);
                        sub_ok[m] = __shfl_sync(0xffffffffu, res.valid, src) != 0;
                    }
                    if (active && k == 0) write_echoes(echo, gi, ns, sub_range, sub_I, sub_tri, sub_ok);
                }
            }
            continue;
        }
        for (int j0 = 0; j0 < tile_rays; j0 += 32) {
            const int64_t pos = base + j0 + lane;
            const bool active = pos < sd.n_beams;
            if (!__any_sync(0xffffffffu, active)) break;
            if (!active) continue;
            const uint32_t beam = sd.order ? __ldg(&sd.order[pos]) : (uint32_t)pos;
            float P[12];
            sweep_pose(f, __ldg(&sd.sweep[beam]), P);
            const RayW beam_ray = world_ray(P, __ldg(&sd.dirs[3 * (int64_t)beam]),
                                            __ldg(&sd.dirs[3 * (int64_t)beam + 1]),
                                            __ldg(&sd.dirs[3 * (int64_t)beam + 2]));
            float sub_range[kEcho ? LIDAR_MAX_SUBRAYS : 1], sub_I[kEcho ? LIDAR_MAX_SUBRAYS : 1];
            uint32_t sub_tri[kEcho ? LIDAR_MAX_SUBRAYS : 1];
            bool sub_ok[kEcho ? LIDAR_MAX_SUBRAYS : 1];
            BeamResult best;
            int best_sub = 0;
            float best_I = -1.0f;
            for (int k = 0; k < sd.n_sub; ++k) {
                RayW r = beam_ray;
                if (k > 0) subray_dir(r.dx, r.dy, r.dz, sd.alpha[k], sd.beta[k]);
                const RayPre p = prepare_ray(r);
                HitRec h;
                if (!trace_closest4<false>(S, p, sd.t_max, h, nullptr, nullptr, 0))
                    raise_status(status, h.leaf == kBadIndex ? ST_BOUNDS : ST_STACK);
                BeamResult res;
                shade(S, h, r, sd, T, seed, beam, (uint32_t)f.frame, (uint32_t)f.sensor, (uint32_t)k, res);
                if (kEcho) {
                    sub_range[k] = res.range;
                    sub_I[k] = res.intensity;
                    sub_tri[k] = res.tri;
                    sub_ok[k] = res.valid != 0;
                }
                if (k == 0) best = res;
                if (res.valid && res.intensity > best_I) {
                    best_I = res.intensity;
                    best = res;
                    best_sub = k;
                }
            }
            const int64_t g = f.beam_offset + beam;
            write_beam(out, g, best, P, best_sub);
            if (kEcho) write_echoes(echo, g, sd.n_sub, sub_range, sub_I, sub_tri, sub_ok);
        }
    }
}

}  // namespace

cudaError_t launch_sweep_tiles(cudaStream_t s, const SceneDev& S, const SensorDev* sensors_dev,
                               const SweepDev* frames_dev, int n_frames, const int64_t* tile_prefix_dev,
                               int64_t n_tiles, TableDev T, uint64_t seed, BeamsOut out, EchoOut echo, int* status,
                               unsigned long long* work_counter, const LaunchCfg& cfg, int num_sms)
{
    if (n_tiles == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(work_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t warps = cfg.block_threads / 32;
    int64_t grid = (int64_t)num_sms * cfg.blocks_per_sm;
    if (grid > (n_tiles + warps - 1) / warps) grid = (n_tiles + warps - 1) / warps;
    const int resident = cfg.block_threads * cfg.blocks_per_sm;
    const int bt = cfg.block_threads;
    const dim3 gd((unsigned)grid);
#define LIDAR_SWEEP_LAUNCH(MB, EC)                                                                              \
    k_sweep_tiles<MB, EC><<<gd, bt, 0, s>>>(S, sensors_dev, frames_dev, n_frames, tile_prefix_dev, n_tiles,     \
                                            cfg.tile_rays, T, seed, out, echo, status, work_counter)
    const bool ec = echo.n_echoes > 0;
    if (resident <= 512) {
        if (ec) LIDAR_SWEEP_LAUNCH(2, true); else LIDAR_SWEEP_LAUNCH(2, false);
    } else if (resident <= 768) {
        if (ec) LIDAR_SWEEP_LAUNCH(3, true); else LIDAR_SWEEP_LAUNCH(3, false);
    } else {
        if (ec) LIDAR_SWEEP_LAUNCH(4, true); else LIDAR_SWEEP_LAUNCH(4, false);
    }
#undef LIDAR_SWEEP_LAUNCH
    return cudaGetLastError();
}

}  // namespace lidar
