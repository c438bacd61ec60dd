// Reflectance tables from material parameters, and the adjoint of the
// intensity with respect to the tables and the gain (hits and masks held
// fixed from the forward pass).
//
// Table (Eq. 4's Lambertian law R(theta) = R(0) cos(theta) with R(0) = a, plus
// a specular lobe): T[m][k] = a cos(k deg) + s exp(-k^2 / (2 w^2)), k = 0..90.
//
// Adjoint accumulation is deterministic: every contribution is converted to a
// 64-bit fixed-point integer with a per-call power-of-two scale (chosen from
// the largest contribution, so the sum cannot overflow) and summed with
// integer atomics, first in a block-private shared-memory copy of the
// gradient, then into a global copy; integer addition is associative, so the
// result does not depend on scheduling.
#include "common.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace lidar {
namespace {

constexpr int kAdjThreads = 256;

__global__ void k_build_tables(const float* __restrict__ params, int M, float* __restrict__ table)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * LIDAR_TABLE_SIZE) return;
    const int m = e / LIDAR_TABLE_SIZE, k = e % LIDAR_TABLE_SIZE;
    const float a = params[3 * m], s = params[3 * m + 1], w = params[3 * m + 2];
    const float kf = (float)k;
    table[e] = a * cospif(kf / 180.0f) + s * expf(-(kf * kf) / (2.0f * w * w));
}

// one warp per material; fixed-order reduction over the 91 entries
__global__ void k_build_tables_backward(const float* __restrict__ params, const float* __restrict__ grad_table,
                                        int M, float* __restrict__ grad_params)
{
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= M) return;
    const float s = params[3 * m + 1], w = params[3 * m + 2];
    double ga = 0.0, gs = 0.0, gw = 0.0;
    for (int k = lane; k < LIDAR_TABLE_SIZE; k += 32) {
        const float kf = (float)k;
        const double g = grad_table[m * LIDAR_TABLE_SIZE + k];
        const double e = (double)expf(-(kf * kf) / (2.0f * w * w));
        ga += g * (double)cospif(kf / 180.0f);
        gs += g * e;
        gw += g * (double)s * e * (double)(kf * kf) / ((double)w * w * w);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ga += __shfl_down_sync(0xffffffffu, ga, o);
        gs += __shfl_down_sync(0xffffffffu, gs, o);
        gw += __shfl_down_sync(0xffffffffu, gw, o);
    }
    if (lane == 0) {
        grad_params[3 * m + 0] = (float)ga;
        grad_params[3 * m + 1] = (float)gs;
        grad_params[3 * m + 2] = (float)gw;
    }
}

struct TapeRow {
    bool use;
    int m, i;
    float f, R, rf, gI;  // gI: dL/dI (unnormalised for the MSE variant: 2 (I - I*))
    float res;           // residual I - I* (MSE variant)
};

// Beams per lane per step: a warp takes kAdjPerLane x 32 consecutive beams and
// all of a step's tape loads are in flight before the first is used.  With
// aligned tape arrays (kVec) lane l takes the consecutive beams base + 4 l + j
// through one vector load per array (neighbouring beams often share a table
// bin, which the lane then updates once); otherwise the beams base + 32 j + l
// with scalar loads.  Either way every load instruction is coalesced.
constexpr int kAdjPerLane = 4;

struct TapeIn {
    uint8_t valid[kAdjPerLane], tvalid[kAdjPerLane];
    uint16_t mat[kAdjPerLane];
    float theta[kAdjPerLane], rf[kAdjPerLane], g[kAdjPerLane];  // g: target I (MSE) or dL/dI
};

// kLast: the tape's last read in this call (streaming loads); the first pass
// reads through the cache so the second can find the tape in L2
template <bool kLast, bool kVec>
__device__ __forceinline__ void load_tape(int64_t base, int lane, int64_t n, const uint8_t* valid,
                                          const uint16_t* mat, const float* theta_deg, const float* rf,
                                          const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                          TapeIn& in)
{
    const float* g = target_I ? target_I : grad_I;
    auto ld = [](const auto* p) { return kLast ? __ldcs(p) : __ldg(p); };
    if (kVec && base + 4 * lane + 3 < n) {
        const int64_t b = base + 4 * lane;
        const uchar4 v = ld(reinterpret_cast<const uchar4*>(valid + b));
        const uchar4 tv = target_valid ? ld(reinterpret_cast<const uchar4*>(target_valid + b)) : make_uchar4(1, 1, 1, 1);
        const ushort4 m = ld(reinterpret_cast<const ushort4*>(mat + b));
        const float4 th = ld(reinterpret_cast<const float4*>(theta_deg + b));
        const float4 r = ld(reinterpret_cast<const float4*>(rf + b));
        const float4 gg = ld(reinterpret_cast<const float4*>(g + b));
        in.valid[0] = v.x; in.valid[1] = v.y; in.valid[2] = v.z; in.valid[3] = v.w;
        in.tvalid[0] = tv.x; in.tvalid[1] = tv.y; in.tvalid[2] = tv.z; in.tvalid[3] = tv.w;
        in.mat[0] = m.x; in.mat[1] = m.y; in.mat[2] = m.z; in.mat[3] = m.w;
        in.theta[0] = th.x; in.theta[1] = th.y; in.theta[2] = th.z; in.theta[3] = th.w;
        in.rf[0] = r.x; in.rf[1] = r.y; in.rf[2] = r.z; in.rf[3] = r.w;
        in.g[0] = gg.x; in.g[1] = gg.y; in.g[2] = gg.z; in.g[3] = gg.w;
        return;
    }
#pragma unroll
    for (int j = 0; j < kAdjPerLane; ++j) {
        const int64_t b = kVec ? base + 4 * lane + j : base + j * 32 + lane;
        const bool ok = b < n;
        in.valid[j] = ok ? ld(&valid[b]) : (uint8_t)0;
        in.tvalid[j] = (ok && target_valid) ? ld(&target_valid[b]) : (uint8_t)1;
        in.mat[j] = ok ? ld(&mat[b]) : (uint16_t)0;
        in.theta[j] = ok ? ld(&theta_deg[b]) : 0.0f;
        in.rf[j] = ok ? ld(&rf[b]) : 0.0f;
        in.g[j] = ok ? ld(&g[b]) : 0.0f;
    }
}

__device__ __forceinline__ TapeRow tape_row(const TapeIn& in, int j, TableDev T, float gain, bool mse)
{
    TapeRow r;
    r.use = in.valid[j] != 0 && in.tvalid[j] != 0;
    if (!r.use) return r;
    const int m = in.mat[j] < T.n_mat ? in.mat[j] : T.n_mat - 1;
    const float th = in.theta[j];
    int i = (int)th;
    if (i > LIDAR_TABLE_SIZE - 2) i = LIDAR_TABLE_SIZE - 2;
    const float f = th - (float)i;
    const float* row = T.table + (int64_t)m * LIDAR_TABLE_SIZE;
    const float R = __ldg(&row[i]) * (1.0f - f) + __ldg(&row[i + 1]) * f;
    r.m = m;
    r.i = i;
    r.f = f;
    r.R = R;
    r.rf = in.rf[j];
    if (mse) {
        r.res = gain * R * r.rf - in.g[j];
        r.gI = 2.0f * r.res;
    } else {
        r.res = 0.0f;
        r.gI = in.g[j];
    }
    return r;
}

// pass 1: largest |contribution| bound and the count of used beams
template <bool kVec>
__global__ void __launch_bounds__(kAdjThreads) k_adj_absmax(int64_t n, const uint8_t* __restrict__ valid,
                                                            const uint16_t* __restrict__ mat,
                                                            const float* __restrict__ theta_deg,
                                                            const float* __restrict__ rf, TableDev T, float gain,
                                                            const float* __restrict__ grad_I,
                                                            const float* __restrict__ target_I,
                                                            const uint8_t* __restrict__ target_valid,
                                                            unsigned int* absmax_bits,
                                                            unsigned long long* count)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool mse = target_I != nullptr;
    float mx = 0.0f;
    unsigned long long c = 0;
    for (int64_t base = warp * (32 * kAdjPerLane); base < n; base += n_warps * (32 * kAdjPerLane)) {
        TapeIn in;
        load_tape<false, kVec>(base, lane, n, valid, mat, theta_deg, rf, grad_I, target_I, target_valid, in);
#pragma unroll
        for (int j = 0; j < kAdjPerLane; ++j) {
            const TapeRow r = tape_row(in, j, T, gain, mse);
            if (!r.use) continue;
            ++c;
            const float wt = fmaxf(fabsf(gain * r.rf), fabsf(r.rf * r.R));
            mx = fmaxf(mx, fabsf(r.gI) * wt);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        atomicMax(absmax_bits, __float_as_uint(mx));  // non-negative floats order like their bits
        if (c) atomicAdd(count, c);
    }
}

// power-of-two scale so that n_used * max|term| * scale < 2^62
__device__ __forceinline__ float fixed_scale(unsigned int absmax_bits, unsigned long long count)
{
    const float mx = __uint_as_float(absmax_bits);
    if (!(mx > 0.0f) || count == 0) return 1.0f;
    const double bound = (double)mx * (double)(count + 1);
    int e;
    frexp(bound, &e);            // bound < 2^e
    int sh = 61 - e;
    if (sh > 126) sh = 126;
    if (sh < -126) sh = -126;
    return ldexpf(1.0f, sh);
}

__device__ __forceinline__ long long to_fixed(float v, float scale)
{
    return __float2ll_rn(v * scale);
}

// pass 2: fixed-point accumulation; per-block shared copy when it fits.  The
// gain's term goes to one accumulator for every beam, so each lane sums its
// own terms and each warp adds one total; a lane adds the terms of its
// consecutive beams that share a table bin before updating it (integer sums:
// the order is free).
template <bool kVec>
__global__ void __launch_bounds__(kAdjThreads) k_adj_accumulate(
    int64_t n, const uint8_t* __restrict__ valid, const uint16_t* __restrict__ mat,
    const float* __restrict__ theta_deg, const float* __restrict__ rf, TableDev T, float gain,
    const float* __restrict__ grad_I, const float* __restrict__ target_I, const uint8_t* __restrict__ target_valid,
    const unsigned int* __restrict__ absmax_bits, const unsigned long long* __restrict__ count,
    unsigned long long* acc, double* loss_partials, int use_shared)
{
    extern __shared__ unsigned long long s_acc[];
    const int n_acc = T.n_mat * LIDAR_TABLE_SIZE + 1;  // table entries + gain
    if (use_shared)
        for (int j = threadIdx.x; j < n_acc; j += blockDim.x) s_acc[j] = 0ull;
    __syncthreads();
    unsigned long long* dst = use_shared ? s_acc : acc;
    const float scale = fixed_scale(*absmax_bits, *count);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool mse = target_I != nullptr;
    float loss32 = 0.0f;  // this lane's squared residuals, in its fixed order (FP64 is slow here)
    unsigned long long g_gain = 0;
    for (int64_t base = warp * (32 * kAdjPerLane); base < n; base += n_warps * (32 * kAdjPerLane)) {
        TapeIn in;
        load_tape<true, kVec>(base, lane, n, valid, mat, theta_deg, rf, grad_I, target_I, target_valid, in);
        int cur = -1;
        unsigned long long a0 = 0, a1 = 0;
#pragma unroll
        for (int j = 0; j < kAdjPerLane; ++j) {
            const TapeRow r = tape_row(in, j, T, gain, mse);
            if (!r.use) continue;
            const float w = gain * r.rf * r.gI;
            const int e = r.m * LIDAR_TABLE_SIZE + r.i;
            const unsigned long long lo = (unsigned long long)to_fixed(w * (1.0f - r.f), scale);
            const unsigned long long hi = (unsigned long long)to_fixed(w * r.f, scale);
            if (e != cur) {
                if (cur >= 0) {
                    atomicAdd(&dst[cur], a0);
                    atomicAdd(&dst[cur + 1], a1);
                }
                cur = e;
                a0 = 0;
                a1 = 0;
            }
            a0 += lo;
            a1 += hi;
            g_gain += (unsigned long long)to_fixed(r.rf * r.R * r.gI, scale);
            loss32 = __fmaf_rn(r.res, r.res, loss32);
        }
        if (cur >= 0) {
            atomicAdd(&dst[cur], a0);
            atomicAdd(&dst[cur + 1], a1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) g_gain += __shfl_down_sync(0xffffffffu, g_gain, o);
    if (lane == 0 && g_gain) atomicAdd(&dst[n_acc - 1], g_gain);
    // deterministic per-block loss partial (fixed shuffle order)
    double loss = (double)loss32;
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    __shared__ double s_loss[kAdjThreads / 32];
    if (lane == 0) s_loss[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) t += s_loss[w];
        loss_partials[blockIdx.x] = t;
    }
    if (use_shared)
        for (int j = threadIdx.x; j < n_acc; j += blockDim.x)
            if (s_acc[j]) atomicAdd(&acc[j], s_acc[j]);
}

// pass 3: back to floating point, normalised, accumulated into the outputs;
// block 0 also sums the loss partials in a fixed tree order
constexpr int kFinalizeThreads = 256;
__global__ void __launch_bounds__(kFinalizeThreads) k_adj_finalize(
    int n_acc, const unsigned long long* __restrict__ acc, const unsigned int* __restrict__ absmax_bits,
    const unsigned long long* __restrict__ count, int mse, const double* __restrict__ loss_partials, int n_partials,
    float* grad_table, float* grad_gain, float* loss)
{
    const float scale = fixed_scale(*absmax_bits, *count);
    const float inv_scale = __frcp_rn(scale);  // exact: the scale is a power of two
    const unsigned long long N = *count;
    // FP32 (FP64 is slow on this part): the integer sum rounded once to 24
    // bits, an exact scaling, one rounded normalisation
    const float norm = mse ? (N ? __frcp_rn((float)N) : 0.0f) : 1.0f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_acc; j += gridDim.x * blockDim.x) {
        const float v = __fmul_rn(__fmul_rn(__ll2float_rn((long long)acc[j]), inv_scale), norm);
        if (j < n_acc - 1) {
            if (grad_table) grad_table[j] += v;
        } else if (grad_gain) {
            *grad_gain += v;
        }
    }
    if (blockIdx.x == 0 && loss) {
        __shared__ double s_part[kFinalizeThreads];
        double t = 0.0;
        for (int k = threadIdx.x; k < n_partials; k += kFinalizeThreads) t += loss_partials[k];
        s_part[threadIdx.x] = t;
        __syncthreads();
        for (int w = kFinalizeThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) s_part[threadIdx.x] += s_part[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) *loss = mse ? (float)(N ? s_part[0] / (double)N : 0.0) : 0.0f;
    }
}

constexpr int kAdjBlocks = 1024;

// ------------------------------------------------------------ one-pass adjoint
//
// The same sums as the passes above with the tape read once.  One block per
// SM (cooperative launch) owns a contiguous run of chunks of kOneChunk beams.
// Its chunks stream into shared memory by bulk asynchronous copies (TMA,
// cp.async.bulk) kOneStages deep, completion tracked by one mbarrier per
// stage; with tape arrays the copy engine cannot address (not 16-byte
// aligned) and for the tape's last, partial chunk the threads load the beams
// themselves.  The block sums its contributions exactly in 64-bit fixed point
// in shared memory at its own power-of-two scale, chosen from the largest
// contribution seen so far and the block's beam count; when a chunk raises
// that maximum past the scale's headroom, the accumulators are rescaled
// (a rounding shift) before the chunk is added.  After one bounded grid-wide
// wait every block knows every block's maximum, converts its sums to the
// common scale of the whole tape (a rounding shift) and adds them into the
// global accumulators with integer atomics; the last block to finish turns
// them into the gradients and sums the per-block loss partials in block
// order.  Every step is a deterministic function of the tape and the grid
// size, so the result is bit-reproducible run to run.

constexpr int kOneThreads = 512;
constexpr int kOneBPT = 4;                          // consecutive beams per thread per chunk
constexpr int kOneChunk = kOneThreads * kOneBPT;    // 2048 beams
constexpr int kOneStages = 4;
constexpr int kOneStageBytes = kOneChunk * 16;      // valid 1, target valid 1, mat 2, theta 4, rf 4, g 4
constexpr int kOneWarps = kOneThreads / 32;

struct OneArgs {
    int64_t n;
    const uint8_t* valid;
    const uint16_t* mat;
    const float* theta;
    const float* rf;
    const float* g;             // target intensities (MSE) or dL/dI
    const uint8_t* tvalid;      // target valid flags, NULL: all valid
    TableDev T;
    float gain;
    int mse;
    int n_acc;                  // table entries + the gain
    unsigned long long* acc;    // [n_acc] global accumulators, cleared in the kernel
    float* blk_max;             // [grid] per block: largest contribution
    int* blk_sh;                // [grid] its fixed-point shift
    double* blk_loss;           // [grid] sum of squared residuals
    unsigned long long* blk_n;  // [grid] beams used
    unsigned* ctl;              // [0] grid-wait arrivals, [1] finished blocks; 0 between calls
    int* status;
    uint64_t wait_ns;
    float* loss;
    float* grad_table;
    float* grad_gain;
};

__device__ __forceinline__ uint64_t adj_global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// fixed-point shift for sums of up to `count` terms of magnitude <= m: every
// partial sum stays below 2^61 (m < 2^em, count + 1 <= 2^ec)
__device__ __forceinline__ int one_shift(float m, int64_t count)
{
    int em;
    frexpf(m, &em);
    const int ec = 64 - __clzll((long long)(count + 1));
    int sh = 61 - em - ec;
    return sh > 126 ? 126 : (sh < -126 ? -126 : sh);
}

// v / 2^d rounded to nearest (ties up), d >= 0
__device__ __forceinline__ long long round_shift(long long v, int d)
{
    if (d == 0) return v;
    if (d > 62) return 0;
    return (v + (1ll << (d - 1))) >> d;
}

__device__ __forceinline__ void bar_init(uint64_t* bar)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
}

__device__ __forceinline__ void bar_expect(uint64_t* bar, unsigned bytes)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// waits for the stage's phase `parity` to complete; false after wait_ns
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity, uint64_t wait_ns)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    uint64_t t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it == 0) t0 = adj_global_ns();
        else if (adj_global_ns() - t0 > wait_ns) return false;
    }
}

template <bool kTma>
__global__ void __launch_bounds__(kOneThreads, 1) k_adj_onepass(const __grid_constant__ OneArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stages = smem;
    unsigned long long* s_acc = (unsigned long long*)(smem + (kTma ? kOneStages * kOneStageBytes : 0));
    uint64_t* s_bar = (uint64_t*)(s_acc + ((a.n_acc + 1) & ~1));
    __shared__ float s_wmax[2][kOneWarps];
    __shared__ double s_red[kOneWarps];
    __shared__ unsigned long long s_cnt[kOneWarps];
    __shared__ int s_flag;
    __shared__ float s_gmax;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, blk = blockIdx.x;
    const int64_t n = a.n;
    const int64_t n_chunks = (n + kOneChunk - 1) / kOneChunk;
    const int64_t k0 = (int64_t)blk * n_chunks / G, k1 = ((int64_t)blk + 1) * n_chunks / G;
    const int64_t first = k0 * kOneChunk;
    const int64_t last = min(k1 * kOneChunk, n);
    const int64_t L = last > first ? last - first : 0;   // beams of this block
    const bool has_tv = a.tvalid != nullptr;

    for (int j = tid; j < a.n_acc; j += kOneThreads) s_acc[j] = 0ull;
    for (int64_t j = (int64_t)blk * kOneThreads + tid; j < a.n_acc; j += (int64_t)G * kOneThreads) a.acc[j] = 0ull;
    if (kTma && tid == 0) {
        for (int st = 0; st < kOneStages; ++st) bar_init(&s_bar[st]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // a chunk is copied by the copy engine iff it is whole (the tape's last
    // chunk may be partial: its byte counts need not be multiples of 16)
    auto whole = [&](int64_t k) { return (k + 1) * (int64_t)kOneChunk <= n; };
    auto issue = [&](int64_t k) {
        const int slot = (int)((k - k0) % kOneStages);
        unsigned char* d = stages + slot * kOneStageBytes;
        const int64_t c0 = k * kOneChunk;
        const unsigned bytes = kOneChunk * (has_tv ? 16u : 15u);
        bar_expect(&s_bar[slot], bytes);
        bulk_copy(d, a.valid + c0, kOneChunk, &s_bar[slot]);
        if (has_tv) bulk_copy(d + kOneChunk, a.tvalid + c0, kOneChunk, &s_bar[slot]);
        bulk_copy(d + 2 * kOneChunk, a.mat + c0, 2 * kOneChunk, &s_bar[slot]);
        bulk_copy(d + 4 * kOneChunk, a.theta + c0, 4 * kOneChunk, &s_bar[slot]);
        bulk_copy(d + 8 * kOneChunk, a.rf + c0, 4 * kOneChunk, &s_bar[slot]);
        bulk_copy(d + 12 * kOneChunk, a.g + c0, 4 * kOneChunk, &s_bar[slot]);
    };
    int64_t issued = k0;  // next chunk to copy (meaningful in thread 0)
    if (kTma && tid == 0)
        for (; issued < k1 && issued < k0 + kOneStages && whole(issued); ++issued) issue(issued);

    float blk_max = 0.0f;
    int sh = 126;
    float loss32 = 0.0f;
    unsigned cnt = 0;
    bool failed = false;
    int64_t k_fail = k1;  // first chunk whose stage wait ran out
    const float* Tt = a.T.table;
    for (int64_t k = k0; k < k1; ++k) {
        const int64_t c0 = k * kOneChunk;
        TapeIn in;
        bool ok = true;
        if (kTma && whole(k)) {
            const int slot = (int)((k - k0) % kOneStages);
            ok = bar_wait(&s_bar[slot], (unsigned)(((k - k0) / kOneStages) & 1), a.wait_ns);
            if (ok) {
                const unsigned char* d = stages + slot * kOneStageBytes;
                const uchar4 v = reinterpret_cast<const uchar4*>(d)[tid];
                const uchar4 tv = has_tv ? reinterpret_cast<const uchar4*>(d + kOneChunk)[tid] : make_uchar4(1, 1, 1, 1);
                const ushort4 m = reinterpret_cast<const ushort4*>(d + 2 * kOneChunk)[tid];
                const float4 th = reinterpret_cast<const float4*>(d + 4 * kOneChunk)[tid];
                const float4 r = reinterpret_cast<const float4*>(d + 8 * kOneChunk)[tid];
                const float4 gg = reinterpret_cast<const float4*>(d + 12 * kOneChunk)[tid];
                in.valid[0] = v.x; in.valid[1] = v.y; in.valid[2] = v.z; in.valid[3] = v.w;
                in.tvalid[0] = tv.x; in.tvalid[1] = tv.y; in.tvalid[2] = tv.z; in.tvalid[3] = tv.w;
                in.mat[0] = m.x; in.mat[1] = m.y; in.mat[2] = m.z; in.mat[3] = m.w;
                in.theta[0] = th.x; in.theta[1] = th.y; in.theta[2] = th.z; in.theta[3] = th.w;
                in.rf[0] = r.x; in.rf[1] = r.y; in.rf[2] = r.z; in.rf[3] = r.w;
                in.g[0] = gg.x; in.g[1] = gg.y; in.g[2] = gg.z; in.g[3] = gg.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kOneBPT; ++j) {
                const int64_t b = c0 + kOneBPT * tid + j;
                const bool inb = b < n;
                in.valid[j] = inb ? __ldcs(&a.valid[b]) : (uint8_t)0;
                in.tvalid[j] = (inb && has_tv) ? __ldcs(&a.tvalid[b]) : (uint8_t)1;
                in.mat[j] = inb ? __ldcs(&a.mat[b]) : (uint16_t)0;
                in.theta[j] = inb ? __ldcs(&a.theta[b]) : 0.0f;
                in.rf[j] = inb ? __ldcs(&a.rf[b]) : 0.0f;
                in.g[j] = inb ? __ldcs(&a.g[b]) : 0.0f;
            }
        }
        float t_lo[kOneBPT], t_hi[kOneBPT], t_g[kOneBPT];
        int e[kOneBPT];
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < kOneBPT; ++j) {
            e[j] = -1;
            t_lo[j] = t_hi[j] = t_g[j] = 0.0f;
            if (!ok) continue;
            const TapeRow r = tape_row(in, j, TableDev{Tt, a.T.n_mat}, a.gain, a.mse != 0);
            if (!r.use) continue;
            const float w = a.gain * r.rf * r.gI;
            e[j] = r.m * LIDAR_TABLE_SIZE + r.i;
            t_lo[j] = w * (1.0f - r.f);
            t_hi[j] = w * r.f;
            t_g[j] = r.rf * r.R * r.gI;
            mx = fmaxf(mx, fmaxf(fabsf(t_g[j]), fmaxf(fabsf(t_lo[j]), fabsf(t_hi[j]))));
            loss32 = __fmaf_rn(r.res, r.res, loss32);
            ++cnt;
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_wmax[k & 1][warp] = mx;
        // every thread has read this chunk's stage and published its maximum
        if (__syncthreads_or(!ok)) {
            failed = true;
            k_fail = k;
            break;
        }
        if (kTma && tid == 0 && issued < k1 && whole(issued)) {
            // the stage just read is free: order the generic reads before the
            // copy engine's writes, then refill it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(issued);
            ++issued;
        }
        float cm = 0.0f;
#pragma unroll
        for (int w = 0; w < kOneWarps; ++w) cm = fmaxf(cm, s_wmax[k & 1][w]);
        if (cm > blk_max) {
            const int nsh = one_shift(cm, L);
            if (nsh < sh && blk_max > 0.0f) {
                const int d = sh - nsh;
                for (int j = tid; j < a.n_acc; j += kOneThreads)
                    s_acc[j] = (unsigned long long)round_shift((long long)s_acc[j], d);
                __syncthreads();
            }
            if (nsh < sh) sh = nsh;
            blk_max = cm;
        }
        if (blk_max > 0.0f) {
            const float scale = ldexpf(1.0f, sh);
            int cur = -1;
            unsigned long long a0 = 0, a1 = 0, gsum = 0;
#pragma unroll
            for (int j = 0; j < kOneBPT; ++j) {
                if (e[j] < 0) continue;
                if (e[j] != cur) {
                    if (cur >= 0) {
                        atomicAdd(&s_acc[cur], a0);
                        atomicAdd(&s_acc[cur + 1], a1);
                    }
                    cur = e[j];
                    a0 = a1 = 0;
                }
                a0 += (unsigned long long)__float2ll_rn(t_lo[j] * scale);
                a1 += (unsigned long long)__float2ll_rn(t_hi[j] * scale);
                gsum += (unsigned long long)__float2ll_rn(t_g[j] * scale);
            }
            if (cur >= 0) {
                atomicAdd(&s_acc[cur], a0);
                atomicAdd(&s_acc[cur + 1], a1);
            }
            for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
            if (lane == 0 && gsum) atomicAdd(&s_acc[a.n_acc - 1], gsum);
        }
    }
    if (failed && kTma && tid == 0) {
        // let the copies still in flight (chunks k_fail .. issued - 1, at most one
        // per stage) land before the block's shared memory goes away; bounded by
        // at least a second whatever the caller's wait limit
        const uint64_t drain_ns = a.wait_ns > 1000000000ull ? a.wait_ns : 1000000000ull;
        for (int64_t k = k_fail; k < issued; ++k) {
            const int slot = (int)((k - k0) % kOneStages);
            bar_wait(&s_bar[slot], (unsigned)(((k - k0) / kOneStages) & 1), drain_ns);
        }
    }
    if (failed && tid == 0) raise_status(a.status, ST_TIMEOUT);

    // ---- this block's loss partial (fixed order), beam count, maximum and shift
    double l = (double)loss32;
    unsigned long long c = cnt;
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_down_sync(0xffffffffu, l, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        s_red[warp] = l;
        s_cnt[warp] = c;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        unsigned long long ct = 0;
        for (int w = 0; w < kOneWarps; ++w) {
            t += s_red[w];
            ct += s_cnt[w];
        }
        a.blk_loss[blk] = t;
        a.blk_n[blk] = ct;
        a.blk_max[blk] = failed ? 0.0f : blk_max;
        a.blk_sh[blk] = sh;
        // ---- grid-wide wait (cooperative launch: every block is resident)
        __threadfence();
        atomicAdd(&a.ctl[0], 1u);
        int okw = 1;
        const uint64_t t0 = adj_global_ns();
        while (*(volatile unsigned*)&a.ctl[0] < (unsigned)G) {
            if (adj_global_ns() - t0 > a.wait_ns) {
                raise_status(a.status, ST_TIMEOUT);
                okw = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_flag = okw;
    }
    __syncthreads();
    if (s_flag && !failed) {
        // the common scale: the largest contribution of the whole tape
        float gm = 0.0f;
        for (int j = tid; j < G; j += kOneThreads) gm = fmaxf(gm, __ldcg(&a.blk_max[j]));
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if (lane == 0) s_wmax[0][warp] = gm;
        __syncthreads();
        if (tid == 0) {
            float t = 0.0f;
            for (int w = 0; w < kOneWarps; ++w) t = fmaxf(t, s_wmax[0][w]);
            s_gmax = t;
        }
        __syncthreads();
        if (blk_max > 0.0f) {
            const int S = one_shift(s_gmax, n);
            const int d = sh - S;
            for (int j = tid; j < a.n_acc; j += kOneThreads) {
                const long long v = round_shift((long long)s_acc[j], d);
                if (v) atomicAdd(&a.acc[j], (unsigned long long)v);
            }
        }
    }
    // ---- the last block to finish writes the results
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = atomicAdd(&a.ctl[1], 1u) == (unsigned)G - 1;
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    if (tid == 0) {
        float gm = 0.0f;
        unsigned long long N = 0;
        for (int j = 0; j < G; ++j) {
            gm = fmaxf(gm, __ldcg(&a.blk_max[j]));
            N += __ldcg(&a.blk_n[j]);
        }
        s_gmax = gm;
        s_cnt[0] = N;
        if (a.loss) {
            double t = 0.0;
            for (int j = 0; j < G; ++j) t += __ldcg(&a.blk_loss[j]);
            *a.loss = a.mse ? (float)(N ? t / (double)N : 0.0) : 0.0f;
        }
    }
    __syncthreads();
    const unsigned long long N = s_cnt[0];
    if (s_gmax > 0.0f) {
        const float inv_scale = ldexpf(1.0f, -one_shift(s_gmax, n));  // exact: a power of two
        const float norm = a.mse ? (N ? __frcp_rn((float)N) : 0.0f) : 1.0f;
        for (int j = tid; j < a.n_acc; j += kOneThreads) {
            const float v = __fmul_rn(__fmul_rn(__ll2float_rn((long long)__ldcg(&a.acc[j])), inv_scale), norm);
            if (j < a.n_acc - 1) {
                if (a.grad_table) a.grad_table[j] += v;
            } else if (a.grad_gain) {
                *a.grad_gain += v;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        // every block has passed the grid wait and counted itself: ready for the next call
        a.ctl[0] = 0u;
        a.ctl[1] = 0u;
    }
}

}  // namespace

// Scratch of the allocation-free backward variant: a file-scope device array
// sized for kNoAllocMaxMaterials table rows (every device that loads the
// library holds it until the process exits).
constexpr int kNoAllocMaxMaterials = LIDAR_NOALLOC_MAX_MATERIALS;
constexpr size_t kNoAllocScratchBytes =
    256 + (((size_t)kNoAllocMaxMaterials * LIDAR_TABLE_SIZE + 1) * 8 + 255) / 256 * 256 + kAdjBlocks * sizeof(double);
static_assert(kNoAllocScratchBytes == LIDAR_NOALLOC_SCRATCH_BYTES, "lidar.h states the scratch size");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

cudaError_t noalloc_scratch(void** ptr, size_t* bytes)
{
    // cudaGetSymbolAddress resolves the array on the current device
    cudaError_t e = cudaGetSymbolAddress(ptr, g_noalloc_scratch);
    *bytes = kNoAllocScratchBytes;
    return e;
}

cudaError_t launch_build_tables(cudaStream_t s, const float* params, int M, float* table)
{
    const int n = M * LIDAR_TABLE_SIZE;
    if (n == 0) return cudaSuccess;
    k_build_tables<<<(n + 255) / 256, 256, 0, s>>>(params, M, table);
    return cudaGetLastError();
}

cudaError_t launch_build_tables_backward(cudaStream_t s, const float* params, const float* grad_table, int M,
                                         float* grad_params)
{
    if (M == 0) return cudaSuccess;
    k_build_tables_backward<<<(M + 7) / 8, 256, 0, s>>>(params, grad_table, M, grad_params);
    return cudaGetLastError();
}

size_t backward_scratch_bytes(int M)
{
    const size_t n_acc = (size_t)M * LIDAR_TABLE_SIZE + 1;
    return 256 + ((n_acc * 8 + 255) / 256) * 256 + kAdjBlocks * sizeof(double);
}

cudaError_t launch_cast_backward(cudaStream_t s, int64_t n, const uint8_t* valid, const uint16_t* mat,
                                 const float* theta_deg, const float* rf, TableDev T, float gain,
                                 const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                 float* loss, float* grad_table, float* grad_gain, void* scratch,
                                 size_t scratch_bytes)
{
    if (scratch_bytes < backward_scratch_bytes(T.n_mat)) return cudaErrorInvalidValue;
    const int n_acc = T.n_mat * LIDAR_TABLE_SIZE + 1;
    char* p = (char*)scratch;
    unsigned int* absmax = (unsigned int*)p;
    unsigned long long* count = (unsigned long long*)(p + 8);
    p += 256;
    unsigned long long* acc = (unsigned long long*)p;
    p += (((size_t)n_acc * 8 + 255) / 256) * 256;
    double* partials = (double*)p;
    // every call starts from zeroed accumulators (the scratch may hold the last call's)
    const cudaError_t me = cudaMemsetAsync(scratch, 0, 256 + (((size_t)n_acc * 8 + 255) / 256) * 256, s);
    if (me != cudaSuccess) return me;
    // one wave of resident blocks (at most kAdjBlocks), no more than the tape needs
    int device = 0, sms = 0;
    cudaGetDevice(&device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms < 1) sms = 1;
    const int64_t need = (n + kAdjThreads * kAdjPerLane - 1) / (kAdjThreads * kAdjPerLane);
    auto wave = [&](const void* fn, size_t smem_bytes) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kAdjThreads, smem_bytes) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        int64_t b = (int64_t)per_sm * sms;
        if (b > need) b = need;
        if (b > kAdjBlocks) b = kAdjBlocks;
        return (int)(b < 1 ? 1 : b);
    };
    // vector loads need every tape array aligned to its 4-element vector
    const float* g = target_I ? target_I : grad_I;
    auto aligned = [](const void* p, uintptr_t a) { return p == nullptr || ((uintptr_t)p % a) == 0; };
    const bool vec = aligned(valid, 4) && aligned(target_valid, 4) && aligned(mat, 8) && aligned(theta_deg, 16) &&
                     aligned(rf, 16) && aligned(g, 16);
    const int blocks1 = wave(vec ? (const void*)k_adj_absmax<true> : (const void*)k_adj_absmax<false>, 0);
    if (vec)
        k_adj_absmax<true><<<blocks1, kAdjThreads, 0, s>>>(n, valid, mat, theta_deg, rf, T, gain, grad_I, target_I,
                                                           target_valid, absmax, count);
    else
        k_adj_absmax<false><<<blocks1, kAdjThreads, 0, s>>>(n, valid, mat, theta_deg, rf, T, gain, grad_I,
                                                            target_I, target_valid, absmax, count);
    const size_t smem = (size_t)n_acc * sizeof(unsigned long long);
    const void* acc_fn = vec ? (const void*)k_adj_accumulate<true> : (const void*)k_adj_accumulate<false>;
    int use_shared = smem <= 96 * 1024;
    if (use_shared && smem > 48 * 1024) {
        if (cudaFuncSetAttribute(acc_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            use_shared = 0;
        }
    }
    const int blocks = wave(acc_fn, use_shared ? smem : 0);
    if (vec)
        k_adj_accumulate<true><<<blocks, kAdjThreads, use_shared ? smem : 0, s>>>(
            n, valid, mat, theta_deg, rf, T, gain, grad_I, target_I, target_valid, absmax, count, acc, partials,
            use_shared);
    else
        k_adj_accumulate<false><<<blocks, kAdjThreads, use_shared ? smem : 0, s>>>(
            n, valid, mat, theta_deg, rf, T, gain, grad_I, target_I, target_valid, absmax, count, acc, partials,
            use_shared);
    k_adj_finalize<<<(n_acc + kFinalizeThreads - 1) / kFinalizeThreads, kFinalizeThreads, 0, s>>>(
        n_acc, acc, absmax, count, target_I != nullptr, partials, blocks, grad_table, grad_gain, loss);
    return cudaGetLastError();
}

size_t onepass_scratch_bytes(int M, int num_sms)
{
    const size_t n_acc = (size_t)M * LIDAR_TABLE_SIZE + 1;
    const size_t G = (size_t)(num_sms > 0 ? num_sms : 1);
    return ((n_acc * 8 + 255) / 256) * 256 + ((G * 24 + 255) / 256) * 256;
}

cudaError_t launch_cast_backward_onepass(cudaStream_t s, int64_t n, const uint8_t* valid, const uint16_t* mat,
                                         const float* theta_deg, const float* rf, TableDev T, float gain,
                                         const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                         float* loss, float* grad_table, float* grad_gain, void* scratch,
                                         size_t scratch_bytes, unsigned* ctl, int* status, uint64_t wait_ns,
                                         int num_sms)
{
    const int n_acc = T.n_mat * LIDAR_TABLE_SIZE + 1;
    if (num_sms < 1 || scratch_bytes < onepass_scratch_bytes(T.n_mat, num_sms)) return cudaErrorInvalidValue;
    const float* g = target_I ? target_I : grad_I;
    // the copy engine needs 16-byte aligned sources; otherwise the threads load the tape
    auto al16 = [](const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; };
    const bool tma = al16(valid) && al16(target_valid) && al16(mat) && al16(theta_deg) && al16(rf) && al16(g);
    const size_t acc_smem = (size_t)((n_acc + 1) & ~1) * 8;
    const size_t smem = (tma ? (size_t)kOneStages * kOneStageBytes : 0) + acc_smem + kOneStages * 8;
    const void* fn = tma ? (const void*)k_adj_onepass<true> : (const void*)k_adj_onepass<false>;
    {
        // the shared-memory attribute and the residency are asked once per
        // (device, kernel, size); a failure means the accumulators do not fit
        // beside the stages: the caller then takes the separate passes
        static std::mutex mu;
        static std::map<std::tuple<int, bool, size_t>, bool> fits;
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        auto it = fits.find({dev, tma, smem});
        if (it == fits.end()) {
            int per_sm = 0;
            bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
                      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kOneThreads, smem) == cudaSuccess &&
                      per_sm >= 1;
            if (!ok) cudaGetLastError();
            it = fits.emplace(std::make_tuple(dev, tma, smem), ok).first;
        }
        if (!it->second) return cudaErrorNotSupported;
    }
    // one block per SM whatever the occupancy, so the aligned and the unaligned
    // paths split the tape the same way (and give the same sums)
    const int64_t n_chunks = (n + kOneChunk - 1) / kOneChunk;
    int G = (int)std::min<int64_t>(std::max<int64_t>(n_chunks, 1), num_sms);
    char* p = (char*)scratch;
    OneArgs a{};
    a.n = n;
    a.valid = valid;
    a.mat = mat;
    a.theta = theta_deg;
    a.rf = rf;
    a.g = g;
    a.tvalid = target_valid;
    a.T = T;
    a.gain = gain;
    a.mse = target_I != nullptr;
    a.n_acc = n_acc;
    a.acc = (unsigned long long*)p;
    p += (((size_t)n_acc * 8 + 255) / 256) * 256;
    a.blk_max = (float*)p;
    a.blk_sh = (int*)(p + (size_t)G * 4);
    a.blk_loss = (double*)(p + (size_t)G * 8);
    a.blk_n = (unsigned long long*)(p + (size_t)G * 16);
    a.ctl = ctl;
    a.status = status;
    a.wait_ns = wait_ns;
    a.loss = loss;
    a.grad_table = grad_table;
    a.grad_gain = grad_gain;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kOneThreads), args, smem, s);
}

}  // namespace lidar
