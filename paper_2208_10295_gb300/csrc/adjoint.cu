// Reflectance tables from material parameters, and the adjoint of the
// intensity with respect to the tables and the gain (hits and masks held
// fixed from the forward pass).
//
// Table (Eq. 4's Lambertian law R(theta) = R(0) cos(theta) with R(0) = a, plus
// a specular lobe): T[m][k] = a cos(k deg) + s exp(-k^2 / (2 w^2)), k = 0..90.
//
// Adjoint accumulation is deterministic: every contribution is converted to a
// 64-bit fixed-point integer at a power-of-two scale chosen from the largest
// contribution (so no sum can overflow) and summed with integer atomics, first
// in a block-private shared-memory copy of the gradient; integer addition is
// associative, so the result does not depend on scheduling.  Two forms:
//   - one pass (the default): one cooperative launch reads the tape once
//     (copy-engine stages), each block sums at its own scale, rescaled as its
//     maximum grows, and the blocks meet at the common scale after a bounded
//     grid-wide wait;
//   - separate passes (tables too large for shared memory beside the copy
//     stages, devices without cooperative launch, the allocation-free entry
//     point): a scale pass over the tape, the fixed-point accumulation at
//     the global scale, and a finalize kernel.
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
    float* grad_table, float* grad_gain, float* loss, unsigned long long* n_used)
{
    const float scale = fixed_scale(*absmax_bits, *count);
    const float inv_scale = __frcp_rn(scale);  // exact: the scale is a power of two
    const unsigned long long N = *count;
    if (n_used && blockIdx.x == 0 && threadIdx.x == 0) *n_used = N;
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
// (a rounding shift) before the chunk is added.  Each block then writes its
// sums as one row.  After one bounded grid-wide wait every block knows every
// block's maximum and scale; block b adds, over its own slice of the table
// entries, every block's row shifted to the common scale of the whole tape (a
// rounding shift) and writes those gradients; block 0 sums the per-block loss
// partials in block order.  Every step is a deterministic function of the
// tape and the grid size, so the result is bit-reproducible run to run.

constexpr int kOneThreads = 512;
constexpr int kOneBPT = 4;                          // beams per thread per chunk (one per warp step)
constexpr int kOneChunk = kOneThreads * kOneBPT;    // 2048 beams
constexpr int kOneStages = 2;
constexpr int kOneBlocksPerSm = 2;
constexpr int kOneStageBytes = kOneChunk * 16;      // valid 1, target valid 1, mat 2, theta 4, rf 4, g 4
constexpr int kOneWarps = kOneThreads / 32;
constexpr int kOneMaxGrid = 1024;  // blocks of one launch (two per SM on up to 512 SMs)

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
    long long* rows;            // [grid][n_acc] each block's sums at its own scale
    float* blk_max;             // [grid] per block: largest contribution
    int* blk_sh;                // [grid] its fixed-point shift
    double* blk_loss;           // [grid] sum of squared residuals
    unsigned long long* blk_n;  // [grid] beams used
    unsigned long long* arrivals;  // blocks arrived at the grid-wide wait, over every launch (never reset)
    unsigned long long base;       // its value when this launch starts
    int* status;
    uint64_t wait_ns;
    float* loss;
    float* grad_table;
    float* grad_gain;
    unsigned long long* n_used;  // NULL, or the number of beams the mean runs over
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

// round(x 2^sh) as a 64-bit integer for |x| 2^sh < 2^61: y = x 2^sh is exact
// (a power-of-two scale), q = y / 2^31 rounded and r = y - q 2^31 are exact
// in FP32 (|q| < 2^30, |r| <= 2^30), and both convert to 32-bit integers; the
// FP32-to-int64 conversion would run on the FP64 pipe, which is narrow on
// this part.  Ties of r round to even.
__device__ __forceinline__ long long fixed_of(float x, float scale)
{
    const float y = x * scale;
    const float q = rintf(y * 4.656612873077393e-10f);  // 2^-31
    const float r = fmaf(-q, 2147483648.0f, y);
    return ((long long)__float2int_rn(q) << 31) + (long long)__float2int_rn(r);
}

// v / 2^d rounded to nearest (ties up), d >= 0 (d <= 0 returns v unchanged)
__device__ __forceinline__ long long round_shift(long long v, int d)
{
    if (d <= 0) return v;
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
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 2000;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it == 0) t0 = adj_global_ns();
        else if (adj_global_ns() - t0 > wait_ns) return false;
    }
}

// Shared-memory accumulators of the one-pass kernel: each 64-bit two's
// complement fixed-point sum is kept as a low and a high 32-bit word in two
// arrays and added with native 32-bit atomics, the carry out of the low word
// (seen in the value the atomic returns) added into the high word.  Every add
// is exact modulo 2^64 and the adds commute, so the sum is the 64-bit sum.
struct Acc32 {
    unsigned* lo;
    unsigned* hi;
    __device__ __forceinline__ void add(int j, long long v) const
    {
        const unsigned l = (unsigned)(unsigned long long)v;
        const unsigned h = (unsigned)((unsigned long long)v >> 32);
        const unsigned old = atomicAdd(&lo[j], l);
        const unsigned carry = (old + l < old) ? 1u : 0u;
        if (h + carry) atomicAdd(&hi[j], h + carry);
    }
    __device__ __forceinline__ long long get(int j) const
    {
        return (long long)(((unsigned long long)hi[j] << 32) | lo[j]);
    }
    __device__ __forceinline__ void set(int j, long long v) const
    {
        lo[j] = (unsigned)(unsigned long long)v;
        hi[j] = (unsigned)((unsigned long long)v >> 32);
    }
};

// Grid-wide wait of a cooperative launch in two halves: every block arrives
// once (thread 0 publishes the block's writes first), then waits until the
// arrival counter reaches its value at the launch's start plus the grid,
// bounded by wait_ns (then ST_TIMEOUT, and false in every thread of the
// block).  The counter only grows: every block of every launch arrives
// exactly once, timed out or not, so the caller knows its value at the next
// launch and nothing resets it.
__device__ __forceinline__ void grid_arrive(unsigned long long* arrivals)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(arrivals, 1ull);
    }
}

__device__ __forceinline__ bool grid_wait_for(unsigned long long* arrivals, unsigned long long target, int* status,
                                              uint64_t wait_ns, int* s_flag)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = adj_global_ns();
        while (*(volatile unsigned long long*)arrivals < target) {
            if (adj_global_ns() - t0 > wait_ns) {
                raise_status(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

template <bool kTma>
__global__ void __launch_bounds__(kOneThreads, 2) k_adj_onepass(const __grid_constant__ OneArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stages = smem;
    const int n_acc_pad = (a.n_acc + 3) & ~3;
    unsigned* s_words = (unsigned*)(smem + (kTma ? kOneStages * kOneStageBytes : 0));
    const Acc32 acc{s_words, s_words + n_acc_pad};
    uint64_t* s_bar = (uint64_t*)(s_words + 2 * n_acc_pad);
    float* s_table = (float*)(s_bar + kOneStages);  // the reflectance table, [n_mat][91]
    __shared__ __align__(16) float s_wmax[2][kOneWarps];
    __shared__ double s_red[kOneThreads];
    __shared__ unsigned long long s_cnt[kOneWarps];
    __shared__ int s_flag;
    __shared__ float s_gmax;
    __shared__ int s_sh[kOneMaxGrid];  // every block's fixed-point shift

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, blk = blockIdx.x;
    const int64_t n = a.n;
    // this block's beams: an even share of the tape in whole 16-beam groups
    // (16-byte aligned copies of every array), taken in chunks of kOneChunk
    // beams; only the last chunk of a block may be shorter
    const int64_t n16 = (n + 15) / 16;
    const int64_t first = ((int64_t)blk * n16 / G) * 16;
    const int64_t last = min((((int64_t)blk + 1) * n16 / G) * 16, n);
    const int64_t L = last > first ? last - first : 0;
    const int64_t n_chunks = (L + kOneChunk - 1) / kOneChunk;
    const bool has_tv = a.tvalid != nullptr;


    // beams of chunk k, and how many of them the copy engine brings (whole
    // 16-beam groups: only the tape's last few beams are loaded by the threads)
    auto chunk_beams = [&](int64_t k) { return (int)min((int64_t)kOneChunk, L - k * kOneChunk); };
    auto chunk_copied = [&](int64_t k) { return chunk_beams(k) & ~15; };
    auto issue = [&](int64_t k) {
        const int slot = (int)(k % kOneStages);
        unsigned char* d = stages + slot * kOneStageBytes;
        const int64_t c0 = first + k * kOneChunk;
        const unsigned nb = (unsigned)chunk_copied(k);
        bar_expect(&s_bar[slot], nb * (has_tv ? 16u : 15u));
        if (nb == 0) return;
        bulk_copy(d, a.valid + c0, nb, &s_bar[slot]);
        if (has_tv) bulk_copy(d + kOneChunk, a.tvalid + c0, nb, &s_bar[slot]);
        bulk_copy(d + 2 * kOneChunk, a.mat + c0, 2 * nb, &s_bar[slot]);
        bulk_copy(d + 4 * kOneChunk, a.theta + c0, 4 * nb, &s_bar[slot]);
        bulk_copy(d + 8 * kOneChunk, a.rf + c0, 4 * nb, &s_bar[slot]);
        bulk_copy(d + 12 * kOneChunk, a.g + c0, 4 * nb, &s_bar[slot]);
    };
    // the first copies go out before the accumulators are cleared and the
    // table is read (the stages are disjoint from both); the block barrier
    // below orders the barriers' initialisation before any thread waits
    int64_t issued = 0;  // next chunk to copy (meaningful in thread 0)
    if (kTma && tid == 0) {
        for (int st = 0; st < kOneStages; ++st) bar_init(&s_bar[st]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (; issued < n_chunks && issued < kOneStages; ++issued) issue(issued);
    }
    for (int j = tid; j < 2 * n_acc_pad; j += kOneThreads) s_words[j] = 0u;
    for (int j = tid; j < a.T.n_mat * LIDAR_TABLE_SIZE; j += kOneThreads) s_table[j] = __ldg(&a.T.table[j]);
    __syncthreads();

    float blk_max = 0.0f;
    int sh = 126;
    float loss32 = 0.0f, gain32 = 0.0f;  // this thread's squared residuals and gain terms, in its order
    unsigned cnt = 0;
    bool failed = false;
    int64_t k_fail = n_chunks;  // first chunk whose stage wait ran out
    for (int64_t k = 0; k < n_chunks; ++k) {
        const int64_t c0 = first + k * kOneChunk;
        const int nb = chunk_beams(k);
        TapeIn in;
        bool ok = true;
        const unsigned char* d = nullptr;
        if (kTma) {
            const int slot = (int)(k % kOneStages);
            ok = bar_wait(&s_bar[slot], (unsigned)((k / kOneStages) & 1), a.wait_ns);
            d = stages + slot * kOneStageBytes;
        }
        const int r0 = kOneBPT * tid;  // this thread's first beam in the chunk
        if (kTma && ok && r0 + kOneBPT <= chunk_copied(k)) {
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
        } else {
            // the ragged end of the tape, a tape the copy engine cannot address,
            // or a wait that ran out
            const int cp = kTma && ok ? chunk_copied(k) : 0;
#pragma unroll
            for (int j = 0; j < kOneBPT; ++j) {
                const int rr = r0 + j;
                in.valid[j] = 0;
                in.tvalid[j] = 1;
                in.mat[j] = 0;
                in.theta[j] = in.rf[j] = in.g[j] = 0.0f;
                if (!ok || rr >= nb) continue;
                if (rr < cp) {
                    in.valid[j] = d[rr];
                    if (has_tv) in.tvalid[j] = d[kOneChunk + rr];
                    in.mat[j] = reinterpret_cast<const uint16_t*>(d + 2 * kOneChunk)[rr];
                    in.theta[j] = reinterpret_cast<const float*>(d + 4 * kOneChunk)[rr];
                    in.rf[j] = reinterpret_cast<const float*>(d + 8 * kOneChunk)[rr];
                    in.g[j] = reinterpret_cast<const float*>(d + 12 * kOneChunk)[rr];
                } else {
                    const int64_t b = c0 + rr;
                    in.valid[j] = __ldcs(&a.valid[b]);
                    if (has_tv) in.tvalid[j] = __ldcs(&a.tvalid[b]);
                    in.mat[j] = __ldcs(&a.mat[b]);
                    in.theta[j] = __ldcs(&a.theta[b]);
                    in.rf[j] = __ldcs(&a.rf[b]);
                    in.g[j] = __ldcs(&a.g[b]);
                }
            }
        }
        float t_lo[kOneBPT], t_hi[kOneBPT];
        int e[kOneBPT];
        float mx = 0.0f;
        const int n_mat = a.T.n_mat;
        const float gain = a.gain;
        const bool mse = a.mse != 0;
#pragma unroll
        for (int j = 0; j < kOneBPT; ++j) {
            e[j] = -1;
            t_lo[j] = t_hi[j] = 0.0f;
            if (!(in.valid[j] != 0 && in.tvalid[j] != 0)) continue;
            // the forward pass's lerp of the table row (Sec. III), then dL/dI
            const int m = in.mat[j] < n_mat ? in.mat[j] : n_mat - 1;
            const float th = in.theta[j];
            int i = (int)th;
            if (i > LIDAR_TABLE_SIZE - 2) i = LIDAR_TABLE_SIZE - 2;
            const float f = th - (float)i;
            const int ei = m * LIDAR_TABLE_SIZE + i;
            const float R = s_table[ei] * (1.0f - f) + s_table[ei + 1] * f;
            const float rf = in.rf[j];
            float res = 0.0f, gI = in.g[j];
            if (mse) {
                res = gain * R * rf - in.g[j];
                gI = 2.0f * res;
            }
            const float w = gain * rf * gI;
            e[j] = ei;
            t_lo[j] = w * (1.0f - f);
            t_hi[j] = w * f;
            gain32 += rf * R * gI;
            mx = fmaxf(mx, fmaxf(fabsf(t_lo[j]), fabsf(t_hi[j])));
            loss32 = __fmaf_rn(res, res, loss32);
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
        if (kTma && tid == 0 && issued < n_chunks) {
            // the stage just read is free: order the generic reads before the
            // copy engine's writes, then refill it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(issued);
            ++issued;
        }
        float cm = 0.0f;
#pragma unroll
        for (int w = 0; w < kOneWarps; w += 4) {
            const float4 q = *reinterpret_cast<const float4*>(&s_wmax[k & 1][w]);
            cm = fmaxf(fmaxf(cm, fmaxf(q.x, q.y)), fmaxf(q.z, q.w));
        }
        if (cm > blk_max) {
            const int nsh = one_shift(cm, L);
            if (nsh < sh && blk_max > 0.0f) {
                const int dd = sh - nsh;
                for (int j = tid; j < a.n_acc; j += kOneThreads) acc.set(j, round_shift(acc.get(j), dd));
                __syncthreads();
            }
            if (nsh < sh) sh = nsh;
            blk_max = cm;
        }
        if (blk_max > 0.0f) {
            // a thread's neighbouring beams that share a table bin are added once
            // (integer sums: the grouping does not change the result)
            const float scale = ldexpf(1.0f, sh);
            int cur = -1;
            long long a0 = 0, a1 = 0;
#pragma unroll
            for (int j = 0; j < kOneBPT; ++j) {
                if (e[j] < 0) continue;
                if (e[j] != cur) {
                    if (cur >= 0) {
                        acc.add(cur, a0);
                        acc.add(cur + 1, a1);
                    }
                    cur = e[j];
                    a0 = a1 = 0;
                }
                a0 += fixed_of(t_lo[j], scale);
                a1 += fixed_of(t_hi[j], scale);
            }
            if (cur >= 0) {
                acc.add(cur, a0);
                acc.add(cur + 1, a1);
            }
        }
    }
    __syncthreads();  // every thread is done with the last chunk's maxima
    if (failed && kTma && tid == 0) {
        // let the copies still in flight (chunks k_fail .. issued - 1, at most one
        // per stage) land before the block's shared memory goes away; bounded by
        // at least a second whatever the caller's wait limit
        const uint64_t drain_ns = a.wait_ns > 1000000000ull ? a.wait_ns : 1000000000ull;
        for (int64_t k = k_fail; k < issued; ++k)
            bar_wait(&s_bar[k % kOneStages], (unsigned)((k / kOneStages) & 1), drain_ns);
    }
    if (failed && tid == 0) raise_status(a.status, ST_TIMEOUT);

    // ---- this block's gain-term maximum, loss partial (fixed order), beam count:
    // FP32 within a warp (a fixed shuffle tree), FP64 across warps
    float gmx = fabsf(gain32);
    float l = loss32;
    unsigned c = cnt;
    for (int o = 16; o > 0; o >>= 1) {
        gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, o));
        l += __shfl_down_sync(0xffffffffu, l, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        s_red[warp] = (double)l;
        s_cnt[warp] = c;
        s_wmax[0][warp] = gmx;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        unsigned long long ct = 0;
        float gm = 0.0f;
        for (int w = 0; w < kOneWarps; ++w) {
            t += s_red[w];
            ct += s_cnt[w];
            gm = fmaxf(gm, s_wmax[0][w]);
        }
        s_gmax = gm;
        a.blk_loss[blk] = t;
        a.blk_n[blk] = ct;
    }
    __syncthreads();
    // the threads' gain sums join the fixed-point sums: widen the scale first
    // if one of them is larger than every term seen
    if (s_gmax > blk_max && !failed) {
        const int nsh = one_shift(s_gmax, L);
        if (nsh < sh && blk_max > 0.0f) {
            const int dd = sh - nsh;
            for (int j = tid; j < a.n_acc; j += kOneThreads) acc.set(j, round_shift(acc.get(j), dd));
        }
        if (nsh < sh) sh = nsh;
        blk_max = s_gmax;
    }
    __syncthreads();
    if (blk_max > 0.0f) {
        long long gq = fixed_of(gain32, ldexpf(1.0f, sh));
        for (int o = 16; o > 0; o >>= 1) gq += __shfl_xor_sync(0xffffffffu, gq, o);
        if (lane == 0 && gq) acc.add(a.n_acc - 1, gq);
    }
    __syncthreads();  // every warp's gain sum is in before the row is read out
    // this block's slice of the entries, summed over every row after the
    // wait, and the gradients already in its first 32 entries (read now:
    // nothing else writes them during the launch)
    const int j0 = (int)((int64_t)blk * a.n_acc / G), j1 = (int)(((int64_t)blk + 1) * a.n_acc / G);
    float g_prev = 0.0f;
    if (warp == 0 && lane < j1 - j0) {
        const int j = j0 + lane;
        if (j < a.n_acc - 1) {
            if (a.grad_table) g_prev = a.grad_table[j];
        } else if (a.grad_gain) {
            g_prev = *a.grad_gain;
        }
    }
    // this block's sums at its own scale, one dense row, with its maximum and shift
    {
        long long* row = a.rows + (int64_t)blk * a.n_acc;
        for (int j = tid; j < a.n_acc; j += kOneThreads) row[j] = failed ? 0ll : acc.get(j);
    }
    if (tid == 0) {
        a.blk_max[blk] = failed ? 0.0f : blk_max;
        a.blk_sh[blk] = sh;
    }
    // ---- the grid-wide wait: every block's row, maximum, shift, count and loss partial are out
    grid_arrive(a.arrivals);
    if (!grid_wait_for(a.arrivals, a.base + (unsigned long long)G, a.status, a.wait_ns, &s_flag)) failed = true;

    // The merge takes the slice in pieces of up to 32 entries.  For a piece of
    // P entries a warp load covers R = 32 / P rows (lane l: entry l mod P of
    // row sub-group l / P); warp w takes rows (i kOneWarps + w) R + sub for
    // i = 0, 1, ...  The first batch of loads is issued before the per-block
    // maxima are reduced, so both round trips overlap.
    constexpr int kRowLoads = 8;
    auto piece = [&](int e0, int& P, int& R, int& sub, int& j) {
        P = min(32, j1 - e0);
        R = 32 / P;
        sub = lane / P;
        j = e0 + lane % P;
    };
    auto load_batch = [&](int e0, int i0, long long (&v)[kRowLoads]) {
        int P, R, sub, j;
        piece(e0, P, R, sub, j);
#pragma unroll
        for (int u = 0; u < kRowLoads; ++u) {
            const int r = ((i0 + u) * kOneWarps + warp) * R + sub;
            v[u] = (sub < R && r < G) ? __ldcg(&a.rows[(int64_t)r * a.n_acc + j]) : 0ll;
        }
    };
    long long v0[kRowLoads];
    if (j0 < j1) load_batch(j0, 0, v0);
    // the common scale (the largest contribution of the whole tape) and the
    // number of beams used, reduced in a fixed order by every block; every
    // block's shift into shared memory
    {
        float gm = 0.0f;
        unsigned long long N = 0;
        for (int j = tid; j < G; j += kOneThreads) {
            gm = fmaxf(gm, __ldcg(&a.blk_max[j]));
            N += __ldcg(&a.blk_n[j]);
            s_sh[j] = __ldcg(&a.blk_sh[j]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
            N += __shfl_xor_sync(0xffffffffu, N, o);
        }
        if (lane == 0) {
            s_wmax[1][warp] = gm;
            s_cnt[warp] = N;
        }
        __syncthreads();
        if (tid == 0) {
            float g2 = 0.0f;
            unsigned long long n2 = 0;
            for (int w = 0; w < kOneWarps; ++w) {
                g2 = fmaxf(g2, s_wmax[1][w]);
                n2 += s_cnt[w];
            }
            s_gmax = g2;
            s_cnt[0] = n2;
        }
        __syncthreads();
    }
    const float gmax = s_gmax;
    const unsigned long long N = s_cnt[0];
    const int S = one_shift(gmax, n);
    // block 0's last warp writes the loss: the partials in a fixed order (lane
    // l takes blocks l, l + 32, ..., then a fixed shuffle tree)
    if (blk == 0 && tid == 0 && a.n_used) *a.n_used = N;
    if (blk == 0 && warp == kOneWarps - 1 && a.loss) {
        double t = 0.0;
        for (int j = lane; j < G; j += 32) t += __ldcg(&a.blk_loss[j]);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) *a.loss = a.mse ? (float)(N ? t / (double)N : 0.0) : 0.0f;
    }
    // each block sums every row over its slice of the entries, each row
    // shifted from its block's scale to the common one (a rounding shift, as
    // the block would have made), and writes those gradients; the warps' and
    // sub-groups' sums meet in shared memory (integer sums: the order is free)
    if (!failed && gmax > 0.0f) {
        const float inv_scale = ldexpf(1.0f, -S);  // exact: a power of two
        const float norm = a.mse ? (N ? __frcp_rn((float)N) : 0.0f) : 1.0f;
        long long* s_part = reinterpret_cast<long long*>(s_red);  // [kOneWarps][32]
        for (int e0 = j0; e0 < j1; e0 += 32) {
            int P, R, sub, j;
            piece(e0, P, R, sub, j);
            long long t = 0;
            for (int i0 = 0; (i0 * kOneWarps + warp) * R < G; i0 += kRowLoads) {
                long long v[kRowLoads];
                if (e0 == j0 && i0 == 0) {
#pragma unroll
                    for (int u = 0; u < kRowLoads; ++u) v[u] = v0[u];
                } else {
                    load_batch(e0, i0, v);
                }
#pragma unroll
                for (int u = 0; u < kRowLoads; ++u) {
                    const int r = ((i0 + u) * kOneWarps + warp) * R + sub;
                    if (sub < R && r < G) t += round_shift(v[u], s_sh[r] - S);
                }
            }
            s_part[warp * 32 + lane] = t;
            __syncthreads();
            if (warp == 0 && lane < P) {
                long long tot = 0;
                for (int w = 0; w < kOneWarps; ++w)
                    for (int q = 0; q < R; ++q) tot += s_part[w * 32 + q * P + lane];
                const float v = __fmul_rn(__fmul_rn(__ll2float_rn(tot), inv_scale), norm);
                const int jj = e0 + lane;
                if (jj < a.n_acc - 1) {
                    if (a.grad_table) a.grad_table[jj] = (e0 == j0 ? g_prev : a.grad_table[jj]) + v;
                } else if (a.grad_gain) {
                    *a.grad_gain = (e0 == j0 ? g_prev : *a.grad_gain) + v;
                }
            }
            __syncthreads();
        }
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
                                 size_t scratch_bytes, unsigned long long* n_used)
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
        n_acc, acc, absmax, count, target_I != nullptr, partials, blocks, grad_table, grad_gain, loss, n_used);
    return cudaGetLastError();
}

size_t onepass_scratch_bytes(int M, int num_sms)
{
    const size_t n_acc = (size_t)M * LIDAR_TABLE_SIZE + 1;
    const size_t G = (size_t)(num_sms > 0 ? num_sms : 1) * kOneBlocksPerSm;
    return ((G * n_acc * 8 + 255) / 256) * 256 + ((G * 24 + 255) / 256) * 256;
}

cudaError_t launch_cast_backward_onepass(cudaStream_t s, int64_t n, const uint8_t* valid, const uint16_t* mat,
                                         const float* theta_deg, const float* rf, TableDev T, float gain,
                                         const float* grad_I, const float* target_I, const uint8_t* target_valid,
                                         float* loss, float* grad_table, float* grad_gain, void* scratch,
                                         size_t scratch_bytes, unsigned long long* arrivals,
                                         unsigned long long* arrivals_base, int* status, uint64_t wait_ns, int num_sms,
                                         unsigned long long* n_used)
{
    const int n_acc = T.n_mat * LIDAR_TABLE_SIZE + 1;
    if (num_sms < 1 || scratch_bytes < onepass_scratch_bytes(T.n_mat, num_sms)) return cudaErrorInvalidValue;
    const float* g = target_I ? target_I : grad_I;
    // the copy engine needs 16-byte aligned sources; otherwise the threads load the tape
    auto al16 = [](const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; };
    const bool tma = al16(valid) && al16(target_valid) && al16(mat) && al16(theta_deg) && al16(rf) && al16(g);
    const size_t acc_smem = (size_t)((n_acc + 3) & ~3) * 8;  // low and high words, 16-byte aligned
    const size_t table_smem = (size_t)T.n_mat * LIDAR_TABLE_SIZE * 4;
    const size_t smem_tma = (size_t)kOneStages * kOneStageBytes + acc_smem + kOneStages * 8 + table_smem;
    const size_t smem_direct = acc_smem + kOneStages * 8 + table_smem;
    const size_t smem = tma ? smem_tma : smem_direct;
    const void* fn_tma = (const void*)k_adj_onepass<true>;
    const void* fn = tma ? fn_tma : (const void*)k_adj_onepass<false>;
    // blocks per SM: as many as the copy-engine variant can keep resident (up to
    // kOneBlocksPerSm), whichever variant runs, so that the aligned and the
    // unaligned paths split the tape the same way (and give the same sums)
    int bps = 0;
    {
        // the kernel may take up to the device's opt-in shared memory (set once
        // per device and kernel: the attribute is the function's, whatever the
        // size of a launch); residency is asked once per (device, kernel, size).
        // No room for one block means the accumulators do not fit beside the
        // stages: the caller then takes the separate passes.
        static std::mutex mu;
        static std::map<std::pair<int, const void*>, bool> opted;
        static std::map<std::tuple<int, const void*, size_t>, int> resident;
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        auto opt_in = [&](const void* f) {
            auto it = opted.find({dev, f});
            if (it != opted.end()) return it->second;
            int optin = 0;
            cudaFuncAttributes fa{};
            bool ok = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
                      cudaFuncGetAttributes(&fa, f) == cudaSuccess &&
                      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           optin - (int)fa.sharedSizeBytes) == cudaSuccess;
            if (!ok) cudaGetLastError();
            opted[{dev, f}] = ok;
            return ok;
        };
        auto per_sm = [&](const void* f, size_t bytes) {
            auto it = resident.find({dev, f, bytes});
            if (it != resident.end()) return it->second;
            int r = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, f, kOneThreads, bytes) != cudaSuccess) {
                cudaGetLastError();
                r = 0;
            }
            resident[{dev, f, bytes}] = r;
            return r;
        };
        if (!opt_in(fn_tma) || !opt_in(fn)) return cudaErrorNotSupported;
        bps = std::min(per_sm(fn_tma, smem_tma), kOneBlocksPerSm);
        if (bps < 1 || per_sm(fn, smem) < bps) return cudaErrorNotSupported;
    }
    // about a chunk per block at least; a block's share is whole 16-beam groups
    const int64_t n_chunks = (n + kOneChunk - 1) / kOneChunk;
    int G = (int)std::min<int64_t>(std::max<int64_t>(n_chunks, 1), (int64_t)bps * num_sms);
    if (G > kOneMaxGrid) G = kOneMaxGrid;
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
    a.rows = (long long*)p;
    p += (((size_t)G * n_acc * 8 + 255) / 256) * 256;
    a.blk_max = (float*)p;
    a.blk_sh = (int*)(p + (size_t)G * 4);
    a.blk_loss = (double*)(p + (size_t)G * 8);
    a.blk_n = (unsigned long long*)(p + (size_t)G * 16);
    a.arrivals = arrivals;
    a.base = *arrivals_base;
    a.status = status;
    a.wait_ns = wait_ns;
    a.loss = loss;
    a.grad_table = grad_table;
    a.grad_gain = grad_gain;
    a.n_used = n_used;
    void* args[] = {&a};
    const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kOneThreads), args, smem, s);
    if (e != cudaSuccess)
        cudaGetLastError();  // leave no stale launch error for the next call
    else
        *arrivals_base += (unsigned long long)G;  // every block arrives once, whatever happens in the launch
    return e;
}

}  // namespace lidar
