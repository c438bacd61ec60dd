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

}  // namespace lidar
