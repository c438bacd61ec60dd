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

__device__ __forceinline__ TapeRow tape_row(int64_t b, const uint8_t* valid, const uint16_t* mat,
                                            const float* theta_deg, const float* rf, TableDev T, float gain,
                                            const float* grad_I, const float* target_I,
                                            const uint8_t* target_valid)
{
    TapeRow r;
    r.use = valid[b] != 0 && (target_valid == nullptr || target_valid[b] != 0);
    if (!r.use) return r;
    const int m = mat[b] < T.n_mat ? mat[b] : T.n_mat - 1;
    const float th = theta_deg[b];
    int i = (int)th;
    if (i > LIDAR_TABLE_SIZE - 2) i = LIDAR_TABLE_SIZE - 2;
    const float f = th - (float)i;
    const float* row = T.table + (int64_t)m * LIDAR_TABLE_SIZE;
    const float R = row[i] * (1.0f - f) + row[i + 1] * f;
    r.m = m;
    r.i = i;
    r.f = f;
    r.R = R;
    r.rf = rf[b];
    if (target_I) {
        r.res = gain * R * r.rf - target_I[b];
        r.gI = 2.0f * r.res;
    } else {
        r.res = 0.0f;
        r.gI = grad_I[b];
    }
    return r;
}

// pass 1: largest |contribution| bound and the count of used beams
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
    float mx = 0.0f;
    unsigned long long c = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        TapeRow r = tape_row(b, valid, mat, theta_deg, rf, T, gain, grad_I, target_I, target_valid);
        if (!r.use) continue;
        ++c;
        const float wt = fmaxf(fabsf(gain * r.rf), fabsf(r.rf * r.R));
        mx = fmaxf(mx, fabsf(r.gI) * wt);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
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

// pass 2: fixed-point accumulation; per-block shared copy when it fits
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
    double loss = 0.0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        TapeRow r = tape_row(b, valid, mat, theta_deg, rf, T, gain, grad_I, target_I, target_valid);
        if (!r.use) continue;
        const float w = gain * r.rf * r.gI;
        const int e = r.m * LIDAR_TABLE_SIZE + r.i;
        atomicAdd(&dst[e], (unsigned long long)to_fixed(w * (1.0f - r.f), scale));
        atomicAdd(&dst[e + 1], (unsigned long long)to_fixed(w * r.f, scale));
        atomicAdd(&dst[n_acc - 1], (unsigned long long)to_fixed(r.rf * r.R * r.gI, scale));
        loss += (double)r.res * (double)r.res;
    }
    // deterministic per-block loss partial (fixed shuffle order)
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    __shared__ double s_loss[kAdjThreads / 32];
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = loss;
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

// pass 3: back to floating point, normalised, accumulated into the outputs
__global__ void k_adj_finalize(int n_acc, const unsigned long long* __restrict__ acc,
                               const unsigned int* __restrict__ absmax_bits,
                               const unsigned long long* __restrict__ count, int mse,
                               const double* __restrict__ loss_partials, int n_partials, float* grad_table,
                               float* grad_gain, float* loss)
{
    const float scale = fixed_scale(*absmax_bits, *count);
    const unsigned long long N = *count;
    const double norm = mse ? (N ? 1.0 / (double)N : 0.0) : 1.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_acc; j += gridDim.x * blockDim.x) {
        const double v = (double)(long long)acc[j] / (double)scale * norm;
        if (j < n_acc - 1) {
            if (grad_table) grad_table[j] += (float)v;
        } else if (grad_gain) {
            *grad_gain += (float)v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        double t = 0.0;
        for (int k = 0; k < n_partials; ++k) t += loss_partials[k];
        *loss = mse ? (float)(N ? t / (double)N : 0.0) : 0.0f;
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
    cudaMemsetAsync(scratch, 0, 256 + (((size_t)n_acc * 8 + 255) / 256) * 256, s);
    int blocks = (int)((n + kAdjThreads - 1) / kAdjThreads);
    if (blocks > kAdjBlocks) blocks = kAdjBlocks;
    if (blocks < 1) blocks = 1;
    k_adj_absmax<<<blocks, kAdjThreads, 0, s>>>(n, valid, mat, theta_deg, rf, T, gain, grad_I, target_I,
                                                target_valid, absmax, count);
    const size_t smem = (size_t)n_acc * sizeof(unsigned long long);
    int use_shared = smem <= 96 * 1024;
    if (use_shared && smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k_adj_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            use_shared = 0;
        }
    }
    k_adj_accumulate<<<blocks, kAdjThreads, use_shared ? smem : 0, s>>>(
        n, valid, mat, theta_deg, rf, T, gain, grad_I, target_I, target_valid, absmax, count, acc, partials,
        use_shared);
    k_adj_finalize<<<(n_acc + 255) / 256, 256, 0, s>>>(n_acc, acc, absmax, count, target_I != nullptr, partials,
                                                       blocks, grad_table, grad_gain, loss);
    return cudaGetLastError();
}

}  // namespace lidar
