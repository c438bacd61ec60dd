// Stable LSD radix sort of (key, value) pairs, hand-written.
//
// Each pass sorts by one 4-bit digit with three kernels ("reduce, then scan,
// then scatter"):
//   upsweep   : per tile digit histogram, written digit-major [16][n_tiles]
//   scan      : one block turns the histogram into exclusive global offsets
//   downsweep : per tile stable ranking (warp match + cross-warp prefix per
//               round of 256 keys) and scatter to offset[digit][tile] + rank.
// Keys are read in a striped layout (key index = tile*TILE + round*256 + tid),
// so ordering by (round, warp, lane) is the input order and the pass is stable.
#include "common.cuh"

namespace lidar {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 4;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortWarps = kSortThreads / 32;

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_upsweep(const K* __restrict__ keys, int64_t n, int shift,
                                                          int n_tiles, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t s_cnt[kRadix];
    if (threadIdx.x < kRadix) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint32_t local[kRadix];
#pragma unroll
    for (int d = 0; d < kRadix; ++d) local[d] = 0;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < n) {
            uint32_t dg = (uint32_t)(keys[idx] >> shift) & (kRadix - 1);
#pragma unroll
            for (int d = 0; d < kRadix; ++d) local[d] += (dg == (uint32_t)d);
        }
    }
    // warp-reduce each digit count, one shared atomic per warp and digit
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 0; d < kRadix; ++d) {
        uint32_t v = local[d];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(&s_cnt[d], v);
    }
    __syncthreads();
    if (threadIdx.x < kRadix) counts[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = s_cnt[threadIdx.x];
}

// Exclusive scan of `n` counts in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_counts(uint32_t* __restrict__ counts, int64_t n)
{
    __shared__ uint32_t s_sum[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = (int64_t)threadIdx.x * per;
    const int64_t hi = min(lo + per, n);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += counts[i];
    s_sum[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 partial sums
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = (threadIdx.x >= (unsigned)off) ? s_sum[threadIdx.x - off] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = (threadIdx.x == 0) ? 0u : s_sum[threadIdx.x - 1];
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t c = counts[i];
        counts[i] = run;
        run += c;
    }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_downsweep(const K* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            K* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out, int64_t n,
                                                            int shift, int n_tiles,
                                                            const uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t s_off[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_wcnt[kSortWarps][kRadix];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < kRadix) {
        s_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
        s_base[threadIdx.x] = 0;
    }
    if (threadIdx.x < kSortWarps * kRadix) (&s_wcnt[0][0])[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        const bool ok = idx < n;
        K key = ok ? keys_in[idx] : (K)0;
        uint32_t val = ok ? vals_in[idx] : 0u;
        uint32_t dg = ok ? ((uint32_t)(key >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        uint32_t wrank = __popc(peers & lt_mask);
        if (ok && wrank == 0) s_wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < kRadix) {
            uint32_t run = s_base[threadIdx.x];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = s_wcnt[w][threadIdx.x];
                s_wcnt[w][threadIdx.x] = run;
                run += c;
            }
            s_base[threadIdx.x] = run;
        }
        __syncthreads();
        if (ok) {
            uint32_t pos = s_off[dg] + s_wcnt[warp][dg] + wrank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        if (threadIdx.x < kSortWarps * kRadix) (&s_wcnt[0][0])[threadIdx.x] = 0;
        __syncthreads();
    }
}

template <typename K>
cudaError_t radix_sort_pairs(cudaStream_t s, K* keys, uint32_t* vals, int64_t n, int key_bits, void* scratch,
                             size_t scratch_bytes)
{
    if (n <= 1) return cudaSuccess;
    if (scratch_bytes < radix_sort_scratch_bytes(n)) return cudaErrorInvalidValue;
    const int n_tiles = (int)((n + kSortTile - 1) / kSortTile);
    char* p = (char*)scratch;
    K* alt_keys = (K*)p;
    p += ((n * sizeof(uint64_t) + 255) / 256) * 256;
    uint32_t* alt_vals = (uint32_t*)p;
    p += ((n * sizeof(uint32_t) + 255) / 256) * 256;
    uint32_t* counts = (uint32_t*)p;
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    K* kin = keys;
    K* kout = alt_keys;
    uint32_t* vin = vals;
    uint32_t* vout = alt_vals;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kRadixBits;
        k_upsweep<K><<<n_tiles, kSortThreads, 0, s>>>(kin, n, shift, n_tiles, counts);
        k_scan_counts<<<1, 1024, 0, s>>>(counts, (int64_t)kRadix * n_tiles);
        k_downsweep<K><<<n_tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, n_tiles, counts);
        K* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys) {
        cudaMemcpyAsync(keys, kin, n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n)
{
    const int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    return ((n * sizeof(uint64_t) + 255) / 256) * 256 + ((n * sizeof(uint32_t) + 255) / 256) * 256 +
           (size_t)kRadix * n_tiles * sizeof(uint32_t) + 256;
}

cudaError_t radix_sort_pairs_u64(cudaStream_t s, uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                 void* scratch, size_t scratch_bytes)
{
    return radix_sort_pairs<uint64_t>(s, keys, vals, n, key_bits, scratch, scratch_bytes);
}

cudaError_t radix_sort_pairs_u32(cudaStream_t s, uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                 void* scratch, size_t scratch_bytes)
{
    return radix_sort_pairs<uint32_t>(s, keys, vals, n, key_bits, scratch, scratch_bytes);
}

}  // namespace lidar
