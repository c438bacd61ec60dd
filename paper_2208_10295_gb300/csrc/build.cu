// Linear BVH build (Karras, "Maximizing Parallelism in the Construction of
// BVHs, Octrees, and k-d Trees", HPG 2012), hand-written:
//   1. centroid bounds (block reduction + ordered-int atomics), index check
//   2. 63-bit Morton keys of the triangle centroids (21 bits per axis)
//   3. stable radix sort of (key, triangle index)
//   4. leaf-ordered triangle gather (vertices + original index, material, instance)
//   5. internal nodes from the longest common key prefixes (ties on equal keys
//      broken by the leaf index), parent links
//   6. bottom-up refit: each leaf climbs; the second thread to reach a node
//      writes both child boxes (exact FP32 min/max, no rounding) and the node
//      height; the first stops.  The root height bounds the traversal stack.
#include "common.cuh"

#include <utility>

namespace lidar {
namespace {

constexpr int kBuildThreads = 256;

__device__ __forceinline__ int float_to_ordered(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}

__device__ __forceinline__ float ordered_to_float(int i)
{
    return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
}

__device__ __forceinline__ float3 load_vert(const float* v, uint32_t i)
{
    return make_float3(v[3 * (int64_t)i], v[3 * (int64_t)i + 1], v[3 * (int64_t)i + 2]);
}

__global__ void k_init_bounds(int* bounds)
{
    if (threadIdx.x < 3) bounds[threadIdx.x] = float_to_ordered(INFINITY);
    else if (threadIdx.x < 6) bounds[threadIdx.x] = float_to_ordered(-INFINITY);
}

__device__ __forceinline__ float3 centroid(float3 a, float3 b, float3 c)
{
    const float k = 1.0f / 3.0f;
    return make_float3((a.x + b.x + c.x) * k, (a.y + b.y + c.y) * k, (a.z + b.z + c.z) * k);
}

__global__ void __launch_bounds__(kBuildThreads) k_centroid_bounds(const float* __restrict__ verts,
                                                                   int64_t n_verts,
                                                                   const uint32_t* __restrict__ tris,
                                                                   int64_t n, int* bounds, int* status)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t a = tris[3 * i], b = tris[3 * i + 1], c = tris[3 * i + 2];
        if ((int64_t)a >= n_verts || (int64_t)b >= n_verts || (int64_t)c >= n_verts) {
            raise_status(status, ST_INDEX);
            continue;
        }
        float3 ct = centroid(load_vert(verts, a), load_vert(verts, b), load_vert(verts, c));
        lo[0] = fminf(lo[0], ct.x); lo[1] = fminf(lo[1], ct.y); lo[2] = fminf(lo[2], ct.z);
        hi[0] = fmaxf(hi[0], ct.x); hi[1] = fmaxf(hi[1], ct.y); hi[2] = fmaxf(hi[2], ct.z);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[k], float_to_ordered(lo[k]));
            atomicMax(&bounds[3 + k], float_to_ordered(hi[k]));
        }
    }
}

// spread the low 21 bits of x so that bit i lands on bit 3i
__device__ __forceinline__ uint64_t spread3(uint64_t x)
{
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t quantize21(float v, float lo, float inv_ext)
{
    float q = (v - lo) * inv_ext * 2097151.0f;
    q = fminf(fmaxf(q, 0.0f), 2097151.0f);
    return (uint32_t)q;
}

__global__ void __launch_bounds__(kBuildThreads) k_morton(const float* __restrict__ verts,
                                                          const uint32_t* __restrict__ tris, int64_t n,
                                                          int64_t n_verts, const int* __restrict__ bounds,
                                                          uint64_t* __restrict__ keys,
                                                          uint32_t* __restrict__ vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float lo[3], inv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = ordered_to_float(bounds[k]);
        float ext = ordered_to_float(bounds[3 + k]) - lo[k];
        inv[k] = ext > 0.0f ? 1.0f / ext : 0.0f;
    }
    uint32_t a = tris[3 * i], b = tris[3 * i + 1], c = tris[3 * i + 2];
    uint64_t key = 0;
    if ((int64_t)a < n_verts && (int64_t)b < n_verts && (int64_t)c < n_verts) {
        float3 ct = centroid(load_vert(verts, a), load_vert(verts, b), load_vert(verts, c));
        key = (spread3(quantize21(ct.x, lo[0], inv[0])) << 2) | (spread3(quantize21(ct.y, lo[1], inv[1])) << 1) |
              spread3(quantize21(ct.z, lo[2], inv[2]));
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(kBuildThreads) k_gather(const float* __restrict__ verts, int64_t n_verts,
                                                          const uint32_t* __restrict__ tris,
                                                          const uint16_t* __restrict__ mat,
                                                          const uint32_t* __restrict__ inst,
                                                          const uint32_t* __restrict__ order, int64_t n,
                                                          float4* __restrict__ tris_out,
                                                          uint32_t* __restrict__ leaf_tri)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t t = order[i];
    uint32_t a = tris[3 * (int64_t)t], b = tris[3 * (int64_t)t + 1], c = tris[3 * (int64_t)t + 2];
    if ((int64_t)a >= n_verts || (int64_t)b >= n_verts || (int64_t)c >= n_verts) a = b = c = 0;
    float3 va = load_vert(verts, a), vb = load_vert(verts, b), vc = load_vert(verts, c);
    tris_out[3 * i + 0] = make_float4(va.x, va.y, va.z, __int_as_float((int)t));
    tris_out[3 * i + 1] = make_float4(vb.x, vb.y, vb.z, __int_as_float((int)(mat ? mat[t] : 0)));
    tris_out[3 * i + 2] = make_float4(vc.x, vc.y, vc.z, __int_as_float((int)(inst ? inst[t] : 0)));
    leaf_tri[i] = t;
}

// length of the common prefix of keys i and j; -1 outside [0, n)
__device__ __forceinline__ int delta(const uint64_t* __restrict__ keys, int64_t n, int64_t i, int64_t j)
{
    if (j < 0 || j >= n) return -1;
    uint64_t a = keys[i], b = keys[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void __launch_bounds__(kBuildThreads) k_karras(const uint64_t* __restrict__ keys, int64_t n,
                                                          float4* __restrict__ nodes,
                                                          int* __restrict__ parent_node,
                                                          int* __restrict__ parent_leaf)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    // direction of the node's key range
    const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(keys, n, i, i - d);
    // exponential then binary search for the far end of the range
    int64_t lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(keys, n, i, j);
    // split: last position of the range that still shares more than dnode bits with i
    int64_t s = 0;
    int64_t step = l;
    do {
        step = (step + 1) >> 1;
        if (delta(keys, n, i, i + (s + step) * d) > dnode) s += step;
    } while (step > 1);
    const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int left, right;
    if (lo == gamma) {
        left = ~(int)gamma;
        parent_leaf[gamma] = (int)i;
    } else {
        left = (int)gamma;
        parent_node[gamma] = (int)i;
    }
    if (hi == gamma + 1) {
        right = ~(int)(gamma + 1);
        parent_leaf[gamma + 1] = (int)i;
    } else {
        right = (int)(gamma + 1);
        parent_node[gamma + 1] = (int)i;
    }
    nodes[4 * i + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.0f, 0.0f);
    if (i == 0) parent_node[0] = -1;
}

struct Box {
    float lo[3], hi[3];
};

__device__ __forceinline__ Box leaf_box(const float4* __restrict__ tris, int leaf)
{
    float4 a = tris[3 * (int64_t)leaf], b = tris[3 * (int64_t)leaf + 1], c = tris[3 * (int64_t)leaf + 2];
    Box r;
    r.lo[0] = fminf(a.x, fminf(b.x, c.x)); r.hi[0] = fmaxf(a.x, fmaxf(b.x, c.x));
    r.lo[1] = fminf(a.y, fminf(b.y, c.y)); r.hi[1] = fmaxf(a.y, fmaxf(b.y, c.y));
    r.lo[2] = fminf(a.z, fminf(b.z, c.z)); r.hi[2] = fmaxf(a.z, fmaxf(b.z, c.z));
    return r;
}

__device__ __forceinline__ Box node_box(const float4* node_boxes, int node)
{
    float4 lo = __ldcg(&node_boxes[2 * (int64_t)node]);
    float4 hi = __ldcg(&node_boxes[2 * (int64_t)node + 1]);
    Box r;
    r.lo[0] = lo.x; r.lo[1] = lo.y; r.lo[2] = lo.z;
    r.hi[0] = hi.x; r.hi[1] = hi.y; r.hi[2] = hi.z;
    return r;
}

__global__ void __launch_bounds__(kBuildThreads) k_refit(const float4* __restrict__ tris, int64_t n,
                                                         float4* nodes, float4* node_boxes, int* heights,
                                                         const int* __restrict__ parent_node,
                                                         const int* __restrict__ parent_leaf, int* visits,
                                                         int* max_height)
{
    int64_t leaf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= n) return;
    int p = parent_leaf[leaf];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&visits[p], 1) == 0) return;  // the sibling subtree is not finished yet
        __threadfence();
        float4 n3 = __ldcg(&nodes[4 * (int64_t)p + 3]);
        int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
        Box L = cl < 0 ? leaf_box(tris, ~cl) : node_box(node_boxes, cl);
        Box R = cr < 0 ? leaf_box(tris, ~cr) : node_box(node_boxes, cr);
        int hl = cl < 0 ? 0 : __ldcg(&heights[cl]);
        int hr = cr < 0 ? 0 : __ldcg(&heights[cr]);
        nodes[4 * (int64_t)p + 0] = make_float4(L.lo[0], L.hi[0], L.lo[1], L.hi[1]);
        nodes[4 * (int64_t)p + 1] = make_float4(R.lo[0], R.hi[0], R.lo[1], R.hi[1]);
        nodes[4 * (int64_t)p + 2] = make_float4(L.lo[2], L.hi[2], R.lo[2], R.hi[2]);
        node_boxes[2 * (int64_t)p] = make_float4(fminf(L.lo[0], R.lo[0]), fminf(L.lo[1], R.lo[1]),
                                                 fminf(L.lo[2], R.lo[2]), 0.0f);
        node_boxes[2 * (int64_t)p + 1] = make_float4(fmaxf(L.hi[0], R.hi[0]), fmaxf(L.hi[1], R.hi[1]),
                                                     fmaxf(L.hi[2], R.hi[2]), 0.0f);
        int h = 1 + max(hl, hr);
        heights[p] = h;
        if (p == 0) atomicMax(max_height, h);
        p = parent_node[p];
    }
}

// a single triangle: one root whose right child box is empty
__global__ void k_single(const float4* __restrict__ tris, float4* nodes, int* max_height)
{
    Box L = leaf_box(tris, 0);
    nodes[0] = make_float4(L.lo[0], L.hi[0], L.lo[1], L.hi[1]);
    nodes[1] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    nodes[2] = make_float4(L.lo[2], L.hi[2], INFINITY, -INFINITY);
    nodes[3] = make_float4(__int_as_float(~0), __int_as_float(~0), 0.0f, 0.0f);
    *max_height = 1;
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t build_scratch_bytes(int64_t n)
{
    return align256(n * sizeof(uint64_t)) + align256(n * sizeof(uint32_t)) + align256(n * sizeof(int)) * 4 +
           align256((size_t)n * 2 * sizeof(float4)) + align256(64) + radix_sort_scratch_bytes(n);
}

cudaError_t build_ploc(cudaStream_t s, const float4* tris_sorted, int64_t n, float4* nodes_out, int* max_height_dev,
                       int radius, void* scratch, size_t scratch_bytes, unsigned long long* host_total, AreaW w);

cudaError_t build_lbvh(cudaStream_t s, const float* verts, int64_t n_verts, const uint32_t* tris,
                       const uint16_t* mat, const uint32_t* inst, int64_t n, float4* nodes_out,
                       float4* tris_out, uint32_t* leaf_tri_out, int* status, int* max_height_dev,
                       void* scratch, size_t scratch_bytes, int method, int radius, AreaW area_w)
{
    if (n == 0) return cudaSuccess;
    if (scratch_bytes < build_scratch_bytes(n)) return cudaErrorInvalidValue;
    char* p = (char*)scratch;
    uint64_t* keys = (uint64_t*)p; p += align256(n * sizeof(uint64_t));
    uint32_t* vals = (uint32_t*)p; p += align256(n * sizeof(uint32_t));
    int* parent_node = (int*)p; p += align256(n * sizeof(int));
    int* parent_leaf = (int*)p; p += align256(n * sizeof(int));
    int* visits = (int*)p; p += align256(n * sizeof(int));
    int* heights = (int*)p; p += align256(n * sizeof(int));
    float4* node_boxes = (float4*)p; p += align256((size_t)n * 2 * sizeof(float4));
    int* bounds = (int*)p; p += align256(64);
    void* sort_scratch = p;
    size_t sort_bytes = scratch_bytes - (size_t)(p - (char*)scratch);

    const int blocks = (int)((n + kBuildThreads - 1) / kBuildThreads);
    k_init_bounds<<<1, 32, 0, s>>>(bounds);
    const int red_blocks = blocks < 2048 ? blocks : 2048;
    k_centroid_bounds<<<red_blocks, kBuildThreads, 0, s>>>(verts, n_verts, tris, n, bounds, status);
    k_morton<<<blocks, kBuildThreads, 0, s>>>(verts, tris, n, n_verts, bounds, keys, vals);
    cudaError_t e = radix_sort_pairs_u64(s, keys, vals, n, 63, sort_scratch, sort_bytes);
    if (e != cudaSuccess) return e;
    k_gather<<<blocks, kBuildThreads, 0, s>>>(verts, n_verts, tris, mat, inst, vals, n, tris_out, leaf_tri_out);
    cudaMemsetAsync(max_height_dev, 0, sizeof(int), s);
    if (n == 1) {
        k_single<<<1, 1, 0, s>>>(tris_out, nodes_out, max_height_dev);
        return cudaGetLastError();
    }
    if (method == 1) {
        // clustering over the Morton-ordered leaves; the sort's buffers are free again
        unsigned long long total = 0;
        return build_ploc(s, tris_out, n, nodes_out, max_height_dev, radius, scratch, scratch_bytes, &total, area_w);
    }
    const int iblocks = (int)((n - 1 + kBuildThreads - 1) / kBuildThreads);
    k_karras<<<iblocks, kBuildThreads, 0, s>>>(keys, n, nodes_out, parent_node, parent_leaf);
    cudaMemsetAsync(visits, 0, n * sizeof(int), s);
    k_refit<<<blocks, kBuildThreads, 0, s>>>(tris_out, n, nodes_out, node_boxes, heights, parent_node, parent_leaf,
                                             visits, max_height_dev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// PLOC: Parallel Locally-Ordered Clustering (Meister and Bittner, "Parallel
// Locally-Ordered Clustering for Bounding Volume Hierarchy Construction",
// IEEE TVCG 2018), an alternative to the Karras hierarchy over the same
// Morton-ordered leaves.  Clusters start as the leaves; each iteration every
// cluster finds its nearest neighbour within `radius` positions of the
// cluster array (distance: surface area of the union box; ties to the lower
// position), mutual nearest pairs merge into a new node at the lower position,
// and the array is compacted in order.  Node ids count down from n - 2, so the
// last merge is the root at 0.  Boxes are exact FP32 min/max unions.
namespace {

struct PlocClusters {
    int* ref;        // ~leaf or node id
    float4* box;     // [2 per cluster] lo, hi
    int* height;
};

// half the weighted surface of the union of two boxes
__device__ __forceinline__ float union_half_area(float4 alo, float4 ahi, float4 blo, float4 bhi, AreaW w)
{
    const float dx = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
    const float dy = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
    const float dz = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
    return w.z * dx * dy + w.x * dy * dz + w.y * dz * dx;
}

__global__ void __launch_bounds__(kBuildThreads) k_ploc_init(const float4* __restrict__ tris, int64_t n,
                                                             PlocClusters C)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Box b = leaf_box(tris, (int)i);
    C.ref[i] = ~(int)i;
    C.box[2 * i] = make_float4(b.lo[0], b.lo[1], b.lo[2], 0.0f);
    C.box[2 * i + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], 0.0f);
    C.height[i] = 0;
}

__global__ void __launch_bounds__(kBuildThreads) k_ploc_nearest(PlocClusters C, int n, int radius, int* nn, AreaW w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 alo = C.box[2 * (int64_t)i], ahi = C.box[2 * (int64_t)i + 1];
    int best = -1;
    float best_d = INFINITY;
    const int lo = max(i - radius, 0), hi = min(i + radius, n - 1);
    for (int j = lo; j <= hi; ++j) {
        if (j == i) continue;
        const float d = union_half_area(alo, ahi, C.box[2 * (int64_t)j], C.box[2 * (int64_t)j + 1], w);
        if (d < best_d) {  // ascending j: ties keep the lower position
            best_d = d;
            best = j;
        }
    }
    nn[i] = best;
}

// flags: high word 1 if i creates a node, low word 1 if i's cluster survives
__global__ void __launch_bounds__(kBuildThreads) k_ploc_flags(const int* __restrict__ nn, int n, int force_pairs,
                                                              unsigned long long* flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = nn[i];
    bool merge_low, merged_away;
    if (force_pairs) {
        // no mutual pair anywhere (not expected): merge positions 2k, 2k+1
        merge_low = (i % 2 == 0) && i + 1 < n;
        merged_away = (i % 2 == 1);
    } else {
        const bool mutual = j >= 0 && nn[j] == i;
        merge_low = mutual && i < j;
        merged_away = mutual && j < i;
    }
    flags[i] = ((unsigned long long)(merge_low ? 1u : 0u) << 32) | (merged_away ? 0ull : 1ull);
}

__global__ void __launch_bounds__(kBuildThreads) k_ploc_merge(PlocClusters C, PlocClusters D, const int* __restrict__ nn,
                                                              int n, int force_pairs,
                                                              const unsigned long long* __restrict__ flags,
                                                              const unsigned long long* __restrict__ prefix,
                                                              int64_t id_base, float4* nodes, int* max_height)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long f = flags[i];
    if ((f & 0xFFFFFFFFull) == 0) return;  // merged into a lower position
    const int out = (int)(prefix[i] & 0xFFFFFFFFull);
    if ((f >> 32) == 0) {
        D.ref[out] = C.ref[i];
        D.box[2 * (int64_t)out] = C.box[2 * (int64_t)i];
        D.box[2 * (int64_t)out + 1] = C.box[2 * (int64_t)i + 1];
        D.height[out] = C.height[i];
        return;
    }
    const int j = force_pairs ? i + 1 : nn[i];
    const int64_t id = id_base - (int64_t)(prefix[i] >> 32);
    const float4 llo = C.box[2 * (int64_t)i], lhi = C.box[2 * (int64_t)i + 1];
    const float4 rlo = C.box[2 * (int64_t)j], rhi = C.box[2 * (int64_t)j + 1];
    nodes[4 * id + 0] = make_float4(llo.x, lhi.x, llo.y, lhi.y);
    nodes[4 * id + 1] = make_float4(rlo.x, rhi.x, rlo.y, rhi.y);
    nodes[4 * id + 2] = make_float4(llo.z, lhi.z, rlo.z, rhi.z);
    nodes[4 * id + 3] = make_float4(__int_as_float(C.ref[i]), __int_as_float(C.ref[j]), 0.0f, 0.0f);
    const int h = 1 + max(C.height[i], C.height[j]);
    D.ref[out] = (int)id;
    D.box[2 * (int64_t)out] = make_float4(fminf(llo.x, rlo.x), fminf(llo.y, rlo.y), fminf(llo.z, rlo.z), 0.0f);
    D.box[2 * (int64_t)out + 1] = make_float4(fmaxf(lhi.x, rhi.x), fmaxf(lhi.y, rhi.y), fmaxf(lhi.z, rhi.z), 0.0f);
    D.height[out] = h;
    if (id == 0) *max_height = h;
}

// exclusive scan of uint64 flags: per-block scans, one block over the block
// sums, then the block offsets added
constexpr int kScanItems = 1024;

__global__ void __launch_bounds__(kScanItems) k_scan_local(const unsigned long long* __restrict__ in, int n,
                                                          unsigned long long* out, unsigned long long* sums)
{
    __shared__ unsigned long long s[kScanItems];
    const int i = blockIdx.x * kScanItems + threadIdx.x;
    const unsigned long long v = i < n ? in[i] : 0ull;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanItems; o <<= 1) {
        const unsigned long long a = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
        __syncthreads();
        s[threadIdx.x] += a;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == kScanItems - 1) sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void __launch_bounds__(kScanItems) k_scan_sums(unsigned long long* sums, int m)
{
    __shared__ unsigned long long s[kScanItems];
    unsigned long long carry = 0;
    for (int base = 0; base < m; base += kScanItems) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < m ? sums[i] : 0ull;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kScanItems; o <<= 1) {
            const unsigned long long a = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
            __syncthreads();
            s[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < m) sums[i] = carry + s[threadIdx.x] - v;
        const unsigned long long total = s[kScanItems - 1];
        __syncthreads();
        carry += total;
    }
    if (threadIdx.x == 0) sums[m] = carry;
}

__global__ void __launch_bounds__(kScanItems) k_scan_add(unsigned long long* out, int n,
                                                        const unsigned long long* __restrict__ sums)
{
    const int i = blockIdx.x * kScanItems + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

}  // namespace

size_t ploc_scratch_bytes(int64_t n)
{
    const size_t m = (size_t)(n + kScanItems - 1) / kScanItems + 1;
    return 2 * (align256(n * sizeof(int)) + align256((size_t)n * 2 * sizeof(float4)) + align256(n * sizeof(int))) +
           align256(n * sizeof(int)) + 2 * align256(n * sizeof(unsigned long long)) + align256(m * 8) + 256;
}

cudaError_t build_ploc(cudaStream_t s, const float4* tris_sorted, int64_t n, float4* nodes_out, int* max_height_dev,
                       int radius, void* scratch, size_t scratch_bytes, unsigned long long* host_total, AreaW w)
{
    if (n < 2) return cudaErrorInvalidValue;
    if (scratch_bytes < ploc_scratch_bytes(n)) return cudaErrorInvalidValue;
    char* p = (char*)scratch;
    PlocClusters A, B;
    A.ref = (int*)p; p += align256(n * sizeof(int));
    A.box = (float4*)p; p += align256((size_t)n * 2 * sizeof(float4));
    A.height = (int*)p; p += align256(n * sizeof(int));
    B.ref = (int*)p; p += align256(n * sizeof(int));
    B.box = (float4*)p; p += align256((size_t)n * 2 * sizeof(float4));
    B.height = (int*)p; p += align256(n * sizeof(int));
    int* nn = (int*)p; p += align256(n * sizeof(int));
    unsigned long long* flags = (unsigned long long*)p; p += align256(n * sizeof(unsigned long long));
    unsigned long long* prefix = (unsigned long long*)p; p += align256(n * sizeof(unsigned long long));
    unsigned long long* sums = (unsigned long long*)p;
    const int blocks0 = (int)((n + kBuildThreads - 1) / kBuildThreads);
    k_ploc_init<<<blocks0, kBuildThreads, 0, s>>>(tris_sorted, n, A);
    int nc = (int)n;
    int64_t created = 0;
    for (int iter = 0; nc > 1; ++iter) {
        if (iter > 4 * n) return cudaErrorUnknown;
        const int blocks = (nc + kBuildThreads - 1) / kBuildThreads;
        const int sblocks = (nc + kScanItems - 1) / kScanItems;
        int force = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            k_ploc_nearest<<<blocks, kBuildThreads, 0, s>>>(A, nc, radius, nn, w);
            k_ploc_flags<<<blocks, kBuildThreads, 0, s>>>(nn, nc, force, flags);
            k_scan_local<<<sblocks, kScanItems, 0, s>>>(flags, nc, prefix, sums);
            k_scan_sums<<<1, kScanItems, 0, s>>>(sums, sblocks);
            k_scan_add<<<sblocks, kScanItems, 0, s>>>(prefix, nc, sums);
            cudaError_t e = cudaMemcpyAsync(host_total, sums + sblocks, sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            if ((*host_total >> 32) > 0) break;
            force = 1;  // no mutual pair: merge neighbours pairwise
        }
        const unsigned long long total = *host_total;
        k_ploc_merge<<<blocks, kBuildThreads, 0, s>>>(A, B, nn, nc, force, flags, prefix, (n - 2) - created,
                                                      nodes_out, max_height_dev);
        created += (int64_t)(total >> 32);
        nc = (int)(total & 0xFFFFFFFFull);
        std::swap(A, B);
    }
    return cudaGetLastError();
}

}  // namespace lidar

// ---------------------------------------------------------------------------
// Collapse of the binary hierarchy into a W-wide one (W = 4 or 8).  Top-down,
// one frontier of binary nodes per level: each becomes a wide node whose
// children are found by repeatedly opening the child with the largest surface
// area until W children or only leaves remain.  Slots of the next level are
// assigned by an exclusive scan, so the layout is breadth-first and
// deterministic.
//
// Wide node of G = W/4 groups of four children, 8G float4s: for axis a the
// lower planes of group g at (2a)G + g, the upper planes at (2a + 1)G + g, the
// child codes of group g at 6G + g (>= 0: wide node, < 0: ~leaf; empty slots
// have an empty box and code 0), then G float4s of metadata (128 bytes for
// W = 4, 256 for W = 8).  A node keeps its internal children in the first
// slots, in the order of their (consecutive) node ids, and its first metadata
// float4 holds the first internal child's id and the mask of leaf slots, so a
// traversal finds an internal child as first + slot.
//
// Alongside each frontier entry travels the number of stack entries its
// ancestors can leave behind: a traversal that descends into one hit internal
// child pushes at most the node's other internal children, so the deepest
// stack the tree can need is max over nodes of (ancestors' pushes + the
// node's internal children - 1).
namespace lidar {
namespace {

struct ChildBox {
    float lo[3], hi[3];
    int ref;  // binary node (>= 0) or ~leaf (< 0)
};

__device__ __forceinline__ void binary_child(const float4* __restrict__ bn, int node, int side, ChildBox& c)
{
    const float4 n0 = bn[4 * (int64_t)node + 0], n1 = bn[4 * (int64_t)node + 1];
    const float4 n2 = bn[4 * (int64_t)node + 2], n3 = bn[4 * (int64_t)node + 3];
    if (side == 0) {
        c.lo[0] = n0.x; c.hi[0] = n0.y; c.lo[1] = n0.z; c.hi[1] = n0.w; c.lo[2] = n2.x; c.hi[2] = n2.y;
        c.ref = __float_as_int(n3.x);
    } else {
        c.lo[0] = n1.x; c.hi[0] = n1.y; c.lo[1] = n1.z; c.hi[1] = n1.w; c.lo[2] = n2.z; c.hi[2] = n2.w;
        c.ref = __float_as_int(n3.y);
    }
}

__device__ __forceinline__ float half_area(const ChildBox& c, AreaW w)
{
    const float dx = c.hi[0] - c.lo[0], dy = c.hi[1] - c.lo[1], dz = c.hi[2] - c.lo[2];
    return w.z * dx * dy + w.x * dy * dz + w.y * dz * dx;
}

// children of binary node b; returns the number of internal ones
template <int W>
__device__ int gather_children(const float4* __restrict__ bn, int b, ChildBox ch[W], int& count, AreaW w)
{
    binary_child(bn, b, 0, ch[0]);
    binary_child(bn, b, 1, ch[1]);
    count = 2;
    while (count < W) {
        int best = -1;
        float best_a = -1.0f;
        for (int k = 0; k < count; ++k)
            if (ch[k].ref >= 0 && half_area(ch[k], w) > best_a) {
                best_a = half_area(ch[k], w);
                best = k;
            }
        if (best < 0) break;
        const int open = ch[best].ref;
        binary_child(bn, open, 0, ch[best]);
        binary_child(bn, open, 1, ch[count]);
        ++count;
    }
    int internal = 0;
    for (int k = 0; k < count; ++k) internal += ch[k].ref >= 0;
    return internal;
}

// ---- SAH-optimal choice of a wide node's children (a dynamic program over the
// binary tree, in the manner of Ylitie, Karras and Laine, HPG 2017).  Expected
// cost of a tree: c_node x SA(N) summed over its wide nodes N plus c_tri x
// SA(t) over its triangle children t (surface areas relative to the root's).
// For binary node n and a budget of i child slots (i = 1..W):
//   D(n, i) = min over j of C(left, j) + C(right, i - j)   (n spread over i slots)
//   C(n, 1) = c_node SA(n) + D(n, W)                        (n one slot: a wide node)
//   C(n, i) = min(C(n, 1), D(n, i)),  i >= 2
// with C(t, i) = c_tri SA(t) for a triangle.  Per node the argmin split of
// D(n, i) and whether C(n, 1) won are kept; a wide node at n takes the slots
// D(n, W)'s split gives its two children, expanded while they win.
struct CollapseDP {
    const int* parent_node;   // [n_binary] parent of each internal node (-1: root)
    const int* parent_leaf;   // [n_leaves] parent of each triangle
    float* cost;              // [n_binary][W] C(n, i)
    uint8_t* split;           // [n_binary][W] argmin j of D(n, i) (i >= 2)
    uint16_t* single;         // [n_binary] bit i: C(n, 1) <= D(n, i)
    unsigned* visits;         // [n_binary] children finished, bottom-up
    float c_node, c_tri;
    AreaW w;                  // face weights of the area measure (also the largest-area rule's)
};

__global__ void k_parents(const float4* __restrict__ bn, int n_binary, int* parent_node, int* parent_leaf)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_binary) return;
    const float4 n3 = bn[4 * (int64_t)n + 3];
    const int c[2] = {__float_as_int(n3.x), __float_as_int(n3.y)};
    for (int k = 0; k < 2; ++k) {
        if (c[k] >= 0) parent_node[c[k]] = n;
        else parent_leaf[~c[k]] = n;
    }
}

// one thread per triangle climbs towards the root; the second child to finish
// computes its parent's table, so every node is computed once, after both
// children
template <int W>
__global__ void k_collapse_dp(const float4* __restrict__ bn, int n_leaves, CollapseDP dp)
{
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= n_leaves) return;
    int node = dp.parent_leaf[leaf];
    while (node >= 0) {
        __threadfence();
        if (atomicAdd(&dp.visits[node], 1u) == 0u) return;  // the other child is still running
        __threadfence();
        ChildBox cb[2];
        float cc[2][W];
        for (int side = 0; side < 2; ++side) {
            binary_child(bn, node, side, cb[side]);
            if (cb[side].ref < 0) {
                const float v = dp.c_tri * half_area(cb[side], dp.w);
                for (int i = 0; i < W; ++i) cc[side][i] = v;
            } else {
                for (int i = 0; i < W; ++i) cc[side][i] = __ldcg(&dp.cost[(int64_t)cb[side].ref * W + i]);
            }
        }
        ChildBox u;
        for (int a = 0; a < 3; ++a) {
            u.lo[a] = fminf(cb[0].lo[a], cb[1].lo[a]);
            u.hi[a] = fmaxf(cb[0].hi[a], cb[1].hi[a]);
        }
        float D[W + 1];
        int J[W + 1];
        for (int i = 2; i <= W; ++i) {
            D[i] = INFINITY;
            J[i] = 1;
            for (int j = 1; j < i; ++j) {
                const float v = cc[0][j - 1] + cc[1][i - j - 1];
                if (v < D[i]) {
                    D[i] = v;
                    J[i] = j;
                }
            }
        }
        const float c1 = dp.c_node * half_area(u, dp.w) + D[W];
        unsigned mask = 0;
        float* out = dp.cost + (int64_t)node * W;
        uint8_t* sp = dp.split + (int64_t)node * W;
        out[0] = c1;
        sp[0] = 0;
        for (int i = 2; i <= W; ++i) {
            if (c1 <= D[i]) {
                out[i - 1] = c1;
                mask |= 1u << i;
            } else {
                out[i - 1] = D[i];
            }
            sp[i - 1] = (uint8_t)J[i];
        }
        dp.single[node] = (uint16_t)mask;
        node = dp.parent_node[node];
    }
}

// children of binary node b chosen by the dynamic program; returns the number
// of internal ones
template <int W>
__device__ int gather_children_dp(const float4* __restrict__ bn, int b, const CollapseDP& dp, ChildBox ch[W],
                                  int& count)
{
    int budget[W];
    binary_child(bn, b, 0, ch[0]);
    binary_child(bn, b, 1, ch[1]);
    const int j = dp.split[(int64_t)b * W + W - 1];
    budget[0] = j;
    budget[1] = W - j;
    count = 2;
    for (bool more = true; more;) {
        more = false;
        for (int k = 0; k < count; ++k) {
            const int x = ch[k].ref, i = budget[k];
            if (x < 0 || i < 2 || ((dp.single[x] >> i) & 1u)) continue;
            const int jx = dp.split[(int64_t)x * W + i - 1];
            binary_child(bn, x, 0, ch[k]);
            binary_child(bn, x, 1, ch[count]);
            budget[k] = jx;
            budget[count] = i - jx;
            ++count;
            more = true;
            break;
        }
    }
    int internal = 0;
    for (int k = 0; k < count; ++k) internal += ch[k].ref >= 0;
    return internal;
}

template <int W>
__device__ __forceinline__ int gather(const float4* __restrict__ bn, int b, const CollapseDP& dp, int use_dp,
                                      ChildBox ch[W], int& count)
{
    return use_dp ? gather_children_dp<W>(bn, b, dp, ch, count) : gather_children<W>(bn, b, ch, count, dp.w);
}

template <int W>
__global__ void k_collapse_count(const float4* __restrict__ bn, const int* __restrict__ frontier, int n,
                                 uint32_t* __restrict__ n_internal, const CollapseDP dp, int use_dp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ChildBox ch[W];
    int count;
    n_internal[i] = (uint32_t)gather<W>(bn, frontier[i], dp, use_dp, ch, count);
}

__global__ void __launch_bounds__(1024) k_collapse_scan(uint32_t* __restrict__ v, int n, uint32_t* total)
{
    __shared__ uint32_t s_sum[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(lo + per, n);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += v[i];
    s_sum[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t x = (threadIdx.x >= (unsigned)off) ? s_sum[threadIdx.x - off] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = threadIdx.x == 0 ? 0u : s_sum[threadIdx.x - 1];
    for (int i = lo; i < hi; ++i) {
        const uint32_t c = v[i];
        v[i] = run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) *total = s_sum[blockDim.x - 1];
}

// frontier entry i owns wide slot (slot_base + i); its internal children get
// slots next_base + offset[i] + k and enter the next frontier at offset[i] + k.
// With nodes == nullptr only the next frontier and the stack bound are made.
template <int W>
__global__ void k_collapse_write(const float4* __restrict__ bn, const int* __restrict__ frontier,
                                 const int* __restrict__ pushes_in, int n, const uint32_t* __restrict__ offset,
                                 int slot_base, int next_base, float4* __restrict__ nodes,
                                 int* __restrict__ next_frontier, int* __restrict__ pushes_out, int* stack_need,
                                 const CollapseDP dp, int use_dp)
{
    constexpr int G = W / 4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ChildBox ch[W];
    int count;
    const int internal = gather<W>(bn, frontier[i], dp, use_dp, ch, count);
    const int below = pushes_in[i] + (internal > 0 ? internal - 1 : 0);
    atomicMax(stack_need, below);
    {
        // internal children first, keeping their order (a stable partition)
        ChildBox tmp[W];
        int m = 0;
        for (int k = 0; k < count; ++k)
            if (ch[k].ref >= 0) tmp[m++] = ch[k];
        for (int k = 0; k < count; ++k)
            if (ch[k].ref < 0) tmp[m++] = ch[k];
        for (int k = 0; k < count; ++k) ch[k] = tmp[k];
    }
    float lo[3][W], hi[3][W];
    int code[W];
    int k_int = 0;
    unsigned leaf_mask = 0;
    for (int k = 0; k < W; ++k) {
        if (k < count) {
            for (int a = 0; a < 3; ++a) { lo[a][k] = ch[k].lo[a]; hi[a][k] = ch[k].hi[a]; }
            if (ch[k].ref >= 0) {
                const int j = (int)offset[i] + k_int++;
                code[k] = next_base + j;
                next_frontier[j] = ch[k].ref;
                pushes_out[j] = below;
            } else {
                code[k] = ch[k].ref;
                leaf_mask |= 1u << k;
            }
        } else {
            for (int a = 0; a < 3; ++a) { lo[a][k] = INFINITY; hi[a][k] = -INFINITY; }
            code[k] = 0;
        }
    }
    if (!nodes) return;
    float4* out = nodes + 8 * G * (int64_t)(slot_base + i);
    for (int g = 0; g < G; ++g) {
        const int c = 4 * g;
        for (int a = 0; a < 3; ++a) {
            out[(2 * a) * G + g] = make_float4(lo[a][c], lo[a][c + 1], lo[a][c + 2], lo[a][c + 3]);
            out[(2 * a + 1) * G + g] = make_float4(hi[a][c], hi[a][c + 1], hi[a][c + 2], hi[a][c + 3]);
        }
        out[6 * G + g] = make_float4(__int_as_float(code[c]), __int_as_float(code[c + 1]),
                                     __int_as_float(code[c + 2]), __int_as_float(code[c + 3]));
        out[7 * G + g] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    out[7 * G] = make_float4(__int_as_float(internal > 0 ? next_base + (int)offset[i] : 0),
                             __int_as_float((int)leaf_mask), 0.0f, 0.0f);
}

}  // namespace

size_t collapse_scratch_bytes(int64_t n_binary)
{
    const int64_t m = n_binary > 0 ? n_binary : 1;
    const size_t arr = ((m * sizeof(int) + 255) / 256) * 256;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    // frontier and push arrays, counts, total; then the dynamic program's
    // parents (nodes, triangles), costs and splits for up to 8 slots, flags, visits
    return 5 * arr + 256 + arr + al((m + 1) * sizeof(int)) + al(m * 8 * sizeof(float)) + al(m * 8) +
           al(m * sizeof(uint16_t)) + arr;
}

cudaError_t collapse_bvh(cudaStream_t s, int width, const float4* binary_nodes, int64_t n_binary, float4* nodes,
                         int64_t* n_wide, int* levels, int* stack_need, void* scratch, size_t scratch_bytes,
                         int sah_dp, float tri_cost, AreaW area_w)
{
    *n_wide = 0;
    *levels = 0;
    *stack_need = 0;
    if (width != 4 && width != 8) return cudaErrorInvalidValue;
    if (n_binary == 0) return cudaSuccess;
    if (scratch_bytes < collapse_scratch_bytes(n_binary)) return cudaErrorInvalidValue;
    const size_t arr = ((n_binary * sizeof(int) + 255) / 256) * 256;
    int* fa = (int*)scratch;
    int* fbuf = (int*)((char*)scratch + arr);
    int* pa = (int*)((char*)scratch + 2 * arr);
    int* pb = (int*)((char*)scratch + 3 * arr);
    uint32_t* counts = (uint32_t*)((char*)scratch + 4 * arr);
    uint32_t* total = (uint32_t*)((char*)scratch + 5 * arr);
    int* need = (int*)(total + 1);
    CollapseDP dp{};
    dp.w = area_w;  // the largest-area rule reads it too
    if (sah_dp && n_binary < 2) sah_dp = 0;  // a single triangle: nothing to choose
    if (sah_dp) {
        auto al = [](size_t b) { return (b + 255) / 256 * 256; };
        char* q = (char*)scratch + 5 * arr + 256;
        int* parent_node = (int*)q;
        q += arr;
        int* parent_leaf = (int*)q;
        q += al((n_binary + 1) * sizeof(int));
        dp.cost = (float*)q;
        q += al(n_binary * 8 * sizeof(float));
        dp.split = (uint8_t*)q;
        q += al(n_binary * 8);
        dp.single = (uint16_t*)q;
        q += al(n_binary * sizeof(uint16_t));
        dp.visits = (unsigned*)q;
        dp.parent_node = parent_node;
        dp.parent_leaf = parent_leaf;
        dp.c_node = 1.0f;
        dp.c_tri = tri_cost;
        cudaError_t e0 = cudaMemsetAsync(parent_node, 0xFF, (size_t)n_binary * sizeof(int), s);
        if (e0 == cudaSuccess) e0 = cudaMemsetAsync(dp.visits, 0, (size_t)n_binary * sizeof(unsigned), s);
        if (e0 != cudaSuccess) return e0;
        const int nb = (int)n_binary;
        k_parents<<<(nb + 255) / 256, 256, 0, s>>>(binary_nodes, nb, parent_node, parent_leaf);
        if (width == 4)
            k_collapse_dp<4><<<(nb + 1 + 255) / 256, 256, 0, s>>>(binary_nodes, nb + 1, dp);
        else
            k_collapse_dp<8><<<(nb + 1 + 255) / 256, 256, 0, s>>>(binary_nodes, nb + 1, dp);
        e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    const int use_dp = sah_dp ? 1 : 0;
    const int init[2] = {0, 0};  // root, no pushes above it
    cudaError_t e = cudaMemcpyAsync(fa, &init[0], sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pa, &init[1], sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(need, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    int n = 1, slot_base = 0;
    int64_t allocated = 1;
    int* cur = fa;
    int* nxt = fbuf;
    int* pcur = pa;
    int* pnxt = pb;
    while (n > 0) {
        const int blocks = (n + 255) / 256;
        if (width == 4) {
            k_collapse_count<4><<<blocks, 256, 0, s>>>(binary_nodes, cur, n, counts, dp, use_dp);
            k_collapse_scan<<<1, 1024, 0, s>>>(counts, n, total);
            k_collapse_write<4><<<blocks, 256, 0, s>>>(binary_nodes, cur, pcur, n, counts, slot_base,
                                                      (int)allocated, nodes, nxt, pnxt, need, dp, use_dp);
        } else {
            k_collapse_count<8><<<blocks, 256, 0, s>>>(binary_nodes, cur, n, counts, dp, use_dp);
            k_collapse_scan<<<1, 1024, 0, s>>>(counts, n, total);
            k_collapse_write<8><<<blocks, 256, 0, s>>>(binary_nodes, cur, pcur, n, counts, slot_base,
                                                      (int)allocated, nodes, nxt, pnxt, need, dp, use_dp);
        }
        uint32_t next_n = 0;
        e = cudaMemcpyAsync(&next_n, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        slot_base = (int)allocated;
        allocated += next_n;
        n = (int)next_n;
        std::swap(cur, nxt);
        std::swap(pcur, pnxt);
        ++*levels;
    }
    e = cudaMemcpyAsync(stack_need, need, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *n_wide = allocated;
    return cudaGetLastError();
}

}  // namespace lidar

// ---------------------------------------------------------------------------
// Treelet restructuring of the binary hierarchy (Karras and Aila, "Fast
// Parallel Construction of High-Quality Bounding Volume Hierarchies", HPG
// 2013), written here for one thread per treelet.  Cost of a tree under the
// surface-area model: c_node x A(n) over its internal nodes plus c_tri x A(t)
// over its triangles (A: half the surface area of the box).  One round climbs
// the tree bottom-up (the second child to finish processes its parent, so a
// node is processed after its whole subtree).  At node n the thread forms a
// treelet: starting from n's two children it replaces the treelet leaf of
// largest area that is an internal node by that node's children, until there
// are kTreeletLeaves leaves or none is internal.  A dynamic program over the
// subsets S of the treelet's leaves gives the cheapest binary tree over them:
//   c({l}) = cost of leaf l's subtree,
//   c(S)   = c_node x A(S) + min over partitions S = P + Q of c(P) + c(Q).
// If that is cheaper than the treelet's current shape, its internal nodes
// (n first, so n's parent keeps pointing at it) are rewritten in the new
// shape with exact FP32 min/max child boxes.  Only the topology above the
// treelet's leaves changes, so the result is again a valid hierarchy over the
// same triangles.  Every decision depends only on the subtree below the
// node, so the result does not depend on the order threads run in.
namespace lidar {
namespace {

constexpr int kTreeletLeaves = 7;

struct TreeletArgs {
    const float4* tris;
    int n_leaves;
    int n_binary;
    float4* nodes;            // binary nodes, rewritten in place
    const int* parent_node;   // [n_binary], -1 at the root
    const int* parent_leaf;   // [n_leaves]
    unsigned* visits;         // [n_binary] children finished, zero at the start of a round
    float* cost;              // [n_binary] surface-area cost of each node's subtree
    unsigned long long* changed;  // treelets rewritten in the round
    int* status;              // ST_BOUNDS: a child reference out of range, or a climb longer than the bound
    float c_node, c_tri;
    AreaW w;                  // face weights of the area measure
};

// longest climb a valid hierarchy of up to 2^31 triangles can need is far
// below this; a longer one means a broken tree (a cycle), which ends the climb
constexpr int kTreeletMaxClimb = 4096;

struct TBox {
    float lo[3], hi[3];
};

__device__ __forceinline__ float tbox_area(const TBox& b, AreaW w)
{
    const float dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return w.z * dx * dy + w.x * dy * dz + w.y * dz * dx;
}

__device__ __forceinline__ void tbox_grow(TBox& a, const TBox& b)
{
    for (int k = 0; k < 3; ++k) {
        a.lo[k] = fminf(a.lo[k], b.lo[k]);
        a.hi[k] = fmaxf(a.hi[k], b.hi[k]);
    }
}

// child `side` of binary node `node` (read through L2: other threads of the
// round may have written it)
__device__ __forceinline__ void treelet_child(const float4* nodes, int node, int side, int& ref, TBox& b)
{
    const float4 n0 = __ldcg(&nodes[4 * (int64_t)node + 0]), n1 = __ldcg(&nodes[4 * (int64_t)node + 1]);
    const float4 n2 = __ldcg(&nodes[4 * (int64_t)node + 2]), n3 = __ldcg(&nodes[4 * (int64_t)node + 3]);
    if (side == 0) {
        b.lo[0] = n0.x; b.hi[0] = n0.y; b.lo[1] = n0.z; b.hi[1] = n0.w; b.lo[2] = n2.x; b.hi[2] = n2.y;
        ref = __float_as_int(n3.x);
    } else {
        b.lo[0] = n1.x; b.hi[0] = n1.y; b.lo[1] = n1.z; b.hi[1] = n1.w; b.lo[2] = n2.z; b.hi[2] = n2.w;
        ref = __float_as_int(n3.y);
    }
}

__device__ __forceinline__ bool ref_ok(const TreeletArgs& a, int ref)
{
    return ref >= 0 ? ref < a.n_binary : ~ref < a.n_leaves;
}

__device__ __forceinline__ float subtree_cost(const TreeletArgs& a, int ref, const TBox& b)
{
    return ref < 0 ? a.c_tri * tbox_area(b, a.w) : __ldcg(&a.cost[ref]);
}

__device__ void treelet_node(const TreeletArgs& a, int node)
{
    int lref[kTreeletLeaves];
    TBox lbox[kTreeletLeaves];
    float lcost[kTreeletLeaves];
    int inner[kTreeletLeaves - 1];
    treelet_child(a.nodes, node, 0, lref[0], lbox[0]);
    treelet_child(a.nodes, node, 1, lref[1], lbox[1]);
    if (!ref_ok(a, lref[0]) || !ref_ok(a, lref[1])) {
        raise_status(a.status, ST_BOUNDS);
        return;
    }
    lcost[0] = subtree_cost(a, lref[0], lbox[0]);
    lcost[1] = subtree_cost(a, lref[1], lbox[1]);
    TBox whole = lbox[0];
    tbox_grow(whole, lbox[1]);
    // the node's cost in its current shape
    const float c_now = a.c_node * tbox_area(whole, a.w) + lcost[0] + lcost[1];
    inner[0] = node;
    int k = 2, n_inner = 1;
    while (k < kTreeletLeaves) {
        int best = -1;
        float best_a = -1.0f;
        for (int i = 0; i < k; ++i)
            if (lref[i] >= 0 && tbox_area(lbox[i], a.w) > best_a) {
                best_a = tbox_area(lbox[i], a.w);
                best = i;
            }
        if (best < 0) break;
        const int open = lref[best];
        inner[n_inner++] = open;
        treelet_child(a.nodes, open, 0, lref[best], lbox[best]);
        treelet_child(a.nodes, open, 1, lref[k], lbox[k]);
        if (!ref_ok(a, lref[best]) || !ref_ok(a, lref[k])) {
            raise_status(a.status, ST_BOUNDS);
            return;
        }
        lcost[best] = subtree_cost(a, lref[best], lbox[best]);
        lcost[k] = subtree_cost(a, lref[k], lbox[k]);
        ++k;
    }
    if (k < 3) {
        a.cost[node] = c_now;
        return;
    }
    // the cheapest binary tree over the k leaves: subsets in increasing order
    // (every proper subset of S is smaller than S); each partition once (P
    // holds S's lowest leaf)
    float c[1 << kTreeletLeaves];
    unsigned char split[1 << kTreeletLeaves];
    const int full = (1 << k) - 1;
    for (int s = 1; s <= full; ++s) {
        if ((s & (s - 1)) == 0) {
            c[s] = lcost[__ffs(s) - 1];
            split[s] = 0;
            continue;
        }
        TBox u;
        bool first = true;
        for (int i = 0; i < k; ++i)
            if (s & (1 << i)) {
                if (first) u = lbox[i];
                else tbox_grow(u, lbox[i]);
                first = false;
            }
        const int low = s & -s;
        float best = INFINITY;
        int bp = low;
        for (int p = (s - 1) & s; p; p = (p - 1) & s) {
            if (!(p & low)) continue;
            const float v = c[p] + c[s ^ p];
            if (v < best) {
                best = v;
                bp = p;
            }
        }
        c[s] = a.c_node * tbox_area(u, a.w) + best;
        split[s] = (unsigned char)bp;
    }
    // keep the current shape unless the optimum is clearly cheaper (it is
    // one of the shapes the program compares, so it is never dearer beyond
    // rounding)
    if (!(c[full] < c_now * (1.0f - 1e-5f))) {
        a.cost[node] = c_now;
        return;
    }
    // rewrite: subset S at internal node id, its parts as leaves or the next
    // internal nodes of the treelet
    int st_s[kTreeletLeaves], st_id[kTreeletLeaves];
    int sp = 0, next = 1;
    st_s[sp] = full;
    st_id[sp++] = node;
    while (sp > 0) {
        --sp;
        const int s = st_s[sp], id = st_id[sp];
        const int part[2] = {split[s], s ^ split[s]};
        int ref[2];
        TBox box[2];
        for (int side = 0; side < 2; ++side) {
            const int x = part[side];
            bool first = true;
            for (int i = 0; i < k; ++i)
                if (x & (1 << i)) {
                    if (first) box[side] = lbox[i];
                    else tbox_grow(box[side], lbox[i]);
                    first = false;
                }
            if ((x & (x - 1)) == 0) {
                ref[side] = lref[__ffs(x) - 1];
            } else {
                ref[side] = inner[next++];
                st_s[sp] = x;
                st_id[sp++] = ref[side];
            }
        }
        const TBox& L = box[0];
        const TBox& R = box[1];
        a.nodes[4 * (int64_t)id + 0] = make_float4(L.lo[0], L.hi[0], L.lo[1], L.hi[1]);
        a.nodes[4 * (int64_t)id + 1] = make_float4(R.lo[0], R.hi[0], R.lo[1], R.hi[1]);
        a.nodes[4 * (int64_t)id + 2] = make_float4(L.lo[2], L.hi[2], R.lo[2], R.hi[2]);
        a.nodes[4 * (int64_t)id + 3] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), 0.0f, 0.0f);
        a.cost[id] = c[s];
    }
    atomicAdd(a.changed, 1ull);
}

__global__ void __launch_bounds__(128) k_treelet_round(TreeletArgs a)
{
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= a.n_leaves) return;
    int node = a.parent_leaf[leaf];
    for (int step = 0; node >= 0; ++step) {
        if (node >= a.n_binary || step >= kTreeletMaxClimb) {
            raise_status(a.status, ST_BOUNDS);
            return;
        }
        __threadfence();
        if (atomicAdd(&a.visits[node], 1u) == 0u) return;  // the other child is still running
        __threadfence();
        treelet_node(a, node);
        node = a.parent_node[node];
    }
}

__global__ void k_parents_reset(int* parent_node, int n_binary)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_binary) parent_node[i] = -1;
}

}  // namespace

size_t treelet_scratch_bytes(int64_t n_tris)
{
    // parents of nodes and leaves, visit counters, costs, heights, node boxes, counter
    return 5 * align256(n_tris * sizeof(int)) + align256((size_t)n_tris * 2 * sizeof(float4)) + 256;
}

cudaError_t restructure_treelets(cudaStream_t s, const float4* tris, int64_t n, float4* nodes, int* max_height_dev,
                                 int rounds, float tri_cost, void* scratch, size_t scratch_bytes,
                                 unsigned long long* changed_host, int* status, AreaW area_w)
{
    if (changed_host) *changed_host = 0;
    if (n < 3 || rounds <= 0) return cudaSuccess;
    if (scratch_bytes < treelet_scratch_bytes(n)) return cudaErrorInvalidValue;
    const int n_binary = (int)(n - 1);
    char* p = (char*)scratch;
    int* parent_node = (int*)p; p += align256(n * sizeof(int));
    int* parent_leaf = (int*)p; p += align256(n * sizeof(int));
    unsigned* visits = (unsigned*)p; p += align256(n * sizeof(int));
    float* cost = (float*)p; p += align256(n * sizeof(float));
    int* heights = (int*)p; p += align256(n * sizeof(int));
    float4* node_boxes = (float4*)p; p += align256((size_t)n * 2 * sizeof(float4));
    unsigned long long* changed = (unsigned long long*)p;
    const int nb_blocks = (n_binary + 255) / 256;
    TreeletArgs a{tris, (int)n, n_binary, nodes, parent_node, parent_leaf, visits, cost, changed, status,
                  1.0f, tri_cost, area_w};
    cudaError_t e = cudaMemsetAsync(changed, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    for (int r = 0; r < rounds; ++r) {
        k_parents_reset<<<nb_blocks, 256, 0, s>>>(parent_node, n_binary);
        k_parents<<<nb_blocks, 256, 0, s>>>(nodes, n_binary, parent_node, parent_leaf);
        e = cudaMemsetAsync(visits, 0, (size_t)n_binary * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        k_treelet_round<<<(int)((n + 127) / 128), 128, 0, s>>>(a);
    }
    // parents, heights and the root height of the final shape (the boxes the
    // refit writes are the same exact unions)
    k_parents_reset<<<nb_blocks, 256, 0, s>>>(parent_node, n_binary);
    k_parents<<<nb_blocks, 256, 0, s>>>(nodes, n_binary, parent_node, parent_leaf);
    e = cudaMemsetAsync(visits, 0, (size_t)n_binary * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(max_height_dev, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_refit<<<(int)((n + kBuildThreads - 1) / kBuildThreads), kBuildThreads, 0, s>>>(
        tris, n, nodes, node_boxes, heights, parent_node, parent_leaf, (int*)visits, max_height_dev);
    e = cudaGetLastError();
    if (e == cudaSuccess && changed_host)
        e = cudaMemcpyAsync(changed_host, changed, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    return e;
}

}  // namespace lidar
