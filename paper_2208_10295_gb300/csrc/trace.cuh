// Device-side ray geometry: world ray, sub-rays, robust box test, watertight
// triangle test and closest-hit BVH traversal.  Shared by the cast kernel and
// the brute-force debug kernel so both use bit-identical arithmetic.
#pragma once
#include "common.cuh"

namespace lidar {

constexpr float kTEps = 1e-4f;
// Conservative slab test (Ize, "Robust BVH Ray Traversal", JCGT 2013): the far
// slab distance is scaled by 1 + 2 gamma_3, gamma_3 = 3u / (1 - 3u), u = 2^-24;
// rounded up here to 1 + 2^-21.
constexpr float kFarScale = 1.0f + 4.76837158203125e-07f;
// pruning against the current closest hit keeps a slightly wider margin
constexpr float kBestScale = 1.0f + 9.5367431640625e-07f;

// Checked builds (-DLIDAR_BOUNDS): every traversal tests each node and
// triangle index against its array before reading it.  A bad index (corrupt
// scene data) ends the traversal with h.leaf = kBadIndex and false, which the
// cast reports as a bounds error in the status word, instead of reading
// outside the arrays.  Normal builds compile the tests away.
#ifdef LIDAR_BOUNDS
constexpr bool kBoundsChecks = true;
#else
constexpr bool kBoundsChecks = false;
#endif
constexpr int kBadIndex = -2;

__device__ __forceinline__ bool index_ok(int64_t i, int64_t n)
{
    return !kBoundsChecks || (i >= 0 && i < n);
}

struct RayW {
    float ox, oy, oz;
    float dx, dy, dz;
};

// World ray: o = pose translation, d_w[r] = fma(R[r][2], d2, fma(R[r][1], d1, R[r][0] * d0)).
__device__ __forceinline__ RayW world_ray(const float* pose, float d0, float d1, float d2)
{
    RayW r;
    r.dx = __fmaf_rn(pose[2], d2, __fmaf_rn(pose[1], d1, __fmul_rn(pose[0], d0)));
    r.dy = __fmaf_rn(pose[6], d2, __fmaf_rn(pose[5], d1, __fmul_rn(pose[4], d0)));
    r.dz = __fmaf_rn(pose[10], d2, __fmaf_rn(pose[9], d1, __fmul_rn(pose[8], d0)));
    r.ox = pose[3];
    r.oy = pose[7];
    r.oz = pose[11];
    return r;
}

// Sub-ray k of a beam: k = 0 is the beam; otherwise, with u = (d x z)/|d x z|
// (d x x when |d x z| < 1e-3), v = d x u: w = (d + alpha u) + beta v,
// direction w / |w|.  Every operation is rounded as written (no contraction).
__device__ __forceinline__ void subray_dir(float& dx, float& dy, float& dz, float alpha, float beta)
{
    const float n2 = __fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dx, dx));
    float c0, c1, c2;
    if (__fsqrt_rn(n2) >= 1e-3f) {
        c0 = dy; c1 = -dx; c2 = 0.0f;
    } else {
        c0 = 0.0f; c1 = dz; c2 = -dy;
    }
    const float cc = __fadd_rn(__fadd_rn(__fmul_rn(c0, c0), __fmul_rn(c1, c1)), __fmul_rn(c2, c2));
    const float s = __fsqrt_rn(cc);
    const float u0 = __fdiv_rn(c0, s), u1 = __fdiv_rn(c1, s), u2 = __fdiv_rn(c2, s);
    const float v0 = __fsub_rn(__fmul_rn(dy, u2), __fmul_rn(dz, u1));
    const float v1 = __fsub_rn(__fmul_rn(dz, u0), __fmul_rn(dx, u2));
    const float v2 = __fsub_rn(__fmul_rn(dx, u1), __fmul_rn(dy, u0));
    const float w0 = __fadd_rn(__fadd_rn(dx, __fmul_rn(alpha, u0)), __fmul_rn(beta, v0));
    const float w1 = __fadd_rn(__fadd_rn(dy, __fmul_rn(alpha, u1)), __fmul_rn(beta, v1));
    const float w2 = __fadd_rn(__fadd_rn(dz, __fmul_rn(alpha, u2)), __fmul_rn(beta, v2));
    const float ww = __fadd_rn(__fadd_rn(__fmul_rn(w0, w0), __fmul_rn(w1, w1)), __fmul_rn(w2, w2));
    const float sw = __fsqrt_rn(ww);
    dx = __fdiv_rn(w0, sw);
    dy = __fdiv_rn(w1, sw);
    dz = __fdiv_rn(w2, sw);
}

// Per-ray constants of the watertight test (Woop, Benthin, Wald, "Watertight
// Ray/Triangle Intersection", JCGT 2013) and of the slab test.
struct RayPre {
    float ox, oy, oz;
    float ix, iy, iz;     // correctly rounded reciprocals of the direction
    int kx, ky, kz;       // kz: dominant axis; (kx, ky) keep the winding
    float Sx, Sy, Sz;     // shear constants
};

__device__ __forceinline__ float sel3(float a, float b, float c, int k)
{
    return k == 0 ? a : (k == 1 ? b : c);
}

__device__ __forceinline__ RayPre prepare_ray(const RayW& r)
{
    RayPre p;
    p.ox = r.ox; p.oy = r.oy; p.oz = r.oz;
    p.ix = __frcp_rn(r.dx);
    p.iy = __frcp_rn(r.dy);
    p.iz = __frcp_rn(r.dz);
    const float ax = fabsf(r.dx), ay = fabsf(r.dy), az = fabsf(r.dz);
    int kz = (ax > ay) ? ((ax > az) ? 0 : 2) : ((ay > az) ? 1 : 2);
    int kx = kz + 1; if (kx == 3) kx = 0;
    int ky = kx + 1; if (ky == 3) ky = 0;
    const float dkz = sel3(r.dx, r.dy, r.dz, kz);
    if (dkz < 0.0f) { int t = kx; kx = ky; ky = t; }
    p.kx = kx; p.ky = ky; p.kz = kz;
    p.Sx = __fdiv_rn(sel3(r.dx, r.dy, r.dz, kx), dkz);
    p.Sy = __fdiv_rn(sel3(r.dx, r.dy, r.dz, ky), dkz);
    p.Sz = __frcp_rn(dkz);
    return p;
}

struct HitRec {
    float t;
    float cull;       // t * kBestScale: boxes entering beyond this are pruned
    uint32_t idx;     // original triangle index (ties: lowest wins)
    int leaf;         // leaf position, -1 for no hit
};

// Watertight, two-sided ray/triangle test; updates `h` when the triangle is
// closer (or equally close with a lower original index).
__device__ __forceinline__ void intersect_triangle(const float4* __restrict__ tris, int leaf, const RayPre& p,
                                                   float t_max, HitRec& h)
{
    const float4 a = __ldg(&tris[3 * (int64_t)leaf]);
    const float4 b = __ldg(&tris[3 * (int64_t)leaf + 1]);
    const float4 c = __ldg(&tris[3 * (int64_t)leaf + 2]);
    const float A0 = __fsub_rn(a.x, p.ox), A1 = __fsub_rn(a.y, p.oy), A2 = __fsub_rn(a.z, p.oz);
    const float B0 = __fsub_rn(b.x, p.ox), B1 = __fsub_rn(b.y, p.oy), B2 = __fsub_rn(b.z, p.oz);
    const float C0 = __fsub_rn(c.x, p.ox), C1 = __fsub_rn(c.y, p.oy), C2 = __fsub_rn(c.z, p.oz);
    const float Akz = sel3(A0, A1, A2, p.kz), Bkz = sel3(B0, B1, B2, p.kz), Ckz = sel3(C0, C1, C2, p.kz);
    const float Ax = __fmaf_rn(-p.Sx, Akz, sel3(A0, A1, A2, p.kx));
    const float Ay = __fmaf_rn(-p.Sy, Akz, sel3(A0, A1, A2, p.ky));
    const float Bx = __fmaf_rn(-p.Sx, Bkz, sel3(B0, B1, B2, p.kx));
    const float By = __fmaf_rn(-p.Sy, Bkz, sel3(B0, B1, B2, p.ky));
    const float Cx = __fmaf_rn(-p.Sx, Ckz, sel3(C0, C1, C2, p.kx));
    const float Cy = __fmaf_rn(-p.Sy, Ckz, sel3(C0, C1, C2, p.ky));
    // edge functions, antisymmetric under swapping the edge's end points
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        // exact products in double decide edge cases consistently
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return;
    const float Az = __fmul_rn(p.Sz, Akz), Bz = __fmul_rn(p.Sz, Bkz), Cz = __fmul_rn(p.Sz, Ckz);
    const float T = __fmaf_rn(W, Cz, __fmaf_rn(V, Bz, __fmul_rn(U, Az)));
    const float t = __fdiv_rn(T, det);
    if (!(t > kTEps && t <= t_max)) return;
    const uint32_t idx = (uint32_t)__float_as_int(a.w);
    if (t < h.t || (t == h.t && idx < h.idx)) {
        h.t = t;
        h.idx = idx;
        h.leaf = leaf;
        h.cull = t * kBestScale;
    }
}

// Slab test of the two child boxes of one node.  Entry and exit planes are
// chosen by the sign of the direction (not by min/max of the two slab
// distances): a ray parallel to an axis and lying exactly in a box plane gives
// 0 * inf = NaN there, which fmaxf/fminf then ignore, leaving that axis
// unconstrained as it should be for a ray inside the closed slab.
__device__ __forceinline__ float slab_t(float plane, float o, float inv)
{
    return __fmul_rn(__fsub_rn(plane, o), inv);
}

__device__ __forceinline__ void child_boxes(const float4 n0, const float4 n1, const float4 n2, const RayPre& p,
                                            float cull, bool& hitL, bool& hitR, float& tL, float& tR)
{
    const bool nx = p.ix < 0.0f, ny = p.iy < 0.0f, nz = p.iz < 0.0f;
    const float lex = slab_t(nx ? n0.y : n0.x, p.ox, p.ix), lxx = slab_t(nx ? n0.x : n0.y, p.ox, p.ix);
    const float ley = slab_t(ny ? n0.w : n0.z, p.oy, p.iy), lxy = slab_t(ny ? n0.z : n0.w, p.oy, p.iy);
    const float lez = slab_t(nz ? n2.y : n2.x, p.oz, p.iz), lxz = slab_t(nz ? n2.x : n2.y, p.oz, p.iz);
    const float rex = slab_t(nx ? n1.y : n1.x, p.ox, p.ix), rxx = slab_t(nx ? n1.x : n1.y, p.ox, p.ix);
    const float rey = slab_t(ny ? n1.w : n1.z, p.oy, p.iy), rxy = slab_t(ny ? n1.z : n1.w, p.oy, p.iy);
    const float rez = slab_t(nz ? n2.w : n2.z, p.oz, p.iz), rxz = slab_t(nz ? n2.z : n2.w, p.oz, p.iz);
    const float lnear = fmaxf(fmaxf(lex, ley), fmaxf(lez, kTEps));
    const float lfar = fminf(fminf(lxx, lxy), lxz) * kFarScale;
    const float rnear = fmaxf(fmaxf(rex, rey), fmaxf(rez, kTEps));
    const float rfar = fminf(fminf(rxx, rxy), rxz) * kFarScale;
    hitL = lnear <= fminf(lfar, cull);
    hitR = rnear <= fminf(rfar, cull);
    tL = lnear;
    tR = rnear;
}

// Closest hit in (kTEps, t_max] by BVH traversal with a per-thread stack of
// deferred far children.  Returns false if the stack would overflow (the
// build refuses trees deeper than the stack, so this does not happen).
//
// The stack's first kSharedStack entries can live in shared memory, laid out
// [depth][thread] (`sh` points at this thread's column, `sh_stride` = threads
// per block), so lanes at different depths still hit distinct banks; deeper
// entries go to a per-thread local array.  Measured on GB300 the shared part
// does not pay (it shrinks the L1 the node fetches live in), so the default
// depth is 0 and the whole stack is local (L1-cached).
#ifndef LIDAR_SHARED_STACK
#define LIDAR_SHARED_STACK 0
#endif
constexpr int kSharedStack = LIDAR_SHARED_STACK;

struct SplitStack {
    int2* sh;
    int sh_stride;
    int2 local[kTraversalStack - kSharedStack];
    __device__ __forceinline__ void put(int i, int2 e)
    {
        if (i < kSharedStack) sh[i * sh_stride] = e;
        else local[i - kSharedStack] = e;
    }
    __device__ __forceinline__ int2 get(int i) const
    {
        return i < kSharedStack ? sh[i * sh_stride] : local[i - kSharedStack];
    }
};

template <bool kCount = false>
__device__ __forceinline__ bool trace_closest(const SceneDev& S, const RayPre& p, float t_max, HitRec& h,
                                              const WorkCount* wc, int2* sh_stack, int sh_stride,
                                              unsigned* cost = nullptr)
{
    unsigned long long n_nodes = 0, n_tris = 0;
    h.t = t_max;
    h.cull = t_max * kBestScale;
    h.idx = 0xFFFFFFFFu;
    h.leaf = -1;
    if (S.n_tris == 0) return true;
    SplitStack stack;
    stack.sh = sh_stack;
    stack.sh_stride = sh_stride;
    int sp = 0;
    int node = 0;
    while (true) {
        if (kCount) {
            ++n_nodes;
            atomicOr(&wc->node_bits[node >> 5], 1u << (node & 31));
        }
        if (!index_ok(node, S.n_nodes)) {
            h.leaf = kBadIndex;
            return false;
        }
        const float4 n0 = __ldg(&S.nodes[4 * (int64_t)node + 0]);
        const float4 n1 = __ldg(&S.nodes[4 * (int64_t)node + 1]);
        const float4 n2 = __ldg(&S.nodes[4 * (int64_t)node + 2]);
        const float4 n3 = __ldg(&S.nodes[4 * (int64_t)node + 3]);
        bool hitL, hitR;
        float tL, tR;
        child_boxes(n0, n1, n2, p, h.cull, hitL, hitR, tL, tR);
        const int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
        if (!index_ok(hitL && cl < 0 ? ~cl : 0, S.n_tris) || !index_ok(hitR && cr < 0 ? ~cr : 0, S.n_tris)) {
            h.leaf = kBadIndex;
            return false;
        }
        if (hitL && cl < 0) {
            if (kCount) {
                ++n_tris;
                atomicOr(&wc->leaf_bits[(~cl) >> 5], 1u << ((~cl) & 31));
            }
            intersect_triangle(S.tris, ~cl, p, t_max, h);
            hitL = false;
        }
        if (hitR && cr < 0) {
            if (kCount) {
                ++n_tris;
                atomicOr(&wc->leaf_bits[(~cr) >> 5], 1u << ((~cr) & 31));
            }
            intersect_triangle(S.tris, ~cr, p, t_max, h);
            hitR = false;
        }
        hitL = hitL && tL <= h.cull;
        hitR = hitR && tR <= h.cull;
        if (hitL && hitR) {
            const bool lfirst = tL <= tR;
            if (sp >= kTraversalStack) return false;
            stack.put(sp++, make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? tR : tL)));
            node = lfirst ? cl : cr;
            continue;
        }
        if (hitL) { node = cl; continue; }
        if (hitR) { node = cr; continue; }
        bool found = false;
        while (sp > 0) {
            const int2 e = stack.get(--sp);
            if (__int_as_float(e.y) <= h.cull) {
                node = e.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    if (kCount) {
        atomicAdd(&wc->totals[0], n_nodes);
        atomicAdd(&wc->totals[1], n_tris);
        if (cost) *cost += (unsigned)(n_nodes + n_tris);
    }
    return true;
}

// Slab test of the four child boxes of a 4-wide node (child boxes as SoA
// float4 per plane), same rounding and NaN handling as child_boxes.
// Packed FP32 pairs (sm_100+ f32x2 arithmetic): each lane of the pair is
// rounded exactly like the scalar __fsub_rn / __fmul_rn, so the slab distances
// are bit-identical to slab_t, with half the instructions.
__device__ __forceinline__ unsigned long long pack2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ unsigned long long slab2(unsigned long long planes, unsigned long long o2,
                                                    unsigned long long inv2)
{
    unsigned long long d, t;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(planes), "l"(o2));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(d), "l"(inv2));
    return t;
}

// entry/exit planes already chosen by the ray's direction signs
__device__ __forceinline__ void slab4_planes(float4 e, float4 x, unsigned long long o2, unsigned long long i2,
                                             float4& tin, float4& tout)
{
    unpack2(slab2(pack2(e.x, e.y), o2, i2), tin.x, tin.y);
    unpack2(slab2(pack2(e.z, e.w), o2, i2), tin.z, tin.w);
    unpack2(slab2(pack2(x.x, x.y), o2, i2), tout.x, tout.y);
    unpack2(slab2(pack2(x.z, x.w), o2, i2), tout.z, tout.w);
}

// Three-input FP32 max / min (sm_100+): the same result as the two-input
// fmaxf / fminf chains, NaN inputs ignored unless all are NaN, in one
// instruction and one dependent step instead of two.
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Near and far slab distances of four child boxes (entry and exit planes per
// axis already chosen by the direction signs): near = max(axis entries,
// t_eps), far = min(axis exits) * kFarScale, each slab distance rounded as
// slab_t rounds it.
__device__ __forceinline__ void near_far4(float4 xe, float4 xx, float4 ye, float4 yx, float4 ze, float4 zx,
                                          unsigned long long ox2, unsigned long long oy2, unsigned long long oz2,
                                          unsigned long long ix2, unsigned long long iy2, unsigned long long iz2,
                                          float4& kn, float4& kf)
{
    float4 xi, xo, yi, yo, zi, zo;
    slab4_planes(xe, xx, ox2, ix2, xi, xo);
    slab4_planes(ye, yx, oy2, iy2, yi, yo);
    slab4_planes(ze, zx, oz2, iz2, zi, zo);
    kn = make_float4(max3f(xi.x, yi.x, fmaxf(zi.x, kTEps)), max3f(xi.y, yi.y, fmaxf(zi.y, kTEps)),
                     max3f(xi.z, yi.z, fmaxf(zi.z, kTEps)), max3f(xi.w, yi.w, fmaxf(zi.w, kTEps)));
    kf = make_float4(min3f(xo.x, yo.x, zo.x) * kFarScale, min3f(xo.y, yo.y, zo.y) * kFarScale,
                     min3f(xo.z, yo.z, zo.z) * kFarScale, min3f(xo.w, yo.w, zo.w) * kFarScale);
}

// child code of slot j (0..7) of an 8-wide node
__device__ __forceinline__ int code8(const int4& a, const int4& b, unsigned j)
{
    const int4 v = (j & 4u) ? b : a;
    const int lo = (j & 1u) ? v.y : v.x, hi = (j & 1u) ? v.w : v.z;
    return (j & 2u) ? hi : lo;
}

__device__ __forceinline__ void sort2u(unsigned& a, unsigned& b)
{
    const unsigned lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Closest hit by traversal of the 4-wide hierarchy.  Node (128 bytes, eight
// 16-byte loads): lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the four children as
// float4s, the child codes (>= 0 node, < 0 ~leaf; empty slots have an empty
// box), then the id of the first internal child and the mask of leaf slots.
// Internal children fill the first slots with consecutive ids (slot j holds
// node first + j).  Triangle children are tested when met.  Of the hit
// internal children a single one is visited directly; several are ordered near
// to far by a 4-key sorting network over 32-bit keys (the entry distance's
// bits with the low bits replaced by the slot, as in trace_closest8); the
// nearest is visited next and the others pushed far-first.
template <bool kCount = false>
__device__ __forceinline__ bool trace_closest4(const SceneDev& S, const RayPre& p, float t_max, HitRec& h,
                                               const WorkCount* wc, int2* sh_stack, int sh_stride,
                                               unsigned* cost = nullptr)
{
    unsigned long long n_nodes = 0, n_tris = 0;
    h.t = t_max;
    h.cull = t_max * kBestScale;
    h.idx = 0xFFFFFFFFu;
    h.leaf = -1;
    if (S.n_tris == 0) return true;
    SplitStack stack;
    stack.sh = sh_stack;
    stack.sh_stride = sh_stride;
    // entry planes per axis: lo for a positive direction, hi for a negative one;
    // chosen once per ray as load offsets instead of selects per node
    const int ex = p.ix < 0.0f ? 1 : 0, ey = p.iy < 0.0f ? 3 : 2, ez = p.iz < 0.0f ? 5 : 4;
    const unsigned long long ox2 = pack2(p.ox, p.ox), oy2 = pack2(p.oy, p.oy), oz2 = pack2(p.oz, p.oz);
    const unsigned long long ix2 = pack2(p.ix, p.ix), iy2 = pack2(p.iy, p.iy), iz2 = pack2(p.iz, p.iz);
    constexpr unsigned kNone = 0xFFFFFFFFu;
    int sp = 0;
    int node = 0;
    while (true) {
        if (kCount) {
            ++n_nodes;
            atomicOr(&wc->node_bits[node >> 5], 1u << (node & 31));
        }
        if (!index_ok(node, S.n_nodes4)) {
            h.leaf = kBadIndex;
            return false;
        }
        const float4* q = S.nodes4 + 8 * (int64_t)node;
        const int2 meta = __ldg(reinterpret_cast<const int2*>(q + 7));
        float4 kn, kf;
        near_far4(__ldg(q + ex), __ldg(q + (1 - ex)), __ldg(q + ey), __ldg(q + (5 - ey)), __ldg(q + ez),
                  __ldg(q + (9 - ez)), ox2, oy2, oz2, ix2, iy2, iz2, kn, kf);
        const unsigned hit = (kn.x <= fminf(kf.x, h.cull) ? 1u : 0u) | (kn.y <= fminf(kf.y, h.cull) ? 2u : 0u) |
                             (kn.z <= fminf(kf.z, h.cull) ? 4u : 0u) | (kn.w <= fminf(kf.w, h.cull) ? 8u : 0u);
        const unsigned leafm = (unsigned)meta.y;
        unsigned vm = hit & ~leafm;  // hit internal children
        unsigned leaves = hit & leafm;
        if (leaves) {
            // triangle children first, through one call site
            const float cull0 = h.cull;
            const int4 c = __ldg(reinterpret_cast<const int4*>(q + 6));
            while (leaves) {
                const unsigned j = (unsigned)(__ffs(leaves) - 1);
                leaves &= leaves - 1;
                const int leaf = ~((j & 2u) ? ((j & 1u) ? c.w : c.z) : ((j & 1u) ? c.y : c.x));
                if (!index_ok(leaf, S.n_tris)) {
                    h.leaf = kBadIndex;
                    return false;
                }
                if (kCount) {
                    ++n_tris;
                    atomicOr(&wc->leaf_bits[leaf >> 5], 1u << (leaf & 31));
                }
                intersect_triangle(S.tris, leaf, p, t_max, h);
            }
            if (h.cull < cull0) {
                // a closer hit: keep only the internal children still in front of it
                const float cl = h.cull;
                vm &= (kn.x <= cl ? 1u : 0u) | (kn.y <= cl ? 2u : 0u) | (kn.z <= cl ? 4u : 0u) |
                      (kn.w <= cl ? 8u : 0u);
            }
        }
        if (vm) {
            const int first = meta.x;
            if ((vm & (vm - 1u)) == 0u) {
                node = first + (__ffs(vm) - 1);
                continue;
            }
            auto key = [vm](float k, unsigned j) -> unsigned {
                return ((vm >> j) & 1u) ? ((__float_as_uint(k) & ~7u) | j) : kNone;
            };
            unsigned s0 = key(kn.x, 0u), s1 = key(kn.y, 1u), s2 = key(kn.z, 2u), s3 = key(kn.w, 3u);
            sort2u(s0, s1); sort2u(s2, s3); sort2u(s0, s2); sort2u(s1, s3); sort2u(s1, s2);
            if (s3 != kNone) {
                if (sp >= kTraversalStack) return false;
                stack.put(sp++, make_int2(first + (int)(s3 & 7u), (int)(s3 & ~7u)));
            }
            if (s2 != kNone) {
                if (sp >= kTraversalStack) return false;
                stack.put(sp++, make_int2(first + (int)(s2 & 7u), (int)(s2 & ~7u)));
            }
            if (sp >= kTraversalStack) return false;
            stack.put(sp++, make_int2(first + (int)(s1 & 7u), (int)(s1 & ~7u)));
            node = first + (int)(s0 & 7u);
            continue;
        }
        bool found = false;
        while (sp > 0) {
            const int2 e = stack.get(--sp);
            if (__int_as_float(e.y) <= h.cull) {
                node = e.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    if (kCount) {
        atomicAdd(&wc->totals[0], n_nodes);
        atomicAdd(&wc->totals[1], n_tris);
        if (cost) *cost += (unsigned)(n_nodes + n_tris);
    }
    return true;
}

// Closest hit by traversal of the 8-wide hierarchy.  Node (256 bytes): per
// axis the lower planes of children 0-3 and 4-7, then their upper planes, as
// float4s (x at 0-3, y at 4-7, z at 8-11), the eight child codes (12-13), then
// the id of the first internal child and the mask of leaf slots (14).  Internal
// children fill the first slots with consecutive ids, so slot j holds node
// first + j.  Triangle children are tested when met.  Of the hit internal
// children a single one is visited directly; several are ordered near to far
// by a sorting network (4 keys when they all sit in slots 0-3, else Batcher's
// 8-key odd-even merge network) over 32-bit keys: the entry distance's bits with
// the three lowest replaced by the slot.  Entry distances are positive, so their
// bit patterns order like the values; clearing low bits only lowers a key, so
// the stacked keys still prune conservatively.  The nearest child is visited
// next, the others are pushed far-first.
template <bool kCount = false>
__device__ __forceinline__ bool trace_closest8(const SceneDev& S, const RayPre& p, float t_max, HitRec& h,
                                               const WorkCount* wc, int2* sh_stack, int sh_stride,
                                               unsigned* cost = nullptr)
{
    unsigned long long n_nodes = 0, n_tris = 0;
    h.t = t_max;
    h.cull = t_max * kBestScale;
    h.idx = 0xFFFFFFFFu;
    h.leaf = -1;
    if (S.n_tris == 0) return true;
    SplitStack stack;
    stack.sh = sh_stack;
    stack.sh_stride = sh_stride;
    // entry planes per axis (lower ones for a positive direction), as load offsets
    const int ex = p.ix < 0.0f ? 2 : 0, ey = p.iy < 0.0f ? 6 : 4, ez = p.iz < 0.0f ? 10 : 8;
    const unsigned long long ox2 = pack2(p.ox, p.ox), oy2 = pack2(p.oy, p.oy), oz2 = pack2(p.oz, p.oz);
    const unsigned long long ix2 = pack2(p.ix, p.ix), iy2 = pack2(p.iy, p.iy), iz2 = pack2(p.iz, p.iz);
    constexpr unsigned kNone = 0xFFFFFFFFu;
    int sp = 0;
    int node = 0;
    while (true) {
        if (kCount) {
            ++n_nodes;
            atomicOr(&wc->node_bits[node >> 5], 1u << (node & 31));
        }
        if (!index_ok(node, S.n_nodes8)) {
            h.leaf = kBadIndex;
            return false;
        }
        const float4* q = S.nodes8 + 16 * (int64_t)node;
        const int2 meta = __ldg(reinterpret_cast<const int2*>(q + 14));
        float4 ka, fa, kb, fb;
        near_far4(__ldg(q + ex), __ldg(q + (2 - ex)), __ldg(q + ey), __ldg(q + (10 - ey)), __ldg(q + ez),
                  __ldg(q + (18 - ez)), ox2, oy2, oz2, ix2, iy2, iz2, ka, fa);
        near_far4(__ldg(q + ex + 1), __ldg(q + (3 - ex)), __ldg(q + ey + 1), __ldg(q + (11 - ey)),
                  __ldg(q + ez + 1), __ldg(q + (19 - ez)), ox2, oy2, oz2, ix2, iy2, iz2, kb, fb);
        const unsigned hit = (ka.x <= fminf(fa.x, h.cull) ? 1u : 0u) | (ka.y <= fminf(fa.y, h.cull) ? 2u : 0u) |
                             (ka.z <= fminf(fa.z, h.cull) ? 4u : 0u) | (ka.w <= fminf(fa.w, h.cull) ? 8u : 0u) |
                             (kb.x <= fminf(fb.x, h.cull) ? 16u : 0u) | (kb.y <= fminf(fb.y, h.cull) ? 32u : 0u) |
                             (kb.z <= fminf(fb.z, h.cull) ? 64u : 0u) | (kb.w <= fminf(fb.w, h.cull) ? 128u : 0u);
        const unsigned leafm = (unsigned)meta.y;
        unsigned vm = hit & ~leafm;  // hit internal children
        unsigned leaves = hit & leafm;
        if (leaves) {
            const float cull0 = h.cull;
            const int4 ca = __ldg(reinterpret_cast<const int4*>(q + 12));
            const int4 cb = __ldg(reinterpret_cast<const int4*>(q + 13));
            while (leaves) {
                const unsigned j = (unsigned)(__ffs(leaves) - 1);
                leaves &= leaves - 1;
                const int leaf = ~code8(ca, cb, j);
                if (!index_ok(leaf, S.n_tris)) {
                    h.leaf = kBadIndex;
                    return false;
                }
                if (kCount) {
                    ++n_tris;
                    atomicOr(&wc->leaf_bits[leaf >> 5], 1u << (leaf & 31));
                }
                intersect_triangle(S.tris, leaf, p, t_max, h);
            }
            if (h.cull < cull0) {
                // a closer hit: keep only the internal children still in front of it
                const float c = h.cull;
                vm &= (ka.x <= c ? 1u : 0u) | (ka.y <= c ? 2u : 0u) | (ka.z <= c ? 4u : 0u) |
                      (ka.w <= c ? 8u : 0u) | (kb.x <= c ? 16u : 0u) | (kb.y <= c ? 32u : 0u) |
                      (kb.z <= c ? 64u : 0u) | (kb.w <= c ? 128u : 0u);
            }
        }
        if (vm) {
            const int first = meta.x;
            if ((vm & (vm - 1u)) == 0u) {
                node = first + (__ffs(vm) - 1);
                continue;
            }
            auto key = [vm](float k, unsigned j) -> unsigned {
                return ((vm >> j) & 1u) ? ((__float_as_uint(k) & ~7u) | j) : kNone;
            };
            auto push = [&](unsigned s) -> bool {
                if (s == kNone) return true;
                if (sp >= kTraversalStack) return false;
                stack.put(sp++, make_int2(first + (int)(s & 7u), (int)(s & ~7u)));
                return true;
            };
            unsigned s0 = key(ka.x, 0u), s1 = key(ka.y, 1u), s2 = key(ka.z, 2u), s3 = key(ka.w, 3u);
            if ((vm & 0xF0u) == 0u) {
                sort2u(s0, s1); sort2u(s2, s3); sort2u(s0, s2); sort2u(s1, s3); sort2u(s1, s2);
                if (!push(s3) || !push(s2) || !push(s1)) return false;
            } else {
                unsigned s4 = key(kb.x, 4u), s5 = key(kb.y, 5u), s6 = key(kb.z, 6u), s7 = key(kb.w, 7u);
                sort2u(s0, s1); sort2u(s2, s3); sort2u(s4, s5); sort2u(s6, s7);
                sort2u(s0, s2); sort2u(s1, s3); sort2u(s4, s6); sort2u(s5, s7);
                sort2u(s1, s2); sort2u(s5, s6);
                sort2u(s0, s4); sort2u(s1, s5); sort2u(s2, s6); sort2u(s3, s7);
                sort2u(s2, s4); sort2u(s3, s5);
                sort2u(s1, s2); sort2u(s3, s4); sort2u(s5, s6);
                if (!push(s7) || !push(s6) || !push(s5) || !push(s4) || !push(s3) || !push(s2) || !push(s1))
                    return false;
            }
            node = first + (int)(s0 & 7u);
            continue;
        }
        bool found = false;
        while (sp > 0) {
            const int2 e = stack.get(--sp);
            if (__int_as_float(e.y) <= h.cull) {
                node = e.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    if (kCount) {
        atomicAdd(&wc->totals[0], n_nodes);
        atomicAdd(&wc->totals[1], n_tris);
        if (cost) *cost += (unsigned)(n_nodes + n_tris);
    }
    return true;
}

// Warp-synchronous variant of trace_closest (same result).  All 32 lanes of
// the warp must call it together; lanes with `active` false take part in the
// warp votes only.  Triangle tests are postponed: a lane that reaches a leaf
// parks it (at most two, one node's children) and waits while other lanes
// still descend, so the triangle tests run with most lanes busy instead of
// one or two lanes per node step (Aila & Laine, "Understanding the Efficiency
// of Ray Traversal on GPUs", HPG 2009: while-while traversal).
template <bool kCount = false>
__device__ __forceinline__ bool trace_closest_warp(const SceneDev& S, const RayPre& p, float t_max, HitRec& h,
                                                   bool active, const WorkCount* wc = nullptr)
{
    unsigned long long n_nodes = 0, n_tris = 0;
    h.t = t_max;
    h.cull = t_max * kBestScale;
    h.idx = 0xFFFFFFFFu;
    h.leaf = -1;
    int2 stack[kTraversalStack];
    int sp = 0;
    int node = (active && S.n_tris > 0) ? 0 : -1;
    float node_t = 0.0f;  // entry distance of `node` (culled when it exceeds the best hit)
    int pend0 = -1, pend1 = -1;
    bool ok = true;
    bool bad = false;  // a bounds check failed (checked builds)
    while (__any_sync(0xffffffffu, node >= 0 || pend0 >= 0)) {
        // descend until this lane holds a leaf or has nothing left
        while (__any_sync(0xffffffffu, node >= 0 && pend0 < 0)) {
            if (node >= 0 && pend0 < 0) {
                if (node_t > h.cull) {
                    node = -1;
                } else if (!index_ok(node, S.n_nodes)) {
                    ok = false;
                    bad = true;
                    node = -1;
                    sp = 0;
                } else {
                    if (kCount) {
                        ++n_nodes;
                        atomicOr(&wc->node_bits[node >> 5], 1u << (node & 31));
                    }
                    const float4 n0 = __ldg(&S.nodes[4 * (int64_t)node + 0]);
                    const float4 n1 = __ldg(&S.nodes[4 * (int64_t)node + 1]);
                    const float4 n2 = __ldg(&S.nodes[4 * (int64_t)node + 2]);
                    const float4 n3 = __ldg(&S.nodes[4 * (int64_t)node + 3]);
                    bool hitL, hitR;
                    float tL, tR;
                    child_boxes(n0, n1, n2, p, h.cull, hitL, hitR, tL, tR);
                    const int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
                    if (!index_ok(hitL && cl < 0 ? ~cl : 0, S.n_tris) ||
                        !index_ok(hitR && cr < 0 ? ~cr : 0, S.n_tris)) {
                        ok = false;
                        bad = true;
                        hitL = hitR = false;
                    }
                    if (hitL && cl < 0) { pend0 = ~cl; hitL = false; }
                    if (hitR && cr < 0) {
                        if (pend0 < 0) pend0 = ~cr; else pend1 = ~cr;
                        hitR = false;
                    }
                    if (hitL && hitR) {
                        const bool lfirst = tL <= tR;
                        if (sp >= kTraversalStack) {
                            ok = false;
                            node = -1;
                            sp = 0;
                        } else {
                            stack[sp++] = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? tR : tL));
                            node = lfirst ? cl : cr;
                            node_t = lfirst ? tL : tR;
                        }
                    } else if (hitL) {
                        node = cl;
                        node_t = tL;
                    } else if (hitR) {
                        node = cr;
                        node_t = tR;
                    } else {
                        node = -1;
                    }
                }
                if (node < 0) {
                    while (sp > 0) {
                        const int2 e = stack[--sp];
                        if (__int_as_float(e.y) <= h.cull) {
                            node = e.x;
                            node_t = __int_as_float(e.y);
                            break;
                        }
                    }
                }
            }
        }
        // intersect the parked triangles
        if (pend0 >= 0) {
            if (kCount) {
                ++n_tris;
                atomicOr(&wc->leaf_bits[pend0 >> 5], 1u << (pend0 & 31));
            }
            intersect_triangle(S.tris, pend0, p, t_max, h);
            pend0 = -1;
        }
        if (pend1 >= 0) {
            if (kCount) {
                ++n_tris;
                atomicOr(&wc->leaf_bits[pend1 >> 5], 1u << (pend1 & 31));
            }
            intersect_triangle(S.tris, pend1, p, t_max, h);
            pend1 = -1;
        }
    }
    if (kCount) {
        atomicAdd(&wc->totals[0], n_nodes);
        atomicAdd(&wc->totals[1], n_tris);
    }
    if (bad) h.leaf = kBadIndex;
    return ok;
}

}  // namespace lidar
