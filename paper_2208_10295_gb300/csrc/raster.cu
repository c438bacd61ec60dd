// The paper's own sampling path (Sec. II-A..II-C), as compute rasterisation:
// per frame, K pin-hole cameras at the sensor pose share the sensor's 360
// degree horizontal field (camera k looks along sensor azimuth
// -pi + (k + 1/2) 2 pi / K; square W x W image; intrinsics of Eq. 1-2).  Each
// camera renders, through every pixel centre, the depth pass (z-depth, three
// bytes), the incidence angle (three bytes), the material stencil (one byte)
// and the instance colour (three bytes); each beam then reads the pixel its
// direction projects to (Eq. 3 in the corrected form n_x = c + f x/z,
// n_y = c - f y/z) and goes through the same noise, Eq. 4 lookup, Eq. 5
// capability test and intensity as the ray-cast path.
//
// Rasterisation: one thread per triangle finds the cameras whose azimuth
// sectors its horizontal extent can reach, and for each clips the triangle at
// the near plane, projects it and bounds the pixel centres it can cover; each
// of those pixels tests its centre ray against the triangle with the
// watertight test of the ray-cast path and keeps the closest (t, original
// index) by a 64-bit atomicMin — the z-buffer.  Small boxes are tested by that
// thread; larger ones go to a list of row bands that warps take.
#include "common.cuh"
#include "philox.cuh"
#include "trace.cuh"

namespace lidar {
namespace {

constexpr int kSmallBox = 32;           // pixels a triangle's own thread tests
constexpr float kNear = 1e-6f;          // camera-space near plane (metres)
constexpr uint32_t kSky = 0xFFFFFFu;    // depth code of a pixel with no hit
constexpr unsigned long long kNoKey = ~0ull;

struct BigBox {
    uint32_t cam_leaf;   // camera << 26 | leaf
    uint16_t x0, y0, nx, ny;
};

// Pixel-centre ray of camera k in the world, every operation rounded as
// written: a = (i + 1/2 - c)/f, b = (c - (j + 1/2))/f,
// dir = (F + a L + b U) / sqrt(1 + a^2 + b^2); `inv` = 1 / sqrt(...) = dir . F.
__device__ __forceinline__ RayW pixel_ray(const RasterCams& C, const float* pose, int k, int ix, int iy,
                                          float& inv)
{
    const float a = __fdiv_rn(__fsub_rn(__fadd_rn((float)ix, 0.5f), C.c), C.f);
    const float b = __fdiv_rn(__fsub_rn(C.c, __fadd_rn((float)iy, 0.5f)), C.f);
    float s2 = __fadd_rn(1.0f, __fmul_rn(a, a));
    s2 = __fadd_rn(s2, __fmul_rn(b, b));
    inv = __fdiv_rn(1.0f, __fsqrt_rn(s2));
    const float ck = C.ck[k], sk = C.sk[k];
    const float dx = __fmul_rn(__fsub_rn(ck, __fmul_rn(a, sk)), inv);
    const float dy = __fmul_rn(__fadd_rn(sk, __fmul_rn(a, ck)), inv);
    const float dz = __fmul_rn(b, inv);
    return world_ray(pose, dx, dy, dz);
}

// z-test of one pixel centre against one triangle (leaf position)
__device__ __forceinline__ void raster_pixel(const SceneDev& S, const RasterCams& C, const RasterFrame& F, int k,
                                             int leaf, int ix, int iy, unsigned long long* keys)
{
    float inv;
    const RayW r = pixel_ray(C, F.pose, k, ix, iy, inv);
    const RayPre p = prepare_ray(r);
    HitRec h;
    h.t = F.t_max;
    h.cull = F.t_max;
    h.idx = 0xFFFFFFFFu;
    h.leaf = -1;
    intersect_triangle(S.tris, leaf, p, F.t_max, h);
    if (h.leaf < 0) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(h.t) << 32) | h.idx;
    atomicMin(&keys[((int64_t)k * C.W + iy) * C.W + ix], key);
}

// Pixel box of the centres a triangle can cover in camera k (empty: x1 < x0).
// The box only selects pixels to test; the exact test decides coverage, so it
// is widened by a hundredth of a pixel against rounding.
__device__ __forceinline__ void triangle_box(const RasterCams& C, const RasterFrame& F, int k, float4 a, float4 b,
                                             float4 c, int& x0, int& x1, int& y0, int& y1)
{
    const float* Lw = F.axes + 9 * k;      // L, U, F of camera k in the world
    const float vx[3] = {a.x - F.pose[3], b.x - F.pose[3], c.x - F.pose[3]};
    const float vy[3] = {a.y - F.pose[7], b.y - F.pose[7], c.y - F.pose[7]};
    const float vz[3] = {a.z - F.pose[11], b.z - F.pose[11], c.z - F.pose[11]};
    float cx[3], cy[3], cz[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        cx[j] = vx[j] * Lw[0] + vy[j] * Lw[1] + vz[j] * Lw[2];
        cy[j] = vx[j] * Lw[3] + vy[j] * Lw[4] + vz[j] * Lw[5];
        cz[j] = vx[j] * Lw[6] + vy[j] * Lw[7] + vz[j] * Lw[8];
    }
    x0 = 1; x1 = 0; y0 = 1; y1 = 0;
    // a hit at t <= t_max has z-depth <= t_max
    if (fminf(fminf(cz[0], cz[1]), cz[2]) > F.t_max) return;
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    int n = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int m = j == 2 ? 0 : j + 1;
        if (cz[j] > kNear) {
            const float u = cx[j] / cz[j], v = cy[j] / cz[j];
            umin = fminf(umin, u); umax = fmaxf(umax, u);
            vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
            ++n;
        }
        if ((cz[j] > kNear) != (cz[m] > kNear)) {
            // crossing of the near plane
            const float s = (kNear - cz[j]) / (cz[m] - cz[j]);
            const float px = cx[j] + s * (cx[m] - cx[j]), py = cy[j] + s * (cy[m] - cy[j]);
            const float u = px / kNear, v = py / kNear;
            umin = fminf(umin, u); umax = fmaxf(umax, u);
            vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
            ++n;
        }
    }
    if (n == 0) return;
    const float W = (float)C.W;
    // centres i + 1/2 with c + f u in [c + f umin, c + f umax]; rows grow downwards
    const float lx = C.c + C.f * umin - 0.5f - 0.01f, hx = C.c + C.f * umax - 0.5f + 0.01f;
    const float ly = C.c - C.f * vmax - 0.5f - 0.01f, hy = C.c - C.f * vmin - 0.5f + 0.01f;
    if (!(hx >= 0.0f) || !(lx <= W - 1.0f) || !(hy >= 0.0f) || !(ly <= W - 1.0f)) return;
    x0 = (int)ceilf(fmaxf(lx, 0.0f));
    x1 = (int)floorf(fminf(hx, W - 1.0f));
    y0 = (int)ceilf(fmaxf(ly, 0.0f));
    y1 = (int)floorf(fminf(hy, W - 1.0f));
}

// Boxes above kSmallBox pixels go to a list in row bands of at most
// kChunkPixels pixels (a box wider than that: one row per entry), so that one
// warp can take any entry: the pixel work of a large triangle is spread over
// many warps without a scan or a search.
constexpr int kChunkPixels = 256;

// Cameras (bit k = camera k) whose azimuth sector [-pi + k 2pi/K, -pi + (k+1)
// 2pi/K) the triangle can reach: camera k's pixel centres see only directions
// of azimuth inside its sector (u = tan of the azimuth off its axis), so a
// triangle whose horizontal projection, seen from the sensor axis, spans the
// arc [lo, lo + len] (len < pi: the projection leaves out the axis) reaches
// the sectors that arc meets.  Widened by 1e-3 rad against rounding; every
// camera when a vertex lies (nearly) on the axis or the arc cannot be bounded.
__device__ __forceinline__ unsigned long long camera_mask(const RasterCams& C, const float* pose, float4 a, float4 b,
                                                          float4 c)
{
    const unsigned long long all = C.K >= 64 ? ~0ull : ((1ull << C.K) - 1ull);
    const float vx[3] = {a.x - pose[3], b.x - pose[3], c.x - pose[3]};
    const float vy[3] = {a.y - pose[7], b.y - pose[7], c.y - pose[7]};
    const float vz[3] = {a.z - pose[11], b.z - pose[11], c.z - pose[11]};
    float az[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // sensor-frame x and y: the pose's rotation transposed
        const float sx = vx[j] * pose[0] + vy[j] * pose[4] + vz[j] * pose[8];
        const float sy = vx[j] * pose[1] + vy[j] * pose[5] + vz[j] * pose[9];
        // sx, sy carry rounding errors of ~2e-7 of the vertex's distance: keep
        // their angle's error below the margin, else take every camera
        if (fabsf(sx) + fabsf(sy) < 1e-3f * (fabsf(vx[j]) + fabsf(vy[j]) + fabsf(vz[j])) + 1e-6f) return all;
        az[j] = atan2f(sy, sx);
    }
    // sort the three azimuths, then the arc is the circle minus the largest gap
    float t;
    if (az[0] > az[1]) { t = az[0]; az[0] = az[1]; az[1] = t; }
    if (az[1] > az[2]) { t = az[1]; az[1] = az[2]; az[2] = t; }
    if (az[0] > az[1]) { t = az[0]; az[0] = az[1]; az[1] = t; }
    const float two_pi = 6.28318530717958648f;
    const float g0 = az[1] - az[0], g1 = az[2] - az[1], g2 = az[0] + two_pi - az[2];
    float lo, gap;
    if (g0 >= g1 && g0 >= g2) { gap = g0; lo = az[1]; }
    else if (g1 >= g2) { gap = g1; lo = az[2]; }
    else { gap = g2; lo = az[0]; }
    if (gap <= 3.14159265358979324f + 2e-3f) return all;  // the projection may surround the axis
    const float eps = 1e-3f;
    const float sector = two_pi / (float)C.K;
    const float start = lo - eps + 3.14159265358979324f;  // measured from -pi
    const float len = two_pi - gap + 2.0f * eps;
    int k0 = (int)floorf(start / sector);
    const int k1 = (int)floorf((start + len) / sector);
    const int count = min(k1 - k0 + 1, C.K);
    k0 = ((k0 % C.K) + C.K) % C.K;
    unsigned long long m = 0;
    for (int i = 0; i < count; ++i) m |= 1ull << ((k0 + i) % C.K);
    return m;
}

__global__ void __launch_bounds__(256) k_raster_tris(SceneDev S, RasterCams C, RasterFrame F,
                                                     unsigned long long* keys, BigBox* big,
                                                     unsigned long long* n_big, unsigned big_cap)
{
    for (int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; leaf < S.n_tris;
         leaf += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(&S.tris[3 * leaf]);
        const float4 b = __ldg(&S.tris[3 * leaf + 1]);
        const float4 c = __ldg(&S.tris[3 * leaf + 2]);
        unsigned long long cams = camera_mask(C, F.pose, a, b, c);
        while (cams) {
            const int k = __ffsll((long long)cams) - 1;
            cams &= cams - 1;
            int x0, x1, y0, y1;
            triangle_box(C, F, k, a, b, c, x0, x1, y0, y1);
            if (x1 < x0 || y1 < y0) continue;
            const int nx = x1 - x0 + 1, ny = y1 - y0 + 1;
            int y_here = y0;  // rows from here on are tested by this thread
            if (nx * ny > kSmallBox) {
                const int rows = max(1, kChunkPixels / nx);
                const int n_chunks = (ny + rows - 1) / rows;
                // a 64-bit counter cannot wrap; every slot below the capacity is
                // written by the box that took it, the bands past it are tested here
                const unsigned long long slot = atomicAdd(n_big, (unsigned long long)n_chunks);
                const int fit = slot >= big_cap ? 0 : (int)min((unsigned long long)n_chunks, big_cap - slot);
                for (int q = 0; q < fit; ++q) {
                    const int r0 = q * rows;
                    BigBox& e = big[slot + q];
                    e.cam_leaf = ((uint32_t)k << 26) | (uint32_t)leaf;
                    e.x0 = (uint16_t)x0;
                    e.y0 = (uint16_t)(y0 + r0);
                    e.nx = (uint16_t)nx;
                    e.ny = (uint16_t)min(rows, ny - r0);
                }
                y_here = y0 + min(ny, fit * rows);
            }
            for (int iy = y_here; iy <= y1; ++iy)
                for (int ix = x0; ix <= x1; ++ix) raster_pixel(S, C, F, k, (int)leaf, ix, iy, keys);
        }
    }
}

// the listed row bands, one warp per band
__global__ void __launch_bounds__(256) k_raster_big(SceneDev S, RasterCams C, RasterFrame F, const BigBox* big,
                                                    const unsigned long long* n_big, unsigned big_cap,
                                                    unsigned long long* keys)
{
    const unsigned n = (unsigned)min(*n_big, (unsigned long long)big_cap);
    const int lane = threadIdx.x & 31;
    const unsigned n_warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n; e += n_warps) {
        const BigBox bx = big[e];
        const int k = (int)(bx.cam_leaf >> 26), leaf = (int)(bx.cam_leaf & ((1u << 26) - 1));
        const int nxy = (int)bx.nx * bx.ny;
        for (int q = lane; q < nxy; q += 32)
            raster_pixel(S, C, F, k, leaf, bx.x0 + q % bx.nx, bx.y0 + q / bx.nx, keys);
    }
}

// G-buffer of every pixel: depth code (24 bits), angle code (24 bits) | stencil
// << 24, colour (24 bits), triangle (original index)
__global__ void __launch_bounds__(256) k_gbuffer(SceneDev S, RasterCams C, RasterFrame F,
                                                 const unsigned long long* __restrict__ keys,
                                                 const uint32_t* __restrict__ orig_to_leaf, GBuffer G)
{
    const int64_t n = (int64_t)C.K * C.W * C.W;
    const float qs = __fdiv_rn(16777215.0f, F.t_max);
    const float qa_s = __fdiv_rn(16777215.0f, 90.0f);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[p];
        if (key == kNoKey) {
            G.depth[p] = kSky;
            G.angle_mat[p] = 0u;
            G.inst[p] = 0u;
            if (G.tri) G.tri[p] = LIDAR_NO_HIT;
            continue;
        }
        const int k = (int)(p / ((int64_t)C.W * C.W));
        const int rem = (int)(p - (int64_t)k * C.W * C.W);
        const int iy = rem / C.W, ix = rem - iy * C.W;
        const uint32_t orig = (uint32_t)(key & 0xFFFFFFFFull);
        const float t = __uint_as_float((uint32_t)(key >> 32));
        float inv;
        const RayW r = pixel_ray(C, F.pose, k, ix, iy, inv);
        // depth pass: z-depth in three bytes
        const float z = __fmul_rn(t, inv);
        uint32_t q = __float2uint_rn(__fmul_rn(z, qs));
        if (q > kSky - 1u) q = kSky - 1u;
        // incidence angle on the face (two-sided), three bytes
        const int leaf = (int)orig_to_leaf[orig];
        const float4 a = __ldg(&S.tris[3 * (int64_t)leaf]);
        const float4 b = __ldg(&S.tris[3 * (int64_t)leaf + 1]);
        const float4 c = __ldg(&S.tris[3 * (int64_t)leaf + 2]);
        const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
        const float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
        float nx = e1y * e2z - e1z * e2y;
        float ny = e1z * e2x - e1x * e2z;
        float nz = e1x * e2y - e1y * e2x;
        const float inl = rsqrtf(nx * nx + ny * ny + nz * nz);
        nx *= inl; ny *= inl; nz *= inl;
        const float dn = r.dx * nx + r.dy * ny + r.dz * nz;
        const float cx = r.dy * nz - r.dz * ny, cy = r.dz * nx - r.dx * nz, cz = r.dx * ny - r.dy * nx;
        const float theta = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), fabsf(dn)) * 57.295779513082320876798f;
        uint32_t qa = __float2uint_rn(__fmul_rn(theta, qa_s));
        if (qa > 0xFFFFFFu) qa = 0xFFFFFFu;
        const uint32_t m8 = (uint32_t)__float_as_int(b.w) & 0xFFu;
        G.depth[p] = q;
        G.angle_mat[p] = qa | (m8 << 24);
        G.inst[p] = (uint32_t)__float_as_int(c.w) & 0xFFFFFFu;
        if (G.tri) G.tri[p] = orig;
    }
}

// Each beam of one frame reads the pixel its direction projects to.
__global__ void __launch_bounds__(256) k_resample(RasterCams C, RasterFrame F, const SensorDev* __restrict__ sensors,
                                                  int sensor, int frame_id, int64_t beam_offset, TableDev T,
                                                  uint64_t seed, GBuffer G, BeamsOut out)
{
    const SensorDev& sd = sensors[sensor];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= sd.n_beams) return;
    const float dx = __ldg(&sd.dirs[3 * (int64_t)b]), dy = __ldg(&sd.dirs[3 * (int64_t)b + 1]);
    const float dz = __ldg(&sd.dirs[3 * (int64_t)b + 2]);
    // camera: largest d . F_k (ties to the lowest k)
    int k = 0;
    float zk = 0.0f;
    for (int j = 0; j < C.K; ++j) {
        const float zj = __fadd_rn(__fmul_rn(dx, C.ck[j]), __fmul_rn(dy, C.sk[j]));
        if (j == 0 || zj > zk) {
            zk = zj;
            k = j;
        }
    }
    const int64_t o = beam_offset + b;
    bool hit = false;
    uint32_t q = kSky, am = 0u, inst = 0u, tri = LIDAR_NO_HIT;
    if (zk > 0.0f) {
        const float x = __fadd_rn(__fmul_rn(dx, -C.sk[k]), __fmul_rn(dy, C.ck[k]));
        const float nxp = __fadd_rn(C.c, __fmul_rn(C.f, __fdiv_rn(x, zk)));
        const float nyp = __fsub_rn(C.c, __fmul_rn(C.f, __fdiv_rn(dz, zk)));
        float fx = floorf(nxp);
        const float fy = floorf(nyp);
        if (fx == fx && fy >= 0.0f && fy < (float)C.W) {
            fx = fminf(fmaxf(fx, 0.0f), (float)(C.W - 1));  // a beam on the border of two cameras
            const int64_t p = ((int64_t)k * C.W + (int)fy) * C.W + (int)fx;
            q = G.depth[p];
            am = G.angle_mat[p];
            inst = G.inst[p];
            if (G.tri) tri = G.tri[p];
            hit = q != kSky;
        }
    }
    if (!hit) {
        if (out.valid) out.valid[o] = 0;
        if (out.tri) out.tri[o] = LIDAR_NO_HIT;
        if (out.t) out.t[o] = INFINITY;
        if (out.range) out.range[o] = INFINITY;
        if (out.intensity) out.intensity[o] = 0.0f;
        if (out.normal) out.normal[3 * o] = out.normal[3 * o + 1] = out.normal[3 * o + 2] = 0.0f;
        if (out.mat) out.mat[o] = 0;
        if (out.inst) out.inst[o] = 0;
        if (out.sub) out.sub[o] = 0;
        if (out.theta_deg) out.theta_deg[o] = 0.0f;
        if (out.rf) out.rf[o] = 0.0f;
        return;
    }
    // the pixel's depth read along the beam, then the model of the ray-cast path
    const float zq = __fmul_rn((float)q, __fdiv_rn(F.t_max, 16777215.0f));
    const float theta_deg = __fmul_rn((float)(am & 0xFFFFFFu), __fdiv_rn(90.0f, 16777215.0f));
    const uint32_t m = am >> 24;
    const float d_beam = __fdiv_rn(zq, zk);
    const uint32_t mrow = m < (uint32_t)T.n_mat ? m : (uint32_t)(T.n_mat - 1);
    int i = (int)theta_deg;
    if (i > LIDAR_TABLE_SIZE - 2) i = LIDAR_TABLE_SIZE - 2;
    const float f = theta_deg - (float)i;
    const float* row = T.table + (int64_t)mrow * LIDAR_TABLE_SIZE;
    const float R = __ldg(&row[i]) * (1.0f - f) + __ldg(&row[i + 1]) * f;
    const float zn = range_noise_normal(seed, (uint32_t)b, (uint32_t)frame_id, (uint32_t)sensor, 0u);
    const float d = d_beam + __fmaf_rn(sd.sigma_k, d_beam, sd.sigma) * zn;
    const float RLd = __fdiv_rn(__fmul_rn(sd.RL_max, d), sd.d_max);
    const int valid = (d >= sd.r_min) && (d <= sd.r_max) && (d <= sd.d_max) && (RLd <= R);
    const float rf = (sd.range_exp == 0.0f) ? 1.0f : powf(sd.r_ref / d, sd.range_exp);
    if (out.valid) out.valid[o] = (uint8_t)valid;
    if (out.tri) out.tri[o] = tri;
    if (out.t) out.t[o] = d_beam;
    if (out.range) out.range[o] = d;
    if (out.intensity) out.intensity[o] = sd.gain * R * rf;
    if (out.normal) out.normal[3 * o] = out.normal[3 * o + 1] = out.normal[3 * o + 2] = 0.0f;  // not in the G-buffer
    if (out.mat) out.mat[o] = (uint16_t)m;
    if (out.inst) out.inst[o] = inst;
    if (out.sub) out.sub[o] = 0;
    if (out.theta_deg) out.theta_deg[o] = theta_deg;
    if (out.rf) out.rf[o] = rf;
}

__global__ void k_invert_leaf_order(const uint32_t* __restrict__ leaf_tri, int64_t n, uint32_t* orig_to_leaf)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) orig_to_leaf[leaf_tri[i]] = (uint32_t)i;
}

}  // namespace

size_t raster_scratch_bytes(int width, int n_cameras, int64_t n_tris, bool with_tri)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t px = (size_t)n_cameras * width * width;
    const size_t cap = raster_big_capacity(n_cameras, n_tris);
    return al(px * 8) + 3 * al(px * 4) + (with_tri ? al(px * 4) : 0) + al(cap * sizeof(BigBox)) + 256;
}

size_t raster_big_capacity(int n_cameras, int64_t n_tris)
{
    return (size_t)(((int64_t)n_cameras * n_tris) / 4 + 65536);
}

cudaError_t launch_invert_leaf_order(cudaStream_t s, const uint32_t* leaf_tri, int64_t n, uint32_t* orig_to_leaf)
{
    if (n == 0) return cudaSuccess;
    k_invert_leaf_order<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(leaf_tri, n, orig_to_leaf);
    return cudaGetLastError();
}

cudaError_t launch_rasterise(cudaStream_t s, const SceneDev& S, const RasterCams& C, const RasterFrame& F,
                             const uint32_t* orig_to_leaf, void* scratch, bool with_tri, GBuffer* G_out, int num_sms)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t px = (size_t)C.K * C.W * C.W;
    const unsigned cap = (unsigned)raster_big_capacity(C.K, S.n_tris);
    char* p = (char*)scratch;
    unsigned long long* keys = (unsigned long long*)p;
    p += al(px * 8);
    GBuffer G;
    G.depth = (uint32_t*)p; p += al(px * 4);
    G.angle_mat = (uint32_t*)p; p += al(px * 4);
    G.inst = (uint32_t*)p; p += al(px * 4);
    G.tri = with_tri ? (uint32_t*)p : nullptr;
    if (with_tri) p += al(px * 4);
    BigBox* big = (BigBox*)p; p += al((size_t)cap * sizeof(BigBox));
    unsigned long long* n_big = (unsigned long long*)p;
    cudaError_t e = cudaMemsetAsync(keys, 0xFF, px * 8, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(n_big, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (S.n_tris > 0) {
        const int64_t blocks = std::min<int64_t>((S.n_tris + 255) / 256, (int64_t)num_sms * 16);
        k_raster_tris<<<(unsigned)blocks, 256, 0, s>>>(S, C, F, keys, big, n_big, cap);
        k_raster_big<<<(unsigned)num_sms * 16, 256, 0, s>>>(S, C, F, big, n_big, cap, keys);
    }
    const int64_t gb = std::min<int64_t>(((int64_t)px + 255) / 256, (int64_t)num_sms * 16);
    k_gbuffer<<<(unsigned)gb, 256, 0, s>>>(S, C, F, keys, orig_to_leaf, G);
    *G_out = G;
    return cudaGetLastError();
}

cudaError_t launch_resample(cudaStream_t s, const RasterCams& C, const RasterFrame& F, const SensorDev* sensors_dev,
                            int sensor, int n_beams, int frame_id, int64_t beam_offset, TableDev T, uint64_t seed,
                            const GBuffer& G, BeamsOut out)
{
    if (n_beams == 0) return cudaSuccess;
    k_resample<<<(unsigned)((n_beams + 255) / 256), 256, 0, s>>>(C, F, sensors_dev, sensor, frame_id, beam_offset,
                                                                  T, seed, G, out);
    return cudaGetLastError();
}

}  // namespace lidar
