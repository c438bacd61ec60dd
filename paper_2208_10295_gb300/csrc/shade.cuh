// Per-ray shading and the dense per-beam record, shared by the cast kernels.
#pragma once

#include "common.cuh"
#include "philox.cuh"
#include "trace.cuh"

namespace lidar {
namespace {

struct BeamResult {
    float t, range, intensity, theta_deg, rf;
    float nx, ny, nz;   // world frame, facing the sensor
    uint32_t tri, inst;
    uint32_t mat;
    int valid;
};

// Everything after the closest hit for one ray (Sec. II-A..II-D).
__device__ __forceinline__ void shade(const SceneDev& S, const HitRec& h, const RayW& r, const SensorDev& sd,
                                      const TableDev& T, uint64_t seed, uint32_t beam, uint32_t frame,
                                      uint32_t sensor, uint32_t sub, BeamResult& out)
{
    if (h.leaf < 0) {
        out.t = INFINITY;
        out.range = INFINITY;
        out.intensity = 0.0f;
        out.theta_deg = 0.0f;
        out.rf = 0.0f;
        out.nx = out.ny = out.nz = 0.0f;
        out.tri = LIDAR_NO_HIT;
        out.inst = 0;
        out.mat = 0;
        out.valid = 0;
        return;
    }
    const float4 a = __ldg(&S.tris[3 * (int64_t)h.leaf]);
    const float4 b = __ldg(&S.tris[3 * (int64_t)h.leaf + 1]);
    const float4 c = __ldg(&S.tris[3 * (int64_t)h.leaf + 2]);
    // face normal, turned towards the sensor
    const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    float nx = e1y * e2z - e1z * e2y;
    float ny = e1z * e2x - e1x * e2z;
    float nz = e1x * e2y - e1y * e2x;
    const float inl = rsqrtf(nx * nx + ny * ny + nz * nz);
    nx *= inl; ny *= inl; nz *= inl;
    float dn = r.dx * nx + r.dy * ny + r.dz * nz;
    if (dn > 0.0f) { nx = -nx; ny = -ny; nz = -nz; dn = -dn; }
    // incidence angle between beam and normal (Sec. II-C)
    const float cx = r.dy * nz - r.dz * ny, cy = r.dz * nx - r.dx * nz, cz = r.dx * ny - r.dy * nx;
    const float theta = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), fabsf(dn));
    const float theta_deg = theta * 57.295779513082320876798f;
    // reflectance: linear interpolation of the material's 1-degree table (Eq. 4, Sec. III)
    uint32_t m = (uint32_t)__float_as_int(b.w);
    const uint32_t mrow = m < (uint32_t)T.n_mat ? m : (uint32_t)(T.n_mat - 1);
    int i = (int)theta_deg;
    if (i > LIDAR_TABLE_SIZE - 2) i = LIDAR_TABLE_SIZE - 2;
    const float f = theta_deg - (float)i;
    const float* row = T.table + (int64_t)mrow * LIDAR_TABLE_SIZE;
    const float R0 = __ldg(&row[i]), R1 = __ldg(&row[i + 1]);
    const float R = R0 * (1.0f - f) + R1 * f;
    // range with Gaussian noise (Sec. II-A)
    const float z = range_noise_normal(seed, beam, frame, sensor, sub);
    const float d = h.t + __fmaf_rn(sd.sigma_k, h.t, sd.sigma) * z;
    // capability model (Eq. 5) and range limits
    const float RLd = __fdiv_rn(__fmul_rn(sd.RL_max, d), sd.d_max);
    const int valid = (d >= sd.r_min) && (d <= sd.r_max) && (d <= sd.d_max) && (RLd <= R);
    const float rf = (sd.range_exp == 0.0f) ? 1.0f : powf(sd.r_ref / d, sd.range_exp);
    out.t = h.t;
    out.range = d;
    out.intensity = sd.gain * R * rf;
    out.theta_deg = theta_deg;
    out.rf = rf;
    out.nx = nx; out.ny = ny; out.nz = nz;
    out.tri = h.idx;
    out.inst = (uint32_t)__float_as_int(c.w);
    out.mat = m;
    out.valid = valid;
}

// Dense per-beam record of one beam (normal rotated into the sensor frame).
__device__ __forceinline__ void write_beam(const BeamsOut& out, int64_t o, const BeamResult& b, const float* P,
                                           int sub)
{
    if (out.valid) out.valid[o] = (uint8_t)b.valid;
    if (out.tri) out.tri[o] = b.tri;
    if (out.t) out.t[o] = b.t;
    if (out.range) out.range[o] = b.range;
    if (out.intensity) out.intensity[o] = b.intensity;
    if (out.normal) {
        // n_s = R^T n_w
        out.normal[3 * o + 0] = P[0] * b.nx + P[4] * b.ny + P[8] * b.nz;
        out.normal[3 * o + 1] = P[1] * b.nx + P[5] * b.ny + P[9] * b.nz;
        out.normal[3 * o + 2] = P[2] * b.nx + P[6] * b.ny + P[10] * b.nz;
    }
    if (out.mat) out.mat[o] = (uint16_t)b.mat;
    if (out.inst) out.inst[o] = b.inst;
    if (out.sub) out.sub[o] = (uint8_t)sub;
    if (out.theta_deg) out.theta_deg[o] = b.theta_deg;
    if (out.rf) out.rf[o] = b.rf;
}

}  // namespace
}  // namespace lidar
