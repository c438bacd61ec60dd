/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, deliberately unoptimised FP64 CPU implementation of per-beam
 * LiDAR return generation ("Physical LiDAR Simulation in Real-Time Engine",
 * Sec. II).  Only the test-suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no
 * source, header, table or helper with the CUDA library.
 *
 * What it computes, per (frame, beam, sub-ray):
 *   ray       : o = pose translation, d_w = R_pose * d_s, replayed in FP32 with
 *               the fixed operation order the library documents, then promoted.
 *   closest hit (replaces the depth-pass sample of Sec. II-A): brute force over
 *               every triangle, Moller-Trumbore in FP64, two-sided, closest by
 *               (t, triangle index) with t in (T_EPS, T_max].
 *   incidence angle (Sec. II-C): angle between the beam and the face normal,
 *               theta = atan2(|d x n|, |d . n|).
 *   reflectance (Eq. 4, generalised to a 91-entry table per material that is
 *               interpolated linearly over incidence angle, Sec. III).
 *   noise (Sec. II-A): d = t + (sigma + sigma_k t) z (sigma_k = 0: the paper's
 *               constant noise factor), z standard normal drawn by
 *               Box-Muller from Philox4x64-10 (Salmon et al., SC'11).
 *   capability model (Sec. II-D, Eq. 5): detected iff R_L(d) = RL_max/d_max*d
 *               <= R, with d <= d_max, and d inside [r_min, r_max].
 *   intensity : I = g * R * (r_ref / d)^p (p = 0 is the paper's reflectance
 *               intensity).
 *   sub-rays  : the strongest valid return among the beam's sub-rays.
 *   adjoint   : exact chain rule of the mean-squared intensity loss with the
 *               hits and masks held fixed, and of the table builder.
 *
 * Compile with -ffp-contract=off: the FP32 ray replay relies on every
 * operation being rounded exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_NO_HIT 0xFFFFFFFFu
#define ORACLE_T_EPS 1e-4
#define ORACLE_NTAB 91

/* exemption flags (counted by the tests, never silently passed) */
#define ORACLE_FLAG_EDGE 1u    /* a hit or near-miss closer than the hit lies within the edge band */
#define ORACLE_FLAG_TIE 2u     /* second-closest hit within 1e-6 relative of the closest */
#define ORACLE_FLAG_CUTOFF 4u  /* a cut-off decision within 1e-5 relative of its threshold */
#define ORACLE_FLAG_SUBTIE 8u  /* strongest-return choice among sub-rays is not unique */
#define ORACLE_FLAG_GRAZING 16u /* |cos(theta)| < 1e-2: range ill-conditioned in FP32 */

typedef struct {
    int64_t n_beams;
    const double* az;
    const double* el;
    float r_min, r_max, d_max, RL_max, sigma, gain, range_exp, r_ref, divergence;
    int32_t n_sub;
    float sigma_k;   /* noise standard deviation sigma + sigma_k * t at true range t */
} oracle_sensor;

typedef struct {
    int32_t sensor;
    int32_t frame;
    float pose[12]; /* row-major 3x4 [R | t], sensor -> world */
} oracle_frame;

typedef struct {
    /* per sample (one beam of one frame) */
    uint8_t* valid;
    uint32_t* tri;
    double* t;
    double* range;
    double* intensity;
    double* normal;    /* [3], sensor frame, facing the sensor */
    double* xyz;       /* [3], sensor frame */
    uint16_t* mat;
    uint32_t* inst;
    double* theta_deg;
    double* R;
    double* rf;
    int32_t* sub;
    uint32_t* flags;
    /* per sample x n_sub_max (each may be NULL) */
    uint8_t* sub_valid;
    double* sub_I;
    double* sub_range;
    uint32_t* sub_tri;
    uint32_t* sub_flags;
} oracle_out;

/* ------------------------------------------------------------ beam pattern */

/* Unit direction of beam (theta_i azimuth, phi_j elevation), Sec. II-A:
 * (cos phi cos theta, cos phi sin theta, sin phi) in FP64, rounded to FP32. */
void oracle_beam_dirs(int64_t n, const double* az, const double* el, float* out)
{
    for (int64_t b = 0; b < n; ++b) {
        double ce = cos(el[b]);
        out[3 * b + 0] = (float)(ce * cos(az[b]));
        out[3 * b + 1] = (float)(ce * sin(az[b]));
        out[3 * b + 2] = (float)sin(el[b]);
    }
}

/* Sub-ray offsets: sub-ray 0 is the beam itself; sub-rays 1..n-1 sit on a
 * cone of half-angle divergence/2 at azimuths 2*pi*(k-1)/(n-1) around it,
 * offset = tan(divergence/2) * (cos, sin).  FP64, rounded to FP32. */
void oracle_subray_offsets(float divergence, int32_t n_sub, float* alpha, float* beta)
{
    double r = tan(0.5 * (double)divergence);
    alpha[0] = 0.0f;
    beta[0] = 0.0f;
    for (int k = 1; k < n_sub; ++k) {
        double a = 2.0 * M_PI * (double)(k - 1) / (double)(n_sub - 1);
        alpha[k] = (float)(r * cos(a));
        beta[k] = (float)(r * sin(a));
    }
}

/* ----------------------------------------------------------------- FP32 ray */

/* World ray of one beam, in FP32, every operation rounded as written:
 * d_w[r] = fma(R[r][2], d[2], fma(R[r][1], d[1], R[r][0] * d[0])). */
void oracle_world_ray(const float* pose, const float* d, float* o_out, float* d_out)
{
    for (int r = 0; r < 3; ++r) {
        float p0 = pose[4 * r + 0] * d[0];
        float acc = fmaf(pose[4 * r + 1], d[1], p0);
        d_out[r] = fmaf(pose[4 * r + 2], d[2], acc);
        o_out[r] = pose[4 * r + 3];
    }
}

/* Sub-ray k of world direction d, FP32, each operation rounded as written:
 *   c = d x z_hat (or d x x_hat when |d x z_hat| < 1e-3), u = c / |c|,
 *   v = d x u, w = (d + alpha*u) + beta*v, sub = w / |w|.  Sub-ray 0 is d. */
void oracle_subray_dir(const float* d, float alpha, float beta, int k, float* out)
{
    if (k == 0) {
        out[0] = d[0]; out[1] = d[1]; out[2] = d[2];
        return;
    }
    float c0, c1, c2;
    float n2 = d[1] * d[1];
    float dx2 = d[0] * d[0];
    n2 = n2 + dx2;
    if (sqrtf(n2) >= 1e-3f) {
        c0 = d[1]; c1 = -d[0]; c2 = 0.0f;
    } else {
        c0 = 0.0f; c1 = d[2]; c2 = -d[1];
    }
    float cc = c0 * c0;
    float t1 = c1 * c1;
    float t2 = c2 * c2;
    cc = cc + t1;
    cc = cc + t2;
    float s = sqrtf(cc);
    float u0 = c0 / s, u1 = c1 / s, u2 = c2 / s;
    float v0 = d[1] * u2; float v0b = d[2] * u1; v0 = v0 - v0b;
    float v1 = d[2] * u0; float v1b = d[0] * u2; v1 = v1 - v1b;
    float v2 = d[0] * u1; float v2b = d[1] * u0; v2 = v2 - v2b;
    float w[3];
    float au0 = alpha * u0, au1 = alpha * u1, au2 = alpha * u2;
    float bv0 = beta * v0, bv1 = beta * v1, bv2 = beta * v2;
    w[0] = d[0] + au0; w[0] = w[0] + bv0;
    w[1] = d[1] + au1; w[1] = w[1] + bv1;
    w[2] = d[2] + au2; w[2] = w[2] + bv2;
    float ww = w[0] * w[0];
    float w1 = w[1] * w[1];
    float w2 = w[2] * w[2];
    ww = ww + w1;
    ww = ww + w2;
    float sw = sqrtf(ww);
    out[0] = w[0] / sw;
    out[1] = w[1] / sw;
    out[2] = w[2] / sw;
}

/* ------------------------------------------------------------ Philox4x64-10 */

/* Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
 * multiplies two words by the round constants, swaps the halves and xors the
 * high products with the other words and the key; the key is bumped by the
 * Weyl constants between rounds. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    __uint128_t p = (__uint128_t)a * (__uint128_t)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t* ctr_in, const uint64_t* key_in, uint64_t* out)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t h0, l0, h1, l1;
        mulhilo64(M0, c0, &h0, &l0);
        mulhilo64(M1, c2, &h1, &l1);
        uint64_t n0 = h1 ^ c1 ^ k0;
        uint64_t n1 = l1;
        uint64_t n2 = h0 ^ c3 ^ k1;
        uint64_t n3 = l0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normal for one ray: counter = (beam, frame | sensor << 32, sub, 0),
 * key = (seed, 0); u_j = ((x_j >> 11) + 1/2) 2^-53 in (0, 1); Box-Muller
 * z = sqrt(-2 ln u_0) cos(2 pi u_1), in FP64. */
double oracle_normal(uint64_t seed, uint64_t beam, uint32_t frame, uint32_t sensor, uint32_t sub)
{
    uint64_t ctr[4] = {beam, (uint64_t)frame | ((uint64_t)sensor << 32), (uint64_t)sub, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t x[4];
    oracle_philox4x64_10(ctr, key, x);
    double u0 = ((double)(x[0] >> 11) + 0.5) * 0x1p-53;
    double u1 = ((double)(x[1] >> 11) + 0.5) * 0x1p-53;
    return sqrt(-2.0 * log(u0)) * cos(2.0 * M_PI * u1);
}

/* ------------------------------------------------------------ material table */

/* T[m][k] = a_m cos(k deg) + s_m exp(-k^2 / (2 w_m^2)), k = 0..90 degrees:
 * the Lambertian law of Eq. 4 with R(0) = a_m plus a specular lobe of width w_m. */
void oracle_build_tables(const float* params, int32_t M, double* table)
{
    for (int m = 0; m < M; ++m) {
        double a = params[3 * m + 0], s = params[3 * m + 1], w = params[3 * m + 2];
        for (int k = 0; k < ORACLE_NTAB; ++k) {
            double kd = (double)k;
            table[m * ORACLE_NTAB + k] = a * cos(kd * M_PI / 180.0) + s * exp(-kd * kd / (2.0 * w * w));
        }
    }
}

/* Chain rule of oracle_build_tables: given dL/dT, returns dL/d(a, s, w). */
void oracle_build_tables_backward(const float* params, const double* grad_table, int32_t M,
                                  double* grad_params)
{
    for (int m = 0; m < M; ++m) {
        double s = params[3 * m + 1], w = params[3 * m + 2];
        double ga = 0.0, gs = 0.0, gw = 0.0;
        for (int k = 0; k < ORACLE_NTAB; ++k) {
            double kd = (double)k;
            double g = grad_table[m * ORACLE_NTAB + k];
            double e = exp(-kd * kd / (2.0 * w * w));
            ga += g * cos(kd * M_PI / 180.0);
            gs += g * e;
            gw += g * s * e * kd * kd / (w * w * w);
        }
        grad_params[3 * m + 0] = ga;
        grad_params[3 * m + 1] = gs;
        grad_params[3 * m + 2] = gw;
    }
}

/* Linear interpolation of a table row over the 1-degree grid. */
static double oracle_lerp_row(const double* row, double theta_deg, int* i_out, double* f_out)
{
    int i = (int)floor(theta_deg);
    if (i > ORACLE_NTAB - 2) i = ORACLE_NTAB - 2;
    if (i < 0) i = 0;
    double f = theta_deg - (double)i;
    *i_out = i;
    *f_out = f;
    return row[i] * (1.0 - f) + row[i + 1] * f;
}

/* ------------------------------------------------------------ scene (FP64) */

typedef struct {
    int64_t n;
    double *v0, *e1, *e2; /* [n][3] each, exact promotions of the FP32 input */
    double* vmax;          /* max |coordinate| of the triangle's vertices */
} oracle_tris;

static void oracle_tris_init(oracle_tris* S, const float* verts, const uint32_t* tris, int64_t nt)
{
    S->n = nt;
    S->v0 = (double*)malloc(sizeof(double) * 3 * nt);
    S->e1 = (double*)malloc(sizeof(double) * 3 * nt);
    S->e2 = (double*)malloc(sizeof(double) * 3 * nt);
    S->vmax = (double*)malloc(sizeof(double) * nt);
    for (int64_t i = 0; i < nt; ++i) {
        const float* a = verts + 3 * (int64_t)tris[3 * i + 0];
        const float* b = verts + 3 * (int64_t)tris[3 * i + 1];
        const float* c = verts + 3 * (int64_t)tris[3 * i + 2];
        double vm = 0.0;
        for (int k = 0; k < 3; ++k) {
            S->v0[3 * i + k] = (double)a[k];
            S->e1[3 * i + k] = (double)b[k] - (double)a[k];
            S->e2[3 * i + k] = (double)c[k] - (double)a[k];
            vm = fmax(vm, fabs((double)a[k]));
            vm = fmax(vm, fabs((double)b[k]));
            vm = fmax(vm, fabs((double)c[k]));
        }
        S->vmax[i] = vm;
    }
}

static void oracle_tris_free(oracle_tris* S)
{
    free(S->v0); free(S->e1); free(S->e2); free(S->vmax);
}

static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Moller-Trumbore, two-sided.  Returns 1 on a hit inside the closed triangle
 * (t unrestricted) and writes t, u, v; returns 0 when det == 0 or outside. */
static int mt_intersect(const double* o, const double* d, const double* v0, const double* e1,
                        const double* e2, double* t, double* u_out, double* v_out)
{
    double p[3], s[3], q[3];
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    s[0] = o[0] - v0[0]; s[1] = o[1] - v0[1]; s[2] = o[2] - v0[2];
    double u = dot3(s, p) * inv;
    cross3(s, e1, q);
    double v = dot3(d, q) * inv;
    *t = dot3(e2, q) * inv;
    *u_out = u;
    *v_out = v;
    return (u >= 0.0 && v >= 0.0 && u + v <= 1.0) ? 1 : 0;
}

/* Signed distance (metres, in the triangle's plane) from the ray's crossing of
 * the plane to the nearest edge: >= 0 inside, < 0 outside (a lower bound on the
 * distance to the triangle when outside).  Returns 0 when det == 0. */
static int edge_distance(const double* o, const double* d, const double* v0, const double* e1,
                         const double* e2, double* t_plane, double* dist)
{
    double p[3], s[3], q[3], n[3], e3[3];
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    s[0] = o[0] - v0[0]; s[1] = o[1] - v0[1]; s[2] = o[2] - v0[2];
    double u = dot3(s, p) * inv;
    cross3(s, e1, q);
    double v = dot3(d, q) * inv;
    *t_plane = dot3(e2, q) * inv;
    double w = 1.0 - u - v;
    cross3(e1, e2, n);
    double area2 = sqrt(dot3(n, n));
    e3[0] = e2[0] - e1[0]; e3[1] = e2[1] - e1[1]; e3[2] = e2[2] - e1[2];
    double h0 = area2 / sqrt(dot3(e3, e3)); /* altitude from v0 */
    double h1 = area2 / sqrt(dot3(e2, e2)); /* altitude from v1 */
    double h2 = area2 / sqrt(dot3(e1, e1)); /* altitude from v2 */
    double d0 = w * h0, d1 = u * h1, d2 = v * h2;
    *dist = fmin(d0, fmin(d1, d2));
    return 1;
}

typedef struct {
    uint32_t tri;     /* original triangle index or ORACLE_NO_HIT */
    double t;
    double range;
    double I, R, rf, theta_deg;
    double n_world[3];
    uint32_t flags;
    int valid;
} ray_result;

/* Closest hit of one ray over every triangle (brute force), with the EDGE,
 * TIE and (t near T_max) CUTOFF flags.  Returns the triangle or -1. */
static int64_t oracle_closest(const oracle_tris* S, const double* o, const double* d, double T_max,
                              double* t_out, uint32_t* flags)
{
    double best_t = INFINITY, second_t = INFINITY;
    int64_t best = -1;

    /* closest hit: brute force over every triangle */
    for (int64_t i = 0; i < S->n; ++i) {
        double t, u, v;
        if (!mt_intersect(o, d, S->v0 + 3 * i, S->e1 + 3 * i, S->e2 + 3 * i, &t, &u, &v)) continue;
        if (!(t > ORACLE_T_EPS && t <= T_max)) continue;
        if (t < best_t) {
            second_t = best_t;
            best_t = t;
            best = i;
        } else if (t == best_t) {
            second_t = t; /* equal depth: keep the lower index (loop order) */
        } else if (t < second_t) {
            second_t = t;
        }
    }

    uint32_t res_flags = 0;
    double onorm = fmax(fabs(o[0]), fmax(fabs(o[1]), fabs(o[2])));
    /* edge band: any triangle whose crossing is at or before the hit (or before
     * T_max on a miss) and lies within 1e-6 relative of one of its edges */
    double limit = (best >= 0) ? best_t * (1.0 + 1e-6) : T_max * (1.0 + 1e-5);
    for (int64_t i = 0; i < S->n; ++i) {
        double tp, dist;
        if (!edge_distance(o, d, S->v0 + 3 * i, S->e1 + 3 * i, S->e2 + 3 * i, &tp, &dist)) continue;
        if (!(tp > ORACLE_T_EPS * (1.0 - 1e-6) && tp <= limit)) continue;
        double band = 1e-6 * fmax(onorm, fmax(S->vmax[i], fabs(tp)));
        if (fabs(dist) < band) {
            res_flags |= ORACLE_FLAG_EDGE;
            break;
        }
    }
    if (best >= 0 && second_t <= best_t * (1.0 + 1e-6)) res_flags |= ORACLE_FLAG_TIE;
    if (best >= 0 && fabs(best_t - T_max) <= 1e-5 * T_max) res_flags |= ORACLE_FLAG_CUTOFF;
    *flags = res_flags;
    *t_out = best_t;
    return best;
}

/* One ray through the whole per-beam model (everything but the sub-ray reduce). */
static void oracle_one_ray(const oracle_tris* S, const uint16_t* mat, const double* table, int32_t n_mat,
                           const oracle_sensor* sen, const float* o32, const float* d32, uint64_t seed,
                           uint64_t beam, uint32_t frame, uint32_t sensor_id, uint32_t sub, ray_result* res)
{
    double o[3] = {o32[0], o32[1], o32[2]};
    double d[3] = {d32[0], d32[1], d32[2]};
    double T_max = ((double)fminf(sen->r_max, sen->d_max) + 9.0 * (double)sen->sigma) /
                   (1.0 - 9.0 * (double)sen->sigma_k);
    double best_t;
    int64_t best = oracle_closest(S, o, d, T_max, &best_t, &res->flags);
    if (best < 0) {
        /* a miss whose nearest crossing is just beyond T_max could flip */
        res->tri = ORACLE_NO_HIT;
        res->t = INFINITY;
        res->range = INFINITY;
        res->I = res->R = res->rf = res->theta_deg = 0.0;
        res->n_world[0] = res->n_world[1] = res->n_world[2] = 0.0;
        res->valid = 0;
        return;
    }

    /* surface attributes: face normal facing the sensor */
    const double* e1 = S->e1 + 3 * best;
    const double* e2 = S->e2 + 3 * best;
    double n[3];
    cross3(e1, e2, n);
    double nl = sqrt(dot3(n, n));
    n[0] /= nl; n[1] /= nl; n[2] /= nl;
    if (dot3(n, d) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }

    /* incidence angle */
    double c[3];
    cross3(d, n, c);
    double theta = atan2(sqrt(dot3(c, c)), fabs(dot3(d, n)));
    double theta_deg = theta * 180.0 / M_PI;
    double cos_abs = fabs(dot3(d, n)) / sqrt(dot3(d, d));
    if (cos_abs < 1e-2) res->flags |= ORACLE_FLAG_GRAZING;

    /* reflectance lookup */
    int m = mat[best];
    if (m >= n_mat) m = n_mat - 1;
    int ii;
    double ff;
    double R = oracle_lerp_row(table + (int64_t)m * ORACLE_NTAB, theta_deg, &ii, &ff);

    /* range noise */
    double z = oracle_normal(seed, beam, frame, sensor_id, sub);
    double dist = best_t + ((double)sen->sigma + (double)sen->sigma_k * best_t) * z;

    /* cut-offs */
    double r_min = sen->r_min, r_max = sen->r_max, d_max = sen->d_max, RL = sen->RL_max;
    double RLd = RL * dist / d_max;
    int valid = (dist >= r_min) && (dist <= r_max) && (dist <= d_max) && (RLd <= R);
    double tol = 1e-5 * fabs(dist);
    if (fabs(dist - r_min) <= tol || fabs(dist - r_max) <= tol || fabs(dist - d_max) <= tol ||
        fabs(RLd - R) <= 1e-5 * fmax(fabs(R), fabs(RLd)))
        res->flags |= ORACLE_FLAG_CUTOFF;

    /* intensity */
    double rf = (sen->range_exp == 0.0f) ? 1.0 : pow((double)sen->r_ref / dist, (double)sen->range_exp);
    double I = (double)sen->gain * R * rf;

    res->tri = (uint32_t)best;
    res->t = best_t;
    res->range = dist;
    res->I = I;
    res->R = R;
    res->rf = rf;
    res->theta_deg = theta_deg;
    res->n_world[0] = n[0]; res->n_world[1] = n[1]; res->n_world[2] = n[2];
    res->valid = valid;
}

/* Per-beam return generation for a list of (frame entry, beam) samples.
 * `table` is [n_mat][91] in FP64.  Returns 0 on success, -1 on bad input. */
int oracle_cast(const float* verts, int64_t n_verts, const uint32_t* tris, int64_t n_tris,
                const uint16_t* mat, const uint32_t* inst, const oracle_sensor* sensors, int32_t n_sensors,
                const oracle_frame* frames, int32_t n_frames, const double* table, int32_t n_mat,
                uint64_t seed, const int64_t* sample_frame, const int64_t* sample_beam, int64_t n_samples,
                int32_t n_sub_max, oracle_out* out, int32_t n_threads)
{
    for (int64_t i = 0; i < 3 * n_tris; ++i)
        if ((int64_t)tris[i] >= n_verts) return -1;
    for (int64_t s = 0; s < n_samples; ++s) {
        if (sample_frame[s] < 0 || sample_frame[s] >= n_frames) return -1;
        const oracle_frame* fr = frames + sample_frame[s];
        if (fr->sensor < 0 || fr->sensor >= n_sensors) return -1;
        if (sample_beam[s] < 0 || sample_beam[s] >= sensors[fr->sensor].n_beams) return -1;
        if (sensors[fr->sensor].n_sub > n_sub_max || sensors[fr->sensor].n_sub < 1) return -1;
    }
    oracle_tris S;
    oracle_tris_init(&S, verts, tris, n_tris);

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < n_samples; ++s) {
        const oracle_frame* fr = frames + sample_frame[s];
        const oracle_sensor* sen = sensors + fr->sensor;
        int64_t b = sample_beam[s];
        float ds[3];
        oracle_beam_dirs(1, sen->az + b, sen->el + b, ds);
        float o32[3], dw[3];
        oracle_world_ray(fr->pose, ds, o32, dw);
        float alpha[64], beta[64];
        oracle_subray_offsets(sen->divergence, sen->n_sub, alpha, beta);

        ray_result best_res;
        int chosen = 0;
        double best_I = -1.0, second_I = -1.0;
        uint32_t any_flags = 0;
        ray_result first;
        for (int k = 0; k < sen->n_sub; ++k) {
            float dk[3];
            oracle_subray_dir(dw, alpha[k], beta[k], k, dk);
            ray_result r;
            oracle_one_ray(&S, mat, table, n_mat, sen, o32, dk, seed, (uint64_t)b, (uint32_t)fr->frame,
                           (uint32_t)fr->sensor, (uint32_t)k, &r);
            if (k == 0) first = r;
            any_flags |= r.flags;
            if (out->sub_valid) out->sub_valid[s * n_sub_max + k] = (uint8_t)r.valid;
            if (out->sub_I) out->sub_I[s * n_sub_max + k] = r.I;
            if (out->sub_range) out->sub_range[s * n_sub_max + k] = r.range;
            if (out->sub_tri) out->sub_tri[s * n_sub_max + k] = (r.tri == ORACLE_NO_HIT) ? ORACLE_NO_HIT : r.tri;
            if (out->sub_flags) out->sub_flags[s * n_sub_max + k] = r.flags;
            if (r.valid) {
                if (r.I > best_I) {
                    second_I = best_I;
                    best_I = r.I;
                    best_res = r;
                    chosen = k;
                } else if (r.I > second_I) {
                    second_I = r.I;
                }
            }
        }
        if (best_I < 0.0) {
            best_res = first;
            chosen = 0;
        }
        uint32_t flags = best_res.flags;
        if (sen->n_sub > 1) {
            double tolI = 1e-4 * fabs(best_I) + 1e-7 * (double)sen->gain;
            if ((second_I >= 0.0 && best_I - second_I <= tolI) ||
                (any_flags & (ORACLE_FLAG_EDGE | ORACLE_FLAG_TIE | ORACLE_FLAG_CUTOFF)))
                flags |= ORACLE_FLAG_SUBTIE;
        }
        out->valid[s] = (uint8_t)best_res.valid;
        out->tri[s] = best_res.tri;
        out->t[s] = best_res.t;
        out->range[s] = best_res.range;
        out->intensity[s] = best_res.I;
        out->theta_deg[s] = best_res.theta_deg;
        out->R[s] = best_res.R;
        out->rf[s] = best_res.rf;
        out->sub[s] = chosen;
        out->flags[s] = flags;
        if (best_res.tri != ORACLE_NO_HIT) {
            out->mat[s] = mat[best_res.tri];
            out->inst[s] = inst[best_res.tri];
            /* normal into the sensor frame: n_s = R^T n_w */
            for (int c = 0; c < 3; ++c)
                out->normal[3 * s + c] = (double)fr->pose[0 + c] * best_res.n_world[0] +
                                         (double)fr->pose[4 + c] * best_res.n_world[1] +
                                         (double)fr->pose[8 + c] * best_res.n_world[2];
            for (int c = 0; c < 3; ++c) out->xyz[3 * s + c] = best_res.range * (double)ds[c];
        } else {
            out->mat[s] = 0;
            out->inst[s] = 0;
            for (int c = 0; c < 3; ++c) { out->normal[3 * s + c] = 0.0; out->xyz[3 * s + c] = 0.0; }
        }
    }
    oracle_tris_free(&S);
    return 0;
}

/* ---------------------------------------- rolling shutter and multi-echo */

/* Rolling shutter (Sec. II-A: the camera is turned with the sensor's spin
 * over each time step): beam b fires at the fraction s_b of the sweep, its
 * azimuth over 2 pi taken in [0, 1) (the sweep starts at azimuth 0 and turns
 * towards +y), and sees the pose interpolated between the sweep's start and
 * end poses: translation (1 - s) t0 + s t1, rotation the normalised linear
 * blend (1 - s) q0 + s q1 of the two poses' unit quaternions (taken on the
 * same hemisphere); both blends are exact at s = 0 and s = 1.
 * The quaternions are found from the rotation matrices in FP64 and rounded
 * once; the blend, its normalisation, the matrix of the blended quaternion and
 * the translation are FP32 with every operation rounded as written.
 *
 * Multi-echo (Sec. IV, future work): from the returns of a beam's sub-rays,
 *   mode 0: the n strongest, strongest first (ties to the lower sub-ray),
 *           skipping a return closer than `separation` in range to one kept;
 *   mode 1: the first (smallest range) and the last (largest range) return,
 *           the last only if it lies at least `separation` beyond the first
 *           (ties to the lower sub-ray). */
#define ORACLE_FLAG_ECHO 32u /* echo choice within tolerance of a tie or of the separation */

typedef struct {
    int32_t sensor;
    int32_t frame;
    float pose0[12];
    float pose1[12];
} oracle_sweep_frame;

typedef struct {
    int32_t n_echoes;
    int32_t mode;
    float separation;
    uint8_t* count;
    double* range;      /* [n][n_echoes] */
    double* intensity;
    uint32_t* tri;
    int32_t* sub;
} oracle_echoes;

/* firing fraction of a beam of azimuth az */
float oracle_sweep_fraction(double az)
{
    double s = fmod(az, 2.0 * M_PI) / (2.0 * M_PI);
    if (s < 0.0) s += 1.0;
    if (s >= 1.0) s = 0.0;
    return (float)s;
}

/* unit quaternion (w, x, y, z) of the rotation part of a row-major 3x4 pose,
 * by the largest of the four diagonal combinations (Shepperd 1978), FP64 */
static void pose_quaternion(const float* P, double* q)
{
    const double m00 = P[0], m01 = P[1], m02 = P[2], m10 = P[4], m11 = P[5], m12 = P[6];
    const double m20 = P[8], m21 = P[9], m22 = P[10];
    const double tr = m00 + m11 + m22;
    if (tr >= m00 && tr >= m11 && tr >= m22) {
        const double r = sqrt(1.0 + tr), h = 0.5 / r;
        q[0] = 0.5 * r; q[1] = (m21 - m12) * h; q[2] = (m02 - m20) * h; q[3] = (m10 - m01) * h;
    } else if (m00 >= m11 && m00 >= m22) {
        const double r = sqrt(1.0 + m00 - m11 - m22), h = 0.5 / r;
        q[0] = (m21 - m12) * h; q[1] = 0.5 * r; q[2] = (m01 + m10) * h; q[3] = (m02 + m20) * h;
    } else if (m11 >= m22) {
        const double r = sqrt(1.0 + m11 - m00 - m22), h = 0.5 / r;
        q[0] = (m02 - m20) * h; q[1] = (m01 + m10) * h; q[2] = 0.5 * r; q[3] = (m12 + m21) * h;
    } else {
        const double r = sqrt(1.0 + m22 - m00 - m11), h = 0.5 / r;
        q[0] = (m10 - m01) * h; q[1] = (m02 + m20) * h; q[2] = (m12 + m21) * h; q[3] = 0.5 * r;
    }
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

/* the sweep's two quaternions, same hemisphere, rounded to FP32 */
void oracle_sweep_quaternions(const float* pose0, const float* pose1, float* q0f, float* q1f)
{
    double q0[4], q1[4];
    pose_quaternion(pose0, q0);
    pose_quaternion(pose1, q1);
    const double dq = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2] + q0[3] * q1[3];
    for (int i = 0; i < 4; ++i) {
        q0f[i] = (float)q0[i];
        q1f[i] = (float)(dq < 0.0 ? -q1[i] : q1[i]);
    }
}

/* pose at fraction s of the sweep, FP32, every operation rounded as written */
void oracle_sweep_pose(const float* q0, const float* q1, const float* pose0, const float* pose1, float s,
                       float* P)
{
    const float ms = 1.0f - s;
    float q[4];
    for (int i = 0; i < 4; ++i) {
        float a = ms * q0[i];
        q[i] = fmaf(s, q1[i], a);
    }
    float n2 = q[0] * q[0];
    float t1 = q[1] * q[1];
    float t2 = q[2] * q[2];
    float t3 = q[3] * q[3];
    n2 = n2 + t1;
    n2 = n2 + t2;
    n2 = n2 + t3;
    float inv = 1.0f / sqrtf(n2);
    const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
    float a;
    a = yy + zz; P[0] = 1.0f - 2.0f * a;
    a = xy - wz; P[1] = 2.0f * a;
    a = xz + wy; P[2] = 2.0f * a;
    a = xy + wz; P[4] = 2.0f * a;
    a = xx + zz; P[5] = 1.0f - 2.0f * a;
    a = yz - wx; P[6] = 2.0f * a;
    a = xz - wy; P[8] = 2.0f * a;
    a = yz + wx; P[9] = 2.0f * a;
    a = xx + yy; P[10] = 1.0f - 2.0f * a;
    for (int r = 0; r < 3; ++r) {
        float a = ms * pose0[4 * r + 3];
        P[4 * r + 3] = fmaf(s, pose1[4 * r + 3], a);
    }
}

/* echo choice from the kept sub-ray returns of one beam */
static int oracle_pick_echoes(int n_sub, const ray_result* rr, int mode, int n_echoes, double sep, int* pick,
                              uint32_t* flags)
{
    int n = 0;
    uint32_t f = 0;
    int idx[64], m = 0;
    for (int k = 0; k < n_sub; ++k)
        if (rr[k].valid) idx[m++] = k;
    for (int a = 0; a < m; ++a)
        for (int b = a + 1; b < m; ++b) {
            const ray_result *ra = rr + idx[a], *rb = rr + idx[b];
            const double dI = fabs(ra->I - rb->I), dR = fabs(ra->range - rb->range);
            if (mode == 0 && dI <= 1e-4 * fmax(ra->I, rb->I) + 1e-7) f |= ORACLE_FLAG_ECHO;
            if (mode == 1 && dR <= 1e-5 * fmax(ra->range, rb->range)) f |= ORACLE_FLAG_ECHO;
            if (fabs(dR - sep) <= 1e-5 * fmax(ra->range, rb->range) + 1e-6) f |= ORACLE_FLAG_ECHO;
        }
    for (int k = 0; k < n_sub; ++k)
        if (rr[k].flags & (ORACLE_FLAG_EDGE | ORACLE_FLAG_TIE | ORACLE_FLAG_CUTOFF)) f |= ORACLE_FLAG_ECHO;
    if (mode == 0) {
        int used[64] = {0};
        while (n < n_echoes) {
            int best = -1;
            for (int a = 0; a < m; ++a) {
                if (used[a]) continue;
                if (best < 0 || rr[idx[a]].I > rr[idx[best]].I) best = a;
            }
            if (best < 0) break;
            used[best] = 1;
            int ok = 1;
            for (int j = 0; j < n; ++j)
                if (fabs(rr[idx[best]].range - rr[pick[j]].range) < sep) ok = 0;
            if (ok) pick[n++] = idx[best];
        }
    } else if (m > 0) {
        int first = idx[0], last = idx[0];
        for (int a = 1; a < m; ++a) {
            if (rr[idx[a]].range < rr[first].range) first = idx[a];
            if (rr[idx[a]].range > rr[last].range) last = idx[a];
        }
        pick[n++] = first;
        if (n_echoes > 1 && rr[last].range - rr[first].range >= sep) pick[n++] = last;
    }
    *flags |= f;
    return n;
}

int oracle_cast_sweep(const float* verts, int64_t n_verts, const uint32_t* tris, int64_t n_tris,
                      const uint16_t* mat, const uint32_t* inst, const oracle_sensor* sensors, int32_t n_sensors,
                      const oracle_sweep_frame* frames, int32_t n_frames, const double* table, int32_t n_mat,
                      uint64_t seed, const int64_t* sample_frame, const int64_t* sample_beam, int64_t n_samples,
                      int32_t n_sub_max, oracle_out* out, oracle_echoes* echo, int32_t n_threads)
{
    if (echo && (echo->n_echoes < 1 || echo->n_echoes > 4 || echo->mode < 0 || echo->mode > 1)) return -1;
    for (int64_t i = 0; i < 3 * n_tris; ++i)
        if ((int64_t)tris[i] >= n_verts) return -1;
    for (int64_t s = 0; s < n_samples; ++s) {
        if (sample_frame[s] < 0 || sample_frame[s] >= n_frames) return -1;
        const oracle_sweep_frame* fr = frames + sample_frame[s];
        if (fr->sensor < 0 || fr->sensor >= n_sensors) return -1;
        if (sample_beam[s] < 0 || sample_beam[s] >= sensors[fr->sensor].n_beams) return -1;
        if (sensors[fr->sensor].n_sub > n_sub_max || sensors[fr->sensor].n_sub < 1 ||
            sensors[fr->sensor].n_sub > 64) return -1;
    }
    oracle_tris S;
    oracle_tris_init(&S, verts, tris, n_tris);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < n_samples; ++s) {
        const oracle_sweep_frame* fr = frames + sample_frame[s];
        const oracle_sensor* sen = sensors + fr->sensor;
        const int64_t b = sample_beam[s];
        float q0[4], q1[4], P[12];
        oracle_sweep_quaternions(fr->pose0, fr->pose1, q0, q1);
        oracle_sweep_pose(q0, q1, fr->pose0, fr->pose1, oracle_sweep_fraction(sen->az[b]), P);
        float ds[3], o32[3], dw[3];
        oracle_beam_dirs(1, sen->az + b, sen->el + b, ds);
        oracle_world_ray(P, ds, o32, dw);
        float alpha[64], beta[64];
        oracle_subray_offsets(sen->divergence, sen->n_sub, alpha, beta);
        ray_result rr[64];
        int chosen = 0;
        double best_I = -1.0, second_I = -1.0;
        uint32_t any_flags = 0;
        for (int k = 0; k < sen->n_sub; ++k) {
            float dk[3];
            oracle_subray_dir(dw, alpha[k], beta[k], k, dk);
            oracle_one_ray(&S, mat, table, n_mat, sen, o32, dk, seed, (uint64_t)b, (uint32_t)fr->frame,
                           (uint32_t)fr->sensor, (uint32_t)k, rr + k);
            any_flags |= rr[k].flags;
            if (rr[k].valid) {
                if (rr[k].I > best_I) {
                    second_I = best_I;
                    best_I = rr[k].I;
                    chosen = k;
                } else if (rr[k].I > second_I) {
                    second_I = rr[k].I;
                }
            }
        }
        const ray_result* best = rr + chosen;
        uint32_t flags = best->flags;
        if (sen->n_sub > 1) {
            double tolI = 1e-4 * fabs(best_I) + 1e-7 * (double)sen->gain;
            if ((second_I >= 0.0 && best_I - second_I <= tolI) ||
                (any_flags & (ORACLE_FLAG_EDGE | ORACLE_FLAG_TIE | ORACLE_FLAG_CUTOFF)))
                flags |= ORACLE_FLAG_SUBTIE;
        }
        if (echo) {
            int pick[4];
            const int ne = oracle_pick_echoes(sen->n_sub, rr, echo->mode, echo->n_echoes, (double)echo->separation,
                                              pick, &flags);
            echo->count[s] = (uint8_t)ne;
            for (int j = 0; j < echo->n_echoes; ++j) {
                const int64_t e = s * echo->n_echoes + j;
                if (j < ne) {
                    echo->range[e] = rr[pick[j]].range;
                    echo->intensity[e] = rr[pick[j]].I;
                    echo->tri[e] = rr[pick[j]].tri;
                    echo->sub[e] = pick[j];
                } else {
                    echo->range[e] = 0.0;
                    echo->intensity[e] = 0.0;
                    echo->tri[e] = ORACLE_NO_HIT;
                    echo->sub[e] = -1;
                }
            }
        }
        out->valid[s] = (uint8_t)best->valid;
        out->tri[s] = best->tri;
        out->t[s] = best->t;
        out->range[s] = best->range;
        out->intensity[s] = best->I;
        out->theta_deg[s] = best->theta_deg;
        out->R[s] = best->R;
        out->rf[s] = best->rf;
        out->sub[s] = chosen;
        out->flags[s] = flags;
        if (out->sub_valid)
            for (int k = 0; k < sen->n_sub; ++k) {
                out->sub_valid[s * n_sub_max + k] = (uint8_t)rr[k].valid;
                out->sub_I[s * n_sub_max + k] = rr[k].I;
                out->sub_range[s * n_sub_max + k] = rr[k].range;
                out->sub_tri[s * n_sub_max + k] = rr[k].tri;
                out->sub_flags[s * n_sub_max + k] = rr[k].flags;
            }
        if (best->tri != ORACLE_NO_HIT) {
            out->mat[s] = mat[best->tri];
            out->inst[s] = inst[best->tri];
            for (int c = 0; c < 3; ++c)
                out->normal[3 * s + c] = (double)P[0 + c] * best->n_world[0] + (double)P[4 + c] * best->n_world[1] +
                                         (double)P[8 + c] * best->n_world[2];
            for (int c = 0; c < 3; ++c) out->xyz[3 * s + c] = best->range * (double)ds[c];
        } else {
            out->mat[s] = 0;
            out->inst[s] = 0;
            for (int c = 0; c < 3; ++c) { out->normal[3 * s + c] = 0.0; out->xyz[3 * s + c] = 0.0; }
        }
    }
    oracle_tris_free(&S);
    return 0;
}

/* ------------------------------------------------ raster-and-resample path */

/* The paper's own sampling path (Sec. II-A..II-C): per frame, K pin-hole
 * cameras at the sensor pose share the sensor's 360-degree horizontal field
 * (camera k looks along sensor azimuth -pi + (k + 1/2) 2 pi / K, square W x W
 * image, FOV_c = 2 pi / K); each renders the depth pass, the incidence angle,
 * the material stencil and the instance colour of the surface seen through
 * every pixel centre; each beam then reads the pixel its direction projects to
 * (intrinsics of Eq. 1-2, pixel coordinates of Eq. 3 in the corrected form
 * n_x = c + f x/z, n_y = c - f y/z with (x, y, z) the beam in camera axes).
 *
 *   camera    : the k maximising d . F_k (FP32, ties to the lowest k),
 *               F_k = (cos, sin, 0) of its azimuth, L_k = (-sin, cos, 0), U = z.
 *   pixel     : (floor n_x, floor n_y) in FP32, every operation rounded as
 *               written; the column is clamped to [0, W) (a beam on the border
 *               of two cameras), a row outside [0, W) leaves the beam without
 *               a return.
 *   pixel ray : through the pixel centre, a = (i + 1/2 - c)/f,
 *               b = (c - (j + 1/2))/f, dir = (F + a L + b U) / sqrt(1 + a^2 + b^2)
 *               in FP32, then to the world like a beam.
 *   depth     : z-depth of the closest hit (FP64 brute force), z = t |dir . F|,
 *               rounded to FP32 and stored as 24-bit fixed point of z / T_max
 *               (q = rn(z * (2^24 - 1) / T_max), at most 2^24 - 2; 2^24 - 1
 *               marks no hit) — the "three bytes unsigned precision" of Sec. II-A.
 *   angle     : incidence angle of the pixel ray on the face (Sec. II-C), FP32,
 *               24-bit fixed point of theta / 90 degrees; material in the 8-bit
 *               stencil (mat & 255), instance as a 24-bit colour (inst & 2^24-1).
 *   beam      : range = z' / (d . F_k) (the pixel's depth read along the beam),
 *               theta = theta', then noise, Eq. 4 lookup, Eq. 5 and intensity as
 *               in the ray-cast path (sub-ray 0's noise draw).
 * The FP32 quantisation codes are computed from the FP64 values rounded to
 * FP32, with the library's operation order. */
typedef struct {
    int32_t width;
    int32_t n_cameras;
} oracle_raster_cfg;

typedef struct {
    uint8_t* valid;
    uint8_t* outside;      /* beam projects outside every camera image */
    int32_t* cam;
    int32_t* px;
    int32_t* py;
    uint32_t* tri;         /* triangle seen through the pixel centre */
    uint32_t* q_depth;
    uint32_t* q_angle;
    uint16_t* mat;         /* 8-bit stencil */
    uint32_t* inst;        /* 24-bit colour */
    double* t;             /* pixel ray distance to the hit */
    double* z;             /* z-depth before quantisation */
    double* range;
    double* intensity;
    double* theta_deg;     /* decoded */
    uint32_t* flags;
} oracle_raster_out;

/* camera constants as FP32, from the definitions in FP64 */
static void oracle_raster_consts(const oracle_raster_cfg* cfg, float* f, float* c, float* ck, float* sk)
{
    double fov = 2.0 * M_PI / (double)cfg->n_cameras;
    *f = (float)((double)cfg->width / (2.0 * tan(0.5 * fov)));
    *c = (float)(0.5 * (double)cfg->width);
    for (int k = 0; k < cfg->n_cameras; ++k) {
        double az = -M_PI + ((double)k + 0.5) * fov;
        ck[k] = (float)cos(az);
        sk[k] = (float)sin(az);
    }
}

int oracle_raster(const float* verts, int64_t n_verts, const uint32_t* tris, int64_t n_tris,
                  const uint16_t* mat, const uint32_t* inst, const oracle_sensor* sensors, int32_t n_sensors,
                  const oracle_frame* frames, int32_t n_frames, const double* table, int32_t n_mat,
                  uint64_t seed, const oracle_raster_cfg* cfg, const int64_t* sample_frame,
                  const int64_t* sample_beam, int64_t n_samples, oracle_raster_out* out, int32_t n_threads)
{
    if (cfg->width < 1 || cfg->n_cameras < 3 || cfg->n_cameras > 64) return -1;
    for (int64_t i = 0; i < 3 * n_tris; ++i)
        if ((int64_t)tris[i] >= n_verts) return -1;
    for (int64_t s = 0; s < n_samples; ++s) {
        if (sample_frame[s] < 0 || sample_frame[s] >= n_frames) return -1;
        const oracle_frame* fr = frames + sample_frame[s];
        if (fr->sensor < 0 || fr->sensor >= n_sensors) return -1;
        if (sample_beam[s] < 0 || sample_beam[s] >= sensors[fr->sensor].n_beams) return -1;
    }
    float f, c, ck[64], sk[64];
    oracle_raster_consts(cfg, &f, &c, ck, sk);
    const int W = cfg->width, K = cfg->n_cameras;
    oracle_tris S;
    oracle_tris_init(&S, verts, tris, n_tris);

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < n_samples; ++s) {
        const oracle_frame* fr = frames + sample_frame[s];
        const oracle_sensor* sen = sensors + fr->sensor;
        const int64_t b = sample_beam[s];
        float ds[3];
        oracle_beam_dirs(1, sen->az + b, sen->el + b, ds);
        out->valid[s] = 0;
        out->outside[s] = 1;
        out->cam[s] = -1;
        out->px[s] = out->py[s] = -1;
        out->tri[s] = ORACLE_NO_HIT;
        out->q_depth[s] = 0xFFFFFFu;
        out->q_angle[s] = 0;
        out->mat[s] = 0;
        out->inst[s] = 0;
        out->t[s] = out->z[s] = out->range[s] = INFINITY;
        out->intensity[s] = 0.0;
        out->theta_deg[s] = 0.0;
        out->flags[s] = 0;

        /* camera: largest d . F_k */
        int k = 0;
        float zk = 0.0f;
        for (int j = 0; j < K; ++j) {
            float p0 = ds[0] * ck[j];
            float p1 = ds[1] * sk[j];
            float zj = p0 + p1;
            if (j == 0 || zj > zk) { zk = zj; k = j; }
        }
        out->cam[s] = k;
        if (!(zk > 0.0f)) continue;
        /* projection (corrected Eq. 3) */
        float xa = ds[0] * (-sk[k]);
        float xb = ds[1] * ck[k];
        float x = xa + xb;
        float y = ds[2];
        float rx = x / zk, ry = y / zk;
        float fx = f * rx, fy = f * ry;
        float nx = c + fx;
        float ny = c - fy;
        float fnx = floorf(nx), fny = floorf(ny);
        /* the chosen camera is within half its field of the beam, so a column
         * outside the image is a boundary beam (n_x = 0 or W): clamp it; rows
         * outside the image are beams above or below the camera's field */
        if (!(fnx == fnx) || !(fny >= 0.0f && fny < (float)W)) continue;
        if (fnx < 0.0f) fnx = 0.0f;
        if (fnx > (float)(W - 1)) fnx = (float)(W - 1);
        const int ix = (int)fnx, iy = (int)fny;
        out->outside[s] = 0;
        out->px[s] = ix;
        out->py[s] = iy;
        /* pixel-centre ray */
        float cxp = (float)ix + 0.5f, cyp = (float)iy + 0.5f;
        float an = cxp - c, bn = c - cyp;
        float a = an / f, bb = bn / f;
        float a2 = a * a, b2 = bb * bb;
        float s2 = 1.0f + a2;
        s2 = s2 + b2;
        float inv = 1.0f / sqrtf(s2);
        float as = a * sk[k], ac = a * ck[k];
        float dpx = ck[k] - as, dpy = sk[k] + ac;
        float dps[3] = {dpx * inv, dpy * inv, bb * inv};
        float o32[3], dw[3];
        oracle_world_ray(fr->pose, dps, o32, dw);
        double o[3] = {o32[0], o32[1], o32[2]};
        double d[3] = {dw[0], dw[1], dw[2]};
        const double T_max = ((double)fminf(sen->r_max, sen->d_max) + 9.0 * (double)sen->sigma) /
                             (1.0 - 9.0 * (double)sen->sigma_k);
        double t;
        uint32_t flags;
        int64_t best = oracle_closest(&S, o, d, T_max, &t, &flags);
        out->flags[s] = flags;
        if (best < 0) continue;
        out->tri[s] = (uint32_t)best;
        out->t[s] = t;
        /* depth pass: z-depth, 24-bit */
        const float Tm = (fminf(sen->r_max, sen->d_max) + 9.0f * sen->sigma) / (1.0f - 9.0f * sen->sigma_k);
        double zd = t * (double)inv;
        out->z[s] = zd;
        float z32 = (float)zd;
        float qs = 16777215.0f / Tm;
        float qz = z32 * qs;
        uint32_t q = (uint32_t)rintf(qz);
        if (q > 16777214u) q = 16777214u;
        out->q_depth[s] = q;
        /* incidence angle on the face, 24-bit */
        const double* e1 = S.e1 + 3 * best;
        const double* e2 = S.e2 + 3 * best;
        double n[3], cr[3];
        cross3(e1, e2, n);
        double nl = sqrt(dot3(n, n));
        n[0] /= nl; n[1] /= nl; n[2] /= nl;
        cross3(d, n, cr);
        double theta = atan2(sqrt(dot3(cr, cr)), fabs(dot3(d, n))) * 180.0 / M_PI;
        float th32 = (float)theta;
        float qa_s = 16777215.0f / 90.0f;
        float qa_f = th32 * qa_s;
        uint32_t qa = (uint32_t)rintf(qa_f);
        if (qa > 16777215u) qa = 16777215u;
        out->q_angle[s] = qa;
        const uint32_t m8 = (uint32_t)mat[best] & 0xFFu;
        out->mat[s] = (uint16_t)m8;
        out->inst[s] = inst[best] & 0xFFFFFFu;
        /* resample: the pixel's depth read along the beam */
        double zq = (double)q * ((double)Tm / 16777215.0);
        double th = (double)qa * (90.0 / 16777215.0);
        double d_beam = zq / (double)zk;
        double zn = oracle_normal(seed, (uint64_t)b, (uint32_t)fr->frame, (uint32_t)fr->sensor, 0);
        double dist = d_beam + ((double)sen->sigma + (double)sen->sigma_k * d_beam) * zn;
        int mrow = (int)m8 < n_mat ? (int)m8 : n_mat - 1;
        int ii;
        double ff;
        double R = oracle_lerp_row(table + (int64_t)mrow * ORACLE_NTAB, th, &ii, &ff);
        double r_min = sen->r_min, r_max = sen->r_max, d_max = sen->d_max, RL = sen->RL_max;
        double RLd = RL * dist / d_max;
        int valid = (dist >= r_min) && (dist <= r_max) && (dist <= d_max) && (RLd <= R);
        /* margins: quantisation codes may differ by a few steps between FP32 paths */
        double tol = 1e-5 * fabs(dist) + 4.0 * (double)Tm / 16777215.0;
        if (fabs(dist - r_min) <= tol || fabs(dist - r_max) <= tol || fabs(dist - d_max) <= tol ||
            fabs(RLd - R) <= 1e-5 * fmax(fabs(R), fabs(RLd)) + RL * tol / d_max)
            out->flags[s] |= ORACLE_FLAG_CUTOFF;
        double rf = (sen->range_exp == 0.0f) ? 1.0 : pow((double)sen->r_ref / dist, (double)sen->range_exp);
        out->range[s] = dist;
        out->intensity[s] = (double)sen->gain * R * rf;
        out->theta_deg[s] = th;
        out->valid[s] = (uint8_t)valid;
    }
    oracle_tris_free(&S);
    return 0;
}

/* Camera constants of the raster path (for the tests' pins). */
void oracle_raster_constants(int32_t width, int32_t n_cameras, float* f, float* c, float* ck, float* sk)
{
    oracle_raster_cfg cfg = {width, n_cameras};
    oracle_raster_consts(&cfg, f, c, ck, sk);
}

/* --------------------------------------------------------------- adjoint */

/* Mean squared intensity loss with hits and masks frozen:
 *   L = (1/N) sum_{b in mask} (I_b - I*_b)^2,  I_b = g rf_b lerp(T[m_b], theta_b),
 *   mask = valid_b and target_valid_b, N = |mask| (L = 0 when N = 0). */
double oracle_loss(int64_t n, const uint8_t* valid, const uint16_t* mat, const double* theta_deg,
                   const double* rf, const double* table, int32_t M, double gain, const double* target_I,
                   const uint8_t* target_valid)
{
    double acc = 0.0;
    int64_t N = 0;
    for (int64_t b = 0; b < n; ++b) {
        if (!(valid[b] && target_valid[b])) continue;
        int m = mat[b] < M ? mat[b] : M - 1;
        int i;
        double f;
        double R = oracle_lerp_row(table + (int64_t)m * ORACLE_NTAB, theta_deg[b], &i, &f);
        double r = gain * rf[b] * R - target_I[b];
        acc += r * r;
        ++N;
    }
    return N ? acc / (double)N : 0.0;
}

/* Exact adjoint of oracle_loss: dL/dT [M][91] (overwritten) and dL/dg.
 *   dL/dI_b = 2 (I_b - I*_b) / N
 *   dL/dT[m_b][i_b]   += g rf_b (1 - f_b) dL/dI_b
 *   dL/dT[m_b][i_b+1] += g rf_b f_b dL/dI_b
 *   dL/dg             += rf_b R_b dL/dI_b
 * Returns N. */
int64_t oracle_cast_backward(int64_t n, const uint8_t* valid, const uint16_t* mat, const double* theta_deg,
                             const double* rf, const double* table, int32_t M, double gain,
                             const double* target_I, const uint8_t* target_valid, double* loss,
                             double* grad_table, double* grad_gain)
{
    int64_t N = 0;
    for (int64_t b = 0; b < n; ++b)
        if (valid[b] && target_valid[b]) ++N;
    memset(grad_table, 0, sizeof(double) * (size_t)M * ORACLE_NTAB);
    *grad_gain = 0.0;
    *loss = 0.0;
    if (N == 0) return 0;
    double acc = 0.0;
    for (int64_t b = 0; b < n; ++b) {
        if (!(valid[b] && target_valid[b])) continue;
        int m = mat[b] < M ? mat[b] : M - 1;
        int i;
        double f;
        double R = oracle_lerp_row(table + (int64_t)m * ORACLE_NTAB, theta_deg[b], &i, &f);
        double res = gain * rf[b] * R - target_I[b];
        acc += res * res;
        double gI = 2.0 * res / (double)N;
        grad_table[m * ORACLE_NTAB + i] += gain * rf[b] * (1.0 - f) * gI;
        grad_table[m * ORACLE_NTAB + i + 1] += gain * rf[b] * f * gI;
        *grad_gain += rf[b] * R * gI;
    }
    *loss = acc / (double)N;
    return N;
}

int32_t oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
