/*
 * hdda_oracle.c -- plain, slow, obviously correct CPU definition of the
 * occupancy-grid ray sampler and of the front-to-back compositor.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library, and it must be compiled with
 *     -O2 -ffp-contract=off -fno-fast-math
 * so that every float expression below is one IEEE-754 binary32 operation
 * rounded to nearest (no fused multiply-add, no reassociation, no
 * flush-to-zero).  On aarch64 GCC contracts a*b+c into an FMA unless told not
 * to, which would change the sample set.
 *
 * What it computes (Kato & Tarashima, "Plug-and-Play Acceleration of
 * Occupancy Grid-based NeRF Rendering using VDB Grid and Hierarchical Ray
 * Traversal"):
 *
 *   Sampling (Sec. 3 and Algorithm 1 of the supplementary material).  Every
 *   ray walks one lattice of step parameters t_0 < t_1 < ... that advances by
 *   a step size independent of voxel boundaries (Algorithm 1 adds Delta t to
 *   t_last on every iteration, whatever voxel it is in).  The step is either
 *   constant or grows linearly with t (Sec. 3).  A lattice interval
 *   [t_k, t_{k+1}] is kept when the grid voxel holding its midpoint is
 *   occupied (Algorithm 1 appends a sample only when grid.at(ijk) is true).
 *   With several cascade levels the finest level that contains the point
 *   decides (Sec. 3, last paragraph; the level boxes double in size,
 *   Sec. 4.1).
 *
 *   The recurrence, in binary32 with no contraction:
 *       t_0      = near
 *       dt_k     = min(max(t_k * cone, step), max_step)
 *       t_{k+1}  = t_k + dt_k
 *       candidate k exists iff t_{k+1} <= far
 *       tm_k     = (t_k + t_{k+1}) * 0.5
 *       x_c      = o_c + tm_k * d_c            (c = x, y, z; mul then add)
 *       level    = finest l with lo_l <= x < hi_l on every axis
 *       s_{l,c}  = R / (hi_{l,c} - lo_{l,c})
 *       i_c      = clamp(floor((x_c - lo_{l,c}) * s_{l,c}), 0, R - 1)
 *       keep (r, t_k, t_{k+1}) iff occ[l][i_x][i_y][i_z] != 0
 *
 *   Readings where the paper is silent (each one also listed in the design
 *   notes): the lattice starts at `near` for every ray; intervals are never
 *   clipped; boxes and voxels are half-open [lo, hi); the voxel index is
 *   clamped to R-1 because (x - lo) * s can round up to R just below hi; a
 *   ray with a non-finite origin or direction component has no samples;
 *   min/max follow C fminf/fmaxf; exceeding max_steps candidates is an error.
 *
 *   Compositing (Sec. 1: the sampled points are fed to the radiance field and
 *   their density and colour are accumulated into the pixel).  The radiance
 *   field here is a seeded sum of isotropic Gaussian blobs standing in for
 *   the trained model; the accumulation is done in binary64:
 *       sigma(x) = sum_g a_g exp(-|x - mu_g|^2 / (2 s_g^2))
 *       c(x)     = sum_g a_g exp(...) rgb_g / sigma(x)    (0 when sigma = 0)
 *       alpha    = -expm1(-sigma(x(tm)) * (t1 - t0))
 *       C       += T * alpha * c ;  T *= 1 - alpha       (front to back)
 *       output    (C_r, C_g, C_b, 1 - T), black background, no early stop.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

enum {
    ORACLE_OK = 0,
    ORACLE_ERR_INVALID_ARG = 1,
    ORACLE_ERR_CAPACITY = 3,
    ORACLE_ERR_STEP_LIMIT = 4,
};

/* Parameters are validated the way the sampler's statement needs them:
 * everything finite, a strictly positive step, a non-negative cone. */
static int params_ok(float near_t, float far_t, float step, float cone,
                     float max_step, int64_t max_steps)
{
    if (!isfinite(near_t) || !isfinite(far_t) || !isfinite(step) ||
        !isfinite(cone) || !isfinite(max_step))
        return 0;
    if (!(step > 0.0f) || !(max_step > 0.0f) || !(cone >= 0.0f))
        return 0;
    if (max_steps < 0)
        return 0;
    return 1;
}

static int boxes_ok(const float* aabbs, int levels, int res)
{
    if (levels < 1 || res < 1)
        return 0;
    for (int l = 0; l < levels; ++l) {
        for (int c = 0; c < 3; ++c) {
            float lo = aabbs[l * 6 + c];
            float hi = aabbs[l * 6 + 3 + c];
            if (!isfinite(lo) || !isfinite(hi) || !(lo < hi))
                return 0;
            float s = (float)res / (hi - lo);
            if (!isfinite(s))
                return 0;
        }
    }
    return 1;
}

/*
 * The lattice of one ray (Algorithm 1: t_last starts at t_min and grows by
 * Delta t every iteration; Sec. 3: constant or linearly increasing step).
 * Writes t_0 .. t_K into t_out when there is room and returns K, the number
 * of candidate intervals, through n_candidates.
 */
int oracle_lattice(float near_t, float far_t, float step, float cone,
                   float max_step, int64_t max_steps, float* t_out,
                   int64_t capacity, int64_t* n_candidates)
{
    if (!params_ok(near_t, far_t, step, cone, max_step, max_steps))
        return ORACLE_ERR_INVALID_ARG;
    int64_t k = 0;
    float t = near_t;
    if (capacity > 0)
        t_out[0] = t;
    for (;;) {
        float dt = fminf(fmaxf(t * cone, step), max_step);
        float tn = t + dt;
        if (tn > far_t)
            break;
        if (k == max_steps)
            return ORACLE_ERR_STEP_LIMIT;
        k += 1;
        if (k < capacity)
            t_out[k] = tn;
        t = tn;
    }
    *n_candidates = k;
    return ORACLE_OK;
}

/* Grid lookup of one point: returns 1 when the finest level whose box holds
 * x has its voxel occupied, 0 when it is empty or no level holds x. */
static int occupied_at(const float x[3], const uint8_t* occ, int levels,
                       int res, const float* aabbs)
{
    for (int l = 0; l < levels; ++l) {
        const float* lo = aabbs + l * 6;
        const float* hi = aabbs + l * 6 + 3;
        int inside = 1;
        for (int c = 0; c < 3; ++c)
            if (!(x[c] >= lo[c] && x[c] < hi[c]))
                inside = 0;
        if (!inside)
            continue; /* a coarser level may hold it */
        int64_t idx[3];
        for (int c = 0; c < 3; ++c) {
            float s = (float)res / (hi[c] - lo[c]);
            float u = (x[c] - lo[c]) * s;
            int64_t i = (int64_t)floorf(u);
            if (i < 0)
                i = 0;
            if (i > res - 1)
                i = res - 1;
            idx[c] = i;
        }
        int64_t r = res;
        int64_t lin = (((int64_t)l * r + idx[0]) * r + idx[1]) * r + idx[2];
        return occ[lin] != 0;
    }
    return 0;
}

static int ray_finite(const float* o, const float* d)
{
    for (int c = 0; c < 3; ++c)
        if (!isfinite(o[c]) || !isfinite(d[c]))
            return 0;
    return 1;
}

/*
 * Walks one ray over its whole lattice.  When out_idx is NULL it only counts
 * the kept intervals; otherwise it writes them, in ascending k, starting at
 * out position `base`.
 */
static int walk_ray(int64_t r, const float* o, const float* d,
                    const uint8_t* occ, int levels, int res,
                    const float* aabbs, float near_t, float far_t, float step,
                    float cone, float max_step, int64_t max_steps,
                    int64_t* count, int64_t base, int32_t* out_idx,
                    float* out_t0, float* out_t1)
{
    int64_t kept = 0;
    if (ray_finite(o, d)) {
        int64_t k = 0;
        float t = near_t;
        for (;;) {
            float dt = fminf(fmaxf(t * cone, step), max_step);
            float tn = t + dt;
            if (tn > far_t)
                break;
            if (k == max_steps)
                return ORACLE_ERR_STEP_LIMIT;
            float tm = (t + tn) * 0.5f;
            float x[3];
            for (int c = 0; c < 3; ++c) {
                float p = tm * d[c];
                x[c] = o[c] + p;
            }
            if (occupied_at(x, occ, levels, res, aabbs)) {
                if (out_idx) {
                    out_idx[base + kept] = (int32_t)r;
                    out_t0[base + kept] = t;
                    out_t1[base + kept] = tn;
                }
                kept += 1;
            }
            t = tn;
            k += 1;
        }
    }
    *count = kept;
    return ORACLE_OK;
}

/*
 * Samples every ray.  offsets[0..n_rays] receives the exclusive prefix sum
 * of the per-ray counts (CSR row pointers); *total_out the number of kept
 * intervals.  When capacity >= total the intervals are written as
 * structure-of-arrays (ray index, t_start, t_end), rays in order and each
 * ray's intervals in ascending k.  capacity == 0 only counts; a non-zero
 * capacity below the total returns ORACLE_ERR_CAPACITY and writes nothing.
 */
int oracle_sample(const float* rays_o, const float* rays_d, int64_t n_rays,
                  const uint8_t* occ, int levels, int res, const float* aabbs,
                  float near_t, float far_t, float step, float cone,
                  float max_step, int64_t max_steps, int64_t* offsets,
                  int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                  int64_t* total_out)
{
    if (n_rays < 0 || n_rays > INT32_MAX)
        return ORACLE_ERR_INVALID_ARG;
    if (!params_ok(near_t, far_t, step, cone, max_step, max_steps))
        return ORACLE_ERR_INVALID_ARG;
    if (!boxes_ok(aabbs, levels, res))
        return ORACLE_ERR_INVALID_ARG;
    int64_t total = 0;
    offsets[0] = 0;
    for (int64_t r = 0; r < n_rays; ++r) {
        int64_t cnt = 0;
        int st = walk_ray(r, rays_o + 3 * r, rays_d + 3 * r, occ, levels, res,
                          aabbs, near_t, far_t, step, cone, max_step,
                          max_steps, &cnt, 0, NULL, NULL, NULL);
        if (st != ORACLE_OK)
            return st;
        total += cnt;
        offsets[r + 1] = total;
    }
    *total_out = total;
    if (capacity == 0)
        return ORACLE_OK;
    if (capacity < total)
        return ORACLE_ERR_CAPACITY;
    for (int64_t r = 0; r < n_rays; ++r) {
        int64_t cnt = 0;
        int st = walk_ray(r, rays_o + 3 * r, rays_d + 3 * r, occ, levels, res,
                          aabbs, near_t, far_t, step, cone, max_step,
                          max_steps, &cnt, offsets[r], ray_idx, t0, t1);
        if (st != ORACLE_OK)
            return st;
    }
    return ORACLE_OK;
}

/*
 * Front-to-back compositing in binary64 over the kept intervals (Sec. 1:
 * densities and colours of the sampled points are accumulated into the
 * pixel).  field is n_g records of 8 floats: mu_x, mu_y, mu_z, s, a, r, g, b.
 * rgba_out receives n_rays records of 4 doubles.
 */
int oracle_composite(const float* rays_o, const float* rays_d, int64_t n_rays,
                     const int64_t* offsets, const float* t0, const float* t1,
                     const float* field, int n_g, double* rgba_out)
{
    if (n_rays < 0 || n_g < 0)
        return ORACLE_ERR_INVALID_ARG;
    for (int64_t r = 0; r < n_rays; ++r) {
        double C[3] = {0.0, 0.0, 0.0};
        double T = 1.0;
        for (int64_t s = offsets[r]; s < offsets[r + 1]; ++s) {
            double a0 = (double)t0[s];
            double a1 = (double)t1[s];
            double tm = 0.5 * (a0 + a1);
            double x[3];
            for (int c = 0; c < 3; ++c)
                x[c] = (double)rays_o[3 * r + c] + tm * (double)rays_d[3 * r + c];
            double sigma = 0.0;
            double wc[3] = {0.0, 0.0, 0.0};
            for (int g = 0; g < n_g; ++g) {
                const float* G = field + 8 * g;
                double d2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double e = x[c] - (double)G[c];
                    d2 += e * e;
                }
                double sg = (double)G[3];
                double w = (double)G[4] * exp(-d2 / (2.0 * sg * sg));
                sigma += w;
                for (int c = 0; c < 3; ++c)
                    wc[c] += w * (double)G[5 + c];
            }
            double alpha = -expm1(-sigma * (a1 - a0));
            if (sigma > 0.0) {
                for (int c = 0; c < 3; ++c)
                    C[c] += T * alpha * (wc[c] / sigma);
            }
            T *= 1.0 - alpha;
        }
        rgba_out[4 * r + 0] = C[0];
        rgba_out[4 * r + 1] = C[1];
        rgba_out[4 * r + 2] = C[2];
        rgba_out[4 * r + 3] = 1.0 - T;
    }
    return ORACLE_OK;
}
