/*
 * af_oracle.c -- plain, single-threaded CPU statement of the Accessibility
 * Field hot path: scan-centric TSDF integration with positive clamping
 * (Sec. 3.2), the ray-cleared free band (Sec. 3.4), the weight cap
 * (Sec. 3.6), the occupied / known view of the TSDF, and accessibility
 * scoring of surface points against tool and corridor voxel kernels
 * (Sec. 3.4, 3.5).
 *
 * TEST INFRASTRUCTURE. This file is the correctness reference that the CUDA
 * path is compared against. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product never does.
 *
 * It is written for a reader checking it against the paper, not for speed:
 * one voxel at a time, one return at a time, one direction at a time, every
 * direction scored in full (no early exits), a hash map of single voxels.
 *
 * Floating point. Every decision that yields an integer (the behind-surface
 * cone, the quantised contribution, the voxel a point falls in) is taken in
 * IEEE single precision, one correctly rounded operation at a time, in the
 * order written here; build with -ffp-contract=off and without -ffast-math.
 * The kernel tables are rasterised in double precision.
 *
 * Readings of the paper that this file implements (the paper leaves them
 * open):
 *  - The cone test of Sec. 3.2 EXCLUDES voxels with cos(theta) > cone_cos,
 *    theta the angle between x - p and p - q: the narrow cone behind the
 *    return along its ray. A voxel whose centre coincides with p is kept.
 *  - The "+-tau cube" of Sec. 3.2 is the index-space cube of half-width
 *    m = ceil(tau/v) around the voxel holding p (the (2m+1)^3 cube of
 *    Sec. 3.6).
 *  - Contributions are accumulated exactly: S += round(d * 2^20) in integers
 *    and w += 1, so the result does not depend on the order of the returns.
 *  - The weight cap of Sec. 3.6 is applied once at the end of each scan:
 *    w > w_cap => S = floor(S * w_cap / w), w = w_cap (floor also for a
 *    negative S of the signed ablation).
 *  - With clamp_signed (the [-tau, tau] ablation of Tab. 4) only the clamp
 *    changes: the cube, the cone and the accumulation are the same.
 *  - The cleared band (clear_lo*tau, clear_hi*tau] is sampled at N_s points
 *    dist_j = clear_lo*tau + j*((clear_hi - clear_lo)*tau / N_s), j = 1..N_s,
 *    along the unit vector from p toward q; the voxel holding each sample is
 *    marked cleared.
 *  - occ = (w >= 1) and (S < round(r_c * 2^20) * w), i.e. TSDF < r_c;
 *    known = (w >= 1) or cleared.
 *  - Approach directions are a table of unit vectors shared by both sides;
 *    a direction is a candidate for a point when n . u > cos_theta_max.
 *  - Tool kernel of direction u: voxel offsets o with e = o*v, a = e.u,
 *    0 <= a <= L, |e - a u|^2 <= r^2 and |e|^2 > r_s^2. Corridor kernel:
 *    L < a <= L + L_c and |e - a u|^2 <= r_corr^2.
 *  - Arm samples: offsets floor(0.5 + (f*tau) * u_k / v), f in
 *    {0.6, 1.25, 2.25}; blocked when occupied or unknown (Sec. 3.4).
 *  - Corridor voxels block when occupied (unknown reads free, as for the
 *    tool kernel); with `strict`, unknown corridor voxels block as well.
 *  - Direction score: blocked (arm or corridor) => n_c + 1, else
 *    min(count, n_c); best = lowest index of the minimum; ACCESSIBLE iff the
 *    best score is below n_c; no candidate => BLOCKED with best = -1.
 *  - Points whose voxel has w < w_min are UNSCORED with best = -1.
 *  - The map is confined to a fixed box of voxels (the paper's bounded
 *    window, Sec. 3.3): a return whose cube leaves the box is dropped, and
 *    cleared-band samples outside the box are skipped. Voxels outside the
 *    box read w = 0, not cleared.
 *
 * The differentiable form (soft clearance, not in the paper: a smooth
 * companion of the Sec. 3.4 tool / corridor test) takes these readings:
 *  - SDF of a voxel = S / (w 2^20) divided in double and rounded to single
 *    precision; tau where w = 0 or outside the box (an unobserved voxel reads
 *    as far from any surface).
 *  - SDF(x) = trilinear interpolation over voxel centres: with
 *    g = x / v - 1/2, the cell is floor(g) and the weights g - floor(g).
 *  - Samples along the approach axis at a_j = h + j v, j = 1..J,
 *    J = floor((L + L_c) / v); a sample with j v <= r_s is skipped (the
 *    self-exclusion of Sec. 3.4 in the tool's own frame); its margin is r
 *    when j v <= L (tool) and r_corr beyond (corridor).
 *  - phi_j = SDF(x_j) - margin_j; C = -tau_s log sum_j exp(-phi_j / tau_s).
 *  - Direction u = q / |q|, q = u0 + alpha t1 + beta t2, (t1, t2) the
 *    orthonormal tangent basis of u0 of Duff et al. 2017.
 *  - The cell of every sample is an integer decided by floating point, so
 *    with fp32_cells it is decided as the kernel decides it: in single
 *    precision in the fixed order of pair_frame_f / sample_cell_f below,
 *    relative to the voxel of the point. The weights, SDF, softmin and
 *    gradient are double. Without fp32_cells the cell is floor(g) in double.
 */
#include "af_oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_SCALE 1048576.0f /* 2^20: fixed-point scale of the SDF sum */

/* ------------------------------------------------------------------------- */
/* Voxel store: open addressing over packed voxel indices.                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint64_t key; /* 0 = empty slot */
    int64_t S;    /* sum of quantised contributions, units of 2^-20 m */
    uint32_t w;   /* number of contributions */
    int32_t cleared;
} or_voxel;

struct or_map {
    or_config cfg;
    or_voxel *slot;
    uint64_t cap; /* power of two */
    uint64_t count;
};

/* floor(a / b) for b > 0 (C division truncates toward zero). */
static int64_t floor_div(int64_t a, int64_t b) {
    const int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

static uint64_t pack_key(int32_t ix, int32_t iy, int32_t iz);

/* Weight cap with proportional rescale of the sum (Sec. 3.6), once per scan. */
static void apply_cap(or_map *m);

static uint64_t pack_key(int32_t ix, int32_t iy, int32_t iz) {
    /* 21 bits per axis, offset so that the packed key is never 0. */
    uint64_t x = (uint64_t)(uint32_t)(ix + (1 << 20)) & 0x1FFFFFu;
    uint64_t y = (uint64_t)(uint32_t)(iy + (1 << 20)) & 0x1FFFFFu;
    uint64_t z = (uint64_t)(uint32_t)(iz + (1 << 20)) & 0x1FFFFFu;
    return (x | (y << 21) | (z << 42)) + 1u;
}

static void unpack_key(uint64_t key, int32_t *ix, int32_t *iy, int32_t *iz) {
    uint64_t k = key - 1u;
    *ix = (int32_t)(k & 0x1FFFFFu) - (1 << 20);
    *iy = (int32_t)((k >> 21) & 0x1FFFFFu) - (1 << 20);
    *iz = (int32_t)((k >> 42) & 0x1FFFFFu) - (1 << 20);
}

static uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    return k;
}

static or_voxel *find_slot(const or_map *m, uint64_t key) {
    uint64_t h = mix64(key) & (m->cap - 1);
    for (;;) {
        or_voxel *s = &m->slot[h];
        if (s->key == key || s->key == 0) return s;
        h = (h + 1) & (m->cap - 1);
    }
}

static void grow(or_map *m) {
    or_voxel *old = m->slot;
    uint64_t oldcap = m->cap;
    m->cap *= 2;
    m->slot = (or_voxel *)calloc(m->cap, sizeof(or_voxel));
    for (uint64_t k = 0; k < oldcap; ++k)
        if (old[k].key) *find_slot(m, old[k].key) = old[k];
    free(old);
}

static or_voxel *voxel_ref(or_map *m, int32_t ix, int32_t iy, int32_t iz) {
    if (2 * (m->count + 1) > m->cap) grow(m);
    uint64_t key = pack_key(ix, iy, iz);
    or_voxel *s = find_slot(m, key);
    if (s->key == 0) {
        s->key = key;
        s->S = 0;
        s->w = 0;
        s->cleared = 0;
        m->count++;
    }
    return s;
}

static const or_voxel *voxel_get(const or_map *m, int32_t ix, int32_t iy, int32_t iz) {
    const or_voxel *s = find_slot(m, pack_key(ix, iy, iz));
    return s->key ? s : NULL;
}

static int in_domain(const or_config *c, int32_t ix, int32_t iy, int32_t iz) {
    return ix >= c->dom_min[0] && ix < c->dom_min[0] + c->dom_size[0] &&
           iy >= c->dom_min[1] && iy < c->dom_min[1] + c->dom_size[1] &&
           iz >= c->dom_min[2] && iz < c->dom_min[2] + c->dom_size[2];
}

or_map *or_map_new(const or_config *cfg) {
    or_map *m = (or_map *)calloc(1, sizeof(or_map));
    m->cfg = *cfg;
    m->cap = 1024;
    m->slot = (or_voxel *)calloc(m->cap, sizeof(or_voxel));
    return m;
}

void or_map_free(or_map *m) {
    if (!m) return;
    free(m->slot);
    free(m);
}

static void apply_cap(or_map *m) {
    const or_config *c = &m->cfg;
    for (uint64_t k = 0; k < m->cap; ++k) {
        or_voxel *vx = &m->slot[k];
        if (vx->key && vx->w > c->w_cap) {
            vx->S = floor_div(vx->S * (int64_t)c->w_cap, (int64_t)vx->w);
            vx->w = c->w_cap;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Scan-centric integration (Sec. 3.2, 3.4, 3.6).                            */
/* ------------------------------------------------------------------------- */

/* Voxel index of a coordinate: floor(c / v) in single precision. Returns 0
 * when the index is not representable. */
static int voxel_index(float c, float v, int32_t *out) {
    float f = floorf(c / v);
    if (!(f >= -1.0e9f && f <= 1.0e9f)) return 0;
    *out = (int32_t)f;
    return 1;
}

static float voxel_centre(int32_t i, float v) { return ((float)i + 0.5f) * v; }

int64_t or_integrate(or_map *m, const float *pts, int64_t n, const float pose[16]) {
    return or_integrate_bands(m, pts, n, pose, NULL, NULL);
}

int64_t or_integrate2(or_map *m, const float *pts, int64_t n, const float pose[16],
                      int32_t *voxel_out) {
    return or_integrate_bands(m, pts, n, pose, voxel_out, NULL);
}

int64_t or_integrate_bands(or_map *m, const float *pts, int64_t n, const float pose[16],
                           int32_t *voxel_out, int32_t *band_out) {
    const or_config *c = &m->cfg;
    const float v = c->v, tau = c->tau, lo = c->clamp_signed ? -c->tau : 0.0f;
    const int32_t mr = c->cube_radius;
    /* sensor origin q = translation of the world_from_sensor pose */
    const float q[3] = {pose[3], pose[7], pose[11]};
    int64_t accepted = 0;

    if (voxel_out)
        for (int64_t k = 0; k < 3 * n; ++k) voxel_out[k] = INT32_MIN;
    if (band_out)
        for (int64_t k = 0; k < 3 * n * c->clear_samples; ++k) band_out[k] = INT32_MIN;
    for (int64_t k = 0; k < n; ++k) {
        const float *ps = pts + 3 * k;
        if (!isfinite(ps[0]) || !isfinite(ps[1]) || !isfinite(ps[2])) continue;

        /* p_i = R ps + t, one rounding per operation */
        float p[3];
        for (int r = 0; r < 3; ++r)
            p[r] = ((pose[4 * r + 0] * ps[0] + pose[4 * r + 1] * ps[1]) + pose[4 * r + 2] * ps[2]) +
                   pose[4 * r + 3];

        /* b = p_i - q, the ray from the sensor to the return */
        const float b[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
        const float bb = (b[0] * b[0] + b[1] * b[1]) + b[2] * b[2];
        const float range = sqrtf(bb); /* ||p_i - q|| */
        if (!(range >= c->range_min && range <= c->range_max)) continue;

        int32_t ip[3];
        if (!voxel_index(p[0], v, &ip[0]) || !voxel_index(p[1], v, &ip[1]) ||
            !voxel_index(p[2], v, &ip[2]))
            continue;
        if (!in_domain(c, ip[0] - mr, ip[1] - mr, ip[2] - mr) ||
            !in_domain(c, ip[0] + mr, ip[1] + mr, ip[2] + mr))
            continue;
        accepted++;
        if (voxel_out)
            for (int r = 0; r < 3; ++r) voxel_out[3 * k + r] = ip[r];

        /* every voxel x of the (2m+1)^3 cube around p_i */
        for (int32_t oz = -mr; oz <= mr; ++oz)
            for (int32_t oy = -mr; oy <= mr; ++oy)
                for (int32_t ox = -mr; ox <= mr; ++ox) {
                    const int32_t j[3] = {ip[0] + ox, ip[1] + oy, ip[2] + oz};
                    const float x[3] = {voxel_centre(j[0], v), voxel_centre(j[1], v),
                                        voxel_centre(j[2], v)};
                    /* theta: angle between x - p_i and p_i - q */
                    const float a[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
                    const float aa = (a[0] * a[0] + a[1] * a[1]) + a[2] * a[2];
                    if (aa > 0.0f) {
                        const float cos_theta =
                            ((a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]) / (sqrtf(aa) * range);
                        if (cos_theta > c->cone_cos) continue; /* behind the surface */
                    }
                    /* d = ||p_i - q|| - ||x - q||, clamped to [0, tau]
                       ([-tau, tau] in the signed ablation) */
                    const float e[3] = {x[0] - q[0], x[1] - q[1], x[2] - q[2]};
                    const float ee = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
                    float d = range - sqrtf(ee);
                    if (d < lo) d = lo;
                    if (d > tau) d = tau;
                    const int64_t dq = (int64_t)rintf(d * OR_SCALE);
                    or_voxel *vx = voxel_ref(m, j[0], j[1], j[2]);
                    vx->S += dq;
                    vx->w += 1;
                }

        /* ray-cleared band toward the sensor: (clear_lo*tau, clear_hi*tau] */
        const float u[3] = {(q[0] - p[0]) / range, (q[1] - p[1]) / range, (q[2] - p[2]) / range};
        const float step = ((c->clear_hi - c->clear_lo) * tau) / (float)c->clear_samples;
        const float start = c->clear_lo * tau;
        for (int32_t s = 1; s <= c->clear_samples; ++s) {
            const float dist = start + (float)s * step;
            int32_t js[3];
            if (!voxel_index(p[0] + dist * u[0], v, &js[0]) ||
                !voxel_index(p[1] + dist * u[1], v, &js[1]) ||
                !voxel_index(p[2] + dist * u[2], v, &js[2]))
                continue;
            if (!in_domain(c, js[0], js[1], js[2])) continue;
            voxel_ref(m, js[0], js[1], js[2])->cleared = 1;
            if (band_out)
                for (int r = 0; r < 3; ++r)
                    band_out[3 * (k * c->clear_samples + (s - 1)) + r] = js[r];
        }
    }

    apply_cap(m);
    return accepted;
}

/* ------------------------------------------------------------------------- */
/* Projective integration: the ablation of Tab. 3 (Sec. 3.2).                */
/* ------------------------------------------------------------------------- */

/* Bin of a sensor-frame direction in an N x N octahedral map of the sphere:
 * (u, w) = (d_x, d_y) / (|d_x| + |d_y| + |d_z|), the lower hemisphere folded
 * onto the corners, then N equal cells per axis over [-1, 1]. */
static int32_t octa_bin(const float d[3], int32_t N) {
    const float s = (fabsf(d[0]) + fabsf(d[1])) + fabsf(d[2]);
    float u = d[0] / s, w = d[1] / s;
    if (d[2] < 0.0f) {
        const float uu = (1.0f - fabsf(w)) * (u >= 0.0f ? 1.0f : -1.0f);
        const float ww = (1.0f - fabsf(u)) * (w >= 0.0f ? 1.0f : -1.0f);
        u = uu;
        w = ww;
    }
    const float h = (float)N * 0.5f;
    int32_t bu = (int32_t)floorf((u + 1.0f) * h), bw = (int32_t)floorf((w + 1.0f) * h);
    bu = bu < 0 ? 0 : (bu >= N ? N - 1 : bu);
    bw = bw < 0 ? 0 : (bw >= N ? N - 1 : bw);
    return bw * N + bu;
}

int32_t or_octa_bin(const float d[3], int32_t bins) { return octa_bin(d, bins); }

static int brick_cmp(const void *x, const void *y) {
    const uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : (a > b);
}

int64_t or_integrate_projective(or_map *m, const float *pts, int64_t n, const float pose[16],
                                int32_t bins) {
    const or_config *c = &m->cfg;
    const float v = c->v, tau = c->tau, lo = c->clamp_signed ? -c->tau : 0.0f;
    const int32_t mr = c->cube_radius;
    const float q[3] = {pose[3], pose[7], pose[11]};
    const int64_t N2 = (int64_t)bins * bins;
    float *img = (float *)malloc(sizeof(float) * (size_t)N2);
    uint8_t *hit = (uint8_t *)calloc((size_t)N2, 1);
    const int32_t nb = (2 * mr + 7) / 8 + 1; /* bricks a cube spans per axis, at most */
    uint64_t *bricks = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n * nb * nb * nb + 1));
    int64_t nbr = 0, accepted = 0;

    /* the returns accepted by the scan-centric rules: range image and bricks */
    for (int64_t k = 0; k < n; ++k) {
        const float *ps = pts + 3 * k;
        if (!isfinite(ps[0]) || !isfinite(ps[1]) || !isfinite(ps[2])) continue;
        float p[3];
        for (int r = 0; r < 3; ++r)
            p[r] = ((pose[4 * r + 0] * ps[0] + pose[4 * r + 1] * ps[1]) + pose[4 * r + 2] * ps[2]) +
                   pose[4 * r + 3];
        const float b[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
        const float range = sqrtf((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]);
        if (!(range >= c->range_min && range <= c->range_max)) continue;
        int32_t ip[3];
        if (!voxel_index(p[0], v, &ip[0]) || !voxel_index(p[1], v, &ip[1]) ||
            !voxel_index(p[2], v, &ip[2]))
            continue;
        if (!in_domain(c, ip[0] - mr, ip[1] - mr, ip[2] - mr) ||
            !in_domain(c, ip[0] + mr, ip[1] + mr, ip[2] + mr))
            continue;
        accepted++;
        /* the return's range in the bin of its sensor-frame direction (the nearest wins) */
        if (ps[0] != 0.0f || ps[1] != 0.0f || ps[2] != 0.0f) {
            const int32_t bin = octa_bin(ps, bins);
            if (!hit[bin] || range < img[bin]) img[bin] = range;
            hit[bin] = 1;
        }
        for (int32_t bz = floor_div(ip[2] - mr, 8); bz <= floor_div(ip[2] + mr, 8); ++bz)
            for (int32_t by = floor_div(ip[1] - mr, 8); by <= floor_div(ip[1] + mr, 8); ++by)
                for (int32_t bx = floor_div(ip[0] - mr, 8); bx <= floor_div(ip[0] + mr, 8); ++bx)
                    bricks[nbr++] = pack_key(bx, by, bz);
    }
    qsort(bricks, (size_t)nbr, sizeof(uint64_t), brick_cmp);

    /* every voxel of those bricks looks its range up through its own bin */
    for (int64_t k = 0; k < nbr; ++k) {
        if (k > 0 && bricks[k] == bricks[k - 1]) continue;
        int32_t bx, by, bz;
        unpack_key(bricks[k], &bx, &by, &bz);
        for (int32_t l = 0; l < 512; ++l) {
            const int32_t j[3] = {8 * bx + (l & 7), 8 * by + ((l >> 3) & 7), 8 * bz + (l >> 6)};
            if (!in_domain(c, j[0], j[1], j[2])) continue;
            const float e[3] = {voxel_centre(j[0], v) - q[0], voxel_centre(j[1], v) - q[1],
                                voxel_centre(j[2], v) - q[2]};
            /* sensor-frame direction R^T e */
            float xs[3];
            for (int r = 0; r < 3; ++r)
                xs[r] = (pose[r] * e[0] + pose[4 + r] * e[1]) + pose[8 + r] * e[2];
            if (xs[0] == 0.0f && xs[1] == 0.0f && xs[2] == 0.0f) continue;
            const int32_t bin = octa_bin(xs, bins);
            if (!hit[bin]) continue; /* an empty bin: no observation */
            const float dist = sqrtf((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
            float d = img[bin] - dist;
            if (d < -tau) continue; /* beyond the truncation behind the surface */
            if (d < lo) d = lo;
            if (d > tau) d = tau;
            or_voxel *vx = voxel_ref(m, j[0], j[1], j[2]);
            vx->S += (int64_t)rintf(d * OR_SCALE);
            vx->w += 1;
        }
    }
    apply_cap(m);
    free(img);
    free(hit);
    free(bricks);
    return accepted;
}

int or_get_voxel(const or_map *m, int32_t ix, int32_t iy, int32_t iz, int64_t *S,
                 uint32_t *w, int32_t *cleared) {
    const or_voxel *vx = voxel_get(m, ix, iy, iz);
    *S = vx ? vx->S : 0;
    *w = vx ? vx->w : 0;
    *cleared = vx ? vx->cleared : 0;
    return vx != NULL;
}

void or_set_voxel(or_map *m, int32_t ix, int32_t iy, int32_t iz, int64_t S, uint32_t w,
                  int32_t cleared) {
    or_voxel *vx = voxel_ref(m, ix, iy, iz);
    vx->S = S;
    vx->w = w;
    vx->cleared = cleared;
}

void or_set_voxels(or_map *m, int64_t n, const int32_t *ijk, const int64_t *S,
                   const uint32_t *w, const uint8_t *cleared) {
    for (int64_t k = 0; k < n; ++k)
        or_set_voxel(m, ijk[3 * k], ijk[3 * k + 1], ijk[3 * k + 2], S[k], w[k], cleared[k]);
}

int64_t or_voxel_count(const or_map *m) { return (int64_t)m->count; }

const or_config *or_map_config(const or_map *m) { return &m->cfg; }

/* TSDF < r_c, with r_c on the same 2^-20 m grid as S. */
static int occ_of(const or_map *m, const or_voxel *vx) {
    if (!vx || vx->w == 0) return 0;
    const int64_t rcq = (int64_t)rintf(m->cfg.r_c * OR_SCALE);
    return vx->S < rcq * (int64_t)vx->w;
}

static int known_of(const or_voxel *vx) { return vx && (vx->w >= 1 || vx->cleared); }

int or_occ(const or_map *m, int32_t ix, int32_t iy, int32_t iz) {
    if (!in_domain(&m->cfg, ix, iy, iz)) return 0;
    return occ_of(m, voxel_get(m, ix, iy, iz));
}

int or_known(const or_map *m, int32_t ix, int32_t iy, int32_t iz) {
    if (!in_domain(&m->cfg, ix, iy, iz)) return 0;
    return known_of(voxel_get(m, ix, iy, iz));
}

void or_export(const or_map *m, int32_t *ijk, int64_t *S, uint32_t *w, uint8_t *cleared,
               uint8_t *occ, uint8_t *known) {
    uint64_t o = 0;
    for (uint64_t k = 0; k < m->cap; ++k) {
        const or_voxel *vx = &m->slot[k];
        if (!vx->key) continue;
        unpack_key(vx->key, &ijk[3 * o], &ijk[3 * o + 1], &ijk[3 * o + 2]);
        S[o] = vx->S;
        w[o] = vx->w;
        cleared[o] = (uint8_t)vx->cleared;
        occ[o] = (uint8_t)occ_of(m, vx);
        known[o] = (uint8_t)known_of(vx);
        ++o;
    }
}

/* ------------------------------------------------------------------------- */
/* Tool and corridor kernels (Sec. 3.4), rasterised in double precision.     */
/* ------------------------------------------------------------------------- */

static int in_kernel(const or_tool *t, double v, const double u[3], int32_t ox, int32_t oy,
                     int32_t oz, int which) {
    const double e[3] = {(double)ox * v, (double)oy * v, (double)oz * v};
    const double a = (e[0] * u[0] + e[1] * u[1]) + e[2] * u[2]; /* distance along u */
    const double r[3] = {e[0] - a * u[0], e[1] - a * u[1], e[2] - a * u[2]};
    const double rho2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]; /* squared axis distance */
    const double L = (double)t->length;
    if (which == OR_KERNEL_TOOL) {
        const double ee = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
        const double rad = (double)t->radius, rs = (double)t->self_excl;
        return a >= 0.0 && a <= L && rho2 <= rad * rad && ee > rs * rs;
    } else {
        const double rad = (double)t->corr_radius;
        return a > L && a <= L + (double)t->corr_length && rho2 <= rad * rad;
    }
}

int64_t or_kernel_offsets(const or_tool *t, float v, const float u[3], int which, int32_t *out,
                          int64_t cap) {
    const double dv = (double)v;
    const double du[3] = {(double)u[0], (double)u[1], (double)u[2]};
    /* Every kernel point lies within reach of the tip; enumerate the cube
     * that contains that ball, with one voxel of margin. */
    const double reach = (double)t->length + (double)t->corr_length +
                         ((double)t->radius > (double)t->corr_radius ? (double)t->radius
                                                                     : (double)t->corr_radius);
    const int32_t B = (int32_t)ceil(reach / dv) + 1;
    int64_t count = 0;
    for (int32_t oz = -B; oz <= B; ++oz)
        for (int32_t oy = -B; oy <= B; ++oy)
            for (int32_t ox = -B; ox <= B; ++ox)
                if (in_kernel(t, dv, du, ox, oy, oz, which)) {
                    if (count < cap) {
                        out[3 * count + 0] = ox;
                        out[3 * count + 1] = oy;
                        out[3 * count + 2] = oz;
                    }
                    ++count;
                }
    return count;
}

void or_arm_offsets(float v, float tau, const float u[3], int32_t out[9]) {
    static const double frac[3] = {0.6, 1.25, 2.25};
    for (int s = 0; s < 3; ++s)
        for (int k = 0; k < 3; ++k)
            out[3 * s + k] =
                (int32_t)floor(0.5 + ((frac[s] * (double)tau) * (double)u[k]) / (double)v);
}

/* ------------------------------------------------------------------------- */
/* Accessibility scoring (Sec. 3.4, 3.5).                                    */
/* ------------------------------------------------------------------------- */

struct or_tables {
    or_tool t;
    float v, tau;
    int32_t G;
    float *dirs;
    int32_t **tool, **corr;
    int64_t *ntool, *ncorr;
    int32_t *arm;
};

/* Precomputed kernels, one per direction, no run-time rotation (Sec. 3.6). */
or_tables *or_tables_new(const or_tool *t, float v, float tau, const float *dirs, int32_t G) {
    or_tables *T = (or_tables *)calloc(1, sizeof(or_tables));
    T->t = *t;
    T->v = v;
    T->tau = tau;
    T->G = G;
    T->dirs = (float *)malloc(sizeof(float) * 3 * (size_t)(G > 0 ? G : 1));
    memcpy(T->dirs, dirs, sizeof(float) * 3 * (size_t)G);
    T->tool = (int32_t **)calloc((size_t)G, sizeof(int32_t *));
    T->corr = (int32_t **)calloc((size_t)G, sizeof(int32_t *));
    T->ntool = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    T->ncorr = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    T->arm = (int32_t *)calloc((size_t)G * 9, sizeof(int32_t));
    for (int32_t g = 0; g < G; ++g) {
        const float *u = dirs + 3 * g;
        T->ntool[g] = or_kernel_offsets(t, v, u, OR_KERNEL_TOOL, NULL, 0);
        T->tool[g] = (int32_t *)malloc((size_t)(3 * T->ntool[g] + 1) * sizeof(int32_t));
        or_kernel_offsets(t, v, u, OR_KERNEL_TOOL, T->tool[g], T->ntool[g]);
        T->ncorr[g] = or_kernel_offsets(t, v, u, OR_KERNEL_CORRIDOR, NULL, 0);
        T->corr[g] = (int32_t *)malloc((size_t)(3 * T->ncorr[g] + 1) * sizeof(int32_t));
        or_kernel_offsets(t, v, u, OR_KERNEL_CORRIDOR, T->corr[g], T->ncorr[g]);
        or_arm_offsets(v, tau, u, T->arm + 9 * g);
    }
    return T;
}

void or_tables_free(or_tables *T) {
    if (!T) return;
    for (int32_t g = 0; g < T->G; ++g) {
        free(T->tool[g]);
        free(T->corr[g]);
    }
    free(T->tool);
    free(T->corr);
    free(T->ntool);
    free(T->ncorr);
    free(T->arm);
    free(T->dirs);
    free(T);
}

void or_score(const or_map *m, const or_tool *t, const float *dirs, int32_t G, const float *pts,
              const float *normals, int64_t npts, uint8_t *label, int16_t *best,
              int32_t *dir_score) {
    or_tables *T = or_tables_new(t, m->cfg.v, m->cfg.tau, dirs, G);
    or_score_tables(m, T, pts, normals, npts, label, best, dir_score);
    or_tables_free(T);
}

void or_score_tables(const or_map *m, const or_tables *T, const float *pts, const float *normals,
                     int64_t npts, uint8_t *label, int16_t *best, int32_t *dir_score) {
    const or_config *c = &m->cfg;
    const float v = c->v;
    const or_tool *t = &T->t;
    const int32_t n_c = (int32_t)t->n_c, G = T->G;
    const float *dirs = T->dirs;
    int32_t *const *tool = T->tool, *const *corr = T->corr;
    const int64_t *ntool = T->ntool, *ncorr = T->ncorr;
    const int32_t *arm = T->arm;

    for (int64_t k = 0; k < npts; ++k) {
        const float *s = pts + 3 * k, *nrm = normals + 3 * k;
        int32_t *ds = dir_score ? dir_score + (int64_t)G * k : NULL;
        if (ds)
            for (int32_t g = 0; g < G; ++g) ds[g] = -1;
        label[k] = OR_UNSCORED;
        best[k] = -1;

        /* the point's voxel and its confidence (Sec. 3.5) */
        int32_t i[3];
        if (!voxel_index(s[0], v, &i[0]) || !voxel_index(s[1], v, &i[1]) ||
            !voxel_index(s[2], v, &i[2]))
            continue;
        uint32_t w = 0;
        if (in_domain(c, i[0], i[1], i[2])) {
            const or_voxel *vx = voxel_get(m, i[0], i[1], i[2]);
            w = vx ? vx->w : 0;
        }
        if (w < c->w_min) continue;

        int32_t best_score = -1, best_g = -1;
        for (int32_t g = 0; g < G; ++g) {
            const float *u = dirs + 3 * g;
            /* normal filter: candidate iff n . u > cos(theta_max) */
            const float nu = (nrm[0] * u[0] + nrm[1] * u[1]) + nrm[2] * u[2];
            if (!(nu > t->cos_theta_max)) continue;

            /* arm path: any sample occupied or unknown blocks */
            int blocked = 0;
            for (int sIdx = 0; sIdx < 3; ++sIdx) {
                const int32_t *o = arm + 9 * g + 3 * sIdx;
                const int32_t x = i[0] + o[0], y = i[1] + o[1], z = i[2] + o[2];
                if (or_occ(m, x, y, z) || !or_known(m, x, y, z)) blocked = 1;
            }
            /* approach corridor: any occupied (strict: or unknown) voxel blocks */
            for (int64_t q = 0; q < ncorr[g]; ++q) {
                const int32_t *o = corr[g] + 3 * q;
                const int32_t x = i[0] + o[0], y = i[1] + o[1], z = i[2] + o[2];
                if (or_occ(m, x, y, z) || (t->strict && !or_known(m, x, y, z))) blocked = 1;
            }
            /* tool kernel: collision count (Sec. 3.4) */
            int64_t count = 0;
            for (int64_t q = 0; q < ntool[g]; ++q) {
                const int32_t *o = tool[g] + 3 * q;
                count += or_occ(m, i[0] + o[0], i[1] + o[1], i[2] + o[2]);
            }
            const int32_t score = blocked ? n_c + 1 : (count < n_c ? (int32_t)count : n_c);
            if (ds) ds[g] = score;
            if (best_g < 0 || score < best_score) {
                best_score = score;
                best_g = g;
            }
        }
        best[k] = (int16_t)best_g;
        label[k] = (best_g >= 0 && best_score < n_c) ? OR_ACCESSIBLE : OR_BLOCKED;
    }
}


/* ------------------------------------------------------------------------- */
/* Soft clearance and its gradient (the differentiable form).                */
/* ------------------------------------------------------------------------- */

/* TSDF value of a voxel as single precision data: S / (w 2^20), or tau when
 * the voxel is unobserved or outside the box. */
static double sdf_voxel(const or_map *m, int32_t ix, int32_t iy, int32_t iz) {
    int64_t S;
    uint32_t w;
    int32_t cl;
    if (!in_domain(&m->cfg, ix, iy, iz)) return (double)m->cfg.tau;
    or_get_voxel(m, ix, iy, iz, &S, &w, &cl);
    if (w == 0) return (double)m->cfg.tau;
    return (double)(float)((double)S / ((double)w * 1048576.0));
}

/* Trilinear SDF in the cell whose low corner is `cell`, at fractional
 * position f (normally in [0, 1]); grad receives d SDF / d g (per voxel),
 * each component a weighted sum of corner differences along its axis. */
static double sdf_cell(const or_map *m, const int32_t cell[3], const double f[3], double grad[3]) {
    double D[2][2][2]; /* [dz][dy][dx] */
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                D[dz][dy][dx] = sdf_voxel(m, cell[0] + dx, cell[1] + dy, cell[2] + dz);
    const double w[3][2] = {{1.0 - f[0], f[0]}, {1.0 - f[1], f[1]}, {1.0 - f[2], f[2]}};
    double val = 0.0;
    grad[0] = grad[1] = grad[2] = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            grad[0] += (D[b][a][1] - D[b][a][0]) * w[1][a] * w[2][b];
            grad[1] += (D[b][1][a] - D[b][0][a]) * w[0][a] * w[2][b];
            grad[2] += (D[1][b][a] - D[0][b][a]) * w[0][a] * w[1][b];
            for (int c = 0; c < 2; ++c) val += D[c][b][a] * w[0][a] * w[1][b] * w[2][c];
        }
    return val;
}

/* Orthonormal tangent basis (t1, t2) of the unit vector n (Duff et al. 2017,
 * "Building an orthonormal basis, revisited"), in double ... */
static void onb_d(const double n[3], double t1[3], double t2[3]) {
    const double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    const double a = -1.0 / (sg + n[2]);
    const double b = n[0] * n[1] * a;
    t1[0] = 1.0 + sg * n[0] * n[0] * a;
    t1[1] = sg * b;
    t1[2] = -sg * n[0];
    t2[0] = b;
    t2[1] = sg + n[1] * n[1] * a;
    t2[2] = -n[1];
}

/* ... and in single precision, one rounded operation at a time. */
static void onb_f(const float n[3], float t1[3], float t2[3]) {
    const float sg = n[2] >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + n[2]);
    const float b = (n[0] * n[1]) * a;
    t1[0] = 1.0f + ((sg * n[0]) * n[0]) * a;
    t1[1] = sg * b;
    t1[2] = -(sg * n[0]);
    t2[0] = b;
    t2[1] = sg + (n[1] * n[1]) * a;
    t2[2] = -n[1];
}

void or_soft_seed(const float *normals, int64_t npts, const float *table, int32_t K, float *u0) {
    for (int64_t p = 0; p < npts; ++p) {
        const float *n = normals + 3 * p;
        float t1[3], t2[3];
        onb_f(n, t1, t2);
        for (int32_t k = 0; k < K; ++k) {
            const float *e = table + 3 * k;
            float *o = u0 + 3 * (p * K + k);
            for (int i = 0; i < 3; ++i) o[i] = (e[0] * t1[i] + e[1] * t2[i]) + e[2] * n[i];
        }
    }
}

/* The single-precision frame of one (point, direction) pair: the cell I of
 * the point on the sample grid (g = x / v - 1/2), the point's offset r in it,
 * the direction u and the standoff in voxels h / v. Sample j then sits at
 * g = I + r + (h / v + j) u. */
typedef struct {
    float I[3], r[3], w[3], e;
} pair_frame;

static void pair_frame_f(float v, const float s[3], const float u0[3], float al, float be,
                         float h, pair_frame *F) {
    float t1[3], t2[3], q[3];
    onb_f(u0, t1, t2);
    for (int i = 0; i < 3; ++i) q[i] = (u0[i] + al * t1[i]) + be * t2[i];
    const float nq = sqrtf((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]);
    for (int i = 0; i < 3; ++i) {
        const float o = s[i] / v - 0.5f;
        F->I[i] = floorf(o);
        F->r[i] = o - F->I[i];
        F->w[i] = q[i] / nq;
    }
    F->e = h / v;
}

/* Cell of sample j, decided in single precision; 0 if it is not a usable
 * integer (then the sample is treated as outside the box). */
static int sample_cell_f(const pair_frame *F, int j, int32_t cell[3]) {
    const float t = F->e + (float)j;
    for (int i = 0; i < 3; ++i) {
        const float l = F->r[i] + t * F->w[i];
        if (!(fabsf(l) < 1.0e7f) || !(fabsf(F->I[i]) < 1.0e9f)) return 0;
        cell[i] = (int32_t)F->I[i] + (int32_t)floorf(l);
    }
    return 1;
}

static int all_finite(const float *x, int n) {
    for (int i = 0; i < n; ++i)
        if (!isfinite(x[i])) return 0;
    return 1;
}

/* Soft clearance of one pair and its gradient, in double. */
static double soft_pair(const or_map *m, const or_tool *t, const float s[3], const float u0[3],
                        float al, float be, float h, double tau_s, int fp32_cells,
                        double grad[3], double *cmin) {
    const float vf = m->cfg.v;
    const double v = (double)vf;
    const int J = (int)floorf((t->length + t->corr_length) / vf);
    if (!all_finite(s, 3) || !all_finite(u0, 3) || !isfinite(al) || !isfinite(be) ||
        !isfinite(h)) {
        grad[0] = grad[1] = grad[2] = NAN;
        *cmin = NAN;
        return NAN;
    }
    /* direction and its derivatives */
    double n0[3], t1[3], t2[3], q[3];
    for (int i = 0; i < 3; ++i) n0[i] = (double)u0[i];
    onb_d(n0, t1, t2);
    double nq = 0.0;
    for (int i = 0; i < 3; ++i) {
        q[i] = n0[i] + (double)al * t1[i] + (double)be * t2[i];
        nq += q[i] * q[i];
    }
    nq = sqrt(nq);
    double u[3], du_a[3], du_b[3];
    for (int i = 0; i < 3; ++i) u[i] = q[i] / nq;
    const double ut1 = u[0] * t1[0] + u[1] * t1[1] + u[2] * t1[2];
    const double ut2 = u[0] * t2[0] + u[1] * t2[1] + u[2] * t2[2];
    for (int i = 0; i < 3; ++i) {
        du_a[i] = (t1[i] - u[i] * ut1) / nq;
        du_b[i] = (t2[i] - u[i] * ut2) / nq;
    }
    pair_frame F;
    pair_frame_f(vf, s, u0, al, be, h, &F);

    double *phi = (double *)malloc(sizeof(double) * 4 * (size_t)(J > 0 ? J : 1));
    double *dpa = phi + (J > 0 ? J : 1), *dpb = dpa + (J > 0 ? J : 1), *dph = dpb + (J > 0 ? J : 1);
    int ns = 0;
    double mn = INFINITY;
    for (int j = 1; j <= J; ++j) {
        const float aj = (float)j * vf;
        if (!(aj > t->self_excl)) continue;
        const double margin = aj <= t->length ? (double)t->radius : (double)t->corr_radius;
        const double dist = (double)h + (double)j * v; /* a_j */
        double g[3], f[3], G[3];
        int32_t cell[3];
        for (int i = 0; i < 3; ++i) g[i] = (double)s[i] / v - 0.5 + dist * u[i] / v;
        int ok = 1;
        if (fp32_cells) {
            ok = sample_cell_f(&F, j, cell);
        } else {
            for (int i = 0; i < 3; ++i) {
                if (!(fabs(g[i]) < 1.0e9)) ok = 0;
                else cell[i] = (int32_t)floor(g[i]);
            }
        }
        double D;
        if (ok) {
            for (int i = 0; i < 3; ++i) f[i] = g[i] - (double)cell[i];
            D = sdf_cell(m, cell, f, G);
        } else {
            D = (double)m->cfg.tau;
            G[0] = G[1] = G[2] = 0.0;
        }
        phi[ns] = D - margin;
        /* x_j = s + a_j u: d x / d h = u, d x / d alpha = a_j du/dalpha;
         * d SDF / d x = G / v */
        dph[ns] = (G[0] * u[0] + G[1] * u[1] + G[2] * u[2]) / v;
        dpa[ns] = dist * (G[0] * du_a[0] + G[1] * du_a[1] + G[2] * du_a[2]) / v;
        dpb[ns] = dist * (G[0] * du_b[0] + G[1] * du_b[1] + G[2] * du_b[2]) / v;
        if (phi[ns] < mn) mn = phi[ns];
        ++ns;
    }
    double C;
    *cmin = ns ? mn : NAN;
    if (ns == 0) {
        C = NAN;
        grad[0] = grad[1] = grad[2] = NAN;
    } else {
        /* softmin; d C / d phi_j = exp(-phi_j / tau_s) / sum_i exp(-phi_i / tau_s) */
        double Z = 0.0, ga = 0.0, gb = 0.0, gh = 0.0;
        for (int k = 0; k < ns; ++k) Z += exp(-(phi[k] - mn) / tau_s);
        for (int k = 0; k < ns; ++k) {
            const double wk = exp(-(phi[k] - mn) / tau_s) / Z;
            ga += wk * dpa[k];
            gb += wk * dpb[k];
            gh += wk * dph[k];
        }
        C = mn - tau_s * log(Z);
        grad[0] = ga;
        grad[1] = gb;
        grad[2] = gh;
    }
    free(phi);
    return C;
}

void or_soft_clearance(const or_map *m, const or_tool *t, const float *pts, uint32_t per_point,
                       const float *u0, const float *alpha, const float *beta, const float *h,
                       int64_t npairs, double tau_s, int fp32_cells, double *c,
                       double *g_alpha, double *g_beta, double *g_h, double *cmin) {
    for (int64_t i = 0; i < npairs; ++i) {
        double g[3], mn;
        c[i] = soft_pair(m, t, pts + 3 * (i / per_point), u0 + 3 * i, alpha[i], beta[i], h[i],
                         tau_s, fp32_cells, g, &mn);
        if (cmin) cmin[i] = mn;
        if (g_alpha) g_alpha[i] = g[0];
        if (g_beta) g_beta[i] = g[1];
        if (g_h) g_h[i] = g[2];
    }
}

void or_soft_refine(const or_map *m, const or_tool *t, const float *pts, uint32_t per_point,
                    const float *u0, float *alpha, float *beta, float *h, int64_t npairs,
                    double tau_s, int steps, float lr_dir, float lr_h, float h_max, double *c,
                    double *cmin) {
    for (int64_t i = 0; i < npairs; ++i) {
        const float *s = pts + 3 * (i / per_point);
        double g[3], mn;
        for (int k = 0; k < steps; ++k) {
            soft_pair(m, t, s, u0 + 3 * i, alpha[i], beta[i], h[i], tau_s, 1, g, &mn);
            /* gradient ascent on C, standoff kept in [0, h_max] */
            alpha[i] = (float)((double)alpha[i] + (double)lr_dir * g[0]);
            beta[i] = (float)((double)beta[i] + (double)lr_dir * g[1]);
            double hn = (double)h[i] + (double)lr_h * g[2];
            hn = hn < 0.0 ? 0.0 : (hn > (double)h_max ? (double)h_max : hn);
            h[i] = (float)hn;
        }
        c[i] = soft_pair(m, t, s, u0 + 3 * i, alpha[i], beta[i], h[i], tau_s, 1, g, &mn);
        if (cmin) cmin[i] = mn;
    }
}
