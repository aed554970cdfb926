/*
 * synth_raycast.c -- first-hit ray casting against analytic primitives, for
 * the synthetic LiDAR scan generator (synth.py). Input generation only: no
 * part of the Accessibility Field method is computed here.
 *
 * Primitives are grouped; each group has a bounding capsule (segment a-b,
 * radius) that culls rays before the exact tests. Double precision; every
 * ray is independent, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>

#define EPS 1e-9

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* squared distance between ray o + t d (t >= 0, |d| = 1) and segment a-b */
static double ray_seg_dist2(const double *o, const double *d, const double *a, const double *b) {
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double r[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
    double ee = dot3(ab, ab), de = dot3(d, ab), dr = dot3(d, r), er = dot3(ab, r);
    double den = ee - de * de;
    double s = den > 1e-18 ? (er - de * dr) / den : 0.0;
    s = s < 0 ? 0 : (s > 1 ? 1 : s);
    double t = de * s - dr;
    if (t < 0) t = 0;
    s = ee > 1e-18 ? (er + t * de) / ee : 0.0;
    s = s < 0 ? 0 : (s > 1 ? 1 : s);
    double p[3];
    for (int k = 0; k < 3; ++k) p[k] = r[k] + t * d[k] - s * ab[k];
    return dot3(p, p);
}

static void hit_sphere(const double *o, const double *d, const double *s, double *tb, double *nb) {
    double oc[3] = {o[0] - s[0], o[1] - s[1], o[2] - s[2]};
    double b = dot3(d, oc), c = dot3(oc, oc) - s[3] * s[3];
    double disc = b * b - c;
    if (disc < 0) return;
    double q = sqrt(disc), t = -b - q;
    if (t <= EPS) t = -b + q;
    if (t <= EPS || t >= *tb) return;
    *tb = t;
    for (int k = 0; k < 3; ++k) nb[k] = o[k] + t * d[k] - s[k];
}

static void hit_box(const double *o, const double *d, const double *bx, double *tb, double *nb) {
    double tn = -INFINITY, tf = INFINITY;
    int axis = 0;
    for (int k = 0; k < 3; ++k) {
        if (fabs(d[k]) < 1e-300) {
            if (o[k] < bx[k] || o[k] > bx[k + 3]) return;
            continue;
        }
        double t1 = (bx[k] - o[k]) / d[k], t2 = (bx[k + 3] - o[k]) / d[k];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > tn) { tn = lo; axis = k; }
        if (hi < tf) tf = hi;
    }
    if (tf < tn || tf <= EPS) return;
    double t = tn > EPS ? tn : tf;
    if (t >= *tb) return;
    *tb = t;
    nb[0] = nb[1] = nb[2] = 0.0;
    nb[axis] = d[axis] > 0 ? -1.0 : 1.0;
}

static void hit_cylinder(const double *o, const double *d, const double *cy, double *tb, double *nb) {
    const double *a = cy, *b = cy + 3;
    double r = cy[6];
    double ax[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double h = sqrt(dot3(ax, ax));
    double w[3] = {ax[0] / h, ax[1] / h, ax[2] / h};
    double oa[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
    double dw = dot3(d, w), ow = dot3(oa, w);
    double dp[3], op[3];
    for (int k = 0; k < 3; ++k) { dp[k] = d[k] - dw * w[k]; op[k] = oa[k] - ow * w[k]; }
    double A = dot3(dp, dp), B = dot3(dp, op), Cc = dot3(op, op) - r * r;
    double disc = B * B - A * Cc;
    if (A > 1e-18 && disc >= 0) {
        double q = sqrt(disc);
        double ts[2] = {(-B - q) / A, (-B + q) / A};
        for (int i = 0; i < 2; ++i) {
            double t = ts[i], y = ow + t * dw;
            if (t > EPS && y >= 0 && y <= h && t < *tb) {
                *tb = t;
                for (int k = 0; k < 3; ++k) nb[k] = oa[k] + t * d[k] - y * w[k];
                break;
            }
        }
    }
    if (fabs(dw) > 1e-300) {
        for (int cap = 0; cap < 2; ++cap) {
            double yv = cap ? h : 0.0;
            double t = (yv - ow) / dw;
            if (t <= EPS || t >= *tb) continue;
            double pc[3];
            for (int k = 0; k < 3; ++k) pc[k] = oa[k] + t * d[k] - yv * w[k];
            if (dot3(pc, pc) <= r * r) {
                *tb = t;
                for (int k = 0; k < 3; ++k) nb[k] = cap ? w[k] : -w[k];
            }
        }
    }
}

/* Groups are arranged in clusters (contiguous group ranges, cl_off) with a
 * bounding capsule each (cl_caps, same layout as caps) that encloses every
 * group capsule of the cluster: a ray that misses it skips the cluster. */
void sr_raycast(int64_t n_clusters, const double *cl_caps, const int64_t *cl_off,
                const double *caps, const int64_t *sph_off, const double *sph,
                const int64_t *box_off, const double *box, const int64_t *cyl_off,
                const double *cyl, const double *o, int64_t n, const double *dirs, double *t_out,
                double *n_out) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        const double *d = dirs + 3 * i;
        double tb = INFINITY, nb[3] = {0, 0, 0};
        for (int64_t c = 0; c < n_clusters; ++c) {
            const double *cc = cl_caps + 7 * c;
            if (ray_seg_dist2(o, d, cc, cc + 3) > cc[6] * cc[6]) continue;
            for (int64_t g = cl_off[c]; g < cl_off[c + 1]; ++g) {
                const double *cp = caps + 7 * g;
                if (ray_seg_dist2(o, d, cp, cp + 3) > cp[6] * cp[6]) continue;
                for (int64_t k = sph_off[g]; k < sph_off[g + 1]; ++k) hit_sphere(o, d, sph + 4 * k, &tb, nb);
                for (int64_t k = box_off[g]; k < box_off[g + 1]; ++k) hit_box(o, d, box + 6 * k, &tb, nb);
                for (int64_t k = cyl_off[g]; k < cyl_off[g + 1]; ++k) hit_cylinder(o, d, cyl + 7 * k, &tb, nb);
            }
        }
        double nn = sqrt(dot3(nb, nb));
        t_out[i] = tb;
        for (int k = 0; k < 3; ++k) n_out[3 * i + k] = nn > 0 ? nb[k] / nn : 0.0;
    }
}
