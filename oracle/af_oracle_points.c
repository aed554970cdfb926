/*
 * af_oracle_points.c -- plain CPU statement of the stateful layer around
 * accessibility scoring: the voxel-deduplicated surface point set (Sec. 3.1),
 * PCA normals oriented to the mean historical sensor position and the
 * observation-side filter over stored viewpoints (Sec. 3.4), the incremental
 * re-evaluation triggers with a per-frame budget and a backlog, the TSDF
 * confidence c and the accessibility confidence a (Sec. 3.5).
 *
 * TEST INFRASTRUCTURE, like af_oracle.c: only the test-suite, the smoke
 * check and the benchmark's CPU legs load it.
 *
 * Readings of the paper implemented here (it leaves them open):
 *  - A surface point is the centre of a voxel holding an accepted return;
 *    points are created in order of first observation, the points new in one
 *    frame in (z, y, x) order of their voxels, and numbered in that order.
 *  - Viewpoints: once per scan that observes a point, the scan's sensor
 *    position is added to the point's sum (for the mean sensor position) and,
 *    while fewer than max_views are stored, stored if it lies farther than
 *    view_min_dist from every stored one.
 *  - Normal: PCA over the k_nn nearest surface points (the point included),
 *    searched in the voxel cube of half-width nn_radius, nearest first, ties
 *    in (dz, dy, dx) order; the covariance is formed exactly from integer
 *    voxel offsets (k sum d d^T - (sum d)(sum d)^T, the same eigenvectors);
 *    its eigenvector of the smallest eigenvalue (lowest index on ties) comes
 *    from 8 cyclic Jacobi sweeps in single precision, and it is flipped to
 *    face the mean sensor position. Fewer than 3 neighbours: not evaluated.
 *  - Candidates: n . u > cos_theta_max and, for some stored viewpoint q,
 *    u . (q - s) / |q - s| > obs_dot (u points from the surface outward).
 *  - Triggers, after the frame's integration: (i) the TSDF at the point's
 *    voxel moved by more than trig_tsdf since the previous frame; (ii) a
 *    changed voxel within r_u of the point: |o|^2 <= R^2 for the integer
 *    offset o between the two voxels, R = trig_radius (3 for r_u = 3v). A
 *    voxel changes in a scan when its stored state (S, w, ray-cleared mark)
 *    after the scan, weight cap included, differs from its state before (a
 *    voxel never stored has S = w = 0 and no mark). Like the paper, the
 *    changed voxels are sampled to bound the query: when there are more
 *    than trig_sample (256) of them, the trig_sample with the smallest
 *    h = mix(key ^ mix(f)) are tested, mix the splitmix64 finaliser (a
 *    bijection, so no two voxels tie), key the packed absolute voxel index
 *    and f the layer's frame number (1, 2, ...); trig_sample = 0 tests them
 *    all. The sample is why (i) is not implied by (ii): the point's own
 *    voxel may change without being drawn. (iii) the sensor moved more than
 *    trig_move since the last time this trigger fired: every point labelled
 *    BLOCKED is re-queued; new points are always queued.
 *    The brick rule (trig_exact = 0), a cheaper superset of (ii) taken over
 *    every changed voxel: a brick within one brick of the point's brick was
 *    touched by the scan, i.e. it overlaps the cube of an accepted return or
 *    holds one of its cleared-band samples; every voxel that can change lies
 *    in such a brick, and r_u < one brick.
 *  - Budget: each frame dequeues up to `budget` queued points in id order;
 *    the rest stay queued (the backlog, also drained by or_pts_drain).
 *  - A dequeued point with c = w / (w + k_c) < c_min at its voxel keeps its
 *    state. Otherwise its best score s (n_c + 1 when no candidate) is taken
 *    with the scoring rules of af_oracle.c; the stored score only decreases
 *    (strictly lower replaces it, with its direction); a stored-accessible
 *    point (score < n_c) that scores s >= n_c is a conflict (a *= a_decay),
 *    a score s < n_c confirms (a += a_recover (1 - a)); the label is
 *    ACCESSIBLE iff the stored score < n_c and c a > ca_min, else BLOCKED.
 *  - Coarse-to-fine search (Sec. 3.6), for a direction table in ring order
 *    such as the paper's yaw ring: the directions searched are every
 *    c2f_stride-th one and those within c2f_half indices (circularly) of a
 *    centre. The centre is the stored best direction of the nearest other
 *    point within c2f_radius (voxel-centre distance; ties in (dz, dy, dx)
 *    order) among the points that had one when the batch of evaluations
 *    began; without such a point, the best of the coarse set. The result is
 *    the lowest-index minimum over the searched candidates.
 *
 * Floating point: single precision, one rounded operation at a time, in the
 * order written (build with -ffp-contract=off).
 */
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "af_oracle.h"

#define MAX_VIEWS 8
#define JACOBI_SWEEPS 8

typedef struct {
    int32_t ijk[3];
    float views[MAX_VIEWS][3];
    int32_t nviews;
    float qsum[3];
    uint32_t nobs;
    uint32_t last_scan;
    float last_tsdf;
    uint8_t queued, label;
    int16_t score, best;
    float a;
    float normal[3];
} or_point;

typedef struct {
    uint64_t *key;
    int64_t *val;
    uint64_t cap, count;
} keymap;

struct or_pts {
    or_pts_config pc;
    or_config mc;
    or_tool tool;
    int32_t G;
    float *dirs;
    int32_t **tk, **ck;
    int64_t *ntk, *nck;
    int32_t *arm;
    or_point *p;
    int64_t n, cap;
    keymap ids;        /* voxel key -> point id */
    int32_t (*off)[3]; /* neighbour offsets, nearest first */
    int32_t noff;
    int32_t (*c2f_off)[3]; /* coarse-to-fine neighbour ball, nearest first, origin excluded */
    int32_t c2f_noff;
    int16_t *snap;         /* stored best directions when the current batch began */
    float q_last[3];
    int have_q_last;
    uint32_t scan;
};

/* ---- keys and a small open-addressing map ---- */

static uint64_t vkey(int32_t x, int32_t y, int32_t z) {
    return ((uint64_t)(uint32_t)(x + (1 << 20)) & 0x1FFFFFu) |
           (((uint64_t)(uint32_t)(y + (1 << 20)) & 0x1FFFFFu) << 21) |
           (((uint64_t)(uint32_t)(z + (1 << 20)) & 0x1FFFFFu) << 42);
}

static uint64_t hmix(uint64_t k) {
    k ^= k >> 31;
    k *= 0x7fb5d329728ea185ULL;
    k ^= k >> 27;
    return k;
}

static void km_init(keymap *m, uint64_t cap) {
    m->cap = cap;
    m->count = 0;
    m->key = (uint64_t *)malloc(cap * sizeof(uint64_t));
    m->val = (int64_t *)malloc(cap * sizeof(int64_t));
    for (uint64_t i = 0; i < cap; ++i) m->key[i] = UINT64_MAX;
}

static void km_free(keymap *m) {
    free(m->key);
    free(m->val);
}

static int64_t km_get(const keymap *m, uint64_t k) {
    for (uint64_t h = hmix(k) & (m->cap - 1);; h = (h + 1) & (m->cap - 1)) {
        if (m->key[h] == k) return m->val[h];
        if (m->key[h] == UINT64_MAX) return -1;
    }
}

static void km_put(keymap *m, uint64_t k, int64_t v) {
    if (2 * (m->count + 1) > m->cap) {
        keymap g;
        km_init(&g, m->cap * 2);
        for (uint64_t i = 0; i < m->cap; ++i)
            if (m->key[i] != UINT64_MAX) km_put(&g, m->key[i], m->val[i]);
        km_free(m);
        *m = g;
    }
    uint64_t h = hmix(k) & (m->cap - 1);
    while (m->key[h] != UINT64_MAX && m->key[h] != k) h = (h + 1) & (m->cap - 1);
    if (m->key[h] == UINT64_MAX) m->count++;
    m->key[h] = k;
    m->val[h] = v;
}

static int32_t floor8(int32_t i) { return i >= 0 ? i / 8 : -((-i + 7) / 8); }

static int in_box(const or_config *c, int32_t x, int32_t y, int32_t z) {
    return x >= c->dom_min[0] && x < c->dom_min[0] + c->dom_size[0] && y >= c->dom_min[1] &&
           y < c->dom_min[1] + c->dom_size[1] && z >= c->dom_min[2] &&
           z < c->dom_min[2] + c->dom_size[2];
}

/* TSDF of a voxel: S / (w 2^20) in double rounded to single, tau if w = 0. */
static float tsdf_at(const or_map *m, const int32_t i[3], uint32_t *w_out) {
    int64_t S = 0;
    uint32_t w = 0;
    int32_t cl;
    if (in_box(or_map_config(m), i[0], i[1], i[2])) or_get_voxel(m, i[0], i[1], i[2], &S, &w, &cl);
    if (w_out) *w_out = w;
    if (w == 0) return or_map_config(m)->tau;
    return (float)((double)S / ((double)w * 1048576.0));
}

/* ---- the eigenvector routine ---- */

void or_jacobi3(const float A[9], int sweeps, float evals[3], float V[9]) {
    float a[3][3], v[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            a[i][j] = A[3 * i + j];
            v[i][j] = i == j ? 1.0f : 0.0f;
        }
    static const int pq[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sw = 0; sw < sweeps; ++sw)
        for (int k = 0; k < 3; ++k) {
            const int p = pq[k][0], q = pq[k][1], r = 3 - p - q;
            const float apq = a[p][q];
            if (apq == 0.0f) continue;
            /* rotation angle phi with tan(phi) = t zeroing a[p][q] */
            const float theta = (a[q][q] - a[p][p]) / (2.0f * apq);
            const float t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
            const float c = 1.0f / sqrtf(t * t + 1.0f);
            const float s = t * c;
            const float app = a[p][p] - t * apq;
            const float aqq = a[q][q] + t * apq;
            const float arp = a[r][p], arq = a[r][q];
            const float nrp = c * arp - s * arq;
            const float nrq = s * arp + c * arq;
            a[p][p] = app;
            a[q][q] = aqq;
            a[p][q] = a[q][p] = 0.0f;
            a[r][p] = a[p][r] = nrp;
            a[r][q] = a[q][r] = nrq;
            for (int i = 0; i < 3; ++i) {
                const float vip = v[i][p], viq = v[i][q];
                v[i][p] = c * vip - s * viq;
                v[i][q] = s * vip + c * viq;
            }
        }
    for (int i = 0; i < 3; ++i) {
        evals[i] = a[i][i];
        for (int j = 0; j < 3; ++j) V[3 * i + j] = v[i][j];
    }
}

/* ---- construction ---- */

static int off_cmp(const void *x, const void *y) {
    const int32_t *a = (const int32_t *)x, *b = (const int32_t *)y;
    const int32_t da = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    const int32_t db = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    if (da != db) return da < db ? -1 : 1;
    for (int k = 2; k >= 0; --k) /* (dz, dy, dx) */
        if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
    return 0;
}

or_pts *or_pts_new(const or_map *m, const or_pts_config *pc, const or_tool *t, const float *dirs,
                   int32_t G) {
    or_pts *P = (or_pts *)calloc(1, sizeof(or_pts));
    P->pc = *pc;
    if (P->pc.max_views > MAX_VIEWS) P->pc.max_views = MAX_VIEWS;
    P->mc = *or_map_config(m);
    P->tool = *t;
    P->G = G;
    P->dirs = (float *)malloc(sizeof(float) * 3 * (size_t)G);
    memcpy(P->dirs, dirs, sizeof(float) * 3 * (size_t)G);
    P->tk = (int32_t **)calloc((size_t)G, sizeof(int32_t *));
    P->ck = (int32_t **)calloc((size_t)G, sizeof(int32_t *));
    P->ntk = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    P->nck = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    P->arm = (int32_t *)calloc((size_t)G * 9, sizeof(int32_t));
    for (int32_t g = 0; g < G; ++g) {
        const float *u = dirs + 3 * g;
        P->ntk[g] = or_kernel_offsets(t, P->mc.v, u, OR_KERNEL_TOOL, NULL, 0);
        P->tk[g] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * P->ntk[g] + 1));
        or_kernel_offsets(t, P->mc.v, u, OR_KERNEL_TOOL, P->tk[g], P->ntk[g]);
        P->nck[g] = or_kernel_offsets(t, P->mc.v, u, OR_KERNEL_CORRIDOR, NULL, 0);
        P->ck[g] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * P->nck[g] + 1));
        or_kernel_offsets(t, P->mc.v, u, OR_KERNEL_CORRIDOR, P->ck[g], P->nck[g]);
        or_arm_offsets(P->mc.v, P->mc.tau, u, P->arm + 9 * g);
    }
    const int32_t R = pc->nn_radius, W = 2 * R + 1;
    P->noff = W * W * W;
    P->off = (int32_t (*)[3])malloc(sizeof(int32_t[3]) * (size_t)P->noff);
    int32_t k = 0;
    for (int32_t z = -R; z <= R; ++z)
        for (int32_t y = -R; y <= R; ++y)
            for (int32_t x = -R; x <= R; ++x) {
                P->off[k][0] = x;
                P->off[k][1] = y;
                P->off[k][2] = z;
                ++k;
            }
    qsort(P->off, (size_t)P->noff, sizeof(int32_t[3]), off_cmp);
    if (pc->c2f_stride > 0) {
        /* offsets o != 0 with |o|^2 v^2 <= radius^2, evaluated in double */
        const double v = (double)P->mc.v, r = (double)pc->c2f_radius;
        const int32_t Rb = (int32_t)(r / v) + 1;
        const int32_t Wb = 2 * Rb + 1;
        P->c2f_off = (int32_t (*)[3])malloc(sizeof(int32_t[3]) * (size_t)Wb * Wb * Wb);
        int32_t n = 0;
        for (int32_t z = -Rb; z <= Rb; ++z)
            for (int32_t y = -Rb; y <= Rb; ++y)
                for (int32_t x = -Rb; x <= Rb; ++x) {
                    const int32_t d2 = x * x + y * y + z * z;
                    if (d2 == 0 || (double)d2 * v * v > r * r) continue;
                    P->c2f_off[n][0] = x;
                    P->c2f_off[n][1] = y;
                    P->c2f_off[n][2] = z;
                    ++n;
                }
        P->c2f_noff = n;
        qsort(P->c2f_off, (size_t)n, sizeof(int32_t[3]), off_cmp);
    }
    P->cap = 1024;
    P->p = (or_point *)calloc((size_t)P->cap, sizeof(or_point));
    km_init(&P->ids, 1024);
    return P;
}

void or_pts_free(or_pts *P) {
    if (!P) return;
    for (int32_t g = 0; g < P->G; ++g) {
        free(P->tk[g]);
        free(P->ck[g]);
    }
    free(P->tk);
    free(P->ck);
    free(P->ntk);
    free(P->nck);
    free(P->arm);
    free(P->dirs);
    free(P->off);
    free(P->c2f_off);
    free(P->snap);
    free(P->p);
    km_free(&P->ids);
    free(P);
}

int64_t or_pts_count(const or_pts *P) { return P->n; }

/* ---- one evaluation ---- */

static void centre(const or_pts *P, const int32_t i[3], float s[3]) {
    for (int k = 0; k < 3; ++k) s[k] = ((float)i[k] + 0.5f) * P->mc.v;
}

/* Full score of direction g at voxel i (the rules of or_score). */
static int32_t dir_score(const or_pts *P, const or_map *m, const int32_t i[3], int32_t g) {
    const int32_t n_c = (int32_t)P->tool.n_c;
    int blocked = 0;
    for (int s = 0; s < 3; ++s) {
        const int32_t *o = P->arm + 9 * g + 3 * s;
        const int32_t x = i[0] + o[0], y = i[1] + o[1], z = i[2] + o[2];
        if (or_occ(m, x, y, z) || !or_known(m, x, y, z)) blocked = 1;
    }
    for (int64_t q = 0; q < P->nck[g]; ++q) {
        const int32_t *o = P->ck[g] + 3 * q;
        const int32_t x = i[0] + o[0], y = i[1] + o[1], z = i[2] + o[2];
        if (or_occ(m, x, y, z) || (P->tool.strict && !or_known(m, x, y, z))) blocked = 1;
    }
    int64_t count = 0;
    for (int64_t q = 0; q < P->ntk[g]; ++q) {
        const int32_t *o = P->tk[g] + 3 * q;
        count += or_occ(m, i[0] + o[0], i[1] + o[1], i[2] + o[2]);
    }
    return blocked ? n_c + 1 : (count < n_c ? (int32_t)count : n_c);
}

/* PCA normal of point pt (0 if fewer than 3 neighbours). */
static int pca_normal(const or_pts *P, const or_point *pt, float nrm[3]) {
    int64_t kk = 0, sx = 0, sy = 0, sz = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    for (int32_t k = 0; k < P->noff && kk < (int64_t)P->pc.k_nn; ++k) {
        const int32_t *o = P->off[k];
        if (km_get(&P->ids, vkey(pt->ijk[0] + o[0], pt->ijk[1] + o[1], pt->ijk[2] + o[2])) < 0)
            continue;
        kk++;
        sx += o[0];
        sy += o[1];
        sz += o[2];
        sxx += o[0] * o[0];
        syy += o[1] * o[1];
        szz += o[2] * o[2];
        sxy += o[0] * o[1];
        sxz += o[0] * o[2];
        syz += o[1] * o[2];
    }
    if (kk < 3) return 0;
    /* k * sum d d^T - (sum d)(sum d)^T: k times the covariance, exact */
    const float A[9] = {(float)(kk * sxx - sx * sx), (float)(kk * sxy - sx * sy),
                        (float)(kk * sxz - sx * sz), (float)(kk * sxy - sx * sy),
                        (float)(kk * syy - sy * sy), (float)(kk * syz - sy * sz),
                        (float)(kk * sxz - sx * sz), (float)(kk * syz - sy * sz),
                        (float)(kk * szz - sz * sz)};
    float ev[3], V[9];
    or_jacobi3(A, JACOBI_SWEEPS, ev, V);
    int j = 0;
    for (int k = 1; k < 3; ++k)
        if (ev[k] < ev[j]) j = k;
    for (int k = 0; k < 3; ++k) nrm[k] = V[3 * k + j];
    /* face the mean historical sensor position */
    float s[3], d[3];
    centre(P, pt->ijk, s);
    for (int k = 0; k < 3; ++k) d[k] = pt->qsum[k] / (float)pt->nobs - s[k];
    const float nd = (nrm[0] * d[0] + nrm[1] * d[1]) + nrm[2] * d[2];
    if (nd < 0.0f)
        for (int k = 0; k < 3; ++k) nrm[k] = -nrm[k];
    return 1;
}

/* Normal filter and observation-side filter of direction g (Sec. 3.4). */
static int is_candidate(const or_pts *P, const float nrm[3], const float (*vu)[3], int32_t nv,
                        int32_t g) {
    const float *u = P->dirs + 3 * g;
    const float nu = (nrm[0] * u[0] + nrm[1] * u[1]) + nrm[2] * u[2];
    if (!(nu > P->tool.cos_theta_max)) return 0;
    for (int32_t k = 0; k < nv; ++k)
        if ((u[0] * vu[k][0] + u[1] * vu[k][1]) + u[2] * vu[k][2] > P->pc.obs_dot) return 1;
    return 0;
}

/* Stored best direction, at the start of the batch, of the nearest other
 * point within the coarse-to-fine radius that had one; -1 if none. */
static int32_t nearest_resolved(const or_pts *P, const or_point *pt) {
    for (int32_t k = 0; k < P->c2f_noff; ++k) {
        const int32_t *o = P->c2f_off[k];
        const int64_t id = km_get(&P->ids, vkey(pt->ijk[0] + o[0], pt->ijk[1] + o[1],
                                               pt->ijk[2] + o[2]));
        if (id >= 0 && P->snap[id] >= 0) return P->snap[id];
    }
    return -1;
}

static void evaluate(or_pts *P, const or_map *m, or_point *pt) {
    const int32_t n_c = (int32_t)P->tool.n_c;
    pt->queued = 0;
    uint32_t w = 0;
    tsdf_at(m, pt->ijk, &w);
    const float c = (float)w / ((float)w + P->pc.k_c);
    if (!(c >= P->pc.c_min)) return;
    float nrm[3];
    if (!pca_normal(P, pt, nrm)) return;
    for (int k = 0; k < 3; ++k) pt->normal[k] = nrm[k];

    /* unit vectors from the point toward its stored viewpoints */
    float s[3], vu[MAX_VIEWS][3];
    centre(P, pt->ijk, s);
    for (int32_t k = 0; k < pt->nviews; ++k) {
        float d[3];
        for (int r = 0; r < 3; ++r) d[r] = pt->views[k][r] - s[r];
        const float len = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
        for (int r = 0; r < 3; ++r) vu[k][r] = d[r] / len;
    }

    /* the directions searched: all, or the coarse set and a window */
    uint8_t *in_e = (uint8_t *)malloc((size_t)P->G);
    const int32_t stride = (int32_t)P->pc.c2f_stride;
    for (int32_t g = 0; g < P->G; ++g) in_e[g] = stride == 0 || g % stride == 0;
    if (stride > 0) {
        int32_t centre = nearest_resolved(P, pt);
        if (centre < 0) { /* no resolved neighbour: the coarse set's own best */
            int32_t cs = 0, found = 0;
            for (int32_t g = 0; g < P->G; g += stride) {
                if (!is_candidate(P, nrm, vu, pt->nviews, g)) continue;
                const int32_t sc = dir_score(P, m, pt->ijk, g);
                if (!found || sc < cs) {
                    cs = sc;
                    centre = g;
                    found = 1;
                }
            }
        }
        if (centre >= 0)
            for (int32_t g = 0; g < P->G; ++g) {
                const int32_t d = abs(g - centre);
                if ((d < P->G - d ? d : P->G - d) <= (int32_t)P->pc.c2f_half) in_e[g] = 1;
            }
    }
    int32_t best_s = n_c + 1, best_g = -1, found = 0;
    for (int32_t g = 0; g < P->G; ++g) {
        if (!in_e[g] || !is_candidate(P, nrm, vu, pt->nviews, g)) continue;
        const int32_t sc = dir_score(P, m, pt->ijk, g);
        if (!found || sc < best_s) {
            best_s = sc;
            best_g = g;
            found = 1;
        }
    }
    free(in_e);
    if (!found) best_g = -1; /* no candidate: blocked, no direction */

    or_pts_state_step(&P->pc, n_c, best_s, best_g, c, &pt->score, &pt->best, &pt->a, &pt->label);
}

void or_pts_state_step(const or_pts_config *pc, int32_t n_c, int32_t s, int32_t g, float c,
                       int16_t *score, int16_t *best, float *a, uint8_t *label) {
    const int prev_acc = *score >= 0 && *score < n_c;
    /* the stored score only decreases */
    if (*score < 0 || s < *score) {
        *score = (int16_t)s;
        *best = (int16_t)g;
    }
    if (prev_acc && s >= n_c)
        *a = pc->a_decay * *a; /* conflicting evaluation */
    else if (s < n_c)
        *a = *a + pc->a_recover * (1.0f - *a); /* confirming evaluation */
    *label = (*score < n_c && c * *a > pc->ca_min) ? OR_ACCESSIBLE : OR_BLOCKED;
}

int64_t or_pts_drain(or_pts *P, const or_map *m, int64_t max) {
    int64_t done = 0;
    if (P->pc.c2f_stride > 0) { /* neighbours' directions as they were before this batch */
        free(P->snap);
        P->snap = (int16_t *)malloc(sizeof(int16_t) * (size_t)(P->n > 0 ? P->n : 1));
        for (int64_t id = 0; id < P->n; ++id) P->snap[id] = P->p[id].best;
    }
    for (int64_t id = 0; id < P->n && done < max; ++id)
        if (P->p[id].queued) {
            evaluate(P, m, &P->p[id]);
            done++;
        }
    return done;
}

/* ---- one frame ---- */

static int key_cmp(const void *x, const void *y) {
    const int32_t *a = (const int32_t *)x, *b = (const int32_t *)y;
    for (int k = 2; k >= 0; --k) /* (z, y, x) */
        if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
    return 0;
}

/* The stored state of every voxel: key -> index into (S, w, cleared). */
typedef struct {
    keymap at;
    int64_t *S;
    uint32_t *w;
    uint8_t *cl;
    int32_t *ijk;
    int64_t n;
} snapshot;

static void state_snapshot(const or_map *m, snapshot *out) {
    const int64_t nv = or_voxel_count(m);
    const size_t cnt = (size_t)(nv > 0 ? nv : 1);
    out->n = nv;
    out->ijk = (int32_t *)malloc(sizeof(int32_t) * 3 * cnt);
    out->S = (int64_t *)malloc(sizeof(int64_t) * cnt);
    out->w = (uint32_t *)malloc(sizeof(uint32_t) * cnt);
    out->cl = (uint8_t *)malloc(cnt);
    uint8_t *oc = (uint8_t *)malloc(cnt), *kn = (uint8_t *)malloc(cnt);
    or_export(m, out->ijk, out->S, out->w, out->cl, oc, kn);
    free(oc);
    free(kn);
    km_init(&out->at, 1024);
    for (int64_t k = 0; k < nv; ++k)
        km_put(&out->at, vkey(out->ijk[3 * k], out->ijk[3 * k + 1], out->ijk[3 * k + 2]), k);
}

static void snapshot_free(snapshot *s) {
    km_free(&s->at);
    free(s->ijk);
    free(s->S);
    free(s->w);
    free(s->cl);
}

/* splitmix64's output function (Steele, Lea, Flood 2014): a bijection of
 * 64-bit words. */
uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static int u64_cmp(const void *x, const void *y) {
    const uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* The changed voxels of the scan that trigger (ii) tests (see the header):
 * all of them, or the `sample` with the smallest h. */
static void changed_sample(const snapshot *before, const snapshot *after, uint32_t sample,
                           uint32_t f, keymap *out) {
    const uint64_t salt = or_mix64((uint64_t)f);
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(after->n > 0 ? after->n : 1));
    uint64_t *h = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(after->n > 0 ? after->n : 1));
    int64_t nc = 0;
    for (int64_t k = 0; k < after->n; ++k) {
        const uint64_t kk = vkey(after->ijk[3 * k], after->ijk[3 * k + 1], after->ijk[3 * k + 2]);
        const int64_t b = km_get(&before->at, kk);
        const int same = b >= 0 ? (before->S[b] == after->S[k] && before->w[b] == after->w[k] &&
                                   before->cl[b] == after->cl[k])
                                : (after->S[k] == 0 && after->w[k] == 0 && after->cl[k] == 0);
        if (same) continue;
        key[nc] = kk;
        h[nc] = or_mix64(kk ^ salt);
        ++nc;
    }
    uint64_t t = UINT64_MAX; /* the largest h tested */
    if (sample > 0 && nc > (int64_t)sample) {
        uint64_t *sorted = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nc);
        memcpy(sorted, h, sizeof(uint64_t) * (size_t)nc);
        qsort(sorted, (size_t)nc, sizeof(uint64_t), u64_cmp);
        t = sorted[sample - 1];
        free(sorted);
    }
    km_init(out, 1024);
    for (int64_t k = 0; k < nc; ++k)
        if (h[k] <= t) km_put(out, key[k], 1);
    free(key);
    free(h);
}

int64_t or_pts_frame(or_pts *P, or_map *m, const float *pts, int64_t n, const float pose[16]) {
    const float q[3] = {pose[3], pose[7], pose[11]};
    const int32_t mr = P->mc.cube_radius, ns = P->mc.clear_samples;
    const int exact = P->pc.trig_exact != 0;
    snapshot before;
    keymap tested; /* the changed voxels trigger (ii) tests */
    if (exact) state_snapshot(m, &before);
    int32_t *vox = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * (n > 0 ? n : 1)));
    int32_t *band = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * (n > 0 ? n : 1) * (ns > 0 ? ns : 1)));
    or_integrate_bands(m, pts, n, pose, vox, band);
    P->scan++;
    if (exact) {
        snapshot after;
        state_snapshot(m, &after);
        changed_sample(&before, &after, P->pc.trig_sample, P->scan, &tested);
        snapshot_free(&after);
        snapshot_free(&before);
    }

    /* bricks touched by the scan: the cubes and cleared-band samples of the
       accepted returns (the brick rule) */
    keymap changed;
    km_init(&changed, 1024);
    for (int64_t k = 0; k < n * ns; ++k) {
        const int32_t *j = band + 3 * k;
        if (j[0] != INT32_MIN) km_put(&changed, vkey(floor8(j[0]), floor8(j[1]), floor8(j[2])), 1);
    }
    /* new points, unique, in (z, y, x) order */
    int32_t *fresh = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * (n > 0 ? n : 1)));
    int64_t nf = 0;
    keymap seen;
    km_init(&seen, 1024);
    for (int64_t k = 0; k < n; ++k) {
        const int32_t *i = vox + 3 * k;
        if (i[0] == INT32_MIN) continue;
        for (int32_t bz = floor8(i[2] - mr); bz <= floor8(i[2] + mr); ++bz)
            for (int32_t by = floor8(i[1] - mr); by <= floor8(i[1] + mr); ++by)
                for (int32_t bx = floor8(i[0] - mr); bx <= floor8(i[0] + mr); ++bx)
                    km_put(&changed, vkey(bx, by, bz), 1);
        const uint64_t key = vkey(i[0], i[1], i[2]);
        if (km_get(&P->ids, key) < 0 && km_get(&seen, key) < 0) {
            km_put(&seen, key, 1);
            memcpy(fresh + 3 * nf, i, sizeof(int32_t) * 3);
            nf++;
        }
    }
    qsort(fresh, (size_t)nf, sizeof(int32_t) * 3, key_cmp);
    for (int64_t f = 0; f < nf; ++f) {
        if (P->n == P->cap) {
            P->cap *= 2;
            P->p = (or_point *)realloc(P->p, sizeof(or_point) * (size_t)P->cap);
        }
        or_point *pt = &P->p[P->n];
        memset(pt, 0, sizeof *pt);
        memcpy(pt->ijk, fresh + 3 * f, sizeof(int32_t) * 3);
        pt->last_tsdf = tsdf_at(m, pt->ijk, NULL);
        pt->queued = 1;
        pt->label = OR_UNSCORED;
        pt->score = -1;
        pt->best = -1;
        pt->a = 1.0f;
        km_put(&P->ids, vkey(pt->ijk[0], pt->ijk[1], pt->ijk[2]), P->n);
        P->n++;
    }

    /* viewpoints: once per scan that observes the point */
    const float md2 = P->pc.view_min_dist * P->pc.view_min_dist;
    for (int64_t k = 0; k < n; ++k) {
        const int32_t *i = vox + 3 * k;
        if (i[0] == INT32_MIN) continue;
        or_point *pt = &P->p[km_get(&P->ids, vkey(i[0], i[1], i[2]))];
        if (pt->last_scan == P->scan) continue;
        pt->last_scan = P->scan;
        for (int r = 0; r < 3; ++r) pt->qsum[r] = pt->qsum[r] + q[r];
        pt->nobs++;
        if ((uint32_t)pt->nviews < P->pc.max_views) {
            int far = 1;
            for (int32_t v = 0; v < pt->nviews; ++v) {
                const float d[3] = {q[0] - pt->views[v][0], q[1] - pt->views[v][1],
                                    q[2] - pt->views[v][2]};
                if (!((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] > md2)) far = 0;
            }
            if (far) {
                memcpy(pt->views[pt->nviews], q, sizeof(float) * 3);
                pt->nviews++;
            }
        }
    }

    /* triggers (i) and (ii) */
    const int32_t R = P->pc.trig_radius;
    for (int64_t id = 0; id < P->n; ++id) {
        or_point *pt = &P->p[id];
        const float cur = tsdf_at(m, pt->ijk, NULL);
        if (fabsf(cur - pt->last_tsdf) > P->pc.trig_tsdf) pt->queued = 1;
        pt->last_tsdf = cur;
        if (exact) {
            for (int32_t dz = -R; dz <= R && !pt->queued; ++dz)
                for (int32_t dy = -R; dy <= R && !pt->queued; ++dy)
                    for (int32_t dx = -R; dx <= R && !pt->queued; ++dx)
                        if (dx * dx + dy * dy + dz * dz <= R * R &&
                            km_get(&tested, vkey(pt->ijk[0] + dx, pt->ijk[1] + dy,
                                                 pt->ijk[2] + dz)) >= 0)
                            pt->queued = 1;
        } else {
            const int32_t bx = floor8(pt->ijk[0]), by = floor8(pt->ijk[1]), bz = floor8(pt->ijk[2]);
            for (int32_t dz = -1; dz <= 1 && !pt->queued; ++dz)
                for (int32_t dy = -1; dy <= 1 && !pt->queued; ++dy)
                    for (int32_t dx = -1; dx <= 1 && !pt->queued; ++dx)
                        if (km_get(&changed, vkey(bx + dx, by + dy, bz + dz)) >= 0) pt->queued = 1;
        }
    }
    /* trigger (iii) */
    if (P->have_q_last) {
        const float d[3] = {q[0] - P->q_last[0], q[1] - P->q_last[1], q[2] - P->q_last[2]};
        if ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] > P->pc.trig_move * P->pc.trig_move) {
            for (int64_t id = 0; id < P->n; ++id)
                if (P->p[id].label == OR_BLOCKED) P->p[id].queued = 1;
            memcpy(P->q_last, q, sizeof q);
        }
    } else {
        memcpy(P->q_last, q, sizeof q);
        P->have_q_last = 1;
    }

    km_free(&changed);
    if (exact) km_free(&tested);
    km_free(&seen);
    free(fresh);
    free(vox);
    free(band);
    return or_pts_drain(P, m, (int64_t)P->pc.budget);
}

void or_pts_export(const or_pts *P, int32_t *ijk, float *normal, uint8_t *label, int16_t *score,
                   int16_t *best, float *a, uint8_t *queued, int32_t *nviews) {
    for (int64_t id = 0; id < P->n; ++id) {
        const or_point *pt = &P->p[id];
        for (int k = 0; k < 3; ++k) {
            if (ijk) ijk[3 * id + k] = pt->ijk[k];
            if (normal) normal[3 * id + k] = pt->normal[k];
        }
        if (label) label[id] = pt->label;
        if (score) score[id] = pt->score;
        if (best) best[id] = pt->best;
        if (a) a[id] = pt->a;
        if (queued) queued[id] = pt->queued;
        if (nviews) nviews[id] = pt->nviews;
    }
}
