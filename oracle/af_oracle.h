/*
 * af_oracle.h -- declarations of the plain CPU oracle for the Accessibility
 * Field hot path.
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this code. The product (the CUDA library
 * and its Python binding) never includes, links or calls it, and this file
 * includes nothing from the product.
 *
 * Units: metres. Voxel indices are integers i with voxel i covering
 * [i*v, (i+1)*v) on each axis; its centre is ((float)i + 0.5f) * v.
 */
#ifndef AF_ORACLE_H
#define AF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float v;            /* voxel size (Sec. 3.2)                                  */
    float tau;          /* truncation distance tau (Sec. 3.2)                     */
    float r_c;          /* collision threshold on the TSDF (Sec. 3.4)             */
    float cone_cos;     /* behind-surface cone, cos(theta) > cone_cos excluded    */
    float range_min;    /* returns with |p - q| outside [range_min, range_max]   */
    float range_max;    /*   are dropped                                          */
    float clear_lo;     /* ray-cleared band (clear_lo*tau, clear_hi*tau]          */
    float clear_hi;     /*   toward the sensor (Sec. 3.4)                         */
    int32_t cube_radius;   /* m = ceil(tau / v): cube (2m+1)^3 (Sec. 3.6)        */
    int32_t clear_samples; /* N_s samples in the cleared band                    */
    uint32_t w_min;     /* confidence gate: scored iff w >= w_min (Sec. 3.5)      */
    uint32_t w_cap;     /* weight cap with proportional rescale of S (Sec. 3.6)   */
    int32_t dom_min[3]; /* map domain: voxel indices [dom_min, dom_min+dom_size) */
    int32_t dom_size[3];
    int32_t clamp_signed; /* 0: d clamped to [0, tau] (Sec. 3.2); 1: [-tau, tau],
                             the ablation of Tab. 4                              */
} or_config;

typedef struct {
    float radius;          /* tool cylinder radius r                              */
    float length;          /* tool cylinder length L (tip at the surface point)   */
    float self_excl;       /* self-exclusion radius r_s (Sec. 3.4)                */
    float corr_radius;     /* approach corridor radius                            */
    float corr_length;     /* approach corridor length beyond the tool            */
    float cos_theta_max;   /* candidate iff n . u > cos_theta_max (Sec. 3.4)      */
    uint32_t n_c;          /* collision-count threshold n_c (Sec. 3.4, 4.1)       */
    int32_t strict;        /* 1: unknown voxels block the corridor too            */
} or_tool;

typedef struct or_map or_map;

enum { OR_UNSCORED = 0, OR_ACCESSIBLE = 1, OR_BLOCKED = 2 };
enum { OR_KERNEL_TOOL = 0, OR_KERNEL_CORRIDOR = 1 };

or_map *or_map_new(const or_config *cfg);
void or_map_free(or_map *m);

/* One scan (Sec. 3.2 scan-centric update, Sec. 3.4 ray-cleared band,
 * Sec. 3.6 weight cap). pts: n x 3 floats in the sensor frame; pose: 4x4
 * row-major world_from_sensor. Returns the number of accepted returns. */
int64_t or_integrate(or_map *m, const float *pts, int64_t n, const float pose[16]);
/* Projective integration, the ablation of Tab. 3: the returns accepted by the
 * scan-centric rules fill a range image over bins x bins octahedral direction
 * cells (the nearest return per cell); every voxel of the 8^3 bricks that
 * their cubes overlap takes d = (range in its own cell) - |x - q|, skipped
 * if the cell is empty or d < -tau, clamped as the scan-centric path clamps;
 * no cone and no cleared band. Returns the accepted returns. */
int64_t or_integrate_projective(or_map *m, const float *pts, int64_t n, const float pose[16],
                                int32_t bins);
/* The octahedral cell (row-major, bins x bins) of direction d (exposed for its pins). */
int32_t or_octa_bin(const float d[3], int32_t bins);
/* The same, also writing the voxel of every accepted return to voxel_out
 * (n x 3, INT32_MIN for dropped returns) when it is not NULL. */
int64_t or_integrate2(or_map *m, const float *pts, int64_t n, const float pose[16],
                      int32_t *voxel_out);
/* As or_integrate2; band_out (n x clear_samples x 3, or NULL) receives the
 * voxel of each cleared-band sample marked for return k, sample s at row
 * k * clear_samples + (s - 1) (INT32_MIN where the return was dropped or the
 * sample fell outside the box). */
int64_t or_integrate_bands(or_map *m, const float *pts, int64_t n, const float pose[16],
                           int32_t *voxel_out, int32_t *band_out);

/* Voxel state. Absent voxels report S = 0, w = 0, cleared = 0. */
int or_get_voxel(const or_map *m, int32_t ix, int32_t iy, int32_t iz,
                 int64_t *S, uint32_t *w, int32_t *cleared);
void or_set_voxel(or_map *m, int32_t ix, int32_t iy, int32_t iz,
                  int64_t S, uint32_t w, int32_t cleared);
void or_set_voxels(or_map *m, int64_t n, const int32_t *ijk, const int64_t *S,
                   const uint32_t *w, const uint8_t *cleared);
int64_t or_voxel_count(const or_map *m);
const or_config *or_map_config(const or_map *m);
/* Writes every stored voxel: ijk (count x 3), S, w, cleared, occ, known. */
void or_export(const or_map *m, int32_t *ijk, int64_t *S, uint32_t *w,
               uint8_t *cleared, uint8_t *occ, uint8_t *known);
int or_occ(const or_map *m, int32_t ix, int32_t iy, int32_t iz);
int or_known(const or_map *m, int32_t ix, int32_t iy, int32_t iz);

/* Tool / corridor voxel kernel for one approach direction u (Sec. 3.4).
 * Writes up to cap offsets (x,y,z int32 triples) in z-major, then y, then x
 * order; returns the full count. */
int64_t or_kernel_offsets(const or_tool *t, float v, const float u[3], int which,
                          int32_t *out, int64_t cap);
/* The three arm-path sample offsets {0.6, 1.25, 2.25} tau along u (Sec. 3.4). */
void or_arm_offsets(float v, float tau, const float u[3], int32_t out[9]);

/* Accessibility scoring (Sec. 3.4, 3.5). dirs: G x 3 unit vectors.
 * label[k] in {UNSCORED, ACCESSIBLE, BLOCKED}; best[k] = index into dirs or -1.
 * dir_score (optional, m x G int32) receives each direction's score, or -1
 * for directions that are not candidates / points that are not scored. */
void or_score(const or_map *m, const or_tool *t, const float *dirs, int32_t G,
              const float *pts, const float *normals, int64_t npts,
              uint8_t *label, int16_t *best, int32_t *dir_score);

/* The same scoring with the kernel tables built once (Sec. 3.6: the kernels
 * are precomputed at initialisation): or_score is or_tables_new,
 * or_score_tables, or_tables_free. The tables hold the tool, the directions
 * and the voxel size and truncation they were built for, which must be the
 * map's. */
typedef struct or_tables or_tables;
or_tables *or_tables_new(const or_tool *t, float v, float tau, const float *dirs, int32_t G);
void or_tables_free(or_tables *T);
void or_score_tables(const or_map *m, const or_tables *T, const float *pts,
                     const float *normals, int64_t npts, uint8_t *label, int16_t *best,
                     int32_t *dir_score);

/* The differentiable form: soft clearance of (point, direction) pairs.
 * Pair i belongs to point i / per_point. For pair i with base direction u0,
 * tangent coordinates (alpha, beta) and standoff h it writes
 * C = softmin_{tau_s} over the axis samples of (SDF - margin),
 * dC/d(alpha, beta, h) and the hard clearance min_j (SDF - margin)
 * (gradients and cmin optional). Readings in af_oracle.c. */
void or_soft_clearance(const or_map *m, const or_tool *t, const float *pts, uint32_t per_point,
                       const float *u0, const float *alpha, const float *beta, const float *h,
                       int64_t npairs, double tau_s, int fp32_cells, double *c,
                       double *g_alpha, double *g_beta, double *g_h, double *cmin);
/* Seed directions: u0[p*K + k] = table_k rotated into the tangent frame of
 * normal p (table +z -> normal), single precision in a fixed order. */
void or_soft_seed(const float *normals, int64_t npts, const float *table, int32_t K, float *u0);
/* `steps` gradient-ascent steps on C (alpha, beta += lr_dir * grad;
 * h += lr_h * grad, kept in [0, h_max]; state rounded to single precision
 * after each step), then C and the hard clearance at the final state. */
void or_soft_refine(const or_map *m, const or_tool *t, const float *pts, uint32_t per_point,
                    const float *u0, float *alpha, float *beta, float *h, int64_t npairs,
                    double tau_s, int steps, float lr_dir, float lr_h, float h_max, double *c,
                    double *cmin);

/* ---- The stateful layer around scoring (Sec. 3.4 normals and
 * observation-side filter, Sec. 3.5 incremental updates and confidence). ---- */
typedef struct {
    uint32_t k_nn;        /* neighbours of the PCA normal, the point included (10)   */
    int32_t nn_radius;    /* neighbour search cube half-width, voxels (3)              */
    uint32_t max_views;   /* stored historical viewpoints per point, <= 8              */
    float view_min_dist;  /* a viewpoint is stored if farther than this from all others */
    float obs_dot;        /* observation-side filter threshold (0.25)                  */
    float trig_tsdf;      /* re-evaluate when the point's TSDF moves more (2v)         */
    float trig_move;      /* sensor motion that re-queues blocked points (0.1 m)      */
    uint32_t budget;      /* evaluations per frame; the rest waits in the backlog      */
    float k_c;            /* confidence c = w / (w + k_c)                              */
    float c_min;          /* points with c below are not evaluated (0.2)               */
    float a_decay;        /* accessibility confidence a *= a_decay on conflict (0.75)  */
    float a_recover;      /* a += a_recover (1 - a) on confirmation (0.15)             */
    float ca_min;         /* confident-accessible iff score < n_c and c a > ca_min    */
    /* Coarse-to-fine search (Sec. 3.6) over a direction table in ring order
     * (the yaw ring): 0 = off. The evaluated directions are the coarse set
     * {g : g mod c2f_stride = 0} and the window of indices within c2f_half
     * (circularly) of a centre: the best direction of the nearest other point
     * within c2f_radius whose stored best direction was set before this
     * batch of evaluations, else the coarse set's own best. */
    uint32_t c2f_stride;
    uint32_t c2f_half;
    float c2f_radius;
    /* Trigger (ii) of Sec. 3.5. trig_exact = 1: a voxel within trig_radius
     * voxels (|o|^2 <= trig_radius^2; r_u = 3v: 3) of the point's voxel
     * changed its stored state (S, w or ray-cleared mark) in this scan, among
     * the changed voxels sampled for the frame: at most trig_sample (256) of
     * them, those with the smallest or_mix64(key ^ or_mix64(frame)); 0 = all.
     * trig_exact = 0 (the brick rule): a brick within one brick of the point's
     * brick was touched by the scan (a return's cube or cleared-band sample
     * lies in it), a superset of the unsampled exact rule. */
    int32_t trig_exact;
    int32_t trig_radius;
    uint32_t trig_sample;
} or_pts_config;

/* splitmix64's output function: a bijection of 64-bit words (the hash that
 * draws the sample of trigger (ii)). */
uint64_t or_mix64(uint64_t z);

typedef struct or_pts or_pts;

/* A point set that follows map m, scored with tool t over the G directions. */
or_pts *or_pts_new(const or_map *m, const or_pts_config *pc, const or_tool *t, const float *dirs,
                   int32_t G);
void or_pts_free(or_pts *P);
/* One frame: integrate the scan into m, then ingest its returns as surface
 * points, raise the re-evaluation triggers and evaluate up to `budget`
 * queued points in id order. Returns the number of evaluations. */
int64_t or_pts_frame(or_pts *P, or_map *m, const float *pts, int64_t n, const float pose[16]);
/* Evaluate up to max queued points (the backlog between frames). */
int64_t or_pts_drain(or_pts *P, const or_map *m, int64_t max);
int64_t or_pts_count(const or_pts *P);
/* Per point in id order: voxel (n x 3), normal (n x 3), label, stored score
 * (-1 never scored), stored best direction, accessibility confidence a,
 * queued flag, number of stored viewpoints. */
void or_pts_export(const or_pts *P, int32_t *ijk, float *normal, uint8_t *label, int16_t *score,
                   int16_t *best, float *a, uint8_t *queued, int32_t *nviews);
/* The state update of one evaluation (exposed for its pins): score s and
 * direction g of the evaluation at confidence c update the stored score and
 * direction, the accessibility confidence a and the label. */
void or_pts_state_step(const or_pts_config *pc, int32_t n_c, int32_t s, int32_t g, float c,
                       int16_t *score, int16_t *best, float *a, uint8_t *label);
/* The symmetric-eigenvector routine of the normal (exposed for its pins):
 * cyclic Jacobi on A (3 x 3, row-major), `sweeps` sweeps; writes the
 * eigenvalues (diagonal after the sweeps) and eigenvectors (columns of V). */
void or_jacobi3(const float A[9], int sweeps, float evals[3], float V[9]);

#ifdef __cplusplus
}
#endif
#endif
