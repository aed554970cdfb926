/*
 * af.h -- C ABI of the Accessibility Field hot path on NVIDIA GB300 (sm_103a).
 *
 * The library integrates LiDAR scans into a truncated signed distance field
 * (TSDF) held in a sparse voxel-brick hash map, keeps a bit-packed occupied /
 * known view of it, and scores surface points for tool accessibility against
 * precomputed tool and approach-corridor voxel kernels (Scott, Schofield,
 * Green, "Beyond Visibility: Real-Time Surface Accessibility Fields from
 * Sparse LiDAR": Sec. 3.2 scan-centric TSDF, Sec. 3.4 accessibility scoring,
 * Sec. 3.5 confidence, Sec. 3.6 GPU implementation).
 *
 * Conventions for every entry point:
 *  - Units are metres; voxel i covers [i v, (i+1) v) on each axis and its
 *    centre is ((float)i + 0.5f) * v.
 *  - Pointers named d_* are device memory owned by the caller; pointers named
 *    h_* are host memory owned by the caller. The library owns the map, the
 *    kernel tables and its scratch, allocated in af_create / af_set_tool, and
 *    on first use by the calls that say so (af_points_enable, the af_soft_*
 *    views, the projective range image, work-sharing records beyond
 *    max_points); all of it is freed by af_destroy.
 *
 * Entry points: the map (af_create, af_integrate_scan, af_set_tool,
 * af_score, af_frame_host), batched ticks (af_batch_*), the differentiable
 * form (af_soft_*), the stateful point layer (af_points_*), the paper's
 * variants (af_integrate_scan_projective; clamp_signed in af_config; the
 * coarse-to-fine search in af_points_config), scheduling (af_set_score_split),
 * an allocation-free integration (af_integrate_scan_noalloc), and status,
 * statistics, export, profiling and kernel-table inspection calls.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *    that take a stream are asynchronous on it unless stated otherwise.
 *  - Argument errors are returned synchronously and nothing is enqueued.
 *    Errors found on the device (capacity) are latched in a device status
 *    word; af_sync_status returns them. AF_ERR_CAPACITY is sticky: later
 *    integrations are skipped, the map keeps the last committed scan, and
 *    scoring keeps working on it.
 *  - A context is not thread-safe; use it from one host thread.
 *  - The library is built twice with the same entry points: libaf.so, and
 *    libaf_checked.so (compiled with AF_CHECKED), where every pool index,
 *    plane-word index and run-table index that the integration, bit-view and
 *    scoring kernels use is checked before the access; a failed check skips
 *    the access (a read gives 0) and latches AF_ERR_CHECK in the device
 *    status word, which af_sync_status returns. af_version names the build.
 *  - Fault injection for tests: when the environment variable
 *    AF_FAIL_ALLOC_AT holds k >= 0, af_create's k-th device allocation
 *    (counting from 0) fails as if the device were out of memory: af_create
 *    frees what it allocated and returns AF_ERR_CUDA.
 */
#ifndef AF_H
#define AF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct af_ctx af_ctx;

typedef enum {
    AF_OK = 0,
    AF_ERR_INVALID_ARG = 1, /* bad argument; nothing was enqueued          */
    AF_ERR_CAPACITY = 2,    /* hash, brick pool or per-call size exceeded */
    AF_ERR_CUDA = 3,        /* a CUDA call failed; see af_last_error       */
    AF_ERR_TIMEOUT = 4,     /* a bounded device wait gave up               */
    AF_ERR_STATE = 5,       /* call out of order (e.g. score before tool)  */
    AF_ERR_CHECK = 6        /* a bounds check of the checked build failed  */
} af_status;

/* Per-point labels written by af_score (Fig. 1: green / red / grey). */
enum { AF_UNSCORED = 0, AF_ACCESSIBLE = 1, AF_BLOCKED = 2 };
/* Kernel selectors for af_kernel_offsets. */
enum { AF_KERNEL_TOOL = 0, AF_KERNEL_CORRIDOR = 1 };

/*
 * Map parameters (Sec. 3.2 - 3.6). Integers that the paper derives from
 * v and tau are passed explicitly so both ends agree on them exactly.
 */
typedef struct {
    float voxel_size;     /* v                                                  */
    float truncation;     /* tau; contributions are clamped to [0, tau]        *
                           * ([-tau, tau] with clamp_signed)                   */
    float r_c;            /* collision threshold: occupied iff TSDF < r_c      */
    float cone_cos;       /* voxels with cos(theta) > cone_cos behind a return
                             are not updated (Sec. 3.2; 0.95)                  */
    float range_min;      /* returns with range outside [range_min, range_max] */
    float range_max;      /*   are dropped (0.1 m, 40 m)                       */
    float clear_lo;       /* ray-cleared band (clear_lo tau, clear_hi tau]     */
    float clear_hi;       /*   toward the sensor (Sec. 3.4; 1.0, 2.25)         */
    int32_t cube_radius;  /* m = ceil(tau / v): (2m+1)^3 cube (Sec. 3.6), 1..8 */
    int32_t clear_samples;/* samples N_s along the cleared band, 0..64         */
    uint32_t w_min;       /* points are scored iff their voxel has w >= w_min  */
    uint32_t w_cap;       /* weight cap with proportional rescale (Sec. 3.6)   */
    uint32_t block_edge;  /* voxels per brick edge; must be 8                  */
    int32_t domain_min[3];     /* map box, in bricks: bricks [min, min+size)  */
    uint32_t domain_bricks[3]; /*   (the paper's bounded window, Sec. 3.3)    */
    uint32_t hash_capacity;    /* hash slots, a power of two                  */
    uint32_t pool_blocks;      /* bricks that can be allocated                */
    uint32_t max_returns;      /* largest n per af_integrate_scan            */
    uint32_t max_points;       /* largest m per af_frame_host                */
    int32_t clamp_signed;      /* 0: the paper's positive clamp [0, tau];     *
                                * 1: [-tau, tau], the ablation of Tab. 4.     *
                                * Only the clamp changes; S may then be < 0.  */
} af_config;

/* A cylinder tool of radius r and length L whose tip (the interaction point)
 * sits on the surface point and whose body extends along the approach
 * direction u, followed by a coaxial approach corridor (Sec. 3.4). */
typedef struct {
    float radius;          /* r                                                */
    float length;          /* L                                                */
    float self_excl;       /* r_s: kernel voxels within r_s of the tip ignored */
    float corr_radius;     /* corridor radius                                  */
    float corr_length;     /* corridor extends over (L, L + corr_length]       */
    float cos_theta_max;   /* direction u is a candidate iff n . u > this      */
    uint32_t n_c;          /* collision threshold n_c (Sec. 3.4, 4.1; 5)       */
    int32_t corridor_strict; /* 1: unknown corridor voxels also block          */
} af_tool;

typedef struct {
    uint64_t scans;             /* af_integrate_scan calls                      */
    uint64_t returns_in;        /* returns offered                              */
    uint64_t returns_accepted;  /* returns integrated                           */
    uint64_t blocks_allocated;  /* bricks in use                                */
    uint64_t blocks_dirty_last; /* bricks touched by the last scan              */
    uint64_t points_in;         /* points offered to af_score                  */
    uint64_t points_scored;     /* points that passed the confidence gate       */
    uint64_t tests;             /* (scored point, candidate direction) pairs    */
} af_stats;

/* Library version string (static storage). */
const char *af_version(void);

/* Creates a context on the current CUDA device and allocates all map memory
 * (hash, brick pool, occupancy planes, scratch). Returns AF_ERR_INVALID_ARG
 * for inconsistent parameters, AF_ERR_CUDA if allocation fails. */
af_status af_create(const af_config *cfg, af_ctx **out);

/* Frees everything the context owns. Synchronises the device first. */
af_status af_destroy(af_ctx *ctx);

/*
 * Integrates one LiDAR scan (Sec. 3.2, 3.4, 3.6).
 *  d_xyz : n x 3 float32, returns in the sensor frame, row-major (x,y,z).
 *  n     : 0 <= n <= max_returns (n = 0 is a no-op that still counts a scan).
 *  pose  : host float[16], row-major 4x4 world_from_sensor; its translation
 *          is the sensor origin q; the point is p = R ps + t.
 * Per return: dropped if non-finite, out of range, or its cube leaves the
 * map box. Otherwise every voxel x of its (2m+1)^3 cube outside the
 * behind-surface cone receives d = |p - q| - |x - q| clamped to [0, tau]
 * (accumulated exactly as round(d 2^20) in integers, w += 1), and the voxels
 * of N_s samples of the band toward the sensor are marked ray-cleared. At the
 * end of the call weights above w_cap are capped with proportional rescaling
 * and the occupied / known view of every touched brick is rebuilt.
 * Asynchronous on `stream`; d_xyz must stay valid until the work completes.
 */
af_status af_integrate_scan(af_ctx *ctx, const float *d_xyz, uint32_t n,
                            const float pose[16], void *stream);

/*
 * Projective integration, the ablation of Tab. 3 (Sec. 3.2): the same
 * arguments and return acceptance as af_integrate_scan, but the accepted
 * returns only build a range image -- the nearest range in each cell of a
 * bins x bins octahedral map of sensor-frame directions ((u, w) =
 * (d_x, d_y) / (|d_x| + |d_y| + |d_z|), the lower hemisphere folded onto the
 * corners; 812 gives the mean solid angle of a 0.25 x 0.25 degree bin) --
 * and every voxel x of the bricks their cubes overlap takes
 * d = (range of the cell of R^T (x - q)) - |x - q|, skipped if that cell is
 * empty or d < -tau, clamped as the map clamps. No cone, no cleared band;
 * the weight cap and the view rebuild as af_integrate_scan. 2 <= bins <= 8192;
 * the range image (bins^2 x 4 bytes) is allocated on first use and kept.
 * Asynchronous on `stream`.
 */
af_status af_integrate_scan_projective(af_ctx *ctx, const float *d_xyz, uint32_t n,
                                       const float pose[16], uint32_t bins, void *stream);

/*
 * Sets the tool and the approach-direction table (Sec. 3.4, 3.6): for each
 * of the G unit directions (h_dirs: host G x 3 float32, world frame) the
 * library rasterises the tool and corridor kernels and the three arm-path
 * samples once, and keeps them on the device (no rotation at run time).
 * 1 <= G <= 4096. Synchronous; replaces any previous tool.
 */
af_status af_set_tool(af_ctx *ctx, const af_tool *tool, const float *h_dirs, uint32_t G);

/*
 * Scores m surface points (Sec. 3.4, 3.5).
 *  d_pts, d_normals : m x 3 float32 (points; outward unit normals).
 *  d_label : m uint8  -> AF_UNSCORED (voxel weight below w_min),
 *                        AF_ACCESSIBLE (best direction score < n_c),
 *                        AF_BLOCKED.
 *  d_best  : m int16  -> index of the best direction (lowest index among the
 *                        minimum scores), -1 if unscored or no candidate.
 * A direction's score is n_c + 1 when an arm sample is occupied or unknown or
 * the corridor holds an occupied voxel, else min(#occupied tool voxels, n_c).
 * Requires af_set_tool (else AF_ERR_STATE). Asynchronous on `stream`. Calls
 * on one context must not overlap on different streams: the scorer takes
 * points from a counter that the context owns.
 */
af_status af_score(af_ctx *ctx, const float *d_pts, const float *d_normals, uint32_t m,
                   uint8_t *d_label, int16_t *d_best, void *stream);

/*
 * Work sharing of af_score (and af_frame_host): a point whose search takes
 * more than `budget` candidate directions past the arm screen hands the rest
 * of its directions to a second kernel that searches them one warp per
 * (point, direction); the labels and best directions are identical to the
 * single-pass search for every budget. budget = -1: single pass, one warp
 * per point (the default); 0 .. 4096: the hand-off threshold. The hand-off
 * records take 12 bytes per point, allocated for max_points at af_create and
 * grown (synchronously) for larger m. Adds two launches per af_score call.
 */
af_status af_set_score_split(af_ctx *ctx, int32_t budget);

/*
 * One whole frame from host buffers: copies the scan and the points to the
 * device, integrates, scores, copies labels and best directions back, and
 * waits for `stream`. Sizes are bounded by max_returns / max_points. Returns
 * the latched device status as well (AF_ERR_CAPACITY if the map is full).
 * Host buffers should be page-locked for asynchronous copies.
 */
af_status af_frame_host(af_ctx *ctx, const float *h_xyz, uint32_t n, const float pose[16],
                        const float *h_pts, const float *h_normals, uint32_t m,
                        uint8_t *h_label, int16_t *h_best, void *stream);

/* Waits for the context's last stream and returns the latched device status
 * (AF_OK, AF_ERR_CAPACITY, or AF_ERR_CHECK in the checked build). Does not
 * clear it. */
af_status af_sync_status(af_ctx *ctx);

/* Synchronises and fills *out. */
af_status af_get_stats(af_ctx *ctx, af_stats *out);

/* Synchronises and returns the number of allocated bricks. */
af_status af_block_count(af_ctx *ctx, uint32_t *out);

/*
 * Synchronises and copies the allocated bricks to host memory, at most `cap`
 * of them (order unspecified). Brick b covers voxels
 * (domain_min + key) * 8 + (lx, ly, lz), voxel l = lx + 8 ly + 64 lz.
 *  h_key     : cap x 3 int32   brick coordinates (absolute, in bricks)
 *  h_S       : cap x 512 int64  SDF sums in units of 2^-20 m (negative only
 *              with clamp_signed)
 *  h_w       : cap x 512 uint32 weights
 *  h_flags   : cap x 512 uint8  bit0 cleared, bit1 occupied, bit2 known
 * *out_count receives the number written.
 */
af_status af_export_blocks(af_ctx *ctx, uint32_t cap, int32_t *h_key, int64_t *h_S,
                           uint32_t *h_w, uint8_t *h_flags, uint32_t *out_count);

/*
 * Host-only: the integer voxel offsets of the tool (which = AF_KERNEL_TOOL)
 * or corridor (AF_KERNEL_CORRIDOR) kernel that the library rasterises for
 * direction u (Sec. 3.4). Writes min(count, cap) x 3 int32 to h_out (any
 * order) and the full count to *count. Needs no GPU.
 */
af_status af_kernel_offsets(const af_tool *tool, float voxel_size, const float u[3],
                            int32_t which, int32_t *h_out, int64_t cap, int64_t *count);

/* Host-only: the three arm-path sample offsets at {0.6, 1.25, 2.25} tau along
 * u (Sec. 3.4), as 3 x 3 int32 rows. Needs no GPU. */
af_status af_arm_offsets(float voxel_size, float truncation, const float u[3], int32_t h_out[9]);

/*
 * Batched ticks: many maps (scenes), each with its own scan, tool and
 * direction table, integrated and scored together -- one CUDA graph launch
 * per tick whose persistent kernels share the GPU across scenes of uneven
 * size. The result of a tick is exactly that of af_integrate_scan followed
 * by af_score on every scene (Sec. 3.2 - 3.5; the batching itself is the
 * implementation's, not the paper's).
 *
 * af_batch_create groups existing contexts (same device, same cube_radius,
 * each at most once); they must outlive the batch and must not be used on
 * another stream while a tick is in flight. Each tick reads the scenes' tools
 * as set at that time.
 */
typedef struct af_batch af_batch;

typedef struct {
    const float *d_xyz;      /* n x 3 returns, sensor frame (as af_integrate_scan) */
    uint32_t n;              /* 0 <= n <= the scene's max_returns                  */
    float pose[16];          /* world_from_sensor, row-major                       */
    const float *d_pts;      /* m x 3 points to score after integration            */
    const float *d_normals;  /* m x 3 normals                                      */
    uint32_t m;              /* 0 = score nothing for this scene                   */
    uint8_t *d_label;        /* m labels (as af_score)                             */
    int16_t *d_best;         /* m best-direction indices                           */
} af_batch_item;

/* Launch shape of a batch: integration tile and scoring CTA size. */
typedef struct {
    uint32_t returns_per_tile;  /* returns per integration CTA: 8, 16 or 32      */
    uint32_t warps_per_cta;     /* warps per scoring CTA: 2, 4 or 8              */
    uint32_t explored;          /* candidate shapes timed so far (of 9)         */
    uint32_t done;              /* 1 once the shape is final                     */
    float ms[9];                /* mean tick time per candidate (tile-major), 0 if untimed */
} af_batch_tuning;

af_status af_batch_create(af_ctx *const *scenes, uint32_t count, af_batch **out);
af_status af_batch_destroy(af_batch *batch);

/* One tick: items[s] is scene s's scan and points (count items). Asynchronous
 * on `stream`; the item buffers must stay valid until the tick completes. The
 * first 18 ticks time the 9 candidate launch shapes twice each (the online
 * autotuner), later ticks use the fastest; results never depend on the shape. */
af_status af_batch_tick(af_batch *batch, const af_batch_item *items, void *stream);

/* Fixes the launch shape (tile 8/16/32, warps 2/4/8); (0, 0) returns to tuning. */
af_status af_batch_set_tuning(af_batch *batch, uint32_t returns_per_tile, uint32_t warps_per_cta);

/* Synchronises and reports the tuner's state and the chosen shape. */
af_status af_batch_get_tuning(af_batch *batch, af_batch_tuning *out);

/*
 * The differentiable form: soft clearance. Not in the paper -- a smooth
 * companion of the tool / corridor test of Sec. 3.4 whose gradient refines an
 * approach direction and a standoff continuously.
 *
 * A pair is a surface point s and an approach direction. Pair i belongs to
 * point i / per_point (points' pairs adjacent; the last point may have
 * fewer). Its direction is u = (u0 + alpha t1 + beta t2) / |u0 + alpha t1 +
 * beta t2|, (t1, t2) the orthonormal tangent basis of the unit vector u0
 * (Duff et al. 2017), and its tool starts at standoff h along u. The axis is
 * sampled at a_j = h + j v, j = 1..floor((L + L_c) / v), skipping j v <= r_s
 * (the tool's self-exclusion); sample j has margin r while j v <= L, r_corr
 * beyond (the af_tool set on the context). With SDF the trilinear
 * interpolation over voxel centres of the TSDF S / (w 2^20) (Sec. 3.2; tau
 * where w = 0 or outside the map box), phi_j = SDF(x_j) - margin_j and
 *     C = -tau_s log sum_j exp(-phi_j / tau_s)   (softmin; C <= min_j phi_j).
 * C > 0 means every axis sample clears its margin. Where every sample reads
 * tau the gradient is exactly zero (truncation).
 *
 * Buffers are device memory owned by the caller; pairs are float32: d_pts
 * (points x 3), d_u0 (n x 3, unit), d_alpha, d_beta, d_h, outputs (n).
 * The first call builds a single-precision view of the map (dense: 36 bytes
 * per voxel of the box; brick-sparse: 16 KB per brick near an observed one;
 * see af_soft_set_view; AF_ERR_CAPACITY if it cannot be allocated) and later
 * calls rebuild it when scans were integrated since; the map's updates must be
 * ordered before the call on `stream`. AF_ERR_STATE without a tool or when
 * no axis sample lies beyond r_s. Asynchronous on `stream`. Non-finite
 * inputs give NaN outputs.
 */
typedef struct {
    uint32_t steps;  /* ascent steps                                      */
    float lr_dir;    /* alpha, beta += lr_dir * dC/d(alpha, beta)         */
    float lr_h;      /* h += lr_h * dC/dh, then h kept in [0, h_max]      */
    float h_max;
} af_refine;

/* Seeds: u0[p*K + k] = table_k rotated into the tangent frame of normal p
 * (table +z -> the normal): h_table is K x 3 host floats (a hemisphere set
 * of K approach orientations around +z), d_normals m x 3 unit normals.
 * The table is uploaded when it differs from the previous call's (the
 * device is synchronised first); repeated calls with the same table are
 * asynchronous. */
af_status af_soft_seed(af_ctx *ctx, const float *d_normals, uint32_t m, const float *h_table,
                       uint32_t K, float *d_u0, void *stream);

/* Start directions of refinement from the plain path: for each of m points
 * scored by af_score, u0[p] = the context's direction best[p] when label[p]
 * is AF_ACCESSIBLE, NaN otherwise (the soft calls return NaN for such pairs
 * without sampling). d_label / d_best are af_score's outputs, d_u0 m x 3. */
af_status af_soft_start(af_ctx *ctx, const uint8_t *d_label, const int16_t *d_best, uint32_t m,
                        float *d_u0, void *stream);

/* C of n pairs -> d_c; if d_cmin is given, also the hard clearance
 * min_j phi_j of each pair (> 0: every axis sample clears its margin). */
af_status af_soft_clearance(af_ctx *ctx, const float *d_pts, uint32_t per_point,
                            const float *d_u0, const float *d_alpha, const float *d_beta,
                            const float *d_h, uint64_t n, float tau_s, float *d_c,
                            float *d_cmin, void *stream);

/* Adjoint: with g = d_gc[i] (1 if d_gc is NULL), writes g dC/dalpha,
 * g dC/dbeta, g dC/dh (any of d_ga, d_gb, d_gh, d_c may be NULL to skip it;
 * d_c receives C). Recomputes every sample from the map: nothing from the
 * forward call is kept. */
af_status af_soft_clearance_adjoint(af_ctx *ctx, const float *d_pts, uint32_t per_point,
                                    const float *d_u0, const float *d_alpha, const float *d_beta,
                                    const float *d_h, uint64_t n, float tau_s, const float *d_gc,
                                    float *d_c, float *d_ga, float *d_gb, float *d_gh,
                                    void *stream);

/* R->steps gradient-ascent steps on C for every pair in one launch (alpha,
 * beta, h updated in place), then C (and, if d_cmin is given, the hard
 * clearance) at the final state. */
af_status af_soft_refine(af_ctx *ctx, const float *d_pts, uint32_t per_point, const float *d_u0,
                         float *d_alpha, float *d_beta, float *d_h, uint64_t n, float tau_s,
                         const af_refine *R, float *d_c, float *d_cmin, void *stream);

/* The SDF view the soft calls sample (the same values either way, so the
 * same results bit for bit): mode 1, dense -- one FP32 value per voxel of the
 * map box plus a 32-byte corner record per interpolation cell (36 bytes per
 * box voxel; boxes under 2^31 cells); mode 2, brick-sparse -- a 4-byte slot
 * per brick of the box (plus one layer below it) and 16 KB of corner records
 * for every brick within one brick below an allocated brick on each axis
 * (every cell whose corners touch an observed voxel; the others read tau),
 * sized by the map instead of the box, one more dependent load per sample;
 * mode 0 (default): dense when it fits (under 2^31 cells and within half
 * the free device memory), else sparse. Frees the current views; the next
 * soft call builds the chosen one. Synchronous. */
af_status af_soft_set_view(af_ctx *ctx, int32_t mode);

/* Per point of n pairs (per_point each, as above): the index within its
 * pairs of the largest d_c (lowest index on ties, -1 if all are NaN) ->
 * d_best_k, that value -> d_best_c, and, if d_best_u0 is given, that pair's
 * base direction from d_u0 (NaN for -1). Outputs may be NULL to skip. Needs
 * no map. */
af_status af_soft_best(af_ctx *ctx, const float *d_c, uint64_t n, uint32_t per_point,
                       const float *d_u0, int32_t *d_best_k, float *d_best_c, float *d_best_u0,
                       void *stream);

/*
 * The stateful layer around scoring (Sec. 3.4 normals and observation-side
 * filter, Sec. 3.5 incremental updates and confidence). The context keeps a
 * growing, voxel-deduplicated set of surface points (the centres of voxels
 * that received an accepted return) and, per point, its stored best score and
 * direction, accessibility confidence a, label, and up to 8 historical
 * viewpoints. Each af_points_frame integrates a scan (as af_integrate_scan),
 * adds its new points, raises the re-evaluation triggers and evaluates up to
 * `budget` queued points in point-id order; af_points_drain evaluates more of
 * the backlog between frames. Points are numbered in order of first
 * observation, the points new in one frame in (z, y, x) order of their
 * voxels. The rules:
 *  - viewpoints: once per scan that observes a point, the sensor position is
 *    added to its sum and, while fewer than max_views are stored, stored if
 *    farther than view_min_dist from every stored one;
 *  - normal: PCA over the k_nn nearest surface points (itself included) in the
 *    voxel cube of half-width nn_radius (ties in (dz, dy, dx) order), from
 *    the exact integer covariance of the voxel offsets, its smallest-eigenvalue
 *    eigenvector by 8 cyclic Jacobi sweeps in single precision, facing the
 *    mean sensor position; fewer than 3 neighbours: not evaluated;
 *  - candidates: n . u > cos_theta_max and u . (q - s) / |q - s| > obs_dot for
 *    some stored viewpoint q; scores as af_score (no candidate: n_c + 1);
 *  - triggers: new points; (i) TSDF at the voxel moved more than trig_tsdf
 *    since the previous frame; (ii) a changed voxel within r_u of the point
 *    (|o|^2 <= trig_radius^2 for the integer voxel offset o; r_u = 3v: 3):
 *    a voxel changes when its stored state (S, w, ray-cleared mark) after the
 *    frame's scan, weight cap included, differs from its state before; as in
 *    the paper, only a sample of the changed voxels is tested: when there are
 *    more than trig_sample (256), the trig_sample with the smallest
 *    h = mix(key ^ mix(f)), mix splitmix64's output function, key the
 *    absolute voxel index (x + 2^20) | (y + 2^20) << 21 | (z + 2^20) << 42,
 *    f the layer's frame number 1, 2, ... (trig_sample = 0 tests all);
 *    trig_exact = 0 replaces (ii) with the brick rule, a cheaper superset:
 *    a brick within one brick of the point's brick was touched by the scan
 *    (a return's cube or cleared-band sample lies in it); (iii) a sensor
 *    move of more than trig_move since the motion trigger last fired
 *    re-queues the points labelled AF_BLOCKED;
 *  - evaluation: points with c = w / (w + k_c) < c_min keep their state; the
 *    stored score only decreases (strictly lower replaces it and its
 *    direction); an accessible stored score (< n_c) with a new score >= n_c is
 *    a conflict (a *= a_decay), a new score < n_c confirms
 *    (a += a_recover (1 - a)); label AF_ACCESSIBLE iff stored score < n_c and
 *    c a > ca_min, else AF_BLOCKED (AF_UNSCORED before the first evaluation);
 *  - coarse-to-fine search (Sec. 3.6; c2f_stride > 0), for a direction table
 *    in ring order such as the paper's 180-direction yaw ring: the directions
 *    searched are every c2f_stride-th one and those within c2f_half indices
 *    (circularly) of a centre: the stored best direction of the nearest
 *    other point within c2f_radius (voxel-centre distance, ties in
 *    (dz, dy, dx) order) among those that had one when the batch began, else
 *    the coarse set's own best; lowest-index minimum over the searched
 *    candidates.
 * Needs af_set_tool before the first frame. Asynchronous on `stream`; the
 * export and stats calls synchronise.
 */
typedef struct {
    uint32_t capacity;     /* maximum number of points (AF_ERR_CAPACITY latched beyond) */
    uint32_t k_nn;         /* 10: neighbours of the normal, 3..343                      */
    int32_t nn_radius;     /* 3: neighbour search cube half-width in voxels, 1..3        */
    uint32_t max_views;    /* 8: stored viewpoints per point, <= 8                       */
    float view_min_dist;   /* 0.1 m                                                      */
    float obs_dot;         /* 0.25                                                       */
    float trig_tsdf;       /* 2 v                                                        */
    float trig_move;       /* 0.1 m                                                      */
    uint32_t budget;       /* evaluations per frame                                      */
    float k_c;             /* 5                                                          */
    float c_min;           /* 0.2                                                        */
    float a_decay;         /* 0.75                                                       */
    float a_recover;       /* 0.15                                                       */
    float ca_min;          /* 0.7                                                        */
    uint32_t c2f_stride;   /* 0: full search; yaw ring of 180: 10 (20 degrees)           */
    uint32_t c2f_half;     /* window half-width in directions; yaw ring: 12 (+-24 deg)   */
    float c2f_radius;      /* neighbour radius, 0.3 m; below 32 voxels                   */
    int32_t trig_exact;    /* 1: trigger (ii) over changed voxels; 0: the brick rule      */
    int32_t trig_radius;   /* 3: r_u in voxels, 0..7                                      */
    uint32_t trig_sample;  /* 256: changed voxels drawn per frame; 0: all of them         */
} af_points_config;

/* Allocates the layer: 2 KB per pool brick plus 200 B per point of capacity;
 * with trig_exact another 4.2 KB per pool brick (the touched bricks' state
 * before each scan). */
af_status af_points_enable(af_ctx *ctx, const af_points_config *cfg);
/* Integrate one scan and update the point layer (see above). */
af_status af_points_frame(af_ctx *ctx, const float *d_xyz, uint32_t n, const float pose[16],
                          void *stream);
/* Evaluate up to max_evals queued points in id order. */
af_status af_points_drain(af_ctx *ctx, uint32_t max_evals, void *stream);
/* Synchronises; number of points and evaluations of the last frame / drain. */
af_status af_points_stats(af_ctx *ctx, uint32_t *count, uint32_t *last_evals);
/* Synchronises; the first min(cap, count) points in id order (host arrays,
 * any may be NULL): absolute voxel (x 3), normal (x 3), label, stored score
 * (-1: never scored), stored direction, a, queued flag, stored viewpoints. */
af_status af_points_export(af_ctx *ctx, uint32_t cap, int32_t *h_ijk, float *h_normal,
                           uint8_t *h_label, int16_t *h_score, int16_t *h_best, float *h_a,
                           uint8_t *h_queued, int32_t *h_nviews, uint32_t *out_count);

/*
 * Kernel timing: when enabled, every launch of the context is bracketed by
 * CUDA events recorded on the launch's own stream. Index 0 = brick
 * allocation, 1 = cube integration, 2 = weight cap + bit view, 3 = scoring,
 * 4 = SDF view build, 5 = soft clearance, 6 = its adjoint, 7 = refinement,
 * 8 = seeding (af_soft_seed, af_soft_start), 9 = per-point best.
 * af_profile_read synchronises, sums the elapsed times of the recorded
 * launches (milliseconds) and, if `reset`, forgets them. launches[] counts
 * kernels: an af_score call with work sharing on is three (k_score,
 * k_score_split, k_score_finish) timed as one bracket.
 */
typedef struct {
    uint64_t launches[10];
    double ms[10];
} af_profile;
af_status af_profile_enable(af_ctx *ctx, int enable);
af_status af_profile_read(af_ctx *ctx, af_profile *out, int reset);

/*
 * Allocation-free scan integration. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- a real-time
 * loop whose memory is budgeted once at start-up, a host framework that owns
 * every device buffer through its own arena, code that must not enter the
 * CUDA allocator while other work runs. af_create allocates the hashed map,
 * so those callers integrate into a dense voxel box that they own instead.
 *
 * The call integrates one scan exactly as af_integrate_scan does (same drop
 * rules, same arithmetic, same weight cap and occupied / known rule; `cfg`'s
 * geometry and map box are used, its capacities are ignored) and ADDS it to
 * the box's current contents, so consecutive calls accumulate scans like a
 * map. The caller clears the box once before the first scan. The weight cap
 * and the flags are applied to the voxels the scan touches (the cubes and
 * cleared-band samples of its accepted returns); other voxels keep their
 * words and flags, so the cost follows the scan, not the box.
 *  box_min, box_dim : the output box in absolute voxel indices; voxel
 *                     (x, y, z) is element ((z - z0) * dy + (y - y0)) * dx +
 *                     (x - x0). Contributions outside the box are not kept.
 *  d_vox   : per voxel, S 2^20 + w in two's complement: S the SDF sum in
 *            units of 2^-20 m (negative only with clamp_signed; recover it
 *            by an arithmetic shift of the word as int64 by 20), w the
 *            weight (device memory, caller-owned, in/out).
 *  d_flags : per voxel, bit0 ray-cleared, bit1 occupied, bit2 known
 *            (device memory, caller-owned, in/out).
 * The library allocates nothing: its per-return scratch is a fixed device
 * array of AF_NOALLOC_MAX_RETURNS float4 (1 MiB) that every GPU loading the
 * library holds until the process exits. n > AF_NOALLOC_MAX_RETURNS returns
 * AF_ERR_CAPACITY (split the scan). A box of more than
 * AF_NOALLOC_MAX_BOX_VOXELS (2^40) voxels returns AF_ERR_INVALID_ARG. The
 * first call on a device looks up the
 * array's device address once; make that first call before any stream
 * capture. All calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller. Asynchronous on `stream`; errors are
 * reported through af_last_error(NULL).
 */
#define AF_NOALLOC_MAX_RETURNS 65536
#define AF_NOALLOC_MAX_BOX_VOXELS (1ull << 40)
af_status af_integrate_scan_noalloc(const af_config *cfg, const float *d_xyz, uint32_t n,
                                    const float pose[16], const int32_t box_min[3],
                                    const uint32_t box_dim[3], uint64_t *d_vox,
                                    uint8_t *d_flags, void *stream);

/*
 * The library's L2 read-bandwidth probe (no counterpart in the paper: the
 * denominator of the roofline of the kernels whose working set stays in L2).
 * Allocates a working set of `bytes` (a multiple of 16 in [1 MiB, 96 MiB],
 * well inside the L2) on the current device, brings it into L2, then reads it
 * `reps` times per launch with 16-byte L2-only loads from a persistent grid,
 * `launches` launches each timed with CUDA events on a stream of its own;
 * *gbs receives bytes * reps / (fastest launch's time) in GB/s. Synchronous;
 * frees what it allocated; errors through af_last_error(NULL).
 */
af_status af_probe_l2_read(uint64_t bytes, uint32_t reps, uint32_t launches, double *gbs);

/* Last error message of the context (static storage if ctx is NULL). */
const char *af_last_error(const af_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* AF_H */
