// af_internal.cuh -- device-side layout shared by the integration and scoring
// kernels of libaf (sm_103a).
//
// Map layout in HBM (all allocated once in af_create):
//  * hash   : open addressing, hash_capacity 16-byte slots of (u64 brick key,
//             u32 pool index, u32 scan stamp for dirty-brick deduplication).
//             Keys are domain-relative brick coordinates packed 21 bits per
//             axis; all ones marks an empty slot.
//  * pool   : bricks of 8^3 voxels. Each voxel is ONE u64 word holding
//             S 2^20 + w in two's complement (S is negative only in the
//             signed-clamp ablation), so a contribution is a single 64-bit
//             atomic add of round(d 2^20) 2^20 + 1 and integer addition makes
//             the sum independent of the order of the returns. w < 2^20 is
//             guaranteed by max_returns + w_cap < 2^20, |S| < 2^40 by
//             tau <= 1 m; S is the arithmetic shift of the word by 20.
//             Next to it: 512 cleared bits per brick and the brick key.
//  * planes : the occupied and known views as dense bit planes over the map
//             box, one bit per voxel, rows along x (64 voxels per u64 word),
//             row index z * Y + y. A brick row of 8 voxels is one byte, so the
//             view of a brick is 64 byte stores per plane. The occupied view
//             is also kept with rows along y (row index z * X + x) and along
//             z (row index y * X + x), so a kernel run can follow whichever
//             axis its direction is closest to.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace af {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kNoBlock = ~0u;
constexpr uint32_t kUnused = ~0u - 2;  // brick-table slot outside the return's cube
constexpr int kBrick = 8;
constexpr int kBrickVox = 512;
constexpr int kWBits = 20;
constexpr uint64_t kWMask = (1ull << kWBits) - 1;
constexpr float kScale = 1048576.0f;  // 2^20

// Latched device status (values of af_status).
constexpr uint32_t kStatusCapacity = 2;
constexpr uint32_t kStatusChecked = 6;  // AF_ERR_CHECK: a bounds check of the checked build

struct Control {
  uint32_t status;       // latched af_status of device-side failures
  uint32_t pool_count;   // bricks handed out
  uint32_t dirty_count;  // bricks touched by the current scan
  uint32_t pad;
  unsigned long long returns_accepted;
  unsigned long long points_scored;
  unsigned long long tests;
};

// One hash slot, 16 bytes, so that one load returns the brick key, its pool
// index and the scan stamp that deduplicates dirty-brick marks. All ones =
// empty slot (key ~0, pool index kNoBlock, stamp never equal to a scan).
struct alignas(16) HashSlot {
  unsigned long long key;
  uint32_t val;
  uint32_t stamp;
};

// Everything a kernel needs about the map; passed by value.
// The signed sum S of a voxel word (arithmetic shift: exact for any sign).
__host__ __device__ inline long long word_S(unsigned long long word) {
  return (long long)word >> kWBits;
}

// A voxel word from S and w (w < 2^20).
__host__ __device__ inline unsigned long long make_word(long long S, unsigned long long w) {
  return ((unsigned long long)S << kWBits) | w;
}

// Sec. 3.6's proportional rescale S w_cap / w, rounded toward minus infinity.
__host__ __device__ inline long long capped_S(long long S, long long w_cap, long long w) {
  const long long a = S * w_cap, q = a / w;
  return (a % w != 0 && a < 0) ? q - 1 : q;
}

struct MapView {
  // geometry
  float v, tau, r_c, cone_cos, range_min, range_max, clear_lo, clear_hi;
  float inv_v;        // 1 / v rounded to single precision
  int m;              // cube radius
  int ns;             // cleared-band samples
  uint32_t w_min, w_cap;
  uint64_t rcq;       // round(r_c 2^20)
  int clamp_signed;   // 1: contributions clamped to [-tau, tau] (Tab. 4 ablation)
  float dlo;          // lower clamp of d: 0, or -tau with clamp_signed
  int dom_vox[3];     // absolute voxel index of the box's min corner
  int dim_vox[3];     // box size in voxels (multiples of 8)
  int row_words;      // u64 words per plane row
  unsigned long long* occ_y;  // occupied, rows along y: row z * X + x
  unsigned long long* occ_z;  // occupied, rows along z: row y * X + x
  int row_words_y, row_words_z;
  // hash
  struct HashSlot* slots;
  uint32_t hmask;     // capacity - 1
  // pool
  unsigned long long* vox;  // pool_blocks * 512 packed words
  uint32_t* cleared;        // pool_blocks * 16
  uint64_t* bkey;           // pool_blocks
  uint32_t* dirty;          // pool_blocks
  uint32_t pool_blocks;
  // per-scan scratch: the pool index of each cube brick of each return
  uint32_t* rtab;           // max_returns * nbmax
  int nbmax;                // bricks a cube can span: ((2m + 7) / 8 + 1)^3
  // planes
  unsigned long long* occ;
  unsigned long long* known;
  Control* ctl;
  size_t words_x, words_y, words_z;  // 64-bit words of the x-row views, of occ_y, of occ_z
};

// Tool tables on the device (built by af_set_tool).
// Work sharing of the plain scorer: points whose search uses up its budget
// hand their remaining directions to a second kernel (one warp per
// (point, direction)), which folds them into a packed lowest-index minimum.
struct ScoreSplit {
  int2* over;        // (point, first direction not yet searched)
  uint32_t* res;     // packed (score << 16 | direction) of the search so far
  uint32_t* count;   // points handed off
  int budget;        // directions past the arm screen before a hand-off; < 0: never
  uint32_t* work;    // the staged scorer's next-point and finished-warp counters (zero
                     // between launches)
};

struct ToolView {
  const float* dirs;      // G x 3 unit directions
  const short4* runs;     // x-runs (dx0, len, dy, dz), len in 1..64
  const int2* fruns;      // the same runs as (row delta in plane words, dx0 | len << 16)
  const int4* dtab;       // per direction: tool runs [x, y), corridor runs [z, w)
  const short4* arm;      // G x 3 arm-sample offsets
  int ntool;              // every direction's tool runs come first: runs [0, ntool)
  int G;
  int n_c;
  float cos_max;
  int strict;
  int reach[3];           // largest |offset| per axis over every kernel and arm sample
  int nruns;              // entries of runs / fruns
  Control* ctl;           // the map's status word (the checked build's run-index checks)
};

__host__ __device__ inline uint64_t pack_brick(uint32_t bx, uint32_t by, uint32_t bz) {
  return (uint64_t)bx | ((uint64_t)by << 21) | ((uint64_t)bz << 42);
}

// splitmix64's output function (Steele, Lea, Flood 2014): a bijection of
// 64-bit words.
__host__ __device__ inline uint64_t mix64(uint64_t key) {
  key ^= key >> 30;
  key *= 0xbf58476d1ce4e5b9ull;
  key ^= key >> 27;
  key *= 0x94d049bb133111ebull;
  key ^= key >> 31;
  return key;
}

__device__ inline uint32_t hash_slot(uint64_t key, uint32_t mask) {
  return (uint32_t)mix64(key) & mask;
}

// One 16-byte slot read: key, pool index, stamp.
__device__ inline void load_slot(const MapView& M, uint32_t h, unsigned long long* key,
                                 uint32_t* val, uint32_t* stamp) {
  const uint4 s = __ldcg(reinterpret_cast<const uint4*>(M.slots) + h);
  *key = (unsigned long long)s.x | ((unsigned long long)s.y << 32);
  *val = s.z;
  *stamp = s.w;
}

// Slot holding `key` (or -1) with its pool index and stamp. Read-only probe;
// never spins: at most hmask + 1 slots are visited.
__device__ inline int find_slot(const MapView& M, uint64_t key, uint32_t* val, uint32_t* stamp) {
  uint32_t h = hash_slot(key, M.hmask);
  for (uint32_t probe = 0; probe <= M.hmask; ++probe) {
    unsigned long long k;
    load_slot(M, h, &k, val, stamp);
    if (k == key) return (int)h;
    if (k == kEmptyKey) return -1;
    h = (h + 1) & M.hmask;
  }
  return -1;
}

// Pool index of a brick, or kNoBlock.
__device__ inline uint32_t lookup_brick(const MapView& M, uint64_t key) {
  uint32_t val, stamp;
  if (find_slot(M, key, &val, &stamp) < 0) return kNoBlock;
  return val < M.pool_blocks ? val : kNoBlock;
}

__device__ inline void latch_status(Control* c, uint32_t code) {
  atomicCAS(&c->status, 0u, code);
}

// The checked build (libaf_checked.so, -DAF_CHECKED): `ok` is the bounds
// check of an index about to be used; a failure latches AF_ERR_CHECK and the
// caller skips the access. In the normal build the check is not compiled.
__device__ inline bool check_index(bool ok, Control* c) {
#ifdef AF_CHECKED
  if (!ok) latch_status(c, kStatusChecked);
  return ok;
#else
  (void)ok;
  (void)c;
  return true;
#endif
}

// Voxel index of a coordinate, floor(c / v) with c / v rounded in IEEE single
// precision. The product with the rounded reciprocal 1/v lies within
// |c / v| 2^-22 of the rounded quotient; when no integer lies within
// |c / v| 2^-20 of the product the floor is already decided by it, and
// otherwise the correctly rounded division decides. Same result either way.
__device__ inline bool voxel_index(float c, const MapView& M, int* out) {
  const float qa = c * M.inv_v;
  const float e = fabsf(qa) * 9.5367431640625e-07f;  // 2^-20
  float f;
  if (fabsf(qa) > 1e-30f && floorf(qa - e) == floorf(qa + e))
    f = floorf(qa);
  else
    f = floorf(__fdiv_rn(c, M.v));
  if (!(f >= -1.0e9f && f <= 1.0e9f)) return false;
  *out = (int)f;
  return true;
}

__device__ inline float voxel_centre(int i, float v) {
  return __fmul_rn(__fadd_rn((float)i, 0.5f), v);
}


// ---- per-return steps shared by the integration kernels (Sec. 3.2, 3.4) ----

struct Pose {
  float r[3][4];  // row-major [R | t]
};

// ---- the differentiable form (soft clearance) ----

// What the soft-clearance kernels read: the cell view of the map and the
// axis samples of the tool. Built per call by the host.
struct SoftView {
  const float4* cells;  // dense: ncell[0] * ncell[1] * ncell[2] cells, 2 float4 each;
                        // sparse: 512 cells (2 float4 each) per slot of bgrid
  int lo[3];            // absolute voxel index of the lowest cell's low corner
  int ncell[3];         // cells per axis: box voxels + 1
  int sparse;           // 1: the brick-sparse view
  const uint32_t* bgrid;  // sparse: per grid brick, the slot of its cells (kNoBlock: all tau)
  int glo[3];           // sparse: absolute voxel index of the grid's first brick corner
  int gdim[3];          // sparse: grid bricks per axis (box bricks + the layer below)
  float v, tau;
  float r, r_corr;      // margins: tool, corridor
  int j0, jt, J;        // samples j0..J; tool margin for j <= jt
  float k2;             // log2(e) / tau_s
  float ln2_tau_s;      // tau_s ln 2
  int fixed;            // 1: softmin weights against the fixed bound `ref`
  float ref;            // lower bound of every phi: -max(r, r_corr)
};

struct RefineArgs {
  int steps;
  float lr_dir, lr_h, h_max;
};

// ---- the stateful layer around scoring (Sec. 3.4, 3.5) ----

// One surface point (64 bytes). Its stored viewpoints live in a separate
// array, max 8 per point.
struct PtState {
  int32_t x, y, z;    // box-relative voxel
  uint32_t blk;       // pool index of its brick
  float qsum[3];      // sum of the sensor positions of the scans that saw it
  uint32_t nobs;      // number of such scans
  uint32_t last_scan; // stamp of the last of them
  float last_tsdf;    // TSDF at its voxel after the previous frame
  float a;            // accessibility confidence
  float n[3];         // normal of the last evaluation
  int16_t score, best;  // stored best score (-1: never scored) and direction
  uint8_t queued, label, nviews, pad;
};

struct PtCounters {
  uint32_t count;     // points
  uint32_t nnew;      // points new in this frame
  uint32_t nchanged;  // voxels whose stored state the frame's scan changed
  uint32_t nsnap;     // bricks whose state was copied before the frame's scan
  uint32_t nsel;      // points selected for evaluation
  uint32_t evals;     // evaluations of the last call
  uint32_t pad[2];
};

// The draw of changed voxels for the neighbourhood trigger: a radix
// selection of the `trig_sample` smallest hashes, 11 bits per pass.
struct PtSample {
  unsigned long long prefix;  // high bits of the selected bound found so far
  unsigned long long t;       // the largest hash drawn (all ones: every changed voxel)
  uint32_t below;             // changed voxels known to lie below the prefix's range
  uint32_t done;              // 1 once t is final
};

// Parameters of the layer as the kernels read them.
struct PtView {
  PtState* st;
  float4* views;         // capacity * 8
  int32_t* pid;          // point id per voxel of every pool brick, -1 none, -2 being created
  unsigned long long* newkeys;
  uint32_t* near;        // per pool brick: stamp of the last frame with a touched brick next to it
  unsigned long long* snapw;  // per dirty brick of the frame: its 512 voxel words before the scan
  uint32_t* snapc;            // ... and its 16 cleared-mark words
  uint32_t* chgmask;          // per dirty brick: 512 bits, voxels whose state changed
  uint32_t* hist;             // 2048 bins of the draw's radix selection
  PtSample* samp;
  int trig_exact;             // 1: changed voxels within trig_radius; 0: touched bricks
  int trig_radius;
  uint32_t trig_sample;       // changed voxels drawn per frame (0: all)
  unsigned long long salt;    // mix64(frame number of the layer)
  uint32_t* sel;
  uint32_t* blocksum;
  PtCounters* C;
  const int4* nnoff;     // neighbour offsets, nearest first, ties in (dz, dy, dx) order
  int noff;
  uint32_t capacity;
  int k_nn, nn_radius, max_views;
  float view_min_dist2, obs_dot, trig_tsdf, k_c, c_min, a_decay, a_recover, ca_min;
  // coarse-to-fine search (stride 0: off)
  int c2f_stride, c2f_half;
  int c2f_R;             // ball radius in whole voxels (<= 31)
  const int4* c2foff;    // the ball's offsets, origin excluded, nearest first
  int c2f_noff;
  int16_t* snap;         // stored best directions when the batch began
};

// ---- batched ticks: many maps in one set of persistent launches ----

// One map's share of a batched tick, rewritten every tick. The offsets are
// exclusive prefix sums over the batch, so a global work index maps to its
// map by a binary search.
struct SceneDesc {
  MapView M;
  ToolView T;
  Pose P;
  const float* xyz;     // n returns, sensor frame
  float4* ret;          // per-return scratch of the map's context
  const float* pts;     // m points and normals
  const float* nrm;
  uint8_t* label;
  int16_t* best;
  uint32_t n, m, frame;
  uint32_t alloc_off;   // allocation threads: n * (nbmax + N_s)
  uint32_t tile_off;    // integration tiles: ceil(n / returns per tile)
  uint32_t pt_off;      // scored points: m
};

struct BatchHdr {
  uint32_t count;
  uint32_t total_alloc, total_tiles, total_points;
};

// Largest s with off_F(s) <= x (F: 0 allocation, 1 tiles, 2 points). Maps
// with no work share their successor's offset, so the one found owns x.
template <int F>
__device__ inline int scene_of(const SceneDesc* __restrict__ D, int count, uint32_t x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const uint32_t off = F == 0 ? D[mid].alloc_off : (F == 1 ? D[mid].tile_off : D[mid].pt_off);
    if (off <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Transform, validate, voxel-index one return. Returns false if dropped.
__device__ inline bool prepare_return(const MapView& M, const Pose& P, float sx, float sy,
                                      float sz, float p[3], float* range, int rel[3]) {
  if (!isfinite(sx) || !isfinite(sy) || !isfinite(sz)) return false;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    p[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P.r[r][0], sx), __fmul_rn(P.r[r][1], sy)),
                               __fmul_rn(P.r[r][2], sz)),
                     P.r[r][3]);
  const float b0 = __fsub_rn(p[0], P.r[0][3]);
  const float b1 = __fsub_rn(p[1], P.r[1][3]);
  const float b2 = __fsub_rn(p[2], P.r[2][3]);
  const float bb = __fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2));
  *range = __fsqrt_rn(bb);
  if (!(*range >= M.range_min && *range <= M.range_max)) return false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int i;
    if (!voxel_index(p[k], M, &i)) return false;
    rel[k] = i - M.dom_vox[k];
    if (rel[k] - M.m < 0 || rel[k] + M.m >= M.dim_vox[k]) return false;
  }
  return true;
}

// Sample s (1..ns) of the ray-cleared band toward the sensor. Returns the
// domain-relative voxel, or false if it falls outside the map box.
__device__ inline bool band_sample(const MapView& M, const float p[3], const float q[3],
                                   float range, int s, int rel[3]) {
  const float step = __fdiv_rn(__fmul_rn(__fsub_rn(M.clear_hi, M.clear_lo), M.tau), (float)M.ns);
  const float start = __fmul_rn(M.clear_lo, M.tau);
  const float dist = __fadd_rn(start, __fmul_rn((float)s, step));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = __fdiv_rn(__fsub_rn(q[k], p[k]), range);
    int i;
    if (!voxel_index(__fadd_rn(p[k], __fmul_rn(dist, u)), M, &i)) return false;
    rel[k] = i - M.dom_vox[k];
    if (rel[k] < 0 || rel[k] >= M.dim_vox[k]) return false;
  }
  return true;
}

}  // namespace af
