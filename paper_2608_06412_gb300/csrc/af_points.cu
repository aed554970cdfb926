// af_points.cu -- the stateful layer around scoring (Sec. 3.4, 3.5 of the
// paper): the voxel-deduplicated surface point set of a map, PCA normals
// oriented to the mean historical sensor position, the observation-side
// filter over stored viewpoints, incremental re-evaluation triggers with a
// per-frame budget and a backlog, the TSDF confidence c and the
// accessibility confidence a.
//
// Per frame, after the scan's integration, on the caller's stream:
//  k_pts_snapshot (inside the scan's integration, after brick allocation)
//                 the state of every brick the scan touches, before the scan
//  k_pts_mark     one thread per return: new point voxels (claimed in the
//                 per-brick point-id table)
//  k_pts_near     (brick rule) bricks next to the scan's touched bricks
//  k_pts_create   new points numbered by key order within the frame, so ids
//                 never depend on thread timing
//  k_pts_views    once per (point, scan): sensor sum and stored viewpoints
//  k_pts_diff     per touched brick: the voxels whose stored state changed
//  k_pts_hist / k_pts_pick
//                 the draw: radix selection, 11 bits per pass, of the
//                 trig_sample smallest hashes of the changed voxels
//  k_pts_scatter  every drawn changed voxel queues the points within r_u
//  k_pts_trigger  one thread per point: TSDF change, brick rule, sensor
//                 motion for blocked points
//  k_pts_count / k_pts_scan / k_pts_select
//                 the first `budget` queued ids in id order
//  k_pts_snap     (coarse-to-fine search only) the stored best directions
//                 as they are before the batch
//  k_pts_eval     one warp per selected point: confidence gate, nearest
//                 neighbours, exact integer covariance, Jacobi eigenvector,
//                 view-filtered scoring (the plain path's exact search, or
//                 its coarse-to-fine form), state update
// The integer decisions (neighbour choice, eigenvector, orientation,
// candidate tests, gates) are taken in single precision with correctly
// rounded operations in a fixed order, as the CPU oracle takes them.
#include <af.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "af_ctx.cuh"
#include "af_internal.cuh"
#include "af_score.cuh"

namespace af {
cudaError_t launch_alloc(const MapView& M, const float* d_xyz, uint32_t n, const float pose[16],
                         float4* d_ret, uint32_t frame, cudaStream_t stream);
cudaError_t launch_cube(const MapView& M, uint32_t n, const float pose[16], const float4* d_ret,
                        uint32_t frame, cudaStream_t stream);
cudaError_t launch_bitview(const MapView& M, int num_sms, cudaStream_t stream);
}  // namespace af

namespace af {
namespace {

constexpr int kJacobiSweeps = 8;
constexpr int kSelBlock = 1024;  // ids per selection block

__device__ inline bool box_rel(const MapView& M, int x, int y, int z) {
  return (unsigned)x < (unsigned)M.dim_vox[0] && (unsigned)y < (unsigned)M.dim_vox[1] &&
         (unsigned)z < (unsigned)M.dim_vox[2];
}

__device__ inline unsigned long long rel_key(int x, int y, int z) {
  return (unsigned long long)x | ((unsigned long long)y << 21) | ((unsigned long long)z << 42);
}

__device__ inline int vox_slot(int x, int y, int z) { return (x & 7) | ((y & 7) << 3) | ((z & 7) << 6); }

// TSDF of a voxel word: S / (w 2^20) in double rounded to single, tau if w = 0.
__device__ inline float tsdf_word(unsigned long long word, float tau) {
  const unsigned long long w = word & kWMask;
  const long long S = word_S(word);
  return w ? __double2float_rn((double)S / ((double)w * 1048576.0)) : tau;
}

// The accepted return k's voxel (box-relative); false if it was dropped.
__device__ inline bool return_voxel(const MapView& M, const float4* ret, uint32_t k, int r[3]) {
  const float4 p = ret[k];
  if (p.w == 0.f) return false;
  int i[3];
  if (!voxel_index(p.x, M, &i[0]) || !voxel_index(p.y, M, &i[1]) || !voxel_index(p.z, M, &i[2]))
    return false;
  for (int a = 0; a < 3; ++a) r[a] = i[a] - M.dom_vox[a];
  return true;
}

// One thread per return: the voxel of an accepted return becomes a new
// point if it has none (claimed with -2 until k_pts_create numbers it).
__global__ void __launch_bounds__(256) k_pts_mark(MapView M, const float4* __restrict__ ret,
                                                  uint32_t n, PtView V) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int r[3];
  if (!return_voxel(M, ret, k, r)) return;
  const uint32_t b = lookup_brick(M, pack_brick(r[0] >> 3, r[1] >> 3, r[2] >> 3));
  if (b == kNoBlock) return;
  int32_t* slot = V.pid + (size_t)b * kBrickVox + vox_slot(r[0], r[1], r[2]);
  if (*slot == -1 && atomicCAS(slot, -1, -2) == -1)
    V.newkeys[atomicAdd(&V.C->nnew, 1u)] = rel_key(r[0], r[1], r[2]);
}

// Brick rule: one thread per (brick touched by the scan, neighbour of its
// 3 x 3 x 3 block). The scan's dirty list holds exactly the bricks that its
// cubes and cleared-band samples touch.
__global__ void __launch_bounds__(256) k_pts_near(MapView M, PtView V, uint32_t frame) {
  const uint32_t count = __ldcg(&M.ctl->dirty_count) * 27u;
  const int BX = M.dim_vox[0] >> 3, BY = M.dim_vox[1] >> 3, BZ = M.dim_vox[2] >> 3;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint64_t key = M.bkey[M.dirty[i / 27u]];
    const int o = (int)(i % 27u);
    const int x = (int)(key & 0x1FFFFF) + o % 3 - 1, y = (int)((key >> 21) & 0x1FFFFF) + (o / 3) % 3 - 1,
              z = (int)(key >> 42) + o / 9 - 1;
    if ((unsigned)x >= (unsigned)BX || (unsigned)y >= (unsigned)BY || (unsigned)z >= (unsigned)BZ)
      continue;
    const uint32_t b = lookup_brick(M, pack_brick(x, y, z));
    if (b != kNoBlock) V.near[b] = frame;
  }
}

// ---- trigger (ii): changed voxels near a point (Sec. 3.5) ----

// Copies the voxel words and cleared marks of every brick the scan touches;
// runs after brick allocation, which lists them all, and before integration.
__global__ void __launch_bounds__(512) k_pts_snapshot(MapView M, PtView V) {
  const uint32_t count = __ldcg(&M.ctl->dirty_count);
  if (blockIdx.x == 0 && threadIdx.x == 0) V.C->nsnap = count;
  const int l = threadIdx.x;
  for (uint32_t d = blockIdx.x; d < count; d += gridDim.x) {
    const uint32_t blk = M.dirty[d];
    V.snapw[(size_t)d * kBrickVox + l] = __ldcg(M.vox + (size_t)blk * kBrickVox + l);
    if (l < 16) V.snapc[(size_t)d * 16 + l] = __ldcg(M.cleared + (size_t)blk * 16 + l);
  }
}

// Absolute voxel of the box-relative voxel (x, y, z) packed as the draw's key.
__device__ inline unsigned long long draw_key(const MapView& M, int x, int y, int z) {
  return ((unsigned long long)(uint32_t)(x + M.dom_vox[0] + (1 << 20)) & 0x1FFFFFull) |
         (((unsigned long long)(uint32_t)(y + M.dom_vox[1] + (1 << 20)) & 0x1FFFFFull) << 21) |
         (((unsigned long long)(uint32_t)(z + M.dom_vox[2] + (1 << 20)) & 0x1FFFFFull) << 42);
}

// Box-relative voxel l of brick blk.
__device__ inline void brick_voxel(const MapView& M, uint32_t blk, int l, int* x, int* y, int* z) {
  const uint64_t key = M.bkey[blk];
  *x = (int)(key & 0x1FFFFF) * 8 + (l & 7);
  *y = (int)((key >> 21) & 0x1FFFFF) * 8 + ((l >> 3) & 7);
  *z = (int)(key >> 42) * 8 + (l >> 6);
}

// Per touched brick (after the weight cap): voxels whose word or cleared mark
// differs from the snapshot, as a 512-bit mask, and their count.
__global__ void __launch_bounds__(512) k_pts_diff(MapView M, PtView V) {
  const uint32_t count = __ldcg(&M.ctl->dirty_count), nsnap = V.C->nsnap;
  if (count > nsnap && blockIdx.x == 0 && threadIdx.x == 0)
    latch_status(M.ctl, kStatusCapacity);  // a brick missed by the snapshot: never expected
  const int l = threadIdx.x, lane = l & 31, wi = l >> 5;
  const uint32_t nd = min(count, nsnap);
  for (uint32_t d = blockIdx.x; d < nd; d += gridDim.x) {
    const uint32_t blk = M.dirty[d];
    const bool cl_now = (__ldcg(M.cleared + (size_t)blk * 16 + wi) >> lane) & 1u;
    const bool cl_then = (V.snapc[(size_t)d * 16 + wi] >> lane) & 1u;
    const bool ch = __ldcg(M.vox + (size_t)blk * kBrickVox + l) != V.snapw[(size_t)d * kBrickVox + l] ||
                    cl_now != cl_then;
    const unsigned b = __ballot_sync(0xffffffffu, ch);
    if (lane == 0) {
      V.chgmask[(size_t)d * 16 + wi] = b;
      if (b) atomicAdd(&V.C->nchanged, (unsigned)__popc(b));
    }
  }
}

// The draw's radix selection: digits of kDrawBits bits from the top of the
// hash down (the last one narrower), at most kDrawPasses passes; it stops as
// soon as a digit's bin holds exactly the draws still missing.
constexpr int kDrawBits = 11;
constexpr int kDrawBins = 1 << kDrawBits;
constexpr int kDrawPasses = (64 + kDrawBits - 1) / kDrawBits;

__device__ inline int draw_hi(int pass) { return 64 - kDrawBits * pass; }  // bits above the digit
__device__ inline int draw_lo(int pass) { return max(0, 64 - kDrawBits * (pass + 1)); }

// One pass of the draw: histogram (per CTA in shared memory, then merged) of
// this pass's digit of the hashes of the changed voxels whose higher bits
// equal the prefix found so far.
__global__ void __launch_bounds__(512) k_pts_hist(MapView M, PtView V, int pass) {
  __shared__ uint32_t s_hist[kDrawBins];
  const uint32_t k = V.trig_sample;
  if (V.samp->done || k == 0 || V.C->nchanged <= k) return;  // uniform
  const unsigned long long prefix = V.samp->prefix;
  const int hi = draw_hi(pass), lo = draw_lo(pass);
  const unsigned long long dmask = (1ull << (hi - lo)) - 1ull;
  const int l = threadIdx.x, lane = l & 31, wi = l >> 5;
  for (int b = l; b < kDrawBins; b += 512) s_hist[b] = 0u;
  __syncthreads();
  const uint32_t nd = min(__ldcg(&M.ctl->dirty_count), V.C->nsnap);
  for (uint32_t d = blockIdx.x; d < nd; d += gridDim.x) {
    if (!((V.chgmask[(size_t)d * 16 + wi] >> lane) & 1u)) continue;
    int x, y, z;
    brick_voxel(M, M.dirty[d], l, &x, &y, &z);
    const unsigned long long h = mix64(draw_key(M, x, y, z) ^ V.salt);
    if (pass > 0 && (h >> hi) != prefix) continue;
    atomicAdd(s_hist + ((h >> lo) & dmask), 1u);
  }
  __syncthreads();
  for (int b = l; b < kDrawBins; b += 512)
    if (s_hist[b]) atomicAdd(V.hist + b, s_hist[b]);
}

// Picks this pass's digit (one CTA, 2 bins per thread) and clears the
// histogram. When the digit's bin holds exactly the draws still missing, or
// after the last pass, t is final: every hash up to t is drawn, trig_sample
// of them (hashes of distinct voxels never tie: mix64 is a bijection).
__global__ void __launch_bounds__(1024) k_pts_pick(PtView V, int pass) {
  __shared__ uint32_t part[1024];
  PtSample* S = V.samp;
  const int tid = threadIdx.x;
  const uint32_t k = V.trig_sample;
  const bool all = k == 0 || V.C->nchanged <= k;
  if (!S->done && all) {
    if (tid == 0) {
      S->t = ~0ull;
      S->done = 1;
    }
  } else if (!S->done) {
    const uint32_t need = k - S->below;
    const uint32_t h0 = V.hist[2 * tid], h1 = V.hist[2 * tid + 1];
    const uint32_t sum = h0 + h1;
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan
      const uint32_t t = tid >= off ? part[tid - off] : 0u;
      __syncthreads();
      part[tid] += t;
      __syncthreads();
    }
    const uint32_t excl = part[tid] - sum;
    if (excl < need && need <= part[tid]) {
      const bool first = excl + h0 >= need;
      const uint32_t dg = 2 * tid + (first ? 0 : 1), before = excl + (first ? 0u : h0);
      const uint32_t cnt = first ? h0 : h1;
      const int hi = draw_hi(pass), lo = draw_lo(pass);
      S->below += before;
      S->prefix = (S->prefix << (hi - lo)) | (unsigned long long)dg;
      if (before + cnt == need || lo == 0) {
        S->t = lo == 0 ? S->prefix : ((S->prefix << lo) | ((1ull << lo) - 1ull));
        S->done = 1;
      }
    }
  }
  __syncthreads();
  V.hist[2 * tid] = 0u;
  V.hist[2 * tid + 1] = 0u;
}

// Every drawn changed voxel (hash <= t) queues the points within r_u of it;
// one CTA per touched brick, the pool indices of its 27 neighbours looked up
// once. r_u < 8 voxels, so the ball stays inside those bricks.
__global__ void __launch_bounds__(512) k_pts_scatter(MapView M, PtView V) {
  __shared__ uint32_t s_nb[27];
  const unsigned long long t = V.samp->t;
  const int R = V.trig_radius, R2 = R * R;
  const int l = threadIdx.x, lane = l & 31, wi = l >> 5;
  const int BX = M.dim_vox[0] >> 3, BY = M.dim_vox[1] >> 3, BZ = M.dim_vox[2] >> 3;
  const uint32_t nd = min(__ldcg(&M.ctl->dirty_count), V.C->nsnap);
  for (uint32_t d = blockIdx.x; d < nd; d += gridDim.x) {
    const uint32_t blk = M.dirty[d];
    const uint64_t key = M.bkey[blk];
    const int bx = (int)(key & 0x1FFFFF), by = (int)((key >> 21) & 0x1FFFFF), bz = (int)(key >> 42);
    __syncthreads();  // s_nb of the previous brick is no longer read
    if (l < 27) {
      const int x = bx + l % 3 - 1, y = by + (l / 3) % 3 - 1, z = bz + l / 9 - 1;
      s_nb[l] = ((unsigned)x < (unsigned)BX && (unsigned)y < (unsigned)BY && (unsigned)z < (unsigned)BZ)
                    ? lookup_brick(M, pack_brick(x, y, z))
                    : kNoBlock;
    }
    __syncthreads();
    if (!((V.chgmask[(size_t)d * 16 + wi] >> lane) & 1u)) continue;
    int x, y, z;
    brick_voxel(M, blk, l, &x, &y, &z);
    if (mix64(draw_key(M, x, y, z) ^ V.salt) > t) continue;
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          if (dx * dx + dy * dy + dz * dz > R2) continue;
          const int nx = x + dx, ny = y + dy, nz = z + dz;
          if (!box_rel(M, nx, ny, nz)) continue;
          const uint32_t b = s_nb[((nx >> 3) - bx + 1) + 3 * (((ny >> 3) - by + 1) + 3 * ((nz >> 3) - bz + 1))];
          if (b == kNoBlock) continue;
          const int32_t id = V.pid[(size_t)b * kBrickVox + vox_slot(nx, ny, nz)];
          if (id >= 0 && check_index((uint32_t)id < V.capacity, M.ctl)) V.st[id].queued = 1;
        }
  }
}

// New points: id = count + rank of the key among the frame's new keys.
__global__ void __launch_bounds__(256) k_pts_create(MapView M, PtView V) {
  __shared__ unsigned long long tile[256];
  const uint32_t nnew = V.C->nnew, base = V.C->count;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < nnew; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const unsigned long long key = i < nnew ? V.newkeys[i] : ~0ull;
    uint32_t rank = 0;
    for (uint32_t t0 = 0; t0 < nnew; t0 += 256) {
      __syncthreads();
      tile[threadIdx.x] = t0 + threadIdx.x < nnew ? V.newkeys[t0 + threadIdx.x] : ~0ull;
      __syncthreads();
      const uint32_t lim = min(256u, nnew - t0);
      for (uint32_t j = 0; j < lim; ++j) rank += tile[j] < key;
    }
    if (i >= nnew) continue;
    const int x = (int)(key & 0x1FFFFF), y = (int)((key >> 21) & 0x1FFFFF), z = (int)(key >> 42);
    const uint32_t blk = lookup_brick(M, pack_brick(x >> 3, y >> 3, z >> 3));
    if (blk == kNoBlock) continue;  // claimed in k_pts_mark, so present
    const uint32_t id = base + rank;
    int32_t* slot = V.pid + (size_t)blk * kBrickVox + vox_slot(x, y, z);
    if (id >= V.capacity) {  // the point set is full: the voxel stays free
      *slot = -1;
      latch_status(M.ctl, kStatusCapacity);
      continue;
    }
    *slot = (int32_t)id;
    PtState s;
    s.x = x;
    s.y = y;
    s.z = z;
    s.blk = blk;
    s.qsum[0] = s.qsum[1] = s.qsum[2] = 0.f;
    s.nobs = 0;
    s.last_scan = 0;
    s.last_tsdf = tsdf_word(__ldcg(M.vox + (size_t)blk * kBrickVox + vox_slot(x, y, z)), M.tau);
    s.a = 1.0f;
    s.n[0] = s.n[1] = s.n[2] = 0.f;
    s.score = -1;
    s.best = -1;
    s.queued = 1;
    s.label = 0;
    s.nviews = 0;
    s.pad = 0;
    V.st[id] = s;
  }
}

__global__ void k_pts_commit(PtView V) {
  V.C->count = min(V.C->count + V.C->nnew, V.capacity);
}

__global__ void __launch_bounds__(256) k_pts_views(MapView M, const float4* __restrict__ ret,
                                                   uint32_t n, PtView V, float q0, float q1,
                                                   float q2, uint32_t frame) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int r[3];
  if (!return_voxel(M, ret, k, r)) return;
  const uint32_t blk = lookup_brick(M, pack_brick(r[0] >> 3, r[1] >> 3, r[2] >> 3));
  if (blk == kNoBlock) return;
  const int32_t id = V.pid[(size_t)blk * kBrickVox + vox_slot(r[0], r[1], r[2])];
  if (id < 0 || !check_index((uint32_t)id < V.capacity, M.ctl)) return;
  PtState* s = V.st + id;
  if (atomicExch(&s->last_scan, frame) == frame) return;  // once per (point, scan)
  s->qsum[0] = __fadd_rn(s->qsum[0], q0);
  s->qsum[1] = __fadd_rn(s->qsum[1], q1);
  s->qsum[2] = __fadd_rn(s->qsum[2], q2);
  s->nobs += 1;
  const int nv = s->nviews;
  if (nv < V.max_views) {
    float4* vw = V.views + (size_t)id * 8;
    bool far = true;
    for (int j = 0; j < nv; ++j) {
      const float4 o = vw[j];
      const float d0 = __fsub_rn(q0, o.x), d1 = __fsub_rn(q1, o.y), d2 = __fsub_rn(q2, o.z);
      const float dd = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
      if (!(dd > V.view_min_dist2)) far = false;
    }
    if (far) {
      vw[nv] = make_float4(q0, q1, q2, 0.f);
      s->nviews = (uint8_t)(nv + 1);
    }
  }
}

__global__ void __launch_bounds__(256) k_pts_trigger(MapView M, PtView V, uint32_t frame, int moved) {
  const uint32_t count = V.C->count;
  for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < count; id += gridDim.x * blockDim.x) {
    PtState* s = V.st + id;
    const float cur = tsdf_word(__ldcg(M.vox + (size_t)s->blk * kBrickVox + vox_slot(s->x, s->y, s->z)), M.tau);
    bool q = s->queued != 0;
    if (fabsf(__fsub_rn(cur, s->last_tsdf)) > V.trig_tsdf) q = true;
    s->last_tsdf = cur;
    if (!V.trig_exact && V.near[s->blk] == frame) q = true;  // (ii) by the brick rule
    if (moved && s->label == 2) q = true;
    s->queued = q ? 1 : 0;
  }
}

// Selection of the first `budget` queued ids: per-block counts, one scan, scatter.
__global__ void __launch_bounds__(kSelBlock) k_pts_count(PtView V) {
  __shared__ uint32_t part[kSelBlock / 32];
  const uint32_t id = blockIdx.x * kSelBlock + threadIdx.x;
  const bool q = id < V.C->count && V.st[id].queued;
  const unsigned b = __ballot_sync(0xffffffffu, q);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = part[threadIdx.x];
    v = __reduce_add_sync(0xffffffffu, v);
    if (threadIdx.x == 0) V.blocksum[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(1024) k_pts_scan(PtView V, uint32_t nblocks, uint32_t budget) {
  // exclusive scan of the block counts, 1024 at a time
  __shared__ uint32_t buf[1024];
  uint32_t carry = 0;
  for (uint32_t b0 = 0; b0 < nblocks; b0 += 1024) {
    const uint32_t b = b0 + threadIdx.x;
    const uint32_t v = b < nblocks ? V.blocksum[b] : 0u;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {
      const uint32_t t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0u;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (b < nblocks) V.blocksum[b] = carry + buf[threadIdx.x] - v;
    const uint32_t total = buf[1023];
    __syncthreads();
    carry += total;
  }
  if (threadIdx.x == 0) {
    V.C->nsel = min(carry, budget);
    V.C->evals = 0;
  }
}

__global__ void __launch_bounds__(kSelBlock) k_pts_select(PtView V, uint32_t budget) {
  __shared__ uint32_t part[kSelBlock / 32];
  const uint32_t id = blockIdx.x * kSelBlock + threadIdx.x;
  const bool q = id < V.C->count && V.st[id].queued;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, q);
  if (lane == 0) part[wi] = __popc(b);
  __syncthreads();
  uint32_t before = 0;
  for (int j = 0; j < wi; ++j) before += part[j];
  const uint32_t rank = V.blocksum[blockIdx.x] + before + __popc(b & ((1u << lane) - 1u));
  if (q && rank < budget) V.sel[rank] = id;
}

// Candidate test of the layer: the normal filter and the observation-side
// filter (some stored viewpoint on the approach side, u . v > obs_dot).
struct NormalViewFilter {
  float n0, n1, n2;
  float v[8][3];
  int nv;
  float obs_dot;
  __device__ bool operator()(const ToolView& T, int g) const {
    if (!candidate(T, g, n0, n1, n2)) return false;
    const float u0 = __ldg(T.dirs + 3 * g), u1 = __ldg(T.dirs + 3 * g + 1),
                u2 = __ldg(T.dirs + 3 * g + 2);
    bool seen = false;
    for (int k = 0; k < nv; ++k)
      seen = seen || __fadd_rn(__fadd_rn(__fmul_rn(u0, v[k][0]), __fmul_rn(u1, v[k][1])),
                               __fmul_rn(u2, v[k][2])) > obs_dot;
    return seen;
  }
};

// Cyclic Jacobi on a symmetric 3 x 3 matrix; the eigenvector of the
// smallest diagonal element after the sweeps (lowest index on ties).
__device__ inline void jacobi_min(float a[3][3], float out[3]) {
  float v[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  for (int sw = 0; sw < kJacobiSweeps; ++sw)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int p = k == 2 ? 1 : 0, q = k == 0 ? 1 : 2, r = 3 - p - q;
      const float apq = a[p][q];
      if (apq == 0.0f) continue;
      const float theta = __fdiv_rn(__fsub_rn(a[q][q], a[p][p]), __fmul_rn(2.0f, apq));
      const float t = __fdiv_rn(theta >= 0.0f ? 1.0f : -1.0f,
                                __fadd_rn(fabsf(theta), __fsqrt_rn(__fadd_rn(__fmul_rn(theta, theta), 1.0f))));
      const float c = __fdiv_rn(1.0f, __fsqrt_rn(__fadd_rn(__fmul_rn(t, t), 1.0f)));
      const float s = __fmul_rn(t, c);
      const float app = __fsub_rn(a[p][p], __fmul_rn(t, apq));
      const float aqq = __fadd_rn(a[q][q], __fmul_rn(t, apq));
      const float arp = a[r][p], arq = a[r][q];
      const float nrp = __fsub_rn(__fmul_rn(c, arp), __fmul_rn(s, arq));
      const float nrq = __fadd_rn(__fmul_rn(s, arp), __fmul_rn(c, arq));
      a[p][p] = app;
      a[q][q] = aqq;
      a[p][q] = a[q][p] = 0.0f;
      a[r][p] = a[p][r] = nrp;
      a[r][q] = a[q][r] = nrq;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float vip = v[i][p], viq = v[i][q];
        v[i][p] = __fsub_rn(__fmul_rn(c, vip), __fmul_rn(s, viq));
        v[i][q] = __fadd_rn(__fmul_rn(s, vip), __fmul_rn(c, viq));
      }
    }
  int j = 0;
  for (int k = 1; k < 3; ++k)
    if (a[k][k] < a[j][j]) j = k;
  for (int i = 0; i < 3; ++i) out[i] = v[i][j];
}

// Stored best directions before a batch of evaluations (coarse-to-fine).
__global__ void __launch_bounds__(256) k_pts_snap(PtView V) {
  const uint32_t n = min(V.C->count, V.capacity);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    V.snap[i] = V.st[i].best;
}

// Coarse-to-fine direction subsets over a ring-ordered table.
struct CoarseFilter {
  const NormalViewFilter& F;
  int stride;
  __device__ bool operator()(const ToolView& T, int g) const {
    return g < T.G && g % stride == 0 && F(T, g);
  }
};
// The window around `centre`; with `coarse` also every stride-th direction,
// else without them (they were searched already).
struct WindowFilter {
  const NormalViewFilter& F;
  int centre, half, stride;
  bool coarse;
  __device__ bool operator()(const ToolView& T, int g) const {
    if (g >= T.G) return false;
    const int d = abs(g - centre);
    const bool in_coarse = g % stride == 0;
    return (min(d, T.G - d) <= half ? (coarse || !in_coarse) : (coarse && in_coarse)) && F(T, g);
  }
};

// Lowest-index minimum of two (score, index) results; index -1 = none.
__device__ inline int2 better(int2 a, int2 b) {
  if (b.y < 0) return a;
  if (a.y < 0) return b;
  return (b.x < a.x || (b.x == a.x && b.y < a.y)) ? b : a;
}

constexpr int kC2FTab = 729;  // bricks a ball of radius <= 31 voxels can span (9^3)
constexpr int kC2FNear = 64;  // ball offsets probed directly before the brick table

// Stored best direction (before the batch) of the nearest other point in
// the coarse-to-fine ball that had one; -1 if none. tb: this warp's table of
// the ball's bricks.
__device__ int nearest_resolved(const MapView& M, const PtView& V, const PtState& st, uint32_t* tb,
                                int lane) {
  // the nearest offsets first, one hash probe per lane: most points have a
  // resolved neighbour within a voxel or two
  const int near = min(V.c2f_noff, kC2FNear);
  for (int c0 = 0; c0 < near; c0 += 32) {
    const int j = c0 + lane;
    int16_t b = -1;
    if (j < near) {
      const int4 o = __ldg(V.c2foff + j);
      const int x = st.x + o.x, y = st.y + o.y, z = st.z + o.z;
      if (box_rel(M, x, y, z)) {
        const uint32_t bb = lookup_brick(M, pack_brick(x >> 3, y >> 3, z >> 3));
        if (bb != kNoBlock) {
          const int32_t id = __ldcg(V.pid + (size_t)bb * kBrickVox + vox_slot(x, y, z));
          if (id >= 0) b = __ldcg(V.snap + id);
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, b >= 0);
    if (bal) return __shfl_sync(0xffffffffu, (int)b, __ffs(bal) - 1);
  }
  if (near == V.c2f_noff) return -1;
  // the rest of the ball through a table of its bricks
  const int R = V.c2f_R;
  const int b0x = (st.x - R) >> 3, b0y = (st.y - R) >> 3, b0z = (st.z - R) >> 3;
  const int nx = ((st.x + R) >> 3) - b0x + 1, ny = ((st.y + R) >> 3) - b0y + 1,
            nz = ((st.z + R) >> 3) - b0z + 1;
  for (int k = lane; k < nx * ny * nz; k += 32) {
    const int bx = b0x + k % nx, by = b0y + (k / nx) % ny, bz = b0z + k / (nx * ny);
    uint32_t b = kNoBlock;
    if (bx >= 0 && by >= 0 && bz >= 0 && bx < (M.dim_vox[0] >> 3) && by < (M.dim_vox[1] >> 3) &&
        bz < (M.dim_vox[2] >> 3))
      b = lookup_brick(M, pack_brick(bx, by, bz));
    tb[k] = b;
  }
  __syncwarp();
  int res = -1;
  for (int c0 = near; c0 < V.c2f_noff; c0 += 32) {
    const int j = c0 + lane;
    int16_t b = -1;
    if (j < V.c2f_noff) {
      const int4 o = __ldg(V.c2foff + j);
      const int x = st.x + o.x, y = st.y + o.y, z = st.z + o.z;
      if (box_rel(M, x, y, z)) {
        const uint32_t bb = tb[((x >> 3) - b0x) + nx * (((y >> 3) - b0y) + ny * ((z >> 3) - b0z))];
        if (bb != kNoBlock) {
          const int32_t id = __ldcg(V.pid + (size_t)bb * kBrickVox + vox_slot(x, y, z));
          if (id >= 0) b = __ldcg(V.snap + id);
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, b >= 0);
    if (bal) {
      res = __shfl_sync(0xffffffffu, (int)b, __ffs(bal) - 1);
      break;
    }
  }
  __syncwarp();  // the table is rewritten for the warp's next point
  return res;
}

__global__ void __launch_bounds__(128) k_pts_eval(MapView M, ToolView T, PtView V) {
  __shared__ uint32_t s_c2f[4][kC2FTab];
  const int lane = threadIdx.x & 31;
  const uint32_t nsel = V.C->nsel;
  const uint32_t wstride = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nsel; i += wstride) {
    const uint32_t id = V.sel[i];
    PtState st = V.st[id];
    if (lane == 0) {
      V.st[id].queued = 0;
      atomicAdd(&V.C->evals, 1u);
    }
    // confidence gate, c = w / (w + k_c)
    const int l = vox_slot(st.x, st.y, st.z);
    const uint32_t w = (uint32_t)(__ldcg(M.vox + (size_t)st.blk * kBrickVox + l) & kWMask);
    const float c = __fdiv_rn((float)w, __fadd_rn((float)w, V.k_c));
    if (!(c >= V.c_min)) continue;

    // nearest neighbours: the sorted offsets, present points taken in order;
    // the cube spans at most two bricks per axis, looked up once by lanes 0-7
    const int R = V.nn_radius;
    const int b0x = (st.x - R) >> 3, b0y = (st.y - R) >> 3, b0z = (st.z - R) >> 3;
    uint32_t myb = kNoBlock;
    if (lane < 8) {
      const int bx = b0x + (lane & 1), by = b0y + ((lane >> 1) & 1), bz = b0z + ((lane >> 2) & 1);
      if (bx >= 0 && by >= 0 && bz >= 0 && bx < (M.dim_vox[0] >> 3) && by < (M.dim_vox[1] >> 3) &&
          bz < (M.dim_vox[2] >> 3))
        myb = lookup_brick(M, pack_brick(bx, by, bz));
    }
    int found = 0;
    int sx = 0, sy = 0, sz = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    for (int c0 = 0; c0 < V.noff && found < V.k_nn; c0 += 32) {
      const int j = c0 + lane;
      int4 o = make_int4(0, 0, 0, 0);
      bool in = false;
      int bi = 0, vl = 0;
      if (j < V.noff) {
        o = __ldg(V.nnoff + j);
        const int x = st.x + o.x, y = st.y + o.y, z = st.z + o.z;
        in = box_rel(M, x, y, z);
        bi = ((x >> 3) - b0x) | (((y >> 3) - b0y) << 1) | (((z >> 3) - b0z) << 2);
        vl = vox_slot(x, y, z);
      }
      const uint32_t bb = __shfl_sync(0xffffffffu, myb, in ? bi : 0);
      const bool present = in && bb != kNoBlock && __ldcg(V.pid + (size_t)bb * kBrickVox + vl) >= 0;
      const unsigned bal = __ballot_sync(0xffffffffu, present);
      const int take = min(__popc(bal), V.k_nn - found);
      const bool mine = present && __popc(bal & ((1u << lane) - 1u)) < take;
      if (mine) {
        sx += o.x;
        sy += o.y;
        sz += o.z;
        sxx += o.x * o.x;
        syy += o.y * o.y;
        szz += o.z * o.z;
        sxy += o.x * o.y;
        sxz += o.x * o.z;
        syz += o.y * o.z;
      }
      found += take;
    }
    if (found < 3) continue;
    sx = __reduce_add_sync(0xffffffffu, sx);
    sy = __reduce_add_sync(0xffffffffu, sy);
    sz = __reduce_add_sync(0xffffffffu, sz);
    sxx = __reduce_add_sync(0xffffffffu, sxx);
    syy = __reduce_add_sync(0xffffffffu, syy);
    szz = __reduce_add_sync(0xffffffffu, szz);
    sxy = __reduce_add_sync(0xffffffffu, sxy);
    sxz = __reduce_add_sync(0xffffffffu, sxz);
    syz = __reduce_add_sync(0xffffffffu, syz);
    // k sum d d^T - (sum d)(sum d)^T: exact integers, the same eigenvectors as the covariance
    const int kk = found;
    float a[3][3];
    a[0][0] = (float)(kk * sxx - sx * sx);
    a[1][1] = (float)(kk * syy - sy * sy);
    a[2][2] = (float)(kk * szz - sz * sz);
    a[0][1] = a[1][0] = (float)(kk * sxy - sx * sy);
    a[0][2] = a[2][0] = (float)(kk * sxz - sx * sz);
    a[1][2] = a[2][1] = (float)(kk * syz - sy * sz);
    float nrm[3];
    jacobi_min(a, nrm);
    // face the mean historical sensor position
    const float s0 = voxel_centre(st.x + M.dom_vox[0], M.v), s1 = voxel_centre(st.y + M.dom_vox[1], M.v),
                s2 = voxel_centre(st.z + M.dom_vox[2], M.v);
    const float fn = (float)st.nobs;
    const float d0 = __fsub_rn(__fdiv_rn(st.qsum[0], fn), s0), d1 = __fsub_rn(__fdiv_rn(st.qsum[1], fn), s1),
                d2 = __fsub_rn(__fdiv_rn(st.qsum[2], fn), s2);
    const float nd = __fadd_rn(__fadd_rn(__fmul_rn(nrm[0], d0), __fmul_rn(nrm[1], d1)), __fmul_rn(nrm[2], d2));
    if (nd < 0.0f) {
      nrm[0] = -nrm[0];
      nrm[1] = -nrm[1];
      nrm[2] = -nrm[2];
    }
    // unit vectors toward the stored viewpoints
    NormalViewFilter F;
    F.n0 = nrm[0];
    F.n1 = nrm[1];
    F.n2 = nrm[2];
    F.nv = st.nviews;
    F.obs_dot = V.obs_dot;
    for (int k = 0; k < F.nv; ++k) {
      const float4 q = V.views[(size_t)id * 8 + k];
      const float e0 = __fsub_rn(q.x, s0), e1 = __fsub_rn(q.y, s1), e2 = __fsub_rn(q.z, s2);
      const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2)));
      F.v[k][0] = __fdiv_rn(e0, len);
      F.v[k][1] = __fdiv_rn(e1, len);
      F.v[k][2] = __fdiv_rn(e2, len);
    }
    // the plain path's exact search with the layer's candidate test
    Pt P;
    P.px = st.x;
    P.py = st.y;
    P.pz = st.z;
    const bool fast = P.px >= T.reach[0] && P.px + T.reach[0] < M.dim_vox[0] &&
                      P.py >= T.reach[1] && P.py + T.reach[1] < M.dim_vox[1] &&
                      P.pz >= T.reach[2] && P.pz + T.reach[2] < M.dim_vox[2];
    int2 res;
    if (fast) set_rows(M, P); else P.row = P.rowy = P.rowz = 0;
    if (V.c2f_stride == 0) {
      res = fast ? best_direction<true>(M, T, P, F, lane) : best_direction<false>(M, T, P, F, lane);
    } else {
      // coarse set, then the window around the nearest resolved neighbour's
      // direction (else around the coarse best); lowest-index minimum of both
      const int nb = nearest_resolved(M, V, st, s_c2f[threadIdx.x >> 5], lane);
      if (nb >= 0) {  // one pass over the coarse set and the neighbour's window
        const WindowFilter Fu{F, nb, V.c2f_half, V.c2f_stride, true};
        res = fast ? best_direction<true>(M, T, P, Fu, lane) : best_direction<false>(M, T, P, Fu, lane);
      } else {  // the coarse set, then the window around its best
        const CoarseFilter Fc{F, V.c2f_stride};
        res = fast ? best_direction<true>(M, T, P, Fc, lane) : best_direction<false>(M, T, P, Fc, lane);
        if (res.y >= 0) {
          const WindowFilter Fw{F, res.y, V.c2f_half, V.c2f_stride, false};
          res = better(res, fast ? best_direction<true>(M, T, P, Fw, lane)
                                 : best_direction<false>(M, T, P, Fw, lane));
        }
      }
    }
    const int nc = T.n_c;
    const int sc = res.y >= 0 ? res.x : nc + 1;
    const int g = res.y;
    if (lane == 0) {
      // the stored score only decreases; a on conflict / confirmation
      const bool prev_acc = st.score >= 0 && st.score < nc;
      if (st.score < 0 || sc < st.score) {
        st.score = (int16_t)sc;
        st.best = (int16_t)g;
      }
      if (prev_acc && sc >= nc)
        st.a = __fmul_rn(V.a_decay, st.a);
      else if (sc < nc)
        st.a = __fadd_rn(st.a, __fmul_rn(V.a_recover, __fsub_rn(1.0f, st.a)));
      st.label = (st.score < nc && __fmul_rn(c, st.a) > V.ca_min) ? 1 : 2;
      st.n[0] = nrm[0];
      st.n[1] = nrm[1];
      st.n[2] = nrm[2];
      st.queued = 0;
      PtState* d = V.st + id;
      d->score = st.score;
      d->best = st.best;
      d->a = st.a;
      d->label = st.label;
      d->n[0] = st.n[0];
      d->n[1] = st.n[1];
      d->n[2] = st.n[2];
      atomicAdd(&M.ctl->points_scored, 1ull);
    }
  }
}

unsigned grid_cap(size_t n, int threads, int num_sms, int per_sm) {
  const size_t want = (n + threads - 1) / threads;
  const size_t cap = (size_t)num_sms * per_sm;
  return (unsigned)std::max<size_t>(1, std::min(want, cap));
}

af_status pfail(af_ctx* c, af_status s, const char* fmt, ...) {
  if (!c) return s;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof c->err, fmt, ap);
  va_end(ap);
  return s;
}

#define PT_CUDA(ctx, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return af::pfail((ctx), AF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

PtView pt_view(af_ctx* ctx) {
  PtView V;
  const af_points_config& c = ctx->pcfg;
  V.st = ctx->d_pst;
  V.views = ctx->d_pviews;
  V.pid = ctx->d_pid;
  V.newkeys = ctx->d_pnew;
  V.near = ctx->d_pnear;
  V.snapw = ctx->d_psnapw;
  V.snapc = ctx->d_psnapc;
  V.chgmask = ctx->d_pchgmask;
  V.hist = ctx->d_phist;
  V.samp = ctx->d_psamp;
  V.trig_exact = c.trig_exact;
  V.trig_radius = c.trig_radius;
  V.trig_sample = c.trig_sample;
  V.salt = mix64((uint64_t)ctx->pts_frames);
  V.sel = ctx->d_psel;
  V.blocksum = ctx->d_pblock;
  V.C = ctx->d_pcount;
  V.nnoff = ctx->d_pnnoff;
  V.noff = ctx->pnoff;
  V.capacity = c.capacity;
  V.k_nn = (int)c.k_nn;
  V.nn_radius = c.nn_radius;
  V.max_views = (int)c.max_views;
  V.view_min_dist2 = c.view_min_dist * c.view_min_dist;
  V.obs_dot = c.obs_dot;
  V.trig_tsdf = c.trig_tsdf;
  V.k_c = c.k_c;
  V.c_min = c.c_min;
  V.a_decay = c.a_decay;
  V.a_recover = c.a_recover;
  V.ca_min = c.ca_min;
  V.c2f_stride = (int)c.c2f_stride;
  V.c2f_half = (int)c.c2f_half;
  V.c2f_R = ctx->pc2f_R;
  V.c2foff = ctx->d_pc2f;
  V.c2f_noff = ctx->pc2f_noff;
  V.snap = ctx->d_psnap;
  return V;
}

af_status select_and_eval(af_ctx* ctx, uint32_t budget, cudaStream_t s) {
  const PtView V = pt_view(ctx);
  const uint32_t nblocks = (ctx->pcfg.capacity + kSelBlock - 1) / kSelBlock;
  k_pts_count<<<nblocks, kSelBlock, 0, s>>>(V);
  k_pts_scan<<<1, 1024, 0, s>>>(V, nblocks, budget);
  k_pts_select<<<nblocks, kSelBlock, 0, s>>>(V, budget);
  if (V.c2f_stride > 0) k_pts_snap<<<grid_cap(ctx->pcfg.capacity, 256, ctx->num_sms, 8), 256, 0, s>>>(V);
  k_pts_eval<<<(unsigned)ctx->num_sms * 8, 128, 0, s>>>(ctx->M, ctx->T, V);
  PT_CUDA(ctx, cudaGetLastError());
  return AF_OK;
}

}  // namespace

cudaError_t launch_pts_snapshot(af_ctx* ctx, cudaStream_t s) {
  k_pts_snapshot<<<(unsigned)ctx->num_sms * 4, 512, 0, s>>>(ctx->M, pt_view(ctx));
  return cudaGetLastError();
}

}  // namespace af

using af::MapView;

extern "C" af_status af_points_enable(af_ctx* ctx, const af_points_config* cfg) {
  if (!ctx || !cfg) return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_enable: NULL argument");
  if (ctx->pts_on) return af::pfail(ctx, AF_ERR_STATE, "af_points_enable: already enabled");
  const af_points_config& c = *cfg;
  const float f[10] = {c.view_min_dist, c.obs_dot, c.trig_tsdf, c.trig_move, c.k_c,
                       c.c_min,        c.a_decay, c.a_recover, c.ca_min, 0.f};
  for (float x : f)
    if (!std::isfinite(x)) return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_enable: non-finite parameter");
  if (c.capacity < 1 || c.capacity > (1u << 30) || c.k_nn < 3 || c.k_nn > 343 || c.nn_radius < 1 ||
      c.nn_radius > 3 || c.max_views > 8 || !(c.k_c > 0.f) || c.view_min_dist < 0.f ||
      (c.trig_exact != 0 && c.trig_exact != 1) || c.trig_radius < 0 || c.trig_radius > 7 ||
      c.trig_sample > (1u << 24))
    return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_enable: parameter out of range");
  // coarse-to-fine ball: offsets o != 0 with |o|^2 v^2 <= radius^2 in double
  std::vector<int4> ball;
  int c2fR = 0;
  if (c.c2f_stride > 0) {
    const double v = (double)ctx->cfg.voxel_size, r = (double)c.c2f_radius;
    if (!(c.c2f_radius > 0.f) || !std::isfinite(c.c2f_radius) || r / v >= 32.0 || c.c2f_half > 4096)
      return af::pfail(ctx, AF_ERR_INVALID_ARG,
                       "af_points_enable: coarse-to-fine radius must be in (0, 32 v), half <= 4096");
    const int Rb = (int)(r / v) + 1;
    for (int z = -Rb; z <= Rb; ++z)
      for (int y = -Rb; y <= Rb; ++y)
        for (int x = -Rb; x <= Rb; ++x) {
          const int d2 = x * x + y * y + z * z;
          if (d2 == 0 || (double)d2 * v * v > r * r) continue;
          ball.push_back(make_int4(x, y, z, d2));
          c2fR = std::max(c2fR, std::max(std::abs(x), std::max(std::abs(y), std::abs(z))));
        }
    std::sort(ball.begin(), ball.end(), [](const int4& a, const int4& b) {
      if (a.w != b.w) return a.w < b.w;
      if (a.z != b.z) return a.z < b.z;
      if (a.y != b.y) return a.y < b.y;
      return a.x < b.x;
    });
    if (c2fR > 31)
      return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_enable: coarse-to-fine ball beyond 31 voxels");
  }
  ctx->pcfg = c;
  const size_t B = ctx->cfg.pool_blocks, P = c.capacity, R = ctx->cfg.max_returns;
  const size_t nblocks = (P + 1023) / 1024;
  auto alloc = [&](void** p, size_t bytes, int fill) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) e = cudaMemset(*p, fill, bytes ? bytes : 16);
    return e;
  };
  cudaError_t e = alloc((void**)&ctx->d_pid, B * af::kBrickVox * 4, 0xFF);
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_pst, P * sizeof(af::PtState), 0);
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_pviews, P * 8 * sizeof(float4), 0);
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_pnew, R * 8, 0);
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_pnear, B * 4, 0);
  if (c.trig_exact) {  // the dirty list holds at most every pool brick
    if (e == cudaSuccess) e = alloc((void**)&ctx->d_psnapw, B * af::kBrickVox * 8, 0);
    if (e == cudaSuccess) e = alloc((void**)&ctx->d_psnapc, B * 16 * 4, 0);
    if (e == cudaSuccess) e = alloc((void**)&ctx->d_pchgmask, B * 16 * 4, 0);
    if (e == cudaSuccess) e = alloc((void**)&ctx->d_phist, af::kDrawBins * 4, 0);
    if (e == cudaSuccess) e = alloc((void**)&ctx->d_psamp, sizeof(af::PtSample), 0);
  }
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_psel, P * 4, 0);
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_pblock, nblocks * 4, 0);
  if (e == cudaSuccess) e = alloc((void**)&ctx->d_pcount, sizeof(af::PtCounters), 0);
  // neighbour offsets, nearest first, ties in (dz, dy, dx) order
  std::vector<int4> off;
  const int Rr = c.nn_radius;
  for (int z = -Rr; z <= Rr; ++z)
    for (int y = -Rr; y <= Rr; ++y)
      for (int x = -Rr; x <= Rr; ++x) off.push_back(make_int4(x, y, z, x * x + y * y + z * z));
  std::sort(off.begin(), off.end(), [](const int4& a, const int4& b) {
    if (a.w != b.w) return a.w < b.w;
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_pnnoff, off.size() * sizeof(int4));
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->d_pnnoff, off.data(), off.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !ball.empty()) {
    e = cudaMalloc((void**)&ctx->d_pc2f, ball.size() * sizeof(int4));
    if (e == cudaSuccess)
      e = cudaMemcpy(ctx->d_pc2f, ball.data(), ball.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = alloc((void**)&ctx->d_psnap, P * sizeof(int16_t), 0xFF);
  }
  if (e != cudaSuccess)
    return af::pfail(ctx, AF_ERR_CUDA, "af_points_enable: allocation failed: %s", cudaGetErrorString(e));
  ctx->pc2f_noff = (int)ball.size();
  ctx->pc2f_R = c2fR;
  ctx->pnoff = (int)off.size();
  ctx->pts_on = true;
  ctx->have_q_last = false;
  return AF_OK;
}

extern "C" af_status af_points_frame(af_ctx* ctx, const float* d_xyz, uint32_t n,
                                     const float pose[16], void* stream) {
  if (!ctx) return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_frame: NULL context");
  if (!ctx->pts_on) return af::pfail(ctx, AF_ERR_STATE, "af_points_frame: call af_points_enable first");
  if (!ctx->has_tool) return af::pfail(ctx, AF_ERR_STATE, "af_points_frame: call af_set_tool first");
  const bool exact = ctx->pcfg.trig_exact != 0;
  ctx->pts_snapshot = exact;
  af_status st = af_integrate_scan(ctx, d_xyz, n, pose, stream);
  ctx->pts_snapshot = false;
  if (st != AF_OK) return st;
  ctx->pts_frames += 1;
  cudaStream_t s = (cudaStream_t)stream;
  const MapView& M = ctx->M;
  const af::PtView V = af::pt_view(ctx);
  const uint32_t frame = ctx->frame;
  PT_CUDA(ctx, cudaMemsetAsync(&ctx->d_pcount->nnew, 0, 2 * sizeof(uint32_t), s));  // nnew, nchanged
  if (n > 0) af::k_pts_mark<<<(n + 255) / 256, 256, 0, s>>>(M, ctx->d_ret, n, V);
  if (!exact)
    af::k_pts_near<<<af::grid_cap((size_t)M.pool_blocks * 27, 256, ctx->num_sms, 8), 256, 0, s>>>(M, V, frame);
  af::k_pts_create<<<af::grid_cap(ctx->cfg.max_returns, 256, ctx->num_sms, 8), 256, 0, s>>>(M, V);
  af::k_pts_commit<<<1, 1, 0, s>>>(V);
  const float q[3] = {pose[3], pose[7], pose[11]};
  if (n > 0) af::k_pts_views<<<(n + 255) / 256, 256, 0, s>>>(M, ctx->d_ret, n, V, q[0], q[1], q[2], frame);
  if (exact) {  // trigger (ii): the changed voxels, their draw, the points near the drawn ones
    const unsigned grid = (unsigned)ctx->num_sms * 4;
    PT_CUDA(ctx, cudaMemsetAsync(ctx->d_psamp, 0, sizeof(af::PtSample), s));
    af::k_pts_diff<<<grid, 512, 0, s>>>(M, V);
    for (int pass = 0; pass < af::kDrawPasses; ++pass) {
      af::k_pts_hist<<<grid, 512, 0, s>>>(M, V, pass);
      af::k_pts_pick<<<1, 1024, 0, s>>>(V, pass);
    }
    af::k_pts_scatter<<<grid, 512, 0, s>>>(M, V);
  }
  // sensor motion since the motion trigger last fired
  int moved = 0;
  if (ctx->have_q_last) {
    const float d[3] = {q[0] - ctx->q_last[0], q[1] - ctx->q_last[1], q[2] - ctx->q_last[2]};
    const float dd = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    if (dd > ctx->pcfg.trig_move * ctx->pcfg.trig_move) {
      moved = 1;
      std::memcpy(ctx->q_last, q, sizeof q);
    }
  } else {
    std::memcpy(ctx->q_last, q, sizeof q);
    ctx->have_q_last = true;
  }
  af::k_pts_trigger<<<af::grid_cap(ctx->pcfg.capacity, 256, ctx->num_sms, 8), 256, 0, s>>>(M, V, frame, moved);
  PT_CUDA(ctx, cudaGetLastError());
  return af::select_and_eval(ctx, ctx->pcfg.budget, s);
}

extern "C" af_status af_points_drain(af_ctx* ctx, uint32_t max_evals, void* stream) {
  if (!ctx) return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_drain: NULL context");
  if (!ctx->pts_on) return af::pfail(ctx, AF_ERR_STATE, "af_points_drain: call af_points_enable first");
  if (!ctx->has_tool) return af::pfail(ctx, AF_ERR_STATE, "af_points_drain: call af_set_tool first");
  return af::select_and_eval(ctx, max_evals, (cudaStream_t)stream);
}

extern "C" af_status af_points_stats(af_ctx* ctx, uint32_t* count, uint32_t* last_evals) {
  if (!ctx || !count || !last_evals) return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_stats: NULL argument");
  if (!ctx->pts_on) return af::pfail(ctx, AF_ERR_STATE, "af_points_stats: call af_points_enable first");
  af::PtCounters h;
  PT_CUDA(ctx, cudaDeviceSynchronize());
  PT_CUDA(ctx, cudaMemcpy(&h, ctx->d_pcount, sizeof h, cudaMemcpyDeviceToHost));
  *count = h.count;
  *last_evals = h.evals;
  return AF_OK;
}

extern "C" af_status af_points_export(af_ctx* ctx, uint32_t cap, int32_t* h_ijk, float* h_normal,
                                      uint8_t* h_label, int16_t* h_score, int16_t* h_best,
                                      float* h_a, uint8_t* h_queued, int32_t* h_nviews,
                                      uint32_t* out_count) {
  uint32_t count = 0, ev = 0;
  af_status st = af_points_stats(ctx, &count, &ev);
  if (st != AF_OK) return st;
  if (!out_count) return af::pfail(ctx, AF_ERR_INVALID_ARG, "af_points_export: NULL count");
  count = std::min(count, cap);
  *out_count = count;
  if (count == 0) return AF_OK;
  std::vector<af::PtState> p(count);
  PT_CUDA(ctx, cudaMemcpy(p.data(), ctx->d_pst, count * sizeof(af::PtState), cudaMemcpyDeviceToHost));
  for (uint32_t i = 0; i < count; ++i) {
    const af::PtState& s = p[i];
    if (h_ijk) {
      h_ijk[3 * i] = s.x + ctx->M.dom_vox[0];
      h_ijk[3 * i + 1] = s.y + ctx->M.dom_vox[1];
      h_ijk[3 * i + 2] = s.z + ctx->M.dom_vox[2];
    }
    if (h_normal)
      for (int k = 0; k < 3; ++k) h_normal[3 * i + k] = s.n[k];
    if (h_label) h_label[i] = s.label;
    if (h_score) h_score[i] = s.score;
    if (h_best) h_best[i] = s.best;
    if (h_a) h_a[i] = s.a;
    if (h_queued) h_queued[i] = s.queued;
    if (h_nviews) h_nviews[i] = s.nviews;
  }
  return AF_OK;
}
