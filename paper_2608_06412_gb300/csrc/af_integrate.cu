// af_integrate.cu -- scan-centric TSDF integration on sm_103a (Sec. 3.2, 3.4,
// 3.6 of the paper), three launches per scan:
//
//  k_alloc     one thread per (return, brick key): pose transform, validity,
//              voxel index; inserts the bricks of the return's (2m+1)^3 cube
//              and of its ray-cleared band samples into the hash. Lanes of a
//              warp that carry the same key are merged with __match_any_sync,
//              so one probe per distinct key per warp reaches L2. The pool
//              index of each cube brick goes into a per-return brick table,
//              and the brick is marked dirty.
//  k_integrate one CTA per tile of 8 returns, one thread per cube offset: the
//              tile's brick tables are loaded once (bricks created by this
//              scan are looked up here), and the per-axis terms of every
//              return's sums (squares, products, brick / slot codes) are
//              computed once into shared memory; then each thread walks the
//              tile's returns for its offset, computes d and adds
//              (round(d 2^20) << 20) | 1 to the voxel word with one 64-bit
//              atomic; integer addition makes the result order-independent.
//              The cleared-band marks follow, off the barrier path.
//  k_bitview   persistent over the scan's dirty bricks: weight cap with
//              proportional rescale, then occupied / known bits packed with
//              __ballot_sync into the dense bit planes.
//
// Every floating-point operation that decides an integer is an explicitly
// rounded IEEE single-precision operation, in the order the method states
// it, so the result is reproducible bit for bit on any IEEE machine; where a
// cheaper approximate value is used, it only takes decisions that the exact
// value is certain to agree with (margins of 2^-16).

#include "af_internal.cuh"

namespace af {

// Inserts a brick key (bounded probe) and returns its pool index: the index
// this thread took if it inserted the key, the stored index if the key was
// already there, or kNoBlock if another thread of this launch is inserting it
// right now (or the pool is full).
// *slot receives the slot index and *stamp the slot's scan stamp as read.
__device__ uint32_t insert_brick(const MapView& M, uint64_t key, uint32_t* slot,
                                 uint32_t* stamp) {
  uint32_t h = hash_slot(key, M.hmask);
  for (uint32_t probe = 0; probe <= M.hmask; ++probe) {
    unsigned long long k;
    uint32_t val;
    load_slot(M, h, &k, &val, stamp);
    if (k == kEmptyKey) {
      k = atomicCAS(&M.slots[h].key, kEmptyKey, key);
      if (k == kEmptyKey) {
        *slot = h;
        const uint32_t idx = atomicAdd(&M.ctl->pool_count, 1u);
        if (idx < M.pool_blocks) {
          M.bkey[idx] = key;
          M.slots[h].val = idx;
          return idx;
        }
        latch_status(M.ctl, kStatusCapacity);
        return kNoBlock;
      }
      val = kNoBlock;  // another thread is filling this slot right now
    }
    if (k == key) {
      *slot = h;
      return val < M.pool_blocks ? val : kNoBlock;
    }
    h = (h + 1) & M.hmask;
  }
  latch_status(M.ctl, kStatusCapacity);
  return kNoBlock;
}

// Appends blk (hash slot h, whose stamp was read as `seen`) to the scan's
// dirty list once per scan: the stamp decides which thread appends. Appends
// are aggregated over the threads of the same map (`group`) that call
// together: one counter atomic per map and call instead of one per brick.
// Threads of different maps may call together (batched ticks, MULTI), and
// each map's appends go through its own counter; without MULTI every calling
// thread belongs to the same map.
template <bool MULTI>
__device__ inline void mark_dirty(const MapView& M, uint32_t h, uint32_t blk, uint32_t frame,
                                  uint32_t seen, uint32_t group) {
  const unsigned active = __activemask();
  const unsigned same = MULTI ? __match_any_sync(active, group) : active;
  const bool need = seen != frame && atomicExch(&M.slots[h].stamp, frame) != frame;
  const unsigned nm = __ballot_sync(active, need) & same;
  const int lane = threadIdx.x & 31;
  const int first = nm ? __ffs(nm) - 1 : lane;
  uint32_t base = 0;
  if (nm && lane == first) base = atomicAdd(&M.ctl->dirty_count, (unsigned)__popc(nm));
  base = __shfl_sync(active, base, first);
  const uint32_t at = base + __popc(nm & ((1u << lane) - 1u));
  if (need && check_index(at < M.pool_blocks, M.ctl)) M.dirty[at] = blk;
}

// Cube bricks of a return: first brick b0 and count nb per axis.
__device__ inline void cube_bricks(const MapView& M, const int rel[3], int b0[3], int nb[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b0[a] = (rel[a] - M.m) >> 3;
    nb[a] = ((rel[a] + M.m) >> 3) - b0[a] + 1;
  }
}

// One thread per (return, brick key): key slots [0, nbmax) are the bricks of
// the return's cube, slots [nbmax, nbmax + N_s) its cleared-band samples. The
// pose transform is recomputed by every thread of a return (cheap next to an
// L2 probe); slot 0 also writes the return's world position for k_integrate.
// All 32 lanes of the warp call this together; `group` tells lanes of
// different maps apart (MULTI; without it every lane is of one map), `e` is
// the thread's slot index within its map's scan (slots past the scan are
// inactive).
template <bool MULTI>
__device__ void alloc_slot(const MapView& M, const float* __restrict__ xyz, uint32_t n,
                           const Pose& P, float4* __restrict__ ret, uint32_t frame, uint32_t e,
                           uint32_t group) {
  const int nbmax = M.nbmax;
  const int per = nbmax + M.ns;
  const uint32_t k = e / per;
  const int j = (int)(e % per);
  const int lane = threadIdx.x & 31;

  float p[3] = {0.f, 0.f, 0.f}, range = 0.f;
  int rel[3] = {0, 0, 0};
  bool valid = false;
  if (k < n) {
    valid = prepare_return(M, P, xyz[3 * k], xyz[3 * k + 1], xyz[3 * k + 2], p, &range, rel);
    if (j == 0) ret[k] = make_float4(p[0], p[1], p[2], valid ? 1.f : 0.f);
  }
  const unsigned same_map = MULTI ? __match_any_sync(0xffffffffu, group) : 0xffffffffu;
  const unsigned acc = __ballot_sync(0xffffffffu, valid && j == 0) & same_map;
  if (lane == __ffs(same_map) - 1 && acc)
    atomicAdd(&M.ctl->returns_accepted, (unsigned long long)__popc(acc));

  uint64_t key = kEmptyKey;
  bool cube_slot = false;
  if (valid) {
    int b0[3], nb[3];
    cube_bricks(M, rel, b0, nb);
    if (j < nbmax) {
      // table layout shared with k_integrate: slot j = bx + BA (by + BA bz)
      const int ba = (2 * M.m + 7) / 8 + 1;
      const int bx = j % ba, by = (j / ba) % ba, bz = j / (ba * ba);
      if (bx < nb[0] && by < nb[1] && bz < nb[2]) {
        key = pack_brick(b0[0] + bx, b0[1] + by, b0[2] + bz);
        cube_slot = true;
      }
    } else {
      const float q[3] = {P.r[0][3], P.r[1][3], P.r[2][3]};
      int sv[3];
      if (band_sample(M, p, q, range, j - nbmax + 1, sv)) {
        const int sb[3] = {sv[0] >> 3, sv[1] >> 3, sv[2] >> 3};
        // bricks of the cube are inserted by the cube slots
        const bool in_cube = sb[0] >= b0[0] && sb[0] - b0[0] < nb[0] && sb[1] >= b0[1] &&
                             sb[1] - b0[1] < nb[1] && sb[2] >= b0[2] && sb[2] - b0[2] < nb[2];
        if (!in_cube) key = pack_brick(sb[0], sb[1], sb[2]);
      }
    }
  }
  const bool ins = key != kEmptyKey;
  const unsigned act = __ballot_sync(0xffffffffu, ins);
  uint32_t blk = kNoBlock;
  if (ins) {
    const unsigned peers =
        __match_any_sync(act, key) & (MULTI ? __match_any_sync(act, group) : act);
    const int leader = __ffs(peers) - 1;
    if (lane == leader) {
      uint32_t h, seen;
      blk = insert_brick(M, key, &h, &seen);
      if (blk != kNoBlock) mark_dirty<MULTI>(M, h, blk, frame, seen, group);
    }
    blk = __shfl_sync(peers, blk, leader);
  }
  // kNoBlock: created by another thread of this launch, resolved (and marked
  // dirty) in k_integrate
  if (k < n && j < nbmax) M.rtab[(size_t)k * nbmax + j] = cube_slot ? blk : kUnused;
}

__global__ void __launch_bounds__(256) k_alloc(MapView M, const float* __restrict__ xyz,
                                                uint32_t n, Pose P, float4* __restrict__ ret,
                                                uint32_t frame) {
  alloc_slot<false>(M, xyz, n, P, ret, frame, blockIdx.x * blockDim.x + threadIdx.x, 0u);
}

// Approximate square root (MUFU reciprocal square root), relative error well
// below 2^-20 for the normal arguments it is used on. Only ever used to take
// a decision that the exact result is certain to agree with (margins of
// 2^-16 relative); near any threshold the exact IEEE operation decides.
__device__ inline float sqrt_approx(float x) { return x * rsqrtf(x); }

constexpr float kMargin = 1.52587890625e-05f;  // 2^-16

// The exact cone decision, RN(dot / RN(RN(sqrt(aa)) range)) > cone, out of
// line: it runs only within 2^-16 of the threshold, so divergent lanes call it
// instead of every lane carrying its instructions.
__device__ __noinline__ bool cone_excludes_exact(float dot, float aa, float range, float cone) {
  return __fdiv_rn(dot, __fmul_rn(__fsqrt_rn(aa), range)) > cone;
}

template <int W>
struct CubeShape {
  static constexpr int C = W * W * W;                                 // offsets
  static constexpr int NT = ((C + 31) / 32) * 32 <= 1024 ? ((C + 31) / 32) * 32 : 1024;
  static constexpr int OPT = (C + NT - 1) / NT;                       // offsets per thread
  static constexpr int BA = (W + 6) / 8 + 1;                          // bricks per edge
  static constexpr int NB = BA * BA * BA;
  static constexpr int MR = W / 2;
};

// A tile of one scan: returns [r0, r1), r1 - r0 <= T; called by the whole
// CTA of CubeShape<W>::NT threads. W = 2m + 1 voxels per cube edge.
template <int W, int T>
__device__ void integrate_tile(const MapView& M, const float4* __restrict__ ret, uint32_t r0,
                               uint32_t r1, float q0, float q1, float q2, uint32_t frame) {
  using S = CubeShape<W>;
  constexpr int C = S::C, NT = S::NT, OPT = S::OPT, BA = S::BA, NB = S::NB, MR = S::MR;
  __shared__ float4 s_p[T];        // p, valid flag
  // what the pair loop reads of a return, in one record: range |p - q|,
  // RN(|p - q|^2), RN(1 / range) (for the approximate cone test), valid flag
  __shared__ float4 s_pr[T];
  __shared__ uint32_t s_blk[T][NB];
  // Per return, axis and cube offset k (voxel rel + k - MR on that axis),
  // the rounded per-axis terms of the three sums the arithmetic needs --
  // (x - p)^2, (x - p)(p - q), (x - q)^2 -- and the brick / voxel-slot code
  // of that coordinate (as float bits), one 16-byte record: a pair then adds
  // three terms per sum in the order written (x, y, z), so every rounding is
  // the same as computing it whole.
  __shared__ float4 s_term[T][3][W];

  // A latched error (sticky capacity error) skips the scan. Another CTA may
  // latch one while this CTA runs, so the whole CTA decides together; the
  // barrier also keeps a previous tile of this CTA from still reading the
  // tables.
  if (__syncthreads_or(__ldcg(&M.ctl->status) != 0u)) return;
  const int tid = threadIdx.x;
  const float q[3] = {q0, q1, q2};

  if (tid < T) {
    const uint32_t k = r0 + tid;
    float4 p = k < r1 ? ret[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    float bb = 0.f, range = 0.f, ir = 0.f;
    if (p.w != 0.f) {
      const float b[3] = {__fsub_rn(p.x, q0), __fsub_rn(p.y, q1), __fsub_rn(p.z, q2)};
      bb = __fadd_rn(__fadd_rn(__fmul_rn(b[0], b[0]), __fmul_rn(b[1], b[1])), __fmul_rn(b[2], b[2]));
      range = __fsqrt_rn(bb);
      ir = __frcp_rn(range);
    }
    s_p[tid] = p;
    s_pr[tid] = make_float4(range, bb, ir, p.w);
  }
  // Per-axis terms of every (return, axis, offset), each thread from the
  // return itself (no barrier between the per-return and per-axis steps).
  const float v = M.v, tau = M.tau, cone = M.cone_cos;
  for (int e = tid; e < T * 3 * W; e += NT) {
    const int t = e / (3 * W), ax = (e / W) % 3, k = e % W;
    if (r0 + t >= r1) continue;
    const float4 p = ret[r0 + t];
    if (p.w == 0.f) continue;
    const float pa = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
    int i;
    voxel_index(pa, M, &i);
    const int rel = i - M.dom_vox[ax];                 // box-relative voxel of p on this axis
    const int j = rel + k - MR;                        // ... of the cube voxel
    const float x = voxel_centre(j + M.dom_vox[ax], v);
    const float a = __fsub_rn(x, pa), b = __fsub_rn(pa, q[ax]), c = __fsub_rn(x, q[ax]);
    // brick offset within the tile's brick table (weight 1, BA, BA^2) in the
    // high half, the voxel's slot bits within its brick in the low half
    const int bk = (j >> 3) - ((rel - MR) >> 3);
    const int code = ((bk * (ax == 0 ? 1 : (ax == 1 ? BA : BA * BA))) << 16) | ((j & 7) << (3 * ax));
    s_term[t][ax][k] = make_float4(__fmul_rn(a, a), __fmul_rn(a, b), __fmul_rn(c, c),
                                   __int_as_float(code));
  }
  // The tile's brick tables; bricks created by this scan are looked up now.
  for (int e = tid; e < T * NB; e += NT) {
    const int t = e / NB, j = e % NB;
    const uint32_t k = r0 + t;
    uint32_t blk = kUnused;
    if (k < r1) {
      blk = M.rtab[(size_t)k * NB + j];
      if (blk == kNoBlock) {
        const float4 p = ret[k];
        int i[3];
        voxel_index(p.x, M, &i[0]);
        voxel_index(p.y, M, &i[1]);
        voxel_index(p.z, M, &i[2]);
        const int rel[3] = {i[0] - M.dom_vox[0], i[1] - M.dom_vox[1], i[2] - M.dom_vox[2]};
        int b0[3], nb[3];
        cube_bricks(M, rel, b0, nb);
        const int bx = j % BA, by = (j / BA) % BA, bz = j / (BA * BA);
        uint32_t val, seen;
        const int h = find_slot(M, pack_brick(b0[0] + bx, b0[1] + by, b0[2] + bz), &val, &seen);
        blk = (h >= 0 && val < M.pool_blocks) ? val : kNoBlock;
        if (blk != kNoBlock) mark_dirty<false>(M, (uint32_t)h, blk, frame, seen, 0u);
      }
    }
    s_blk[t][j] = blk;
  }
  __syncthreads();

  // This thread's cube offsets (ox fastest, so neighbouring threads update
  // neighbouring voxel words), as indices k = o + MR.
  int kx[OPT], ky[OPT], kz[OPT];
#pragma unroll
  for (int s = 0; s < OPT; ++s) {
    const int o = tid + s * NT;
    kx[s] = o % W;
    ky[s] = (o / W) % W;
    kz[s] = o / (W * W);
  }

  for (int t = 0; t < T; ++t) {
    const float4 pr = s_pr[t];
    if (pr.w == 0.f) continue;  // uniform across the block
    const float range = pr.x, bb = pr.y, ir = pr.z;
#pragma unroll
    for (int s = 0; s < OPT; ++s) {
      if (tid + s * NT >= C) break;
      const float4 tx = s_term[t][0][kx[s]], ty = s_term[t][1][ky[s]], tz = s_term[t][2][kz[s]];
      const float aa = __fadd_rn(__fadd_rn(tx.x, ty.x), tz.x);
      // behind-surface cone: theta between x - p and p - q; excluded iff
      // RN(dot / RN(RN(sqrt(aa)) * range)) > cone
      if (aa > 0.f) {
        const float dot = __fadd_rn(__fadd_rn(tx.y, ty.y), tz.y);
        // dot <= 0 makes the rounded cosine <= 0, so with cone >= 0 it is kept
        if (dot > 0.f || cone < 0.f) {
          bool decided = false;
          if (aa > 1e-20f) {
            // a few ulp from the exact cosine (rsqrtf, two products, RN(1 / range))
            const float ca = dot * rsqrtf(aa) * ir;
            if (ca > cone + kMargin) continue;  // certainly excluded
            decided = ca < cone - kMargin;      // certainly kept
          }
          if (!decided && cone_excludes_exact(dot, aa, range, cone)) continue;
        }
      }
      // d = |p - q| - |x - q|, clamped to [0, tau] ([-tau, tau] in the ablation)
      const float cc = __fadd_rn(__fadd_rn(tx.z, ty.z), tz.z);
      float d;
      if (cc >= bb && !M.clamp_signed) {
        d = 0.f;  // |x - q| >= |p - q|: the rounded difference is <= 0
      } else if (cc > 1e-20f && range - sqrt_approx(cc) > tau + range * kMargin) {
        d = tau;  // the exact difference exceeds tau
      } else {
        d = __fsub_rn(range, __fsqrt_rn(cc));
        d = d < M.dlo ? M.dlo : d;
        d = d > tau ? tau : d;
      }
      // |d| <= tau <= 1 m, so |d 2^20| < 2^31: the 32-bit conversion rounds
      // exactly as a 64-bit one would, and stays off the FP64 pipe
      const long long dq = (long long)__float2int_rn(__fmul_rn(d, kScale));
      const int code = __float_as_int(tx.w) + __float_as_int(ty.w) + __float_as_int(tz.w);
      const uint32_t blk = s_blk[t][code >> 16];
      if (blk >= M.pool_blocks) continue;
      atomicAdd(M.vox + (size_t)blk * kBrickVox + (code & 0xFFFF), make_word(dq, 1ull));
    }
  }

  // Ray-cleared band toward the sensor (append-only, does not touch S or w).
  for (int e = tid; e < T * M.ns; e += NT) {
    const int t = e / M.ns, s = e % M.ns + 1;
    if (s_p[t].w == 0.f) continue;
    const float p[3] = {s_p[t].x, s_p[t].y, s_p[t].z};
    int sv[3];
    if (!band_sample(M, p, q, s_pr[t].x, s, sv)) continue;
    uint32_t blk, seen;
    const int h = find_slot(M, pack_brick(sv[0] >> 3, sv[1] >> 3, sv[2] >> 3), &blk, &seen);
    if (h < 0 || blk >= M.pool_blocks) continue;
    const int l = (sv[0] & 7) | ((sv[1] & 7) << 3) | ((sv[2] & 7) << 6);
    atomicOr(M.cleared + blk * 16 + (l >> 5), 1u << (l & 31));
    mark_dirty<false>(M, (uint32_t)h, blk, frame, seen, 0u);
  }
}

// Tiles of 8 returns for the single-map path, one CTA each (measured against
// 12, 16, 20, 26 and 32 on the pine stream, and against persistent CTAs that
// each take an equal share of the returns: slower, 40.9 against 35.4 us).
constexpr int kTile = 8;

template <int W>
__global__ void __launch_bounds__(CubeShape<W>::NT) k_integrate(MapView M,
                                                                const float4* __restrict__ ret,
                                                                uint32_t n, float q0, float q1,
                                                                float q2, uint32_t frame) {
  const uint32_t r0 = blockIdx.x * kTile;
  integrate_tile<W, kTile>(M, ret, r0, min(r0 + kTile, n), q0, q1, q2, frame);
}

// Weight cap and bit view of one dirty brick; called by a CTA of NT threads
// (512 / NT voxels each, NT a multiple of 128). The x-row bytes come straight
// from the ballots; the y- and z-row bytes of the occupied view are gathered
// from the brick's 512 bits in shared memory.
template <int NT>
__device__ void bitview_brick(const MapView& M, uint32_t blk) {
  static_assert(NT >= 128 && 512 % NT == 0, "bitview_brick: NT must divide 512, >= 128");
  __shared__ unsigned s_ob[16];
  if (!check_index(blk < M.pool_blocks, M.ctl)) return;  // uniform over the CTA
  const int lane = threadIdx.x & 31;
  unsigned char* occ = reinterpret_cast<unsigned char*>(M.occ);
  unsigned char* known = reinterpret_cast<unsigned char*>(M.known);
  const size_t row_bytes = (size_t)M.row_words * 8;
  const uint64_t key = M.bkey[blk];
  const uint32_t bx = (uint32_t)(key & 0x1FFFFF), by = (uint32_t)((key >> 21) & 0x1FFFFF),
                 bz = (uint32_t)(key >> 42);
  unsigned long long word[512 / NT];
#pragma unroll
  for (int s = 0; s < 512 / NT; ++s) word[s] = M.vox[(size_t)blk * kBrickVox + threadIdx.x + s * NT];
#pragma unroll
  for (int s = 0; s < 512 / NT; ++s) {
    const int l = threadIdx.x + s * NT, wi = l >> 5;
    unsigned long long w = word[s] & kWMask;
    long long S = word_S(word[s]);
    if (w > M.w_cap) {
      S = capped_S(S, M.w_cap, (long long)w);  // |S| < 2^40, w_cap < 2^20: no overflow
      w = M.w_cap;
      M.vox[(size_t)blk * kBrickVox + l] = make_word(S, w);
    }
    const bool o = w >= 1 && S < (long long)M.rcq * (long long)w;
    const bool cl = (M.cleared[blk * 16 + wi] >> lane) & 1u;
    const bool kn = w >= 1 || cl;
    const unsigned ob = __ballot_sync(0xffffffffu, o);
    const unsigned kb = __ballot_sync(0xffffffffu, kn);
    if (lane == 0) s_ob[wi] = ob;
    if (lane < 4) {
      const size_t y = (size_t)by * 8 + (wi & 1) * 4 + lane;
      const size_t z = (size_t)bz * 8 + (wi >> 1);
      const size_t at = (z * (size_t)M.dim_vox[1] + y) * row_bytes + bx;
      if (check_index(at < M.words_x * 8, M.ctl)) {
        occ[at] = (unsigned char)(ob >> (8 * lane));
        known[at] = (unsigned char)(kb >> (8 * lane));
      }
    }
  }
  __syncthreads();
  const int l = threadIdx.x;
  if (l < 128) {
    // l < 64: the y row at (x, z) = (l & 7, l >> 3); else the z row at (x, y)
    const int x = l & 7, c = (l >> 3) & 7;
    unsigned byte = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int v = l < 64 ? x + 8 * k + 64 * c : x + 8 * c + 64 * k;
      byte |= ((s_ob[v >> 5] >> (v & 31)) & 1u) << k;
    }
    const size_t X = (size_t)M.dim_vox[0], xa = (size_t)bx * 8 + x;
    if (l < 64) {
      const size_t z = (size_t)bz * 8 + c;
      const size_t at = (z * X + xa) * ((size_t)M.row_words_y * 8) + by;
      if (check_index(at < M.words_y * 8, M.ctl))
        reinterpret_cast<unsigned char*>(M.occ_y)[at] = (unsigned char)byte;
    } else {
      const size_t y = (size_t)by * 8 + c;
      const size_t at = (y * X + xa) * ((size_t)M.row_words_z * 8) + bz;
      if (check_index(at < M.words_z * 8, M.ctl))
        reinterpret_cast<unsigned char*>(M.occ_z)[at] = (unsigned char)byte;
    }
  }
  __syncthreads();  // s_ob is rewritten for the CTA's next brick
}

// CTAs of 256 threads (two voxels each): eight per SM, so a scan's dirty
// bricks (about a thousand per pine frame) take one brick per CTA.
constexpr int kBitviewThreads = 256;

__global__ void __launch_bounds__(kBitviewThreads, 2048 / kBitviewThreads) k_bitview(MapView M) {
  const uint32_t count = __ldcg(&M.ctl->dirty_count);
  for (uint32_t d = blockIdx.x; d < count; d += gridDim.x)
    bitview_brick<kBitviewThreads>(M, M.dirty[d]);
}

// Per-voxel flags of allocated bricks for export: bit0 cleared, bit1
// occupied, bit2 known.
__global__ void __launch_bounds__(512) k_export_flags(MapView M, uint8_t* __restrict__ flags) {
  const uint32_t blk = blockIdx.x;
  const int l = threadIdx.x;
  const uint64_t key = M.bkey[blk];
  const int x = (int)(key & 0x1FFFFF) * 8 + (l & 7);
  const int y = (int)((key >> 21) & 0x1FFFFF) * 8 + ((l >> 3) & 7);
  const int z = (int)(key >> 42) * 8 + (l >> 6);
  const size_t word = ((size_t)z * M.dim_vox[1] + y) * M.row_words + (x >> 6);
  const unsigned cl = (M.cleared[blk * 16 + (l >> 5)] >> (l & 31)) & 1u;
  const unsigned oc = (unsigned)(M.occ[word] >> (x & 63)) & 1u;
  const unsigned kn = (unsigned)(M.known[word] >> (x & 63)) & 1u;
  flags[(size_t)blk * kBrickVox + l] = (uint8_t)(cl | (oc << 1) | (kn << 2));
}

cudaError_t launch_export_flags(const MapView& M, uint32_t count, uint8_t* d_flags,
                                cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  k_export_flags<<<count, 512, 0, stream>>>(M, d_flags);
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : cudaStreamSynchronize(stream);
}

// Host-side launchers of the three integration kernels (on `stream`).
cudaError_t launch_alloc(const MapView& M, const float* d_xyz, uint32_t n, const float pose[16],
                         float4* d_ret, uint32_t frame, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(&M.ctl->dirty_count, 0, sizeof(uint32_t), stream);
  if (e != cudaSuccess || n == 0) return e;
  Pose P;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) P.r[r][c] = pose[4 * r + c];
  const uint64_t threads = (uint64_t)n * (M.nbmax + M.ns);
  k_alloc<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(M, d_xyz, n, P, d_ret, frame);
  return cudaGetLastError();
}

cudaError_t launch_cube(const MapView& M, uint32_t n, const float pose[16], const float4* d_ret,
                        uint32_t frame, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (n + kTile - 1) / kTile;
  switch (2 * M.m + 1) {
#define AF_CASE(W)                                                                          \
  case W:                                                                                   \
    k_integrate<W><<<grid, CubeShape<W>::NT, 0, stream>>>(M, d_ret, n, pose[3], pose[7],   \
                                                          pose[11], frame);                 \
    break;
    AF_CASE(3) AF_CASE(5) AF_CASE(7) AF_CASE(9) AF_CASE(11) AF_CASE(13) AF_CASE(15) AF_CASE(17)
#undef AF_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bitview(const MapView& M, int num_sms, cudaStream_t stream) {
  k_bitview<<<num_sms * (2048 / kBitviewThreads), kBitviewThreads, 0, stream>>>(M);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Batched ticks: the same per-map bodies, driven by persistent grids over
// the work of every map of the batch (see af_batch.cu).
// ---------------------------------------------------------------------------

__global__ void k_batch_begin(const BatchHdr* __restrict__ B, const SceneDesc* __restrict__ D) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < B->count;
       s += gridDim.x * blockDim.x)
    D[s].M.ctl->dirty_count = 0;
}

__global__ void __launch_bounds__(256) k_alloc_batch(const BatchHdr* __restrict__ B,
                                                      const SceneDesc* __restrict__ D) {
  const uint32_t total = B->total_alloc;
  const int count = (int)B->count;
  const uint32_t stride = gridDim.x * blockDim.x;
  // warp-uniform trip count: alloc_slot is a warp-wide call
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total;
       base += stride) {
    const uint32_t e = base + (threadIdx.x & 31u);
    const bool act = e < total;
    const int s = act ? scene_of<0>(D, count, e) : 0;
    const SceneDesc& d = D[s];
    alloc_slot<true>(d.M, d.xyz, act ? d.n : 0u, d.P, d.ret, d.frame, act ? e - d.alloc_off : 0u,
               act ? (uint32_t)s : 0xFFFFFFFFu);
  }
}

template <int W, int T>
__global__ void __launch_bounds__(CubeShape<W>::NT) k_integrate_batch(
    const BatchHdr* __restrict__ B, const SceneDesc* __restrict__ D) {
  const uint32_t total = B->total_tiles;
  const int count = (int)B->count;
  for (uint32_t tg = blockIdx.x; tg < total; tg += gridDim.x) {
    const int s = scene_of<1>(D, count, tg);
    const SceneDesc& d = D[s];
    const uint32_t r0 = (tg - d.tile_off) * T;
    integrate_tile<W, T>(d.M, d.ret, r0, min(r0 + T, d.n), d.P.r[0][3], d.P.r[1][3],
                         d.P.r[2][3], d.frame);
  }
}

// Dirty bricks of all maps as one concatenated list, strided over the CTAs.
__global__ void __launch_bounds__(512) k_bitview_batch(const BatchHdr* __restrict__ B,
                                                        const SceneDesc* __restrict__ D) {
  const uint32_t count = B->count, grid = gridDim.x;
  uint32_t acc = 0;
  for (uint32_t s = 0; s < count; ++s) {
    const MapView& M = D[s].M;
    const uint32_t cnt = __ldcg(&M.ctl->dirty_count);
    // this CTA takes the global indices acc + r with (acc + r) % grid == blockIdx.x
    for (uint32_t r = (blockIdx.x + grid - acc % grid) % grid; r < cnt; r += grid)
      bitview_brick<512>(M, M.dirty[r]);
    acc += cnt;
  }
}

template <int W, int T>
int blocks_per_sm_integrate() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_integrate_batch<W, T>, CubeShape<W>::NT, 0);
  return b > 0 ? b : 1;
}

cudaError_t launch_batch_integrate(const BatchHdr* B, const SceneDesc* D, uint32_t count, int m,
                                   int tile, int num_sms, cudaStream_t stream) {
  k_batch_begin<<<(count + 127) / 128, 128, 0, stream>>>(B, D);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_alloc_batch, 256, 0);
  k_alloc_batch<<<num_sms * (per > 0 ? per : 1), 256, 0, stream>>>(B, D);
  switch ((2 * m + 1) * 100 + tile) {
#define AF_BCASE(W, TT)                                                                \
  case W * 100 + TT:                                                                   \
    k_integrate_batch<W, TT><<<num_sms * blocks_per_sm_integrate<W, TT>(),             \
                               CubeShape<W>::NT, 0, stream>>>(B, D);                   \
    break;
#define AF_BW(W) AF_BCASE(W, 8) AF_BCASE(W, 16) AF_BCASE(W, 32)
    AF_BW(3) AF_BW(5) AF_BW(7) AF_BW(9) AF_BW(11) AF_BW(13) AF_BW(15) AF_BW(17)
#undef AF_BW
#undef AF_BCASE
    default: return cudaErrorInvalidValue;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bitview_batch, 512, 0);
  k_bitview_batch<<<num_sms * (per > 0 ? per : 1), 512, 0, stream>>>(B, D);
  return cudaGetLastError();
}

}  // namespace af
