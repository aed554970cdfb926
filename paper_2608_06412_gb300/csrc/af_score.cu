// af_score.cu -- accessibility scoring on sm_103a (Sec. 3.4, 3.5 of the paper).
//
// One warp per surface point. The lanes first evaluate the normal filter for
// 32 directions at a time (ballot -> candidate mask); the candidates are then
// visited in index order, each by the whole warp:
//   * tool kernel: lanes take x-runs of the precomputed kernel (32 runs per
//     step), fetch the run's bits from the occupied plane with one or two
//     64-bit loads, AND with the run mask and __popc; a warp sum saturates
//     at the score to beat, so counting stops as soon as the direction can
//     no longer improve the point;
//   * arm samples: three single-bit lookups (occupied or unknown blocks);
//   * corridor: runs as above, any set bit blocks (__any_sync early exit).
// The best direction is the lowest-index minimum; a score of 0 ends the
// point. Every early exit returns exactly what a full evaluation of every
// candidate would (the score to beat only shrinks; ties keep the lower
// index).
//
// Kernels are x-runs rather than voxel lists: a cylinder meets every x-row
// in one interval (two at most next to the self-exclusion ball), so a run
// of up to 64 voxels costs one or two loads of the bit plane. A point whose
// whole kernel reach lies inside the map box takes the FAST path: the run
// table then holds each run's row as a plane-word offset from the point's
// row, and no bound is checked.
#include "af_internal.cuh"

namespace af {

struct Pt {
  int px, py, pz;  // box-relative voxel of the point
  int row;         // plane-word index of the point's row (FAST path only)
};

// Bits x0 .. x0+len-1 of plane row (y, z), bit i = voxel x0 + i; voxels
// outside the map box read 0 and set *outside.
__device__ inline unsigned long long row_bits(const unsigned long long* __restrict__ plane,
                                              const MapView& M, int x0, int y, int z, int len,
                                              bool* outside) {
  if ((unsigned)y >= (unsigned)M.dim_vox[1] || (unsigned)z >= (unsigned)M.dim_vox[2]) {
    *outside = true;
    return 0ull;
  }
  int xa = x0, xb = x0 + len - 1;
  if (xa < 0 || xb >= M.dim_vox[0]) {
    *outside = true;
    xa = max(xa, 0);
    xb = min(xb, M.dim_vox[0] - 1);
    if (xa > xb) return 0ull;
  }
  const unsigned long long* row = plane + ((size_t)z * M.dim_vox[1] + y) * M.row_words;
  const int wa = xa >> 6, wb = xb >> 6, sh = xa & 63;
  unsigned long long win = __ldg(row + wa) >> sh;
  if (wb != wa) win |= __ldg(row + wb) << (64 - sh);
  const int n = xb - xa + 1;
  if (n < 64) win &= (1ull << n) - 1ull;
  return win << (xa - x0);
}

// One run-table entry: the fast form (plane-word row offset, dx0 | len << 16)
// or the plain form (dx0 | len << 16, dy | dz << 16), 16-bit fields.
struct RunEntry {
  int a, b;
};

template <bool FAST>
__device__ inline RunEntry load_run(const ToolView& T, int r) {
  if (FAST) {
    const int2 f = __ldg(T.fruns + r);
    return {f.x, f.y};
  }
  const short4 s = __ldg(T.runs + r);
  return {(int)((uint32_t)(uint16_t)s.x | ((uint32_t)(uint16_t)s.y << 16)),
          (int)((uint32_t)(uint16_t)s.z | ((uint32_t)(uint16_t)s.w << 16))};
}

// Bits of the run of entry e for point P; *len receives the run length.
template <bool FAST>
__device__ inline unsigned long long run_bits(const unsigned long long* __restrict__ plane,
                                              const MapView& M, RunEntry e, const Pt& P,
                                              int* len, bool* outside) {
  const int dx0 = (int)(short)(e.a & 0xffff), dxy = (int)(short)(e.b & 0xffff);
  if (FAST) {
    const int n = e.b >> 16;
    const int xa = P.px + dxy;
    const int row = P.row + e.a;
    const int wa = xa >> 6, wb = (xa + n - 1) >> 6, sh = xa & 63;
    unsigned long long win = __ldg(plane + row + wa) >> sh;
    if (wb != wa) win |= __ldg(plane + row + wb) << (64 - sh);
    if (n < 64) win &= (1ull << n) - 1ull;
    *len = n;
    return win;
  }
  const int n = (int)((uint32_t)e.a >> 16), dz = (int)(short)((uint32_t)e.b >> 16);
  *len = n;
  return row_bits(plane, M, P.px + dx0, P.py + dxy, P.pz + dz, n, outside);
}

// Walks runs [r0, r1) of the tables a warp step (32 runs, one per lane) at a
// time; the caller's `step(entry, valid)` returns true to stop the walk.
template <bool FAST, class F>
__device__ inline void walk_runs(const ToolView& T, int r0, int r1, int lane, F&& step) {
  for (int b = r0; b < r1; b += 32) {
    const int r = b + lane;
    const RunEntry e = r < r1 ? load_run<FAST>(T, r) : RunEntry{0, 0};
    if (step(e, r < r1)) return;
  }
}

template <bool FAST>
__device__ inline bool bit_at(const unsigned long long* __restrict__ plane, const MapView& M,
                              const Pt& P, short4 a) {
  const int x = P.px + a.x, y = P.py + a.y, z = P.pz + a.z;
  if (!FAST && ((unsigned)x >= (unsigned)M.dim_vox[0] || (unsigned)y >= (unsigned)M.dim_vox[1] ||
                (unsigned)z >= (unsigned)M.dim_vox[2]))
    return false;
  const size_t w = FAST ? (size_t)(P.row + (a.z * M.dim_vox[1] + a.y) * M.row_words + (x >> 6))
                        : ((size_t)z * M.dim_vox[1] + y) * M.row_words + (x >> 6);
  return (__ldg(plane + w) >> (x & 63)) & 1ull;
}

// Occupied tool voxels of direction g at point P, saturated at `sat`.
template <bool FAST>
__device__ inline int tool_count(const MapView& M, const ToolView& T, int g, const Pt& P, int sat,
                                 int lane) {
  const int4 dt = __ldg(T.dtab + g);
  int total = 0;
  walk_runs<FAST>(T, dt.x, dt.y, lane, [&](RunEntry e, bool valid) {
    int c = 0;
    if (valid) {
      int len;
      bool out = false;
      c = __popcll(run_bits<FAST>(M.occ, M, e, P, &len, &out));
    }
    total += __reduce_add_sync(0xffffffffu, c);
    return total >= sat;
  });
  return total >= sat ? sat : total;
}

// The three arm samples of direction g (one lane): clear iff none is
// occupied or unknown. All nine loads are issued together (no short
// circuit), so the screen costs two dependent round trips, not up to nine.
template <bool FAST>
__device__ inline bool arm_clear(const MapView& M, const ToolView& T, int g, const Pt& P) {
  short4 a[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) a[s] = __ldg(T.arm + 3 * g + s);
  bool blocked = false;
#pragma unroll
  for (int s = 0; s < 3; ++s)
    blocked = blocked | bit_at<FAST>(M.occ, M, P, a[s]) | !bit_at<FAST>(M.known, M, P, a[s]);
  return !blocked;
}

// Corridor of direction g: any occupied voxel (strict: or unknown) blocks.
template <bool FAST>
__device__ inline bool corridor_blocked(const MapView& M, const ToolView& T, int g, const Pt& P,
                                        int lane) {
  const int4 dt = __ldg(T.dtab + g);
  bool blocked = false;
  walk_runs<FAST>(T, dt.z, dt.w, lane, [&](RunEntry e, bool valid) {
    bool h = false;
    if (valid) {
      int len;
      bool out = false;
      h = run_bits<FAST>(M.occ, M, e, P, &len, &out) != 0ull;
      if (T.strict && !h) {
        const unsigned long long kb = run_bits<FAST>(M.known, M, e, P, &len, &out);
        const unsigned long long full = len == 64 ? ~0ull : ((1ull << len) - 1ull);
        h = out || (kb != full);
      }
    }
    blocked = __any_sync(0xffffffffu, h);
    return blocked;
  });
  return blocked;
}

__device__ inline bool candidate(const ToolView& T, int g, float n0, float n1, float n2) {
  if (g >= T.G) return false;
  const float u0 = __ldg(T.dirs + 3 * g), u1 = __ldg(T.dirs + 3 * g + 1),
              u2 = __ldg(T.dirs + 3 * g + 2);
  const float nu = __fadd_rn(__fadd_rn(__fmul_rn(n0, u0), __fmul_rn(n1, u1)), __fmul_rn(n2, u2));
  return nu > T.cos_max;
}

// The candidate loop of one point: lowest-index minimum of the direction
// scores, with exact early exits. Returns (best score, best index).
template <bool FAST>
__device__ inline int2 best_direction(const MapView& M, const ToolView& T, const Pt& P, float n0,
                                      float n1, float n2, int lane) {
  const int nc = T.n_c;
  int bscore = nc + 2, best = -1;
  for (int gb = 0; gb < T.G && bscore != 0; gb += 32) {
    // lane-parallel screen: candidates, and the arm samples of each candidate
    const bool cand = candidate(T, gb + lane, n0, n1, n2);
    unsigned mask = __ballot_sync(0xffffffffu, cand);
    const unsigned arm_ok = __ballot_sync(0xffffffffu, cand && arm_clear<FAST>(M, T, gb + lane, P));
    while (mask) {
      const int bit = __ffs(mask) - 1;
      const int g = gb + bit;
      mask &= mask - 1u;
      if (!((arm_ok >> bit) & 1u)) {
        // blocked (n_c + 1): improves only the first candidate's empty best
        if (best < 0) {
          bscore = nc + 1;
          best = g;
        }
        continue;
      }
      if (bscore <= nc) {
        // improves only if not blocked and strictly fewer collisions
        const int cnt = tool_count<FAST>(M, T, g, P, bscore, lane);
        if (cnt >= bscore) continue;
        if (corridor_blocked<FAST>(M, T, g, P, lane)) continue;
        bscore = cnt;
        best = g;
      } else {
        // nothing unblocked yet: any unblocked direction improves
        if (corridor_blocked<FAST>(M, T, g, P, lane)) {
          if (best < 0) {
            bscore = nc + 1;
            best = g;
          }
          continue;
        }
        bscore = tool_count<FAST>(M, T, g, P, nc, lane);
        best = g;
      }
      if (bscore == 0) break;
    }
  }
  return make_int2(bscore, best);
}

// Scores point pi with the whole warp (all 32 lanes call this together).
__device__ void score_point(const MapView& M, const ToolView& T, const float* __restrict__ pts,
                            const float* __restrict__ nrm, uint32_t pi,
                            uint8_t* __restrict__ label, int16_t* __restrict__ best_out,
                            int lane) {
  const float s0 = pts[3 * pi], s1 = pts[3 * pi + 1], s2 = pts[3 * pi + 2];
  const float n0 = nrm[3 * pi], n1 = nrm[3 * pi + 1], n2 = nrm[3 * pi + 2];

  // the point's voxel and its weight (confidence gate, Sec. 3.5)
  int i0, i1, i2;
  const bool ok =
      voxel_index(s0, M, &i0) && voxel_index(s1, M, &i1) && voxel_index(s2, M, &i2);
  Pt P;
  P.px = i0 - M.dom_vox[0];
  P.py = i1 - M.dom_vox[1];
  P.pz = i2 - M.dom_vox[2];
  uint32_t w = 0;
  if (ok && (unsigned)P.px < (unsigned)M.dim_vox[0] && (unsigned)P.py < (unsigned)M.dim_vox[1] &&
      (unsigned)P.pz < (unsigned)M.dim_vox[2]) {
    uint32_t blk = kNoBlock;
    if (lane == 0) blk = lookup_brick(M, pack_brick(P.px >> 3, P.py >> 3, P.pz >> 3));
    blk = __shfl_sync(0xffffffffu, blk, 0);
    if (blk != kNoBlock) {
      const int l = (P.px & 7) | ((P.py & 7) << 3) | ((P.pz & 7) << 6);
      w = (uint32_t)(__ldcg(M.vox + (size_t)blk * kBrickVox + l) & kWMask);
    }
  }
  if (w < M.w_min) {
    if (lane == 0) {
      label[pi] = 0;
      best_out[pi] = -1;
    }
    return;
  }

  // nominal tests: every candidate direction of this point
  int ncand = 0;
  for (int gb = 0; gb < T.G; gb += 32)
    ncand += __popc(__ballot_sync(0xffffffffu, candidate(T, gb + lane, n0, n1, n2)));

  const bool fast = P.px >= T.reach[0] && P.px + T.reach[0] < M.dim_vox[0] &&
                    P.py >= T.reach[1] && P.py + T.reach[1] < M.dim_vox[1] &&
                    P.pz >= T.reach[2] && P.pz + T.reach[2] < M.dim_vox[2];
  int2 res;
  if (fast) {
    P.row = (P.pz * M.dim_vox[1] + P.py) * M.row_words;
    res = best_direction<true>(M, T, P, n0, n1, n2, lane);
  } else {
    P.row = 0;
    res = best_direction<false>(M, T, P, n0, n1, n2, lane);
  }

  if (lane == 0) {
    label[pi] = (res.y >= 0 && res.x < T.n_c) ? 1 : 2;
    best_out[pi] = (int16_t)res.y;
    atomicAdd(&M.ctl->points_scored, 1ull);
    atomicAdd(&M.ctl->tests, (unsigned long long)ncand);
  }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 2048 / (WARPS * 32))
    k_score(MapView M, ToolView T, const float* __restrict__ pts, const float* __restrict__ nrm,
            uint32_t m, uint8_t* __restrict__ label, int16_t* __restrict__ best_out) {
  const uint32_t pi = blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (pi >= m) return;  // whole warp
  score_point(M, T, pts, nrm, pi, label, best_out, threadIdx.x & 31);
}

cudaError_t launch_score(const MapView& M, const ToolView& T, const float* d_pts,
                         const float* d_nrm, uint32_t m, uint8_t* d_label, int16_t* d_best,
                         cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  constexpr int WARPS = 2;
  k_score<WARPS><<<(m + WARPS - 1) / WARPS, WARPS * 32, 0, stream>>>(M, T, d_pts, d_nrm, m,
                                                                      d_label, d_best);
  return cudaGetLastError();
}


// Batched ticks: every point of every map of the batch, one warp per point,
// persistent grid (see af_batch.cu).
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 2048 / (WARPS * 32))
    k_score_batch(const BatchHdr* __restrict__ B, const SceneDesc* __restrict__ D) {
  const uint32_t total = B->total_points;
  const int count = (int)B->count;
  const uint32_t nw = gridDim.x * WARPS;
  for (uint32_t pg = blockIdx.x * WARPS + (threadIdx.x >> 5); pg < total; pg += nw) {
    const int s = scene_of<2>(D, count, pg);
    const SceneDesc& d = D[s];
    score_point(d.M, d.T, d.pts, d.nrm, pg - d.pt_off, d.label, d.best, threadIdx.x & 31);
  }
}

template <int WARPS>
static cudaError_t launch_score_batch_w(const BatchHdr* B, const SceneDesc* D, int num_sms,
                                        cudaStream_t stream) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_score_batch<WARPS>, WARPS * 32, 0);
  k_score_batch<WARPS><<<num_sms * (per > 0 ? per : 1), WARPS * 32, 0, stream>>>(B, D);
  return cudaGetLastError();
}

cudaError_t launch_score_batch(const BatchHdr* B, const SceneDesc* D, int warps, int num_sms,
                               cudaStream_t stream) {
  switch (warps) {
    case 2: return launch_score_batch_w<2>(B, D, num_sms, stream);
    case 4: return launch_score_batch_w<4>(B, D, num_sms, stream);
    case 8: return launch_score_batch_w<8>(B, D, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace af
