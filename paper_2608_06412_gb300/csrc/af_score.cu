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
// of up to 64 voxels costs one or two loads of the bit plane.
#include "af_internal.cuh"

namespace af {

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

__device__ inline bool bit_at(const unsigned long long* __restrict__ plane, const MapView& M,
                              int x, int y, int z) {
  if ((unsigned)x >= (unsigned)M.dim_vox[0] || (unsigned)y >= (unsigned)M.dim_vox[1] ||
      (unsigned)z >= (unsigned)M.dim_vox[2])
    return false;
  const unsigned long long wd =
      __ldg(plane + ((size_t)z * M.dim_vox[1] + y) * M.row_words + (x >> 6));
  return (wd >> (x & 63)) & 1ull;
}

// Occupied tool voxels of direction g at voxel (px,py,pz), saturated at `sat`.
__device__ inline int tool_count(const MapView& M, const ToolView& T, int g, int px, int py,
                                 int pz, int sat, int lane) {
  const int4 dt = __ldg(T.dtab + g);
  int total = 0;
  for (int r0 = dt.x; r0 < dt.y; r0 += 32) {
    const int r = r0 + lane;
    int c = 0;
    if (r < dt.y) {
      const short4 run = __ldg(T.runs + r);
      bool out = false;
      c = __popcll(row_bits(M.occ, M, px + run.x, py + run.z, pz + run.w, run.y, &out));
    }
    total += __reduce_add_sync(0xffffffffu, c);
    if (total >= sat) return sat;
  }
  return total;
}

// Arm samples (occupied or unknown) or corridor (occupied; strict: or unknown).
__device__ inline bool path_blocked(const MapView& M, const ToolView& T, int g, int px, int py,
                                    int pz, int lane) {
  bool hit = false;
  if (lane < 3) {
    const short4 a = __ldg(T.arm + 3 * g + lane);
    const int x = px + a.x, y = py + a.y, z = pz + a.z;
    hit = bit_at(M.occ, M, x, y, z) || !bit_at(M.known, M, x, y, z);
  }
  if (__any_sync(0xffffffffu, hit)) return true;
  const int4 dt = __ldg(T.dtab + g);
  for (int r0 = dt.z; r0 < dt.w; r0 += 32) {
    const int r = r0 + lane;
    bool h = false;
    if (r < dt.w) {
      const short4 run = __ldg(T.runs + r);
      bool out = false;
      const unsigned long long o =
          row_bits(M.occ, M, px + run.x, py + run.z, pz + run.w, run.y, &out);
      h = o != 0ull;
      if (T.strict && !h) {
        const unsigned long long k =
            row_bits(M.known, M, px + run.x, py + run.z, pz + run.w, run.y, &out);
        const unsigned long long full = run.y == 64 ? ~0ull : ((1ull << run.y) - 1ull);
        h = out || (k != full);
      }
    }
    if (__any_sync(0xffffffffu, h)) return true;
  }
  return false;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_score(MapView M, ToolView T,
                                                       const float* __restrict__ pts,
                                                       const float* __restrict__ nrm, uint32_t m,
                                                       uint8_t* __restrict__ label,
                                                       int16_t* __restrict__ best_out) {
  const int lane = threadIdx.x & 31;
  const uint32_t pi = blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (pi >= m) return;  // whole warp

  const float s0 = pts[3 * pi], s1 = pts[3 * pi + 1], s2 = pts[3 * pi + 2];
  const float n0 = nrm[3 * pi], n1 = nrm[3 * pi + 1], n2 = nrm[3 * pi + 2];

  // the point's voxel and its weight (confidence gate, Sec. 3.5)
  int i0, i1, i2;
  bool ok = voxel_index(s0, M.v, &i0) && voxel_index(s1, M.v, &i1) && voxel_index(s2, M.v, &i2);
  const int px = i0 - M.dom_vox[0], py = i1 - M.dom_vox[1], pz = i2 - M.dom_vox[2];
  uint32_t w = 0;
  if (ok && (unsigned)px < (unsigned)M.dim_vox[0] && (unsigned)py < (unsigned)M.dim_vox[1] &&
      (unsigned)pz < (unsigned)M.dim_vox[2]) {
    uint32_t blk = kNoBlock;
    if (lane == 0) blk = lookup_brick(M, pack_brick(px >> 3, py >> 3, pz >> 3));
    blk = __shfl_sync(0xffffffffu, blk, 0);
    if (blk != kNoBlock) {
      const int l = (px & 7) | ((py & 7) << 3) | ((pz & 7) << 6);
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
  for (int gb = 0; gb < T.G; gb += 32) {
    const int g = gb + lane;
    bool cand = false;
    if (g < T.G) {
      const float u0 = __ldg(T.dirs + 3 * g), u1 = __ldg(T.dirs + 3 * g + 1),
                  u2 = __ldg(T.dirs + 3 * g + 2);
      const float nu = __fadd_rn(__fadd_rn(__fmul_rn(n0, u0), __fmul_rn(n1, u1)), __fmul_rn(n2, u2));
      cand = nu > T.cos_max;
    }
    ncand += __popc(__ballot_sync(0xffffffffu, cand));
  }

  const int nc = T.n_c;
  int bscore = nc + 2, best = -1;
  for (int gb = 0; gb < T.G && bscore != 0; gb += 32) {
    const int g = gb + lane;
    bool cand = false;
    if (g < T.G) {
      const float u0 = __ldg(T.dirs + 3 * g), u1 = __ldg(T.dirs + 3 * g + 1),
                  u2 = __ldg(T.dirs + 3 * g + 2);
      const float nu = __fadd_rn(__fadd_rn(__fmul_rn(n0, u0), __fmul_rn(n1, u1)), __fmul_rn(n2, u2));
      cand = nu > T.cos_max;
    }
    unsigned mask = __ballot_sync(0xffffffffu, cand);
    while (mask) {
      const int gg = gb + __ffs(mask) - 1;
      mask &= mask - 1u;
      if (bscore <= nc) {
        // improves only if not blocked and strictly fewer collisions
        const int cnt = tool_count(M, T, gg, px, py, pz, bscore, lane);
        if (cnt >= bscore) continue;
        if (path_blocked(M, T, gg, px, py, pz, lane)) continue;
        bscore = cnt;
        best = gg;
      } else {
        // nothing unblocked yet: any unblocked direction improves
        if (path_blocked(M, T, gg, px, py, pz, lane)) {
          if (best < 0) {
            bscore = nc + 1;
            best = gg;
          }
          continue;
        }
        bscore = tool_count(M, T, gg, px, py, pz, nc, lane);
        best = gg;
      }
      if (bscore == 0) break;
    }
  }

  if (lane == 0) {
    label[pi] = (best >= 0 && bscore < nc) ? 1 : 2;
    best_out[pi] = (int16_t)best;
    atomicAdd(&M.ctl->points_scored, 1ull);
    atomicAdd(&M.ctl->tests, (unsigned long long)ncand);
  }
}

cudaError_t launch_score(const MapView& M, const ToolView& T, const float* d_pts,
                         const float* d_nrm, uint32_t m, uint8_t* d_label, int16_t* d_best,
                         cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  constexpr int WARPS = 4;
  k_score<WARPS><<<(m + WARPS - 1) / WARPS, WARPS * 32, 0, stream>>>(M, T, d_pts, d_nrm, m,
                                                                      d_label, d_best);
  return cudaGetLastError();
}

}  // namespace af
