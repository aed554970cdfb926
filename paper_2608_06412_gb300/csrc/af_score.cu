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
// The device functions live in af_score.cuh.
#include "af_score.cuh"

namespace af {

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
    res = best_direction<true>(M, T, P, NormalFilter{n0, n1, n2}, lane);
  } else {
    P.row = 0;
    res = best_direction<false>(M, T, P, NormalFilter{n0, n1, n2}, lane);
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
