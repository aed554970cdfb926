// af_score.cu -- accessibility scoring on sm_103a (Sec. 3.4, 3.5 of the paper).
//
// One warp per surface point. The plain form (k_score_staged) is a persistent
// grid whose CTAs first copy the direction table, the arm offsets and the
// tool runs into shared memory; the batched form and tables too large to
// stage read them through the read-only path (k_score, k_score_batch).
// The lanes first evaluate the normal filter for
// 32 directions at a time (ballot -> candidate mask); the candidates are then
// visited in index order, each by the whole warp:
//   * tool kernel: lanes take x-runs of the precomputed kernel (32 runs per
//     step), fetch the run's bits from the occupied plane with one or two
//     64-bit loads, AND with the run mask and __popc; a warp sum saturates
//     at the score to beat, so counting stops as soon as the direction can
//     no longer improve the point;
//   * arm samples: three single-bit lookups (occupied or unknown blocks);
//   * corridor: runs as above, any set bit blocks (__any_sync early exit);
//   * once a best exists, the arm-clear candidates are counted two at a time
//     (half a warp each) and then decided in index order.
// The best direction is the lowest-index minimum; a score of 0 ends the
// point. Every early exit returns exactly what a full evaluation of every
// candidate would (the score to beat only shrinks; ties keep the lower
// index).
//
// Work sharing (ScoreSplit): a point whose search takes more than `budget`
// directions past the arm screen stops there and hands the rest of its
// directions to k_score_split, where one warp takes each (point, direction)
// item, prunes it against the point's packed best so far (read at the start
// of the item; the best only ever decreases) and folds its exact score in
// with atomicMin. The packed lowest-index minimum is the result of the full
// search whatever the order the items run in; k_score_finish writes it out.
// The split bounds the span of the launch by the heaviest direction instead
// of the heaviest point.
//
// The device functions live in af_score.cuh.
#include <algorithm>

#include "af_score.cuh"

namespace af {

// Scores point pi with the whole warp (all 32 lanes call this together).
template <bool SPLIT, bool SM = false>
__device__ void score_point(const MapView& M, const ToolView& T, const float* __restrict__ pts,
                            const float* __restrict__ nrm, uint32_t pi,
                            uint8_t* __restrict__ label, int16_t* __restrict__ best_out,
                            int lane, const ScoreSplit& S) {
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
  int next = -1;
  if (fast) set_rows(M, P); else P.row = P.rowy = P.rowz = 0;
  const NormalFilter F{n0, n1, n2};
  if (!SPLIT)
    res = fast ? best_direction<true, NormalFilter, SM>(M, T, P, F, lane)
               : best_direction<false, NormalFilter, SM>(M, T, P, F, lane);
  else
    res = fast ? best_direction_budget<true, NormalFilter, SM>(M, T, P, F, lane, S.budget, &next)
               : best_direction_budget<false, NormalFilter, SM>(M, T, P, F, lane, S.budget, &next);

  if (lane == 0) {
    if (next < 0) {
      label[pi] = (res.y >= 0 && res.x < T.n_c) ? 1 : 2;
      best_out[pi] = (int16_t)res.y;
    } else {  // hand the directions from `next` on to k_score_split
      const uint32_t o = atomicAdd(S.count, 1u);
      S.over[o] = make_int2((int)pi, next);
      S.res[o] = pack_result(res);
    }
    atomicAdd(&M.ctl->points_scored, 1ull);
    atomicAdd(&M.ctl->tests, (unsigned long long)ncand);
  }
}

template <int WARPS, bool SPLIT>
__global__ void __launch_bounds__(WARPS * 32, 2048 / (WARPS * 32))
    k_score(MapView M, ToolView T, const float* __restrict__ pts, const float* __restrict__ nrm,
            uint32_t m, uint8_t* __restrict__ label, int16_t* __restrict__ best_out,
            ScoreSplit S) {
  const uint32_t pi = blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (pi >= m) return;  // whole warp
  score_point<SPLIT>(M, T, pts, nrm, pi, label, best_out, threadIdx.x & 31, S);
}

// Shared-memory bytes of the staged scorer's tables: direction table (16 B
// per direction), arm offsets (24 B per direction), tool runs (8 B per run).
__host__ __device__ inline size_t staged_bytes(const ToolView& T) {
  return (size_t)T.G * 40 + (size_t)T.ntool * 8;
}
// Tables up to 100 KB are staged (two CTAs of 32 warps still fit an SM's
// 228 KB); larger ones (many directions, long tools) are read through the
// read-only path.
constexpr size_t kStagedMaxBytes = 100 * 1024;

// The staged form of k_score: a persistent CTA copies the direction table,
// the arm offsets and every direction's tool runs into shared memory once,
// so that each step of a point's search waits on one L2 load (the plane
// word) instead of a table entry and then a plane word. A warp scores point
// (its warp index) first, then takes points from a launch-wide counter; the
// last warp to finish zeroes the counters for the next launch (every other
// warp has then taken its last point). The search itself is the same.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 2048 / (WARPS * 32))
    k_score_staged(MapView M, ToolView T, const float* __restrict__ pts,
                   const float* __restrict__ nrm, uint32_t m, uint8_t* __restrict__ label,
                   int16_t* __restrict__ best_out, uint32_t* __restrict__ work) {
  short4* s_arm = reinterpret_cast<short4*>(af_staged_tab + T.G);
  int2* s_runs = reinterpret_cast<int2*>(reinterpret_cast<char*>(af_staged_tab) + 40 * T.G);
  for (int i = threadIdx.x; i < T.G; i += WARPS * 32) af_staged_tab[i] = __ldg(T.dtab + i);
  for (int i = threadIdx.x; i < 3 * T.G; i += WARPS * 32) s_arm[i] = __ldg(T.arm + i);
  for (int i = threadIdx.x; i < T.ntool; i += WARPS * 32) s_runs[i] = __ldg(T.fruns + i);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t nw = gridDim.x * WARPS;
  uint32_t pi = blockIdx.x * WARPS + (threadIdx.x >> 5);
  while (pi < m) {
    score_point<false, true>(M, T, pts, nrm, pi, label, best_out, lane,
                             ScoreSplit{nullptr, nullptr, nullptr, -1, nullptr});
    uint32_t nxt = 0;
    if (lane == 0) nxt = nw + atomicAdd(work, 1u);
    pi = __shfl_sync(0xffffffffu, nxt, 0);
  }
  if (lane == 0 && atomicAdd(work + 1, 1u) == nw - 1u) {
    work[0] = 0u;
    work[1] = 0u;
  }
}

// One (point, direction) item of a handed-off search; the whole warp.
template <bool FAST>
__device__ void split_item(const MapView& M, const ToolView& T, const Pt& P, int g, uint32_t* res,
                           int lane) {
  const int nc = T.n_c;
  const uint32_t cur = __ldcg(res);
  const int bs = (int)(cur >> 16), bg = (int)(cur & 0xFFFFu);  // bg 0xFFFF: none yet
  bool arm_ok = false;
  if (lane == 0) arm_ok = arm_clear<FAST>(M, T, g, P);
  arm_ok = __shfl_sync(0xffffffffu, arm_ok, 0);
  uint32_t mine;
  if (!arm_ok) {
    if (bs <= nc) return;  // blocked (n_c + 1) cannot beat an unblocked best
    mine = pack_result(make_int2(nc + 1, g));
  } else {
    // counts below `sat` may improve the best; `exact` counts up to n_c
    const bool exact = bs > nc || (g < bg && bs == nc);
    const int sat = exact ? nc : (g < bg ? bs + 1 : bs);
    if (!exact && sat == 0) return;
    const int c = tool_count<FAST>(M, T, g, P, sat, lane);
    if (!exact && c >= sat) return;
    mine = corridor_blocked<FAST>(M, T, g, P, lane) ? pack_result(make_int2(nc + 1, g))
                                                   : pack_result(make_int2(min(c, nc), g));
  }
  if (lane == 0 && mine < cur) atomicMin(res, mine);
}

__global__ void __launch_bounds__(128, 16)
    k_score_split(MapView M, ToolView T, const float* __restrict__ pts,
                  const float* __restrict__ nrm, ScoreSplit S) {
  const int lane = threadIdx.x & 31;
  const uint64_t items = (uint64_t)__ldcg(S.count) * (uint64_t)T.G;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t it = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nw) {
    const uint32_t o = (uint32_t)(it / (uint64_t)T.G);
    const int g = (int)(it - (uint64_t)o * T.G);
    const int2 ov = __ldcg(S.over + o);
    if (g < ov.y) continue;
    const uint32_t pi = (uint32_t)ov.x;
    if (!candidate(T, g, nrm[3 * pi], nrm[3 * pi + 1], nrm[3 * pi + 2])) continue;
    // the point passed the gate in k_score, so its voxel is inside the box
    int i0, i1, i2;
    voxel_index(pts[3 * pi], M, &i0);
    voxel_index(pts[3 * pi + 1], M, &i1);
    voxel_index(pts[3 * pi + 2], M, &i2);
    Pt P;
    P.px = i0 - M.dom_vox[0];
    P.py = i1 - M.dom_vox[1];
    P.pz = i2 - M.dom_vox[2];
    const bool fast = P.px >= T.reach[0] && P.px + T.reach[0] < M.dim_vox[0] &&
                      P.py >= T.reach[1] && P.py + T.reach[1] < M.dim_vox[1] &&
                      P.pz >= T.reach[2] && P.pz + T.reach[2] < M.dim_vox[2];
    if (fast) set_rows(M, P); else P.row = P.rowy = P.rowz = 0;
    if (fast)
      split_item<true>(M, T, P, g, S.res + o, lane);
    else
      split_item<false>(M, T, P, g, S.res + o, lane);
  }
}

__global__ void __launch_bounds__(256) k_score_finish(ScoreSplit S, int n_c,
                                                      uint8_t* __restrict__ label,
                                                      int16_t* __restrict__ best_out) {
  const uint32_t n = __ldcg(S.count);
  for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    const uint32_t r = S.res[o];
    const uint32_t pi = (uint32_t)S.over[o].x;
    const int sc = (int)(r >> 16), g = (int)(r & 0xFFFFu);
    best_out[pi] = g == 0xFFFF ? (int16_t)-1 : (int16_t)g;
    label[pi] = (g != 0xFFFF && sc < n_c) ? 1 : 2;
  }
}

cudaError_t launch_score(const MapView& M, const ToolView& T, const float* d_pts,
                         const float* d_nrm, uint32_t m, uint8_t* d_label, int16_t* d_best,
                         const ScoreSplit& S, int num_sms, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  constexpr int kStagedWarps = 32;
  if (S.budget < 0 && S.work != nullptr && staged_bytes(T) <= kStagedMaxBytes) {
    const size_t smem = staged_bytes(T);
    int per = 0;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) {  // above the default dynamic shared-memory limit: opt in
      e = cudaFuncSetAttribute(k_score_staged<kStagedWarps>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per, k_score_staged<kStagedWarps>, kStagedWarps * 32, smem);
    if (e != cudaSuccess) return e;
    const uint32_t need = (m + kStagedWarps - 1) / kStagedWarps;
    const uint32_t grid = std::min<uint32_t>(need, (uint32_t)num_sms * (uint32_t)(per > 0 ? per : 1));
    k_score_staged<kStagedWarps><<<grid, kStagedWarps * 32, smem, stream>>>(
        M, T, d_pts, d_nrm, m, d_label, d_best, S.work);
    return cudaGetLastError();
  }
  constexpr int WARPS = 2;
  if (S.budget >= 0) {
    cudaError_t e = cudaMemsetAsync(S.count, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
  }
  if (S.budget >= 0)
    k_score<WARPS, true><<<(m + WARPS - 1) / WARPS, WARPS * 32, 0, stream>>>(M, T, d_pts, d_nrm,
                                                                            m, d_label, d_best, S);
  else
    k_score<WARPS, false><<<(m + WARPS - 1) / WARPS, WARPS * 32, 0, stream>>>(M, T, d_pts, d_nrm,
                                                                             m, d_label, d_best, S);
  if (S.budget >= 0) {
    k_score_split<<<num_sms * 16, 128, 0, stream>>>(M, T, d_pts, d_nrm, S);
    k_score_finish<<<num_sms, 256, 0, stream>>>(S, T.n_c, d_label, d_best);
  }
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
    score_point<false>(d.M, d.T, d.pts, d.nrm, pg - d.pt_off, d.label, d.best, threadIdx.x & 31,
                       ScoreSplit{nullptr, nullptr, nullptr, -1});
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
