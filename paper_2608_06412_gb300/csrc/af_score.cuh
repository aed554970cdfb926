// af_score.cuh -- the scoring device functions (Sec. 3.4, 3.5), shared by the
// plain, batched and stateful-layer scoring kernels.
//
// Kernels are x-runs rather than voxel lists: a cylinder meets every x-row
// in one interval (two at most next to the self-exclusion ball), so a run
// of up to 64 voxels costs one or two loads of the bit plane. A point whose
// whole kernel reach lies inside the map box takes the FAST path: the run
// table then holds each run's row as a plane-word offset from the point's
// row, and no bound is checked.
#pragma once

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

// One corridor run: occupied (strict: or not known) anywhere in it.
template <bool FAST>
__device__ inline bool corridor_run_hit(const MapView& M, const ToolView& T, int r, const Pt& P) {
  const RunEntry e = load_run<FAST>(T, r);
  int len;
  bool out = false;
  bool h = run_bits<FAST>(M.occ, M, e, P, &len, &out) != 0ull;
  if (T.strict && !h) {
    const unsigned long long kb = run_bits<FAST>(M.known, M, e, P, &len, &out);
    const unsigned long long full = len == 64 ? ~0ull : ((1ull << len) - 1ull);
    h = out || (kb != full);
  }
  return h;
}

// Corridor of direction g: any occupied voxel (strict: or unknown) blocks.
// The first warp step tests 32 runs (most blocked corridors end there); later
// steps test 64, then 128 runs, each lane issuing its runs' loads together,
// so a clear corridor costs fewer dependent round trips.
template <bool FAST>
__device__ inline bool corridor_blocked(const MapView& M, const ToolView& T, int g, const Pt& P,
                                        int lane) {
  const int4 dt = __ldg(T.dtab + g);
  int b = dt.z, per = 1;
  while (b < dt.w) {
    bool h = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = b + 32 * k + lane;
      if (k < per && r < dt.w) h |= corridor_run_hit<FAST>(M, T, r, P);
    }
    if (__any_sync(0xffffffffu, h)) return true;
    b += 32 * per;
    per = per < 4 ? 2 * per : 4;
  }
  return false;
}

__device__ inline bool candidate(const ToolView& T, int g, float n0, float n1, float n2) {
  if (g >= T.G) return false;
  const float u0 = __ldg(T.dirs + 3 * g), u1 = __ldg(T.dirs + 3 * g + 1),
              u2 = __ldg(T.dirs + 3 * g + 2);
  const float nu = __fadd_rn(__fadd_rn(__fmul_rn(n0, u0), __fmul_rn(n1, u1)), __fmul_rn(n2, u2));
  return nu > T.cos_max;
}

// The normal filter of Sec. 3.4 as a candidate test.
struct NormalFilter {
  float n0, n1, n2;
  __device__ bool operator()(const ToolView& T, int g) const { return candidate(T, g, n0, n1, n2); }
};

// The candidate loop of one point: lowest-index minimum of the direction
// scores, with exact early exits; `cand(T, g)` says whether direction g is a
// candidate of the point. Returns (best score, best index), (n_c + 2, -1)
// without candidates.
template <bool FAST, class Cand>
__device__ inline int2 best_direction(const MapView& M, const ToolView& T, const Pt& P,
                                      const Cand& cand_of, int lane) {
  const int nc = T.n_c;
  int bscore = nc + 2, best = -1;
  for (int gb = 0; gb < T.G && bscore != 0; gb += 32) {
    // lane-parallel screen: candidates, and the arm samples of each candidate
    const bool cand = cand_of(T, gb + lane);
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


// best_direction with a budget: at most `budget` directions are taken past
// the arm screen (tool count and corridor). If the search stops early,
// *next receives the first direction index not searched and the result is
// exact over the directions before it; *next = -1 when the search finished.
template <bool FAST, class Cand>
__device__ inline int2 best_direction_budget(const MapView& M, const ToolView& T, const Pt& P,
                                             const Cand& cand_of, int lane, int budget,
                                             int* next) {
  const int nc = T.n_c;
  int bscore = nc + 2, best = -1, spent = 0;
  *next = -1;
  for (int gb = 0; gb < T.G && bscore != 0; gb += 32) {
    const bool cand = cand_of(T, gb + lane);
    unsigned mask = __ballot_sync(0xffffffffu, cand);
    const unsigned arm_ok = __ballot_sync(0xffffffffu, cand && arm_clear<FAST>(M, T, gb + lane, P));
    while (mask) {
      const int bit = __ffs(mask) - 1;
      const int g = gb + bit;
      mask &= mask - 1u;
      if (!((arm_ok >> bit) & 1u)) {
        if (best < 0) {
          bscore = nc + 1;
          best = g;
        }
        continue;
      }
      if (spent == budget) {
        *next = g;
        return make_int2(bscore, best);
      }
      ++spent;
      if (bscore <= nc) {
        const int cnt = tool_count<FAST>(M, T, g, P, bscore, lane);
        if (cnt >= bscore) continue;
        if (corridor_blocked<FAST>(M, T, g, P, lane)) continue;
        bscore = cnt;
        best = g;
      } else {
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

// A (score, direction) result packed so that the lowest-index minimum is the
// smallest word: score in the high half, direction (0xFFFF: none) below.
__device__ inline uint32_t pack_result(int2 r) {
  return ((uint32_t)r.x << 16) | (r.y < 0 ? 0xFFFFu : (uint32_t)r.y);
}

}  // namespace af
