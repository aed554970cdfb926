// af_score.cuh -- the scoring device functions (Sec. 3.4, 3.5), shared by the
// plain, batched and stateful-layer scoring kernels.
//
// Kernels are runs rather than voxel lists: a cylinder meets every row in
// one interval (two at most next to the self-exclusion ball), so a run of up
// to 64 voxels costs one or two loads of a bit plane. Each direction's runs
// follow the axis it is closest to, read from the occupied view with rows
// along that axis, so a kernel is a few long runs instead of many short
// ones. A point whose whole kernel reach lies inside the map box takes the
// FAST path: the run table then holds each run's row as a plane-word offset
// from the point's row on that plane, and no bound is checked.
#pragma once

#include "af_internal.cuh"

namespace af {

struct Pt {
  int px, py, pz;  // box-relative voxel of the point
  int row;         // plane-word index of the point's x row (FAST path only)
  int rowy, rowz;  // ... of its y row and z row
};

// The point's row bases on the three planes (FAST path).
__device__ inline void set_rows(const MapView& M, Pt& P) {
  P.row = (P.pz * M.dim_vox[1] + P.py) * M.row_words;
  P.rowy = (P.pz * M.dim_vox[0] + P.px) * M.row_words_y;
  P.rowz = (P.py * M.dim_vox[0] + P.px) * M.row_words_z;
}

// Bits a0 .. a0+len-1 along axis `ax` of the plane row at the other two
// coordinates (o1, o2) (o1 the lower axis), bit i = voxel a0 + i; voxels
// outside the map box read 0 and set *outside.
__device__ inline unsigned long long row_bits(const unsigned long long* __restrict__ plane,
                                              const MapView& M, int ax, int x0, int o1, int o2,
                                              int len, bool* outside) {
  const int A = M.dim_vox[ax];
  const int O1 = ax == 0 ? M.dim_vox[1] : M.dim_vox[0];
  const int O2 = ax == 2 ? M.dim_vox[1] : M.dim_vox[2];
  const int rw = ax == 0 ? M.row_words : (ax == 1 ? M.row_words_y : M.row_words_z);
  if ((unsigned)o1 >= (unsigned)O1 || (unsigned)o2 >= (unsigned)O2) {
    *outside = true;
    return 0ull;
  }
  int xa = x0, xb = x0 + len - 1;
  if (xa < 0 || xb >= A) {
    *outside = true;
    xa = max(xa, 0);
    xb = min(xb, A - 1);
    if (xa > xb) return 0ull;
  }
  const unsigned long long* row = plane + ((size_t)o2 * O1 + o1) * rw;
  const int wa = xa >> 6, wb = xb >> 6, sh = xa & 63;
  const size_t words = ax == 0 ? M.words_x : (ax == 1 ? M.words_y : M.words_z);
  if (!check_index(((size_t)o2 * O1 + o1) * rw + wb < words, M.ctl)) return 0ull;
  unsigned long long win = __ldg(row + wa) >> sh;
  if (wb != wa) win |= __ldg(row + wb) << (64 - sh);
  const int n = xb - xa + 1;
  if (n < 64) win &= (1ull << n) - 1ull;
  return win << (xa - x0);
}

// One run-table entry: the fast form (plane-word row offset,
// d0 | len << 16 | axis << 24) or the plain form (d0 | (len | axis << 8) << 16,
// d1 | d2 << 16), d0 along the run's axis, d1 < d2 the other two axes.
struct RunEntry {
  int a, b;
};

// The staged scorer's copy of the tool tables in dynamic shared memory, in
// this order: the direction table (G int4), the arm offsets (3 G short4) and
// the tool runs in fast form (ntool int2, byte offset 40 G).
extern __shared__ int4 af_staged_tab[];

__device__ __forceinline__ int4 dtab_entry(const ToolView& T, int g, bool staged) {
  return staged ? af_staged_tab[g] : __ldg(T.dtab + g);
}

__device__ __forceinline__ short4 arm_entry(const ToolView& T, int i, bool staged) {
  return staged ? reinterpret_cast<const short4*>(af_staged_tab + T.G)[i] : __ldg(T.arm + i);
}

// Run r of the tables; SM: a tool run read from the staged copy.
template <bool FAST, bool SM = false>
__device__ inline RunEntry load_run(const ToolView& T, int r) {
  if (!check_index((unsigned)r < (unsigned)(SM ? T.ntool : T.nruns), T.ctl)) return {0, 0};  // an empty run
  if (FAST) {
    const int2 f = SM ? reinterpret_cast<const int2*>(
                            reinterpret_cast<const char*>(af_staged_tab) + 40 * T.G)[r]
                      : __ldg(T.fruns + r);
    return {f.x, f.y};
  }
  const short4 s = __ldg(T.runs + r);
  return {(int)((uint32_t)(uint16_t)s.x | ((uint32_t)(uint16_t)s.y << 16)),
          (int)((uint32_t)(uint16_t)s.z | ((uint32_t)(uint16_t)s.w << 16))};
}

// Bits of the run of entry e for point P; *len receives the run length.
// `px`, `py`, `pz`: the view with rows along x, y, z (a view kept with x
// rows only is passed for all three; its runs are all along x).
template <bool FAST>
__device__ inline unsigned long long run_bits(const unsigned long long* __restrict__ px,
                                              const unsigned long long* __restrict__ py,
                                              const unsigned long long* __restrict__ pz,
                                              const MapView& M, RunEntry e, const Pt& P,
                                              int* len, bool* outside) {
  if (FAST) {
    const int d0 = (int)(short)(e.b & 0xffff), n = (e.b >> 16) & 0xFF, ax = (e.b >> 24) & 3;
    const int xa = (ax == 0 ? P.px : (ax == 1 ? P.py : P.pz)) + d0;
    const int row = (ax == 0 ? P.row : (ax == 1 ? P.rowy : P.rowz)) + e.a;
    const unsigned long long* plane = ax == 0 ? px : (ax == 1 ? py : pz);
    const int wa = xa >> 6, wb = (xa + n - 1) >> 6, sh = xa & 63;
    const size_t words = ax == 0 ? M.words_x : (ax == 1 ? M.words_y : M.words_z);
    if (!check_index(row + wa >= 0 && (size_t)(row + wb) < words, M.ctl)) {
      *len = n;
      return 0ull;
    }
    unsigned long long win = __ldg(plane + row + wa) >> sh;
    if (wb != wa) win |= __ldg(plane + row + wb) << (64 - sh);
    if (n < 64) win &= (1ull << n) - 1ull;
    *len = n;
    return win;
  }
  const int d0 = (int)(short)(e.a & 0xffff), n = (int)(((uint32_t)e.a >> 16) & 0xFF),
            ax = (int)(((uint32_t)e.a >> 24) & 3);
  const int d1 = (int)(short)(e.b & 0xffff), d2 = (int)(short)((uint32_t)e.b >> 16);
  *len = n;
  // (a, o1, o2) coordinates of the run's first voxel
  const int a0 = (ax == 0 ? P.px : (ax == 1 ? P.py : P.pz)) + d0;
  const int o1 = (ax == 0 ? P.py : P.px) + d1;
  const int o2 = (ax == 2 ? P.py : P.pz) + d2;
  return row_bits(ax == 0 ? px : (ax == 1 ? py : pz), M, ax, a0, o1, o2, n, outside);
}

// Walks runs [r0, r1) of the tables a warp step (32 runs, one per lane) at a
// time; the caller's `step(entry, valid)` returns true to stop the walk.
template <bool FAST, bool SM, class F>
__device__ inline void walk_runs(const ToolView& T, int r0, int r1, int lane, F&& step) {
  for (int b = r0; b < r1; b += 32) {
    const int r = b + lane;
    const RunEntry e = r < r1 ? load_run<FAST, SM>(T, r) : RunEntry{0, 0};
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
  if (!check_index(w < M.words_x, M.ctl)) return false;
  return (__ldg(plane + w) >> (x & 63)) & 1ull;
}

// Occupied tool voxels of direction g at point P, saturated at `sat`.
// SM: the direction table and the tool runs are staged in shared memory.
template <bool FAST, bool SM = false>
__device__ inline int tool_count(const MapView& M, const ToolView& T, int g, const Pt& P, int sat,
                                 int lane) {
  const int4 dt = dtab_entry(T, g, SM);
  int total = 0;
  walk_runs<FAST, SM && FAST>(T, dt.x, dt.y, lane, [&](RunEntry e, bool valid) {
    int c = 0;
    if (valid) {
      int len;
      bool out = false;
      c = __popcll(run_bits<FAST>(M.occ, M.occ_y, M.occ_z, M, e, P, &len, &out));
    }
    total += __reduce_add_sync(0xffffffffu, c);
    return total >= sat;
  });
  return total >= sat ? sat : total;
}

// Occupied tool voxels of directions g1 and g2 at point P, each saturated at
// `sat`, counted side by side: lanes 0-15 walk g1's runs and lanes 16-31
// g2's, two runs per lane per step, so both counts take the round trips of
// one. Each count is what tool_count returns for its direction: every run is
// counted until the running sum reaches `sat`.
template <bool FAST, bool SM>
__device__ inline int2 tool_count2(const MapView& M, const ToolView& T, int g1, int g2,
                                   const Pt& P, int sat, int lane) {
  const int half = lane >> 4, hl = lane & 15;
  const int4 dt = dtab_entry(T, half ? g2 : g1, SM);
  const int len1 = __shfl_sync(0xffffffffu, dt.y - dt.x, 0);
  const int len2 = __shfl_sync(0xffffffffu, dt.y - dt.x, 16);
  int t1 = 0, t2 = 0;
  for (int b = 0; (b < len1 && t1 < sat) || (b < len2 && t2 < sat); b += 32) {
    const bool mine = half ? (t2 < sat) : (t1 < sat);
    int c = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = dt.x + b + hl + 16 * j;
      if (mine && r < dt.y) {
        int len;
        bool out = false;
        c += __popcll(run_bits<FAST>(M.occ, M.occ_y, M.occ_z, M, load_run<FAST, SM>(T, r), P,
                                     &len, &out));
      }
    }
    t1 += __reduce_add_sync(0xffffffffu, half ? 0 : c);
    t2 += __reduce_add_sync(0xffffffffu, half ? c : 0);
  }
  return make_int2(t1 >= sat ? sat : t1, t2 >= sat ? sat : t2);
}

// The three arm samples of direction g (one lane): clear iff none is
// occupied or unknown. All nine loads are issued together (no short
// circuit), so the screen costs two dependent round trips, not up to nine.
template <bool FAST, bool SM = false>
__device__ inline bool arm_clear(const MapView& M, const ToolView& T, int g, const Pt& P) {
  short4 a[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) a[s] = arm_entry(T, 3 * g + s, SM);
  bool blocked = false;
#pragma unroll
  for (int s = 0; s < 3; ++s)
    blocked = blocked | bit_at<FAST>(M.occ, M, P, a[s]) | !bit_at<FAST>(M.known, M, P, a[s]);
  return !blocked;
}

// Corridor of direction g: any occupied voxel (strict: or unknown) blocks.
template <bool FAST, bool SM = false>
__device__ inline bool corridor_blocked(const MapView& M, const ToolView& T, int g, const Pt& P,
                                        int lane) {
  const int4 dt = dtab_entry(T, g, SM);
  bool blocked = false;
  walk_runs<FAST, false>(T, dt.z, dt.w, lane, [&](RunEntry e, bool valid) {
    bool h = false;
    if (valid) {
      int len;
      bool out = false;
      h = run_bits<FAST>(M.occ, M.occ_y, M.occ_z, M, e, P, &len, &out) != 0ull;
      if (T.strict && !h) {  // strict corridors run along x (the known view's rows)
        const unsigned long long kb = run_bits<FAST>(M.known, M.known, M.known, M, e, P, &len, &out);
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

// The normal filter of Sec. 3.4 as a candidate test.
struct NormalFilter {
  float n0, n1, n2;
  __device__ bool operator()(const ToolView& T, int g) const { return candidate(T, g, n0, n1, n2); }
};

// The candidate loop of one point: lowest-index minimum of the direction
// scores, with exact early exits; `cand(T, g)` says whether direction g is a
// candidate of the point. Returns (best score, best index), (n_c + 2, -1)
// without candidates.
// SM: the direction table, the arm offsets and the tool runs are staged in
// shared memory (af_staged_tab).
// Once a search has a best (score <= n_c), it takes the remaining arm-clear
// candidates two at a time (tool_count2, FAST path): a long search waits on
// half as many tool-count round trips. Both counts are saturated at the score
// to beat before the pair and the pair is then decided in index order, so the
// result is the sequential one.
template <bool FAST, class Cand, bool SM = false>
__device__ inline int2 best_direction(const MapView& M, const ToolView& T, const Pt& P,
                                      const Cand& cand_of, int lane) {
  const int nc = T.n_c;
  int bscore = nc + 2, best = -1;
  for (int gb = 0; gb < T.G && bscore != 0; gb += 32) {
    // lane-parallel screen: candidates, and the arm samples of each candidate
    const bool cand = cand_of(T, gb + lane);
    unsigned mask = __ballot_sync(0xffffffffu, cand);
    const unsigned arm_ok = __ballot_sync(0xffffffffu, cand && arm_clear<FAST, SM>(M, T, gb + lane, P));
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
      const unsigned rest = mask & arm_ok;  // arm-clear candidates after g in this group
      if (FAST && bscore <= nc && rest) {
        // g and the next arm-clear candidate g2; the candidates between them
        // are arm-blocked (n_c + 1) and cannot beat the best there is
        const int bit2 = __ffs(rest) - 1;
        const int g2 = gb + bit2;
        mask &= ~((2u << bit2) - 1u);
        const int2 c = tool_count2<FAST, SM>(M, T, g, g2, P, bscore, lane);
        if (c.x < bscore && !corridor_blocked<FAST, SM>(M, T, g, P, lane)) {
          bscore = c.x;
          best = g;
          if (bscore == 0) break;
        }
        // c.y saturated at the score before g: at or above any score after it
        if (c.y < bscore && !corridor_blocked<FAST, SM>(M, T, g2, P, lane)) {
          bscore = c.y;
          best = g2;
        }
        if (bscore == 0) break;
        continue;
      }
      if (bscore <= nc) {
        // improves only if not blocked and strictly fewer collisions
        const int cnt = tool_count<FAST, SM>(M, T, g, P, bscore, lane);
        if (cnt >= bscore) continue;
        if (corridor_blocked<FAST, SM>(M, T, g, P, lane)) continue;
        bscore = cnt;
        best = g;
      } else {
        // nothing unblocked yet: any unblocked direction improves
        if (corridor_blocked<FAST, SM>(M, T, g, P, lane)) {
          if (best < 0) {
            bscore = nc + 1;
            best = g;
          }
          continue;
        }
        bscore = tool_count<FAST, SM>(M, T, g, P, nc, lane);
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
template <bool FAST, class Cand, bool SM = false>
__device__ inline int2 best_direction_budget(const MapView& M, const ToolView& T, const Pt& P,
                                             const Cand& cand_of, int lane, int budget,
                                             int* next) {
  const int nc = T.n_c;
  int bscore = nc + 2, best = -1, spent = 0;
  *next = -1;
  for (int gb = 0; gb < T.G && bscore != 0; gb += 32) {
    const bool cand = cand_of(T, gb + lane);
    unsigned mask = __ballot_sync(0xffffffffu, cand);
    const unsigned arm_ok = __ballot_sync(0xffffffffu, cand && arm_clear<FAST, SM>(M, T, gb + lane, P));
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
        const int cnt = tool_count<FAST, SM>(M, T, g, P, bscore, lane);
        if (cnt >= bscore) continue;
        if (corridor_blocked<FAST, SM>(M, T, g, P, lane)) continue;
        bscore = cnt;
        best = g;
      } else {
        if (corridor_blocked<FAST, SM>(M, T, g, P, lane)) {
          if (best < 0) {
            bscore = nc + 1;
            best = g;
          }
          continue;
        }
        bscore = tool_count<FAST, SM>(M, T, g, P, nc, lane);
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
