// af_soft.cu -- the differentiable form: soft clearance of (point, direction)
// pairs, its adjoint, fused gradient-ascent refinement, and the SDF views
// they sample.
//
// Soft clearance of a pair (not in the paper; a smooth companion of the tool /
// corridor test of Sec. 3.4): the approach axis from surface point s along
// u = (u0 + alpha t1 + beta t2) / |.| is sampled at a_j = h + j v; sample j
// contributes phi_j = SDF(x_j) - margin_j (tool radius up to the tool length
// L, corridor radius beyond it; samples inside the self-exclusion radius are
// skipped), and C = -tau_s log sum_j exp(-phi_j / tau_s). SDF is trilinear
// interpolation of the TSDF (Sec. 3.2) over voxel centres, tau where
// unobserved.
//
// Views. The hashed map is flattened twice, lazily and only when the map has
// changed since the last build:
//  * dense : one FP32 SDF per voxel of the map box, row-major (x fastest);
//  * cells : for every interpolation cell (low corner from one voxel below
//            the box to its last voxel) its 8 corner values as two float4,
//            (c000, c100, c010, c110) then (c001, c101, c011, c111), so a
//            sample costs ONE 32-byte sector read. 8x the dense view's size
//            (3.7 GB for a 8 x 8 x 14 m box at 2 cm), traded for sector
//            efficiency -- the memory is there on this part.
//
// Precision. The sample's cell is an integer decided by floating point; it is
// decided in single precision in a fixed order of correctly rounded
// operations (the CPU oracle takes the same decision). The point's position
// is split into its cell I and the offset r in it, so sample positions
// r + (h / v + j) u carry rounding relative to the lever arm, not to the
// distance from the map origin -- which keeps central differences of C in
// single precision meaningful. Interpolation, softmin and gradient use FMA
// and exp2 / log2 freely.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "af_internal.cuh"

namespace af {

// ---------------------------------------------------------------------------
// View builds
// ---------------------------------------------------------------------------

__global__ void k_fill(float* __restrict__ out, size_t n, float value) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = value;
}

// Dense SDF of every allocated brick: S / (w 2^20) divided in double and
// rounded to single precision; tau where w = 0.
__global__ void __launch_bounds__(256) k_dense_view(MapView M, float* __restrict__ dense) {
  const uint32_t count = min(__ldcg(&M.ctl->pool_count), M.pool_blocks);
  const size_t X = (size_t)M.dim_vox[0], Y = (size_t)M.dim_vox[1];
  for (uint32_t b = blockIdx.x; b < count; b += gridDim.x) {
    const uint64_t key = M.bkey[b];
    const size_t bx = (size_t)(key & 0x1FFFFF) * 8, by = (size_t)((key >> 21) & 0x1FFFFF) * 8,
                 bz = (size_t)(key >> 42) * 8;
    for (int l = threadIdx.x; l < kBrickVox; l += blockDim.x) {
      const unsigned long long word = __ldcg(M.vox + (size_t)b * kBrickVox + l);
      const unsigned long long w = word & kWMask;
      const long long S = word_S(word);
      const float d = w ? __double2float_rn((double)S / ((double)w * 1048576.0)) : M.tau;
      dense[((bz + (l >> 6)) * Y + by + ((l >> 3) & 7)) * X + bx + (l & 7)] = d;
    }
  }
}

__device__ inline float dense_at(const float* __restrict__ dense, int x, int y, int z, int X,
                                 int Y, int Z, float tau) {
  if (x < 0 || y < 0 || z < 0 || x >= X || y >= Y || z >= Z) return tau;
  return dense[((size_t)z * Y + y) * X + x];
}

// Corner records of every cell whose low corner lies in [-1, dim) per axis.
__global__ void __launch_bounds__(256) k_cell_view(const float* __restrict__ dense, int X, int Y,
                                                   int Z, float tau, float4* __restrict__ cells) {
  const size_t NX = (size_t)X + 1, NY = (size_t)Y + 1, n = NX * NY * ((size_t)Z + 1);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % NX) - 1, y = (int)((i / NX) % NY) - 1, z = (int)(i / (NX * NY)) - 1;
    float c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      c[k] = dense_at(dense, x + (k & 1), y + ((k >> 1) & 1), z + (k >> 2), X, Y, Z, tau);
    cells[2 * i] = make_float4(c[0], c[1], c[2], c[3]);
    cells[2 * i + 1] = make_float4(c[4], c[5], c[6], c[7]);
  }
}

// ---------------------------------------------------------------------------
// Pair geometry, single precision in a fixed order
// ---------------------------------------------------------------------------

// Orthonormal tangent basis (t1, t2) of the unit vector n (Duff et al. 2017,
// "Building an orthonormal basis, revisited").
__device__ inline void onb(const float n[3], float t1[3], float t2[3]) {
  const float sg = n[2] >= 0.0f ? 1.0f : -1.0f;
  const float a = __fdiv_rn(-1.0f, __fadd_rn(sg, n[2]));
  const float b = __fmul_rn(__fmul_rn(n[0], n[1]), a);
  t1[0] = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sg, n[0]), n[0]), a));
  t1[1] = __fmul_rn(sg, b);
  t1[2] = -__fmul_rn(sg, n[0]);
  t2[0] = b;
  t2[1] = __fadd_rn(sg, __fmul_rn(__fmul_rn(n[1], n[1]), a));
  t2[2] = -n[1];
}

// The point's cell on the sample grid (g = x / v - 1/2) and its offset r in
// it, once per pair. `ok` is false for a point whose cell is not a usable
// integer (then every sample reads as outside the view).
struct PointCell {
  float I[3], r[3];
  bool finite, ok;
};

__device__ inline PointCell point_cell(const SoftView& S, const float s[3]) {
  PointCell pc;
  pc.finite = isfinite(s[0]) && isfinite(s[1]) && isfinite(s[2]);
  pc.ok = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float o = __fsub_rn(__fdiv_rn(s[i], S.v), 0.5f);
    pc.I[i] = floorf(o);
    pc.r[i] = __fsub_rn(o, pc.I[i]);
    pc.ok = pc.ok && fabsf(pc.I[i]) < 1.0e9f;
  }
  return pc;
}

// The direction of (alpha, beta) around u0 and the standoff in voxels.
struct Dir {
  float u[3];  // unit direction
  float e;     // h / v
  float inq;   // 1 / |u0 + alpha t1 + beta t2|
  bool finite;
};

__device__ inline Dir make_dir(const SoftView& S, const float u0[3], const float t1[3],
                               const float t2[3], float al, float be, float h) {
  Dir d;
  float q[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    q[i] = __fadd_rn(__fadd_rn(u0[i], __fmul_rn(al, t1[i])), __fmul_rn(be, t2[i]));
  const float nq = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])),
                                        __fmul_rn(q[2], q[2])));
#pragma unroll
  for (int i = 0; i < 3; ++i) d.u[i] = __fdiv_rn(q[i], nq);
  d.e = __fdiv_rn(h, S.v);
  d.inq = 1.0f / nq;
  d.finite = isfinite(al) && isfinite(be) && isfinite(h) && isfinite(u0[0]) &&
             isfinite(u0[1]) && isfinite(u0[2]);
  return d;
}

// Cell of sample j: false when the cell lies outside the view (all corners
// read tau). f receives the fractional position in the cell; *idx the record
// index (dense view) or the cell's brick in the brick grid, *loc then its cell
// within the brick (sparse view).
template <bool SPARSE>
__device__ inline bool sample_cell(const SoftView& S, const PointCell& pc, const Dir& d, int j,
                                   float f[3], uint32_t* idx, uint32_t* loc) {
  const float t = __fadd_rn(d.e, (float)j);
  int c[3];
  bool in = pc.ok;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float l = __fadd_rn(pc.r[i], __fmul_rn(t, d.u[i]));
    const float fl = floorf(l);
    f[i] = l - fl;  // exact
    const bool ok = fabsf(l) < 1.0e7f;
    const int base = SPARSE ? S.glo[i] : S.lo[i];
    const int lim = SPARSE ? 8 * S.gdim[i] : S.ncell[i];
    c[i] = ok ? (int)pc.I[i] + (int)fl - base : -1;
    in = in && ok && (unsigned)c[i] < (unsigned)lim;
  }
  if (SPARSE) {
    *idx = ((uint32_t)(c[2] >> 3) * (uint32_t)S.gdim[1] + (uint32_t)(c[1] >> 3)) *
               (uint32_t)S.gdim[0] + (uint32_t)(c[0] >> 3);
    *loc = (uint32_t)((c[0] & 7) | ((c[1] & 7) << 3) | ((c[2] & 7) << 6));
  } else {
    *idx = ((uint32_t)c[2] * (uint32_t)S.ncell[1] + (uint32_t)c[1]) * (uint32_t)S.ncell[0] +
           (uint32_t)c[0];
    *loc = 0;
  }
  return in;
}

__device__ inline float lerp(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

__device__ inline float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ inline float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Pairs are split across kLanes adjacent lanes: lane g of a pair's group
// takes the samples j0 + g, j0 + g + kLanes, ... and the group merges its
// partial softmin states in a fixed tree onto its first lane, whose result is
// broadcast. Every soft kernel uses the same split, so a pair's C is the same
// bit for bit whichever kernel computes it.
constexpr int kLanes = 4;
constexpr unsigned kFull = 0xffffffffu;

// Softmin state over samples. With FIXED the weights are taken against a
// fixed lower bound `ref` of every phi (no rescaling; the host picks FIXED
// only when the exponents cannot underflow), otherwise against the running
// minimum. m = min phi, Z = sum of exp(-(phi - base) / tau_s), and with GRAD
// the weighted sums sum w_j (h/v + j) G_j and sum w_j G_j of the per-voxel
// SDF gradients G_j.
template <bool GRAD, bool FIXED>
struct Softmin {
  float m = INFINITY, Z = 0.f;
  float at[3] = {0.f, 0.f, 0.f}, a0[3] = {0.f, 0.f, 0.f};

  __device__ inline void scale(float sc) {
    Z *= sc;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        at[i] *= sc;
        a0[i] *= sc;
      }
    }
  }

  __device__ inline void add(float phi, float t, const float G[3], const SoftView& S) {
    float w;
    if (FIXED) {
      w = ex2((S.ref - phi) * S.k2);
      m = fminf(m, phi);
    } else if (phi < m) {
      scale(ex2((phi - m) * S.k2));
      m = phi;
      w = 1.0f;
    } else {
      w = ex2((m - phi) * S.k2);
    }
    Z += w;
    if (GRAD) {
      const float wt = w * t;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        at[i] = __fmaf_rn(wt, G[i], at[i]);
        a0[i] = __fmaf_rn(w, G[i], a0[i]);
      }
    }
  }

  // this <- this (+) o
  __device__ inline void merge(const Softmin& o, float k2) {
    float sa = 1.f, sb = 1.f;
    const float mm = fminf(m, o.m);
    if (!FIXED) {
      sa = m == INFINITY ? 0.f : ex2((mm - m) * k2);
      sb = o.m == INFINITY ? 0.f : ex2((mm - o.m) * k2);
    }
    Z = Z * sa + o.Z * sb;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        at[i] = at[i] * sa + o.at[i] * sb;
        a0[i] = a0[i] * sa + o.a0[i] * sb;
      }
    }
    m = mm;
  }

  // Merge the kLanes partial states of the group; every lane gets the result.
  __device__ inline void reduce(float k2) {
#pragma unroll
    for (int off = kLanes / 2; off >= 1; off >>= 1) {
      Softmin o;
      o.m = __shfl_down_sync(kFull, m, off, kLanes);
      o.Z = __shfl_down_sync(kFull, Z, off, kLanes);
      if (GRAD) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          o.at[i] = __shfl_down_sync(kFull, at[i], off, kLanes);
          o.a0[i] = __shfl_down_sync(kFull, a0[i], off, kLanes);
        }
      }
      merge(o, k2);
    }
    m = __shfl_sync(kFull, m, 0, kLanes);
    Z = __shfl_sync(kFull, Z, 0, kLanes);
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        at[i] = __shfl_sync(kFull, at[i], 0, kLanes);
        a0[i] = __shfl_sync(kFull, a0[i], 0, kLanes);
      }
    }
  }
};

// One corner record, 32 bytes, in one 256-bit read-only load.
__device__ inline void load_cell(const SoftView& S, size_t idx, float4& lo, float4& hi) {
  const float4* p = S.cells + 2 * (size_t)idx;
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z),
        "=f"(hi.w)
      : "l"(p));
}

// Trilinear value (and with GRAD its per-voxel gradient) of one record.
template <bool GRAD>
__device__ inline float trilinear(const float4& lo, const float4& hi, const float f[3],
                                  float G[3]) {
  const float dx00 = lo.y - lo.x, dx10 = lo.w - lo.z, dx01 = hi.y - hi.x, dx11 = hi.w - hi.z;
  const float a00 = __fmaf_rn(f[0], dx00, lo.x), a10 = __fmaf_rn(f[0], dx10, lo.z);
  const float a01 = __fmaf_rn(f[0], dx01, hi.x), a11 = __fmaf_rn(f[0], dx11, hi.z);
  const float dy0 = a10 - a00, dy1 = a11 - a01;
  const float b0 = __fmaf_rn(f[1], dy0, a00), b1 = __fmaf_rn(f[1], dy1, a01);
  if (GRAD) {
    G[0] = lerp(lerp(dx00, dx10, f[1]), lerp(dx01, dx11, f[1]), f[2]);
    G[1] = lerp(dy0, dy1, f[2]);
    G[2] = b1 - b0;
  }
  return __fmaf_rn(f[2], b1 - b0, b0);
}

// Records in flight per lane (NF): the lane computes NF sample cells, issues
// their loads, then folds them into the softmin in sample order, so the
// result does not depend on NF. The field takes 3, the refinement 4
// (measured best; more in flight trade registers for memory parallelism).
constexpr int kInFlightField = 3;
constexpr int kInFlightRefine = 4;

// C of one pair and, with GRAD, dC / d(alpha, beta, h); *cmin = min_j phi_j.
// Called by all kLanes lanes of the pair's group (lane g of it); with
// `live` false the lane samples nothing.
template <bool GRAD, bool FIXED, bool SPARSE, int NF>
__device__ inline float soft_eval(const SoftView& S, const PointCell& pc, const Dir& d,
                                  const float t1[3], const float t2[3], bool live, int g,
                                  float* ga, float* gb, float* gh, float* cmin) {
  Softmin<GRAD, FIXED> sm;
  if (live) {
    for (int j = S.j0 + g; j <= S.J; j += NF * kLanes) {
      float f[NF][3];
      uint32_t id[NF], loc[NF];
      size_t rec[NF];
      bool has[NF], in[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        has[q] = j + q * kLanes <= S.J;
        in[q] = has[q] && sample_cell<SPARSE>(S, pc, d, j + q * kLanes, f[q], &id[q], &loc[q]);
        rec[q] = id[q];
      }
      if (SPARSE) {  // the slots of the cells' bricks first, then the records
        uint32_t slot[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) slot[q] = in[q] ? __ldg(S.bgrid + id[q]) : kNoBlock;
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          in[q] = in[q] && slot[q] != kNoBlock;
          rec[q] = (size_t)slot[q] * kBrickVox + loc[q];
        }
      }
      float4 lo[NF], hi[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q)
        if (in[q]) load_cell(S, rec[q], lo[q], hi[q]);
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        if (!has[q]) break;
        const int jq = j + q * kLanes;
        float G[3] = {0.f, 0.f, 0.f};
        const float D = in[q] ? trilinear<GRAD>(lo[q], hi[q], f[q], G) : S.tau;
        sm.add(D - (jq <= S.jt ? S.r : S.r_corr), d.e + (float)jq, G, S);
      }
    }
  }
  sm.reduce(S.k2);
  const float C = (FIXED ? S.ref : sm.m) - S.ln2_tau_s * lg2(sm.Z);
  *cmin = sm.m;
  if (GRAD) {
    // du/dalpha = (t1 - u (u . t1)) / |q|, likewise for beta with t2
    const float iz = 1.0f / sm.Z;
    const float au = sm.at[0] * d.u[0] + sm.at[1] * d.u[1] + sm.at[2] * d.u[2];
    const float ut1 = d.u[0] * t1[0] + d.u[1] * t1[1] + d.u[2] * t1[2];
    const float ut2 = d.u[0] * t2[0] + d.u[1] * t2[1] + d.u[2] * t2[2];
    const float at1 = sm.at[0] * t1[0] + sm.at[1] * t1[1] + sm.at[2] * t1[2];
    const float at2 = sm.at[0] * t2[0] + sm.at[1] * t2[1] + sm.at[2] * t2[2];
    *ga = (at1 - au * ut1) * d.inq * iz;
    *gb = (at2 - au * ut2) * d.inq * iz;
    *gh = (sm.a0[0] * d.u[0] + sm.a0[1] * d.u[1] + sm.a0[2] * d.u[2]) * iz / S.v;
  }
  return C;
}

__device__ inline void load3(const float* __restrict__ p, size_t i, float o[3]) {
  o[0] = __ldg(p + 3 * i);
  o[1] = __ldg(p + 3 * i + 1);
  o[2] = __ldg(p + 3 * i + 2);
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_soft_seed(const float* __restrict__ nrm, uint32_t m,
                                                   const float* __restrict__ table, uint32_t K,
                                                   float* __restrict__ u0) {
  const size_t n = (size_t)m * K;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float nv[3], e[3], t1[3], t2[3];
    load3(nrm, i / K, nv);
    load3(table, i % K, e);
    onb(nv, t1, t2);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      u0[3 * i + k] = __fadd_rn(__fadd_rn(__fmul_rn(e[0], t1[k]), __fmul_rn(e[1], t2[k])),
                                __fmul_rn(e[2], nv[k]));
  }
}

// Pair groups of a warp, walked so that every lane of the warp takes the same
// number of iterations (the group merges are warp-wide shuffles).
struct GroupWalk {
  size_t first, stride;
  int g, slot;
  __device__ GroupWalk() {
    const int lane = threadIdx.x & 31;
    g = lane % kLanes;
    slot = lane / kLanes;
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
    first = warp * (32 / kLanes);
    stride = warps * (32 / kLanes);
  }
};

template <bool GRAD, bool FIXED, bool SPARSE>
__global__ void __launch_bounds__(128) k_soft(SoftView S, const float* __restrict__ pts,
                                              uint32_t per_point, const float* __restrict__ u0,
                                              const float* __restrict__ alpha,
                                              const float* __restrict__ beta,
                                              const float* __restrict__ hh, uint64_t n,
                                              const float* __restrict__ gc, float* __restrict__ c,
                                              float* __restrict__ cmin, float* __restrict__ ga,
                                              float* __restrict__ gb, float* __restrict__ gh) {
  const GroupWalk w;
  for (size_t base = w.first; base < n; base += w.stride) {
    const size_t i0 = base + w.slot;
    const bool act = i0 < n;
    const size_t i = act ? i0 : n - 1;
    float s[3], u[3], t1[3], t2[3];
    load3(pts, i / per_point, s);
    load3(u0, i, u);
    onb(u, t1, t2);
    const PointCell pc = point_cell(S, s);
    const Dir d = make_dir(S, u, t1, t2, __ldg(alpha + i), __ldg(beta + i), __ldg(hh + i));
    const bool fin = pc.finite && d.finite;
    float da, db, dh, mn;
    float C = soft_eval<GRAD, FIXED, SPARSE, kInFlightField>(S, pc, d, t1, t2, fin && act, w.g,
                                                             &da, &db, &dh, &mn);
    if (!act || w.g != 0) continue;
    if (!fin) C = mn = da = db = dh = NAN;
    if (c) c[i] = C;
    if (cmin) cmin[i] = mn;
    if (GRAD) {
      const float gg = gc ? __ldg(gc + i) : 1.0f;
      if (ga) ga[i] = gg * da;
      if (gb) gb[i] = gg * db;
      if (gh) gh[i] = gg * dh;
    }
  }
}

// `steps` ascent steps on C per pair in registers, then C at the final state.
// The group's lanes update identical copies of (alpha, beta, h).
template <bool FIXED, bool SPARSE>
__global__ void __launch_bounds__(128) k_soft_refine(SoftView S, RefineArgs R,
                                                     const float* __restrict__ pts,
                                                     uint32_t per_point,
                                                     const float* __restrict__ u0,
                                                     float* __restrict__ alpha,
                                                     float* __restrict__ beta,
                                                     float* __restrict__ hh, uint64_t n,
                                                     float* __restrict__ c,
                                                     float* __restrict__ cmin) {
  const GroupWalk w;
  for (size_t base = w.first; base < n; base += w.stride) {
    const size_t i0 = base + w.slot;
    const bool act = i0 < n;
    const size_t i = act ? i0 : n - 1;
    float s[3], u[3], t1[3], t2[3];
    load3(pts, i / per_point, s);
    load3(u0, i, u);
    onb(u, t1, t2);
    const PointCell pc = point_cell(S, s);
    float al = alpha[i], be = beta[i], h = hh[i];
    // a pair that is not finite (e.g. a point with no start) samples nothing
    const bool fin = pc.finite && make_dir(S, u, t1, t2, al, be, h).finite;
    for (int k = 0; k < R.steps; ++k) {
      const Dir d = make_dir(S, u, t1, t2, al, be, h);
      const bool live = fin && act && d.finite;
      float da, db, dh, mn;
      soft_eval<true, FIXED, SPARSE, kInFlightRefine>(S, pc, d, t1, t2, live, w.g, &da, &db, &dh,
                                                      &mn);
      if (live) {
        al = __fmaf_rn(R.lr_dir, da, al);
        be = __fmaf_rn(R.lr_dir, db, be);
        h = fminf(fmaxf(__fmaf_rn(R.lr_h, dh, h), 0.0f), R.h_max);
      }
    }
    const Dir d = make_dir(S, u, t1, t2, al, be, h);
    const bool ok = fin && d.finite;
    float mn;
    float C = soft_eval<false, FIXED, SPARSE, kInFlightRefine>(S, pc, d, t1, t2, ok && act, w.g,
                                                                nullptr, nullptr, nullptr, &mn);
    if (!act || w.g != 0) continue;
    if (!ok) C = mn = al = be = h = NAN;
    alpha[i] = al;
    beta[i] = be;
    hh[i] = h;
    c[i] = C;
    if (cmin) cmin[i] = mn;
  }
}

// Start of each point's refinement from the plain path's result: the best
// direction of an ACCESSIBLE point, NaN otherwise (refinement skips it).
__global__ void __launch_bounds__(256) k_soft_start(const uint8_t* __restrict__ label,
                                                    const int16_t* __restrict__ best, uint32_t m,
                                                    const float* __restrict__ dirs, int G,
                                                    float* __restrict__ u0) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < m; p += gridDim.x * blockDim.x) {
    const int b = best[p];
    const bool ok = label[p] == 1 && b >= 0 && b < G;
#pragma unroll
    for (int d = 0; d < 3; ++d) u0[3 * p + d] = ok ? __ldg(dirs + 3 * b + d) : NAN;
  }
}

// Per point: the index (within the point's pairs) and value of the largest C,
// lowest index on ties, -1 when every C is NaN; optionally that pair's base
// direction (NaN for -1).
__global__ void __launch_bounds__(256) k_soft_best(const float* __restrict__ c, uint64_t n,
                                                   uint32_t per_point, uint64_t points,
                                                   const float* __restrict__ u0,
                                                   int32_t* __restrict__ best_k,
                                                   float* __restrict__ best_c,
                                                   float* __restrict__ best_u0) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < points;
       p += (size_t)gridDim.x * blockDim.x) {
    const size_t a = p * per_point, b = min((size_t)n, a + per_point);
    int32_t k = -1;
    float v = NAN;
    for (size_t i = a; i < b; ++i) {
      const float x = c[i];
      if (x == x && (k < 0 || x > v)) {
        k = (int32_t)(i - a);
        v = x;
      }
    }
    if (best_k) best_k[p] = k;
    if (best_c) best_c[p] = v;
    if (best_u0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) best_u0[3 * p + d] = k >= 0 ? u0[3 * (a + k) + d] : NAN;
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static unsigned grid_for(size_t n, int threads, int num_sms, int per_sm) {
  const size_t want = (n + threads - 1) / threads;
  const size_t cap = (size_t)num_sms * per_sm;
  return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

// ---- the brick-sparse view ----
//
// A cell (low corner c, corners c + {0,1}^3) has corners in the bricks of c
// and the ones above it on each axis, so a cell with a corner in an
// allocated brick B has its low corner in B - e for some e in {0,1}^3; every
// other cell reads tau at all corners. The grid covers the box's bricks and
// one layer below (cells whose low corner lies one voxel below the box);
// each brick of {B - e} gets a slot of 512 corner records, the others none.

// Marks every grid brick B - e (B allocated, e in {0,1}^3) with a slot; one
// thread per (allocated brick, e).
__global__ void __launch_bounds__(256) k_sview_mark(MapView M, uint32_t* __restrict__ bgrid,
                                                    int gx, int gy, uint32_t* __restrict__ keys,
                                                    uint32_t* __restrict__ nslots) {
  const uint32_t count = min(__ldcg(&M.ctl->pool_count), M.pool_blocks);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count * 8u;
       i += gridDim.x * blockDim.x) {
    const uint64_t key = M.bkey[i >> 3];
    const int e = (int)(i & 7u);
    // grid coordinates: box-relative brick + 1 (the layer below the box is 0)
    const int x = (int)(key & 0x1FFFFF) + 1 - (e & 1), y = (int)((key >> 21) & 0x1FFFFF) + 1 - ((e >> 1) & 1),
              z = (int)(key >> 42) + 1 - (e >> 2);
    const uint32_t t = ((uint32_t)z * (uint32_t)gy + (uint32_t)y) * (uint32_t)gx + (uint32_t)x;
    if (atomicCAS(bgrid + t, kNoBlock, kNoBlock - 1u) == kNoBlock) {
      const uint32_t s = atomicAdd(nslots, 1u);
      keys[s] = t;
      bgrid[t] = s;
    }
  }
}

// The 512 corner records of every slot: one CTA of 512 threads per slot, the
// pool indices of the 8 bricks its cells' corners can lie in looked up once.
__global__ void __launch_bounds__(512) k_sview_fill(MapView M, const uint32_t* __restrict__ keys,
                                                    uint32_t nslots, int gx, int gy,
                                                    float4* __restrict__ cells) {
  __shared__ uint32_t s_nb[8];
  const int l = threadIdx.x;
  const int X = M.dim_vox[0], Y = M.dim_vox[1], Z = M.dim_vox[2];
  for (uint32_t s = blockIdx.x; s < nslots; s += gridDim.x) {
    const uint32_t t = keys[s];
    // box-relative brick of the slot's low corners
    const int bx = (int)(t % (uint32_t)gx) - 1, by = (int)((t / (uint32_t)gx) % (uint32_t)gy) - 1,
              bz = (int)(t / ((uint32_t)gx * (uint32_t)gy)) - 1;
    __syncthreads();  // s_nb of the previous slot is no longer read
    if (l < 8) {
      const int x = bx + (l & 1), y = by + ((l >> 1) & 1), z = bz + (l >> 2);
      s_nb[l] = (x >= 0 && y >= 0 && z >= 0 && x * 8 < X && y * 8 < Y && z * 8 < Z)
                    ? lookup_brick(M, pack_brick(x, y, z))
                    : kNoBlock;
    }
    __syncthreads();
    const int vx = bx * 8 + (l & 7), vy = by * 8 + ((l >> 3) & 7), vz = bz * 8 + (l >> 6);
    float c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int x = vx + (k & 1), y = vy + ((k >> 1) & 1), z = vz + (k >> 2);
      float d = M.tau;  // outside the box, unallocated, or w = 0
      if (x >= 0 && y >= 0 && z >= 0 && x < X && y < Y && z < Z) {
        const uint32_t b = s_nb[((x >> 3) - bx) | (((y >> 3) - by) << 1) | (((z >> 3) - bz) << 2)];
        if (b != kNoBlock) {
          const unsigned long long word =
              __ldcg(M.vox + (size_t)b * kBrickVox + ((x & 7) | ((y & 7) << 3) | ((z & 7) << 6)));
          const unsigned long long w = word & kWMask;
          if (w) d = __double2float_rn((double)word_S(word) / ((double)w * 1048576.0));
        }
      }
      c[k] = d;
    }
    float4* rec = cells + 2 * ((size_t)s * kBrickVox + l);
    rec[0] = make_float4(c[0], c[1], c[2], c[3]);
    rec[1] = make_float4(c[4], c[5], c[6], c[7]);
  }
}

cudaError_t launch_sview_mark(const MapView& M, int num_sms, uint32_t* bgrid, size_t gcount,
                              int gx, int gy, uint32_t* keys, uint32_t* nslots, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(bgrid, 0xFF, gcount * 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(nslots, 0, 4, stream);
  if (e != cudaSuccess) return e;
  k_sview_mark<<<num_sms * 8, 256, 0, stream>>>(M, bgrid, gx, gy, keys, nslots);
  return cudaGetLastError();
}

cudaError_t launch_sview_fill(const MapView& M, int num_sms, const uint32_t* keys, uint32_t nslots,
                              int gx, int gy, float4* cells, cudaStream_t stream) {
  if (nslots == 0) return cudaSuccess;
  k_sview_fill<<<(unsigned)std::min<uint32_t>(nslots, (uint32_t)num_sms * 4), 512, 0, stream>>>(
      M, keys, nslots, gx, gy, cells);
  return cudaGetLastError();
}

cudaError_t launch_views(const MapView& M, int num_sms, bool fill, float* dense, float4* cells,
                         cudaStream_t stream) {
  const size_t nd = (size_t)M.dim_vox[0] * M.dim_vox[1] * M.dim_vox[2];
  if (fill) k_fill<<<grid_for(nd, 256, num_sms, 8), 256, 0, stream>>>(dense, nd, M.tau);
  k_dense_view<<<(unsigned)num_sms * 8, 256, 0, stream>>>(M, dense);
  const size_t nc = ((size_t)M.dim_vox[0] + 1) * (M.dim_vox[1] + 1) * (M.dim_vox[2] + 1);
  k_cell_view<<<grid_for(nc, 256, num_sms, 8), 256, 0, stream>>>(dense, M.dim_vox[0], M.dim_vox[1],
                                                                  M.dim_vox[2], M.tau, cells);
  return cudaGetLastError();
}

cudaError_t launch_soft_seed(const float* d_nrm, uint32_t m, const float* d_table, uint32_t K,
                             float* d_u0, int num_sms, cudaStream_t stream) {
  const size_t n = (size_t)m * K;
  if (n == 0) return cudaSuccess;
  k_soft_seed<<<grid_for(n, 256, num_sms, 8), 256, 0, stream>>>(d_nrm, m, d_table, K, d_u0);
  return cudaGetLastError();
}

cudaError_t launch_soft(const SoftView& S, bool grad, const float* pts, uint32_t per_point,
                        const float* u0, const float* al, const float* be, const float* h,
                        uint64_t n, const float* gc, float* c, float* cmin, float* ga,
                        float* gb, float* gh, int num_sms, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const unsigned g = grid_for(n * kLanes, 128, num_sms, 16);
#define AF_SOFT_LAUNCH(GR, FX)                                                                  \
  (S.sparse ? k_soft<GR, FX, true><<<g, 128, 0, stream>>>(S, pts, per_point, u0, al, be, h, n, gc, \
                                                         c, cmin, ga, gb, gh)                    \
            : k_soft<GR, FX, false><<<g, 128, 0, stream>>>(S, pts, per_point, u0, al, be, h, n,   \
                                                          gc, c, cmin, ga, gb, gh))
  if (grad && S.fixed)
    AF_SOFT_LAUNCH(true, true);
  else if (grad)
    AF_SOFT_LAUNCH(true, false);
  else if (S.fixed)
    AF_SOFT_LAUNCH(false, true);
  else
    AF_SOFT_LAUNCH(false, false);
#undef AF_SOFT_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_soft_refine(const SoftView& S, const RefineArgs& R, const float* pts,
                               uint32_t per_point, const float* u0, float* al, float* be,
                               float* h, uint64_t n, float* c, float* cmin, int num_sms,
                               cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const unsigned g = grid_for(n * kLanes, 128, num_sms, 16);
#define AF_REFINE_LAUNCH(FX, SP) \
  k_soft_refine<FX, SP><<<g, 128, 0, stream>>>(S, R, pts, per_point, u0, al, be, h, n, c, cmin)
  if (S.fixed && S.sparse)
    AF_REFINE_LAUNCH(true, true);
  else if (S.fixed)
    AF_REFINE_LAUNCH(true, false);
  else if (S.sparse)
    AF_REFINE_LAUNCH(false, true);
  else
    AF_REFINE_LAUNCH(false, false);
#undef AF_REFINE_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_soft_start(const uint8_t* label, const int16_t* best, uint32_t m,
                              const float* dirs, int G, float* u0, int num_sms,
                              cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  k_soft_start<<<grid_for(m, 256, num_sms, 8), 256, 0, stream>>>(label, best, m, dirs, G, u0);
  return cudaGetLastError();
}

cudaError_t launch_soft_best(const float* c, uint64_t n, uint32_t per_point, const float* u0,
                             int32_t* best_k, float* best_c, float* best_u0, int num_sms,
                             cudaStream_t stream) {
  const uint64_t points = (n + per_point - 1) / per_point;
  if (points == 0) return cudaSuccess;
  k_soft_best<<<grid_for(points, 256, num_sms, 8), 256, 0, stream>>>(c, n, per_point, points, u0,
                                                                      best_k, best_c, best_u0);
  return cudaGetLastError();
}

}  // namespace af
