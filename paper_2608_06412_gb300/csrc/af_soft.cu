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
      const unsigned long long w = word & kWMask, S = word >> kWBits;
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

struct Pair {
  float I[3];          // cell of the point on the sample grid (g = x / v - 1/2)
  float r[3];          // the point's offset in that cell
  float u[3];          // unit direction
  float e;             // h / v
  float dua[3], dub[3];  // du / dalpha, du / dbeta
  bool finite;
};

__device__ inline Pair make_pair(const SoftView& S, const float s[3], const float u0[3],
                                 const float t1[3], const float t2[3], float al, float be,
                                 float h) {
  Pair P;
  float q[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) q[i] = __fadd_rn(__fadd_rn(u0[i], __fmul_rn(al, t1[i])), __fmul_rn(be, t2[i]));
  const float nq = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])),
                                        __fmul_rn(q[2], q[2])));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    P.u[i] = __fdiv_rn(q[i], nq);
    const float o = __fsub_rn(__fdiv_rn(s[i], S.v), 0.5f);
    P.I[i] = floorf(o);
    P.r[i] = __fsub_rn(o, P.I[i]);
  }
  P.e = __fdiv_rn(h, S.v);
  const float ut1 = P.u[0] * t1[0] + P.u[1] * t1[1] + P.u[2] * t1[2];
  const float ut2 = P.u[0] * t2[0] + P.u[1] * t2[1] + P.u[2] * t2[2];
  const float inq = 1.0f / nq;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    P.dua[i] = (t1[i] - P.u[i] * ut1) * inq;
    P.dub[i] = (t2[i] - P.u[i] * ut2) * inq;
  }
  bool fin = isfinite(al) && isfinite(be) && isfinite(h);
#pragma unroll
  for (int i = 0; i < 3; ++i) fin = fin && isfinite(s[i]) && isfinite(u0[i]);
  P.finite = fin;
  return P;
}

// Corner record of sample j: false when the cell lies outside the view (all
// corners read tau). f receives the fractional position in the cell.
__device__ inline bool sample_cell(const SoftView& S, const Pair& P, int j, float f[3],
                                   size_t* idx) {
  const float t = __fadd_rn(P.e, (float)j);
  int c[3];
  bool in = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float l = __fadd_rn(P.r[i], __fmul_rn(t, P.u[i]));
    const float fl = floorf(l);
    f[i] = l - fl;  // exact
    const bool ok = fabsf(l) < 1.0e7f && fabsf(P.I[i]) < 1.0e9f;
    c[i] = ok ? (int)P.I[i] + (int)fl - S.lo[i] : -1;
    in = in && ok && (unsigned)c[i] < (unsigned)S.ncell[i];
  }
  *idx = ((size_t)c[2] * S.ncell[1] + c[1]) * S.ncell[0] + c[0];
  return in;
}

__device__ inline float lerp(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

// Online softmin over the samples; with GRAD also the weighted sums
// sum w_j (h/v + j) G_j and sum w_j G_j of the per-voxel SDF gradients G_j.
template <bool GRAD>
struct Softmin {
  float m = INFINITY, Z = 0.f;
  float at[3] = {0.f, 0.f, 0.f}, a0[3] = {0.f, 0.f, 0.f};

  __device__ inline void add(float phi, float t, const float G[3], float k2) {
    float w;
    if (phi < m) {
      const float sc = exp2f((phi - m) * k2);
      Z *= sc;
      if (GRAD) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          at[i] *= sc;
          a0[i] *= sc;
        }
      }
      m = phi;
      w = 1.0f;
    } else {
      w = exp2f((m - phi) * k2);
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
};

// C of one pair and, with GRAD, dC / d(alpha, beta, h).
template <bool GRAD>
__device__ inline float soft_eval(const SoftView& S, const Pair& P, float* ga, float* gb,
                                  float* gh, float* cmin) {
  Softmin<GRAD> sm;
  for (int j = S.j0; j <= S.J; ++j) {
    const float margin = j <= S.jt ? S.r : S.r_corr;
    float f[3];
    size_t idx;
    float D, G[3] = {0.f, 0.f, 0.f};
    if (sample_cell(S, P, j, f, &idx)) {
      const float4 lo = __ldg(S.cells + 2 * idx), hi = __ldg(S.cells + 2 * idx + 1);
      const float dx00 = lo.y - lo.x, dx10 = lo.w - lo.z, dx01 = hi.y - hi.x, dx11 = hi.w - hi.z;
      const float a00 = __fmaf_rn(f[0], dx00, lo.x), a10 = __fmaf_rn(f[0], dx10, lo.z);
      const float a01 = __fmaf_rn(f[0], dx01, hi.x), a11 = __fmaf_rn(f[0], dx11, hi.z);
      const float dy0 = a10 - a00, dy1 = a11 - a01;
      const float b0 = __fmaf_rn(f[1], dy0, a00), b1 = __fmaf_rn(f[1], dy1, a01);
      D = __fmaf_rn(f[2], b1 - b0, b0);
      if (GRAD) {
        G[0] = lerp(lerp(dx00, dx10, f[1]), lerp(dx01, dx11, f[1]), f[2]);
        G[1] = lerp(dy0, dy1, f[2]);
        G[2] = b1 - b0;
      }
    } else {
      D = S.tau;
    }
    sm.add(D - margin, P.e + (float)j, G, S.k2);
  }
  const float C = sm.m - S.ln2_tau_s * log2f(sm.Z);
  *cmin = sm.m;
  if (GRAD) {
    const float iz = 1.0f / sm.Z;
    *ga = (sm.at[0] * P.dua[0] + sm.at[1] * P.dua[1] + sm.at[2] * P.dua[2]) * iz;
    *gb = (sm.at[0] * P.dub[0] + sm.at[1] * P.dub[1] + sm.at[2] * P.dub[2]) * iz;
    *gh = (sm.a0[0] * P.u[0] + sm.a0[1] * P.u[1] + sm.a0[2] * P.u[2]) * iz / S.v;
  }
  return C;
}

__device__ inline void load3(const float* __restrict__ p, size_t i, float o[3]) {
  o[0] = __ldg(p + 3 * i);
  o[1] = __ldg(p + 3 * i + 1);
  o[2] = __ldg(p + 3 * i + 2);
}

// ---------------------------------------------------------------------------
// Kernels: one thread per pair, pairs of a point adjacent
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

template <bool GRAD>
__global__ void __launch_bounds__(128) k_soft(SoftView S, const float* __restrict__ pts,
                                              uint32_t per_point, const float* __restrict__ u0,
                                              const float* __restrict__ alpha,
                                              const float* __restrict__ beta,
                                              const float* __restrict__ hh, uint64_t n,
                                              const float* __restrict__ gc, float* __restrict__ c,
                                              float* __restrict__ cmin, float* __restrict__ ga,
                                              float* __restrict__ gb, float* __restrict__ gh) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float s[3], u[3], t1[3], t2[3];
    load3(pts, i / per_point, s);
    load3(u0, i, u);
    onb(u, t1, t2);
    const Pair P = make_pair(S, s, u, t1, t2, __ldg(alpha + i), __ldg(beta + i), __ldg(hh + i));
    float da = 0.f, db = 0.f, dh = 0.f, mn;
    float C = soft_eval<GRAD>(S, P, &da, &db, &dh, &mn);
    if (!P.finite) C = mn = da = db = dh = NAN;
    if (c) c[i] = C;
    if (cmin) cmin[i] = mn;
    if (GRAD) {
      const float g = gc ? __ldg(gc + i) : 1.0f;
      if (ga) ga[i] = g * da;
      if (gb) gb[i] = g * db;
      if (gh) gh[i] = g * dh;
    }
  }
}

// `steps` ascent steps on C per pair in registers, then C at the final state.
__global__ void __launch_bounds__(128) k_soft_refine(SoftView S, RefineArgs R,
                                                     const float* __restrict__ pts,
                                                     uint32_t per_point,
                                                     const float* __restrict__ u0,
                                                     float* __restrict__ alpha,
                                                     float* __restrict__ beta,
                                                     float* __restrict__ hh, uint64_t n,
                                                     float* __restrict__ c,
                                                     float* __restrict__ cmin) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float s[3], u[3], t1[3], t2[3];
    load3(pts, i / per_point, s);
    load3(u0, i, u);
    onb(u, t1, t2);
    float al = alpha[i], be = beta[i], h = hh[i];
    for (int k = 0; k < R.steps; ++k) {
      const Pair P = make_pair(S, s, u, t1, t2, al, be, h);
      float da, db, dh, mn;
      soft_eval<true>(S, P, &da, &db, &dh, &mn);
      al = __fmaf_rn(R.lr_dir, da, al);
      be = __fmaf_rn(R.lr_dir, db, be);
      h = fminf(fmaxf(__fmaf_rn(R.lr_h, dh, h), 0.0f), R.h_max);
    }
    const Pair P = make_pair(S, s, u, t1, t2, al, be, h);
    float mn;
    float C = soft_eval<false>(S, P, nullptr, nullptr, nullptr, &mn);
    if (!P.finite) C = mn = al = be = h = NAN;
    alpha[i] = al;
    beta[i] = be;
    hh[i] = h;
    c[i] = C;
    if (cmin) cmin[i] = mn;
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
  const unsigned g = grid_for(n, 128, num_sms, 16);
  if (grad)
    k_soft<true><<<g, 128, 0, stream>>>(S, pts, per_point, u0, al, be, h, n, gc, c, cmin, ga, gb,
                                        gh);
  else
    k_soft<false><<<g, 128, 0, stream>>>(S, pts, per_point, u0, al, be, h, n, nullptr, c, cmin,
                                         nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_soft_refine(const SoftView& S, const RefineArgs& R, const float* pts,
                               uint32_t per_point, const float* u0, float* al, float* be,
                               float* h, uint64_t n, float* c, float* cmin, int num_sms,
                               cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  k_soft_refine<<<grid_for(n, 128, num_sms, 16), 128, 0, stream>>>(S, R, pts, per_point, u0, al,
                                                                    be, h, n, c, cmin);
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
