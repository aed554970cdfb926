// af_projective.cu -- projective TSDF integration, the ablation of Tab. 3
// (Sec. 3.2 of the paper): the comparison the paper makes against
// nvblox-style integration, in which voxels look their distance up in a
// range image instead of being updated from the returns around them.
//
// Per scan, on the caller's stream:
//  k_alloc        (the scan-centric allocation, without cleared-band bricks;
//                 launched by af_integrate_scan_projective in af_host.cu)
//                 bricks overlapped by the cubes of the accepted returns,
//                 listed once each in the map's dirty list
//  k_proj_image   one thread per return: the nearest range in each cell of
//                 a bins x bins octahedral map of sensor-frame directions
//                 (atomicMin on the bits of non-negative floats)
//  k_proj_update  one CTA per listed brick, one thread per voxel: the voxel's
//                 own direction cell gives a range D; d = D - |x - q| unless
//                 the cell is empty or d < -tau, clamped as the map clamps,
//                 added to the voxel word (one writer per voxel per scan)
//  k_bitview      weight cap and occupied / known bits, as after a
//                 scan-centric scan
// The octahedral cells take only +, -, *, / and |.| in a fixed order, so
// the cell of every direction is the same on any IEEE machine.
#include <af.h>

#include <cmath>

#include "af_ctx.cuh"
#include "af_internal.cuh"

namespace af {
namespace {

constexpr unsigned kEmptyCell = 0xFFFFFFFFu;

// Cell of a non-zero direction: (u, w) = (d0, d1) / (|d0| + |d1| + |d2|), the
// lower hemisphere folded onto the corners, N equal cells per axis of [-1, 1].
__device__ inline int octa_cell(float d0, float d1, float d2, int N) {
  const float s = __fadd_rn(__fadd_rn(fabsf(d0), fabsf(d1)), fabsf(d2));
  float u = __fdiv_rn(d0, s), w = __fdiv_rn(d1, s);
  if (d2 < 0.f) {
    const float uu = __fmul_rn(__fsub_rn(1.f, fabsf(w)), u >= 0.f ? 1.f : -1.f);
    const float ww = __fmul_rn(__fsub_rn(1.f, fabsf(u)), w >= 0.f ? 1.f : -1.f);
    u = uu;
    w = ww;
  }
  const float h = __fmul_rn((float)N, 0.5f);
  int bu = (int)floorf(__fmul_rn(__fadd_rn(u, 1.f), h));
  int bw = (int)floorf(__fmul_rn(__fadd_rn(w, 1.f), h));
  bu = bu < 0 ? 0 : (bu >= N ? N - 1 : bu);
  bw = bw < 0 ? 0 : (bw >= N ? N - 1 : bw);
  return bw * N + bu;
}

__global__ void __launch_bounds__(256) k_proj_image(const float* __restrict__ xyz,
                                                     const float4* __restrict__ ret, uint32_t n,
                                                     float q0, float q1, float q2,
                                                     unsigned* __restrict__ img, int N) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float4 p = ret[k];
  if (p.w == 0.f) return;  // not accepted
  const float sx = xyz[3 * k], sy = xyz[3 * k + 1], sz = xyz[3 * k + 2];
  if (sx == 0.f && sy == 0.f && sz == 0.f) return;
  const float b0 = __fsub_rn(p.x, q0), b1 = __fsub_rn(p.y, q1), b2 = __fsub_rn(p.z, q2);
  const float range =
      __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2)));
  atomicMin(img + octa_cell(sx, sy, sz, N), __float_as_uint(range));
}

__global__ void __launch_bounds__(512) k_proj_update(MapView M, Pose P,
                                                      const unsigned* __restrict__ img, int N) {
  const uint32_t count = __ldcg(&M.ctl->dirty_count);
  const int l = threadIdx.x;
  const float q0 = P.r[0][3], q1 = P.r[1][3], q2 = P.r[2][3];
  for (uint32_t d = blockIdx.x; d < count; d += gridDim.x) {
    const uint32_t blk = M.dirty[d];
    const uint64_t key = M.bkey[blk];
    const int jx = (int)(key & 0x1FFFFF) * 8 + (l & 7);
    const int jy = (int)((key >> 21) & 0x1FFFFF) * 8 + ((l >> 3) & 7);
    const int jz = (int)(key >> 42) * 8 + (l >> 6);
    const float e0 = __fsub_rn(voxel_centre(jx + M.dom_vox[0], M.v), q0);
    const float e1 = __fsub_rn(voxel_centre(jy + M.dom_vox[1], M.v), q1);
    const float e2 = __fsub_rn(voxel_centre(jz + M.dom_vox[2], M.v), q2);
    // sensor-frame direction R^T e
    float xs[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      xs[r] = __fadd_rn(__fadd_rn(__fmul_rn(P.r[0][r], e0), __fmul_rn(P.r[1][r], e1)),
                        __fmul_rn(P.r[2][r], e2));
    if (xs[0] == 0.f && xs[1] == 0.f && xs[2] == 0.f) continue;
    const unsigned D = __ldg(img + octa_cell(xs[0], xs[1], xs[2], N));
    if (D == kEmptyCell) continue;
    const float dist =
        __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2)));
    float sd = __fsub_rn(__uint_as_float(D), dist);
    if (sd < -M.tau) continue;  // beyond the truncation behind the surface
    sd = sd < M.dlo ? M.dlo : sd;
    sd = sd > M.tau ? M.tau : sd;
    M.vox[(size_t)blk * kBrickVox + l] += make_word(__float2ll_rn(__fmul_rn(sd, kScale)), 1ull);
  }
}

}  // namespace
}  // namespace af

namespace af {

// The projective update of one scan (the range image, then every voxel of
// the scan's bricks); the allocation and the bit view are launched by the
// caller around it.
cudaError_t launch_projective(const MapView& M, const float* d_xyz, uint32_t n,
                              const float pose[16], const float4* d_ret, unsigned* d_img,
                              uint32_t bins, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_img, 0xFF, (size_t)bins * bins * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (n > 0)
    k_proj_image<<<(n + 255) / 256, 256, 0, s>>>(d_xyz, d_ret, n, pose[3], pose[7], pose[11], d_img,
                                                 (int)bins);
  Pose P;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) P.r[r][c] = pose[4 * r + c];
  k_proj_update<<<num_sms * 4, 512, 0, s>>>(M, P, d_img, (int)bins);
  return cudaGetLastError();
}

}  // namespace af
