// af_noalloc.cu -- af_integrate_scan_noalloc: scan integration for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a real-time loop whose memory
// is budgeted once at start-up, a host framework that owns every device
// buffer through its own arena, or code that must not enter the CUDA
// allocator while other work is in flight. af_create allocates the hashed
// map, so it is out of reach for them. This entry point integrates one scan
// into a dense voxel box that the caller owns and passes in; the only other
// memory it needs -- the per-return scratch that the allocating path keeps in
// its context -- lives in the file-scope device array below. The library
// itself allocates nothing here: no cudaMalloc, no cudaFree, no allocating
// library routine.
//
// The scratch array is AF_NOALLOC_MAX_RETURNS float4 (1 MiB). Every GPU that
// loads the library holds it until the process exits. All calls share it and
// it keeps the last call's contents; each call writes every element it reads
// before reading it, so nothing in it has to start at zero. Calls that
// overlap on the GPU (on different streams, or from several threads) race on
// the array: serialise them.
#include <af.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "af_internal.cuh"

namespace af {
void set_global_error(const char* msg);  // af_last_error(NULL) reports it

namespace {

static __device__ __align__(256) float4 g_scan_scratch[AF_NOALLOC_MAX_RETURNS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float4* g_scratch_dev[kMaxDevices] = {nullptr};  // device address of the array, per device
af_status nfail(af_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_global_error(buf);
  return s;
}

// Device address of the scratch array on the current device; looked up once
// per device (the host-side name of the array is not a device address).
af_status scratch_address(float4** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(AF_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(AF_ERR_CUDA, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scan_scratch);
    if (e != cudaSuccess || !p)
      return nfail(AF_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_dev[dev] = static_cast<float4*>(p);
  }
  *out = g_scratch_dev[dev];
  return AF_OK;
}

struct Box {
  int lo[3];       // domain-relative voxel index of the box corner
  int dim[3];
  unsigned long long* vox;
  uint8_t* flags;
};

__device__ inline bool box_index(const Box& B, int x, int y, int z, size_t* at) {
  x -= B.lo[0];
  y -= B.lo[1];
  z -= B.lo[2];
  if ((unsigned)x >= (unsigned)B.dim[0] || (unsigned)y >= (unsigned)B.dim[1] ||
      (unsigned)z >= (unsigned)B.dim[2])
    return false;
  *at = ((size_t)z * B.dim[1] + y) * B.dim[0] + x;
  return true;
}

__global__ void __launch_bounds__(256) k_na_prepare(MapView M, const float* __restrict__ xyz,
                                                     uint32_t n, Pose P,
                                                     float4* __restrict__ scratch) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float p[3], range;
  int rel[3];
  const bool valid = prepare_return(M, P, xyz[3 * k], xyz[3 * k + 1], xyz[3 * k + 2], p, &range, rel);
  scratch[k] = make_float4(p[0], p[1], p[2], valid ? 1.f : 0.f);
}

// One thread per (return, cube offset), the same arithmetic as the hashed
// path, accumulating into the caller's dense box; cleared-band marks too.
__global__ void __launch_bounds__(256) k_na_integrate(MapView M, const float4* __restrict__ scratch,
                                                       uint32_t n, float q0, float q1, float q2,
                                                       Box B) {
  const int W = 2 * M.m + 1;
  const uint64_t C = (uint64_t)W * W * W;
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t pairs = C * n;
  const uint64_t band = (uint64_t)M.ns * n;
  if (e < pairs) {
    const uint32_t k = (uint32_t)(e / C);
    const int o = (int)(e % C);
    const float4 p = scratch[k];
    if (p.w == 0.f) return;
    const float b0 = __fsub_rn(p.x, q0), b1 = __fsub_rn(p.y, q1), b2 = __fsub_rn(p.z, q2);
    const float range =
        __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2)));
    int i[3];
    // k_na_prepare accepted the return, so its voxel index exists; checked
    // again here so that no index is used unchecked
    if (!(voxel_index(p.x, M, &i[0]) && voxel_index(p.y, M, &i[1]) &&
          voxel_index(p.z, M, &i[2])))
      return;
    const int jx = i[0] - M.dom_vox[0] + o % W - M.m;
    const int jy = i[1] - M.dom_vox[1] + (o / W) % W - M.m;
    const int jz = i[2] - M.dom_vox[2] + o / (W * W) - M.m;
    size_t at;
    if (!box_index(B, jx, jy, jz, &at)) return;
    const float x0 = voxel_centre(jx + M.dom_vox[0], M.v);
    const float x1 = voxel_centre(jy + M.dom_vox[1], M.v);
    const float x2 = voxel_centre(jz + M.dom_vox[2], M.v);
    const float a0 = __fsub_rn(x0, p.x), a1 = __fsub_rn(x1, p.y), a2 = __fsub_rn(x2, p.z);
    const float aa = __fadd_rn(__fadd_rn(__fmul_rn(a0, a0), __fmul_rn(a1, a1)), __fmul_rn(a2, a2));
    if (aa > 0.f) {
      const float dot = __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
      if (__fdiv_rn(dot, __fmul_rn(__fsqrt_rn(aa), range)) > M.cone_cos) return;
    }
    const float c0 = __fsub_rn(x0, q0), c1 = __fsub_rn(x1, q1), c2 = __fsub_rn(x2, q2);
    const float cc = __fadd_rn(__fadd_rn(__fmul_rn(c0, c0), __fmul_rn(c1, c1)), __fmul_rn(c2, c2));
    float d = __fsub_rn(range, __fsqrt_rn(cc));
    d = d < M.dlo ? M.dlo : d;
    d = d > M.tau ? M.tau : d;
    const long long dq = __float2ll_rn(__fmul_rn(d, kScale));
    atomicAdd(B.vox + at, make_word(dq, 1ull));
  } else if (e < pairs + band) {
    const uint64_t f = e - pairs;
    const uint32_t k = (uint32_t)(f / M.ns);
    const int s = (int)(f % M.ns) + 1;
    const float4 p4 = scratch[k];
    if (p4.w == 0.f) return;
    const float p[3] = {p4.x, p4.y, p4.z}, q[3] = {q0, q1, q2};
    const float b0 = __fsub_rn(p[0], q0), b1 = __fsub_rn(p[1], q1), b2 = __fsub_rn(p[2], q2);
    const float range =
        __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2)));
    int sv[3];
    if (!band_sample(M, p, q, range, s, sv)) return;
    size_t at;
    if (box_index(B, sv[0], sv[1], sv[2], &at)) B.flags[at] |= 1u;  // every writer sets bit 0
  }
}

// Weight cap and occupied / known flags of box voxel `at`. Idempotent (a
// capped weight is not capped again), so threads that reach the same voxel
// through different returns write the same word and flags.
__device__ inline void finalize_voxel(const MapView& M, const Box& B, size_t at) {
  unsigned long long word = B.vox[at];
  unsigned long long w = word & kWMask;
  long long S = word_S(word);
  if (w > M.w_cap) {
    S = capped_S(S, M.w_cap, (long long)w);
    w = M.w_cap;
    B.vox[at] = make_word(S, w);
  }
  const unsigned cl = B.flags[at] & 1u;
  const unsigned occ = (w >= 1 && S < (long long)M.rcq * (long long)w) ? 1u : 0u;
  const unsigned kn = (w >= 1 || cl) ? 1u : 0u;
  B.flags[at] = (uint8_t)(cl | (occ << 1) | (kn << 2));
}

// Weight cap and flags of every voxel this scan touched -- the cube voxels
// and cleared-band samples of its accepted returns, enumerated as in
// k_na_integrate -- after all of the scan's additions (a launch of its own).
// Voxels the scan does not touch keep their words and flags.
__global__ void __launch_bounds__(256) k_na_finalize(MapView M, const float4* __restrict__ scratch,
                                                      uint32_t n, float q0, float q1, float q2,
                                                      Box B) {
  const int W = 2 * M.m + 1;
  const uint64_t C = (uint64_t)W * W * W;
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t pairs = C * n;
  const uint64_t band = (uint64_t)M.ns * n;
  size_t at;
  if (e < pairs) {
    const uint32_t k = (uint32_t)(e / C);
    const int o = (int)(e % C);
    const float4 p = scratch[k];
    if (p.w == 0.f) return;
    int i[3];
    if (!(voxel_index(p.x, M, &i[0]) && voxel_index(p.y, M, &i[1]) &&
          voxel_index(p.z, M, &i[2])))
      return;
    const int jx = i[0] - M.dom_vox[0] + o % W - M.m;
    const int jy = i[1] - M.dom_vox[1] + (o / W) % W - M.m;
    const int jz = i[2] - M.dom_vox[2] + o / (W * W) - M.m;
    if (box_index(B, jx, jy, jz, &at)) finalize_voxel(M, B, at);
  } else if (e < pairs + band) {
    const uint64_t f = e - pairs;
    const uint32_t k = (uint32_t)(f / M.ns);
    const int s = (int)(f % M.ns) + 1;
    const float4 p4 = scratch[k];
    if (p4.w == 0.f) return;
    const float p[3] = {p4.x, p4.y, p4.z}, q[3] = {q0, q1, q2};
    const float b0 = __fsub_rn(p[0], q0), b1 = __fsub_rn(p[1], q1), b2 = __fsub_rn(p[2], q2);
    const float range =
        __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2)));
    int sv[3];
    if (!band_sample(M, p, q, range, s, sv)) return;
    if (box_index(B, sv[0], sv[1], sv[2], &at)) finalize_voxel(M, B, at);
  }
}

bool finite_f(float x) { return std::isfinite(x); }

}  // namespace
}  // namespace af

extern "C" af_status af_integrate_scan_noalloc(const af_config* cfg, const float* d_xyz,
                                               uint32_t n, const float pose[16],
                                               const int32_t box_min[3], const uint32_t box_dim[3],
                                               uint64_t* d_vox, uint8_t* d_flags, void* stream) {
  using namespace af;
  if (!cfg || !pose || !box_min || !box_dim || !d_vox || !d_flags || (n > 0 && !d_xyz))
    return nfail(AF_ERR_INVALID_ARG, "af_integrate_scan_noalloc: NULL argument");
  if (n > AF_NOALLOC_MAX_RETURNS)
    return nfail(AF_ERR_CAPACITY,
                 "af_integrate_scan_noalloc: n = %u returns exceeds the fixed scratch of %d "
                 "returns; split the scan",
                 n, AF_NOALLOC_MAX_RETURNS);
  const float f[8] = {cfg->voxel_size, cfg->truncation, cfg->r_c,      cfg->cone_cos,
                      cfg->range_min,  cfg->range_max,  cfg->clear_lo, cfg->clear_hi};
  for (float x : f)
    if (!finite_f(x)) return nfail(AF_ERR_INVALID_ARG, "af_integrate_scan_noalloc: non-finite parameter");
  if (!(cfg->voxel_size > 0.f) || !(cfg->truncation > 0.f && cfg->truncation <= 1.f) ||
      !(cfg->r_c > 0.f && cfg->r_c <= 1.f) || cfg->cube_radius < 1 || cfg->cube_radius > 8 ||
      cfg->clear_samples < 0 || cfg->clear_samples > 64 || cfg->block_edge != 8 ||
      cfg->w_cap < 1 || (uint64_t)AF_NOALLOC_MAX_RETURNS + cfg->w_cap >= (1ull << kWBits) ||
      !(cfg->range_max > cfg->range_min) || !(cfg->clear_hi >= cfg->clear_lo) ||
      (cfg->clamp_signed != 0 && cfg->clamp_signed != 1))
    return nfail(AF_ERR_INVALID_ARG, "af_integrate_scan_noalloc: parameter out of range");
  uint64_t count = 1;
  for (int k = 0; k < 3; ++k) {
    if (cfg->domain_bricks[k] < 1 || cfg->domain_bricks[k] >= (1u << 21) ||
        std::abs((long long)cfg->domain_min[k]) > (1 << 25) || box_dim[k] < 1 ||
        box_dim[k] >= (1u << 24) || std::abs((long long)box_min[k]) > (1 << 28))
      return nfail(AF_ERR_INVALID_ARG, "af_integrate_scan_noalloc: domain or box out of range");
    // each factor is below 2^24, so the running product (at most 2^40 before
    // this step) cannot wrap before the check
    count *= box_dim[k];
    if (count > AF_NOALLOC_MAX_BOX_VOXELS)
      return nfail(AF_ERR_INVALID_ARG,
                   "af_integrate_scan_noalloc: the box holds more than 2^40 voxels");
  }
  for (int k = 0; k < 12; ++k)
    if (!finite_f(pose[k])) return nfail(AF_ERR_INVALID_ARG, "af_integrate_scan_noalloc: non-finite pose");

  float4* scratch = nullptr;
  af_status st = scratch_address(&scratch);
  if (st != AF_OK) return st;

  MapView M{};
  M.v = cfg->voxel_size;
  M.inv_v = 1.0f / cfg->voxel_size;
  M.tau = cfg->truncation;
  M.r_c = cfg->r_c;
  M.cone_cos = cfg->cone_cos;
  M.range_min = cfg->range_min;
  M.range_max = cfg->range_max;
  M.clear_lo = cfg->clear_lo;
  M.clear_hi = cfg->clear_hi;
  M.m = cfg->cube_radius;
  M.ns = cfg->clear_samples;
  M.w_min = cfg->w_min;
  M.w_cap = cfg->w_cap;
  M.rcq = (uint64_t)rintf(cfg->r_c * kScale);
  M.clamp_signed = cfg->clamp_signed;
  M.dlo = cfg->clamp_signed ? -cfg->truncation : 0.f;
  for (int k = 0; k < 3; ++k) {
    M.dom_vox[k] = cfg->domain_min[k] * 8;
    M.dim_vox[k] = (int)cfg->domain_bricks[k] * 8;
  }
  Box B;
  for (int k = 0; k < 3; ++k) {
    B.lo[k] = box_min[k] - M.dom_vox[k];
    B.dim[k] = (int)box_dim[k];
  }
  B.vox = reinterpret_cast<unsigned long long*>(d_vox);
  B.flags = d_flags;
  Pose P;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) P.r[r][c] = pose[4 * r + c];

  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    k_na_prepare<<<(n + 255) / 256, 256, 0, s>>>(M, d_xyz, n, P, scratch);
    const int W = 2 * M.m + 1;
    const uint64_t work = (uint64_t)n * W * W * W + (uint64_t)n * M.ns;
    const unsigned grid = (unsigned)((work + 255) / 256);
    k_na_integrate<<<grid, 256, 0, s>>>(M, scratch, n, pose[3], pose[7], pose[11], B);
    k_na_finalize<<<grid, 256, 0, s>>>(M, scratch, n, pose[3], pose[7], pose[11], B);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(AF_ERR_CUDA, "af_integrate_scan_noalloc: launch failed: %s",
                                     cudaGetErrorString(e));
  return AF_OK;
}

