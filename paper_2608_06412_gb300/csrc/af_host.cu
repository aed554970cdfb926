// af_host.cu -- the C ABI of libaf (include/af.h): context lifetime, argument
// checks, the tool / corridor kernel tables (rasterised once on the host,
// Sec. 3.4 and 3.6 of the paper: no rotation at run time), launches, and
// host-side export of the map.
#include <af.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

#include "af_ctx.cuh"
#include "af_internal.cuh"

namespace af {
cudaError_t launch_alloc(const MapView& M, const float* d_xyz, uint32_t n, const float pose[16],
                         float4* d_ret, uint32_t frame, cudaStream_t stream);
cudaError_t launch_cube(const MapView& M, uint32_t n, const float pose[16], const float4* d_ret,
                        uint32_t frame, cudaStream_t stream);
cudaError_t launch_bitview(const MapView& M, int num_sms, cudaStream_t stream);
cudaError_t launch_projective(const MapView& M, const float* d_xyz, uint32_t n,
                              const float pose[16], const float4* d_ret, unsigned* d_img,
                              uint32_t bins, int num_sms, cudaStream_t s);
cudaError_t launch_score(const MapView& M, const ToolView& T, const float* d_pts,
                         const float* d_nrm, uint32_t m, uint8_t* d_label, int16_t* d_best,
                         const ScoreSplit& S, int num_sms, cudaStream_t stream);
cudaError_t launch_export_flags(const MapView& M, uint32_t count, uint8_t* d_flags,
                                cudaStream_t stream);
cudaError_t launch_views(const MapView& M, int num_sms, bool fill, float* dense, float4* cells,
                         cudaStream_t stream);
cudaError_t launch_soft_seed(const float* d_nrm, uint32_t m, const float* d_table, uint32_t K,
                             float* d_u0, int num_sms, cudaStream_t stream);
cudaError_t launch_soft(const SoftView& S, bool grad, const float* pts, uint32_t per_point,
                        const float* u0, const float* al, const float* be, const float* h,
                        uint64_t n, const float* gc, float* c, float* cmin, float* ga,
                        float* gb, float* gh, int num_sms, cudaStream_t stream);
cudaError_t launch_soft_refine(const SoftView& S, const RefineArgs& R, const float* pts,
                               uint32_t per_point, const float* u0, float* al, float* be,
                               float* h, uint64_t n, float* c, float* cmin, int num_sms,
                               cudaStream_t stream);
cudaError_t launch_soft_best(const float* c, uint64_t n, uint32_t per_point, const float* u0,
                             int32_t* best_k, float* best_c, float* best_u0, int num_sms,
                             cudaStream_t stream);
cudaError_t launch_soft_start(const uint8_t* label, const int16_t* best, uint32_t m,
                              const float* dirs, int G, float* u0, int num_sms,
                              cudaStream_t stream);
cudaError_t launch_pts_snapshot(af_ctx* ctx, cudaStream_t stream);
cudaError_t launch_sview_mark(const MapView& M, int num_sms, uint32_t* bgrid, size_t gcount,
                              int gx, int gy, uint32_t* keys, uint32_t* nslots, cudaStream_t stream);
cudaError_t launch_sview_fill(const MapView& M, int num_sms, const uint32_t* keys, uint32_t nslots,
                              int gx, int gy, float4* cells, cudaStream_t stream);
}  // namespace af

using af::MapView;


namespace {

cudaEvent_t take_event(af_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Runs `launch` on `s`, bracketed by events when profiling is on.
template <class F>
cudaError_t timed(af_ctx* c, int kernel, cudaStream_t s, F&& launch, int kernels = 1) {
  if (!c->prof_on) return launch();
  af_ctx::ProfRec r{kernel, take_event(c), take_event(c), kernels};
  cudaEventRecord(r.a, s);
  const cudaError_t e = launch();
  cudaEventRecord(r.b, s);
  c->prof.push_back(r);
  return e;
}

}  // namespace

static char g_err[512] = "no error";

static af_status fail(af_ctx* c, af_status s, const char* fmt, ...) {
  char* buf = c ? c->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

#define AF_CUDA(ctx, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((ctx), AF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

#ifdef AF_CHECKED
extern "C" const char* af_version(void) { return "libaf 0.2 (sm_103a, checked)"; }
#else
extern "C" const char* af_version(void) { return "libaf 0.2 (sm_103a)"; }
#endif

extern "C" const char* af_last_error(const af_ctx* ctx) { return ctx ? ctx->err : g_err; }

namespace af {
void set_global_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace af

// ---------------------------------------------------------------------------
// Kernel rasterisation (Sec. 3.4). An offset o belongs to the kernel of unit
// direction u when, with e = o v, a = e . u and rho^2 = |e - a u|^2 (double
// precision, summed x, y, z):
//   tool:     0 <= a <= L,  rho^2 <= r^2,  |e|^2 > r_s^2
//   corridor: L < a <= L + L_c,  rho^2 <= r_c^2
// ---------------------------------------------------------------------------
namespace {

struct Offset {
  int x, y, z;
};

bool member(const af_tool& t, double v, const double u[3], int ox, int oy, int oz, int which) {
  const double ex = (double)ox * v, ey = (double)oy * v, ez = (double)oz * v;
  const double a = (ex * u[0] + ey * u[1]) + ez * u[2];
  const double rx = ex - a * u[0], ry = ey - a * u[1], rz = ez - a * u[2];
  const double rho2 = (rx * rx + ry * ry) + rz * rz;
  const double L = (double)t.length;
  if (which == AF_KERNEL_TOOL) {
    const double e2 = (ex * ex + ey * ey) + ez * ez;
    const double r = (double)t.radius, rs = (double)t.self_excl;
    return a >= 0.0 && a <= L && rho2 <= r * r && e2 > rs * rs;
  }
  const double r = (double)t.corr_radius;
  return a > L && a <= L + (double)t.corr_length && rho2 <= r * r;
}

// Offsets of one kernel, enumerating the axis-aligned box that holds the
// cylinder (with one voxel of margin), z-major.
std::vector<Offset> rasterise(const af_tool& t, double v, const double u[3], int which) {
  std::vector<Offset> out;
  const double a0 = which == AF_KERNEL_TOOL ? 0.0 : (double)t.length;
  const double a1 = which == AF_KERNEL_TOOL ? (double)t.length
                                            : (double)t.length + (double)t.corr_length;
  const double r = which == AF_KERNEL_TOOL ? (double)t.radius : (double)t.corr_radius;
  if (which == AF_KERNEL_CORRIDOR && !(t.corr_length > 0.f)) return out;
  int lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    const double p = a0 * u[k], q = a1 * u[k];
    lo[k] = (int)std::floor((std::min(p, q) - r) / v) - 1;
    hi[k] = (int)std::ceil((std::max(p, q) + r) / v) + 1;
  }
  for (int oz = lo[2]; oz <= hi[2]; ++oz)
    for (int oy = lo[1]; oy <= hi[1]; ++oy)
      for (int ox = lo[0]; ox <= hi[0]; ++ox)
        if (member(t, v, u, ox, oy, oz, which)) out.push_back({ox, oy, oz});
  return out;
}

// The axis a direction's runs follow: the one it is closest to (largest
// |u_k|, the lowest k on ties).
int run_axis(const double u[3]) {
  int a = std::fabs(u[1]) > std::fabs(u[0]) ? 1 : 0;
  return std::fabs(u[2]) > std::fabs(u[a]) ? 2 : a;
}

// Groups offsets into runs of at most 64 voxels along `axis`, ordered by the
// axial distance of their first voxel (near runs first: blocking geometry
// next to the surface is met early). A run is (d_axis, len | axis << 8,
// d_o1, d_o2), o1 < o2 the other two axes.
void to_runs(const std::vector<Offset>& offs, double v, const double u[3], int axis,
             std::vector<short4>* runs) {
  struct R {
    double a;
    short4 s;
  };
  const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
  std::vector<std::array<int, 3>> c(offs.size());
  for (size_t k = 0; k < offs.size(); ++k) c[k] = {offs[k].x, offs[k].y, offs[k].z};
  std::sort(c.begin(), c.end(), [&](const std::array<int, 3>& p, const std::array<int, 3>& q) {
    if (p[o2] != q[o2]) return p[o2] < q[o2];
    if (p[o1] != q[o1]) return p[o1] < q[o1];
    return p[axis] < q[axis];
  });
  std::vector<R> rs;
  size_t i = 0;
  while (i < c.size()) {
    size_t j = i + 1;
    while (j < c.size() && c[j][o1] == c[i][o1] && c[j][o2] == c[i][o2] &&
           c[j][axis] == c[j - 1][axis] + 1 && (int)(j - i) < 64)
      ++j;
    const std::array<int, 3>& o = c[i];
    const double a = ((double)o[0] * v * u[0] + (double)o[1] * v * u[1]) + (double)o[2] * v * u[2];
    rs.push_back({a, make_short4((short)o[axis], (short)((int)(j - i) | (axis << 8)), (short)o[o1],
                                 (short)o[o2])});
    i = j;
  }
  std::stable_sort(rs.begin(), rs.end(), [](const R& p, const R& q) { return p.a < q.a; });
  for (const R& r : rs) runs->push_back(r.s);
}

void arm_offsets(double v, double tau, const double u[3], int out[9]) {
  static const double frac[3] = {0.6, 1.25, 2.25};
  for (int s = 0; s < 3; ++s)
    for (int k = 0; k < 3; ++k) out[3 * s + k] = (int)std::floor(0.5 + ((frac[s] * tau) * u[k]) / v);
}

bool finite3(const float* u) { return std::isfinite(u[0]) && std::isfinite(u[1]) && std::isfinite(u[2]); }

af_status check_tool(const af_tool* t) {
  if (!t) return fail(nullptr, AF_ERR_INVALID_ARG, "tool is NULL");
  const float f[6] = {t->radius, t->length, t->self_excl, t->corr_radius, t->corr_length,
                      t->cos_theta_max};
  for (float x : f)
    if (!std::isfinite(x)) return fail(nullptr, AF_ERR_INVALID_ARG, "non-finite tool parameter");
  if (!(t->radius > 0.f) || t->length < 0.f || t->self_excl < 0.f || t->corr_radius < 0.f ||
      t->corr_length < 0.f || t->n_c < 1 || t->n_c > 1000000 || t->cos_theta_max < -1.f ||
      t->cos_theta_max > 1.f || (t->corridor_strict != 0 && t->corridor_strict != 1))
    return fail(nullptr, AF_ERR_INVALID_ARG, "tool parameter out of range");
  return AF_OK;
}

}  // namespace

extern "C" af_status af_kernel_offsets(const af_tool* tool, float voxel_size, const float u[3],
                                       int32_t which, int32_t* h_out, int64_t cap,
                                       int64_t* count) {
  af_status s = check_tool(tool);
  if (s != AF_OK) return s;
  if (!(voxel_size > 0.f) || !std::isfinite(voxel_size) || !u || !finite3(u) || !count ||
      (which != AF_KERNEL_TOOL && which != AF_KERNEL_CORRIDOR) || cap < 0 || (cap > 0 && !h_out))
    return fail(nullptr, AF_ERR_INVALID_ARG, "af_kernel_offsets: bad argument");
  const double du[3] = {(double)u[0], (double)u[1], (double)u[2]};
  const std::vector<Offset> offs = rasterise(*tool, (double)voxel_size, du, which);
  *count = (int64_t)offs.size();
  for (int64_t k = 0; k < std::min<int64_t>(cap, (int64_t)offs.size()); ++k) {
    h_out[3 * k] = offs[k].x;
    h_out[3 * k + 1] = offs[k].y;
    h_out[3 * k + 2] = offs[k].z;
  }
  return AF_OK;
}

extern "C" af_status af_arm_offsets(float voxel_size, float truncation, const float u[3],
                                    int32_t h_out[9]) {
  if (!(voxel_size > 0.f) || !(truncation > 0.f) || !u || !finite3(u) || !h_out)
    return fail(nullptr, AF_ERR_INVALID_ARG, "af_arm_offsets: bad argument");
  const double du[3] = {(double)u[0], (double)u[1], (double)u[2]};
  int o[9];
  arm_offsets((double)voxel_size, (double)truncation, du, o);
  for (int k = 0; k < 9; ++k) h_out[k] = o[k];
  return AF_OK;
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

static void free_tool(af_ctx* c) {
  cudaFree(c->d_dirs);
  cudaFree(c->d_runs);
  cudaFree(c->d_fruns);
  cudaFree(c->d_dtab);
  cudaFree(c->d_arm);
  c->d_dirs = nullptr;
  c->d_runs = nullptr;
  c->d_fruns = nullptr;
  c->d_dtab = nullptr;
  c->d_arm = nullptr;
  c->has_tool = false;
}

static void free_all(af_ctx* c) {
  free_tool(c);
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  c->prof.clear();
  c->ev_free.clear();
  MapView& M = c->M;
  cudaFree(M.slots);
  cudaFree(M.vox);
  cudaFree(M.cleared);
  cudaFree(M.bkey);
  cudaFree(M.dirty);
  cudaFree(M.rtab);
  cudaFree(M.occ);
  cudaFree(M.known);
  cudaFree(M.occ_y);
  cudaFree(M.occ_z);
  cudaFree(M.ctl);
  cudaFree(c->d_ret);
  cudaFree(c->d_xyz);
  cudaFree(c->d_pts);
  cudaFree(c->d_nrm);
  cudaFree(c->d_label);
  cudaFree(c->d_best);
  cudaFree(c->d_over);
  cudaFree(c->d_sres);
  cudaFree(c->d_scount);
  cudaFree(c->d_dense);
  cudaFree(c->d_cells);
  cudaFree(c->d_bgrid);
  cudaFree(c->d_skeys);
  cudaFree(c->d_nslots);
  cudaFree(c->d_scells);
  cudaFree(c->d_table);
  cudaFree(c->d_img);
  for (void* p : {(void*)c->d_pid, (void*)c->d_pst, (void*)c->d_pviews, (void*)c->d_pnew,
                  (void*)c->d_pnear, (void*)c->d_psnapw, (void*)c->d_psnapc, (void*)c->d_pchgmask,
                  (void*)c->d_phist, (void*)c->d_psamp, (void*)c->d_psel, (void*)c->d_pblock,
                  (void*)c->d_pcount, (void*)c->d_pnnoff, (void*)c->d_pc2f, (void*)c->d_psnap})
    cudaFree(p);
  cudaFreeHost(c->h_status);
}

static af_status check_config(const af_config* c) {
  auto bad = [](const char* what) { return fail(nullptr, AF_ERR_INVALID_ARG, "af_config: %s", what); };
  const float f[8] = {c->voxel_size, c->truncation, c->r_c, c->cone_cos,
                      c->range_min, c->range_max, c->clear_lo, c->clear_hi};
  for (float x : f)
    if (!std::isfinite(x)) return bad("non-finite parameter");
  if (!(c->voxel_size > 0.f)) return bad("voxel_size must be > 0");
  if (!(c->truncation > 0.f && c->truncation <= 1.f)) return bad("truncation must be in (0, 1] m");
  if (!(c->r_c > 0.f && c->r_c <= 1.f)) return bad("r_c must be in (0, 1] m");
  if (c->cone_cos < -1.f || c->cone_cos > 1.f) return bad("cone_cos must be in [-1, 1]");
  if (!(c->range_min >= 0.f && c->range_max > c->range_min)) return bad("range bounds");
  if (!(c->clear_lo >= 0.f && c->clear_hi >= c->clear_lo)) return bad("cleared band bounds");
  if (c->cube_radius < 1 || c->cube_radius > 8) return bad("cube_radius must be in 1..8");
  if (c->clear_samples < 0 || c->clear_samples > 64) return bad("clear_samples must be in 0..64");
  if (c->block_edge != 8) return bad("block_edge must be 8");
  if (c->w_cap < 1) return bad("w_cap must be >= 1");
  if (c->clamp_signed != 0 && c->clamp_signed != 1) return bad("clamp_signed must be 0 or 1");
  if (c->max_returns < 1) return bad("max_returns must be >= 1");
  if ((uint64_t)c->max_returns + c->w_cap >= (1ull << af::kWBits))
    return bad("max_returns + w_cap must be below 2^20");
  for (int k = 0; k < 3; ++k) {
    if (c->domain_bricks[k] < 1 || c->domain_bricks[k] >= (1u << 21)) return bad("domain_bricks");
    if (std::abs((int64_t)c->domain_min[k]) > (1 << 25) ||
        std::abs((int64_t)c->domain_min[k] + c->domain_bricks[k]) > (1 << 25))
      return bad("domain out of range");
  }
  if (c->hash_capacity < 2 || (c->hash_capacity & (c->hash_capacity - 1)) != 0 ||
      c->hash_capacity > (1u << 31))
    return bad("hash_capacity must be a power of two >= 2");
  if (c->pool_blocks < 1 || c->pool_blocks >= 0xFFFFFFF0u) return bad("pool_blocks");
  return AF_OK;
}

extern "C" af_status af_create(const af_config* cfg, af_ctx** out) {
  if (!cfg || !out) return fail(nullptr, AF_ERR_INVALID_ARG, "af_create: NULL argument");
  *out = nullptr;
  af_status s = check_config(cfg);
  if (s != AF_OK) return s;
  af_ctx* c = new af_ctx();
  c->cfg = *cfg;
  MapView& M = c->M;
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
  M.rcq = (uint64_t)rintf(cfg->r_c * af::kScale);
  M.clamp_signed = cfg->clamp_signed;
  M.dlo = cfg->clamp_signed ? -cfg->truncation : 0.f;
  for (int k = 0; k < 3; ++k) {
    M.dom_vox[k] = cfg->domain_min[k] * 8;
    M.dim_vox[k] = (int)cfg->domain_bricks[k] * 8;
  }
  M.row_words = (M.dim_vox[0] + 63) / 64;
  M.row_words_y = (M.dim_vox[1] + 63) / 64;
  M.row_words_z = (M.dim_vox[2] + 63) / 64;
  M.words_x = (size_t)M.row_words * M.dim_vox[1] * M.dim_vox[2];
  M.words_y = (size_t)M.row_words_y * M.dim_vox[0] * M.dim_vox[2];
  M.words_z = (size_t)M.row_words_z * M.dim_vox[0] * M.dim_vox[1];
  M.hmask = cfg->hash_capacity - 1;
  M.pool_blocks = cfg->pool_blocks;
  {
    const int ba = (2 * M.m + 1 + 6) / 8 + 1;  // bricks a cube edge can span
    M.nbmax = ba * ba * ba;
  }

  // fault injection for tests: the k-th allocation fails (AF_FAIL_ALLOC_AT)
  long fail_at = -1, nalloc = 0;
  if (const char* f = std::getenv("AF_FAIL_ALLOC_AT")) fail_at = std::strtol(f, nullptr, 10);
  auto alloc = [&](void** p, size_t bytes, int fill) -> af_status {
    if (nalloc++ == fail_at) {
      fail(c, AF_ERR_CUDA, "device allocation of %zu bytes failed: injected failure at "
                           "allocation %ld (AF_FAIL_ALLOC_AT)", bytes, fail_at);
      return AF_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) e = cudaMemset(*p, fill, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      fail(c, AF_ERR_CUDA, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
      return AF_ERR_CUDA;
    }
    return AF_OK;
  };
  const size_t H = cfg->hash_capacity, P = cfg->pool_blocks;
  const size_t plane = (size_t)M.row_words * 8 * M.dim_vox[1] * M.dim_vox[2];
  const size_t R = cfg->max_returns, Pm = cfg->max_points;
  af_status st = AF_OK;
  if (st == AF_OK) st = alloc((void**)&M.slots, H * sizeof(af::HashSlot), 0xFF);
  if (st == AF_OK) st = alloc((void**)&M.vox, P * af::kBrickVox * 8, 0);
  if (st == AF_OK) st = alloc((void**)&M.cleared, P * 16 * 4, 0);
  if (st == AF_OK) st = alloc((void**)&M.bkey, P * 8, 0);
  if (st == AF_OK) st = alloc((void**)&M.dirty, P * 4, 0);
  if (st == AF_OK) st = alloc((void**)&M.occ, plane, 0);
  if (st == AF_OK) st = alloc((void**)&M.known, plane, 0);
  if (st == AF_OK)
    st = alloc((void**)&M.occ_y, (size_t)M.row_words_y * 8 * M.dim_vox[0] * M.dim_vox[2], 0);
  if (st == AF_OK)
    st = alloc((void**)&M.occ_z, (size_t)M.row_words_z * 8 * M.dim_vox[0] * M.dim_vox[1], 0);
  if (st == AF_OK) st = alloc((void**)&M.ctl, sizeof(af::Control), 0);
  if (st == AF_OK) st = alloc((void**)&c->d_ret, R * sizeof(float4), 0);
  if (st == AF_OK) st = alloc((void**)&M.rtab, R * (size_t)M.nbmax * 4, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_xyz, R * 12, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_pts, Pm * 12, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_nrm, Pm * 12, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_label, Pm, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_best, Pm * 2, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_over, Pm * sizeof(int2), 0);
  if (st == AF_OK) st = alloc((void**)&c->d_sres, Pm * 4, 0);
  if (st == AF_OK) st = alloc((void**)&c->d_scount, 16, 0);  // split count, staged counters
  c->split_cap = (uint32_t)Pm;
  if (st == AF_OK && cudaMallocHost((void**)&c->h_status, 64) != cudaSuccess)
    st = fail(c, AF_ERR_CUDA, "pinned allocation failed");
  int dev = 0;
  if (st == AF_OK && (cudaGetDevice(&dev) != cudaSuccess ||
                      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) !=
                          cudaSuccess))
    st = fail(c, AF_ERR_CUDA, "device query failed");
  if (st == AF_OK && cudaDeviceSynchronize() != cudaSuccess)
    st = fail(c, AF_ERR_CUDA, "initialisation failed");
  if (st != AF_OK) {
    snprintf(g_err, sizeof g_err, "%s", c->err);
    free_all(c);
    delete c;
    return st;
  }
  *out = c;
  return AF_OK;
}

extern "C" af_status af_destroy(af_ctx* ctx) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_destroy: NULL context");
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return AF_OK;
}

extern "C" af_status af_integrate_scan(af_ctx* ctx, const float* d_xyz, uint32_t n,
                                       const float pose[16], void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_integrate_scan: NULL context");
  if (!pose) return fail(ctx, AF_ERR_INVALID_ARG, "af_integrate_scan: NULL pose");
  if (n > 0 && !d_xyz) return fail(ctx, AF_ERR_INVALID_ARG, "af_integrate_scan: NULL points");
  if (n > ctx->cfg.max_returns)
    return fail(ctx, AF_ERR_CAPACITY, "af_integrate_scan: n = %u exceeds max_returns = %u", n,
                ctx->cfg.max_returns);
  for (int k = 0; k < 12; ++k)
    if (!std::isfinite(pose[k])) return fail(ctx, AF_ERR_INVALID_ARG, "non-finite pose");
  // scan stamps: 1 .. 2^32 - 2 (all ones marks a slot that no scan touched)
  ctx->frame = ctx->frame + 1 >= 0xFFFFFFFFu ? 1 : ctx->frame + 1;
  cudaStream_t s = (cudaStream_t)stream;
  const MapView& M = ctx->M;
  AF_CUDA(ctx, timed(ctx, 0, s, [&] { return af::launch_alloc(M, d_xyz, n, pose, ctx->d_ret, ctx->frame, s); }));
  // the point layer's neighbourhood trigger compares the touched bricks
  // after the scan with their state before it
  if (ctx->pts_snapshot) AF_CUDA(ctx, af::launch_pts_snapshot(ctx, s));
  if (n > 0)
    AF_CUDA(ctx, timed(ctx, 1, s, [&] { return af::launch_cube(M, n, pose, ctx->d_ret, ctx->frame, s); }));
  AF_CUDA(ctx, timed(ctx, 2, s, [&] { return af::launch_bitview(M, ctx->num_sms, s); }));
  ctx->last_stream = s;
  ctx->scans++;
  ctx->returns_in += n;
  return AF_OK;
}

// Projective integration (the ablation of Tab. 3): the scan-centric
// allocation without band bricks, the range-image update (af_projective.cu),
// then the weight cap and bit view. Profiling slots as af_integrate_scan.
extern "C" af_status af_integrate_scan_projective(af_ctx* ctx, const float* d_xyz, uint32_t n,
                                                  const float pose[16], uint32_t bins,
                                                  void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_integrate_scan_projective: NULL context");
  if (!pose) return fail(ctx, AF_ERR_INVALID_ARG, "af_integrate_scan_projective: NULL pose");
  if (n > 0 && !d_xyz) return fail(ctx, AF_ERR_INVALID_ARG, "af_integrate_scan_projective: NULL points");
  if (n > ctx->cfg.max_returns)
    return fail(ctx, AF_ERR_CAPACITY, "af_integrate_scan_projective: n exceeds max_returns");
  if (bins < 2 || bins > 8192)
    return fail(ctx, AF_ERR_INVALID_ARG, "af_integrate_scan_projective: bins must be in 2..8192");
  for (int k = 0; k < 12; ++k)
    if (!std::isfinite(pose[k])) return fail(ctx, AF_ERR_INVALID_ARG, "non-finite pose");
  const size_t cells = (size_t)bins * bins;
  if (cells > ctx->img_cap) {
    cudaFree(ctx->d_img);
    ctx->d_img = nullptr;
    ctx->img_cap = 0;
    AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_img, cells * sizeof(unsigned)));
    ctx->img_cap = cells;
  }
  ctx->frame = ctx->frame + 1 >= 0xFFFFFFFFu ? 1 : ctx->frame + 1;
  cudaStream_t s = (cudaStream_t)stream;
  af::MapView M = ctx->M;
  M.ns = 0;  // no cleared band: the projective update has none
  AF_CUDA(ctx, timed(ctx, 0, s, [&] { return af::launch_alloc(M, d_xyz, n, pose, ctx->d_ret, ctx->frame, s); }));
  AF_CUDA(ctx, timed(ctx, 1, s, [&] {
            return af::launch_projective(M, d_xyz, n, pose, ctx->d_ret, ctx->d_img, bins, ctx->num_sms, s);
          }, n > 0 ? 2 : 1));
  AF_CUDA(ctx, timed(ctx, 2, s, [&] { return af::launch_bitview(M, ctx->num_sms, s); }));
  ctx->last_stream = s;
  ctx->scans++;
  ctx->returns_in += n;
  return AF_OK;
}

extern "C" af_status af_set_tool(af_ctx* ctx, const af_tool* tool, const float* h_dirs,
                                 uint32_t G) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_set_tool: NULL context");
  af_status s = check_tool(tool);
  if (s != AF_OK) return fail(ctx, s, "%s", g_err);
  if (!h_dirs || G < 1 || G > 4096) return fail(ctx, AF_ERR_INVALID_ARG, "af_set_tool: need 1 <= G <= 4096 directions");
  for (uint32_t g = 0; g < G; ++g)
    if (!finite3(h_dirs + 3 * g)) return fail(ctx, AF_ERR_INVALID_ARG, "non-finite direction");

  const double v = (double)ctx->cfg.voxel_size, tau = (double)ctx->cfg.truncation;
  int reach[3] = {0, 0, 0};
  std::vector<short4> runs, cruns;  // tool runs of every direction, then corridor runs
  std::vector<int4> dtab(G);
  std::vector<short4> arm(3 * G);
  for (uint32_t g = 0; g < G; ++g) {
    const double u[3] = {(double)h_dirs[3 * g], (double)h_dirs[3 * g + 1], (double)h_dirs[3 * g + 2]};
    const std::vector<Offset> tool_o = rasterise(*tool, v, u, AF_KERNEL_TOOL);
    const std::vector<Offset> corr_o = rasterise(*tool, v, u, AF_KERNEL_CORRIDOR);
    for (const std::vector<Offset>* o : {&tool_o, &corr_o})
      for (const Offset& x : *o)
        if (std::abs(x.x) > 32000 || std::abs(x.y) > 32000 || std::abs(x.z) > 32000)
          return fail(ctx, AF_ERR_INVALID_ARG, "tool reach exceeds 32000 voxels");
    // runs along the direction's closest axis; the strict corridor also reads
    // the known view, which has x rows only
    const int ax = run_axis(u);
    dtab[g].x = (int)runs.size();
    to_runs(tool_o, v, u, ax, &runs);
    dtab[g].y = (int)runs.size();
    dtab[g].z = (int)cruns.size();
    to_runs(corr_o, v, u, tool->corridor_strict ? 0 : ax, &cruns);
    dtab[g].w = (int)cruns.size();
    for (const std::vector<Offset>* o : {&tool_o, &corr_o})
      for (const Offset& x : *o) {
        reach[0] = std::max(reach[0], std::abs(x.x));
        reach[1] = std::max(reach[1], std::abs(x.y));
        reach[2] = std::max(reach[2], std::abs(x.z));
      }
    int a[9];
    arm_offsets(v, tau, u, a);
    for (int k = 0; k < 3; ++k)
      arm[3 * g + k] = make_short4((short)a[3 * k], (short)a[3 * k + 1], (short)a[3 * k + 2], 0);
  }
  const int ntool = (int)runs.size();
  for (uint32_t g = 0; g < G; ++g) {
    dtab[g].z += ntool;
    dtab[g].w += ntool;
  }
  runs.insert(runs.end(), cruns.begin(), cruns.end());
  if (runs.empty()) runs.push_back(make_short4(0, 1, 0, 0));  // keep the buffer non-empty
  // Fast-path form of the runs: the plane-word offset of the run's row relative to
  // the point's row, valid while every plane index fits in 31 bits. `reach` bounds
  // every offset, so a point at least `reach` voxels inside the box needs no checks.
  const MapView& M = ctx->M;
  const int X = M.dim_vox[0], Y = M.dim_vox[1], Z = M.dim_vox[2];
  const bool fast_ok = (int64_t)M.row_words * Y * Z < (1ll << 31) &&
                       (int64_t)M.row_words_y * X * Z < (1ll << 31) &&
                       (int64_t)M.row_words_z * X * Y < (1ll << 31);
  // plane rows: axis x -> row z * Y + y; axis y -> z * X + x; axis z -> y * X + x
  const int dim_o1[3] = {Y, X, X};
  const int rw[3] = {M.row_words, M.row_words_y, M.row_words_z};
  std::vector<int2> fruns(runs.size());
  for (size_t r = 0; r < runs.size(); ++r) {
    const short4 s = runs[r];
    const int ax = ((uint16_t)s.y >> 8) & 3, len = (uint16_t)s.y & 0xFF;
    const int64_t delta = ((int64_t)s.w * dim_o1[ax] + s.z) * rw[ax];
    fruns[r] = make_int2((int)delta, (int)(uint16_t)s.x | (len << 16) | (ax << 24));
  }
  for (const short4& a : arm) {
    reach[0] = std::max(reach[0], std::abs((int)a.x));
    reach[1] = std::max(reach[1], std::abs((int)a.y));
    reach[2] = std::max(reach[2], std::abs((int)a.z));
  }
  if (!fast_ok) reach[0] = reach[1] = reach[2] = 1 << 30;  // never take the fast path
  AF_CUDA(ctx, cudaDeviceSynchronize());
  free_tool(ctx);
  AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_dirs, (size_t)G * 12));
  AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_runs, runs.size() * sizeof(short4)));
  AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_fruns, fruns.size() * sizeof(int2)));
  AF_CUDA(ctx, cudaMemcpy(ctx->d_fruns, fruns.data(), fruns.size() * sizeof(int2), cudaMemcpyHostToDevice));
  for (int k = 0; k < 3; ++k) ctx->T.reach[k] = reach[k];
  ctx->T.fruns = ctx->d_fruns;
  ctx->T.ntool = ntool;
  ctx->T.nruns = (int)runs.size();
  ctx->T.ctl = ctx->M.ctl;
  AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_dtab, (size_t)G * sizeof(int4)));
  AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_arm, (size_t)G * 3 * sizeof(short4)));
  AF_CUDA(ctx, cudaMemcpy(ctx->d_dirs, h_dirs, (size_t)G * 12, cudaMemcpyHostToDevice));
  AF_CUDA(ctx, cudaMemcpy(ctx->d_runs, runs.data(), runs.size() * sizeof(short4), cudaMemcpyHostToDevice));
  AF_CUDA(ctx, cudaMemcpy(ctx->d_dtab, dtab.data(), (size_t)G * sizeof(int4), cudaMemcpyHostToDevice));
  AF_CUDA(ctx, cudaMemcpy(ctx->d_arm, arm.data(), (size_t)G * 3 * sizeof(short4), cudaMemcpyHostToDevice));
  ctx->T.dirs = ctx->d_dirs;
  ctx->T.runs = ctx->d_runs;
  ctx->T.dtab = ctx->d_dtab;
  ctx->T.arm = ctx->d_arm;
  ctx->T.G = (int)G;
  ctx->T.n_c = (int)tool->n_c;
  ctx->T.cos_max = tool->cos_theta_max;
  ctx->T.strict = tool->corridor_strict;
  ctx->tool = *tool;
  ctx->has_tool = true;
  return AF_OK;
}

extern "C" af_status af_score(af_ctx* ctx, const float* d_pts, const float* d_normals,
                              uint32_t m, uint8_t* d_label, int16_t* d_best, void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_score: NULL context");
  if (!ctx->has_tool) return fail(ctx, AF_ERR_STATE, "af_score: call af_set_tool first");
  if (m > 0 && (!d_pts || !d_normals || !d_label || !d_best))
    return fail(ctx, AF_ERR_INVALID_ARG, "af_score: NULL buffer");
  if (m > (1u << 31)) return fail(ctx, AF_ERR_INVALID_ARG, "af_score: m too large");
  cudaStream_t s = (cudaStream_t)stream;
  if (ctx->score_budget >= 0 && m > ctx->split_cap) {  // hand-off records for every point
    cudaFree(ctx->d_over);
    cudaFree(ctx->d_sres);
    ctx->d_over = nullptr;
    ctx->d_sres = nullptr;
    ctx->split_cap = 0;
    AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_over, (size_t)m * sizeof(int2)));
    AF_CUDA(ctx, cudaMalloc((void**)&ctx->d_sres, (size_t)m * 4));
    ctx->split_cap = m;
  }
  const af::ScoreSplit S{ctx->d_over, ctx->d_sres, ctx->d_scount, ctx->score_budget,
                         ctx->d_scount + 1};
  if (m > 0)
    AF_CUDA(ctx, timed(ctx, 3, s, [&] {
              return af::launch_score(ctx->M, ctx->T, d_pts, d_normals, m, d_label, d_best, S,
                                      ctx->num_sms, s);
            }, S.budget >= 0 ? 3 : 1));
  ctx->last_stream = s;
  ctx->points_in += m;
  return AF_OK;
}

extern "C" af_status af_set_score_split(af_ctx* ctx, int32_t budget) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_set_score_split: NULL context");
  if (budget < -1 || budget > 4096) return fail(ctx, AF_ERR_INVALID_ARG, "af_set_score_split: budget must be in -1..4096");
  ctx->score_budget = budget;
  return AF_OK;
}

extern "C" af_status af_frame_host(af_ctx* ctx, const float* h_xyz, uint32_t n,
                                   const float pose[16], const float* h_pts,
                                   const float* h_normals, uint32_t m, uint8_t* h_label,
                                   int16_t* h_best, void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_frame_host: NULL context");
  if (n > ctx->cfg.max_returns || m > ctx->cfg.max_points)
    return fail(ctx, AF_ERR_CAPACITY, "af_frame_host: n or m exceeds max_returns / max_points");
  if ((n > 0 && !h_xyz) || (m > 0 && (!h_pts || !h_normals || !h_label || !h_best)))
    return fail(ctx, AF_ERR_INVALID_ARG, "af_frame_host: NULL buffer");
  if (m > 0 && !ctx->has_tool) return fail(ctx, AF_ERR_STATE, "af_frame_host: call af_set_tool first");
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) AF_CUDA(ctx, cudaMemcpyAsync(ctx->d_xyz, h_xyz, (size_t)n * 12, cudaMemcpyHostToDevice, s));
  if (m > 0) {
    AF_CUDA(ctx, cudaMemcpyAsync(ctx->d_pts, h_pts, (size_t)m * 12, cudaMemcpyHostToDevice, s));
    AF_CUDA(ctx, cudaMemcpyAsync(ctx->d_nrm, h_normals, (size_t)m * 12, cudaMemcpyHostToDevice, s));
  }
  af_status st = af_integrate_scan(ctx, ctx->d_xyz, n, pose, stream);
  if (st != AF_OK) return st;
  if (m > 0) {
    st = af_score(ctx, ctx->d_pts, ctx->d_nrm, m, ctx->d_label, ctx->d_best, stream);
    if (st != AF_OK) return st;
    AF_CUDA(ctx, cudaMemcpyAsync(h_label, ctx->d_label, m, cudaMemcpyDeviceToHost, s));
    AF_CUDA(ctx, cudaMemcpyAsync(h_best, ctx->d_best, (size_t)m * 2, cudaMemcpyDeviceToHost, s));
  }
  AF_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, &ctx->M.ctl->status, 4, cudaMemcpyDeviceToHost, s));
  AF_CUDA(ctx, cudaStreamSynchronize(s));
  if (*ctx->h_status != 0)
    return fail(ctx, (af_status)*ctx->h_status, "map capacity exceeded; integration stopped");
  return AF_OK;
}

extern "C" af_status af_sync_status(af_ctx* ctx) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_sync_status: NULL context");
  AF_CUDA(ctx, cudaDeviceSynchronize());
  uint32_t st = 0;
  AF_CUDA(ctx, cudaMemcpy(&st, &ctx->M.ctl->status, 4, cudaMemcpyDeviceToHost));
  if (st == AF_ERR_CHECK) return fail(ctx, AF_ERR_CHECK, "a bounds check of the checked build failed");
  if (st != 0) return fail(ctx, (af_status)st, "map capacity exceeded; integration stopped");
  return AF_OK;
}

extern "C" af_status af_get_stats(af_ctx* ctx, af_stats* out) {
  if (!ctx || !out) return fail(ctx, AF_ERR_INVALID_ARG, "af_get_stats: NULL argument");
  AF_CUDA(ctx, cudaDeviceSynchronize());
  af::Control c;
  AF_CUDA(ctx, cudaMemcpy(&c, ctx->M.ctl, sizeof c, cudaMemcpyDeviceToHost));
  out->scans = ctx->scans;
  out->returns_in = ctx->returns_in;
  out->returns_accepted = c.returns_accepted;
  out->blocks_allocated = std::min<uint64_t>(c.pool_count, ctx->cfg.pool_blocks);
  out->blocks_dirty_last = c.dirty_count;
  out->points_in = ctx->points_in;
  out->points_scored = c.points_scored;
  out->tests = c.tests;
  return AF_OK;
}

extern "C" af_status af_block_count(af_ctx* ctx, uint32_t* out) {
  if (!ctx || !out) return fail(ctx, AF_ERR_INVALID_ARG, "af_block_count: NULL argument");
  AF_CUDA(ctx, cudaDeviceSynchronize());
  uint32_t pc = 0;
  AF_CUDA(ctx, cudaMemcpy(&pc, &ctx->M.ctl->pool_count, 4, cudaMemcpyDeviceToHost));
  *out = std::min(pc, ctx->cfg.pool_blocks);
  return AF_OK;
}

extern "C" af_status af_export_blocks(af_ctx* ctx, uint32_t cap, int32_t* h_key, int64_t* h_S,
                                      uint32_t* h_w, uint8_t* h_flags, uint32_t* out_count) {
  if (!ctx || !out_count) return fail(ctx, AF_ERR_INVALID_ARG, "af_export_blocks: NULL argument");
  if (cap > 0 && (!h_key || !h_S || !h_w || !h_flags))
    return fail(ctx, AF_ERR_INVALID_ARG, "af_export_blocks: NULL buffer");
  uint32_t count = 0;
  af_status s = af_block_count(ctx, &count);
  if (s != AF_OK) return s;
  count = std::min(count, cap);
  *out_count = count;
  if (count == 0) return AF_OK;
  std::vector<uint64_t> keys(count), words((size_t)count * af::kBrickVox);
  AF_CUDA(ctx, cudaMemcpy(keys.data(), ctx->M.bkey, (size_t)count * 8, cudaMemcpyDeviceToHost));
  AF_CUDA(ctx, cudaMemcpy(words.data(), ctx->M.vox, words.size() * 8, cudaMemcpyDeviceToHost));
  uint8_t* d_flags = nullptr;
  AF_CUDA(ctx, cudaMalloc((void**)&d_flags, (size_t)count * af::kBrickVox));
  cudaError_t e = af::launch_export_flags(ctx->M, count, d_flags, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpy(h_flags, d_flags, (size_t)count * af::kBrickVox, cudaMemcpyDeviceToHost);
  cudaFree(d_flags);
  if (e != cudaSuccess) return fail(ctx, AF_ERR_CUDA, "export failed: %s", cudaGetErrorString(e));
  for (uint32_t b = 0; b < count; ++b) {
    const uint64_t k = keys[b];
    h_key[3 * b] = (int32_t)(k & 0x1FFFFF) + ctx->cfg.domain_min[0];
    h_key[3 * b + 1] = (int32_t)((k >> 21) & 0x1FFFFF) + ctx->cfg.domain_min[1];
    h_key[3 * b + 2] = (int32_t)(k >> 42) + ctx->cfg.domain_min[2];
    for (int l = 0; l < af::kBrickVox; ++l) {
      const uint64_t wd = words[(size_t)b * af::kBrickVox + l];
      h_S[(size_t)b * af::kBrickVox + l] = af::word_S(wd);
      h_w[(size_t)b * af::kBrickVox + l] = (uint32_t)(wd & af::kWMask);
    }
  }
  return AF_OK;
}

extern "C" af_status af_profile_enable(af_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_profile_enable: NULL context");
  ctx->prof_on = enable != 0;
  return AF_OK;
}

extern "C" af_status af_profile_read(af_ctx* ctx, af_profile* out, int reset) {
  if (!ctx || !out) return fail(ctx, AF_ERR_INVALID_ARG, "af_profile_read: NULL argument");
  AF_CUDA(ctx, cudaDeviceSynchronize());
  std::memset(out, 0, sizeof *out);
  for (const auto& r : ctx->prof) {
    float ms = 0.f;
    AF_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
    out->launches[r.kernel] += r.kernels;
    out->ms[r.kernel] += ms;
  }
  if (reset) {
    for (auto& r : ctx->prof) {
      ctx->ev_free.push_back(r.a);
      ctx->ev_free.push_back(r.b);
    }
    ctx->prof.clear();
  }
  return AF_OK;
}

// ---------------------------------------------------------------------------
// The differentiable form
// ---------------------------------------------------------------------------

// Whether the dense views of the map box fit: fewer than 2^31 cells, and
// 36 bytes per box voxel within half the device's free memory.
static bool dense_views_fit(const af_ctx* ctx) {
  const MapView& M = ctx->M;
  const uint64_t cells = ((uint64_t)M.dim_vox[0] + 1) * (M.dim_vox[1] + 1) * (M.dim_vox[2] + 1);
  if (cells >= (1ull << 31)) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cells * 36ull <= free_b / 2;
}

// Builds (or rebuilds, if the map changed since) the SDF views: the dense
// view of the box and its cell records, or the brick-sparse cell records
// (the view chosen by af_soft_set_view; automatic: dense when it fits).
static af_status ensure_views(af_ctx* ctx, cudaStream_t s) {
  const MapView& M = ctx->M;
  if (!ctx->d_cells && !ctx->d_bgrid)
    ctx->views_sparse = ctx->soft_mode == 2 || (ctx->soft_mode == 0 && !dense_views_fit(ctx));
  const bool stale = !ctx->views_valid || ctx->views_frame != ctx->frame;
  if (!ctx->views_sparse) {
    bool fill = false;
    if (!ctx->d_cells) {
      const size_t nd = (size_t)M.dim_vox[0] * M.dim_vox[1] * M.dim_vox[2];
      const size_t nc = ((size_t)M.dim_vox[0] + 1) * (M.dim_vox[1] + 1) * (M.dim_vox[2] + 1);
      if (nc >= (1ull << 31))
        return fail(ctx, AF_ERR_CAPACITY, "soft clearance: the map box has too many cells for the dense SDF view");
      if (cudaMalloc(&ctx->d_dense, nd * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&ctx->d_cells, nc * 2 * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->d_dense);
        ctx->d_dense = nullptr;
        ctx->d_cells = nullptr;
        return fail(ctx, AF_ERR_CAPACITY,
                    "soft clearance: cannot allocate the SDF views (%zu + %zu bytes) of the map box",
                    nd * sizeof(float), nc * 2 * sizeof(float4));
      }
      fill = true;
    }
    if (fill || stale) {
      AF_CUDA(ctx, timed(ctx, 4, s, [&] {
        return af::launch_views(M, ctx->num_sms, fill, ctx->d_dense, ctx->d_cells, s);
      }));
    }
  } else {
    const int gx = M.dim_vox[0] / 8 + 1, gy = M.dim_vox[1] / 8 + 1, gz = M.dim_vox[2] / 8 + 1;
    const size_t gcount = (size_t)gx * gy * gz;
    if (gcount >= (1ull << 32))
      return fail(ctx, AF_ERR_CAPACITY, "soft clearance: the map box has too many bricks for the sparse view");
    if (!ctx->d_bgrid) {
      if (cudaMalloc((void**)&ctx->d_bgrid, gcount * 4) != cudaSuccess ||
          cudaMalloc((void**)&ctx->d_skeys, (size_t)ctx->cfg.pool_blocks * 8 * 4) != cudaSuccess ||
          cudaMalloc((void**)&ctx->d_nslots, 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->d_bgrid);
        cudaFree(ctx->d_skeys);
        ctx->d_bgrid = nullptr;
        ctx->d_skeys = nullptr;
        ctx->d_nslots = nullptr;
        return fail(ctx, AF_ERR_CAPACITY, "soft clearance: cannot allocate the sparse view's brick grid");
      }
    }
    if (stale) {
      AF_CUDA(ctx, timed(ctx, 4, s, [&] {
        return af::launch_sview_mark(M, ctx->num_sms, ctx->d_bgrid, gcount, gx, gy, ctx->d_skeys,
                                     ctx->d_nslots, s);
      }));
      uint32_t nslots = 0;
      AF_CUDA(ctx, cudaMemcpyAsync(&nslots, ctx->d_nslots, 4, cudaMemcpyDeviceToHost, s));
      AF_CUDA(ctx, cudaStreamSynchronize(s));
      if (nslots > ctx->scells_cap) {  // the records of every slot, 16 KB each
        cudaFree(ctx->d_scells);
        ctx->d_scells = nullptr;
        ctx->scells_cap = 0;
        const size_t bytes = (size_t)nslots * af::kBrickVox * 2 * sizeof(float4);
        if (cudaMalloc((void**)&ctx->d_scells, bytes) != cudaSuccess) {
          cudaGetLastError();
          ctx->views_valid = false;
          return fail(ctx, AF_ERR_CAPACITY, "soft clearance: cannot allocate %zu bytes of sparse cell records", bytes);
        }
        ctx->scells_cap = nslots;
      }
      AF_CUDA(ctx, timed(ctx, 4, s, [&] {
        return af::launch_sview_fill(M, ctx->num_sms, ctx->d_skeys, nslots, gx, gy, ctx->d_scells, s);
      }));
    }
  }
  ctx->views_valid = true;
  ctx->views_frame = ctx->frame;
  return AF_OK;
}

// The view fields of S after ensure_views.
static void view_fields(const af_ctx* ctx, af::SoftView* S) {
  const MapView& M = ctx->M;
  S->sparse = ctx->views_sparse ? 1 : 0;
  S->cells = ctx->views_sparse ? ctx->d_scells : ctx->d_cells;
  S->bgrid = ctx->d_bgrid;
  for (int k = 0; k < 3; ++k) {
    S->glo[k] = M.dom_vox[k] - 8;
    S->gdim[k] = M.dim_vox[k] / 8 + 1;
  }
}

// The axis samples of the tool, decided in single precision: j = j0..J with
// j v > r_s, tool margin while j v <= L.
static af_status soft_view(af_ctx* ctx, float tau_s, af::SoftView* S) {
  if (!ctx->has_tool) return fail(ctx, AF_ERR_STATE, "soft clearance: call af_set_tool first");
  if (!(tau_s > 0.f) || !std::isfinite(tau_s))
    return fail(ctx, AF_ERR_INVALID_ARG, "soft clearance: tau_s must be finite and > 0");
  const af_tool& t = ctx->tool;
  const float v = ctx->cfg.voxel_size;
  const float span = t.length + t.corr_length;
  const float q = span / v;
  if (!(q < 1.0e6f)) return fail(ctx, AF_ERR_INVALID_ARG, "soft clearance: tool too long");
  const int J = (int)std::floor(q);
  int j0 = J + 1, jt = 0;
  for (int j = J; j >= 1; --j) {
    const float a = (float)j * v;
    if (a > t.self_excl) j0 = j;
    if (a <= t.length && jt == 0) jt = j;
  }
  if (j0 > J)
    return fail(ctx, AF_ERR_STATE, "soft clearance: no axis sample lies beyond the self-exclusion radius");
  const MapView& M = ctx->M;
  S->cells = ctx->d_cells;
  for (int k = 0; k < 3; ++k) {
    S->lo[k] = M.dom_vox[k] - 1;
    S->ncell[k] = M.dim_vox[k] + 1;
  }
  S->v = v;
  S->tau = ctx->cfg.truncation;
  S->r = t.radius;
  S->r_corr = t.corr_radius;
  S->j0 = j0;
  S->jt = jt;
  S->J = J;
  S->k2 = (float)(1.4426950408889634 / (double)tau_s);
  S->ln2_tau_s = (float)(0.6931471805599453 * (double)tau_s);
  // phi = SDF - margin lies in [-max margin, tau - min margin] (the TSDF is
  // clamped to [0, tau]); weights against the lower bound then span at most
  // 2^-E, and below E = 96 no weight underflows single precision.
  const double mx = std::max(t.radius, t.corr_radius), mnm = std::min(t.radius, t.corr_radius);
  const double E = ((double)ctx->cfg.truncation + 1e-3 + mx - mnm) * 1.4426950408889634 / (double)tau_s;
  S->fixed = E <= 96.0 ? 1 : 0;
  S->ref = (float)-mx;
  S->sparse = 0;
  S->bgrid = nullptr;
  return AF_OK;
}

static af_status check_pairs(af_ctx* ctx, const char* fn, const float* d_pts, uint32_t per_point,
                             const float* d_u0, const float* a, const float* b, const float* h,
                             uint64_t n) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "%s: NULL context", fn);
  if (per_point < 1) return fail(ctx, AF_ERR_INVALID_ARG, "%s: per_point must be >= 1", fn);
  if (n > (1ull << 40)) return fail(ctx, AF_ERR_INVALID_ARG, "%s: too many pairs", fn);
  if (n > 0 && (!d_pts || !d_u0 || !a || !b || !h))
    return fail(ctx, AF_ERR_INVALID_ARG, "%s: NULL input", fn);
  return AF_OK;
}

extern "C" af_status af_soft_seed(af_ctx* ctx, const float* d_normals, uint32_t m,
                                  const float* h_table, uint32_t K, float* d_u0, void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_soft_seed: NULL context");
  if (K < 1 || K > 65536 || !h_table)
    return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_seed: need a table of 1..65536 directions");
  if (m > 0 && (!d_normals || !d_u0)) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_seed: NULL buffer");
  for (uint32_t k = 0; k < 3 * K; ++k)
    if (!std::isfinite(h_table[k])) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_seed: non-finite table");
  cudaStream_t s = (cudaStream_t)stream;
  const bool same = ctx->h_table.size() == (size_t)K * 3 &&
                    std::memcmp(ctx->h_table.data(), h_table, (size_t)K * 3 * sizeof(float)) == 0;
  if (!same) {
    // the previous table may still be read by earlier launches
    AF_CUDA(ctx, cudaDeviceSynchronize());
    if (K > ctx->table_cap) {
      cudaFree(ctx->d_table);
      ctx->d_table = nullptr;
      ctx->table_cap = 0;
      AF_CUDA(ctx, cudaMalloc(&ctx->d_table, (size_t)K * 3 * sizeof(float)));
      ctx->table_cap = K;
    }
    AF_CUDA(ctx, cudaMemcpy(ctx->d_table, h_table, (size_t)K * 3 * sizeof(float),
                            cudaMemcpyHostToDevice));
    ctx->h_table.assign(h_table, h_table + (size_t)K * 3);
  }
  AF_CUDA(ctx, timed(ctx, 8, s, [&] {
    return af::launch_soft_seed(d_normals, m, ctx->d_table, K, d_u0, ctx->num_sms, s);
  }));
  ctx->last_stream = s;
  return AF_OK;
}

extern "C" af_status af_soft_clearance(af_ctx* ctx, const float* d_pts, uint32_t per_point,
                                       const float* d_u0, const float* d_alpha,
                                       const float* d_beta, const float* d_h, uint64_t n,
                                       float tau_s, float* d_c, float* d_cmin, void* stream) {
  af_status st = check_pairs(ctx, "af_soft_clearance", d_pts, per_point, d_u0, d_alpha, d_beta, d_h, n);
  if (st != AF_OK) return st;
  if (n > 0 && !d_c) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_clearance: NULL output");
  af::SoftView S;
  if ((st = soft_view(ctx, tau_s, &S)) != AF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = ensure_views(ctx, s)) != AF_OK) return st;
  view_fields(ctx, &S);
  AF_CUDA(ctx, timed(ctx, 5, s, [&] {
    return af::launch_soft(S, false, d_pts, per_point, d_u0, d_alpha, d_beta, d_h, n, nullptr,
                           d_c, d_cmin, nullptr, nullptr, nullptr, ctx->num_sms, s);
  }));
  ctx->last_stream = s;
  return AF_OK;
}

extern "C" af_status af_soft_clearance_adjoint(af_ctx* ctx, const float* d_pts, uint32_t per_point,
                                               const float* d_u0, const float* d_alpha,
                                               const float* d_beta, const float* d_h, uint64_t n,
                                               float tau_s, const float* d_gc, float* d_c,
                                               float* d_ga, float* d_gb, float* d_gh,
                                               void* stream) {
  af_status st = check_pairs(ctx, "af_soft_clearance_adjoint", d_pts, per_point, d_u0, d_alpha,
                             d_beta, d_h, n);
  if (st != AF_OK) return st;
  af::SoftView S;
  if ((st = soft_view(ctx, tau_s, &S)) != AF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = ensure_views(ctx, s)) != AF_OK) return st;
  view_fields(ctx, &S);
  AF_CUDA(ctx, timed(ctx, 6, s, [&] {
    return af::launch_soft(S, true, d_pts, per_point, d_u0, d_alpha, d_beta, d_h, n, d_gc, d_c,
                           nullptr, d_ga, d_gb, d_gh, ctx->num_sms, s);
  }));
  ctx->last_stream = s;
  return AF_OK;
}

extern "C" af_status af_soft_refine(af_ctx* ctx, const float* d_pts, uint32_t per_point,
                                    const float* d_u0, float* d_alpha, float* d_beta, float* d_h,
                                    uint64_t n, float tau_s, const af_refine* R, float* d_c,
                                    float* d_cmin, void* stream) {
  af_status st = check_pairs(ctx, "af_soft_refine", d_pts, per_point, d_u0, d_alpha, d_beta, d_h, n);
  if (st != AF_OK) return st;
  if (!R) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_refine: NULL parameters");
  if (R->steps > 100000 || !std::isfinite(R->lr_dir) || !std::isfinite(R->lr_h) ||
      !(R->h_max >= 0.f) || !std::isfinite(R->h_max))
    return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_refine: bad steps / step sizes / h_max");
  if (n > 0 && !d_c) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_refine: NULL output");
  af::SoftView S;
  if ((st = soft_view(ctx, tau_s, &S)) != AF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = ensure_views(ctx, s)) != AF_OK) return st;
  view_fields(ctx, &S);
  const af::RefineArgs A{(int)R->steps, R->lr_dir, R->lr_h, R->h_max};
  AF_CUDA(ctx, timed(ctx, 7, s, [&] {
    return af::launch_soft_refine(S, A, d_pts, per_point, d_u0, d_alpha, d_beta, d_h, n, d_c,
                                  d_cmin, ctx->num_sms, s);
  }));
  ctx->last_stream = s;
  return AF_OK;
}

extern "C" af_status af_soft_set_view(af_ctx* ctx, int32_t mode) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_soft_set_view: NULL context");
  if (mode < 0 || mode > 2) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_set_view: mode must be 0, 1 or 2");
  AF_CUDA(ctx, cudaDeviceSynchronize());
  cudaFree(ctx->d_dense);
  cudaFree(ctx->d_cells);
  cudaFree(ctx->d_bgrid);
  cudaFree(ctx->d_skeys);
  cudaFree(ctx->d_nslots);
  cudaFree(ctx->d_scells);
  ctx->d_dense = nullptr;
  ctx->d_cells = nullptr;
  ctx->d_bgrid = nullptr;
  ctx->d_skeys = nullptr;
  ctx->d_nslots = nullptr;
  ctx->d_scells = nullptr;
  ctx->scells_cap = 0;
  ctx->views_valid = false;
  ctx->soft_mode = mode;
  return AF_OK;
}

extern "C" af_status af_soft_best(af_ctx* ctx, const float* d_c, uint64_t n, uint32_t per_point,
                                  const float* d_u0, int32_t* d_best_k, float* d_best_c,
                                  float* d_best_u0, void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_soft_best: NULL context");
  if (per_point < 1) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_best: per_point must be >= 1");
  if (n > (1ull << 40)) return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_best: too many pairs");
  if (n > 0 && (!d_c || (d_best_u0 && !d_u0)))
    return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_best: NULL input");
  cudaStream_t s = (cudaStream_t)stream;
  AF_CUDA(ctx, timed(ctx, 9, s, [&] {
    return af::launch_soft_best(d_c, n, per_point, d_u0, d_best_k, d_best_c, d_best_u0,
                                ctx->num_sms, s);
  }));
  ctx->last_stream = s;
  return AF_OK;
}

extern "C" af_status af_soft_start(af_ctx* ctx, const uint8_t* d_label, const int16_t* d_best,
                                   uint32_t m, float* d_u0, void* stream) {
  if (!ctx) return fail(nullptr, AF_ERR_INVALID_ARG, "af_soft_start: NULL context");
  if (!ctx->has_tool) return fail(ctx, AF_ERR_STATE, "af_soft_start: call af_set_tool first");
  if (m > 0 && (!d_label || !d_best || !d_u0))
    return fail(ctx, AF_ERR_INVALID_ARG, "af_soft_start: NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  AF_CUDA(ctx, timed(ctx, 8, s, [&] {
    return af::launch_soft_start(d_label, d_best, m, ctx->T.dirs, ctx->T.G, d_u0, ctx->num_sms, s);
  }));
  ctx->last_stream = s;
  return AF_OK;
}
