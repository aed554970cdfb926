// af_batch.cu -- batched ticks: many maps (scenes), each with its own scan,
// tool and direction set, integrated and scored together by one CUDA graph
// of persistent kernels (allocation, integration, bit view, scoring) per
// tick. Work is laid out as prefix sums over the batch, so uneven scenes
// share the grid without idle CTAs. The integration tile (returns per CTA)
// and the scoring CTA size are chosen online by an autotuner that times the
// candidate launch shapes on the first ticks; every shape computes the same
// result, so tuning never changes a label.
#include <af.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "af_ctx.cuh"
#include "af_internal.cuh"

namespace af {
cudaError_t launch_batch_integrate(const BatchHdr* B, const SceneDesc* D, uint32_t count, int m,
                                   int tile, int num_sms, cudaStream_t stream);
cudaError_t launch_score_batch(const BatchHdr* B, const SceneDesc* D, int warps, int num_sms,
                               cudaStream_t stream);
void set_global_error(const char* msg);
}  // namespace af

namespace {

constexpr int kTiles[3] = {8, 16, 32};
constexpr int kWarps[3] = {2, 4, 8};
constexpr int kCandidates = 9;  // kTiles x kWarps
constexpr int kRepeats = 2;     // ticks timed per candidate

af_status bfail(af_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  af::set_global_error(buf);
  return s;
}

}  // namespace

struct af_batch {
  std::vector<af_ctx*> scenes;
  uint32_t count = 0;
  int m = 0;  // shared cube radius
  int num_sms = 0;
  size_t bytes = 0;                 // header + descriptors
  unsigned char* d_desc = nullptr;  // device copy read by the kernels
  unsigned char* h_desc[2] = {nullptr, nullptr};  // pinned, alternating ticks
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int buf = 0;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec[2][kCandidates] = {};
  // tuning
  cudaEvent_t t0[2] = {nullptr, nullptr}, t1[2] = {nullptr, nullptr};
  int timed_cfg[2] = {-1, -1};
  float sum_ms[kCandidates] = {0};
  int runs[kCandidates] = {0};
  uint64_t ticks = 0;
  int fixed = -1;   // candidate set by af_batch_set_tuning
  int chosen = -1;  // candidate chosen by the tuner
};

namespace {

int cand_of(int tile_i, int warps_i) { return tile_i * 3 + warps_i; }

void destroy(af_batch* b) {
  for (int i = 0; i < 2; ++i) {
    for (int c = 0; c < kCandidates; ++c)
      if (b->exec[i][c]) cudaGraphExecDestroy(b->exec[i][c]);
    if (b->done[i]) cudaEventDestroy(b->done[i]);
    if (b->t0[i]) cudaEventDestroy(b->t0[i]);
    if (b->t1[i]) cudaEventDestroy(b->t1[i]);
    if (b->h_desc[i]) cudaFreeHost(b->h_desc[i]);
  }
  if (b->capture) cudaStreamDestroy(b->capture);
  cudaFree(b->d_desc);
  delete b;
}

// Captures the graph of candidate c reading the pinned descriptors of buffer i.
af_status build_graph(af_batch* b, int i, int c) {
  const auto* B = reinterpret_cast<const af::BatchHdr*>(b->d_desc);
  const auto* D = reinterpret_cast<const af::SceneDesc*>(b->d_desc + 64);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemcpyAsync(b->d_desc, b->h_desc[i], b->bytes, cudaMemcpyHostToDevice, b->capture);
    af::launch_batch_integrate(B, D, b->count, b->m, kTiles[c / 3], b->num_sms, b->capture);
    af::launch_score_batch(B, D, kWarps[c % 3], b->num_sms, b->capture);
    e = cudaStreamEndCapture(b->capture, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[i][c], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return bfail(AF_ERR_CUDA, "af_batch: graph capture failed: %s", cudaGetErrorString(e));
  return AF_OK;
}

// Mean time of candidate c, or a large value while untimed.
float mean_ms(const af_batch* b, int c) {
  return b->runs[c] ? b->sum_ms[c] / b->runs[c] : 1e30f;
}

int choose(af_batch* b) {
  if (b->fixed >= 0) return b->fixed;
  if (b->chosen >= 0) return b->chosen;
  const uint64_t t = b->ticks;
  if (t < (uint64_t)kCandidates * kRepeats) return (int)(t / kRepeats);  // explore
  bool all = true;
  for (int c = 0; c < kCandidates; ++c) all = all && b->runs[c] >= kRepeats;
  int best = 0;
  for (int c = 1; c < kCandidates; ++c)
    if (mean_ms(b, c) < mean_ms(b, best)) best = c;
  if (all) b->chosen = best;
  return best;
}

}  // namespace

extern "C" af_status af_batch_create(af_ctx* const* scenes, uint32_t count, af_batch** out) {
  if (!scenes || !out || count < 1 || count > 4096)
    return bfail(AF_ERR_INVALID_ARG, "af_batch_create: need 1 <= count <= 4096 contexts");
  *out = nullptr;
  for (uint32_t s = 0; s < count; ++s) {
    if (!scenes[s]) return bfail(AF_ERR_INVALID_ARG, "af_batch_create: NULL context %u", s);
    for (uint32_t r = 0; r < s; ++r)
      if (scenes[r] == scenes[s])
        return bfail(AF_ERR_INVALID_ARG, "af_batch_create: context %u appears twice", s);
    if (scenes[s]->cfg.cube_radius != scenes[0]->cfg.cube_radius)
      return bfail(AF_ERR_INVALID_ARG, "af_batch_create: all maps need the same cube radius");
  }
  af_batch* b = new af_batch();
  b->scenes.assign(scenes, scenes + count);
  b->count = count;
  b->m = scenes[0]->cfg.cube_radius;
  b->num_sms = scenes[0]->num_sms;
  b->bytes = 64 + (size_t)count * sizeof(af::SceneDesc);
  cudaError_t e = cudaMalloc((void**)&b->d_desc, b->bytes);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMallocHost((void**)&b->h_desc[i], b->bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t0[i]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t1[i]);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    destroy(b);
    return bfail(AF_ERR_CUDA, "af_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return AF_OK;
}

extern "C" af_status af_batch_destroy(af_batch* b) {
  if (!b) return bfail(AF_ERR_INVALID_ARG, "af_batch_destroy: NULL batch");
  cudaDeviceSynchronize();
  destroy(b);
  return AF_OK;
}

extern "C" af_status af_batch_set_tuning(af_batch* b, uint32_t returns_per_tile,
                                         uint32_t warps_per_cta) {
  if (!b) return bfail(AF_ERR_INVALID_ARG, "af_batch_set_tuning: NULL batch");
  if (returns_per_tile == 0 && warps_per_cta == 0) {
    b->fixed = -1;  // back to the online tuner
    return AF_OK;
  }
  int ti = -1, wi = -1;
  for (int k = 0; k < 3; ++k) {
    if ((int)returns_per_tile == kTiles[k]) ti = k;
    if ((int)warps_per_cta == kWarps[k]) wi = k;
  }
  if (ti < 0 || wi < 0)
    return bfail(AF_ERR_INVALID_ARG, "af_batch_set_tuning: tile must be 8/16/32, warps 2/4/8");
  b->fixed = cand_of(ti, wi);
  return AF_OK;
}

extern "C" af_status af_batch_get_tuning(af_batch* b, af_batch_tuning* out) {
  if (!b || !out) return bfail(AF_ERR_INVALID_ARG, "af_batch_get_tuning: NULL argument");
  for (int i = 0; i < 2; ++i)
    if (b->used[i]) cudaEventSynchronize(b->done[i]);
  // collect any timing still pending
  for (int i = 0; i < 2; ++i)
    if (b->timed_cfg[i] >= 0) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, b->t0[i], b->t1[i]) == cudaSuccess) {
        b->sum_ms[b->timed_cfg[i]] += ms;
        b->runs[b->timed_cfg[i]] += 1;
      }
      b->timed_cfg[i] = -1;
    }
  const int c = b->fixed >= 0 ? b->fixed : (b->chosen >= 0 ? b->chosen : -1);
  std::memset(out, 0, sizeof *out);
  out->returns_per_tile = c >= 0 ? kTiles[c / 3] : 0;
  out->warps_per_cta = c >= 0 ? kWarps[c % 3] : 0;
  out->done = c >= 0;
  for (int k = 0; k < kCandidates; ++k) {
    out->ms[k] = b->runs[k] ? b->sum_ms[k] / b->runs[k] : 0.f;
    out->explored += b->runs[k] > 0;
  }
  return AF_OK;
}

extern "C" af_status af_batch_tick(af_batch* b, const af_batch_item* items, void* stream) {
  if (!b || !items) return bfail(AF_ERR_INVALID_ARG, "af_batch_tick: NULL argument");
  for (uint32_t s = 0; s < b->count; ++s) {
    const af_batch_item& it = items[s];
    const af_ctx* c = b->scenes[s];
    if (it.n > c->cfg.max_returns)
      return bfail(AF_ERR_CAPACITY, "af_batch_tick: scene %u: n exceeds max_returns", s);
    if ((it.n > 0 && !it.d_xyz) ||
        (it.m > 0 && (!it.d_pts || !it.d_normals || !it.d_label || !it.d_best)))
      return bfail(AF_ERR_INVALID_ARG, "af_batch_tick: scene %u: NULL buffer", s);
    if (it.m > 0 && !c->has_tool)
      return bfail(AF_ERR_STATE, "af_batch_tick: scene %u has no tool (af_set_tool)", s);
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(it.pose[k]))
        return bfail(AF_ERR_INVALID_ARG, "af_batch_tick: scene %u: non-finite pose", s);
  }
  const int i = b->buf;
  if (b->used[i]) {
    cudaError_t e = cudaEventSynchronize(b->done[i]);  // the tick that last read h_desc[i]
    if (e != cudaSuccess) return bfail(AF_ERR_CUDA, "af_batch_tick: %s", cudaGetErrorString(e));
    if (b->timed_cfg[i] >= 0) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, b->t0[i], b->t1[i]) == cudaSuccess) {
        b->sum_ms[b->timed_cfg[i]] += ms;
        b->runs[b->timed_cfg[i]] += 1;
      }
      b->timed_cfg[i] = -1;
    }
  }
  const int c = choose(b);
  const int tile = kTiles[c / 3];

  // descriptors: header, then one SceneDesc per map
  auto* H = reinterpret_cast<af::BatchHdr*>(b->h_desc[i]);
  auto* D = reinterpret_cast<af::SceneDesc*>(b->h_desc[i] + 64);
  uint32_t alloc_off = 0, tile_off = 0, pt_off = 0;
  for (uint32_t s = 0; s < b->count; ++s) {
    af_ctx* ctx = b->scenes[s];
    const af_batch_item& it = items[s];
    af::SceneDesc& d = D[s];
    std::memset(&d, 0, sizeof d);
    d.M = ctx->M;
    d.T = ctx->T;
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 4; ++k) d.P.r[r][k] = it.pose[4 * r + k];
    d.xyz = it.d_xyz;
    d.ret = ctx->d_ret;
    d.pts = it.d_pts;
    d.nrm = it.d_normals;
    d.label = it.d_label;
    d.best = it.d_best;
    d.n = it.n;
    d.m = it.m;
    ctx->frame = ctx->frame + 1 >= 0xFFFFFFFFu ? 1 : ctx->frame + 1;
    d.frame = ctx->frame;
    d.alloc_off = alloc_off;
    d.tile_off = tile_off;
    d.pt_off = pt_off;
    alloc_off += it.n * (uint32_t)(ctx->M.nbmax + ctx->M.ns);
    tile_off += (it.n + tile - 1) / tile;
    pt_off += it.m;
  }
  H->count = b->count;
  H->total_alloc = alloc_off;
  H->total_tiles = tile_off;
  H->total_points = pt_off;

  if (!b->exec[i][c]) {
    const af_status st = build_graph(b, i, c);
    if (st != AF_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool timing = b->fixed < 0 && b->chosen < 0;
  if (timing) cudaEventRecord(b->t0[i], s);
  cudaError_t e = cudaGraphLaunch(b->exec[i][c], s);
  if (e != cudaSuccess)
    return bfail(AF_ERR_CUDA, "af_batch_tick: graph launch failed: %s", cudaGetErrorString(e));
  if (timing) {
    cudaEventRecord(b->t1[i], s);
    b->timed_cfg[i] = c;
  }
  cudaEventRecord(b->done[i], s);
  b->used[i] = true;
  b->buf ^= 1;
  b->ticks++;
  for (uint32_t k = 0; k < b->count; ++k) {
    af_ctx* ctx = b->scenes[k];
    ctx->scans++;
    ctx->returns_in += items[k].n;
    ctx->points_in += items[k].m;
    ctx->last_stream = s;
  }
  return AF_OK;
}
