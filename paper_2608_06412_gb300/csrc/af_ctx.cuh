// af_ctx.cuh -- the context behind the opaque af_ctx handle of include/af.h,
// shared by the host-side files of libaf.
#pragma once

#include <af.h>

#include <vector>

#include "af_internal.cuh"

struct af_ctx {
  af_config cfg;
  af::MapView M;
  int num_sms = 0;
  uint32_t frame = 0;
  cudaStream_t last_stream = nullptr;
  // scratch
  float4* d_ret = nullptr;
  float* d_xyz = nullptr;
  float* d_pts = nullptr;
  float* d_nrm = nullptr;
  uint8_t* d_label = nullptr;
  int16_t* d_best = nullptr;
  uint32_t* h_status = nullptr;  // pinned
  // tool tables
  bool has_tool = false;
  af::ToolView T{};
  float* d_dirs = nullptr;
  short4* d_runs = nullptr;
  int2* d_fruns = nullptr;
  int4* d_dtab = nullptr;
  short4* d_arm = nullptr;
  af_tool tool{};
  // views of the differentiable form (built on first use, rebuilt when the
  // map has changed since)
  float* d_dense = nullptr;
  float4* d_cells = nullptr;
  uint32_t* d_bgrid = nullptr;   // the brick-sparse view: slot per grid brick
  uint32_t* d_skeys = nullptr;   // grid brick of every slot
  uint32_t* d_nslots = nullptr;
  float4* d_scells = nullptr;    // 512 cell records per slot
  uint32_t scells_cap = 0;
  int soft_mode = 0;             // af_soft_set_view: 0 automatic, 1 dense, 2 sparse
  bool views_sparse = false;     // the view built is the sparse one
  bool views_valid = false;
  uint32_t views_frame = 0;
  float* d_table = nullptr;  // seed directions, and their host copy
  uint32_t table_cap = 0;
  std::vector<float> h_table;
  // the stateful point layer (af_points_enable)
  bool pts_on = false;
  af_points_config pcfg{};
  int32_t* d_pid = nullptr;
  af::PtState* d_pst = nullptr;
  float4* d_pviews = nullptr;
  unsigned long long* d_pnew = nullptr;
  uint32_t* d_pnear = nullptr;
  unsigned long long* d_psnapw = nullptr;  // trigger (ii): dirty bricks before the scan
  uint32_t* d_psnapc = nullptr;
  uint32_t* d_pchgmask = nullptr;
  uint32_t* d_phist = nullptr;
  af::PtSample* d_psamp = nullptr;
  uint32_t pts_frames = 0;       // af_points_frame calls (the draw's salt)
  bool pts_snapshot = false;     // af_integrate_scan copies the dirty bricks after allocation
  uint32_t* d_psel = nullptr;
  uint32_t* d_pblock = nullptr;
  af::PtCounters* d_pcount = nullptr;
  int4* d_pnnoff = nullptr;
  int pnoff = 0;
  int4* d_pc2f = nullptr;     // coarse-to-fine neighbour ball
  int pc2f_noff = 0, pc2f_R = 0;
  int16_t* d_psnap = nullptr;
  // work sharing of af_score (af_set_score_split)
  int2* d_over = nullptr;
  uint32_t* d_sres = nullptr;
  uint32_t* d_scount = nullptr;
  uint32_t split_cap = 0;
  int score_budget = -1;
  // the projective ablation's range image (af_integrate_scan_projective)
  unsigned* d_img = nullptr;
  size_t img_cap = 0;
  float q_last[3] = {0.f, 0.f, 0.f};
  bool have_q_last = false;
  // host counters
  uint64_t scans = 0, returns_in = 0, points_in = 0;
  // kernel profiling: CUDA events around each launch on its own stream
  bool prof_on = false;
  struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
    int kernels;  // kernel launches inside the bracket
  };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_free;
  char err[512] = {0};
};
