// api.cu -- C ABI of libhweno (declared in include/hweno.h).
//
// Host logic only: argument validation, workspace allocation, ordering
// against the caller's stream, the device-resident time-step control and the
// CUDA graph that replays whole SSP-RK3 steps (ctl_begin, stage 1, stage 2,
// stage 3, ctl_end).  All arithmetic of the scheme runs in the kernels.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hweno.h"
#include "hweno_types.h"
#include "kernels.h"

namespace {

thread_local std::string g_err = "no error";

hweno_status fail(hweno_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define HW_CK(x)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? HWENO_ERR_OOM : HWENO_ERR_CUDA, \
                  "%s failed: %s", #x, cudaGetErrorString(e_));                     \
  } while (0)

#define HW_TRY(x)                       \
  do {                                          \
    hweno_status s_ = (x);                      \
    if (s_ != HWENO_OK) return s_;              \
  } while (0)

constexpr int kGraphSteps = 16;

// NVTX range over a scope: the library's phases (state transfer, graph
// capture and replay, stage launches, indicator, autotuning) show up by name
// on an Nsight timeline; without an attached tool each call is a no-op.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

hweno_status validate(const hweno_config* c, int expect_dim) {
  if (!c) return fail(HWENO_ERR_ARG, "config is NULL");
  if (c->dim != 1 && c->dim != 2) return fail(HWENO_ERR_ARG, "dim must be 1 or 2 (got %d)", c->dim);
  if (expect_dim && c->dim != expect_dim) return fail(HWENO_ERR_ARG, "all configs of a batch need the same dim");
  if (c->nx < 3 || (c->dim == 2 && c->ny < 3))
    return fail(HWENO_ERR_ARG, "need at least 3 cells per direction (nx=%d ny=%d)", c->nx, c->ny);
  if ((long long)c->nx * (c->dim == 2 ? c->ny : 1) > (1LL << 31))
    return fail(HWENO_ERR_ARG, "grid too large (more than 2^31 cells)");
  if (!std::isfinite(c->xlo) || !std::isfinite(c->xhi) ||
      (c->dim == 2 && (!std::isfinite(c->ylo) || !std::isfinite(c->yhi))))
    return fail(HWENO_ERR_ARG, "domain bounds must be finite");
  if (!(c->xhi > c->xlo) || (c->dim == 2 && !(c->yhi > c->ylo)))
    return fail(HWENO_ERR_ARG, "empty domain");
  if (c->equation < 0 || c->equation > 2) return fail(HWENO_ERR_ARG, "unknown equation %d", c->equation);
  if (c->equation == HWENO_EQ_EULER && !(c->gamma_gas > 1.0 && std::isfinite(c->gamma_gas)))
    return fail(HWENO_ERR_ARG, "gamma_gas must be finite and exceed 1");
  if (c->equation == HWENO_EQ_ADVECTION &&
      (!std::isfinite(c->adv_x) || (c->dim == 2 && !std::isfinite(c->adv_y))))
    return fail(HWENO_ERR_ARG, "advection speeds must be finite");
  const int nw = c->dim == 1 ? 3 : 5;
  double s = 0.0;
  for (int m = 0; m < nw; ++m) {
    if (!(c->lin_w[m] > 0.0)) return fail(HWENO_ERR_ARG, "linear weight %d must be positive", m);
    s += c->lin_w[m];
  }
  if (std::fabs(s - 1.0) > 1e-12) return fail(HWENO_ERR_ARG, "linear weights must sum to 1 (sum %.17g)", s);
  if (!(c->eps > 0.0) || !std::isfinite(c->eps)) return fail(HWENO_ERR_ARG, "eps must be positive and finite");
  if (c->weight_pow != 1 && c->weight_pow != 2) return fail(HWENO_ERR_ARG, "weight_pow must be 1 or 2");
  if (c->smoothness != HWENO_BETA_MOMENT && c->smoothness != HWENO_BETA_TYPICAL)
    return fail(HWENO_ERR_ARG, "smoothness must be HWENO_BETA_MOMENT or HWENO_BETA_TYPICAL");
  if (!(c->cfl > 0.0) || !std::isfinite(c->cfl)) return fail(HWENO_ERR_ARG, "cfl must be positive and finite");
  if (c->dt_rule != HWENO_DT_CFL && c->dt_rule != HWENO_DT_CFL_DX53) return fail(HWENO_ERR_ARG, "bad dt_rule");
  if (c->precision != HWENO_FP64 && c->precision != HWENO_FP32 && c->precision != HWENO_FP32_IND64)
    return fail(HWENO_ERR_ARG, "bad precision");
  const int nsides = c->dim == 1 ? 2 : 4;
  for (int k = 0; k < nsides; ++k) {
    if (c->bc[k] < 0 || c->bc[k] > HWENO_BC_SHOCK) return fail(HWENO_ERR_ARG, "bad boundary condition on side %d", k);
    if (c->dim == 1 && c->bc[k] >= HWENO_BC_SPLIT)
      return fail(HWENO_ERR_ARG, "split and moving-shock boundaries need a 2D grid (side %d)", k);
  }
  for (int a = 0; a < c->dim; ++a)
    if ((c->bc[2 * a] == HWENO_BC_PERIODIC) != (c->bc[2 * a + 1] == HWENO_BC_PERIODIC))
      return fail(HWENO_ERR_ARG, "periodic boundaries must be paired (axis %d)", a);
  return HWENO_OK;
}

// The 2D grid descriptor of a configuration.
hw::Grid2 grid_of(const hweno_config& c) {
  hw::Grid2 g{};
  g.nx = c.nx;
  g.ny = c.ny;
  for (int q = 0; q < 4; ++q) {
    g.bc[q] = c.bc[q];
    for (int r = 0; r < 4; ++r) {
      g.st[q][r] = c.bc_state[q][r];
      g.st2[q][r] = c.bc_state2[q][r];
    }
    g.bcp[q][0] = c.bc_param[q][0];
    g.bcp[q][1] = c.bc_param[q][1];
  }
  g.dx = (c.xhi - c.xlo) / c.nx;
  g.dy = (c.yhi - c.ylo) / c.ny;
  g.xlo = c.xlo;
  g.ylo = c.ylo;
  return g;
}

}  // namespace

namespace hw {
// Error reporting and config validation for entry points defined in other
// translation units (the allocation-free step).
hweno_status report_error(hweno_status st, const char* msg) { return fail(st, "%s", msg); }
hweno_status check_config(const hweno_config* cfg, int expect_dim) { return validate(cfg, expect_dim); }
}  // namespace hw

// A device buffer or an event owned by one scope: released on every return
// path, the error returns of HW_CK included.
struct ScopedDev {
  void* p = nullptr;
  ~ScopedDev() { if (p) cudaFree(p); }
};
struct ScopedEvent {
  cudaEvent_t e = nullptr;
  ~ScopedEvent() { if (e) cudaEventDestroy(e); }
};

// One engine serves both a single grid (n_inst = 1) and a 1D batch.
struct Engine {
  hweno_config cfg{};
  int dim = 1, nc = 1, nf = 2, nd = 1, prec = HWENO_FP64;
  size_t esz = 8;
  long long cells = 0;   // per field plane (all instances)
  int n_inst = 0;
  int num_sms = 148;
  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ev = nullptr;
  void *S = nullptr, *A = nullptr, *B = nullptr, *H = nullptr;
  hw::Ctl* ctl = nullptr;        // device: advance control
  hw::Ctl* ctl_manual = nullptr; // device: hweno_step control
  hw::Ctl* ctl_host = nullptr;   // pinned mirror
  std::vector<hw::Ctl> ctl_init;
  hw::Inst1* inst_d = nullptr;
  std::vector<hw::Inst1> inst_h;
  std::vector<long long> offsets;
  int2* tasks_d = nullptr;
  int ntasks = 0;
  double* alpha_op = nullptr;    // device [n_inst] (1D) or [n_inst][2] (2D batch)
  hw::Grid2 grid{};
  // 2D batch: per-instance descriptors and the tile table over all instances
  bool batch2 = false;
  std::vector<hw::Inst2> inst2_h;
  hw::Inst2* inst2_d = nullptr;
  hw::Tile2* tiles2_d = nullptr;
  long long ntiles2 = 0;
  unsigned* sched_d = nullptr;   // the 2D stage kernel's tile scheduler (2 words, self-resetting)
  hw::WeightParams wp{};
  cudaGraphExec_t gexec = nullptr;
  bool has_state = false;
  hw::LaunchShape shape;          // chosen by the autotuner
  // opt-in timing of every stage launch with CUDA events (direct launches)
  bool prof = false;
  std::vector<cudaEvent_t> pev;   // 2 per stage launch of one poll window
  int pev_used = 0;
  double prof_stage_ms = 0.0, prof_total_ms = 0.0;
  long long prof_stage_launches = 0, prof_launches = 0;
  // learned troubled-cell indicator (2D): FP16 weights and the per-step masks
  bool learned = false;
  __half* mlp_w = nullptr;            // W1h [32][80] then W2h [32][32]
  float* mlp_bias = nullptr;          // b1, b2, w3, b3
  unsigned char* troubled = nullptr;  // network output per cell
  unsigned char* smooth = nullptr;    // dilated complement: 1 = linear path
  float z_thresh = 0.f;
  // hweno_stage: the stage that ran last (0: none pending) and its step's
  // dt, alpha and start time
  int stage_done = 0;
  double st_dt = 0.0, st_ax = 0.0, st_ay = 0.0, st_t0 = 0.0;

  ~Engine() {
    for (cudaEvent_t e : pev) cudaEventDestroy(e);
    if (gexec) cudaGraphExecDestroy(gexec);
    cudaFree(S); cudaFree(A); cudaFree(B); cudaFree(H);
    cudaFree(ctl); cudaFree(ctl_manual); cudaFree(inst_d); cudaFree(tasks_d); cudaFree(alpha_op);
    cudaFree(inst2_d); cudaFree(tiles2_d); cudaFree(sched_d);
    cudaFree(mlp_w); cudaFree(mlp_bias); cudaFree(troubled); cudaFree(smooth);
    if (ctl_host) cudaFreeHost(ctl_host);
    if (ev) cudaEventDestroy(ev);
    if (own) cudaStreamDestroy(own);
  }

  hweno_status init(int n, const hweno_config* cfgs, void* stream, bool batch = false) {
    cfg = cfgs[0];
    batch2 = batch && cfg.dim == 2;
    dim = cfg.dim;
    nc = cfg.equation == HWENO_EQ_EULER ? (dim == 1 ? 3 : 4) : 1;
    nf = nc * (dim + 1);
    nd = nc * dim;
    prec = cfg.precision;
    esz = prec == HWENO_FP64 ? 8 : 4;
    n_inst = n;
    user = static_cast<cudaStream_t>(stream);
    int dev = 0;
    HW_CK(cudaGetDevice(&dev));
    HW_CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    HW_CK(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    HW_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    wp = hw::weight_params(cfg);

    ctl_init.resize(n);
    if (dim == 1) {
      inst_h.resize(n);
      offsets.resize(n + 1);
      std::vector<int2> tasks;
      long long off = 0;
      for (int k = 0; k < n; ++k) {
        const hweno_config& c = cfgs[k];
        hw::Inst1& I = inst_h[k];
        I.off = off;
        I.n = c.nx;
        I.bc_lo = c.bc[0];
        I.bc_hi = c.bc[1];
        hw::set_spacing(I, c.xlo, c.xhi, c.nx);
        for (int q = 0; q < 4; ++q) { I.st_lo[q] = c.bc_state[0][q]; I.st_hi[q] = c.bc_state[1][q]; }
        offsets[k] = off;
        for (int s = 0; s < c.nx; s += hw::kTile1) tasks.push_back(make_int2(k, s));
        off += c.nx;
        hw::Ctl& C = ctl_init[k];
        std::memset(&C, 0, sizeof C);
        C.hx = c.dt_rule == HWENO_DT_CFL_DX53 ? std::pow(I.dx, 5.0 / 3.0) : I.dx;
        C.hy = 1.0;
        C.cfl = c.cfl;
        C.done = 1;
      }
      offsets[n] = off;
      cells = off;
      ntasks = (int)tasks.size();
      HW_CK(cudaMalloc(&inst_d, sizeof(hw::Inst1) * n));
      HW_CK(cudaMemcpy(inst_d, inst_h.data(), sizeof(hw::Inst1) * n, cudaMemcpyHostToDevice));
      HW_CK(cudaMalloc(&tasks_d, sizeof(int2) * tasks.size()));
      HW_CK(cudaMemcpy(tasks_d, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice));
    } else if (batch2) {
      inst2_h.resize(n);
      offsets.resize(n + 1);
      std::vector<hw::Tile2> tiles;
      long long off = 0;
      for (int k = 0; k < n; ++k) {
        const hweno_config& c = cfgs[k];
        hw::Inst2& I = inst2_h[k];
        I.off = off;
        I.grid = grid_of(c);
        I.idx = 1.0 / I.grid.dx;
        I.idy = 1.0 / I.grid.dy;
        I.dyx = I.grid.dy / I.grid.dx;
        I.dxy = I.grid.dx / I.grid.dy;
        I.idxf = (float)I.idx; I.idyf = (float)I.idy; I.dyxf = (float)I.dyx; I.dxyf = (float)I.dxy;
        offsets[k] = off;
        for (int j0 = 0; j0 < c.ny; j0 += hw::kTile2)
          for (int i0 = 0; i0 < c.nx; i0 += hw::kTile2) tiles.push_back(hw::Tile2{k, i0, j0, 0});
        off += (long long)c.nx * c.ny;
        hw::Ctl& C = ctl_init[k];
        std::memset(&C, 0, sizeof C);
        const bool r53 = c.dt_rule == HWENO_DT_CFL_DX53;
        C.hx = r53 ? std::pow(I.grid.dx, 5.0 / 3.0) : I.grid.dx;
        C.hy = r53 ? std::pow(I.grid.dy, 5.0 / 3.0) : I.grid.dy;
        C.cfl = c.cfl;
        C.done = 1;
      }
      offsets[n] = off;
      cells = off;
      grid = inst2_h[0].grid;
      ntiles2 = (long long)tiles.size();
      HW_CK(cudaMalloc(&inst2_d, sizeof(hw::Inst2) * n));
      HW_CK(cudaMemcpy(inst2_d, inst2_h.data(), sizeof(hw::Inst2) * n, cudaMemcpyHostToDevice));
      HW_CK(cudaMalloc(&tiles2_d, sizeof(hw::Tile2) * tiles.size()));
      HW_CK(cudaMemcpy(tiles2_d, tiles.data(), sizeof(hw::Tile2) * tiles.size(), cudaMemcpyHostToDevice));
      HW_CK(hw::prepare_stage2d(prec, cfg.equation, cfg.charwise, wp, true));
    } else {
      grid = grid_of(cfg);
      cells = (long long)cfg.nx * cfg.ny;
      offsets = {0, cells};
      hw::Ctl& C = ctl_init[0];
      std::memset(&C, 0, sizeof C);
      const bool r53 = cfg.dt_rule == HWENO_DT_CFL_DX53;
      C.hx = r53 ? std::pow(grid.dx, 5.0 / 3.0) : grid.dx;
      C.hy = r53 ? std::pow(grid.dy, 5.0 / 3.0) : grid.dy;
      C.cfl = cfg.cfl;
      C.done = 1;
      HW_CK(hw::prepare_stage2d(prec, cfg.equation, cfg.charwise, wp, false));
    }
    const size_t plane = (size_t)cells * esz;
    HW_CK(cudaMalloc(&S, plane * nf));
    HW_CK(cudaMalloc(&A, plane * nf));
    HW_CK(cudaMalloc(&B, plane * nf));
    HW_CK(cudaMalloc(&H, plane * nd));
    HW_CK(cudaMalloc(&ctl, sizeof(hw::Ctl) * n));
    HW_CK(cudaMalloc(&ctl_manual, sizeof(hw::Ctl) * n));
    HW_CK(cudaMalloc(&alpha_op, sizeof(double) * 2 * n));
    HW_CK(cudaMalloc(&sched_d, sizeof(unsigned) * 2));
    HW_CK(cudaMemset(sched_d, 0, sizeof(unsigned) * 2));
    HW_CK(cudaMallocHost(&ctl_host, sizeof(hw::Ctl) * n));
    HW_CK(cudaMemcpy(ctl, ctl_init.data(), sizeof(hw::Ctl) * n, cudaMemcpyHostToDevice));
    HW_CK(cudaMemcpy(ctl_manual, ctl_init.data(), sizeof(hw::Ctl) * n, cudaMemcpyHostToDevice));
    return HWENO_OK;
  }

  // order own stream after the caller's, and the caller's after own
  hweno_status enter() {
    HW_CK(cudaEventRecord(ev, user));
    HW_CK(cudaStreamWaitEvent(own, ev, 0));
    return HWENO_OK;
  }
  hweno_status leave() {
    HW_CK(cudaEventRecord(ev, own));
    HW_CK(cudaStreamWaitEvent(user, ev, 0));
    return HWENO_OK;
  }

  hweno_status stage(int s, const void* in, void* out, hw::Ctl* c, double ax, double ay,
                     void* hat) {
    static const char* kNames[4] = {"hweno.operator", "hweno.stage1", "hweno.stage2", "hweno.stage3"};
    Range r(kNames[s]);
    if (dim == 1) {
      hw::Stage1Args a{};
      a.in = in; a.base = S; a.out = out; a.hat = hat;
      a.inst = inst_d; a.tasks = tasks_d; a.ntasks = ntasks; a.total = cells;
      a.ctl = c; a.alpha_op = alpha_op; a.stage = s;
      a.gamma_gas = cfg.gamma_gas; a.adv = cfg.adv_x; a.wp = wp;
      a.gammaf = (float)cfg.gamma_gas; a.advf = (float)cfg.adv_x;
      HW_CK(hw::launch_stage1d(prec, cfg.equation, cfg.charwise, a, num_sms, own, shape));
    } else {
      hw::Stage2Args a{};
      a.in = in; a.base = S; a.out = out; a.hat = hat;
      a.grid = grid; a.ctl = c; a.ax_op = ax; a.ay_op = ay; a.stage = s;
      a.gamma_gas = cfg.gamma_gas; a.adv_x = cfg.adv_x; a.adv_y = cfg.adv_y; a.wp = wp;
      a.f32 = hw::stage2_f32(grid, ax, ay, cfg.gamma_gas, cfg.adv_x, cfg.adv_y);
      a.plane = cells;
      a.smooth = learned && s > 0 ? smooth : nullptr;
      a.sched = sched_d;
      if (batch2) {
        a.batched = 1;
        a.inst = inst2_d;
        a.tiles = tiles2_d;
        a.ntiles = ntiles2;
        a.alpha_op = alpha_op;
      }
      HW_CK(hw::launch_stage2d(prec, cfg.equation, cfg.charwise, a, num_sms, own, shape));
    }
    return HWENO_OK;
  }

  // the three stages of Step 4 under control block c
  hweno_status timed_stage(int s, const void* in, void* out, hw::Ctl* c) {
    const bool t = prof && pev_used + 2 <= (int)pev.size();
    if (t) HW_CK(cudaEventRecord(pev[pev_used], own));
    HW_TRY(stage(s, in, out, c, 0, 0, H));
    if (t) {
      HW_CK(cudaEventRecord(pev[pev_used + 1], own));
      pev_used += 2;
    }
    return HWENO_OK;
  }

  hweno_status rk_stages(hw::Ctl* c) {
    HW_TRY(timed_stage(1, S, A, c));
    HW_TRY(timed_stage(2, A, B, c));
    HW_TRY(timed_stage(3, B, S, c));
    return HWENO_OK;
  }

  hweno_status run_indicator() {
    Range r("hweno.indicator");
    hw::MlpDev m{mlp_w, mlp_w + 32 * 80, mlp_bias, z_thresh};
    HW_CK(hw::launch_mlp_infer2d(prec, cfg.equation, S, grid, cells, m, ctl, troubled, smooth, num_sms, own));
    return HWENO_OK;
  }

  hweno_status one_step() {
    HW_CK(hw::launch_ctl_begin(ctl, n_inst, dim, own));
    if (learned) HW_TRY(run_indicator());  // once per step, on u^n; reused by the 3 stages
    HW_TRY(rk_stages(ctl));
    HW_CK(hw::launch_ctl_end(ctl, n_inst, own));
    return HWENO_OK;
  }

  // fold the recorded stage timings of the last poll window into the totals
  hweno_status collect_prof() {
    for (int k = 0; k + 1 < pev_used; k += 2) {
      float ms = 0.f;
      HW_CK(cudaEventElapsedTime(&ms, pev[k], pev[k + 1]));
      prof_stage_ms += ms;
      prof_stage_launches += 1;
    }
    pev_used = 0;
    return HWENO_OK;
  }

  hweno_status set_profiling(int enable) {
    prof = enable != 0;
    if (prof && pev.empty()) {
      pev.resize(2 * 3 * kGraphSteps);
      for (auto& e : pev) HW_CK(cudaEventCreate(&e));
    }
    prof_stage_ms = prof_total_ms = 0.0;
    prof_stage_launches = prof_launches = 0;
    pev_used = 0;
    return HWENO_OK;
  }

  hweno_status alpha_init() {
    if (dim == 1)
      HW_CK(hw::launch_alpha1d(prec, cfg.equation, S, cells, inst_d, tasks_d, ntasks, cfg.gamma_gas,
                               cfg.adv_x, ctl, num_sms, own));
    else if (batch2)
      for (int k = 0; k < n_inst; ++k)
        HW_CK(hw::launch_alpha2d(prec, cfg.equation, static_cast<const char*>(S) + offsets[k] * esz,
                                 offsets[k + 1] - offsets[k], cells, cfg.gamma_gas, cfg.adv_x, cfg.adv_y,
                                 ctl + k, num_sms, own));
    else
      HW_CK(hw::launch_alpha2d(prec, cfg.equation, S, cells, cells, cfg.gamma_gas, cfg.adv_x, cfg.adv_y, ctl,
                               num_sms, own));
    HW_CK(hw::launch_ctl_commit_alpha(ctl, n_inst, own));
    return HWENO_OK;
  }

  hweno_status set_state(const void* U, int on_device) {
    Range r("hweno.set_state");
    if (!U) return fail(HWENO_ERR_ARG, "state pointer is NULL");
    HW_TRY(enter());
    HW_CK(cudaStreamSynchronize(own));
    for (int k = 0; k < n_inst; ++k) {
      ctl_host[k] = ctl_init[k];
    }
    HW_CK(cudaMemcpyAsync(ctl, ctl_host, sizeof(hw::Ctl) * n_inst, cudaMemcpyHostToDevice, own));
    HW_CK(cudaMemcpyAsync(S, U, (size_t)cells * esz * nf,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, own));
    HW_TRY(alpha_init());
    has_state = true;
    return leave();
  }

  hweno_status get_state(void* U, int on_device) {
    Range r("hweno.get_state");
    if (!U) return fail(HWENO_ERR_ARG, "state pointer is NULL");
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    HW_TRY(enter());
    HW_CK(cudaMemcpyAsync(U, S, (size_t)cells * esz * nf,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, own));
    if (!on_device) HW_CK(cudaStreamSynchronize(own));
    return leave();
  }

  hweno_status read_ctl() {
    HW_CK(cudaMemcpyAsync(ctl_host, ctl, sizeof(hw::Ctl) * n_inst, cudaMemcpyDeviceToHost, own));
    HW_CK(cudaStreamSynchronize(own));
    return HWENO_OK;
  }

  hweno_status build_graph() {
    Range r("hweno.capture");
    if (gexec) return HWENO_OK;
    cudaGraph_t g = nullptr;
    HW_CK(cudaStreamBeginCapture(own, cudaStreamCaptureModeThreadLocal));
    hweno_status st = HWENO_OK;
    for (int s = 0; s < kGraphSteps && st == HWENO_OK; ++s) st = one_step();
    cudaError_t e = cudaStreamEndCapture(own, &g);
    if (st != HWENO_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return fail(HWENO_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(HWENO_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    return HWENO_OK;
  }

  hweno_status advance(const double* t_final, int max_steps) {
    Range r("hweno.advance");
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (max_steps < 0) return fail(HWENO_ERR_ARG, "max_steps must be >= 0");
    for (int k = 0; k < n_inst; ++k)
      if (!std::isfinite(t_final[k])) return fail(HWENO_ERR_ARG, "t_final must be finite");
    HW_TRY(enter());
    HW_TRY(read_ctl());
    for (int k = 0; k < n_inst; ++k) {
      hw::Ctl& C = ctl_host[k];
      if (C.err) return fail((hweno_status)C.err, "instance %d is in an error state", k);
      C.t_final = t_final[k];
      C.max_steps = max_steps;
      C.steps = 0;
      C.done = 0;
      C.last = 0;
    }
    HW_CK(cudaMemcpyAsync(ctl, ctl_host, sizeof(hw::Ctl) * n_inst, cudaMemcpyHostToDevice, own));
    if (!prof) HW_TRY(build_graph());
    long long remaining = max_steps;
    while (remaining > 0) {
      const int chunk = remaining >= kGraphSteps ? kGraphSteps : (int)remaining;
      if (chunk == kGraphSteps && !prof) {
        Range g("hweno.graph16");
        HW_CK(cudaGraphLaunch(gexec, own));
      } else {
        for (int s = 0; s < chunk; ++s) HW_TRY(one_step());
      }
      remaining -= chunk;
      prof_launches += 5LL * chunk;
      HW_TRY(read_ctl());
      if (prof) HW_TRY(collect_prof());
      bool all = true;
      for (int k = 0; k < n_inst; ++k) all = all && (ctl_host[k].done || ctl_host[k].steps >= max_steps);
      if (all) break;
    }
    HW_TRY(leave());
    for (int k = 0; k < n_inst; ++k)
      if (ctl_host[k].err)
        return fail((hweno_status)ctl_host[k].err, "non-physical state in instance %d at t=%.17g", k,
                    ctl_host[k].t);
    return HWENO_OK;
  }

  hweno_status manual_step(double dt, double ax, double ay) {
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (!(dt >= 0.0) || !std::isfinite(dt) || !(ax >= 0.0) || !(ay >= 0.0))
      return fail(HWENO_ERR_ARG, "dt and alpha must be finite and non-negative");
    HW_TRY(enter());
    HW_TRY(read_ctl());
    std::vector<double> t_now(n_inst);
    for (int k = 0; k < n_inst; ++k) t_now[k] = ctl_host[k].t;
    if (learned) HW_TRY(run_indicator());
    for (int k = 0; k < n_inst; ++k) {
      ctl_host[k] = ctl_init[k];
      ctl_host[k].t = t_now[k];
      ctl_host[k].dt = dt;
      ctl_host[k].ax = ax;
      ctl_host[k].ay = ay;
      ctl_host[k].dtf = (float)dt;
      ctl_host[k].axf = (float)ax;
      ctl_host[k].ayf = (float)ay;
      ctl_host[k].done = 0;
    }
    HW_CK(cudaMemcpyAsync(ctl_manual, ctl_host, sizeof(hw::Ctl) * n_inst, cudaMemcpyHostToDevice, own));
    HW_TRY(rk_stages(ctl_manual));
    HW_CK(cudaStreamSynchronize(own));
    // the solver's time moves by dt; the new state's alpha for the next advance
    HW_TRY(read_ctl());
    for (int k = 0; k < n_inst; ++k) ctl_host[k].t = t_now[k] + dt;
    HW_CK(cudaMemcpyAsync(ctl, ctl_host, sizeof(hw::Ctl) * n_inst, cudaMemcpyHostToDevice, own));
    HW_TRY(alpha_init());
    return leave();
  }

  // One RK stage of a step with given dt and alpha (hweno_stage): stage 1
  // reads S and writes A (and the limited derivatives H), stage 2 reads A and
  // writes B, stage 3 reads B and writes S and moves the time by dt.
  hweno_status stage_manual(int s, double dt, double ax, double ay) {
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (dim != 2 || batch2) return fail(HWENO_ERR_ARG, "hweno_stage serves single 2D solvers");
    if (s < 1 || s > 3) return fail(HWENO_ERR_ARG, "stage must be 1, 2 or 3");
    if (!(dt >= 0.0) || !std::isfinite(dt) || !(ax >= 0.0) || !(ay >= 0.0) || !std::isfinite(ax) ||
        !std::isfinite(ay))
      return fail(HWENO_ERR_ARG, "dt and alpha must be finite and non-negative");
    if (s != stage_done + 1) return fail(HWENO_ERR_STATE, "stage %d follows stage %d: stages run 1, 2, 3", s,
                                         stage_done);
    if (s > 1 && (dt != st_dt || ax != st_ax || ay != st_ay))
      return fail(HWENO_ERR_ARG, "the three stages of a step take the same dt and alpha");
    HW_TRY(enter());
    if (s == 1) {
      HW_TRY(read_ctl());
      st_t0 = ctl_host[0].t;
      st_dt = dt;
      st_ax = ax;
      st_ay = ay;
      if (learned) HW_TRY(run_indicator());
      hw::Ctl c = ctl_init[0];
      c.t = st_t0;
      c.dt = dt;
      c.ax = ax;
      c.ay = ay;
      c.dtf = (float)dt;
      c.axf = (float)ax;
      c.ayf = (float)ay;
      c.done = 0;
      ctl_host[0] = c;
      HW_CK(cudaMemcpyAsync(ctl_manual, ctl_host, sizeof(hw::Ctl), cudaMemcpyHostToDevice, own));
      HW_CK(cudaStreamSynchronize(own));
    }
    const void* in = s == 1 ? S : (s == 2 ? A : B);
    void* out = s == 1 ? A : (s == 2 ? B : S);
    HW_TRY(timed_stage(s, in, out, ctl_manual));
    stage_done = s == 3 ? 0 : s;
    if (s == 3) {
      // the solver's time moves by dt; alpha of the new state (hweno_alpha_update
      // again once rows of it have been replaced)
      HW_TRY(read_ctl());
      if (prof) HW_TRY(collect_prof());
      ctl_host[0].t = st_t0 + dt;
      HW_CK(cudaMemcpyAsync(ctl, ctl_host, sizeof(hw::Ctl), cudaMemcpyHostToDevice, own));
      HW_TRY(alpha_init());
    }
    return leave();
  }

  // Rows [row0, row0 + nrows) of every field plane of buffer `which` (0: the
  // state S, 1: stage-1 output A, 2: stage-2 output B) to or from a device
  // buffer laid out [nf][nrows][nx].
  hweno_status rows(int which, int row0, int nrows, void* buf, int to_solver) {
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (dim != 2 || batch2) return fail(HWENO_ERR_ARG, "hweno_rows serves single 2D solvers");
    if (which < 0 || which > 2) return fail(HWENO_ERR_ARG, "buffer must be 0 (state), 1 or 2 (stage outputs)");
    if (!buf) return fail(HWENO_ERR_ARG, "row buffer is NULL");
    if (row0 < 0 || nrows < 1 || row0 + nrows > cfg.ny)
      return fail(HWENO_ERR_ARG, "rows [%d, %d) lie outside [0, %d)", row0, row0 + nrows, cfg.ny);
    HW_TRY(enter());
    char* base = static_cast<char*>(which == 0 ? S : (which == 1 ? A : B));
    const size_t width = (size_t)nrows * cfg.nx * esz, plane = (size_t)cells * esz;
    char* p = base + (size_t)row0 * cfg.nx * esz;
    if (to_solver)
      HW_CK(cudaMemcpy2DAsync(p, plane, buf, width, width, nf, cudaMemcpyDeviceToDevice, own));
    else
      HW_CK(cudaMemcpy2DAsync(buf, width, p, plane, width, nf, cudaMemcpyDeviceToDevice, own));
    return leave();
  }

  hweno_status apply_operator(const double* ax, double ay, void* L, void* dh) {
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (!L || !dh) return fail(HWENO_ERR_ARG, "output pointer is NULL");
    HW_TRY(enter());
    if (dim == 1 || batch2) {
      HW_CK(cudaStreamSynchronize(own));
      HW_CK(cudaMemcpy(alpha_op, ax, sizeof(double) * n_inst * (batch2 ? 2 : 1), cudaMemcpyHostToDevice));
    }
    HW_TRY(stage(0, S, L, ctl, ax[0], ay, dh));
    return leave();
  }

  hweno_status load_indicator(const float* theta, int n, double p_threshold) {
    if (dim != 2 || batch2) return fail(HWENO_ERR_ARG, "the learned indicator serves single 2D solvers");
    if (!theta || n != hw::kMlpParams) return fail(HWENO_ERR_ARG, "expected %d network parameters", hw::kMlpParams);
    if (!(p_threshold > 0.0 && p_threshold < 1.0)) return fail(HWENO_ERR_ARG, "threshold must lie in (0, 1)");
    for (int k = 0; k < n; ++k)
      if (!std::isfinite(theta[k])) return fail(HWENO_ERR_ARG, "parameter %d is not finite", k);
    if (!mlp_w) {
      HW_CK(hw::prepare_mlp_infer2d());
      HW_CK(cudaMalloc(&mlp_w, sizeof(__half) * (32 * 80 + 32 * 32)));
      HW_CK(cudaMalloc(&mlp_bias, sizeof(float) * 97));
      HW_CK(cudaMalloc(&troubled, (size_t)cells));
      HW_CK(cudaMalloc(&smooth, (size_t)cells));
    }
    std::vector<__half> w(32 * 80 + 32 * 32);
    std::vector<float> b(97);
    for (int r = 0; r < 32; ++r)
      for (int c = 0; c < 80; ++c) w[r * 80 + c] = __float2half(c < 75 ? theta[r * 75 + c] : 0.0f);
    const int ob1 = 32 * 75, ow2 = ob1 + 32, ob2 = ow2 + 32 * 32, ow3 = ob2 + 32, ob3 = ow3 + 32;
    for (int k = 0; k < 32 * 32; ++k) w[32 * 80 + k] = __float2half(theta[ow2 + k]);
    for (int k = 0; k < 32; ++k) {
      b[k] = theta[ob1 + k];
      b[32 + k] = theta[ob2 + k];
      b[64 + k] = theta[ow3 + k];
    }
    b[96] = theta[ob3];
    HW_CK(cudaStreamSynchronize(own));
    HW_CK(cudaMemcpy(mlp_w, w.data(), sizeof(__half) * w.size(), cudaMemcpyHostToDevice));
    HW_CK(cudaMemcpy(mlp_bias, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice));
    z_thresh = (float)std::log(p_threshold / (1.0 - p_threshold));
    learned = true;
    drop_graph();
    return HWENO_OK;
  }

  // Time every candidate launch shape on the current state (operator mode,
  // reps launches each, CUDA events) and keep the fastest.
  hweno_status autotune(int reps, double* best_ms) {
    Range r("hweno.autotune");
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (reps < 1 || reps > 1000) return fail(HWENO_ERR_ARG, "reps must lie in [1, 1000]");
    HW_TRY(enter());
    std::vector<hw::LaunchShape> cand;
    if (dim == 1) {
      for (int wpb : {2, 4, 8})
        for (int bps : {4, 8, 16, 32}) {
          hw::LaunchShape s;
          s.warps1d = wpb;
          s.blocks_per_sm1d = bps;
          cand.push_back(s);
        }
    } else {
      for (int p : {1, 0}) {
        hw::LaunchShape s;
        s.persistent2d = p;
        cand.push_back(s);
      }
    }
    ScopedDev L, D;
    HW_CK(cudaMalloc(&L.p, (size_t)cells * esz * nf));
    HW_CK(cudaMalloc(&D.p, (size_t)cells * esz * nd));
    ScopedEvent e0, e1;
    HW_CK(cudaEventCreate(&e0.e));
    HW_CK(cudaEventCreate(&e1.e));
    std::vector<double> a0(2 * n_inst, 1.0);
    if (dim == 1 || batch2) HW_CK(cudaMemcpy(alpha_op, a0.data(), sizeof(double) * a0.size(), cudaMemcpyHostToDevice));
    const hw::LaunchShape keep = shape;
    double best = 1e300;
    hw::LaunchShape pick = keep;
    hweno_status st = HWENO_OK;
    for (const hw::LaunchShape& c : cand) {
      shape = c;
      st = stage(0, S, L.p, ctl, 1.0, 1.0, D.p);  // warm-up
      if (st != HWENO_OK) break;
      cudaEventRecord(e0.e, own);
      for (int r = 0; r < reps && st == HWENO_OK; ++r) st = stage(0, S, L.p, ctl, 1.0, 1.0, D.p);
      cudaEventRecord(e1.e, own);
      if (st != HWENO_OK) break;
      cudaEventSynchronize(e1.e);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0.e, e1.e);
      if (ms < best) { best = ms; pick = c; }
    }
    shape = st == HWENO_OK ? pick : keep;
    if (st != HWENO_OK) return st;
    if (best_ms) *best_ms = best / reps;
    drop_graph();
    return leave();
  }

  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
};

struct hweno_solver { Engine e; };

namespace {

// Gauss-Legendre nodes and weights on [-1/2, 1/2] (weights sum to 1): roots
// of P_n by Newton's method from the Chebyshev-like initial guesses, weights
// 1 / ((1 - x^2) P_n'(x)^2) on [-1, 1], halved.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * z;
    w[i] = 0.5 * 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace
struct hweno_batch { Engine e; };

extern "C" {

const char* hweno_last_error(void) { return g_err.c_str(); }
const char* hweno_version(void) { return "libhweno 0.1 (sm_103a)"; }

hweno_status hweno_create(const hweno_config* cfg, void* cuda_stream, hweno_solver** out) {
  if (!out) return fail(HWENO_ERR_ARG, "out is NULL");
  *out = nullptr;
  HW_TRY(validate(cfg, 0));
  hweno_solver* s = new (std::nothrow) hweno_solver();
  if (!s) return fail(HWENO_ERR_OOM, "host allocation failed");
  hweno_status st = s->e.init(1, cfg, cuda_stream);
  if (st != HWENO_OK) {
    delete s;
    return st;
  }
  *out = s;
  return HWENO_OK;
}

void hweno_destroy(hweno_solver* s) { delete s; }
void* hweno_stream(hweno_solver* s) { return s ? (void*)s->e.own : nullptr; }

hweno_status hweno_shape(const hweno_solver* s, int* nfields, size_t* ncells) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (nfields) *nfields = s->e.nf;
  if (ncells) *ncells = (size_t)s->e.cells;
  return HWENO_OK;
}

hweno_status hweno_set_state(hweno_solver* s, const void* U, int on_device) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.set_state(U, on_device);
}

hweno_status hweno_get_state(hweno_solver* s, void* U, int on_device) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.get_state(U, on_device);
}

hweno_status hweno_alpha(hweno_solver* s, double* alpha_x, double* alpha_y) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (!s->e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(s->e.enter());
  HW_TRY(s->e.read_ctl());
  if (alpha_x) *alpha_x = s->e.ctl_host[0].ax;
  if (alpha_y) *alpha_y = s->e.ctl_host[0].ay;
  if (s->e.ctl_host[0].err) return fail(HWENO_ERR_NONPHYSICAL, "non-physical state");
  return s->e.leave();
}

hweno_status hweno_apply_operator(hweno_solver* s, double alpha_x, double alpha_y, void* L_out,
                                  void* dhat_out) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (!(alpha_x >= 0.0) || !(alpha_y >= 0.0)) return fail(HWENO_ERR_ARG, "alpha must be >= 0");
  return s->e.apply_operator(&alpha_x, alpha_y, L_out, dhat_out);
}

hweno_status hweno_step(hweno_solver* s, double dt, double alpha_x, double alpha_y) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.manual_step(dt, alpha_x, alpha_y);
}

hweno_status hweno_stage(hweno_solver* s, int stage, double dt, double alpha_x, double alpha_y) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.stage_manual(stage, dt, alpha_x, alpha_y);
}

hweno_status hweno_rows(hweno_solver* s, int buffer, int row0, int nrows, void* rows, int to_solver) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.rows(buffer, row0, nrows, rows, to_solver);
}

hweno_status hweno_alpha_update(hweno_solver* s, double* alpha_x, double* alpha_y) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (!s->e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(s->e.enter());
  HW_TRY(s->e.alpha_init());
  HW_TRY(s->e.leave());
  return hweno_alpha(s, alpha_x, alpha_y);
}

hweno_status hweno_advance(hweno_solver* s, double t_final, int max_steps, double* t_out,
                           int* steps_out) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  hweno_status st = s->e.advance(&t_final, max_steps);
  if (t_out) *t_out = s->e.ctl_host[0].t;
  if (steps_out) *steps_out = s->e.ctl_host[0].steps;
  return st;
}

hweno_status hweno_set_profiling(hweno_solver* s, int enable) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.set_profiling(enable);
}

hweno_status hweno_profile(hweno_solver* s, double* stage_ms, long long* stage_launches,
                           long long* kernel_launches) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (stage_ms) *stage_ms = s->e.prof_stage_ms;
  if (stage_launches) *stage_launches = s->e.prof_stage_launches;
  if (kernel_launches) *kernel_launches = s->e.prof_launches;
  return HWENO_OK;
}

hweno_status hweno_batch_create(int n, const hweno_config* cfgs, void* cuda_stream, hweno_batch** out) {
  if (!out) return fail(HWENO_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !cfgs) return fail(HWENO_ERR_ARG, "need at least one config");
  for (int k = 0; k < n; ++k) {
    HW_TRY(validate(&cfgs[k], cfgs[0].dim));
    const hweno_config &a = cfgs[0], &b = cfgs[k];
    bool same = a.equation == b.equation && a.precision == b.precision && a.charwise == b.charwise &&
                a.linear_weights == b.linear_weights && a.weight_pow == b.weight_pow && a.eps == b.eps &&
                a.smoothness == b.smoothness &&
                a.gamma_gas == b.gamma_gas && a.adv_x == b.adv_x && (a.dim == 1 || a.adv_y == b.adv_y);
    for (int m = 0; m < (a.dim == 1 ? 3 : 5); ++m) same = same && a.lin_w[m] == b.lin_w[m];
    if (!same) return fail(HWENO_ERR_ARG, "config %d differs from config 0 in a batch-wide parameter", k);
  }
  hweno_batch* b = new (std::nothrow) hweno_batch();
  if (!b) return fail(HWENO_ERR_OOM, "host allocation failed");
  hweno_status st = b->e.init(n, cfgs, cuda_stream, true);
  if (st != HWENO_OK) {
    delete b;
    return st;
  }
  *out = b;
  return HWENO_OK;
}

void hweno_batch_destroy(hweno_batch* b) { delete b; }
void* hweno_batch_stream(hweno_batch* b) { return b ? (void*)b->e.own : nullptr; }

hweno_status hweno_batch_layout(const hweno_batch* b, size_t* total_cells, size_t* offsets) {
  if (!b) return fail(HWENO_ERR_ARG, "batch is NULL");
  if (total_cells) *total_cells = (size_t)b->e.cells;
  if (offsets)
    for (int k = 0; k <= b->e.n_inst; ++k) offsets[k] = (size_t)b->e.offsets[k];
  return HWENO_OK;
}

hweno_status hweno_batch_set_state(hweno_batch* b, const void* U, int on_device) {
  if (!b) return fail(HWENO_ERR_ARG, "batch is NULL");
  return b->e.set_state(U, on_device);
}

hweno_status hweno_batch_get_state(hweno_batch* b, void* U, int on_device) {
  if (!b) return fail(HWENO_ERR_ARG, "batch is NULL");
  return b->e.get_state(U, on_device);
}

hweno_status hweno_batch_advance(hweno_batch* b, const double* t_final, int max_steps, double* t_out,
                                 int* steps_out) {
  if (!b || !t_final) return fail(HWENO_ERR_ARG, "batch or t_final is NULL");
  hweno_status st = b->e.advance(t_final, max_steps);
  for (int k = 0; k < b->e.n_inst; ++k) {
    if (t_out) t_out[k] = b->e.ctl_host[k].t;
    if (steps_out) steps_out[k] = b->e.ctl_host[k].steps;
  }
  return st;
}

hweno_status hweno_batch_set_profiling(hweno_batch* b, int enable) {
  if (!b) return fail(HWENO_ERR_ARG, "batch is NULL");
  return b->e.set_profiling(enable);
}

hweno_status hweno_batch_profile(hweno_batch* b, double* stage_ms, long long* stage_launches,
                                 long long* kernel_launches) {
  if (!b) return fail(HWENO_ERR_ARG, "batch is NULL");
  if (stage_ms) *stage_ms = b->e.prof_stage_ms;
  if (stage_launches) *stage_launches = b->e.prof_stage_launches;
  if (kernel_launches) *kernel_launches = b->e.prof_launches;
  return HWENO_OK;
}

hweno_status hweno_batch_apply_operator(hweno_batch* b, const double* alpha, void* L_out,
                                        void* dhat_out) {
  if (!b || !alpha) return fail(HWENO_ERR_ARG, "batch or alpha is NULL");
  for (int k = 0; k < b->e.n_inst * b->e.dim; ++k)
    if (!(alpha[k] >= 0.0)) return fail(HWENO_ERR_ARG, "alpha must be >= 0");
  return b->e.apply_operator(alpha, 0.0, L_out, dhat_out);
}

}  // extern "C"

// ---- learned troubled-cell indicator ----
struct hweno_mlp {
  cudaStream_t stream = nullptr;
  int max_batch = 0;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  hw::MlpWork w{};
  int t = 0;
  ~hweno_mlp() {
    cudaFree(theta); cudaFree(m); cudaFree(v); cudaFree(grad);
    cudaFree(w.h1); cudaFree(w.dh1); cudaFree(w.h2); cudaFree(w.dh2); cudaFree(w.dz); cudaFree(w.loss);
    cudaFree(w.loss_acc);
  }
};

extern "C" {

hweno_status hweno_indicator_load(hweno_solver* s, const float* theta, int nparams, double p_threshold) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  return s->e.load_indicator(theta, nparams, p_threshold);
}

hweno_status hweno_indicator_off(hweno_solver* s) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  s->e.learned = false;
  s->e.drop_graph();
  return HWENO_OK;
}

hweno_status hweno_indicator_mask(hweno_solver* s, void* smooth_out, void* troubled_out) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  Engine& e = s->e;
  if (!e.learned) return fail(HWENO_ERR_STATE, "no indicator loaded");
  if (!e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(e.enter());
  HW_TRY(e.run_indicator());
  if (smooth_out) HW_CK(cudaMemcpyAsync(smooth_out, e.smooth, (size_t)e.cells, cudaMemcpyDeviceToDevice, e.own));
  if (troubled_out)
    HW_CK(cudaMemcpyAsync(troubled_out, e.troubled, (size_t)e.cells, cudaMemcpyDeviceToDevice, e.own));
  return e.leave();
}

hweno_status hweno_indicator_features(hweno_solver* s, float* feat_out) {
  if (!s || !feat_out) return fail(HWENO_ERR_ARG, "solver or output is NULL");
  Engine& e = s->e;
  if (e.dim != 2) return fail(HWENO_ERR_ARG, "the learned indicator serves 2D solvers");
  if (!e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(e.enter());
  HW_CK(hw::launch_features2d(e.prec, e.cfg.equation, e.S, e.grid, e.cells, e.ctl, feat_out, e.num_sms, e.own));
  return e.leave();
}

hweno_status hweno_indicator_labels(hweno_solver* s, float* dev_out) {
  if (!s || !dev_out) return fail(HWENO_ERR_ARG, "solver or output is NULL");
  Engine& e = s->e;
  if (e.dim != 2) return fail(HWENO_ERR_ARG, "the learned indicator serves 2D solvers");
  if (!e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(e.enter());
  HW_CK(hw::launch_labels2d(e.prec, e.cfg.equation, e.cfg.charwise, e.S, e.grid, e.cells, e.wp, e.cfg.gamma_gas,
                            e.ctl, dev_out, e.num_sms, e.own));
  return e.leave();
}

hweno_status hweno_mlp_create(int max_batch, void* cuda_stream, hweno_mlp** out) {
  if (!out) return fail(HWENO_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (max_batch < 1 || max_batch > (1 << 24)) return fail(HWENO_ERR_ARG, "max_batch must be in [1, 2^24]");
  hweno_mlp* m = new (std::nothrow) hweno_mlp();
  if (!m) return fail(HWENO_ERR_OOM, "host allocation failed");
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  m->max_batch = max_batch;
  const size_t P = sizeof(float) * hw::kMlpParams, H = sizeof(float) * 32 * (size_t)max_batch;
  cudaError_t e = cudaSuccess;
  float** bufs[] = {&m->theta, &m->m, &m->v, &m->grad};
  for (float** b : bufs) if (e == cudaSuccess) e = cudaMalloc(b, P);
  float** hb[] = {&m->w.h1, &m->w.dh1, &m->w.h2, &m->w.dh2};
  for (float** b : hb) if (e == cudaSuccess) e = cudaMalloc(b, H);
  if (e == cudaSuccess) e = cudaMalloc(&m->w.dz, sizeof(float) * max_batch);
  if (e == cudaSuccess) e = cudaMalloc(&m->w.loss, sizeof(float) * max_batch);
  if (e == cudaSuccess) e = cudaMalloc(&m->w.loss_acc, sizeof(float) * 2);
  if (e == cudaSuccess) e = cudaMemset(m->w.loss_acc, 0, sizeof(float) * 2);
  if (e != cudaSuccess) {
    delete m;
    return fail(e == cudaErrorMemoryAllocation ? HWENO_ERR_OOM : HWENO_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  *out = m;
  return HWENO_OK;
}

void hweno_mlp_destroy(hweno_mlp* m) { delete m; }

hweno_status hweno_mlp_set_params(hweno_mlp* m, const float* theta) {
  if (!m || !theta) return fail(HWENO_ERR_ARG, "mlp or parameters NULL");
  HW_CK(cudaStreamSynchronize(m->stream));
  HW_CK(cudaMemcpy(m->theta, theta, sizeof(float) * hw::kMlpParams, cudaMemcpyHostToDevice));
  HW_CK(cudaMemset(m->m, 0, sizeof(float) * hw::kMlpParams));
  HW_CK(cudaMemset(m->v, 0, sizeof(float) * hw::kMlpParams));
  HW_CK(cudaMemset(m->w.loss_acc, 0, sizeof(float) * 2));
  m->t = 0;
  return HWENO_OK;
}

hweno_status hweno_mlp_get_params(hweno_mlp* m, float* theta) {
  if (!m || !theta) return fail(HWENO_ERR_ARG, "mlp or output NULL");
  HW_CK(cudaStreamSynchronize(m->stream));
  HW_CK(cudaMemcpy(theta, m->theta, sizeof(float) * hw::kMlpParams, cudaMemcpyDeviceToHost));
  return HWENO_OK;
}

static hweno_status mlp_check(hweno_mlp* m, const float* feat, const float* dev, const int* idx, int B) {
  if (!m || !feat || !dev || !idx) return fail(HWENO_ERR_ARG, "NULL argument");
  if (B < 1 || B > m->max_batch) return fail(HWENO_ERR_ARG, "batch size %d outside [1, %d]", B, m->max_batch);
  return HWENO_OK;
}

hweno_status hweno_mlp_gradient(hweno_mlp* m, const float* feat, const float* dev, const int* idx, int B,
                                double delta, double pos_weight, float* grad_out, double* loss_out) {
  HW_TRY(mlp_check(m, feat, dev, idx, B));
  if (!grad_out) return fail(HWENO_ERR_ARG, "grad_out is NULL");
  HW_CK(cudaMemsetAsync(m->w.loss_acc, 0, sizeof(float) * 2, m->stream));
  HW_CK(hw::launch_mlp_train(m->theta, feat, dev, idx, B, (float)delta, (float)pos_weight, m->w, m->grad, m->stream));
  float acc[2];
  HW_CK(cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * hw::kMlpParams, cudaMemcpyDeviceToHost, m->stream));
  HW_CK(cudaMemcpyAsync(acc, m->w.loss_acc, sizeof acc, cudaMemcpyDeviceToHost, m->stream));
  HW_CK(cudaStreamSynchronize(m->stream));
  if (loss_out) *loss_out = acc[0];
  return HWENO_OK;
}

hweno_status hweno_mlp_train_step(hweno_mlp* m, const float* feat, const float* dev, const int* idx, int B,
                                  double delta, double pos_weight, double lr) {
  HW_TRY(mlp_check(m, feat, dev, idx, B));
  if (!(lr > 0.0)) return fail(HWENO_ERR_ARG, "learning rate must be positive");
  HW_CK(hw::launch_mlp_train(m->theta, feat, dev, idx, B, (float)delta, (float)pos_weight, m->w, m->grad, m->stream));
  m->t += 1;
  HW_CK(hw::launch_mlp_adam(m->theta, m->m, m->v, m->grad, (float)lr, m->t, m->stream));
  return HWENO_OK;
}

hweno_status hweno_mlp_mean_loss(hweno_mlp* m, double* loss) {
  if (!m || !loss) return fail(HWENO_ERR_ARG, "NULL argument");
  float acc[2];
  HW_CK(cudaMemcpyAsync(acc, m->w.loss_acc, sizeof acc, cudaMemcpyDeviceToHost, m->stream));
  HW_CK(cudaMemsetAsync(m->w.loss_acc, 0, sizeof(float) * 2, m->stream));
  HW_CK(cudaStreamSynchronize(m->stream));
  *loss = acc[1] > 0.f ? acc[0] / acc[1] : 0.0;
  return HWENO_OK;
}

// SplitMix64 (Steele, Lea and Flood, 2014): the generator of the training
// permutations and of the default initialisation.
static unsigned long long splitmix64(unsigned long long& state) {
  state += 0x9E3779B97F4A7C15ull;
  unsigned long long z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void hweno_train_permutation(unsigned long long seed, int epoch, long long n, int* perm) {
  if (!perm || n < 1) return;
  unsigned long long st = seed + (unsigned long long)(epoch + 1) * 0xD1B54A32D192ED03ull;
  for (long long i = 0; i < n; ++i) perm[i] = (int)i;
  for (long long i = n - 1; i > 0; --i) {
    const long long j = (long long)(splitmix64(st) % (unsigned long long)(i + 1));
    const int t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

hweno_status hweno_indicator_train(const float* feat, const float* dev, long long n, const hweno_train_opts* o,
                                   const float* init_params, float* params_out, double* losses_out,
                                   void* cuda_stream) {
  if (!feat || !dev || !o || !params_out) return fail(HWENO_ERR_ARG, "NULL argument");
  if (n < 1 || n > INT32_MAX) return fail(HWENO_ERR_ARG, "n must lie in [1, 2^31)");
  if (o->epochs < 1 || o->batch < 1 || o->batch > n || o->batch > (1 << 24))
    return fail(HWENO_ERR_ARG, "need epochs >= 1 and 1 <= batch <= min(n, 2^24)");
  if (!(o->lr > 0.0) || !std::isfinite(o->lr) || !std::isfinite(o->delta))
    return fail(HWENO_ERR_ARG, "lr must be positive and delta finite");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int devno = 0, sms = 148;
  HW_CK(cudaGetDevice(&devno));
  HW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devno));
  // class weight of the positives
  double pw = o->pos_weight;
  unsigned long long* cnt = nullptr;
  int* perm_d = nullptr;
  hweno_mlp* m = nullptr;
  hweno_status rc = HWENO_OK;
  std::vector<int> perm((size_t)n);
  std::vector<float> theta(hw::kMlpParams);
  {
    cudaError_t e = cudaMalloc(&cnt, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&perm_d, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = hw::launch_count_above(dev, n, (float)o->delta, cnt, sms, st);
    unsigned long long pos = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&pos, cnt, sizeof pos, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = fail(e == cudaErrorMemoryAllocation ? HWENO_ERR_OOM : HWENO_ERR_CUDA, "%s", cudaGetErrorString(e));
      goto done;
    }
    if (!(pw > 0.0)) {
      const double frac = (double)pos / (double)n;
      pw = std::min(50.0, std::max(1.0, (1.0 - frac) / std::max(frac, 1e-6)));
    }
  }
  if (init_params) {
    std::copy(init_params, init_params + hw::kMlpParams, theta.begin());
  } else {
    // He-normal hidden layers, N(0, 1/32) output layer, zero biases; normal
    // deviates by the Box-Muller transform of SplitMix64 uniforms
    unsigned long long stt = o->seed;
    auto normal = [&stt]() {
      const double u1 = ((splitmix64(stt) >> 11) + 1.0) * 0x1p-53, u2 = (splitmix64(stt) >> 11) * 0x1p-53;
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    std::fill(theta.begin(), theta.end(), 0.0f);
    for (int k = 0; k < 32 * 75; ++k) theta[k] = (float)(normal() * std::sqrt(2.0 / 75.0));
    const int ow2 = 32 * 75 + 32, ow3 = ow2 + 32 * 32 + 32;
    for (int k = 0; k < 32 * 32; ++k) theta[ow2 + k] = (float)(normal() * std::sqrt(2.0 / 32.0));
    for (int k = 0; k < 32; ++k) theta[ow3 + k] = (float)(normal() * std::sqrt(1.0 / 32.0));
  }
  rc = hweno_mlp_create(o->batch, cuda_stream, &m);
  if (rc != HWENO_OK) goto done;
  rc = hweno_mlp_set_params(m, theta.data());
  if (rc != HWENO_OK) goto done;
  for (int ep = 0; ep < o->epochs; ++ep) {
    hweno_train_permutation(o->seed, ep, n, perm.data());
    cudaError_t e = cudaMemcpyAsync(perm_d, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { rc = fail(HWENO_ERR_CUDA, "%s", cudaGetErrorString(e)); goto done; }
    for (long long b0 = 0; b0 + o->batch <= n; b0 += o->batch) {
      rc = hweno_mlp_train_step(m, feat, dev, perm_d + b0, o->batch, o->delta, pw, o->lr);
      if (rc != HWENO_OK) goto done;
    }
    double loss = 0.0;
    rc = hweno_mlp_mean_loss(m, &loss);
    if (rc != HWENO_OK) goto done;
    if (losses_out) losses_out[ep] = loss;
  }
  rc = hweno_mlp_get_params(m, params_out);
done:
  if (m) hweno_mlp_destroy(m);
  cudaFree(cnt);
  cudaFree(perm_d);
  return rc;
}

hweno_status hweno_mlp_predict(hweno_mlp* m, const float* feat, long long n, float* prob) {
  if (!m || !feat || !prob || n < 1) return fail(HWENO_ERR_ARG, "bad argument");
  int dev = 0, sms = 148;
  HW_CK(cudaGetDevice(&dev));
  HW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HW_CK(hw::launch_mlp_predict(m->theta, feat, n, prob, sms, m->stream));
  return HWENO_OK;
}

}  // extern "C"

extern "C" hweno_status hweno_get_time(hweno_solver* s, double* t, int* steps) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (!s->e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(s->e.enter());
  HW_TRY(s->e.read_ctl());
  if (t) *t = s->e.ctl_host[0].t;
  if (steps) *steps = s->e.ctl_host[0].steps;
  return s->e.leave();
}

extern "C" hweno_status hweno_set_time(hweno_solver* s, double t) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  if (!std::isfinite(t) || t < 0.0) return fail(HWENO_ERR_ARG, "t must be finite and non-negative");
  Engine& e = s->e;
  if (!e.has_state) return fail(HWENO_ERR_STATE, "no state set");
  HW_TRY(e.enter());
  HW_TRY(e.read_ctl());
  e.ctl_host[0].t = t;
  HW_CK(cudaMemcpyAsync(e.ctl, e.ctl_host, sizeof(hw::Ctl), cudaMemcpyHostToDevice, e.own));
  HW_CK(cudaStreamSynchronize(e.own));
  return e.leave();
}

extern "C" hweno_status hweno_autotune(hweno_solver* s, int reps, double* best_ms, int* shape_out) {
  if (!s) return fail(HWENO_ERR_ARG, "solver is NULL");
  HW_TRY(s->e.autotune(reps, best_ms));
  if (shape_out) {
    shape_out[0] = s->e.shape.warps1d;
    shape_out[1] = s->e.shape.blocks_per_sm1d;
    shape_out[2] = s->e.shape.persistent2d;
  }
  return HWENO_OK;
}

extern "C" hweno_status hweno_batch_autotune(hweno_batch* b, int reps, double* best_ms, int* shape_out) {
  if (!b) return fail(HWENO_ERR_ARG, "batch is NULL");
  HW_TRY(b->e.autotune(reps, best_ms));
  if (shape_out) {
    shape_out[0] = b->e.shape.warps1d;
    shape_out[1] = b->e.shape.blocks_per_sm1d;
    shape_out[2] = b->e.shape.persistent2d;
  }
  return HWENO_OK;
}

extern "C" hweno_status hweno_project(hweno_solver* s, hweno_u0_fn u0, void* ctx, int nq) {
  if (!s || !u0) return fail(HWENO_ERR_ARG, "solver or u0 is NULL");
  if (nq < 1 || nq > 16) return fail(HWENO_ERR_ARG, "nq must lie in [1, 16]");
  Engine& e = s->e;
  if (e.n_inst != 1) return fail(HWENO_ERR_ARG, "projection serves single-grid solvers");
  const hweno_config& c = e.cfg;
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  const int nc = e.nc, nx = c.nx, ny = c.dim == 2 ? c.ny : 1;
  const double dx = (c.xhi - c.xlo) / nx, dy = c.dim == 2 ? (c.yhi - c.ylo) / ny : 1.0;
  const size_t cells = (size_t)nx * ny;
  std::vector<double> U((size_t)e.nf * cells, 0.0);
  // one callback per row: every quadrature / face point of the row at once
  const int per_cell = c.dim == 2 ? nq * nq + 4 * nq : nq + 2;
  std::vector<double> X((size_t)nx * per_cell), Y((size_t)nx * per_cell), V((size_t)nx * per_cell * nc);
  for (int j = 0; j < ny; ++j) {
    const double yc = c.dim == 2 ? c.ylo + (j + 0.5) * dy : 0.0;
    size_t p = 0;
    for (int i = 0; i < nx; ++i) {
      const double xc = c.xlo + (i + 0.5) * dx;
      if (c.dim == 1) {
        for (int a = 0; a < nq; ++a) { X[p] = xc + dx * gx[a]; Y[p++] = 0.0; }
        X[p] = xc - 0.5 * dx; Y[p++] = 0.0;
        X[p] = xc + 0.5 * dx; Y[p++] = 0.0;
      } else {
        for (int b = 0; b < nq; ++b)
          for (int a = 0; a < nq; ++a) { X[p] = xc + dx * gx[a]; Y[p++] = yc + dy * gx[b]; }
        for (int b = 0; b < nq; ++b) { X[p] = xc - 0.5 * dx; Y[p++] = yc + dy * gx[b]; }
        for (int b = 0; b < nq; ++b) { X[p] = xc + 0.5 * dx; Y[p++] = yc + dy * gx[b]; }
        for (int a = 0; a < nq; ++a) { X[p] = xc + dx * gx[a]; Y[p++] = yc - 0.5 * dy; }
        for (int a = 0; a < nq; ++a) { X[p] = xc + dx * gx[a]; Y[p++] = yc + 0.5 * dy; }
      }
    }
    u0((int)p, X.data(), Y.data(), V.data(), ctx);
    for (size_t q = 0; q < p * nc; ++q)
      if (!std::isfinite(V[q])) return fail(HWENO_ERR_ARG, "u0 returned a non-finite value");
    for (int i = 0; i < nx; ++i) {
      const double* v = V.data() + (size_t)i * per_cell * nc;
      const size_t cell = (size_t)j * nx + i;
      for (int k = 0; k < nc; ++k) {
        double avg = 0.0, vb = 0.0, wb = 0.0;
        if (c.dim == 1) {
          for (int a = 0; a < nq; ++a) avg += gw[a] * v[a * nc + k];
          vb = (v[(nq + 1) * nc + k] - v[nq * nc + k]) / dx;  // mean of u_x over the cell
        } else {
          for (int b = 0; b < nq; ++b)
            for (int a = 0; a < nq; ++a) avg += gw[a] * gw[b] * v[(b * nq + a) * nc + k];
          const int o = nq * nq;
          for (int b = 0; b < nq; ++b) vb += gw[b] * (v[(o + nq + b) * nc + k] - v[(o + b) * nc + k]);
          for (int a = 0; a < nq; ++a) wb += gw[a] * (v[(o + 3 * nq + a) * nc + k] - v[(o + 2 * nq + a) * nc + k]);
        }
        U[(size_t)k * cells + cell] = avg;
        U[(size_t)(nc + k) * cells + cell] = vb;
        if (c.dim == 2) U[(size_t)(2 * nc + k) * cells + cell] = wb;
      }
    }
  }
  if (e.prec == HWENO_FP64) return e.set_state(U.data(), 0);
  std::vector<float> Uf(U.begin(), U.end());
  return e.set_state(Uf.data(), 0);
}
