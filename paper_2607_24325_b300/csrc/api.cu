// api.cu -- C ABI of libhweno (declared in include/hweno.h).
//
// Host logic only: argument validation, workspace allocation, ordering
// against the caller's stream, the device-resident time-step control and the
// CUDA graph that replays whole SSP-RK3 steps (ctl_begin, stage 1, stage 2,
// stage 3, ctl_end).  All arithmetic of the scheme runs in the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

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

hweno_status validate(const hweno_config* c, int expect_dim) {
  if (!c) return fail(HWENO_ERR_ARG, "config is NULL");
  if (c->dim != 1 && c->dim != 2) return fail(HWENO_ERR_ARG, "dim must be 1 or 2 (got %d)", c->dim);
  if (expect_dim && c->dim != expect_dim) return fail(HWENO_ERR_ARG, "batches hold 1D problems only");
  if (c->nx < 3 || (c->dim == 2 && c->ny < 3))
    return fail(HWENO_ERR_ARG, "need at least 3 cells per direction (nx=%d ny=%d)", c->nx, c->ny);
  if ((long long)c->nx * (c->dim == 2 ? c->ny : 1) > (1LL << 31))
    return fail(HWENO_ERR_ARG, "grid too large (more than 2^31 cells)");
  if (!(c->xhi > c->xlo) || (c->dim == 2 && !(c->yhi > c->ylo)))
    return fail(HWENO_ERR_ARG, "empty domain");
  if (c->equation < 0 || c->equation > 2) return fail(HWENO_ERR_ARG, "unknown equation %d", c->equation);
  if (c->equation == HWENO_EQ_EULER && !(c->gamma_gas > 1.0))
    return fail(HWENO_ERR_ARG, "gamma_gas must exceed 1");
  const int nw = c->dim == 1 ? 3 : 5;
  double s = 0.0;
  for (int m = 0; m < nw; ++m) {
    if (!(c->lin_w[m] > 0.0)) return fail(HWENO_ERR_ARG, "linear weight %d must be positive", m);
    s += c->lin_w[m];
  }
  if (std::fabs(s - 1.0) > 1e-12) return fail(HWENO_ERR_ARG, "linear weights must sum to 1 (sum %.17g)", s);
  if (!(c->eps > 0.0)) return fail(HWENO_ERR_ARG, "eps must be positive");
  if (c->weight_pow != 1 && c->weight_pow != 2) return fail(HWENO_ERR_ARG, "weight_pow must be 1 or 2");
  if (!(c->cfl > 0.0)) return fail(HWENO_ERR_ARG, "cfl must be positive");
  if (c->dt_rule != HWENO_DT_CFL && c->dt_rule != HWENO_DT_CFL_DX53) return fail(HWENO_ERR_ARG, "bad dt_rule");
  if (c->precision != HWENO_FP64 && c->precision != HWENO_FP32) return fail(HWENO_ERR_ARG, "bad precision");
  const int nsides = c->dim == 1 ? 2 : 4;
  for (int k = 0; k < nsides; ++k)
    if (c->bc[k] < 0 || c->bc[k] > 3) return fail(HWENO_ERR_ARG, "bad boundary condition on side %d", k);
  for (int a = 0; a < c->dim; ++a)
    if ((c->bc[2 * a] == HWENO_BC_PERIODIC) != (c->bc[2 * a + 1] == HWENO_BC_PERIODIC))
      return fail(HWENO_ERR_ARG, "periodic boundaries must be paired (axis %d)", a);
  return HWENO_OK;
}

}  // namespace

namespace hw {
// Error reporting and config validation for entry points defined in other
// translation units (the allocation-free step).
hweno_status report_error(hweno_status st, const char* msg) { return fail(st, "%s", msg); }
hweno_status check_config(const hweno_config* cfg, int expect_dim) { return validate(cfg, expect_dim); }
}  // namespace hw

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
  double* alpha_op = nullptr;    // device [n_inst]
  hw::Grid2 grid{};
  hw::WeightParams wp{};
  cudaGraphExec_t gexec = nullptr;
  bool has_state = false;
  // opt-in timing of every stage launch with CUDA events (direct launches)
  bool prof = false;
  std::vector<cudaEvent_t> pev;   // 2 per stage launch of one poll window
  int pev_used = 0;
  double prof_stage_ms = 0.0, prof_total_ms = 0.0;
  long long prof_stage_launches = 0, prof_launches = 0;

  ~Engine() {
    for (cudaEvent_t e : pev) cudaEventDestroy(e);
    if (gexec) cudaGraphExecDestroy(gexec);
    cudaFree(S); cudaFree(A); cudaFree(B); cudaFree(H);
    cudaFree(ctl); cudaFree(ctl_manual); cudaFree(inst_d); cudaFree(tasks_d); cudaFree(alpha_op);
    if (ctl_host) cudaFreeHost(ctl_host);
    if (ev) cudaEventDestroy(ev);
    if (own) cudaStreamDestroy(own);
  }

  hweno_status init(int n, const hweno_config* cfgs, void* stream) {
    cfg = cfgs[0];
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
    for (int m = 0; m < 5; ++m) wp.g[m] = cfg.lin_w[m];
    wp.eps = cfg.eps;
    wp.pow2 = cfg.weight_pow == 2;
    wp.linear = cfg.linear_weights != 0;

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
        I.dx = (c.xhi - c.xlo) / c.nx;
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
    } else {
      grid.nx = cfg.nx;
      grid.ny = cfg.ny;
      for (int q = 0; q < 4; ++q) {
        grid.bc[q] = cfg.bc[q];
        for (int r = 0; r < 4; ++r) grid.st[q][r] = cfg.bc_state[q][r];
      }
      grid.dx = (cfg.xhi - cfg.xlo) / cfg.nx;
      grid.dy = (cfg.yhi - cfg.ylo) / cfg.ny;
      cells = (long long)cfg.nx * cfg.ny;
      offsets = {0, cells};
      hw::Ctl& C = ctl_init[0];
      std::memset(&C, 0, sizeof C);
      const bool r53 = cfg.dt_rule == HWENO_DT_CFL_DX53;
      C.hx = r53 ? std::pow(grid.dx, 5.0 / 3.0) : grid.dx;
      C.hy = r53 ? std::pow(grid.dy, 5.0 / 3.0) : grid.dy;
      C.cfl = cfg.cfl;
      C.done = 1;
      HW_CK(hw::prepare_stage2d(prec, cfg.equation, cfg.charwise));
    }
    const size_t plane = (size_t)cells * esz;
    HW_CK(cudaMalloc(&S, plane * nf));
    HW_CK(cudaMalloc(&A, plane * nf));
    HW_CK(cudaMalloc(&B, plane * nf));
    HW_CK(cudaMalloc(&H, plane * nd));
    HW_CK(cudaMalloc(&ctl, sizeof(hw::Ctl) * n));
    HW_CK(cudaMalloc(&ctl_manual, sizeof(hw::Ctl) * n));
    HW_CK(cudaMalloc(&alpha_op, sizeof(double) * n));
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
    if (dim == 1) {
      hw::Stage1Args a{};
      a.in = in; a.base = S; a.out = out; a.hat = hat;
      a.inst = inst_d; a.tasks = tasks_d; a.ntasks = ntasks; a.total = cells;
      a.ctl = c; a.alpha_op = alpha_op; a.stage = s;
      a.gamma_gas = cfg.gamma_gas; a.adv = cfg.adv_x; a.wp = wp;
      HW_CK(hw::launch_stage1d(prec, cfg.equation, cfg.charwise, a, num_sms, own));
    } else {
      hw::Stage2Args a{};
      a.in = in; a.base = S; a.out = out; a.hat = hat;
      a.grid = grid; a.ctl = c; a.ax_op = ax; a.ay_op = ay; a.stage = s;
      a.gamma_gas = cfg.gamma_gas; a.adv_x = cfg.adv_x; a.adv_y = cfg.adv_y; a.wp = wp;
      a.plane = cells;
      HW_CK(hw::launch_stage2d(prec, cfg.equation, cfg.charwise, a, num_sms, own));
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

  hweno_status one_step() {
    HW_CK(hw::launch_ctl_begin(ctl, n_inst, dim, own));
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
    else
      HW_CK(hw::launch_alpha2d(prec, cfg.equation, S, cells, cfg.gamma_gas, cfg.adv_x, cfg.adv_y, ctl,
                               num_sms, own));
    HW_CK(hw::launch_ctl_commit_alpha(ctl, n_inst, own));
    return HWENO_OK;
  }

  hweno_status set_state(const void* U, int on_device) {
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
    HW_CK(cudaStreamSynchronize(own));
    for (int k = 0; k < n_inst; ++k) {
      ctl_host[k] = ctl_init[k];
      ctl_host[k].dt = dt;
      ctl_host[k].ax = ax;
      ctl_host[k].ay = ay;
      ctl_host[k].done = 0;
    }
    HW_CK(cudaMemcpyAsync(ctl_manual, ctl_host, sizeof(hw::Ctl) * n_inst, cudaMemcpyHostToDevice, own));
    HW_TRY(rk_stages(ctl_manual));
    HW_CK(cudaStreamSynchronize(own));
    // the new state's alpha for the next advance
    HW_TRY(alpha_init());
    return leave();
  }

  hweno_status apply_operator(const double* ax, double ay, void* L, void* dh) {
    if (!has_state) return fail(HWENO_ERR_STATE, "no state set");
    if (!L || !dh) return fail(HWENO_ERR_ARG, "output pointer is NULL");
    HW_TRY(enter());
    if (dim == 1) {
      HW_CK(cudaStreamSynchronize(own));
      HW_CK(cudaMemcpy(alpha_op, ax, sizeof(double) * n_inst, cudaMemcpyHostToDevice));
    }
    HW_TRY(stage(0, S, L, ctl, ax[0], ay, dh));
    return leave();
  }
};

struct hweno_solver { Engine e; };
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
    HW_TRY(validate(&cfgs[k], 1));
    const hweno_config &a = cfgs[0], &b = cfgs[k];
    bool same = a.equation == b.equation && a.precision == b.precision && a.charwise == b.charwise &&
                a.linear_weights == b.linear_weights && a.weight_pow == b.weight_pow && a.eps == b.eps &&
                a.gamma_gas == b.gamma_gas && a.adv_x == b.adv_x;
    for (int m = 0; m < 3; ++m) same = same && a.lin_w[m] == b.lin_w[m];
    if (!same) return fail(HWENO_ERR_ARG, "config %d differs from config 0 in a batch-wide parameter", k);
  }
  hweno_batch* b = new (std::nothrow) hweno_batch();
  if (!b) return fail(HWENO_ERR_OOM, "host allocation failed");
  hweno_status st = b->e.init(n, cfgs, cuda_stream);
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

hweno_status hweno_batch_apply_operator(hweno_batch* b, const double* alpha, void* L_out,
                                        void* dhat_out) {
  if (!b || !alpha) return fail(HWENO_ERR_ARG, "batch or alpha is NULL");
  for (int k = 0; k < b->e.n_inst; ++k)
    if (!(alpha[k] >= 0.0)) return fail(HWENO_ERR_ARG, "alpha must be >= 0");
  return b->e.apply_operator(alpha, 0.0, L_out, dhat_out);
}

}  // extern "C"
