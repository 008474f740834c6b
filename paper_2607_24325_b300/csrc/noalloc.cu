// noalloc.cu -- one SSP-RK3 step of a 1D problem without any device
// allocation.
//
// The regular solver (hweno_create / hweno_step) allocates its working
// memory with cudaMalloc.  Some callers cannot do that at the point where
// they want a step: a host application that has handed the whole device
// memory budget to its own pool allocator (so cudaMalloc would fail or
// break its accounting), or a latency-critical loop that must not pay
// cudaMalloc's implicit device-wide synchronisation.  For them this file
// keeps the step's working memory -- the two intermediate stage states, the
// stage-1 limited derivatives, the control block, the instance descriptor
// and the warp-task table -- in one file-scope device array of fixed size.
// Every GPU that loads the library holds that array until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "hweno.h"
#include "hweno_types.h"
#include "kernels.h"

namespace hw {
hweno_status report_error(hweno_status st, const char* msg);
hweno_status check_config(const hweno_config* cfg, int expect_dim);
}  // namespace hw

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr size_t kAlign = 256;

__device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];  // device address of g_step_scratch, per device
int g_sms[kMaxDevices];

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t inst, ctl, tasks, A, B, H, total;
};

Layout layout(long long n, int nc, size_t esz, int ntasks) {
  Layout L{};
  L.inst = 0;
  L.ctl = round_up(sizeof(hw::Inst1));
  L.tasks = L.ctl + round_up(sizeof(hw::Ctl));
  L.A = L.tasks + round_up(sizeof(int2) * (size_t)ntasks);
  L.B = L.A + round_up((size_t)n * 2 * nc * esz);
  L.H = L.B + round_up((size_t)n * 2 * nc * esz);
  L.total = L.H + round_up((size_t)n * nc * esz);
  return L;
}

Layout layout_for(long long n, int nc, size_t esz) {
  return layout(n, nc, esz, (int)((n + hw::kTile1 - 1) / hw::kTile1));
}

// The largest cell count whose layout fits the scratch array (the layout's
// size grows with n, so a bisection finds it exactly).
long long max_cells(int nc, size_t esz) {
  long long lo = 0, hi = (long long)(kScratchBytes / esz) + 1;  // layout(lo) fits, layout(hi) does not
  while (hi - lo > 1) {
    const long long mid = lo + (hi - lo) / 2;
    if (layout_for(mid, nc, esz).total <= kScratchBytes) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Writes the instance descriptor and the control block (next-alpha slot
// zeroed) and the warp-task table of this call into the scratch array.
__global__ void k_noalloc_setup(hw::Inst1 inst, hw::Ctl ctl, hw::Inst1* inst_out, hw::Ctl* ctl_out,
                                int2* tasks, int ntasks) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *inst_out = inst;
    *ctl_out = ctl;
  }
  for (; t < ntasks; t += gridDim.x * blockDim.x) tasks[t] = make_int2(0, t * hw::kTile1);
}

}  // namespace

extern "C" hweno_status hweno_step_1d_noalloc(const hweno_config* cfg, const void* U_in, void* U_out,
                                              double dt, double alpha, void* cuda_stream) {
  if (cfg && cfg->dim != 1)
    return hw::report_error(HWENO_ERR_ARG, "the allocation-free step takes 1D problems only");
  hweno_status st = hw::check_config(cfg, 1);
  if (st != HWENO_OK) return st;
  if (!U_in || !U_out) return hw::report_error(HWENO_ERR_ARG, "state pointer is NULL");
  if (!(dt >= 0.0) || !std::isfinite(dt) || !(alpha >= 0.0) || !std::isfinite(alpha))
    return hw::report_error(HWENO_ERR_ARG, "dt and alpha must be finite and non-negative");
  const int nc = cfg->equation == HWENO_EQ_EULER ? 3 : 1;
  const size_t esz = cfg->precision == HWENO_FP64 ? 8 : 4;
  const long long n = cfg->nx;
  const int ntasks = (int)((n + hw::kTile1 - 1) / hw::kTile1);
  const Layout L = layout(n, nc, esz, ntasks);
  if (L.total > kScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "nx = %lld needs %zu bytes of step scratch; the allocation-free step is limited to %zu bytes "
             "(%lld cells for this equation and precision)",
             n, L.total, kScratchBytes, max_cells(nc, esz));
    return hw::report_error(HWENO_ERR_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hw::report_error(HWENO_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return hw::report_error(HWENO_ERR_ARG, "device ordinal out of range");
  unsigned char* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      // once per device, with that device current: the device address of the
      // array (the host-side name is only a stand-in)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_step_scratch);
      if (e != cudaSuccess) return hw::report_error(HWENO_ERR_CUDA, cudaGetErrorString(e));
      int count = 0;
      e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return hw::report_error(HWENO_ERR_CUDA, cudaGetErrorString(e));
      g_sms[dev] = count;
      g_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    sms = g_sms[dev];
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  hw::Inst1 inst{};
  inst.off = 0;
  inst.n = cfg->nx;
  inst.bc_lo = cfg->bc[0];
  inst.bc_hi = cfg->bc[1];
  hw::set_spacing(inst, cfg->xlo, cfg->xhi, cfg->nx);
  for (int q = 0; q < 4; ++q) {
    inst.st_lo[q] = cfg->bc_state[0][q];
    inst.st_hi[q] = cfg->bc_state[1][q];
  }
  hw::Ctl ctl{};
  ctl.dt = dt;
  ctl.ax = alpha;
  ctl.dtf = (float)dt;
  ctl.axf = (float)alpha;
  ctl.hx = inst.dx;
  ctl.hy = 1.0;
  ctl.cfl = cfg->cfl;
  ctl.done = 0;  // amax_x / amax_y start at zero

  auto* inst_d = reinterpret_cast<hw::Inst1*>(base + L.inst);
  auto* ctl_d = reinterpret_cast<hw::Ctl*>(base + L.ctl);
  auto* tasks_d = reinterpret_cast<int2*>(base + L.tasks);
  void* A = base + L.A;
  void* B = base + L.B;
  void* H = base + L.H;
  const int sblocks = (ntasks + 255) / 256;
  k_noalloc_setup<<<sblocks < 1 ? 1 : sblocks, 256, 0, stream>>>(inst, ctl, inst_d, ctl_d, tasks_d, ntasks);
  e = cudaGetLastError();
  if (e != cudaSuccess) return hw::report_error(HWENO_ERR_CUDA, cudaGetErrorString(e));

  const hw::WeightParams wp = hw::weight_params(*cfg);
  const void* ins[3] = {U_in, A, B};
  void* outs[3] = {A, B, U_out};
  for (int s = 1; s <= 3; ++s) {
    hw::Stage1Args a{};
    a.in = ins[s - 1];
    a.base = U_in;  // u-bar^n of the step
    a.out = outs[s - 1];
    a.hat = H;
    a.inst = inst_d;
    a.tasks = tasks_d;
    a.ntasks = ntasks;
    a.total = n;
    a.ctl = ctl_d;
    a.alpha_op = nullptr;
    a.stage = s;
    a.gamma_gas = cfg->gamma_gas;
    a.adv = cfg->adv_x;
    a.gammaf = (float)cfg->gamma_gas;  // the FP32 kernels read these copies
    a.advf = (float)cfg->adv_x;
    a.wp = wp;
    e = hw::launch_stage1d(cfg->precision, cfg->equation, cfg->charwise, a, sms, stream);
    if (e != cudaSuccess) return hw::report_error(HWENO_ERR_CUDA, cudaGetErrorString(e));
  }
  return HWENO_OK;
}
