// kernels.h -- host-side launch interface of the libhweno kernels.
#pragma once

#include <cuda_runtime.h>

#include "hweno_types.h"

namespace hw {

// Arguments of one 1D stage launch (all instances of a batch at once).
// stage 0: operator mode, out = L (2*nc planes), hat = limited derivatives;
// stage 1..3: SSP-RK3 stage s (Sec. 2.1 Step 4) reading `in`, the step's
// base state `base` (u-bar planes) and the stage-1 limited derivatives `hat`.
struct Stage1Args {
  const void* in;
  const void* base;
  void* out;
  void* hat;
  const Inst1* inst;
  const int2* tasks;      // (instance, first interior cell) per warp task
  int ntasks;
  long long total;        // plane stride (cells of all instances)
  Ctl* ctl;               // per instance
  const double* alpha_op; // stage 0: per-instance alpha
  int stage;
  double gamma_gas, adv;
  WeightParams wp;
};

// Arguments of one 2D stage launch.
struct Stage2Args {
  const void* in;
  const void* base;
  void* out;
  void* hat;              // 2*nc planes: v-hat then w-hat
  Grid2 grid;
  Ctl* ctl;
  double ax_op, ay_op;    // stage 0 alpha
  int stage;
  double gamma_gas, adv_x, adv_y;
  WeightParams wp;
  long long plane;        // nx * ny
};

constexpr int kTile1 = 30;   // interior cells per warp task (32 lanes - 2 ring cells)

cudaError_t launch_stage1d(int precision, int equation, int charwise, const Stage1Args& a,
                           int num_sms, cudaStream_t st);
cudaError_t launch_alpha1d(int precision, int equation, const void* U, long long total,
                           const Inst1* inst, const int2* tasks, int ntasks, double gamma_gas,
                           double adv, Ctl* ctl, int num_sms, cudaStream_t st);
cudaError_t launch_stage2d(int precision, int equation, int charwise, const Stage2Args& a,
                           int num_sms, cudaStream_t st);
cudaError_t prepare_stage2d(int precision, int equation, int charwise);
cudaError_t launch_alpha2d(int precision, int equation, const void* U, long long plane,
                           double gamma_gas, double adv_x, double adv_y, Ctl* ctl, int num_sms,
                           cudaStream_t st);
cudaError_t launch_ctl_begin(Ctl* ctl, int n, int dim, cudaStream_t st);
cudaError_t launch_ctl_end(Ctl* ctl, int n, cudaStream_t st);
cudaError_t launch_ctl_commit_alpha(Ctl* ctl, int n, cudaStream_t st);

}  // namespace hw
