// control.cu -- device-resident time-step control (Sec. 2.1 Step 4 with the
// CFL rule): dt from the step's alpha, last step clipped to t_final, time
// and step counters advanced, next alpha committed, non-physical states
// (NaN or non-positive pressure/density, seen as a NaN alpha) flagged.
#include <cuda_runtime.h>
#include <math.h>

#include "hweno_device.cuh"
#include "kernels.h"

namespace hw {

__global__ void k_ctl_begin(Ctl* ctl, int n, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Ctl* c = ctl + i;
  if (c->done) return;
  if (!(c->t < c->t_final) || c->steps >= c->max_steps) {
    c->done = 1;
    return;
  }
  double dt;
  if (dim == 1) {
    dt = c->ax > 0.0 ? c->cfl * c->hx / c->ax : INFINITY;
  } else {
    const double rate = c->ax / c->hx + c->ay / c->hy;
    dt = rate > 0.0 ? c->cfl / rate : INFINITY;
  }
  if (!(dt > 0.0)) {  // NaN alpha: non-physical state
    c->err = HWENO_ERR_NONPHYSICAL;
    c->done = 1;
    return;
  }
  c->last = 0;
  if (c->t + dt >= c->t_final) {
    dt = c->t_final - c->t;
    c->last = 1;
  }
  c->dt = dt;
  c->dtf = (float)dt;
  c->axf = (float)c->ax;
  c->ayf = (float)c->ay;
}

__global__ void k_ctl_end(Ctl* ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Ctl* c = ctl + i;
  if (c->done) return;
  const double tn = c->t + c->dt;
  c->t = (c->t_final - tn <= 1e-15 * fabs(c->t_final)) ? c->t_final : tn;
  c->steps += 1;
  c->ax = __longlong_as_double((long long)c->amax_x);
  c->ay = __longlong_as_double((long long)c->amax_y);
  c->amax_x = 0ull;
  c->amax_y = 0ull;
  if (!(c->ax <= 1.7976931348623157e308) || !(c->ay <= 1.7976931348623157e308)) {
    c->err = HWENO_ERR_NONPHYSICAL;
    c->done = 1;
  }
}

// alpha of the current state (after an alpha reduction into amax).
__global__ void k_ctl_commit_alpha(Ctl* ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Ctl* c = ctl + i;
  c->ax = __longlong_as_double((long long)c->amax_x);
  c->ay = __longlong_as_double((long long)c->amax_y);
  c->amax_x = 0ull;
  c->amax_y = 0ull;
  if (!(c->ax <= 1.7976931348623157e308) || !(c->ay <= 1.7976931348623157e308))
    c->err = HWENO_ERR_NONPHYSICAL;
}

cudaError_t launch_ctl_begin(Ctl* ctl, int n, int dim, cudaStream_t st) {
  k_ctl_begin<<<(n + 127) / 128, 128, 0, st>>>(ctl, n, dim);
  return cudaGetLastError();
}
cudaError_t launch_ctl_end(Ctl* ctl, int n, cudaStream_t st) {
  k_ctl_end<<<(n + 127) / 128, 128, 0, st>>>(ctl, n);
  return cudaGetLastError();
}
cudaError_t launch_ctl_commit_alpha(Ctl* ctl, int n, cudaStream_t st) {
  k_ctl_commit_alpha<<<(n + 127) / 128, 128, 0, st>>>(ctl, n);
  return cudaGetLastError();
}

}  // namespace hw
