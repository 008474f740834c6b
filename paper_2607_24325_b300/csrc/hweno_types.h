// hweno_types.h -- plain structs shared by the host side of libhweno and its
// kernels (device control block, instance descriptors, launch arguments).
#pragma once

#include <stdint.h>

#include "hweno.h"

namespace hw {

// Scheme constants (Eq. rewrite / rewrite-2D, Eq. nonlinear-weights).
struct WeightParams {
  double g[5];
  double eps;
  int pow2;
  int linear;
  int typical;   // 1: Jiang-Shu integral indicator for p0
  // 1: the mixed precision's FP32 screens clear nothing (every lane takes
  // the FP64 indicator).  Set on the host only, by the screen-off
  // verification build, so that both builds compile the same device code.
  int screen_off;
  // the same in FP32, rounded on the host: FP32 kernels read these
  // parameters directly (a conversion re-done at every use would issue on
  // the FP64 pipe)
  float gf[5];
  float inv_g0f;
  float epsf;
};

// The scheme constants of a configuration, in both precisions.
inline WeightParams weight_params(const hweno_config& c) {
  WeightParams w{};
  for (int m = 0; m < 5; ++m) {
    w.g[m] = c.lin_w[m];
    w.gf[m] = (float)c.lin_w[m];
  }
  w.eps = c.eps;
  w.epsf = (float)c.eps;
  w.inv_g0f = (float)(1.0 / c.lin_w[0]);
  w.pow2 = c.weight_pow == 2;
  w.linear = c.linear_weights != 0;
  w.typical = c.smoothness == HWENO_BETA_TYPICAL;
#ifdef HWENO_SCREEN_OFF
  w.screen_off = 1;
#else
  w.screen_off = 0;
#endif
  return w;
}

// Device-resident time-stepping state of one problem instance.  alpha of
// the step in progress is (ax, ay); stage 3 accumulates the next step's
// alpha into amax_x/amax_y as bit patterns of non-negative doubles.
struct Ctl {
  double t, t_final, dt, ax, ay;
  double hx, hy;        // dx or dx^(5/3) of the dt rule
  double cfl;
  unsigned long long amax_x, amax_y;
  int steps, max_steps, done, last, err;
  int pad;
  float dtf, axf, ayf, fpad;  // dt, ax, ay rounded to FP32 for the FP32 kernels
};

// One 1D instance inside the concatenated field planes.
struct Inst1 {
  long long off;       // first cell of the instance in every field plane
  int n;               // cells
  int bc_lo, bc_hi;    // HWENO_BC_*
  int pad;
  double dx;
  double idx;                 // 1 / dx
  float dxf, idxf;            // the same in FP32 (host-rounded, for the FP32 kernels)
  double st_lo[4], st_hi[4];  // inflow states (conservative)
};

// Grid spacing fields of an instance from its cell count and extent.
inline void set_spacing(Inst1& I, double xlo, double xhi, int nx) {
  I.dx = (xhi - xlo) / nx;
  I.idx = 1.0 / I.dx;
  I.dxf = (float)I.dx;
  I.idxf = (float)I.idx;
}

// 2D grid description.
struct Grid2 {
  int nx, ny;
  int bc[4];
  double dx, dy;
  double xlo, ylo;
  double st[4][4];
  double st2[4][4];   // second state of HWENO_BC_SHOCK sides
  double bcp[4][2];   // HWENO_BC_SPLIT / HWENO_BC_SHOCK parameters
};

// One 2D instance inside the concatenated field planes of a 2D batch.
struct Inst2 {
  long long off;                   // first cell of the instance in every field plane
  Grid2 grid;
  double idx, idy, dyx, dxy;       // 1/dx, 1/dy, dy/dx, dx/dy
  float idxf, idyf, dyxf, dxyf;    // the same rounded to FP32
};

// One 30 x 30 tile of a 2D batch: its instance and its origin.
struct Tile2 {
  int inst, i0, j0, pad;
};

}  // namespace hw
