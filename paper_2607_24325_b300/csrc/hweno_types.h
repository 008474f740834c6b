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
};

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
};

// One 1D instance inside the concatenated field planes.
struct Inst1 {
  long long off;       // first cell of the instance in every field plane
  int n;               // cells
  int bc_lo, bc_hi;    // HWENO_BC_*
  int pad;
  double dx;
  double st_lo[4], st_hi[4];  // inflow states (conservative)
};

// 2D grid description.
struct Grid2 {
  int nx, ny;
  int bc[4];
  double dx, dy;
  double st[4][4];
};

}  // namespace hw
