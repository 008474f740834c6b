// kernels.h -- host-side launch interface of the libhweno kernels.
#pragma once

#include <cuda_fp16.h>
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
  float gammaf, advf;     // the same, host-rounded to FP32
  WeightParams wp;
};

// Arguments of one 2D stage launch.
// The scalar parameters of the 2D stage in FP32, rounded on the host (the
// FP32 kernels use these directly: a double-to-float conversion re-done at
// every use would issue on the FP64 pipe).
struct Stage2F32 {
  float ax_op, ay_op, gamma_gas, adv_x, adv_y;
  float idx, idy, dyx, dxy;   // 1/dx, 1/dy, dy/dx, dx/dy
};
inline Stage2F32 stage2_f32(const Grid2& g, double ax_op, double ay_op, double gamma_gas, double adv_x,
                            double adv_y) {
  Stage2F32 f;
  f.ax_op = (float)ax_op; f.ay_op = (float)ay_op; f.gamma_gas = (float)gamma_gas;
  f.adv_x = (float)adv_x; f.adv_y = (float)adv_y;
  f.idx = (float)(1.0 / g.dx); f.idy = (float)(1.0 / g.dy);
  f.dyx = (float)(g.dy / g.dx); f.dxy = (float)(g.dx / g.dy);
  return f;
}

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
  Stage2F32 f32;
  long long plane;        // field plane stride: nx * ny, or the total cells of a batch
  const unsigned char* smooth;  // learned indicator: 1 = linear path allowed (nullptr: off)
  // 2D batch (batched = 1): per-instance descriptors, the tile table and,
  // for stage 0, per-instance (alpha_x, alpha_y); ctl holds one block per
  // instance.  grid, ax_op, ay_op and f32's grid ratios are then unused.
  int batched;
  const Inst2* inst;
  const Tile2* tiles;
  long long ntiles;
  const double* alpha_op;
  // Dynamic tile scheduler of the persistent launch (nullptr: static
  // stride): sched[0] hands out the tiles after each CTA's first, sched[1]
  // counts finished CTAs; the last CTA to finish zeroes both, so every
  // launch starts from zero.
  unsigned* sched;
};

// Learned troubled-cell indicator: per-sample training buffers and the
// FP16 inference weights.
struct MlpWork {
  float *h1, *dh1, *h2, *dh2, *dz, *loss, *loss_acc;
};
struct MlpDev {
  const __half* W1h;   // [32][80], columns 75..79 zero
  const __half* W2h;   // [32][32]
  const float* bias;   // b1[32], b2[32], w3[32], b3
  float z_thresh;      // logit of the troubled-probability threshold
};
constexpr int kMlpParams = 3521;

constexpr int kTile1 = 30;   // interior cells per warp task (32 lanes - 2 ring cells)
constexpr int kTile2 = 30;   // interior cells per 2D tile edge (the stage kernel's tile)

// Launch shapes chosen by the autotuner: 1D warps per block (1..8) and a cap
// on resident blocks per SM for the persistent grid; 2D persistent grid
// (one CTA per SM slot, tiles looped) or one CTA per tile.
struct LaunchShape {
  int warps1d = 4;
  int blocks_per_sm1d = 16;
  int persistent2d = 1;
};

cudaError_t launch_stage1d(int precision, int equation, int charwise, const Stage1Args& a,
                           int num_sms, cudaStream_t st, const LaunchShape& shape = LaunchShape());
cudaError_t launch_alpha1d(int precision, int equation, const void* U, long long total,
                           const Inst1* inst, const int2* tasks, int ntasks, double gamma_gas,
                           double adv, Ctl* ctl, int num_sms, cudaStream_t st);
cudaError_t launch_stage2d(int precision, int equation, int charwise, const Stage2Args& a,
                           int num_sms, cudaStream_t st, const LaunchShape& shape = LaunchShape());
cudaError_t prepare_stage2d(int precision, int equation, int charwise, const WeightParams& wp, bool batched);
cudaError_t launch_alpha2d(int precision, int equation, const void* U, long long count, long long plane,
                           double gamma_gas, double adv_x, double adv_y, Ctl* ctl, int num_sms,
                           cudaStream_t st);
cudaError_t launch_features2d(int precision, int equation, const void* U, const Grid2& G, long long plane,
                              const Ctl* ctl, float* feat, int num_sms, cudaStream_t st);
cudaError_t launch_labels2d(int precision, int equation, int charwise, const void* U, const Grid2& G,
                            long long plane, const WeightParams& wp, double gamma_gas, const Ctl* ctl, float* dev,
                            int num_sms, cudaStream_t st);
cudaError_t launch_mlp_train(const float* theta, const float* feat, const float* dev, const int* idx, int B,
                             float delta, float pos_weight, MlpWork& w, float* grad, cudaStream_t st);
cudaError_t launch_mlp_adam(float* theta, float* m, float* v, const float* g, float lr, int t, cudaStream_t st);
cudaError_t launch_mlp_predict(const float* theta, const float* feat, long long N, float* prob, int num_sms,
                               cudaStream_t st);
cudaError_t launch_count_above(const float* dev, long long n, float delta, unsigned long long* count, int num_sms,
                               cudaStream_t st);
cudaError_t prepare_mlp_infer2d();
cudaError_t launch_mlp_infer2d(int precision, int equation, const void* U, const Grid2& G, long long plane,
                               const MlpDev& m, const Ctl* ctl, unsigned char* troubled, unsigned char* smooth,
                               int num_sms, cudaStream_t st);
cudaError_t launch_ctl_begin(Ctl* ctl, int n, int dim, cudaStream_t st);
cudaError_t launch_ctl_end(Ctl* ctl, int n, cudaStream_t st);
cudaError_t launch_ctl_commit_alpha(Ctl* ctl, int n, cudaStream_t st);

}  // namespace hw
