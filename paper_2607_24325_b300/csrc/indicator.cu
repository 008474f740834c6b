// indicator.cu -- the learned troubled-cell indicator (no counterpart in the
// paper): a small MLP decides, once per step, which cells may use the linear
// reconstruction p0 (omega = gamma, Eq. rewrite-2D) instead of the full
// nonlinear characteristic HWENO path.  The full path stays the fallback.
//
//   features  5x5 patch of the density's (u-bar, v-bar, w-bar), scaled by
//             s = 1 / (patch range + KAPPA |centre| + TINY), centre
//             subtracted from the averages: 75 inputs, order [field][dy][dx]
//   network   75 -> 32 (ReLU) -> 32 (ReLU) -> 1, p = sigmoid(z)
//   label     plain scheme's largest |omega_m / gamma_m - 1| > delta
//   training  FP32: per-sample forward/backward, per-parameter gradient sums
//             (fixed order, deterministic), Adam
//   inference FP16 weights and features on the tensor cores (mma.sync
//             m16n8k16, FP32 accumulate), then a 3x3 dilation of the
//             troubled mask
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "hweno_stencil2d.cuh"
#include "kernels.h"

namespace hw {

constexpr int kNin = 75, kNinPad = 80, kNh = 32;
constexpr int kNParam = kNh * kNin + kNh + kNh * kNh + kNh + kNh + 1;  // 3521
constexpr float kKappa = 1e-3f, kTiny = 1e-30f;
// offsets of the parameter blocks in the flat vector
constexpr int kOffW1 = 0, kOffB1 = kNh * kNin, kOffW2 = kOffB1 + kNh, kOffB2 = kOffW2 + kNh * kNh,
              kOffW3 = kOffB2 + kNh, kOffB3 = kOffW3 + kNh;

// ---------------------------------------------------------------------------
// Features of one cell from its 5x5 patch (at(field, dy, dx), dy, dx in -2..2).
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ float patch_scale(F at, float& centre) {
  float lo = at(0, -2, -2), hi = lo;
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      const float v = at(0, dy, dx);
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
  centre = at(0, 0, 0);
  return 1.0f / ((hi - lo) + kKappa * fabsf(centre) + kTiny);
}

template <typename F>
__device__ __forceinline__ float feature(F at, int k, float centre, float s) {
  const int f = k / 25, r = k - f * 25, dy = r / 5 - 2, dx = r % 5 - 2;
  const float v = at(f, dy, dx);
  return (f == 0 ? v - centre : v) * s;
}

template <typename T, int EQ, int NC>
__global__ void __launch_bounds__(256) k_features2d(const T* __restrict__ U, Grid2 G, long long plane,
                                                    const Ctl* ctl, float* __restrict__ feat) {
  const double t_bc = ctl->t;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < plane;
       c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / G.nx), i = (int)(c - (long long)j * G.nx);
    auto at = [&](int f, int dy, int dx) -> float {
      const int fld = f * NC;  // density component of field group f
      const int ii = i + dx, jj = j + dy;
      if (ii >= 0 && ii < G.nx && jj >= 0 && jj < G.ny) return (float)U[fld * plane + (long long)jj * G.nx + ii];
      return (float)load_ghost2<T, EQ, NC>(U, plane, G, fld, ii, jj, t_bc);
    };
    float centre;
    const float s = patch_scale(at, centre);
#pragma unroll
    for (int k = 0; k < kNin; ++k) feat[c * kNin + k] = feature(at, k, centre, s);
  }
}

// ---------------------------------------------------------------------------
// Labels: the plain scheme's largest |omega_m / gamma_m - 1| per cell over
// every reconstructed field of both passes (one thread per cell).
// ---------------------------------------------------------------------------
template <typename T, int EQ, bool CHR, int D>
__device__ __forceinline__ void pass_dev(const T* __restrict__ U, long long plane, const Grid2& G, int i, int j,
                                         const WeightsT<T>& w, T g, double t_bc, T& dev) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
  // frame offsets (n along the pass normal, t along the tangent)
  const int on[9] = {-1, 0, 1, -1, 0, 1, -1, 0, 1}, ot[9] = {-1, -1, -1, 0, 0, 0, 1, 1, 1};
  const int fn[4] = {-1, 1, 0, 0}, ft[4] = {0, 0, -1, 1};
  auto val = [&](int fld, int n, int t) -> T {
    const int ii = i + (D == 0 ? n : t), jj = j + (D == 0 ? t : n);
    if (ii >= 0 && ii < G.nx && jj >= 0 && jj < G.ny) return U[fld * plane + (long long)jj * G.nx + ii];
    return load_ghost2<T, EQ, NC>(U, plane, G, fld, ii, jj, t_bc);
  };
  T q[NC][17];
  for (int s = 0; s < 17; ++s) {
    const int dd = s < 9 ? 0 : (s < 13 ? 1 : 2);
    const int n = s < 9 ? on[s] : fn[(s - 9) & 3], t = s < 9 ? ot[s] : ft[(s - 9) & 3];
#pragma unroll
    for (int k = 0; k < NC; ++k) q[k][s] = val(frame_field<D, EQ, NC>(dd, k), n, t);
  }
  if constexpr (CHR) {
    const Eig<T> e = eig2<T>(q[0][4], q[1][4], q[2][4], q[3][4], g);
    for (int s = 0; s < 17; ++s) {
      T x[4], y[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = q[k][s];
      l2_apply<0>(e, x, y);
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k][s] = y[k];
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T cu[15];
    recon2<T, true>(q[k], w, false, cu, &dev);
  }
}

template <typename T, int EQ, bool CHR>
__global__ void __launch_bounds__(128) k_labels2d(const T* __restrict__ U, Grid2 G, long long plane,
                                                  WeightParams wp, double gamma_gas, const Ctl* ctl,
                                                  float* __restrict__ dev_out) {
  const double t_bc = ctl->t;
  const WeightsT<T> wx = make_weights<T>(wp);
  WeightsT<T> wy = wx;
  wy.g[2] = wx.g[4];
  wy.g[4] = wx.g[2];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < plane;
       c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / G.nx), i = (int)(c - (long long)j * G.nx);
    T dev = T(0);
    pass_dev<T, EQ, CHR, 0>(U, plane, G, i, j, wx, (T)gamma_gas, t_bc, dev);
    pass_dev<T, EQ, CHR, 1>(U, plane, G, i, j, wy, (T)gamma_gas, t_bc, dev);
    dev_out[c] = (float)dev;
  }
}

// ---------------------------------------------------------------------------
// Training (FP32, deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float log_sigmoid(float z) { return fminf(z, 0.0f) - log1pf(expf(-fabsf(z))); }

// One thread per sample b of the minibatch (sample index idx[b]): forward
// pass, weighted BCE loss, and the back-propagated deltas.
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(const float* __restrict__ theta, const float* __restrict__ feat,
                                                     const float* __restrict__ dev, const int* __restrict__ idx,
                                                     int B, float delta, float pos_weight, float* h1o, float* dh1o,
                                                     float* h2o, float* dh2o, float* dzo, float* losso) {
  __shared__ float th[kNParam];
  for (int k = threadIdx.x; k < kNParam; k += blockDim.x) th[k] = theta[k];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const long long s = idx[b];
  const float* x = feat + s * kNin;
  const float y = dev[s] > delta ? 1.0f : 0.0f;
  float a1[kNh], a2[kNh];
  for (int n = 0; n < kNh; ++n) {
    float acc = th[kOffB1 + n];
    for (int k = 0; k < kNin; ++k) acc = fmaf(th[kOffW1 + n * kNin + k], x[k], acc);
    a1[n] = acc;
  }
  for (int n = 0; n < kNh; ++n) {
    float acc = th[kOffB2 + n];
    for (int m = 0; m < kNh; ++m) acc = fmaf(th[kOffW2 + n * kNh + m], fmaxf(a1[m], 0.0f), acc);
    a2[n] = acc;
  }
  float z = th[kOffB3];
  for (int m = 0; m < kNh; ++m) z = fmaf(th[kOffW3 + m], fmaxf(a2[m], 0.0f), z);
  const float p = 1.0f / (1.0f + expf(-z));
  const float wt = y > 0.5f ? pos_weight : 1.0f;
  losso[b] = -wt * (y * log_sigmoid(z) + (1.0f - y) * log_sigmoid(-z));
  const float dz = wt * (p - y) / (float)B;
  dzo[b] = dz;
  float d2[kNh];
  for (int n = 0; n < kNh; ++n) {
    d2[n] = a2[n] > 0.0f ? dz * th[kOffW3 + n] : 0.0f;
    h2o[(long long)b * kNh + n] = fmaxf(a2[n], 0.0f);
    dh2o[(long long)b * kNh + n] = d2[n];
  }
  for (int m = 0; m < kNh; ++m) {
    float acc = 0.0f;
    for (int n = 0; n < kNh; ++n) acc = fmaf(th[kOffW2 + n * kNh + m], d2[n], acc);
    h1o[(long long)b * kNh + m] = fmaxf(a1[m], 0.0f);
    dh1o[(long long)b * kNh + m] = a1[m] > 0.0f ? acc : 0.0f;
  }
}

// One thread per parameter: its gradient summed over the batch in sample
// order; the last thread also forms the mean loss.
__global__ void __launch_bounds__(128) k_mlp_grads(const float* __restrict__ feat, const int* __restrict__ idx,
                                                   int B, const float* __restrict__ h1, const float* __restrict__ dh1,
                                                   const float* __restrict__ h2, const float* __restrict__ dh2,
                                                   const float* __restrict__ dz, const float* __restrict__ loss,
                                                   float* __restrict__ grad, float* __restrict__ loss_acc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kNParam) return;
  float acc = 0.0f;
  if (p < kOffB1) {
    const int n = p / kNin, k = p - n * kNin;
    for (int b = 0; b < B; ++b) acc = fmaf(dh1[(long long)b * kNh + n], feat[(long long)idx[b] * kNin + k], acc);
  } else if (p < kOffW2) {
    const int n = p - kOffB1;
    for (int b = 0; b < B; ++b) acc += dh1[(long long)b * kNh + n];
  } else if (p < kOffB2) {
    const int n = (p - kOffW2) / kNh, m = (p - kOffW2) % kNh;
    for (int b = 0; b < B; ++b) acc = fmaf(dh2[(long long)b * kNh + n], h1[(long long)b * kNh + m], acc);
  } else if (p < kOffW3) {
    const int n = p - kOffB2;
    for (int b = 0; b < B; ++b) acc += dh2[(long long)b * kNh + n];
  } else if (p < kOffB3) {
    const int m = p - kOffW3;
    for (int b = 0; b < B; ++b) acc = fmaf(dz[b], h2[(long long)b * kNh + m], acc);
  } else if (p == kOffB3) {
    for (int b = 0; b < B; ++b) acc += dz[b];
  } else {  // p == kNParam: mean loss of the batch, accumulated
    for (int b = 0; b < B; ++b) acc += loss[b];
    loss_acc[0] += acc / (float)B;
    loss_acc[1] += 1.0f;
    return;
  }
  grad[p] = acc;
}

// Adam (Kingma & Ba 2015) with bias correction, step t >= 1.
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNParam) return;
  const float gi = g[p];
  const float mi = b1 * m[p] + (1.0f - b1) * gi;
  const float vi = b2 * v[p] + (1.0f - b2) * gi * gi;
  m[p] = mi;
  v[p] = vi;
  theta[p] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP32 forward for evaluation: probability per sample.
__global__ void __launch_bounds__(128) k_mlp_predict(const float* __restrict__ theta, const float* __restrict__ feat,
                                                     long long N, float* __restrict__ prob) {
  __shared__ float th[kNParam];
  for (int k = threadIdx.x; k < kNParam; k += blockDim.x) th[k] = theta[k];
  __syncthreads();
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const float* x = feat + s * kNin;
    float a1[kNh];
    for (int n = 0; n < kNh; ++n) {
      float acc = th[kOffB1 + n];
      for (int k = 0; k < kNin; ++k) acc = fmaf(th[kOffW1 + n * kNin + k], x[k], acc);
      a1[n] = fmaxf(acc, 0.0f);
    }
    float z = th[kOffB3];
    for (int n = 0; n < kNh; ++n) {
      float acc = th[kOffB2 + n];
      for (int m = 0; m < kNh; ++m) acc = fmaf(th[kOffW2 + n * kNh + m], a1[m], acc);
      z = fmaf(th[kOffW3 + n], fmaxf(acc, 0.0f), z);
    }
    prob[s] = 1.0f / (1.0f + expf(-z));
  }
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores.
// Weights: W1h [32][80] (columns 75..79 zero) and W2h [32][32] in FP16,
// bias b1[32], b2[32], w3[32], b3 in FP32 (MlpDev).
// A CTA (8 warps) takes a 32 x 8 tile of cells: it stages the 36 x 12 box
// of the three density fields, every thread writes its cell's 80 FP16
// features to shared memory, and each warp runs its row's 32 cells as two
// 16-row m-tiles through layer 1 (5 k-steps x 4 n-tiles), layer 2 (2 x 4)
// and the output dot product.
// ---------------------------------------------------------------------------
constexpr int kTX = 32, kTY = 8, kBXW = kTX + 4, kBYH = kTY + 4, kFP = 88;  // feature row pitch (halves)

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <typename T, int EQ, int NC>
__global__ void __launch_bounds__(256) k_mlp_infer2d(const T* __restrict__ U, Grid2 G, long long plane,
                                                     const __half* __restrict__ W1h, const __half* __restrict__ W2h,
                                                     const float* __restrict__ bias, float z_thresh,
                                                     const Ctl* ctl, unsigned char* __restrict__ troubled) {
  const double t_bc = ctl->t;
  __shared__ float box[3][kBYH][kBXW];
  extern __shared__ __align__(16) unsigned char hw_dsm[];
  __half(*feat)[kFP] = reinterpret_cast<__half(*)[kFP]>(hw_dsm);  // [256][kFP], dynamic
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tig = lane & 3;
  // B fragments of both layers stay in registers for the whole kernel
  uint32_t B1[4][5][2], B2[4][2][2];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const __half* r = W1h + (t * 8 + g) * kNinPad + s * 16 + tig * 2;
      B1[t][s][0] = *reinterpret_cast<const uint32_t*>(r);
      B1[t][s][1] = *reinterpret_cast<const uint32_t*>(r + 8);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const __half* r = W2h + (t * 8 + g) * kNh + s * 16 + tig * 2;
      B2[t][s][0] = *reinterpret_cast<const uint32_t*>(r);
      B2[t][s][1] = *reinterpret_cast<const uint32_t*>(r + 8);
    }
  }
  const int tiles_x = (G.nx + kTX - 1) / kTX, tiles = tiles_x * ((G.ny + kTY - 1) / kTY);
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int i0 = (tile % tiles_x) * kTX, j0 = (tile / tiles_x) * kTY;
    __syncthreads();
    for (int e = tid; e < 3 * kBYH * kBXW; e += blockDim.x) {
      const int f = e / (kBYH * kBXW), r = (e / kBXW) % kBYH, cc = e % kBXW;
      int i = i0 - 2 + cc, j = j0 - 2 + r;
      i = min(max(i, -2), G.nx + 1);
      j = min(max(j, -2), G.ny + 1);
      const int fld = f * NC;
      float v;
      if (i >= 0 && i < G.nx && j >= 0 && j < G.ny) v = (float)U[fld * plane + (long long)j * G.nx + i];
      else v = (float)load_ghost2<T, EQ, NC>(U, plane, G, fld, i, j, t_bc);
      box[f][r][cc] = v;
    }
    __syncthreads();
    {
      const int tx = tid & 31, ty = tid >> 5;
      auto at = [&](int f, int dy, int dx) -> float { return box[f][ty + 2 + dy][tx + 2 + dx]; };
      float centre;
      const float s = patch_scale(at, centre);
      __half* row = feat[tid];
#pragma unroll
      for (int k = 0; k < kNin; k += 2) {  // fully unrolled: patch offsets are constants
        const float lo = feature(at, k, centre, s);
        const float hi = k + 1 < kNin ? feature(at, k + 1, centre, s) : 0.0f;
        *reinterpret_cast<__half2*>(row + k) = __floats2half2_rn(lo, hi);
      }
      *reinterpret_cast<__half2*>(row + 76) = __floats2half2_rn(0.0f, 0.0f);
      *reinterpret_cast<__half2*>(row + 78) = __floats2half2_rn(0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = warp * 32 + mt * 16;  // first feature row of this m-tile
      float acc1[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc1[t][q] = 0.0f;
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(&feat[r0 + g][s * 16 + tig * 2]);
        a[1] = *reinterpret_cast<const uint32_t*>(&feat[r0 + g + 8][s * 16 + tig * 2]);
        a[2] = *reinterpret_cast<const uint32_t*>(&feat[r0 + g][s * 16 + tig * 2 + 8]);
        a[3] = *reinterpret_cast<const uint32_t*>(&feat[r0 + g + 8][s * 16 + tig * 2 + 8]);
#pragma unroll
        for (int t = 0; t < 4; ++t) mma16816(acc1[t], a, B1[t][s][0], B1[t][s][1]);
      }
      // bias + ReLU, repacked as the A fragments of layer 2 (C layout = A layout)
      uint32_t a2[2][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n0 = t * 8 + tig * 2;
        const float h0 = fmaxf(acc1[t][0] + bias[n0], 0.0f), h1 = fmaxf(acc1[t][1] + bias[n0 + 1], 0.0f);
        const float h2 = fmaxf(acc1[t][2] + bias[n0], 0.0f), h3 = fmaxf(acc1[t][3] + bias[n0 + 1], 0.0f);
        const int s = t >> 1, hi = t & 1;
        a2[s][hi * 2 + 0] = pack_half2(h0, h1);
        a2[s][hi * 2 + 1] = pack_half2(h2, h3);
      }
      float acc2[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc2[t][q] = 0.0f;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) mma16816(acc2[t], a2[s], B2[t][s][0], B2[t][s][1]);
      float z0 = 0.0f, z1 = 0.0f;  // rows g and g+8
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n0 = t * 8 + tig * 2;
        z0 += bias[64 + n0] * fmaxf(acc2[t][0] + bias[32 + n0], 0.0f) +
              bias[64 + n0 + 1] * fmaxf(acc2[t][1] + bias[32 + n0 + 1], 0.0f);
        z1 += bias[64 + n0] * fmaxf(acc2[t][2] + bias[32 + n0], 0.0f) +
              bias[64 + n0 + 1] * fmaxf(acc2[t][3] + bias[32 + n0 + 1], 0.0f);
      }
      z0 += __shfl_xor_sync(HW_FULL_MASK, z0, 1);
      z0 += __shfl_xor_sync(HW_FULL_MASK, z0, 2);
      z1 += __shfl_xor_sync(HW_FULL_MASK, z1, 1);
      z1 += __shfl_xor_sync(HW_FULL_MASK, z1, 2);
      if (tig == 0) {
        const int j = j0 + warp;
        const int ia = i0 + mt * 16 + g, ib = ia + 8;
        if (j < G.ny) {
          if (ia < G.nx) troubled[(long long)j * G.nx + ia] = (z0 + bias[96]) > z_thresh ? 1 : 0;
          if (ib < G.nx) troubled[(long long)j * G.nx + ib] = (z1 + bias[96]) > z_thresh ? 1 : 0;
        }
      }
    }
  }
}

// smooth[c] = 1 when no cell of c's 3x3 neighbourhood (inside the grid) is troubled.
__global__ void k_dilate(const unsigned char* __restrict__ troubled, int nx, int ny, unsigned char* __restrict__ smooth) {
  const long long n = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
    unsigned char t = 0;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di, jj = j + dj;
        if (ii >= 0 && ii < nx && jj >= 0 && jj < ny) t |= troubled[(long long)jj * nx + ii];
      }
    smooth[c] = t ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static unsigned grid_for(long long n, int threads, int num_sms, int per_sm) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)num_sms * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_features2d(int precision, int equation, const void* U, const Grid2& G, long long plane,
                              const Ctl* ctl, float* feat, int num_sms, cudaStream_t st) {
  const unsigned b = grid_for(plane, 256, num_sms, 8);
#define HW_F(T, EQ, NC) k_features2d<T, EQ, NC><<<b, 256, 0, st>>>(static_cast<const T*>(U), G, plane, ctl, feat)
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) HW_F(double, HWENO_EQ_EULER, 4);
    else if (equation == HWENO_EQ_BURGERS) HW_F(double, HWENO_EQ_BURGERS, 1);
    else HW_F(double, HWENO_EQ_ADVECTION, 1);
  } else {
    if (equation == HWENO_EQ_EULER) HW_F(float, HWENO_EQ_EULER, 4);
    else if (equation == HWENO_EQ_BURGERS) HW_F(float, HWENO_EQ_BURGERS, 1);
    else HW_F(float, HWENO_EQ_ADVECTION, 1);
  }
#undef HW_F
  return cudaGetLastError();
}

cudaError_t launch_labels2d(int precision, int equation, int charwise, const void* U, const Grid2& G,
                            long long plane, const WeightParams& wp, double gamma_gas, const Ctl* ctl, float* dev,
                            int num_sms, cudaStream_t st) {
  const unsigned b = grid_for(plane, 128, num_sms, 8);
  const bool chr = equation == HWENO_EQ_EULER && charwise;
#define HW_L(T, EQ, C) \
  k_labels2d<T, EQ, C><<<b, 128, 0, st>>>(static_cast<const T*>(U), G, plane, wp, gamma_gas, ctl, dev)
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) { if (chr) HW_L(double, HWENO_EQ_EULER, true); else HW_L(double, HWENO_EQ_EULER, false); }
    else if (equation == HWENO_EQ_BURGERS) HW_L(double, HWENO_EQ_BURGERS, false);
    else HW_L(double, HWENO_EQ_ADVECTION, false);
  } else {
    if (equation == HWENO_EQ_EULER) { if (chr) HW_L(float, HWENO_EQ_EULER, true); else HW_L(float, HWENO_EQ_EULER, false); }
    else if (equation == HWENO_EQ_BURGERS) HW_L(float, HWENO_EQ_BURGERS, false);
    else HW_L(float, HWENO_EQ_ADVECTION, false);
  }
#undef HW_L
  return cudaGetLastError();
}

cudaError_t launch_mlp_train(const float* theta, const float* feat, const float* dev, const int* idx, int B,
                             float delta, float pos_weight, MlpWork& w, float* grad, cudaStream_t st) {
  k_mlp_fwd_bwd<<<(B + 127) / 128, 128, 0, st>>>(theta, feat, dev, idx, B, delta, pos_weight, w.h1, w.dh1, w.h2,
                                                  w.dh2, w.dz, w.loss);
  k_mlp_grads<<<(kNParam + 1 + 127) / 128, 128, 0, st>>>(feat, idx, B, w.h1, w.dh1, w.h2, w.dh2, w.dz, w.loss, grad,
                                                          w.loss_acc);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* theta, float* m, float* v, const float* g, float lr, int t, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_mlp_adam<<<(kNParam + 127) / 128, 128, 0, st>>>(theta, m, v, g, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

// Number of label sources above delta (the positives of a training set):
// a warp count per block, one atomic per warp.
__global__ void __launch_bounds__(256) k_count_above(const float* __restrict__ dev, long long n, float delta,
                                                     unsigned long long* count) {
  unsigned c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c += dev[i] > delta ? 1u : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(HW_FULL_MASK, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

cudaError_t launch_count_above(const float* dev, long long n, float delta, unsigned long long* count, int num_sms,
                               cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_count_above<<<grid_for(n, 256, num_sms, 4), 256, 0, st>>>(dev, n, delta, count);
  return cudaGetLastError();
}

cudaError_t launch_mlp_predict(const float* theta, const float* feat, long long N, float* prob, int num_sms,
                               cudaStream_t st) {
  k_mlp_predict<<<grid_for(N, 128, num_sms, 8), 128, 0, st>>>(theta, feat, N, prob);
  return cudaGetLastError();
}

constexpr size_t kFeatBytes = sizeof(__half) * kTX * kTY * kFP;

cudaError_t prepare_mlp_infer2d() {
  cudaError_t e = cudaSuccess;
#define HW_P(T, EQ, NC)                                                                              \
  if (e == cudaSuccess)                                                                              \
    e = cudaFuncSetAttribute(k_mlp_infer2d<T, EQ, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)kFeatBytes);
  HW_P(double, HWENO_EQ_EULER, 4) HW_P(double, HWENO_EQ_BURGERS, 1) HW_P(double, HWENO_EQ_ADVECTION, 1)
  HW_P(float, HWENO_EQ_EULER, 4) HW_P(float, HWENO_EQ_BURGERS, 1) HW_P(float, HWENO_EQ_ADVECTION, 1)
#undef HW_P
  return e;
}

cudaError_t launch_mlp_infer2d(int precision, int equation, const void* U, const Grid2& G, long long plane,
                               const MlpDev& m, const Ctl* ctl, unsigned char* troubled, unsigned char* smooth,
                               int num_sms, cudaStream_t st) {
  const long long tiles = (long long)((G.nx + kTX - 1) / kTX) * ((G.ny + kTY - 1) / kTY);
  const unsigned b = (unsigned)(tiles < (long long)num_sms * 4 ? tiles : (long long)num_sms * 4);
#define HW_I(T, EQ, NC) k_mlp_infer2d<T, EQ, NC><<<b, 256, kFeatBytes, st>>>(static_cast<const T*>(U), G, plane, \
                                                                             m.W1h, m.W2h, m.bias, m.z_thresh, ctl, troubled)
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) HW_I(double, HWENO_EQ_EULER, 4);
    else if (equation == HWENO_EQ_BURGERS) HW_I(double, HWENO_EQ_BURGERS, 1);
    else HW_I(double, HWENO_EQ_ADVECTION, 1);
  } else {
    if (equation == HWENO_EQ_EULER) HW_I(float, HWENO_EQ_EULER, 4);
    else if (equation == HWENO_EQ_BURGERS) HW_I(float, HWENO_EQ_BURGERS, 1);
    else HW_I(float, HWENO_EQ_ADVECTION, 1);
  }
#undef HW_I
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dilate<<<grid_for(plane, 256, num_sms, 8), 256, 0, st>>>(troubled, G.nx, G.ny, smooth);
  return cudaGetLastError();
}

}  // namespace hw
