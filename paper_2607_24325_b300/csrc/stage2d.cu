// stage2d.cu -- fused 2D HWENO stage kernel (Sec. 2.2 Steps 1-4, Remark 1).
//
// A CTA (8 warps) owns a 30 x 30 tile of interior cells.  It stages the
// 34 x 34 box (tile + 2-cell halo) of every field in shared memory, resolving
// ghost cells with the boundary map on the way in, then runs
//   x pass: warp per row, lane l = cell i0-1+l.  Each lane reconstructs its
//           cell (characteristic-wise with the x eigenvectors of its own
//           average for Euler), evaluates u, u_x, u_y at the 3 Gauss points
//           of both x faces, takes its left neighbour's right-face values by
//           shuffle and forms the Lax-Friedrichs fluxes of its LEFT face
//           (each interface once); the right-face flux comes from lane+1.
//           The x part of L and v-hat go to a shared-memory stash.
//   y pass: the same code on the transposed box (warp per column, lanes
//           along y).  Transposing swaps the roles of x and y, of v-bar and
//           w-bar, of the two momentum components and of the stencils S2 and
//           S4, so the y physics is the x physics in the transposed frame.
//           It adds the y part of L and applies the RK stage.
// Interface values, fluxes and L never go through HBM.
#include <cuda_runtime.h>

#include "hweno_device.cuh"
#include "hweno_stencil2d.cuh"
#include "kernels.h"

namespace hw {

static_assert(kT2 == kTile2, "host tile table and kernel tile size differ");

// Lax-Friedrichs fluxes of the pass-frame x physics at one point:
// f, f'(u) v (normal moment), f'(u) w (tangential moment).
template <typename T, int NC, int EQ>
__device__ __forceinline__ void lf_point(const T* Um, const T* Vm, const T* Wm, const T* Up, const T* Vp,
                                         const T* Wp, T alpha, T g, T adv, T* fu, T* fv, T* fw) {
  T Fm[NC], Fp[NC], HVm[NC], HVp[NC], HWm[NC], HWp[NC];
  if constexpr (EQ == HWENO_EQ_EULER) {
    euler2_flux<0>(Um, Vm, Wm, g, Fm, HVm, HWm);
    euler2_flux<0>(Up, Vp, Wp, g, Fp, HVp, HWp);
  } else if constexpr (EQ == HWENO_EQ_BURGERS) {
    Fm[0] = T(0.5) * Um[0] * Um[0]; HVm[0] = Um[0] * Vm[0]; HWm[0] = Um[0] * Wm[0];
    Fp[0] = T(0.5) * Up[0] * Up[0]; HVp[0] = Up[0] * Vp[0]; HWp[0] = Up[0] * Wp[0];
  } else {
    Fm[0] = adv * Um[0]; HVm[0] = adv * Vm[0]; HWm[0] = adv * Wm[0];
    Fp[0] = adv * Up[0]; HVp[0] = adv * Vp[0]; HWp[0] = adv * Wp[0];
  }
  const T ha = T(0.5) * alpha;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    fu[k] = T(0.5) * (Fm[k] + Fp[k]) - ha * (Up[k] - Um[k]);
    fv[k] = T(0.5) * (HVm[k] + HVp[k]) - ha * (Vp[k] - Vm[k]);
    fw[k] = T(0.5) * (HWm[k] + HWp[k]) - ha * (Wp[k] - Wm[k]);
  }
}

// One directional pass for the lane's cell at box index bidx.  Returns the
// Gauss-summed fluxes of the cell's low face (frame components) and the
// limited derivative along the pass normal.  All 32 lanes must call it.
// The direction D (0: x pass, 1: y pass on the transposed stencil) is a
// runtime value: both passes run this one copy of the code, which halves the
// kernel's instruction footprint (instruction fetch was its top stall).
template <typename T, int EQ, bool CHR, bool W64>
__device__ __forceinline__ void pass2d(const T* __restrict__ box, int bidx, int D, const WeightsT<T>& w,
                                       const WeightsT<double>& w64, bool lin, T ihn, T iht, T alpha, T g, T adv,
                                       T* Fu, T* Fv, T* Fw, T* vh) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
  const int SN = D == 0 ? 1 : kBP;
  const int ST = D == 0 ? kBP : 1;
  const int o9[9] = {-SN - ST, -ST, SN - ST, -SN, 0, SN, -SN + ST, ST, SN + ST};
  const int o4[4] = {-SN, SN, -ST, ST};
  T cu[NC][15];
  Eig<T> e{};
  const bool chr = CHR && !lin;
  if (chr) {
    T x0[4];
#pragma unroll
    for (int k = 0; k < NC; ++k) x0[k] = box[frame_field_rt<EQ, NC>(D, 0, k) * kFS + bidx];
    e = eig2<T>(x0[0], x0[1], x0[2], x0[3], g);
  }
  {
    T q[NC][17];
#pragma unroll
    for (int s = 0; s < 17; ++s) {
      T x[NC];
      const int dd = s < 9 ? 0 : (s < 13 ? 1 : 2);
      const int off = s < 9 ? o9[s] : o4[(s - 9) & 3];
#pragma unroll
      for (int k = 0; k < NC; ++k) x[k] = box[frame_field_rt<EQ, NC>(D, dd, k) * kFS + bidx + off];
      if constexpr (CHR) {
        if (chr) {
          T y[4];
          l2_apply<0>(e, x, y);
#pragma unroll
          for (int k = 0; k < NC; ++k) x[k] = y[k];
        }
      }
#pragma unroll
      for (int k = 0; k < NC; ++k) q[k][s] = x[k];
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if constexpr (W64) recon2_w64(q[k], w, w64, lin, cu[k]);
      else recon2<T>(q[k], w, lin, cu[k]);
    }
  }
  if constexpr (CHR) {
    // R applied to the 15 coefficient vectors of the reconstructed
    // characteristic polynomials gives the physical polynomial: every point
    // value, derivative and v-hat below is then a physical quantity.
    if (chr) {
#pragma unroll
      for (int l = 0; l < 15; ++l) {
        T x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = cu[k][l];
        r2_apply<0>(e, x, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) cu[k][l] = y[k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) { Fu[k] = T(0); Fv[k] = T(0); Fw[k] = T(0); vh[k] = T(0); }
  const T sig[3] = {T(5.0 / 18.0), T(8.0 / 18.0), T(5.0 / 18.0)};
  FacePts<T> fr[NC], fl[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    face_points<T>(cu[k], T(1), fr[k]);
    face_points<T>(cu[k], T(-1), fl[k]);
  }
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    T UR[NC], VR[NC], WR[NC], UL[NC], VL[NC], WL[NC];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      T u[NC], un[NC], ut[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const FacePts<T>& fp = side == 0 ? fr[k] : fl[k];
        u[k] = fp.u[mu]; un[k] = fp.un[mu]; ut[k] = fp.ut[mu];
      }
      T* Uo = side == 0 ? UR : UL;
      T* Vo = side == 0 ? VR : VL;
      T* Wo = side == 0 ? WR : WL;
#pragma unroll
      for (int k = 0; k < NC; ++k) { Uo[k] = u[k]; Vo[k] = un[k]; Wo[k] = ut[k]; }
#pragma unroll
      for (int k = 0; k < NC; ++k) { Vo[k] *= ihn; Wo[k] *= iht; }
    }
    // left neighbour's right-face state at this Gauss point
    T Um[NC], Vm[NC], Wm[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Um[k] = __shfl_up_sync(HW_FULL_MASK, UR[k], 1);
      Vm[k] = __shfl_up_sync(HW_FULL_MASK, VR[k], 1);
      Wm[k] = __shfl_up_sync(HW_FULL_MASK, WR[k], 1);
    }
    T fu[NC], fv[NC], fw[NC];
    lf_point<T, NC, EQ>(Um, Vm, Wm, UL, VL, WL, alpha, g, adv, fu, fv, fw);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Fu[k] += sig[mu] * fu[k];
      Fv[k] += sig[mu] * fv[k];
      Fw[k] += sig[mu] * fw[k];
      vh[k] += sig[mu] * (UR[k] - UL[k]);
    }
  }
}

// Per-tile quantities: kernel-wide for one grid, the tile's instance in a
// batch (instance-relative state pointers, grid ratios, stage dt and alpha,
// the boundary time).
template <typename T>
struct TileCtx {
  const T* in;
  const T* base;
  T* out;
  T* hat;
  const unsigned char* smooth;
  T idx, idy, dyx, dxy, tdt, ax, ay;
  double t_bc;
};

// One 30 x 30 tile: halo box fill (ghosts resolved on the way in), x pass,
// y pass and the RK stage update; the stage-3 spectral radius is folded
// into radx / rady.
template <typename T, int EQ, bool CHR, bool W64>
__device__ __forceinline__ void tile2d(const Stage2Args& a, const Grid2& G, int i0, int j0, const TileCtx<T>& c,
                                       T* box, T* stash, const WeightsT<T>& wx, const WeightsT<double>& wx64,
                                       bool lin_all, T g, T advx_t, T advy_t, double& radx, double& rady) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
  constexpr int NF = 3 * NC;
  const long long plane = a.plane;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  __syncthreads();
  const T* __restrict__ in = c.in;
  const T* base = c.base;
  T* out = c.out;
  T* __restrict__ hat = c.hat;
  const unsigned char* __restrict__ smooth = c.smooth;
  const T idx = c.idx, idy = c.idy, dyx = c.dyx, dxy = c.dxy, tdt = c.tdt;
  const bool inner = i0 >= 2 && j0 >= 2 && i0 + kBox - 2 <= G.nx && j0 + kBox - 2 <= G.ny;
  if (a.stage >= 2) {
    // The y pass's stage update reads base and hat at the tile's cells:
    // start pulling those rows into L2 now (3 points cover every 128-byte
    // line of a 30-cell row in either precision).
    for (int e = threadIdx.x; e < 3 * NC * kT2 * 3; e += blockDim.x) {
      const int pl = e / (kT2 * 3), rem = e - pl * (kT2 * 3);
      const int rr = rem / 3, pt = rem - rr * 3;
      const int j = min(j0 + rr, G.ny - 1), i = min(i0 + (pt == 0 ? 0 : (pt == 1 ? 15 : kT2 - 1)), G.nx - 1);
      const T* src = pl < NC ? base + pl * plane : hat + (pl - NC) * plane;
      prefetch_l2(src + (long long)j * G.nx + i);
    }
  }
  if (inner) {
    // whole box in flight at once; ghost-free, so a plain copy: a warp per
    // box row (34 cells: lanes 0-31, then lanes 0-1 for the last two)
    const T* src0 = in + (long long)(j0 - 2) * G.nx + (i0 - 2);
    for (int row = warp; row < NF * kBox; row += nwarps) {
      const int f = row / kBox, rr = row - f * kBox;
      const T* srow = src0 + f * plane + (long long)rr * G.nx;
      T* drow = box + f * kFS + rr * kBP;
      cp_async_elem(drow + lane, srow + lane);
      if (lane < kBox - 32) cp_async_elem(drow + 32 + lane, srow + 32 + lane);
    }
    cp_async_wait_all();
  } else {
    for (int e = threadIdx.x; e < NF * kBox * kBox; e += blockDim.x) {
      const int f = e / (kBox * kBox), rem = e - f * (kBox * kBox);
      const int rr = rem / kBox, cc = rem - rr * kBox;
      const int i = min(max(i0 - 2 + cc, -2), G.nx + 1), j = min(max(j0 - 2 + rr, -2), G.ny + 1);
      T v;
      if (i >= 0 && i < G.nx && j >= 0 && j < G.ny) v = in[f * plane + (long long)j * G.nx + i];
      else v = load_ghost2<T, EQ, NC>(in, plane, G, f, i, j, c.t_bc);
      box[f * kFS + rr * kBP + cc] = v;
    }
  }
  __syncthreads();

  // ---- x pass (D = 0): one row per warp iteration, lane l <-> cell i0-1+l;
  // ---- y pass (D = 1) on the transposed box: one column per iteration.
#pragma unroll 1
  for (int D = 0; D < 2; ++D) {
    if (D == 1) __syncthreads();  // the x pass's stash is complete
    const int lines = D == 0 ? G.ny - j0 : G.nx - i0;
    for (int r = warp; r < kT2; r += nwarps) {
      if (r >= lines) break;
      // learned indicator: a warp whose 32 cells are all smooth takes p0
      bool lin = lin_all;
      if (smooth != nullptr && !lin) {
        const int ii = D == 0 ? min(max(i0 - 1 + lane, 0), G.nx - 1) : i0 + r;
        const int jj = D == 0 ? j0 + r : min(max(j0 - 1 + lane, 0), G.ny - 1);
        lin = __all_sync(HW_FULL_MASK, smooth[(long long)jj * G.nx + ii] != 0);
      }
      const int bidx = D == 0 ? (r + 2) * kBP + lane + 1 : (lane + 1) * kBP + r + 2;
      // the pass's weights by value (S2 <-> S4 in the transposed frame)
      WeightsT<T> wp = wx;
      wp.g[2] = D == 0 ? wx.g[2] : wx.g[4];
      wp.g[4] = D == 0 ? wx.g[4] : wx.g[2];
      WeightsT<double> wp64 = wx64;
      if constexpr (W64) {
        wp64.g[2] = D == 0 ? wx64.g[2] : wx64.g[4];
        wp64.g[4] = D == 0 ? wx64.g[4] : wx64.g[2];
      }
      T Fu[NC], Fv[NC], Fw[NC], vh[NC];
      pass2d<T, EQ, CHR, W64>(box, bidx, D, wp, wp64, lin, D == 0 ? idx : idy, D == 0 ? idy : idx,
                              D == 0 ? c.ax : c.ay, g, D == 0 ? advx_t : advy_t, Fu, Fv, Fw, vh);
      T Gu[NC], Gv[NC], Gw[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        Gu[k] = __shfl_down_sync(HW_FULL_MASK, Fu[k], 1);
        Gv[k] = __shfl_down_sync(HW_FULL_MASK, Fv[k], 1);
        Gw[k] = __shfl_down_sync(HW_FULL_MASK, Fw[k], 1);
      }
      if (D == 0) {
        if (lane >= 1 && lane <= kT2 && i0 - 1 + lane < G.nx) {
          const int sidx = stash_at<T>(r, lane - 1);
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            stash[(0 * NC + k) * kSS + sidx] = -(Gu[k] - Fu[k]) * idx;
            stash[(1 * NC + k) * kSS + sidx] = -(Gv[k] - Fv[k]);
            stash[(2 * NC + k) * kSS + sidx] = -(Gw[k] - Fw[k]) * dyx;
            stash[(3 * NC + k) * kSS + sidx] = vh[k];
          }
        }
        continue;
      }
      const int cc = r, i = i0 + cc;
      const int j = j0 - 1 + lane;
      if (lane >= 1 && lane <= kT2 && j < G.ny) {
        const int sidx = stash_at<T>(lane - 1, cc);
        const long long p = (long long)j * G.nx + i;
        T nu[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const int kk = frame_comp<1, EQ>(k);
          const T Lu = stash[(0 * NC + k) * kSS + sidx] - (Gu[kk] - Fu[kk]) * idy;
          const T Lv = stash[(1 * NC + k) * kSS + sidx] - (Gw[kk] - Fw[kk]) * dxy;
          const T Lw = stash[(2 * NC + k) * kSS + sidx] - (Gv[kk] - Fv[kk]);
          const T vx = stash[(3 * NC + k) * kSS + sidx];
          const T wyv = vh[kk];
          const long long iu = k * plane + p, iv = (NC + k) * plane + p, iw = (2 * NC + k) * plane + p;
          const long long hv = k * plane + p, hw_ = (NC + k) * plane + p;
          if (a.stage == 0) {
            out[iu] = Lu; out[iv] = Lv; out[iw] = Lw;
            hat[hv] = vx; hat[hw_] = wyv;
          } else {
            const T ub = box[k * kFS + (lane + 1) * kBP + cc + 2];
            const T su = ub + tdt * Lu, sv = vx + tdt * Lv, sw = wyv + tdt * Lw;
            if (a.stage == 1) {
              out[iu] = su; out[iv] = sv; out[iw] = sw;
              hat[hv] = vx; hat[hw_] = wyv;
            } else if (a.stage == 2) {
              out[iu] = T(0.75) * base[iu] + T(0.25) * su;
              out[iv] = T(0.75) * hat[hv] + T(0.25) * sv;
              out[iw] = T(0.75) * hat[hw_] + T(0.25) * sw;
            } else {
              nu[k] = base[iu] * T(1.0 / 3.0) + T(2.0 / 3.0) * su;
              out[iv] = hat[hv] * T(1.0 / 3.0) + T(2.0 / 3.0) * sv;
              out[iw] = hat[hw_] * T(1.0 / 3.0) + T(2.0 / 3.0) * sw;
              out[iu] = nu[k];
            }
          }
        }
        if (a.stage == 3) {
          if constexpr (EQ == HWENO_EQ_EULER) {
            const T m2 = nu[1] * nu[1] + nu[2] * nu[2];
            const double rx = euler_radius<T>(nu[0], nu[1], m2, nu[3], g);
            const double ry = euler_radius<T>(nu[0], nu[2], m2, nu[3], g);
            radx = (unsigned long long)__double_as_longlong(rx) > (unsigned long long)__double_as_longlong(radx) ? rx : radx;
            rady = (unsigned long long)__double_as_longlong(ry) > (unsigned long long)__double_as_longlong(rady) ? ry : rady;
          } else if constexpr (EQ == HWENO_EQ_BURGERS) {
            const double rr = fabs((double)nu[0]);
            radx = (unsigned long long)__double_as_longlong(rr) > (unsigned long long)__double_as_longlong(radx) ? rr : radx;
            rady = radx;
          } else {
            radx = fabs(a.adv_x);
            rady = fabs(a.adv_y);
          }
        }
      }
    }
  }
}

// FAST: the paper's configuration (moment indicator, beta + eps) fixed at
// compile time, so no code of the variants is predicated into the hot path
// (4% fewer FP64-pipe instructions in the mixed kernel than with the
// run-time switches).  BATCH: the tiles of many 2D instances of uneven sizes
// (a tile table; per-instance descriptors and control blocks).
template <typename T, int EQ, bool CHR, bool W64, bool FAST, bool BATCH>
__global__ void __launch_bounds__(kThreads2, sizeof(T) == 4 ? 2 : 1) k_stage2d(const Stage2Args a) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
  constexpr int NF = 3 * NC;
  extern __shared__ __align__(16) unsigned char hw_smem[];
  T* box = reinterpret_cast<T*>(hw_smem);
  T* stash = box + NF * kFS;
  WeightsT<T> wx = make_weights<T>(a.wp);
  WeightsT<double> wx64 = make_weights<double>(a.wp);
  if constexpr (FAST) {
    wx.pow2 = 0;
    wx.typical = 0;
    wx64.pow2 = 0;
    wx64.typical = 0;
  }
  const bool lin_all = a.wp.linear != 0;
  // scalars in T; the FP32 kernels take the host-rounded FP32 copies (a
  // conversion the compiler re-did at each use would run on the FP64 pipe)
  T g, advx_t, advy_t;
  if constexpr (sizeof(T) == 4) {
    g = a.f32.gamma_gas; advx_t = a.f32.adv_x; advy_t = a.f32.adv_y;
  } else {
    g = a.gamma_gas; advx_t = a.adv_x; advy_t = a.adv_y;
  }
  const int lane = threadIdx.x & 31;
  double radx = 0.0, rady = 0.0;
  TileCtx<T> c;
  c.smooth = a.smooth;

  if constexpr (!BATCH) {
    const Grid2& G = a.grid;
    if (a.stage != 0 && a.ctl->done) return;
    // time of the stage for time-dependent boundaries: t^n, t^n + dt, t^n + dt/2
    c.t_bc = a.stage <= 1 ? a.ctl->t : a.ctl->t + (a.stage == 2 ? 1.0 : 0.5) * a.ctl->dt;
    c.in = static_cast<const T*>(a.in);
    c.base = static_cast<const T*>(a.base);  // aliases out at stage 3
    c.out = static_cast<T*>(a.out);
    c.hat = static_cast<T*>(a.hat);
    if constexpr (sizeof(T) == 4) {
      c.idx = a.f32.idx; c.idy = a.f32.idy; c.dyx = a.f32.dyx; c.dxy = a.f32.dxy;
      if (a.stage == 0) {
        c.tdt = T(0); c.ax = a.f32.ax_op; c.ay = a.f32.ay_op;
      } else {
        c.tdt = a.ctl->dtf; c.ax = a.ctl->axf; c.ay = a.ctl->ayf;
      }
    } else {
      c.idx = 1.0 / G.dx; c.idy = 1.0 / G.dy; c.dyx = G.dy / G.dx; c.dxy = G.dx / G.dy;
      if (a.stage == 0) {
        c.tdt = T(0); c.ax = a.ax_op; c.ay = a.ay_op;
      } else {
        c.tdt = a.ctl->dt; c.ax = a.ctl->ax; c.ay = a.ctl->ay;
      }
    }
    const int tiles_x = (G.nx + kT2 - 1) / kT2;
    const int ntiles = tiles_x * ((G.ny + kT2 - 1) / kT2);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int i0 = (tile % tiles_x) * kT2, j0 = (tile / tiles_x) * kT2;
      tile2d<T, EQ, CHR, W64>(a, G, i0, j0, c, box, stash, wx, wx64, lin_all, g, advx_t, advy_t, radx, rady);
    }
    if (a.stage == 3) {
      radx = warp_max(radx);
      rady = warp_max(rady);
      if (lane == 0) {
        atomic_max_nonneg(&a.ctl->amax_x, radx);
        atomic_max_nonneg(&a.ctl->amax_y, rady);
      }
    }
  } else {
    for (long long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      const Tile2 tl = a.tiles[tile];
      const Inst2& I = a.inst[tl.inst];
      Ctl* ctl = a.ctl + tl.inst;
      if (a.stage != 0 && ctl->done) continue;  // the same for the whole CTA
      c.t_bc = a.stage <= 1 ? ctl->t : ctl->t + (a.stage == 2 ? 1.0 : 0.5) * ctl->dt;
      c.in = static_cast<const T*>(a.in) + I.off;
      c.base = static_cast<const T*>(a.base) + I.off;
      c.out = static_cast<T*>(a.out) + I.off;
      c.hat = static_cast<T*>(a.hat) + I.off;
      if constexpr (sizeof(T) == 4) {
        c.idx = I.idxf; c.idy = I.idyf; c.dyx = I.dyxf; c.dxy = I.dxyf;
        if (a.stage == 0) {
          c.tdt = T(0); c.ax = (T)a.alpha_op[2 * tl.inst]; c.ay = (T)a.alpha_op[2 * tl.inst + 1];
        } else {
          c.tdt = ctl->dtf; c.ax = ctl->axf; c.ay = ctl->ayf;
        }
      } else {
        c.idx = I.idx; c.idy = I.idy; c.dyx = I.dyx; c.dxy = I.dxy;
        if (a.stage == 0) {
          c.tdt = T(0); c.ax = a.alpha_op[2 * tl.inst]; c.ay = a.alpha_op[2 * tl.inst + 1];
        } else {
          c.tdt = ctl->dt; c.ax = ctl->ax; c.ay = ctl->ay;
        }
      }
      tile2d<T, EQ, CHR, W64>(a, I.grid, tl.i0, tl.j0, c, box, stash, wx, wx64, lin_all, g, advx_t, advy_t, radx,
                              rady);
      if (a.stage == 3) {  // this tile's instance
        radx = warp_max(radx);
        rady = warp_max(rady);
        if (lane == 0) {
          atomic_max_nonneg(&ctl->amax_x, radx);
          atomic_max_nonneg(&ctl->amax_y, rady);
        }
        radx = 0.0;
        rady = 0.0;
      }
    }
  }
}

template <typename T, int EQ>
__global__ void __launch_bounds__(256) k_alpha2d(const T* __restrict__ U, long long count, long long plane,
                                                 double gamma_gas, double adv_x, double adv_y, Ctl* ctl) {
  double rx = 0.0, ry = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < count;
       c += (long long)gridDim.x * blockDim.x) {
    double a, b;
    if constexpr (EQ == HWENO_EQ_EULER) {
      const T r = U[c], mx = U[plane + c], my = U[2 * plane + c], E = U[3 * plane + c];
      const T m2 = mx * mx + my * my;
      a = euler_radius<T>(r, mx, m2, E, (T)gamma_gas);
      b = euler_radius<T>(r, my, m2, E, (T)gamma_gas);
    } else if constexpr (EQ == HWENO_EQ_BURGERS) {
      a = b = fabs((double)U[c]);
    } else {
      a = fabs(adv_x);
      b = fabs(adv_y);
    }
    rx = (unsigned long long)__double_as_longlong(a) > (unsigned long long)__double_as_longlong(rx) ? a : rx;
    ry = (unsigned long long)__double_as_longlong(b) > (unsigned long long)__double_as_longlong(ry) ? b : ry;
  }
  rx = warp_max(rx);
  ry = warp_max(ry);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&ctl->amax_x, rx);
    atomic_max_nonneg(&ctl->amax_y, ry);
  }
}

template <typename T, int EQ, bool CHR, bool W64, bool FAST, bool BATCH>
struct Launch2 {
  static int per_sm;  // resident CTAs per SM, 0 until prepared
  static cudaError_t prepare() {
    if (per_sm > 0) return cudaSuccess;
    constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
    constexpr size_t smem = smem_bytes2<T, NC>();
    cudaError_t e = cudaFuncSetAttribute(k_stage2d<T, EQ, CHR, W64, FAST, BATCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage2d<T, EQ, CHR, W64, FAST, BATCH>, kThreads2,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    per_sm = n;
    return cudaSuccess;
  }
  static cudaError_t go(const Stage2Args& a, int num_sms, cudaStream_t st, const LaunchShape& sh) {
    constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
    constexpr size_t smem = smem_bytes2<T, NC>();
    if (per_sm == 0) {
      cudaError_t e = prepare();
      if (e != cudaSuccess) return e;
    }
    const long long tiles =
        BATCH ? a.ntiles : (long long)((a.grid.nx + kT2 - 1) / kT2) * ((a.grid.ny + kT2 - 1) / kT2);
    if (tiles < 1) return cudaSuccess;
    long long blocks = sh.persistent2d ? (long long)num_sms * per_sm : tiles;
    if (blocks > tiles) blocks = tiles;
    k_stage2d<T, EQ, CHR, W64, FAST, BATCH><<<(unsigned)blocks, kThreads2, smem, st>>>(a);
    return cudaGetLastError();
  }
};
template <typename T, int EQ, bool CHR, bool W64, bool FAST, bool BATCH>
int Launch2<T, EQ, CHR, W64, FAST, BATCH>::per_sm = 0;

// The compile-time fast form exists for the characteristic-wise Euler
// kernels (the workloads' path); every other combination runs the
// run-time switches.
inline bool fast_form(const WeightParams& wp) { return wp.pow2 == 0 && wp.typical == 0; }

template <typename T, int EQ, bool CHR, bool W64 = false>
static cudaError_t go2(const Stage2Args& a, int num_sms, cudaStream_t st, const LaunchShape& sh) {
  if (a.batched) return Launch2<T, EQ, CHR, W64, false, true>::go(a, num_sms, st, sh);
  if constexpr (EQ == HWENO_EQ_EULER && CHR) {
    if (fast_form(a.wp)) return Launch2<T, EQ, CHR, W64, true, false>::go(a, num_sms, st, sh);
  }
  return Launch2<T, EQ, CHR, W64, false, false>::go(a, num_sms, st, sh);
}

template <typename T, bool W64, bool BATCH>
static cudaError_t prep2(int equation, bool chr, bool fast) {
  if (equation == HWENO_EQ_EULER) {
    if (chr)
      return fast && !BATCH ? Launch2<T, HWENO_EQ_EULER, true, W64, true, false>::prepare()
                            : Launch2<T, HWENO_EQ_EULER, true, W64, false, BATCH>::prepare();
    return Launch2<T, HWENO_EQ_EULER, false, W64, false, BATCH>::prepare();
  }
  if (equation == HWENO_EQ_BURGERS) return Launch2<T, HWENO_EQ_BURGERS, false, W64, false, BATCH>::prepare();
  return Launch2<T, HWENO_EQ_ADVECTION, false, W64, false, BATCH>::prepare();
}

cudaError_t prepare_stage2d(int precision, int equation, int charwise, const WeightParams& wp, bool batched) {
  const bool chr = equation == HWENO_EQ_EULER && charwise;
  const bool fast = fast_form(wp);
  // the linear-weight path of a characteristic solver runs the same kernel
  if (batched) {
    if (precision == HWENO_FP64) return prep2<double, false, true>(equation, chr, fast);
    if (precision == HWENO_FP32_IND64) return prep2<float, true, true>(equation, chr, fast);
    return prep2<float, false, true>(equation, chr, fast);
  }
  if (precision == HWENO_FP64) return prep2<double, false, false>(equation, chr, fast);
  if (precision == HWENO_FP32_IND64) return prep2<float, true, false>(equation, chr, fast);
  return prep2<float, false, false>(equation, chr, fast);
}

cudaError_t launch_stage2d(int precision, int equation, int charwise, const Stage2Args& a, int num_sms,
                           cudaStream_t st, const LaunchShape& sh) {
  const bool chr = equation == HWENO_EQ_EULER && charwise;
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) return chr ? go2<double, HWENO_EQ_EULER, true>(a, num_sms, st, sh)
                                               : go2<double, HWENO_EQ_EULER, false>(a, num_sms, st, sh);
    if (equation == HWENO_EQ_BURGERS) return go2<double, HWENO_EQ_BURGERS, false>(a, num_sms, st, sh);
    return go2<double, HWENO_EQ_ADVECTION, false>(a, num_sms, st, sh);
  }
  if (precision == HWENO_FP32_IND64) {
    if (equation == HWENO_EQ_EULER) return chr ? go2<float, HWENO_EQ_EULER, true, true>(a, num_sms, st, sh)
                                               : go2<float, HWENO_EQ_EULER, false, true>(a, num_sms, st, sh);
    if (equation == HWENO_EQ_BURGERS) return go2<float, HWENO_EQ_BURGERS, false, true>(a, num_sms, st, sh);
    return go2<float, HWENO_EQ_ADVECTION, false, true>(a, num_sms, st, sh);
  }
  if (equation == HWENO_EQ_EULER) return chr ? go2<float, HWENO_EQ_EULER, true>(a, num_sms, st, sh)
                                             : go2<float, HWENO_EQ_EULER, false>(a, num_sms, st, sh);
  if (equation == HWENO_EQ_BURGERS) return go2<float, HWENO_EQ_BURGERS, false>(a, num_sms, st, sh);
  return go2<float, HWENO_EQ_ADVECTION, false>(a, num_sms, st, sh);
}

cudaError_t launch_alpha2d(int precision, int equation, const void* U, long long count, long long plane,
                           double gamma_gas, double adv_x, double adv_y, Ctl* ctl, int num_sms, cudaStream_t st) {
  long long blocks = (count + 255) / 256;
  if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
  if (blocks < 1) blocks = 1;
#define HW_A2(T, EQ) k_alpha2d<T, EQ><<<(unsigned)blocks, 256, 0, st>>>( \
    static_cast<const T*>(U), count, plane, gamma_gas, adv_x, adv_y, ctl)
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) HW_A2(double, HWENO_EQ_EULER);
    else if (equation == HWENO_EQ_BURGERS) HW_A2(double, HWENO_EQ_BURGERS);
    else HW_A2(double, HWENO_EQ_ADVECTION);
  } else {
    if (equation == HWENO_EQ_EULER) HW_A2(float, HWENO_EQ_EULER);
    else if (equation == HWENO_EQ_BURGERS) HW_A2(float, HWENO_EQ_BURGERS);
    else HW_A2(float, HWENO_EQ_ADVECTION);
  }
#undef HW_A2
  return cudaGetLastError();
}

}  // namespace hw
