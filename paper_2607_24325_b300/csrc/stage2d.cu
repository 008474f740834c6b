// stage2d.cu -- fused 2D HWENO stage kernel (Sec. 2.2 Steps 1-4, Remark 1).
//
// A CTA (8 warps) owns a 30 x 30 tile of interior cells.  It stages the
// 34 x 34 box (tile + 2-cell halo) of every field in shared memory, resolving
// ghost cells with the boundary map on the way in, then runs
//   y pass: warp per tile column, lanes along y, on the transposed box.
//           Transposing swaps the roles of x and y, of v-bar and w-bar, of
//           the two momentum components and of the stencils S2 and S4, so the
//           y physics is the x physics in the transposed frame and both
//           passes run one copy of the code.  Each lane reconstructs its cell
//           (characteristic-wise with the eigenvectors of its own average for
//           Euler), evaluates u and its two derivatives at the 3 Gauss points
//           of both faces, takes its left neighbour's right-face values by
//           shuffle and forms the Lax-Friedrichs fluxes of its LOW face (each
//           interface once; the high-face flux comes from lane+1).  The y part
//           of L and w-hat go to a shared-memory stash.
//   x pass: warp per tile row, lane l = cell i0-1+l, the same code on the
//           box; it adds the x part of L and applies the RK stage, with
//           coalesced global stores along x (stages 2-3 take u^n, v-hat^n and
//           w-hat^n of the row from shared memory, copied there by cp.async
//           while the row is reconstructed).
// Interface values, fluxes and L never go through HBM.
#include <cuda_runtime.h>

#include "hweno_device.cuh"
#include "hweno_stencil2d.cuh"
#include "kernels.h"

namespace hw {

static_assert(kT2 == kTile2, "host tile table and kernel tile size differ");

// The central part of the Lax-Friedrichs fluxes of the pass-frame x physics
// at one point, doubled: f(u-) + f(u+), f'(u-) v- + f'(u+) v+ (normal
// moment), f'(u-) w- + f'(u+) w+ (tangential moment).  The dissipative part
// -alpha (u+ - u-) is linear in the states, so its Gauss sum over a face is
// formed once from the face averages (pass2d).
template <typename T, int NC, int EQ>
__device__ __forceinline__ void lf_point(const T* Um, const T* Vm, const T* Wm, const T* Up, const T* Vp,
                                         const T* Wp, T g, T adv, T* fu, T* fv, T* fw) {
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
  // twice the central flux: the 1/2 is folded into the Gauss weights by the caller
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    fu[k] = Fm[k] + Fp[k];
    fv[k] = HVm[k] + HVp[k];
    fw[k] = HWm[k] + HWp[k];
  }
}

// Stencil value s of the cell at box index cell, in pass-frame components
// and projected on the characteristic fields of e when chr: s = 0..8 the
// 3 x 3 cell averages (row-major along the pass normal), 9..12 the moments
// along the pass normal and 13..16 those along the tangent of the four face
// neighbours (normal -, +, tangent -, +).
template <typename T, int NC, bool CHR>
__device__ __forceinline__ void stencil_at(const T* __restrict__ box, int cell, int D, int s, const Eig<T>& e,
                                           bool chr, T* x) {
  const int SN = D == 0 ? 1 : kBP;
  const int ST = D == 0 ? kBP : 1;
  const int o9[9] = {-SN - ST, -ST, SN - ST, -SN, 0, SN, -SN + ST, ST, SN + ST};
  const int o4[4] = {-SN, SN, -ST, ST};
  const int dd = s < 9 ? 0 : (s < 13 ? 1 : 2);
  const int off = s < 9 ? o9[s] : o4[(s - 9) & 3];
  // moment group along the pass normal (dd = 1) or tangent (dd = 2)
  const int grp = dd == 0 ? 0 : (D == 0 ? dd : 3 - dd);
  box_load<T, NC>(box, grp, cell + off, D, x);
  if constexpr (CHR) {
    if (chr) {
      T y[4];
      l2_apply<0>(e, x, y);
      // materialised: every reader sees the same rounded values
#pragma unroll
      for (int k = 0; k < NC; ++k) x[k] = opaque(y[k]);
    }
  }
}

// Position of the n-th (from 0) set bit of m; n < popc(m).
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  int pos = 0;
#pragma unroll
  for (int h = 16; h > 0; h >>= 1) {
    const int c = __popc(m & ((1u << h) - 1u));
    if (n >= c) {
      n -= c;
      m >>= h;
      pos += h;
    }
  }
  return pos;
}

// Mixed precision, a deferred warp row: the fields whose FP32 screen did
// not clear every lane (bit k of pend, warp-uniform; bit k of nqb: this
// lane's cell not cleared for field k).  Only the uncleared (lane, field)
// items need the FP64 indicator, so they are packed 32 to a call of
// indicator64 -- the FP64 pipe runs at 1/64 of the FP32 rate, and a warp
// instruction costs it the same with 1 or 32 lanes active.  Lane j of a
// call rebuilds item j's stencil from the box (the owner's cell and
// eigenvectors) and each owner collects its a_m by shuffle into a[k][m]
// (0 on cleared lanes: the screen shows 1 + a_m = 1 there).  Runs between
// rows; not inlined, which keeps its code out of the hot loop (fewer
// instruction-fetch stalls) and its registers off the common path.  The
// indicator's parameters (eps, the power, the form) come by value: a
// reference to a weight set would give the caller's set an address in
// local memory and keep all of it live through the row loop.
template <int NC, bool CHR>
static __device__ __noinline__ void pack64(const float* __restrict__ box, int bidx, int D, bool chr, float g,
                                       unsigned pend, unsigned nqb, double eps, int pow2, int typical,
                                       volatile float (*a)[5]) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int SL = D == 0 ? 1 : kBP;  // box step between neighbouring lanes' cells
  unsigned bal[NC];
  int pre[NC + 1];
  pre[0] = 0;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    bal[k] = ((pend >> k) & 1u) ? __ballot_sync(HW_FULL_MASK, (nqb >> k) & 1u) : 0u;
    pre[k + 1] = pre[k] + __popc(bal[k]);
#pragma unroll
    for (int m = 0; m < 5; ++m) a[k][m] = 0.0f;
  }
  const int n = pre[NC];
#pragma unroll 1
  for (int base = 0; base < n; base += 32) {
    // this lane's item (idle lanes repeat item base): field f, owner L
    const int j = base + lane < n ? base + lane : base;
    int f = 0, pf = 0;
    unsigned mk = bal[0];
#pragma unroll
    for (int k = 1; k < NC; ++k) {
      if (j >= pre[k]) {
        f = k;
        pf = pre[k];
        mk = bal[k];
      }
    }
    const int L = nth_set_bit(mk, j - pf);
    const int cell = bidx + (L - lane) * SL;
    Eig<float> eo{};
    if constexpr (CHR) {
      if (chr) {
        float x0[4];
        box_load<float, 4>(box, 0, cell, D, x0);
        eo = eig2<float>(x0[0], x0[1], x0[2], x0[3], g);
      }
    }
    Stencil17 st;
#pragma unroll
    for (int s = 0; s < 17; ++s) {
      float x[NC];
      stencil_at<float, NC, CHR>(box, cell, D, s, eo, chr, x);
      float v = x[0];
#pragma unroll
      for (int k = 1; k < NC; ++k) v = f == k ? x[k] : v;
      st.q[s] = v;
    }
    const Weights5 r5 = indicator64(st, eps, pow2, typical);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if ((pend >> k) & 1u) {
        const int src = pre[k] + __popc(bal[k] & below) - base;
        const bool mine = ((nqb >> k) & 1u) && src >= 0 && src < 32;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          const float v = __shfl_sync(HW_FULL_MASK, r5.a[m], src & 31);
          if (mine) a[k][m] = v;
        }
      }
    }
  }
}

// One directional pass for the lane's cell at box index bidx.  Returns the
// Gauss-summed fluxes of the cell's low face (frame components) and the
// limited derivative along the pass normal.  All 32 lanes must call it.
// The direction D (0: x pass, 1: y pass on the transposed stencil) is a
// runtime value: both passes run this one copy of the code, which halves the
// kernel's instruction footprint (instruction fetch was its top stall).
//
// Mixed precision (W64): with redo == 0 the FP32 screen runs per field; a
// row where it does not clear every lane of some field returns false at
// once with the fields in *pend and this lane's uncleared ones in *nqb (the
// caller redoes it after pack64).  With redo != 0 the fields in redo take
// their a_m from a64.
template <typename T, int EQ, bool CHR, bool W64>
__device__ __forceinline__ bool pass2d(const T* __restrict__ box, int bidx, int D, const WeightsT<T>& w,
                                       const WeightsT<double>& w64, bool lin, T ihn, T iht, T alpha, T g, T adv,
                                       T* Fu, T* Fv, T* Fw, T* vh, unsigned redo = 0u,
                                       const volatile float (*a64)[5] = nullptr, unsigned* pend = nullptr,
                                       unsigned* nqb = nullptr) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 4 : 1;
  T cu[NC][15];
  Eig<T> e{};
  const bool chr = CHR && !lin;
  if (chr) {
    T x0[4];
    box_load<T, 4>(box, 0, bidx, D, x0);
    e = eig2<T>(x0[0], x0[1], x0[2], x0[3], g);
  }
  {
    T q[NC][17];
#pragma unroll
    for (int s = 0; s < 17; ++s) {
      T x[NC];
      stencil_at<T, NC, CHR>(box, bidx, D, s, e, chr, x);
#pragma unroll
      for (int k = 0; k < NC; ++k) q[k][s] = x[k];
    }
    if constexpr (W64) {
      // FP32 coefficients and weights; a_m = 0 where the screen clears the
      // whole warp, from a64 in a redone row
      unsigned pe = 0u, nb = 0u;
      // the weights of a cleared field (every a_m = 0), once per row
      float r0, om0[5];
      {
        const float z[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        finish2(z, w, r0, om0);
      }
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        Coef2<float> kc;
        coef2<float, float, true, true>(q[k], kc);
        if (lin) {
#pragma unroll
          for (int l = 0; l < 15; ++l) cu[k][l] = kc.c[l];
          continue;
        }
        float r = r0, om[5];
#pragma unroll
        for (int m = 1; m < 5; ++m) om[m] = om0[m];
        if (redo == 0u) {
          const bool quiet = screen2(kc, w64, w);
          if (!__all_sync(HW_FULL_MASK, quiet)) {
            pe |= 1u << k;
            nb |= quiet ? 0u : 1u << k;
          }
        } else if ((redo >> k) & 1u) {
          float a[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) a[m] = a64[k][m];
          finish2(a, w, r, om);
        }
        combine2<float>(kc, r, om, w, cu[k]);
      }
      if (pe != 0u) {
        *pend = pe;
        *nqb = nb;
        return false;
      }
    } else if constexpr (sizeof(T) == 4 && NC == 4) {
      // FP32: Steps 1-3 of two fields per paired instruction
#pragma unroll
      for (int k = 0; k < NC; k += 2) recon2_x2(q[k], q[k + 1], w, lin, cu[k], cu[k + 1]);
    } else {
#pragma unroll
      for (int k = 0; k < NC; ++k) recon2<T>(q[k], w, lin, cu[k]);
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
  const T hsig[3] = {T(5.0 / 36.0), T(8.0 / 36.0), T(5.0 / 36.0)};  // Gauss weights with lf_point's 1/2
  FacePts<T> fr[NC], fl[NC];
  // The dissipation over the low face, -(alpha / 2) times the face average
  // of (u+ - u-) (the Gauss sum of the pointwise terms, exact for these
  // restrictions), starts the flux sums; v-hat is the face average of
  // u(right) - u(left) (Gauss weights summing to 1).
  const T ha = T(0.5) * alpha;
  if constexpr (sizeof(T) == 4 && NC == 4) {
    face_points_x2(cu[0], cu[1], fr[0], fr[1], fl[0], fl[1]);
    face_points_x2(cu[2], cu[3], fr[2], fr[3], fl[2], fl[3]);
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      face_points<T>(cu[k], T(1), fr[k]);
      face_points<T>(cu[k], T(-1), fl[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    Fu[k] = -ha * (fl[k].au - __shfl_up_sync(HW_FULL_MASK, fr[k].au, 1));
    Fv[k] = -ha * (fl[k].an - __shfl_up_sync(HW_FULL_MASK, fr[k].an, 1));
    Fw[k] = -ha * (fl[k].at - __shfl_up_sync(HW_FULL_MASK, fr[k].at, 1));
    vh[k] = fr[k].au - fl[k].au;
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
      // derivatives per unit xi, eta: the moment fluxes are linear in them,
      // so the 1/h scales are applied once to the Gauss sums below
#pragma unroll
      for (int k = 0; k < NC; ++k) { Uo[k] = u[k]; Vo[k] = un[k]; Wo[k] = ut[k]; }
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
    lf_point<T, NC, EQ>(Um, Vm, Wm, UL, VL, WL, g, adv, fu, fv, fw);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Fu[k] += hsig[mu] * fu[k];
      Fv[k] += hsig[mu] * fv[k];
      Fw[k] += hsig[mu] * fw[k];
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    Fv[k] *= ihn;
    Fw[k] *= iht;
  }
  return true;
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
  DeferList* dl = reinterpret_cast<DeferList*>(stash + 4 * NC * kSS);  // after the stash
  // Stages 2-3: the y pass folds w-hat into its w quantity, so the stash's
  // fourth quantity is free during the x pass and holds, per warp, the
  // current row's stage-update inputs (u^n, v-hat^n, w-hat^n of its cells),
  // copied by cp.async while the row is reconstructed.
  T* const stage_in = stash + 3 * NC * kSS;
  static_assert((threads2<T, W64>() / 32) * 3 * NC * 32 <= NC * kSS, "update staging exceeds the stash quantity");
  __syncthreads();
  if constexpr (W64) {
    if (threadIdx.x == 0) dl->n[0] = dl->n[1] = 0;  // published by the fill's barrier
  }
  const T* __restrict__ in = c.in;
  const T* base = c.base;
  T* out = c.out;
  T* __restrict__ hat = c.hat;
  const unsigned char* __restrict__ smooth = c.smooth;
  const T idx = c.idx, idy = c.idy, dyx = c.dyx, dxy = c.dxy, tdt = c.tdt;
  const bool inner = i0 >= 2 && j0 >= 2 && i0 + kBox - 2 <= G.nx && j0 + kBox - 2 <= G.ny;
  if (a.stage >= 2) {
    // The x pass's stage update reads base and hat at the tile's cells:
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
      const int d = f / NC, k = f - d * NC;
      const T* srow = src0 + f * plane + (long long)rr * G.nx;
      const int at = box_at<NC>(d, rr * kBP, k);
      T* drow = box + at;
      const bool row_ok = HW_IN(j0 - 2 + rr, G.ny, 6);
      if (row_ok && HW_IN(at + lane * NC, 3 * NC * kFS, 5) && HW_IN(i0 - 2 + lane, G.nx, 6))
        cp_async_elem(drow + lane * NC, srow + lane);
      if (lane < kBox - 32 && row_ok && HW_IN(at + (32 + lane) * NC, 3 * NC * kFS, 5) &&
          HW_IN(i0 + 30 + lane, G.nx, 6))
        cp_async_elem(drow + (32 + lane) * NC, srow + 32 + lane);
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
      const int at = box_at<NC>(f / NC, rr * kBP + cc, f % NC);
      if (HW_IN(at, 3 * NC * kFS, 7)) box[at] = v;
    }
  }
  __syncthreads();

  // ---- y pass first (D = 1, on the transposed box: one column per warp
  // iteration, lane l <-> cell j0-1+l), its share of L to the stash; then the
  // x pass (D = 0: one row per iteration, lane l <-> cell i0-1+l) and the
  // stage update, whose global loads and stores then run along x
  // (consecutive lanes, consecutive addresses: whole 128-byte lines).
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const int D = 1 - it;
    if (it == 1) __syncthreads();  // the y pass's stash is complete
    const int lines = D == 0 ? G.ny - j0 : G.nx - i0;
    // One warp row of the pass: reconstruction, fluxes, then the stash
    // (first pass) or the stage update (second pass).  False, with the
    // fields (*pend) and this lane's cells (*nqb) the screen did not clear,
    // when the mixed precision defers the row.
    volatile float a64[W64 ? NC : 1][5];
    auto row = [&](const int r, const unsigned redo, unsigned& pend, unsigned& nqb) -> bool {
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
      if constexpr (W64) {
        if (redo != 0u)
          pack64<NC, CHR>(box, bidx, D, CHR && !lin, g, redo & 0xfu, redo >> 4, wx64.eps, wx64.pow2,
                          wx64.typical, a64);
      }
      if (it == 1 && a.stage >= 2) {
        // this row's update inputs, in flight while the row is reconstructed
        // (a deferred row waits for its copies before it returns)
        const int i = i0 - 1 + lane, j = j0 + r;
        if (lane >= 1 && lane <= kT2 && i < G.nx && HW_IN(i, G.nx, 12) && HW_IN(j, G.ny, 12)) {
          const long long p = (long long)j * G.nx + i;
          T* sg = stage_in + warp * (3 * NC * 32) + lane;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            if (HW_IN(warp * (3 * NC * 32) + (2 * NC + k) * 32 + lane, NC * kSS, 12)) {
              cp_async_elem(sg + k * 32, base + k * plane + p);
              cp_async_elem(sg + (NC + k) * 32, hat + k * plane + p);
              cp_async_elem(sg + (2 * NC + k) * 32, hat + (NC + k) * plane + p);
            }
          }
        }
      }
      T Fu[NC], Fv[NC], Fw[NC], vh[NC];
      if (!pass2d<T, EQ, CHR, W64>(box, bidx, D, wp, wp64, lin, D == 0 ? idx : idy, D == 0 ? idy : idx,
                                   D == 0 ? c.ax : c.ay, g, D == 0 ? advx_t : advy_t, Fu, Fv, Fw, vh,
                                   redo & 0xfu, a64, &pend, &nqb)) {
        if (it == 1 && a.stage >= 2) cp_async_wait_all();  // the staging slot is free again
        return false;
      }
      // flux differences across the cell (high face, the next lane's low
      // face, minus low face): the fluxes themselves are dead from here on
      T dFu[NC], dFv[NC], dFw[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        dFu[k] = __shfl_down_sync(HW_FULL_MASK, Fu[k], 1) - Fu[k];
        dFv[k] = __shfl_down_sync(HW_FULL_MASK, Fv[k], 1) - Fv[k];
        dFw[k] = __shfl_down_sync(HW_FULL_MASK, Fw[k], 1) - Fw[k];
      }
      if (it == 0) {  // y pass: column r, lane l <-> tile row l - 1; physical components
        if (lane >= 1 && lane <= kT2 && j0 - 1 + lane < G.ny) {
          T su[NC], sv[NC], sw[NC], sh[NC];
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int kk = frame_comp<1, EQ>(k);
            su[k] = -dFu[kk] * idy;
            sv[k] = -dFw[kk] * dxy;
            sw[k] = -dFv[kk];
            sh[k] = vh[kk];
          }
          if (a.stage >= 2) {
            // the update's y part of w: w-hat + dt L^w_y (quantity 3 is then
            // the x pass's staging area)
#pragma unroll
            for (int k = 0; k < NC; ++k) sw[k] = sh[k] + tdt * sw[k];
          }
          stash_store<T, NC>(stash, 0, lane - 1, r, su);
          stash_store<T, NC>(stash, 1, lane - 1, r, sv);
          stash_store<T, NC>(stash, 2, lane - 1, r, sw);
          if (a.stage < 2) stash_store<T, NC>(stash, 3, lane - 1, r, sh);
        }
        return true;
      }
      // x pass: row r, lane l <-> tile column l - 1, and the stage update
      const int i = i0 - 1 + lane, j = j0 + r;
      if (lane >= 1 && lane <= kT2 && i < G.nx && HW_IN(i, G.nx, 9) && HW_IN(j, G.ny, 9)) {
        const long long p = (long long)j * G.nx + i;
        T yu[NC], yv[NC], yw[NC], yh[NC], ubox[NC];
        stash_load<T, NC>(stash, 0, r, lane - 1, yu);
        stash_load<T, NC>(stash, 1, r, lane - 1, yv);
        stash_load<T, NC>(stash, 2, r, lane - 1, yw);
        if (a.stage < 2) stash_load<T, NC>(stash, 3, r, lane - 1, yh);
        if (a.stage != 0) box_load<T, NC>(box, 0, (r + 2) * kBP + lane + 1, 0, ubox);
        T nu[NC];
        if (a.stage >= 2) {
          // u^n, v-hat^n, w-hat^n of this cell from the staging area (each
          // lane reads only what its own copies wrote)
          cp_async_wait_all();
          const T* sg = stage_in + warp * (3 * NC * 32) + lane;
          const T cA = a.stage == 2 ? T(0.75) : T(1.0 / 3.0), cB = a.stage == 2 ? T(0.25) : T(2.0 / 3.0);
          const T tdx = tdt * dyx;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const T un = sg[k * 32], vn = sg[(NC + k) * 32], wn = sg[(2 * NC + k) * 32];
            const T su = ubox[k] + tdt * (yu[k] - dFu[k] * idx);
            const T sv = vh[k] + tdt * (yv[k] - dFv[k]);
            const T sw = yw[k] - tdx * dFw[k];  // w-hat + dt (L^w_y + L^w_x)
            const long long iu = k * plane + p, iv = (NC + k) * plane + p, iw = (2 * NC + k) * plane + p;
            nu[k] = cA * un + cB * su;
            out[iu] = nu[k];
            out[iv] = cA * vn + cB * sv;
            out[iw] = cA * wn + cB * sw;
          }
        } else {
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const T Lu = yu[k] - dFu[k] * idx;
            const T Lv = yv[k] - dFv[k];
            const T Lw = yw[k] - dFw[k] * dyx;
            const T vx = vh[k];
            const T wyv = yh[k];
            const long long iu = k * plane + p, iv = (NC + k) * plane + p, iw = (2 * NC + k) * plane + p;
            const long long hv = k * plane + p, hw_ = (NC + k) * plane + p;
            if (a.stage == 0) {
              out[iu] = Lu; out[iv] = Lv; out[iw] = Lw;
              hat[hv] = vx; hat[hw_] = wyv;
            } else {
              out[iu] = ubox[k] + tdt * Lu; out[iv] = vx + tdt * Lv; out[iw] = wyv + tdt * Lw;
              hat[hv] = vx; hat[hw_] = wyv;
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
      return true;
    };
    // the warp's own rows r = warp + t nwarps; mixed precision: a row the
    // screen does not clear is listed, and once every warp has listed its
    // rows the list is shared out: each listed row gets its uncleared lanes
    // (from the listing warp's ballots, or by screening it again), its FP64
    // items packed, and is redone.  Two loops, so that the common one holds
    // none of the list's state.
    const int own = (min(kT2, lines) - warp + nwarps - 1) / nwarps;
#pragma unroll 1
    for (int t = 0; t < own; ++t) {
      const int r = warp + t * nwarps;
      unsigned pend = 0u, nqb = 0u;
      if (!row(r, 0u, pend, nqb)) {
        if constexpr (W64) {
          int slot = 0;
          if (lane == 0) {
            slot = atomicAdd(&dl->n[D], 1);
            if (HW_IN(slot, kT2 + 2, 10)) dl->row[slot] = (unsigned char)r;
          }
          slot = __shfl_sync(HW_FULL_MASK, slot, 0);
          if (slot < kDeferBal) {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
              const unsigned b = __ballot_sync(HW_FULL_MASK, (nqb >> k) & 1u);
              if (lane == 0) dl->bal[slot][k] = b;
            }
          }
        }
      }
    }
    if constexpr (W64) {
      __syncthreads();  // every warp's deferred rows are listed
      const int n_def = dl->n[D];
#pragma unroll 1
      for (int e = warp; e < n_def; e += nwarps) {
        const int r = HW_IN(e, kT2 + 2, 11) ? dl->row[e] : 0;
        unsigned redo = 0u;
        if (e < kDeferBal) {  // the listing warp's ballots
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const unsigned b = dl->bal[e][k];
            redo |= (b != 0u ? 1u : 0u) << k;
            redo |= ((b >> lane) & 1u) << (4 + k);
          }
        }
#pragma unroll 1
        for (;;) {  // at most twice: screened again (no ballots kept), then redone
          unsigned pend = 0u, nqb = 0u;
          if (row(r, redo, pend, nqb)) break;
          redo = pend | (nqb << 4);
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
//
// Tiles: with as many CTAs as tiles each CTA takes its own; a persistent
// grid (fewer CTAs than tiles) starts every CTA on the tile of its index
// and then hands out the rest in natural order from a global counter, so a
// CTA whose tiles were cheap (no FP64 indicator work) takes more of them and
// the SMs finish together.
__device__ __forceinline__ int next_tile(unsigned* sched) {
  __shared__ int s_next;
  __syncthreads();  // every thread has read the previous s_next
  if (threadIdx.x == 0) s_next = (int)(atomicAdd(&sched[0], 1u) + gridDim.x);
  __syncthreads();
  return s_next;
}

// After a CTA's last tile: the last CTA of the launch zeroes the scheduler
// for the next launch (every other CTA has drawn its final tile by then).
__device__ __forceinline__ void sched_finish(unsigned* sched) {
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned d = atomicAdd(&sched[1], 1u);
    if (d == gridDim.x - 1) {
      sched[0] = 0u;
      sched[1] = 0u;
      __threadfence();
    }
  }
}

template <typename T, int EQ, bool CHR, bool W64, bool FAST, bool BATCH>
__global__ void __launch_bounds__(threads2<T, W64>(), sizeof(T) == 4 ? 2 : 1) k_stage2d(const Stage2Args a) {
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
    const bool dyn = a.sched != nullptr && (long long)gridDim.x < ntiles;
    for (int tile = blockIdx.x; tile < ntiles; tile = dyn ? next_tile(a.sched) : tile + (int)gridDim.x) {
      const int i0 = (tile % tiles_x) * kT2, j0 = (tile / tiles_x) * kT2;
      tile2d<T, EQ, CHR, W64>(a, G, i0, j0, c, box, stash, wx, wx64, lin_all, g, advx_t, advy_t, radx, rady);
    }
    if (dyn) sched_finish(a.sched);
    if (a.stage == 3) {
      radx = warp_max(radx);
      rady = warp_max(rady);
      if (lane == 0) {
        atomic_max_nonneg(&a.ctl->amax_x, radx);
        atomic_max_nonneg(&a.ctl->amax_y, rady);
      }
    }
  } else {
    const bool dyn = a.sched != nullptr && (long long)gridDim.x < a.ntiles;
    for (long long tile = blockIdx.x; tile < a.ntiles; tile = dyn ? next_tile(a.sched) : tile + gridDim.x) {
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
    if (dyn) sched_finish(a.sched);
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage2d<T, EQ, CHR, W64, FAST, BATCH>, threads2<T, W64>(),
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
    k_stage2d<T, EQ, CHR, W64, FAST, BATCH><<<(unsigned)blocks, threads2<T, W64>(), smem, st>>>(a);
    return cudaGetLastError();
  }
};
template <typename T, int EQ, bool CHR, bool W64, bool FAST, bool BATCH>
int Launch2<T, EQ, CHR, W64, FAST, BATCH>::per_sm = 0;

// The compile-time fast form exists for the characteristic-wise Euler
// kernels (the workloads' path), single grids and batches; every other
// combination runs the run-time switches.
inline bool fast_form(const WeightParams& wp) { return wp.pow2 == 0 && wp.typical == 0; }

template <typename T, int EQ, bool CHR, bool W64 = false>
static cudaError_t go2(const Stage2Args& a, int num_sms, cudaStream_t st, const LaunchShape& sh) {
  if constexpr (EQ == HWENO_EQ_EULER && CHR) {
    if (fast_form(a.wp)) {
      if (a.batched) return Launch2<T, EQ, CHR, W64, true, true>::go(a, num_sms, st, sh);
      return Launch2<T, EQ, CHR, W64, true, false>::go(a, num_sms, st, sh);
    }
  }
  if (a.batched) return Launch2<T, EQ, CHR, W64, false, true>::go(a, num_sms, st, sh);
  return Launch2<T, EQ, CHR, W64, false, false>::go(a, num_sms, st, sh);
}

template <typename T, bool W64, bool BATCH>
static cudaError_t prep2(int equation, bool chr, bool fast) {
  if (equation == HWENO_EQ_EULER) {
    if (chr)
      return fast ? Launch2<T, HWENO_EQ_EULER, true, W64, true, BATCH>::prepare()
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

HW_CHECK_READER(hweno_check_stage2d)
