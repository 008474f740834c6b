// stage1d.cu -- fused 1D HWENO stage kernel (Sec. 2.1 Steps 1-4, Remark 1).
//
// One warp owns a task of 30 consecutive interior cells of one instance:
// lane l holds cell s-1+l (lanes 0 and 31 are the ring cells whose
// reconstructions the two boundary interfaces need).  Each lane
//   1. loads u-bar, v-bar of its cell (ghost cells resolved by the boundary
//      map, nothing padded in memory) and gets its neighbours by shuffles,
//   2. reconstructs its cell (characteristic-wise for Euler),
//   3. evaluates the Lax-Friedrichs flux at its LEFT face from the left
//      neighbour's right-face state (shuffle); the right-face flux comes from
//      lane+1, so every interface flux is computed once,
//   4. applies the RK stage (or writes L in operator mode) and, at stage 3,
//      folds the new state's spectral radius into the instance's alpha.
// No interface value, flux or L ever goes through HBM.
#include <cuda_runtime.h>

#include "hweno_device.cuh"
#include "kernels.h"

namespace hw {

template <typename T, int NC, int EQ>
__device__ __forceinline__ void load_cell1(const T* __restrict__ in, long long total, const Inst1& I,
                                           int c, T* ub, T* vb) {
  const GhostMap g = ghost_map(c, I.n, I.bc_lo, I.bc_hi);
  if (g.fixed) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      ub[k] = (T)(g.side ? I.st_hi[k] : I.st_lo[k]);
      vb[k] = T(0);
    }
    return;
  }
  const long long p = I.off + g.src;
  if (!(HW_IN(g.src, I.n, 21) && HW_IN(p, total, 21))) {
#pragma unroll
    for (int k = 0; k < NC; ++k) ub[k] = vb[k] = T(0);
    return;
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T u = in[k * total + p];
    T v = in[(NC + k) * total + p];
    if (g.flip) {
      if (mirror_negates(EQ, 0, k, 0)) u = -u;
      if (mirror_negates(EQ, 1, k, 0)) v = -v;
    }
    ub[k] = u;
    vb[k] = v;
  }
}

// Global Lax-Friedrichs flux of Sec. 2.1 for (u, v).
template <typename T, int NC, int EQ>
__device__ __forceinline__ void lf_flux1(const T* um, const T* up, const T* vm, const T* vp, T alpha,
                                         T g, T adv, T* fu, T* fv) {
  T Fm[NC], Fp[NC], Hm[NC], Hp[NC];
  if constexpr (EQ == HWENO_EQ_EULER) {
    euler1_flux(um, vm, g, Fm, Hm);
    euler1_flux(up, vp, g, Fp, Hp);
  } else if constexpr (EQ == HWENO_EQ_BURGERS) {
    Fm[0] = T(0.5) * um[0] * um[0]; Hm[0] = um[0] * vm[0];
    Fp[0] = T(0.5) * up[0] * up[0]; Hp[0] = up[0] * vp[0];
  } else {
    Fm[0] = adv * um[0]; Hm[0] = adv * vm[0];
    Fp[0] = adv * up[0]; Hp[0] = adv * vp[0];
  }
  const T ha = T(0.5) * alpha;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    fu[k] = T(0.5) * (Fm[k] + Fp[k]) - ha * (up[k] - um[k]);
    fv[k] = T(0.5) * (Hm[k] + Hp[k]) - ha * (vp[k] - vm[k]);
  }
}

template <typename T, int EQ, bool CHR, bool W64>
__global__ void __launch_bounds__(256) k_stage1d(const Stage1Args a) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 3 : 1;
  const T* __restrict__ in = static_cast<const T*>(a.in);
  const T* base = static_cast<const T*>(a.base);  // aliases out at stage 3
  T* out = static_cast<T*>(a.out);
  T* __restrict__ hat = static_cast<T*>(a.hat);
  const WeightsT<T> w = make_weights<T>(a.wp);
  const WeightsT<double> w64 = make_weights<double>(a.wp);
  // FP32 kernels take host-rounded FP32 scalars (a conversion re-done at
  // each use would issue on the FP64 pipe)
  const T g = sizeof(T) == 4 ? (T)a.gammaf : (T)a.gamma_gas;
  const T adv = sizeof(T) == 4 ? (T)a.advf : (T)a.adv;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const long long total = a.total;
  // stage 3: this lane's running spectral-radius maximum over the warp's
  // tasks of instance rinst, folded into the instance's alpha when the
  // instance changes and after the last task (one atomic per warp and
  // instance instead of one per task: a single-instance grid otherwise
  // serialises hundreds of thousands of atomics on one address)
  double rmax = 0.0;
  int rinst = -1;

  for (int task = blockIdx.x * wpb + (threadIdx.x >> 5); task < a.ntasks; task += gridDim.x * wpb) {
    const int2 tk = a.tasks[task];
    const Inst1 I = a.inst[tk.x];
    T tdt = T(0), alpha;
    if (a.stage == 0) {
      alpha = (T)a.alpha_op[tk.x];
    } else {
      const Ctl* c = a.ctl + tk.x;
      if (c->done) continue;  // warp-uniform
      if constexpr (sizeof(T) == 4) {
        tdt = c->dtf;
        alpha = c->axf;
      } else {
        tdt = c->dt;
        alpha = c->ax;
      }
    }
    const int cell = tk.y - 1 + lane;
    const int lc = min(cell, I.n + 1);
    T ub[NC], vb[NC], um[NC], up[NC], vm[NC], vp[NC];
    load_cell1<T, NC, EQ>(in, total, I, lc, ub, vb);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      um[k] = __shfl_up_sync(HW_FULL_MASK, ub[k], 1);
      vm[k] = __shfl_up_sync(HW_FULL_MASK, vb[k], 1);
      up[k] = __shfl_down_sync(HW_FULL_MASK, ub[k], 1);
      vp[k] = __shfl_down_sync(HW_FULL_MASK, vb[k], 1);
    }
    if (lane == 0) load_cell1<T, NC, EQ>(in, total, I, lc - 1, um, vm);
    if (lane == 31) load_cell1<T, NC, EQ>(in, total, I, min(cell + 1, I.n + 1), up, vp);
    const bool interior = lane >= 1 && lane <= kTile1 && cell < I.n && HW_IN(cell, I.n, 22) &&
                          HW_IN(I.off + cell, total, 22);
    // stages 2-3: the update's u^n and v-hat^n, loaded now so that their
    // latency overlaps the reconstruction (at stage 3 base aliases out; this
    // cell is written only by this lane, after these loads)
    T bn[NC], hn[NC];
    if (a.stage >= 2 && interior) {
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        bn[k] = base[k * total + I.off + cell];
        hn[k] = hat[k * total + I.off + cell];
      }
    }

    T dx, idx;
    if constexpr (sizeof(T) == 4) {
      dx = I.dxf;
      idx = I.idxf;
    } else {
      dx = I.dx;
      idx = I.idx;
    }
    T uL[NC], uR[NC], dL[NC], dR[NC], vh[NC];
    if constexpr (CHR) {
      const Eig<T> e = eig1<T>(ub[0], ub[1], ub[2], g);
      T Wm[3], W0[3], Wp[3], Zm[3], Zp[3];
      l1_apply(e, um, Wm); l1_apply(e, ub, W0); l1_apply(e, up, Wp);
      l1_apply(e, vm, Zm); l1_apply(e, vp, Zp);
      T oL[3], oR[3], odL[3], odR[3], ov[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const Rec1<T> r = recon1<T, W64>(Wm[k], W0[k], Wp[k], Zm[k], Zp[k], dx, idx, w, &w64);
        oL[k] = r.uL; oR[k] = r.uR; odL[k] = r.dL; odR[k] = r.dR; ov[k] = r.vh;
      }
      r1_apply(e, oL, uL); r1_apply(e, oR, uR); r1_apply(e, odL, dL); r1_apply(e, odR, dR);
      r1_apply(e, ov, vh);
    } else {
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const Rec1<T> r = recon1<T, W64>(um[k], ub[k], up[k], vm[k], vp[k], dx, idx, w, &w64);
        uL[k] = r.uL; uR[k] = r.uR; dL[k] = r.dL; dR[k] = r.dR; vh[k] = r.vh;
      }
    }
    // flux at the left face x_{cell-1/2}: (u-, v-) from lane-1's right face
    T Um[NC], Vm[NC], Fu[NC], Fv[NC], Gu[NC], Gv[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Um[k] = __shfl_up_sync(HW_FULL_MASK, uR[k], 1);
      Vm[k] = __shfl_up_sync(HW_FULL_MASK, dR[k], 1);
    }
    lf_flux1<T, NC, EQ>(Um, uL, Vm, dL, alpha, g, adv, Fu, Fv);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Gu[k] = __shfl_down_sync(HW_FULL_MASK, Fu[k], 1);
      Gv[k] = __shfl_down_sync(HW_FULL_MASK, Fv[k], 1);
    }
    double rad = 0.0;
    if (interior) {
      const long long p = I.off + cell;
      T nu[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const T Lu = -(Gu[k] - Fu[k]) * idx;
        const T Lv = -(Gv[k] - Fv[k]) * idx;
        const long long iu = k * total + p, iv = (NC + k) * total + p;
        if (a.stage == 0) {
          out[iu] = Lu;
          out[iv] = Lv;
          hat[k * total + p] = vh[k];
        } else if (a.stage == 1) {
          out[iu] = ub[k] + tdt * Lu;
          out[iv] = vh[k] + tdt * Lv;
          hat[k * total + p] = vh[k];
        } else if (a.stage == 2) {
          out[iu] = T(0.75) * bn[k] + T(0.25) * (ub[k] + tdt * Lu);
          out[iv] = T(0.75) * hn[k] + T(0.25) * (vh[k] + tdt * Lv);
        } else {
          nu[k] = bn[k] * T(1.0 / 3.0) + T(2.0 / 3.0) * (ub[k] + tdt * Lu);
          out[iv] = hn[k] * T(1.0 / 3.0) + T(2.0 / 3.0) * (vh[k] + tdt * Lv);
          out[iu] = nu[k];
        }
      }
      if (a.stage == 3) {
        if constexpr (EQ == HWENO_EQ_EULER) rad = euler_radius<T>(nu[0], nu[1], nu[1] * nu[1], nu[2], g);
        else if constexpr (EQ == HWENO_EQ_BURGERS) rad = fabs((double)nu[0]);
        else rad = fabs((double)adv);
      }
    }
    if (a.stage == 3) {
      if (tk.x != rinst) {  // warp-uniform
        if (rinst >= 0) {
          const double m = warp_max(rmax);
          if (lane == 0) atomic_max_nonneg(&a.ctl[rinst].amax_x, m);
        }
        rinst = tk.x;
        rmax = 0.0;
      }
      // NaN bit patterns exceed every finite one, as in the atomic
      rmax = (unsigned long long)__double_as_longlong(rad) > (unsigned long long)__double_as_longlong(rmax) ? rad : rmax;
    }
  }
  if (a.stage == 3 && rinst >= 0) {
    const double m = warp_max(rmax);
    if (lane == 0) atomic_max_nonneg(&a.ctl[rinst].amax_x, m);
  }
}

// Max spectral radius of a state over all instances (alpha of the first step).
template <typename T, int EQ>
__global__ void __launch_bounds__(128) k_alpha1d(const T* __restrict__ U, long long total,
                                                 const Inst1* inst, const int2* tasks, int ntasks,
                                                 double gamma_gas, double adv, Ctl* ctl) {
  constexpr int NC = EQ == HWENO_EQ_EULER ? 3 : 1;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int task = blockIdx.x * wpb + (threadIdx.x >> 5); task < ntasks; task += gridDim.x * wpb) {
    const int2 tk = tasks[task];
    const int n = inst[tk.x].n;
    const long long off = inst[tk.x].off;
    const int cell = tk.y + lane;
    double rad = 0.0;
    if (lane < kTile1 && cell < n) {
      T s[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) s[k] = U[k * total + off + cell];
      if constexpr (EQ == HWENO_EQ_EULER) rad = euler_radius<T>(s[0], s[1], s[1] * s[1], s[2], (T)gamma_gas);
      else if constexpr (EQ == HWENO_EQ_BURGERS) rad = fabs((double)s[0]);
      else rad = fabs(adv);
    }
    rad = warp_max(rad);
    if (lane == 0) atomic_max_nonneg(&ctl[tk.x].amax_x, rad);
  }
}

template <typename T, int EQ, bool CHR, bool W64 = false>
static cudaError_t go1(const Stage1Args& a, int num_sms, cudaStream_t st, const LaunchShape& sh) {
  const int warps = sh.warps1d < 1 ? 1 : (sh.warps1d > 8 ? 8 : sh.warps1d);
  long long blocks = (a.ntasks + warps - 1) / warps;
  const long long cap = (long long)num_sms * (sh.blocks_per_sm1d < 1 ? 1 : sh.blocks_per_sm1d);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_stage1d<T, EQ, CHR, W64><<<(unsigned)blocks, 32 * warps, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stage1d(int precision, int equation, int charwise, const Stage1Args& a,
                           int num_sms, cudaStream_t st, const LaunchShape& sh) {
  if (a.ntasks <= 0) return cudaSuccess;
  const bool chr = equation == HWENO_EQ_EULER && charwise;
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) return chr ? go1<double, HWENO_EQ_EULER, true>(a, num_sms, st, sh)
                                               : go1<double, HWENO_EQ_EULER, false>(a, num_sms, st, sh);
    if (equation == HWENO_EQ_BURGERS) return go1<double, HWENO_EQ_BURGERS, false>(a, num_sms, st, sh);
    return go1<double, HWENO_EQ_ADVECTION, false>(a, num_sms, st, sh);
  }
  if (precision == HWENO_FP32_IND64) {
    if (equation == HWENO_EQ_EULER) return chr ? go1<float, HWENO_EQ_EULER, true, true>(a, num_sms, st, sh)
                                               : go1<float, HWENO_EQ_EULER, false, true>(a, num_sms, st, sh);
    if (equation == HWENO_EQ_BURGERS) return go1<float, HWENO_EQ_BURGERS, false, true>(a, num_sms, st, sh);
    return go1<float, HWENO_EQ_ADVECTION, false, true>(a, num_sms, st, sh);
  }
  if (equation == HWENO_EQ_EULER) return chr ? go1<float, HWENO_EQ_EULER, true>(a, num_sms, st, sh)
                                             : go1<float, HWENO_EQ_EULER, false>(a, num_sms, st, sh);
  if (equation == HWENO_EQ_BURGERS) return go1<float, HWENO_EQ_BURGERS, false>(a, num_sms, st, sh);
  return go1<float, HWENO_EQ_ADVECTION, false>(a, num_sms, st, sh);
}

cudaError_t launch_alpha1d(int precision, int equation, const void* U, long long total,
                           const Inst1* inst, const int2* tasks, int ntasks, double gamma_gas,
                           double adv, Ctl* ctl, int num_sms, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  long long blocks = (ntasks + 3) / 4;
  if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
#define HW_A1(T, EQ) k_alpha1d<T, EQ><<<(unsigned)blocks, 128, 0, st>>>( \
    static_cast<const T*>(U), total, inst, tasks, ntasks, gamma_gas, adv, ctl)
  if (precision == HWENO_FP64) {
    if (equation == HWENO_EQ_EULER) HW_A1(double, HWENO_EQ_EULER);
    else if (equation == HWENO_EQ_BURGERS) HW_A1(double, HWENO_EQ_BURGERS);
    else HW_A1(double, HWENO_EQ_ADVECTION);
  } else {
    if (equation == HWENO_EQ_EULER) HW_A1(float, HWENO_EQ_EULER);
    else if (equation == HWENO_EQ_BURGERS) HW_A1(float, HWENO_EQ_BURGERS);
    else HW_A1(float, HWENO_EQ_ADVECTION);
  }
#undef HW_A1
  return cudaGetLastError();
}

}  // namespace hw

HW_CHECK_READER(hweno_check_stage1d)
