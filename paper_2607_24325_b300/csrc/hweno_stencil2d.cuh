// hweno_stencil2d.cuh -- the 2D stencil pieces shared by the stage kernel
// and the learned-indicator kernels: tile constants, the pass frame (x pass,
// or the y pass on the transposed stencil), the ghost-cell value map,
// Appendix A's 2D reconstruction with nonlinear weights (Sec. 2.2 Steps 1-3)
// and the face Gauss-point evaluation.
#pragma once

#include "hweno_device.cuh"

namespace hw {

constexpr int kT2 = 30;           // interior tile edge
constexpr int kBox = 34;          // tile + 2 halo cells per side
constexpr int kBP = 35;           // box pitch (odd: conflict-free column walks)
constexpr int kFS = kBox * kBP;   // box field stride
constexpr int kSP = 30;           // stash pitch
constexpr int kSS = kT2 * kSP;    // stash field stride
constexpr int kThreads2 = 256;

template <int NC>
constexpr int stash_fields() { return 4 * NC; }   // L_u, L_v, L_w, v-hat

template <typename T, int NC>
constexpr size_t smem_bytes2() {
  return sizeof(T) * (size_t)(3 * NC * kFS + stash_fields<NC>() * kSS);
}

// Component of the pass frame holding physical component k (an involution).
template <int D, int EQ>
__device__ constexpr int frame_comp(int k) {
  return (EQ == HWENO_EQ_EULER && D == 1 && (k == 1 || k == 2)) ? 3 - k : k;
}
// Box field of frame field (d, k): d = 0 average, 1 moment along the pass
// normal, 2 moment along the tangent.
template <int D, int EQ, int NC>
__device__ constexpr int frame_field(int d, int k) {
  return (d == 0 ? 0 : (D == 0 ? d : 3 - d)) * NC + frame_comp<D, EQ>(k);
}

// Value of field f at cell (i, j), ghost cells resolved as "x sides for the
// interior rows, then y sides for every column".
template <typename T, int EQ, int NC>
__device__ __forceinline__ T load_ghost2(const T* __restrict__ in, long long plane, const Grid2& G,
                                         int f, int i, int j) {
  const int d = f / NC, k = f % NC;
  const GhostMap gx = ghost_map(i, G.nx, G.bc[0], G.bc[1]);
  const GhostMap gy = ghost_map(j, G.ny, G.bc[2], G.bc[3]);
  if (gy.fixed) return d == 0 ? (T)G.st[2 + gy.side][k] : T(0);
  T v;
  if (gx.fixed) {
    v = d == 0 ? (T)G.st[gx.side][k] : T(0);
  } else {
    v = in[f * plane + (long long)gy.src * G.nx + gx.src];
    if (gx.flip && mirror_negates(EQ, d, k, 0)) v = -v;
  }
  if (gy.flip && mirror_negates(EQ, d, k, 1)) v = -v;
  return v;
}

// Appendix A (2D) in the pass frame: the quartic p0 (15 coefficients in the
// basis {1, xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta, xi eta^2, eta^3,
// xi^4, xi^3 eta, xi^2 eta^2, xi eta^3, eta^4}) from q1..q17, and the slopes
// of the linear p1..p4 = q5 + sx xi + sy eta on S1 {W,S}, S2 {E,S}, S3 {E,N},
// S4 {W,N}.  TC is the arithmetic type, TQ the type of the inputs.
template <typename TC>
struct Coef2 {
  TC c[15];
  TC dW, dE, dS, dN, q5;
};

// The coefficients are evaluated on the centre-shifted averages
// d_k = q_k - q5 (k = 1..9, k != 5): p0 reproduces constants, so c_0 gains
// q5 and c_1..c_14 do not see it.  Every q5 term of the appendix's formulas
// cancels exactly, and the rounding of each coefficient scales with the
// local variation instead of with |q5| (in FP32 the difference of two nearby
// averages is exact).  With C0 = false, c_0 is not formed (the smoothness
// indicator does not use it).
template <typename TC, typename TQ, bool C0 = true>
__device__ __forceinline__ void coef2(const TQ* qin, Coef2<TC>& o) {
  const TC q5 = to_tc<TC>(qin[4]);
  const TC d1 = to_tc<TC>(qin[0]) - q5, d2 = to_tc<TC>(qin[1]) - q5, d3 = to_tc<TC>(qin[2]) - q5;
  const TC d4 = to_tc<TC>(qin[3]) - q5, d6 = to_tc<TC>(qin[5]) - q5;
  const TC d7 = to_tc<TC>(qin[6]) - q5, d8 = to_tc<TC>(qin[7]) - q5, d9 = to_tc<TC>(qin[8]) - q5;
  const TC q10 = to_tc<TC>(qin[9]), q11 = to_tc<TC>(qin[10]), q12 = to_tc<TC>(qin[11]);
  const TC q13 = to_tc<TC>(qin[12]), q14 = to_tc<TC>(qin[13]), q15 = to_tc<TC>(qin[14]);
  const TC q16 = to_tc<TC>(qin[15]), q17 = to_tc<TC>(qin[16]);
  const TC s13 = d1 + d3, s79 = d7 + d9, m13 = d1 - d3, m79 = d7 - d9;
  const TC sc = s13 + s79;        // corner sum minus 4 q5
  const TC cx = m13 - m79;
  const TC ax = m13 + m79;
  const TC ay = s13 - s79;
  const TC ex = d4 + d6, ey = d2 + d8;   // minus 2 q5 each
  const TC dxe = d6 - d4, dye = d8 - d2;
  const TC s1011 = q10 + q11, m1110 = q11 - q10, s1213 = q12 + q13, m1213 = q12 - q13;
  const TC s1415 = q14 + q15, m1415 = q14 - q15, s1617 = q16 + q17, m1716 = q17 - q16;
  TC* c = o.c;
  if constexpr (C0) {
    c[0] = q5 + (TC(5) * sc - TC(292) * (ex + ey) + TC(81) * (m1110 + m1716)) * TC(1.0 / 2880.0);
  } else {
    c[0] = TC(0);
  }
  c[1] = (TC(2) * ax + TC(19) * dxe - TC(6) * s1011 + TC(3) * s1213) * TC(1.0 / 24.0);
  c[2] = (TC(2) * ay + TC(19) * dye + TC(3) * s1415 - TC(6) * s1617) * TC(1.0 / 24.0);
  c[3] = (TC(2) * ey + TC(62) * ex - sc - TC(18) * m1110) * TC(1.0 / 48.0);
  c[4] = TC(-0.375) * cx - TC(0.625) * (m1213 + m1415);
  c[5] = (TC(2) * ex + TC(62) * ey - sc - TC(18) * m1716) * TC(1.0 / 48.0);
  c[6] = (TC(4) * (s1011 - dxe) - ax - TC(2) * s1213) * TC(0.05);
  c[7] = TC(-0.25) * ay - TC(0.5) * dye;
  c[8] = TC(-0.25) * ax - TC(0.5) * dxe;
  c[9] = (TC(4) * (s1617 - dye) - ay - TC(2) * s1415) * TC(0.05);
  c[10] = TC(0.25) * m1110 - TC(0.5) * ex;
  c[11] = TC(0.25) * cx + TC(0.5) * m1213;
  c[12] = TC(0.25) * sc - TC(0.5) * (ex + ey);
  c[13] = TC(0.25) * cx + TC(0.5) * m1415;
  c[14] = TC(0.25) * m1716 - TC(0.5) * ey;
  o.dW = -d4;
  o.dE = d6;
  o.dS = -d2;
  o.dN = d8;
  o.q5 = q5;
}

// Steps 2-3 (Sec. 2.2): beta = sum (m! n! c)^2, tau = 1/4 sum |beta_0 - beta_m|,
// the nonlinear weights; r = omega_0 / gamma_0 and om[1..4].  With DEV the
// largest |omega_m / gamma_m - 1| is folded into *dev.
template <typename TW, bool DEV>
__device__ __forceinline__ void weights2(const Coef2<TW>& k, const WeightsT<TW>& w, TW& r, TW* om, TW* dev) {
  const TW* c = k.c;
  const TW b1 = k.dW * k.dW + k.dS * k.dS, b2 = k.dE * k.dE + k.dS * k.dS;
  const TW b3 = k.dE * k.dE + k.dN * k.dN, b4 = k.dW * k.dW + k.dN * k.dN;
  const TW b0 = c[1] * c[1] + c[2] * c[2] + c[4] * c[4] +
                TW(4) * (c[3] * c[3] + c[5] * c[5] + c[7] * c[7] + c[8] * c[8]) +
                TW(36) * (c[6] * c[6] + c[9] * c[9] + c[11] * c[11] + c[13] * c[13]) +
                TW(576) * (c[10] * c[10] + c[14] * c[14]) + TW(16) * c[12] * c[12];
  const TW tau = TW(0.25) * ((fabs_t(b0 - b1) + fabs_t(b0 - b2)) + (fabs_t(b0 - b3) + fabs_t(b0 - b4)));
  const TW beta[5] = {b0, b1, b2, b3, b4};
  nl_weights<TW, 4>(beta, tau, w, r, om);
  if constexpr (DEV) {
    TW d = fabs_t(r - TW(1));
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      const TW x = fabs_t(om[m] / w.g[m] - TW(1));
      d = x > d ? x : d;
    }
    *dev = d > *dev ? d : *dev;
  }
}

// Eq. (hweno-reconstruction-2D): cu = r (p0 - sum gamma_m p_m) + sum omega_m p_m.
template <typename T>
__device__ __forceinline__ void combine2(const Coef2<T>& k, T r, const T* om, const WeightsT<T>& w, T* cu) {
  const T* c = k.c;
  const T gs = (w.g[1] + w.g[2]) + (w.g[3] + w.g[4]);
  const T ws = (om[1] + om[2]) + (om[3] + om[4]);
  cu[0] = r * (c[0] - gs * k.q5) + ws * k.q5;
  cu[1] = r * (c[1] - ((w.g[1] + w.g[4]) * k.dW + (w.g[2] + w.g[3]) * k.dE)) +
          ((om[1] + om[4]) * k.dW + (om[2] + om[3]) * k.dE);
  cu[2] = r * (c[2] - ((w.g[1] + w.g[2]) * k.dS + (w.g[3] + w.g[4]) * k.dN)) +
          ((om[1] + om[2]) * k.dS + (om[3] + om[4]) * k.dN);
#pragma unroll
  for (int l = 3; l < 15; ++l) cu[l] = r * c[l];
}

// Steps 1-3 for one field: the combined polynomial cu (lin: p0 itself).
template <typename T, bool DEV = false>
__device__ __forceinline__ void recon2(const T* q, const WeightsT<T>& w, bool lin, T* cu, T* dev = nullptr) {
  Coef2<T> k;
  coef2<T, T>(q, k);
  if (lin) {
#pragma unroll
    for (int l = 0; l < 15; ++l) cu[l] = k.c[l];
    return;
  }
  T r, om[5];
  weights2<T, DEV>(k, w, r, om, dev);
  combine2<T>(k, r, om, w, cu);
}

// Mixed precision: FP32 inputs and polynomial, but the coefficients that
// enter the smoothness indicators, the indicators and the nonlinear weights
// in FP64 (their epsilon-sensitive differences are where FP32 cancels).  The
// inputs are widened exactly on the integer ALU and the weights narrowed
// (round to nearest) the same way: the hardware conversions would issue on
// the FP64 pipe, which bounds this path.
__device__ __forceinline__ void recon2_w64(const float* q, const WeightsT<float>& w, const WeightsT<double>& w64,
                                           bool lin, float* cu) {
  Coef2<float> k;
  coef2<float, float>(q, k);
  if (lin) {  // linear weights: no indicator, plain FP32 coefficients
#pragma unroll
    for (int l = 0; l < 15; ++l) cu[l] = k.c[l];
    return;
  }
  Coef2<double> k64;
  coef2<double, float, false>(q, k64);
  double r64, om64[5];
  weights2<double, false>(k64, w64, r64, om64, nullptr);
  float om[5];
#pragma unroll
  for (int m = 1; m <= 4; ++m) om[m] = narrow_f64(om64[m]);
  combine2<float>(k, narrow_f64(r64), om, w, cu);
}

// Values at the three Gauss points of the face xi = +-1/2 (sgn = +1 / -1)
// of the pass frame: u, d/dxi u, d/deta u.
template <typename T>
struct FacePts { T u[3], un[3], ut[3]; };

template <typename T>
__device__ __forceinline__ void face_points(const T* c, T sgn, FacePts<T>& o) {
  const T s = T(0.38729833462074168852), s2 = T(0.15), s3 = s * T(0.15), s4 = T(0.0225);
  const T A0 = (c[0] + T(0.25) * c[3] + T(0.0625) * c[10]) + sgn * (T(0.5) * c[1] + T(0.125) * c[6]);
  const T A1 = (c[2] + T(0.25) * c[7]) + sgn * (T(0.5) * c[4] + T(0.125) * c[11]);
  const T A2 = (c[5] + T(0.25) * c[12]) + sgn * (T(0.5) * c[8]);
  const T A3 = c[9] + sgn * (T(0.5) * c[13]);
  const T A4 = c[14];
  const T B0 = (c[1] + T(0.75) * c[6]) + sgn * (c[3] + T(0.5) * c[10]);
  const T B1 = (c[4] + T(0.75) * c[11]) + sgn * c[7];
  const T B2 = c[8] + sgn * c[12];
  const T B3 = c[13];
  const T ue = A0 + A2 * s2 + A4 * s4, uo = A1 * s + A3 * s3;
  const T ne = B0 + B2 * s2, no = B1 * s + B3 * s3;
  const T te = A1 + T(3) * A3 * s2, to = T(2) * A2 * s + T(4) * A4 * s3;
  o.u[0] = ue - uo; o.u[1] = A0; o.u[2] = ue + uo;
  o.un[0] = ne - no; o.un[1] = B0; o.un[2] = ne + no;
  o.ut[0] = te - to; o.ut[1] = A1; o.ut[2] = te + to;
}

}  // namespace hw
