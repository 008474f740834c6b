// hweno_stencil2d.cuh -- the 2D stencil pieces shared by the stage kernel
// and the learned-indicator kernels: tile constants, the pass frame (x pass,
// or the y pass on the transposed stencil), the ghost-cell value map,
// Appendix A's 2D reconstruction with nonlinear weights (Sec. 2.2 Steps 1-3)
// and the face Gauss-point evaluation.
#pragma once

#include <string.h>

#include "hweno_device.cuh"

namespace hw {

constexpr int kT2 = 30;           // interior tile edge
constexpr int kBox = 34;          // tile + 2 halo cells per side
constexpr int kBP = 35;           // box pitch (odd: conflict-free column walks)
constexpr int kFS = kBox * kBP;   // box group stride, in cells
constexpr int kSP = 30;           // stash pitch, in cells
constexpr int kSS = kT2 * kSP + 8;  // stash quantity stride, in cells (room for the row skew)
// Threads per stage-kernel CTA (two CTAs per SM in FP32, one in FP64).
// The tile's 30 rows per pass are dealt to the warps in turn.  Measured on
// the mixed and FP32 kernels: 8 warps at 128 registers beat 6 or 5 warps
// at 168 registers and 10 warps at 96 (fewer warps hide less latency; 96
// registers spill).
template <typename T, bool W64>
__host__ __device__ constexpr int threads2() { return 256; }

// The NC components of one cell as vector loads / stores (16-byte accesses
// for the four Euler components; the address must be 16-byte aligned).
template <typename T, int NC>
__device__ __forceinline__ void vec_load(const T* __restrict__ p, T* x) {
  if constexpr (NC == 4) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(p);
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
      const double2 a = *reinterpret_cast<const double2*>(p);
      const double2 b = *reinterpret_cast<const double2*>(p + 2);
      x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
  } else {
    x[0] = p[0];
  }
}
template <typename T, int NC>
__device__ __forceinline__ void vec_store(T* p, const T* x) {
  if constexpr (NC == 4) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
      *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
      *reinterpret_cast<double2*>(p + 2) = make_double2(x[2], x[3]);
    }
  } else {
    p[0] = x[0];
  }
}

// The stash holds the y pass's results per tile cell: quantity q (L_u,
// L_v, L_w, w-hat), then the cell, then its NC components.  The y pass
// writes columns (lane = row, stride kSP cells); the x pass reads rows
// (consecutive lanes, consecutive cells).  A stride of 30 cells alone puts
// lanes 4 rows apart (16-byte cells: 8 to a 128-byte line) or 16 rows apart
// (4-byte cells) on one bank; skewing the rows by one cell every 4 (16 and
// 32-byte cells), 8 (8-byte) or 16 (4-byte) rows spreads a column walk
// over the banks.
template <typename T, int NC>
__device__ __forceinline__ int stash_at(int q, int r, int c) {
  constexpr int sh = NC == 4 ? 2 : (sizeof(T) == 8 ? 3 : 4);
  return (q * kSS + r * kSP + c + (r >> sh)) * NC;
}

template <int NC>
constexpr int stash_fields() { return 4 * NC; }   // L_u, L_v, L_w, v-hat

// Mixed precision: the rows of a pass that the FP32 screen did not clear,
// listed by the warps that met them and shared out among all warps.  The
// first kDeferBal entries also keep, per field, the ballot of the lanes the
// screen did not clear (0 for a cleared field), so the warp that redoes the
// row needs no second screen; later entries are screened again (shared
// memory is nearly full at two CTAs per SM).
constexpr int kDeferBal = 24;
struct DeferList {
  int n[2];                  // per pass
  unsigned char row[kT2 + 2];
  unsigned bal[kDeferBal][4];
};

template <typename T, int NC>
constexpr size_t smem_bytes2() {
  return sizeof(T) * (size_t)(3 * NC * kFS + stash_fields<NC>() * kSS) + sizeof(DeferList);
}

// The halo box is cell-interleaved: group d (0 averages, 1 x-moments,
// 2 y-moments), then the cell (row * kBP + column), then the NC components,
// so the four Euler components of one stencil value are one 16-byte (FP32)
// or two 16-byte (FP64) shared-memory loads.
template <int NC>
__device__ __forceinline__ int box_at(int d, int cell, int k) {
  return (d * kFS + cell) * NC + k;
}

// The NC components of group d at a box cell, in pass-frame order (the y
// pass swaps the momentum components).
template <typename T, int NC>
__device__ __forceinline__ void box_load(const T* __restrict__ box, int d, int cell, int D, T* x) {
  const int at = box_at<NC>(d, cell, 0);
  if (!HW_IN(at, 3 * NC * kFS - NC + 1, 1)) {
#pragma unroll
    for (int k = 0; k < NC; ++k) x[k] = T(0);
    return;
  }
  vec_load<T, NC>(box + at, x);
  if constexpr (NC == 4) {
    const T a = x[1], b = x[2];
    x[1] = D == 0 ? a : b;
    x[2] = D == 0 ? b : a;
  }
}

// The NC components of tile cell (r, c) of stash quantity q.
template <typename T, int NC>
__device__ __forceinline__ void stash_store(T* stash, int q, int r, int c, const T* x) {
  const int at = stash_at<T, NC>(q, r, c);
  if (HW_IN(at, 4 * NC * kSS - NC + 1, 2)) vec_store<T, NC>(stash + at, x);
}
template <typename T, int NC>
__device__ __forceinline__ void stash_load(const T* stash, int q, int r, int c, T* x) {
  const int at = stash_at<T, NC>(q, r, c);
  if (HW_IN(at, 4 * NC * kSS - NC + 1, 3)) {
    vec_load<T, NC>(stash + at, x);
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) x[k] = T(0);
  }
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

// The rule a side applies to one ghost cell: split walls and moving shocks
// resolve, by the coordinate of the ghost cell's centre along the side
// (lo + (idx + 1/2) h) and the stage time t, into an inflow state or a
// mirror.  The coordinate is formed only for those two kinds of side.
struct SideRule {
  int bc;
  const double* st;
};
__device__ __forceinline__ SideRule side_rule(const Grid2& G, int sd, double lo, int idx, double h, double t) {
  SideRule r{G.bc[sd], G.st[sd]};
  if (r.bc == HWENO_BC_SPLIT || r.bc == HWENO_BC_SHOCK) {
    const double along = lo + (idx + 0.5) * h;
    if (r.bc == HWENO_BC_SPLIT) {
      r.bc = along < G.bcp[sd][0] ? HWENO_BC_INFLOW : HWENO_BC_REFLECT;
    } else {
      r.bc = HWENO_BC_INFLOW;
      if (!(along < G.bcp[sd][0] + G.bcp[sd][1] * t)) r.st = G.st2[sd];
    }
  }
  return r;
}

// Value of field f at cell (i, j), ghost cells resolved as "x sides for the
// interior rows, then y sides for every column"; t is the time the
// time-dependent sides are evaluated at.
template <typename T, int EQ, int NC>
__device__ __forceinline__ T load_ghost2(const T* __restrict__ in, long long plane, const Grid2& G,
                                         int f, int i, int j, double t) {
  const int d = f / NC, k = f % NC;
  // y sides decide by the column's centre x, x sides by the source row's centre y
  const SideRule ry0 = side_rule(G, 2, G.xlo, i, G.dx, t), ry1 = side_rule(G, 3, G.xlo, i, G.dx, t);
  const GhostMap gy = ghost_map(j, G.ny, ry0.bc, ry1.bc);
  if (gy.fixed) return d == 0 ? (T)(gy.side ? ry1.st : ry0.st)[k] : T(0);
  const SideRule rx0 = side_rule(G, 0, G.ylo, gy.src, G.dy, t), rx1 = side_rule(G, 1, G.ylo, gy.src, G.dy, t);
  const GhostMap gx = ghost_map(i, G.nx, rx0.bc, rx1.bc);
  T v;
  if (gx.fixed) {
    v = d == 0 ? (T)(gx.side ? rx1.st : rx0.st)[k] : T(0);
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
// The scale of coefficient l as the FP64 coefficient map forms it (the FP32
// map forms the coefficients themselves).
__host__ __device__ constexpr double sc2(int l) { return l == 6 || l == 9 ? 20.0 : (l >= 7 ? 4.0 : 1.0); }

template <typename TC>
struct Coef2 {
  TC c[15];
  TC dW, dE, dS, dN, q5;
  TC S;  // with SC: the largest |d_k| and |moment| (the FP32 screen's scale)
};

// The coefficients are evaluated on the centre-shifted averages
// d_k = q_k - q5 (k = 1..9, k != 5): p0 reproduces constants, so c_0 gains
// q5 and c_1..c_14 do not see it.  Every q5 term of the appendix's formulas
// cancels exactly, and the rounding of each coefficient scales with the
// local variation instead of with |q5| (in FP32 the difference of two nearby
// averages is exact).  With C0 = false, c_0 is not formed (the smoothness
// indicator does not use it); with SC, S is formed too, so that the stencil
// values are dead once the coefficients exist.
template <typename TC, typename TQ, bool C0 = true, bool SC = false>
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
  if constexpr (sizeof(TC) == 8) {
    // FP64: the denominators folded into the constants (one multiply fewer
    // per coefficient; the constants' own rounding is far below 1e-15)
    if constexpr (C0) {
      c[0] = q5 + TC(5.0 / 2880.0) * sc - TC(292.0 / 2880.0) * (ex + ey) + TC(81.0 / 2880.0) * (m1110 + m1716);
    } else {
      c[0] = TC(0);
    }
    c[1] = TC(1.0 / 12.0) * ax + TC(19.0 / 24.0) * dxe - TC(0.25) * s1011 + TC(0.125) * s1213;
    c[2] = TC(1.0 / 12.0) * ay + TC(19.0 / 24.0) * dye + TC(0.125) * s1415 - TC(0.25) * s1617;
    c[3] = TC(1.0 / 24.0) * ey + TC(31.0 / 24.0) * ex - TC(1.0 / 48.0) * sc - TC(0.375) * m1110;
    c[5] = TC(1.0 / 24.0) * ex + TC(31.0 / 24.0) * ey - TC(1.0 / 48.0) * sc - TC(0.375) * m1716;
  } else {
    if constexpr (C0) {
      c[0] = q5 + (TC(5) * sc - TC(292) * (ex + ey) + TC(81) * (m1110 + m1716)) * TC(1.0 / 2880.0);
    } else {
      c[0] = TC(0);
    }
    c[1] = (TC(2) * ax + TC(19) * dxe - TC(6) * s1011 + TC(3) * s1213) * TC(1.0 / 24.0);
    c[2] = (TC(2) * ay + TC(19) * dye + TC(3) * s1415 - TC(6) * s1617) * TC(1.0 / 24.0);
    c[3] = (TC(2) * ey + TC(62) * ex - sc - TC(18) * m1110) * TC(1.0 / 48.0);
    c[5] = (TC(2) * ex + TC(62) * ey - sc - TC(18) * m1716) * TC(1.0 / 48.0);
  }
  c[4] = TC(-0.375) * cx - TC(0.625) * (m1213 + m1415);
  if constexpr (sizeof(TC) == 8) {
    // FP64: c_6 and c_9 scaled by 20 and c_7, c_8, c_10..c_14 by 4 (sc2): each
    // is then one fused multiply-add of the shared sums, and the scales are
    // folded into the constants of their readers (betas2, face_points); the
    // combination and the back-projection are linear per coefficient
    c[6] = TC(4) * (s1011 - dxe) - ax - TC(2) * s1213;
    c[7] = -ay - TC(2) * dye;
    c[8] = -ax - TC(2) * dxe;
    c[9] = TC(4) * (s1617 - dye) - ay - TC(2) * s1415;
    c[10] = m1110 - TC(2) * ex;
    c[11] = cx + TC(2) * m1213;
    c[12] = sc - TC(2) * (ex + ey);
    c[13] = cx + TC(2) * m1415;
    c[14] = m1716 - TC(2) * ey;
  } else {
    c[6] = (TC(4) * (s1011 - dxe) - ax - TC(2) * s1213) * TC(0.05);
    c[7] = TC(-0.25) * ay - TC(0.5) * dye;
    c[8] = TC(-0.25) * ax - TC(0.5) * dxe;
    c[9] = (TC(4) * (s1617 - dye) - ay - TC(2) * s1415) * TC(0.05);
    c[10] = TC(0.25) * m1110 - TC(0.5) * ex;
    c[11] = TC(0.25) * cx + TC(0.5) * m1213;
    c[12] = TC(0.25) * sc - TC(0.5) * (ex + ey);
    c[13] = TC(0.25) * cx + TC(0.5) * m1415;
    c[14] = TC(0.25) * m1716 - TC(0.5) * ey;
  }
  o.dW = -d4;
  o.dE = d6;
  o.dS = -d2;
  o.dN = d8;
  o.q5 = q5;
  if constexpr (SC) {
    const TC dd[16] = {d1, d2, d3, d4, d6, d7, d8, d9, q10, q11, q12, q13, q14, q15, q16, q17};
    TC S = TC(0);
#pragma unroll
    for (int t = 0; t < 16; ++t) S = fmax(S, fabs_t(dd[t]));
    o.S = S;
  }
}

// Two FP32 lanes of work in one paired instruction (FADD2 / FMUL2 / FFMA2 of
// sm_100 and later; PTX add / sub / mul / fma .rn.f32x2): the same formula
// for two characteristic fields at once, each half rounded as the scalar
// instruction rounds it.
struct f2 { float2 v; };
__device__ __forceinline__ f2 pr(float a, float b) { return f2{make_float2(a, b)}; }
__device__ __forceinline__ f2 sp(float a) { return f2{make_float2(a, a)}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  unsigned long long ra, rb, rd;
  memcpy(&ra, &a.v, 8);
  memcpy(&rb, &b.v, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  f2 d;
  memcpy(&d.v, &rd, 8);
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return f2{__ffma2_rn(a.v, b.v, c.v)}; }

// coef2 (FP32, centre-shifted) for two fields at once: the FP32 formula of
// coef2 term by term, each multiply-add fused as the compiler fuses the
// scalar form; the coefficients and slopes stay paired.
struct Coef2x2 {
  f2 c[15];
  f2 dW, dE, dS, dN, q5;
};
__device__ __forceinline__ void coef2_pair(const float* qa, const float* qb, Coef2x2& o) {
  const f2 q5 = pr(qa[4], qb[4]);
  const f2 d1 = pr(qa[0], qb[0]) - q5, d2 = pr(qa[1], qb[1]) - q5, d3 = pr(qa[2], qb[2]) - q5;
  const f2 d4 = pr(qa[3], qb[3]) - q5, d6 = pr(qa[5], qb[5]) - q5;
  const f2 d7 = pr(qa[6], qb[6]) - q5, d8 = pr(qa[7], qb[7]) - q5, d9 = pr(qa[8], qb[8]) - q5;
  const f2 q10 = pr(qa[9], qb[9]), q11 = pr(qa[10], qb[10]), q12 = pr(qa[11], qb[11]);
  const f2 q13 = pr(qa[12], qb[12]), q14 = pr(qa[13], qb[13]), q15 = pr(qa[14], qb[14]);
  const f2 q16 = pr(qa[15], qb[15]), q17 = pr(qa[16], qb[16]);
  const f2 s13 = d1 + d3, s79 = d7 + d9, m13 = d1 - d3, m79 = d7 - d9;
  const f2 sc = s13 + s79, cx = m13 - m79, ax = m13 + m79, ay = s13 - s79;
  const f2 ex = d4 + d6, ey = d2 + d8, dxe = d6 - d4, dye = d8 - d2;
  const f2 s1011 = q10 + q11, m1110 = q11 - q10, s1213 = q12 + q13, m1213 = q12 - q13;
  const f2 s1415 = q14 + q15, m1415 = q14 - q15, s1617 = q16 + q17, m1716 = q17 - q16;
  o.c[0] = fma2(fma2(sp(81.0f), m1110 + m1716, fma2(sp(-292.0f), ex + ey, sp(5.0f) * sc)), sp(1.0f / 2880.0f), q5);
  o.c[1] = fma2(sp(3.0f), s1213, fma2(sp(-6.0f), s1011, fma2(sp(19.0f), dxe, sp(2.0f) * ax))) * sp(1.0f / 24.0f);
  o.c[2] = fma2(sp(-6.0f), s1617, fma2(sp(3.0f), s1415, fma2(sp(19.0f), dye, sp(2.0f) * ay))) * sp(1.0f / 24.0f);
  o.c[3] = fma2(sp(-18.0f), m1110, fma2(sp(62.0f), ex, sp(2.0f) * ey) - sc) * sp(1.0f / 48.0f);
  o.c[4] = fma2(sp(-0.625f), m1213 + m1415, sp(-0.375f) * cx);
  o.c[5] = fma2(sp(-18.0f), m1716, fma2(sp(62.0f), ey, sp(2.0f) * ex) - sc) * sp(1.0f / 48.0f);
  o.c[6] = fma2(sp(-2.0f), s1213, fma2(sp(4.0f), s1011 - dxe, sp(0.0f) - ax)) * sp(0.05f);
  o.c[7] = fma2(sp(-0.5f), dye, sp(-0.25f) * ay);
  o.c[8] = fma2(sp(-0.5f), dxe, sp(-0.25f) * ax);
  o.c[9] = fma2(sp(-2.0f), s1415, fma2(sp(4.0f), s1617 - dye, sp(0.0f) - ay)) * sp(0.05f);
  o.c[10] = fma2(sp(-0.5f), ex, sp(0.25f) * m1110);
  o.c[11] = fma2(sp(0.5f), m1213, sp(0.25f) * cx);
  o.c[12] = fma2(sp(-0.5f), ex + ey, sp(0.25f) * sc);
  o.c[13] = fma2(sp(0.5f), m1415, sp(0.25f) * cx);
  o.c[14] = fma2(sp(-0.5f), ey, sp(0.25f) * m1716);
  const f2 z = sp(0.0f);
  o.dW = z - d4;
  o.dE = d6;
  o.dS = z - d2;
  o.dN = d8;
  o.q5 = q5;
}
__device__ __forceinline__ void unpack2(const Coef2x2& k, Coef2<float>& a, Coef2<float>& b) {
#pragma unroll
  for (int l = 0; l < 15; ++l) { a.c[l] = k.c[l].v.x; b.c[l] = k.c[l].v.y; }
  a.dW = k.dW.v.x; b.dW = k.dW.v.y;
  a.dE = k.dE.v.x; b.dE = k.dE.v.y;
  a.dS = k.dS.v.x; b.dS = k.dS.v.y;
  a.dN = k.dN.v.x; b.dN = k.dN.v.y;
  a.q5 = k.q5.v.x; b.q5 = k.q5.v.y;
}
__device__ __forceinline__ void coef2_x2(const float* qa, const float* qb, Coef2<float>& oa, Coef2<float>& ob) {
  Coef2x2 k;
  coef2_pair(qa, qb, k);
  unpack2(k, oa, ob);
}

// Jiang-Shu indicator of the 2D quartic, the 2D form of Eq.
// (smoothness-indicator-typical): the sum over 1 <= m + n <= 4 of the
// integrals over [-1/2, 1/2]^2 of (d^{m+n} p / dxi^m deta^n)^2, as the
// closed quadratic form in c_1..c_14 (29 terms; the odd monomial moments
// vanish), grouped by the first coefficient of each product.
template <typename T>
__device__ __forceinline__ T beta_typical_2d(const T* c) {
  T b = c[1] * (c[1] + T(0.5) * c[6] + T(1.0 / 6.0) * c[8]);
  b += c[2] * (c[2] + T(1.0 / 6.0) * c[7] + T(0.5) * c[9]);
  b += c[3] * (T(13.0 / 3.0) * c[3] + T(4.2) * c[10] + T(13.0 / 18.0) * c[12]);
  b += c[5] * (T(13.0 / 3.0) * c[5] + T(4.2) * c[14] + T(13.0 / 18.0) * c[12]);
  b += c[4] * (T(7.0 / 6.0) * c[4] + T(17.0 / 30.0) * (c[11] + c[13]));
  b += c[6] * (T(3129.0 / 80.0) * c[6] + T(1.0 / 24.0) * c[8]);
  b += c[9] * (T(3129.0 / 80.0) * c[9] + T(1.0 / 24.0) * c[7]);
  b += T(3389.0 / 720.0) * (c[7] * c[7] + c[8] * c[8]);
  b += c[10] * (T(87617.0 / 140.0) * c[10] + T(0.35) * c[12]);
  b += c[14] * (T(87617.0 / 140.0) * c[14] + T(0.35) * c[12]);
  b += c[11] * (T(47459.0 / 1120.0) * c[11] + T(11.0 / 80.0) * c[13]);
  b += T(47459.0 / 1120.0) * c[13] * c[13] + T(6799.0 / 360.0) * c[12] * c[12];
  return b;
}

// Step 2 (Sec. 2.2): beta_0 = sum (m! n! c)^2 (or the Jiang-Shu form),
// beta_1..4 of the linear polynomials, and tau = 1/4 sum |beta_0 - beta_m|.
template <typename TW>
__device__ __forceinline__ TW betas2(const Coef2<TW>& k, const WeightsT<TW>& w, TW* beta) {
  const TW* c = k.c;
  const TW b1 = k.dW * k.dW + k.dS * k.dS, b2 = k.dE * k.dE + k.dS * k.dS;
  const TW b3 = k.dE * k.dE + k.dN * k.dN, b4 = k.dW * k.dW + k.dN * k.dN;
  TW b0;
  if constexpr (sizeof(TW) == 8) {
    // the FP64 coefficients carry the scales sc2: the weights (m! n!)^2 / sc2^2
    if (w.typical) {
      TW cu[15];
#pragma unroll
      for (int l = 0; l < 15; ++l) cu[l] = c[l] * TW(1.0 / sc2(l));
      b0 = beta_typical_2d(cu);
    } else {
      b0 = c[1] * c[1] + c[2] * c[2] + c[4] * c[4] + TW(4) * (c[3] * c[3] + c[5] * c[5]) +
           TW(0.25) * (c[7] * c[7] + c[8] * c[8]) + TW(0.09) * (c[6] * c[6] + c[9] * c[9]) +
           TW(2.25) * (c[11] * c[11] + c[13] * c[13]) + TW(36) * (c[10] * c[10] + c[14] * c[14]) +
           c[12] * c[12];
    }
  } else {
    b0 = w.typical ? beta_typical_2d(c)
                   : c[1] * c[1] + c[2] * c[2] + c[4] * c[4] +
                         TW(4) * (c[3] * c[3] + c[5] * c[5] + c[7] * c[7] + c[8] * c[8]) +
                         TW(36) * (c[6] * c[6] + c[9] * c[9] + c[11] * c[11] + c[13] * c[13]) +
                         TW(576) * (c[10] * c[10] + c[14] * c[14]) + TW(16) * c[12] * c[12];
  }
  beta[0] = b0; beta[1] = b1; beta[2] = b2; beta[3] = b3; beta[4] = b4;
  return TW(0.25) * ((fabs_t(b0 - b1) + fabs_t(b0 - b2)) + (fabs_t(b0 - b3) + fabs_t(b0 - b4)));
}

// Steps 2-3 (Sec. 2.2): the indicators and the nonlinear weights;
// r = omega_0 / gamma_0 and om[1..4].  With DEV the largest
// |omega_m / gamma_m - 1| is folded into *dev.
template <typename TW, bool DEV>
__device__ __forceinline__ void weights2(const Coef2<TW>& k, const WeightsT<TW>& w, TW& r, TW* om, TW* dev) {
  TW beta[5];
  const TW tau = betas2<TW>(k, w, beta);
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

// FP64, Steps 2-3 and Eq. (hweno-reconstruction-2D) in one.  With the weight
// numerators f_m (nl_numerators: w~_m P = gamma_m f_m), e_m = gamma_m f_m and
// s = sum_m e_m: r = f_0 / s, omega_m = e_m / s, so the pair sums of omega
// the combination takes are (e_a + e_b) / s, and sum_{m >= 1} omega_m =
// 1 - r gamma_0 (the weights sum to 1).
__device__ __forceinline__ void weights_combine2_f64(const Coef2<double>& k, const WeightsT<double>& w, double* cu) {
  double beta[5], f[5];
  const double tau = betas2<double>(k, w, beta);
  nl_numerators<double, 4>(beta, tau, w, f);
  const double* c = k.c;
  const double e1 = w.g[1] * f[1], e2 = w.g[2] * f[2], e3 = w.g[3] * f[3], e4 = w.g[4] * f[4];
  const double E12 = e1 + e2, E34 = e3 + e4;
  const double inv = rcp_t(fma(w.g[0], f[0], E12 + E34));
  const double r = f[0] * inv;
  const double ws = fma(-r, w.g[0], 1.0);
  const double gs = (w.g[1] + w.g[2]) + (w.g[3] + w.g[4]);
  // r (c_1 - G_W dW - G_E dE) + O_W dW + O_E dE = r c_1 + (O_W - r G_W) dW + (O_E - r G_E) dE,
  // O_W - r G_W = (e_1 + e_4 - f_0 G_W) / s
  const double aW = (fma(-f[0], w.g[1] + w.g[4], e1 + e4)) * inv;
  const double aE = (fma(-f[0], w.g[2] + w.g[3], e2 + e3)) * inv;
  const double aS = (fma(-f[0], w.g[1] + w.g[2], E12)) * inv;
  const double aN = (fma(-f[0], w.g[3] + w.g[4], E34)) * inv;
  cu[0] = r * (c[0] - gs * k.q5) + ws * k.q5;
  cu[1] = r * c[1] + (aW * k.dW + aE * k.dE);
  cu[2] = r * c[2] + (aS * k.dS + aN * k.dN);
#pragma unroll
  for (int l = 3; l < 15; ++l) cu[l] = r * c[l];
}

// Eq. (hweno-reconstruction-2D): cu = r (p0 - sum gamma_m p_m) + sum omega_m p_m.
template <typename T>
__device__ __forceinline__ void combine2(const Coef2<T>& k, T r, const T* om, const WeightsT<T>& w, T* cu) {
  const T* c = k.c;
  const T gs = (w.g[1] + w.g[2]) + (w.g[3] + w.g[4]);
  const T ws = (om[1] + om[2]) + (om[3] + om[4]);
  cu[0] = r * (c[0] - gs * k.q5) + ws * k.q5;
  if constexpr (sizeof(T) == 8) {
    // r (c_1 - G_W dW - G_E dE) + O_W dW + O_E dE = r c_1 + (O_W - r G_W) dW + (O_E - r G_E) dE
    const T aW = (om[1] + om[4]) - r * (w.g[1] + w.g[4]), aE = (om[2] + om[3]) - r * (w.g[2] + w.g[3]);
    const T aS = (om[1] + om[2]) - r * (w.g[1] + w.g[2]), aN = (om[3] + om[4]) - r * (w.g[3] + w.g[4]);
    cu[1] = r * c[1] + (aW * k.dW + aE * k.dE);
    cu[2] = r * c[2] + (aS * k.dS + aN * k.dN);
  } else {
    cu[1] = r * (c[1] - ((w.g[1] + w.g[4]) * k.dW + (w.g[2] + w.g[3]) * k.dE)) +
            ((om[1] + om[4]) * k.dW + (om[2] + om[3]) * k.dE);
    cu[2] = r * (c[2] - ((w.g[1] + w.g[2]) * k.dS + (w.g[3] + w.g[4]) * k.dN)) +
            ((om[1] + om[2]) * k.dS + (om[3] + om[4]) * k.dN);
  }
#pragma unroll
  for (int l = 3; l < 15; ++l) cu[l] = r * c[l];
}

// Steps 2-3 for one field from its coefficients: the combined polynomial cu
// (lin: p0 itself).
template <typename T, bool DEV = false>
__device__ __forceinline__ void recon2_from(const Coef2<T>& k, const WeightsT<T>& w, bool lin, T* cu, T* dev = nullptr) {
  if (lin) {
#pragma unroll
    for (int l = 0; l < 15; ++l) cu[l] = k.c[l];
    return;
  }
  if constexpr (sizeof(T) == 8 && !DEV) {
    weights_combine2_f64(k, w, cu);
  } else {
    T r, om[5];
    weights2<T, DEV>(k, w, r, om, dev);
    combine2<T>(k, r, om, w, cu);
  }
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
  if constexpr (sizeof(T) == 8 && !DEV) {
    weights_combine2_f64(k, w, cu);
  } else {
    T r, om[5];
    weights2<T, DEV>(k, w, r, om, dev);
    combine2<T>(k, r, om, w, cu);
  }
}

// |x| of both halves (the sign bits cleared on the integer ALU).
__device__ __forceinline__ f2 abs2(f2 x) {
  return f2{make_float2(__uint_as_float(__float_as_uint(x.v.x) & 0x7fffffffu),
                        __uint_as_float(__float_as_uint(x.v.y) & 0x7fffffffu))};
}

// FP32, Steps 1-3 for two fields at once (recon2 term by term, paired): the
// coefficient maps, the moment indicator and the weights of Sec. 2.2 with
// the FP32 quotients, and the combination of Eq. (hweno-reconstruction-2D).
// The Jiang-Shu form takes the scalar path.
__device__ __forceinline__ void recon2_x2(const float* qa, const float* qb, const WeightsT<float>& w, bool lin,
                                          float* cua, float* cub) {
  Coef2x2 k;
  coef2_pair(qa, qb, k);
  const f2* c = k.c;
  if (lin) {
#pragma unroll
    for (int l = 0; l < 15; ++l) { cua[l] = c[l].v.x; cub[l] = c[l].v.y; }
    return;
  }
  if (w.typical) {
    Coef2<float> ka, kb;
    unpack2(k, ka, kb);
    recon2_from<float>(ka, w, false, cua);
    recon2_from<float>(kb, w, false, cub);
    return;
  }
  // Step 2: beta_0 = sum (m! n! c)^2, beta_1..4 of the linear polynomials
  const f2 dW2 = k.dW * k.dW, dE2 = k.dE * k.dE, dS2 = k.dS * k.dS, dN2 = k.dN * k.dN;
  f2 beta[5];
  beta[1] = dW2 + dS2;
  beta[2] = dE2 + dS2;
  beta[3] = dE2 + dN2;
  beta[4] = dW2 + dN2;
  const f2 g4 = fma2(c[8], c[8], fma2(c[7], c[7], fma2(c[5], c[5], c[3] * c[3])));
  const f2 g36 = fma2(c[13], c[13], fma2(c[11], c[11], fma2(c[9], c[9], c[6] * c[6])));
  const f2 g576 = fma2(c[14], c[14], c[10] * c[10]);
  f2 b0 = fma2(c[4], c[4], fma2(c[2], c[2], c[1] * c[1]));
  b0 = fma2(sp(16.0f) * c[12], c[12], fma2(sp(576.0f), g576, fma2(sp(36.0f), g36, fma2(sp(4.0f), g4, b0))));
  beta[0] = b0;
  const f2 tau = sp(0.25f) * ((abs2(b0 - beta[1]) + abs2(b0 - beta[2])) + (abs2(b0 - beta[3]) + abs2(b0 - beta[4])));
  // Step 3: w~_m = gamma_m (1 + tau^2 / (beta_m^p + eps)), omega = w~ / sum w~
  const f2 t2 = tau * tau;
  f2 e[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const f2 d = w.pow2 ? fma2(beta[m], beta[m], sp(w.eps)) : beta[m] + sp(w.eps);
    const f2 a = t2 * pr(rcp_approx(d.v.x), rcp_approx(d.v.y));
    e[m] = fma2(sp(w.g[m]), a, sp(w.g[m]));
  }
  const f2 sum = ((e[0] + e[1]) + (e[2] + e[3])) + e[4];
  const f2 inv = pr(rcp_approx(sum.v.x), rcp_approx(sum.v.y));
  const f2 r = (e[0] * inv) * sp(w.inv_g0);
  f2 om[5];
#pragma unroll
  for (int m = 1; m <= 4; ++m) om[m] = e[m] * inv;
  // Eq. (hweno-reconstruction-2D): cu = r (p0 - sum gamma_m p_m) + sum omega_m p_m
  const float gs = (w.g[1] + w.g[2]) + (w.g[3] + w.g[4]);
  const f2 ws = (om[1] + om[2]) + (om[3] + om[4]);
  f2 cu[15];
  cu[0] = fma2(ws, k.q5, r * fma2(sp(-gs), k.q5, c[0]));
  cu[1] = fma2(om[2] + om[3], k.dE, (om[1] + om[4]) * k.dW) +
          r * (c[1] - fma2(sp(w.g[2] + w.g[3]), k.dE, sp(w.g[1] + w.g[4]) * k.dW));
  cu[2] = fma2(om[3] + om[4], k.dN, (om[1] + om[2]) * k.dS) +
          r * (c[2] - fma2(sp(w.g[3] + w.g[4]), k.dN, sp(w.g[1] + w.g[2]) * k.dS));
#pragma unroll
  for (int l = 3; l < 15; ++l) cu[l] = r * c[l];
#pragma unroll
  for (int l = 0; l < 15; ++l) { cua[l] = cu[l].v.x; cub[l] = cu[l].v.y; }
}

// The stencil values of one field, by value (the argument of the FP64
// indicator below).
struct Stencil17 { float q[17]; };
struct Weights5 { float a[5]; };

// Mixed precision, the FP64 part of Steps 2-3 for one field: a_m =
// tau^2 / (beta_m^{1|2} + eps) from the FP32 stencil values q, rounded to
// FP32.
//  * The indicator uses c_1..c_14 only, each c_l = u_l / den_l with u_l an
//    integer-weighted sum of the centre-shifted averages and the moments;
//    the 1/den_l^2 factors are folded into beta_0's weights (m! n!)^2:
//    576 beta_0 = u1^2 + u2^2 + u3^2 + u5^2 + 9 u4^2 + 144 (u7^2 + u8^2)
//                 + 51.84 (u6^2 + u9^2) + 1296 (u11^2 + u13^2)
//                 + 20736 (u10^2 + u14^2) + 576 u12^2.
//  * The inputs are widened exactly on the integer ALU; the differences
//    q_k - q5 are taken in FP32 when that is exact for all 32 lanes (checked
//    with Knuth's TwoSum error term), else in FP64.
//  * beta_m, tau and a_m in FP64 (the reciprocal by rcp_newton).
// Not inlined: it runs only for warps the FP32 screen cannot clear, and as a
// call its register demand is met by saves on that path alone instead of
// spills of the caller's live values on every path.  All 32 lanes call it.
static __device__ __noinline__ Weights5 indicator64(const Stencil17 st, double eps, int pow2, int typical) {
  const float* q = st.q;
  const float q5f = q[4];
  float d32[9];
  bool exact = true;
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    if (s == 4) continue;
    const float a = q[s], b = -q5f;
    const float sum = a + b, bb = sum - a;
    exact = exact && ((a - (sum - bb)) + (b - bb)) == 0.0f;
    d32[s] = sum;
  }
  Weights5 out;
  float* a = out.a;
  double d[9];
  if (__all_sync(HW_FULL_MASK, exact)) {
#pragma unroll
    for (int s = 0; s < 9; ++s)
      if (s != 4) d[s] = widen_f32(d32[s]);
  } else {
    const double q5 = widen_f32(q5f);
#pragma unroll
    for (int s = 0; s < 9; ++s)
      if (s != 4) d[s] = widen_f32(q[s]) - q5;
  }
  const double d1 = d[0], d2 = d[1], d3 = d[2], d4 = d[3], d6 = d[5], d7 = d[6], d8 = d[7], d9 = d[8];
  const double q10 = widen_f32(q[9]), q11 = widen_f32(q[10]), q12 = widen_f32(q[11]), q13 = widen_f32(q[12]);
  const double q14 = widen_f32(q[13]), q15 = widen_f32(q[14]), q16 = widen_f32(q[15]), q17 = widen_f32(q[16]);
  const double s13 = d1 + d3, s79 = d7 + d9, m13 = d1 - d3, m79 = d7 - d9;
  const double sc = s13 + s79, cx = m13 - m79, ax = m13 + m79, ay = s13 - s79;
  const double ex = d4 + d6, ey = d2 + d8, dxe = d6 - d4, dye = d8 - d2;
  const double s1011 = q10 + q11, m1110 = q11 - q10, s1213 = q12 + q13, m1213 = q12 - q13;
  const double s1415 = q14 + q15, m1415 = q14 - q15, s1617 = q16 + q17, m1716 = q17 - q16;
  const double u1 = 2.0 * ax + 19.0 * dxe - 6.0 * s1011 + 3.0 * s1213;
  const double u2 = 2.0 * ay + 19.0 * dye + 3.0 * s1415 - 6.0 * s1617;
  const double u3 = 2.0 * ey - sc + 62.0 * ex - 18.0 * m1110;
  const double u5 = 2.0 * ex - sc + 62.0 * ey - 18.0 * m1716;
  const double u4 = 3.0 * cx + 5.0 * (m1213 + m1415);
  const double u6 = 4.0 * (s1011 - dxe) - ax - 2.0 * s1213;
  const double u9 = 4.0 * (s1617 - dye) - ay - 2.0 * s1415;
  const double u7 = ay + 2.0 * dye, u8 = ax + 2.0 * dxe;
  const double u10 = m1110 - 2.0 * ex, u14 = m1716 - 2.0 * ey;
  const double u11 = cx + 2.0 * m1213, u13 = cx + 2.0 * m1415;
  const double u12 = sc - 2.0 * (ex + ey);
  double b0;
  if (typical) {  // the Jiang-Shu form needs the scaled coefficients c_l = u_l / den_l
    const double c[15] = {0.0,         u1 * (1.0 / 24.0), u2 * (1.0 / 24.0), u3 * (1.0 / 48.0), -0.125 * u4,
                          u5 * (1.0 / 48.0), 0.05 * u6,   -0.25 * u7,        -0.25 * u8,        0.05 * u9,
                          0.25 * u10,  0.25 * u11,        0.25 * u12,        0.25 * u13,        0.25 * u14};
    b0 = beta_typical_2d(c);
  } else {
    double acc = u1 * u1 + u2 * u2 + u3 * u3 + u5 * u5 + 9.0 * u4 * u4;
    acc += 144.0 * (u7 * u7 + u8 * u8) + 51.84 * (u6 * u6 + u9 * u9);
    acc += 1296.0 * (u11 * u11 + u13 * u13) + 20736.0 * (u10 * u10 + u14 * u14) + 576.0 * u12 * u12;
    b0 = acc * (1.0 / 576.0);
  }
  const double w2 = d4 * d4, e2 = d6 * d6, s2 = d2 * d2, n2 = d8 * d8;  // dW, dE, dS, dN squared
  const double b1 = w2 + s2, b2 = e2 + s2, b3 = e2 + n2, b4 = w2 + n2;
  const double tau = 0.25 * ((fabs(b0 - b1) + fabs(b0 - b2)) + (fabs(b0 - b3) + fabs(b0 - b4)));
  // the epsilon-sensitive part in FP64: a_m = tau^2 / (beta_m^{1|2} + eps)
  const double t2 = tau * tau;
  const double beta[5] = {b0, b1, b2, b3, b4};
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const double dm = (pow2 ? beta[m] * beta[m] : beta[m]) + eps;
    a[m] = narrow_f64_ftz(t2 * rcp_newton(dm));
  }
  return out;
}

// Mixed precision, Steps 2-3 for one field, FP32 part: the screen.  True
// where every a_m = tau^2 / (beta_m^p + eps) is provably below 2^-24, so
// that 1 + a_m is 1 in FP32 and a_m = 0 gives the FP64 evaluation's result
// bit for bit.
__device__ __forceinline__ bool screen2(const Coef2<float>& k, const WeightsT<double>& w,
                                        const WeightsT<float>& wf) {
  // verification build (libhweno_noscreen.so, which sets screen_off on the
  // host and compiles the same device code): every lane takes the FP64
  // indicator, to show that the screen never changes an output bit
  if (wf.screen_off) return false;
  // FP32 screen: a sound upper bound on every a_m = tau^2 / (beta_m^p + eps)
  // from the FP32 coefficients k.  Each c~_l combines the stencil differences
  // and moments (largest magnitude S) and errs by at most ~30 u S in FP32
  // (u = 2^-24), bounded here by E = 2^-16 S.  beta_0 is a quadratic form
  // sum_t m_t c_a c_b with positive m_t (the moment form: squares only; the
  // Jiang-Shu form: 29 terms), so
  //   |beta~_0 - beta_0| <= 2^-18 A + E (G + E sum_t m_t),
  // A the form at |c~|, G = sum_l R_l |c~_l| with R_l the form's row sums;
  //   |beta~_m - beta_m| <= 2^-20 beta~_m  (m >= 1),
  // and tau <= tau~ (1 + 2^-20) + D_0 + (D_1 + ... + D_4) / 4.  For the
  // moment form (weights w_l summing to 1331) Cauchy-Schwarz gives
  // G = 2 sum_l w_l |c~_l| <= 2 sqrt(1331 A) <= 72.97 sqrt(beta~_0), taken
  // as 73 sqrt(beta~_0); likewise for the Jiang-Shu form with its matrix.  Where the bound puts every a_m below 2^-25 for
  // all 32 lanes, 1 + a_m is 1 in FP32 whatever the FP64 evaluation gives,
  // so that evaluation is skipped and the result is the same bit for bit
  // (any sound bound keeps this; a looser one only skips less often).
  bool quiet;
  {
    // S: the largest stencil difference or moment (k.S, formed with the coefficients)
    const float S = k.S;
    const float* c = k.c;
    const float E = S * 0x1p-16f;
    float bs[5], Ds[5];
    if (w.typical) {
      float ac[15];
#pragma unroll
      for (int l = 0; l < 15; ++l) ac[l] = fabsf(c[l]);
      bs[0] = beta_typical_2d(c);
      const float A = beta_typical_2d(ac);
      // G = 2 sum_l R_l |c~_l| <= 2 sqrt(R^T M^-1 R) sqrt(A), M the form's
      // (positive definite) matrix: 2 sqrt(R^T M^-1 R) = 76.63, taken as 76.7
      const float G = 76.7f * sqrt_approx(A);
      Ds[0] = 0x1p-18f * A + E * (G + 1469.0f * E);
    } else {
      bs[0] = c[1] * c[1] + c[2] * c[2] + c[4] * c[4] +
              4.0f * (c[3] * c[3] + c[5] * c[5] + c[7] * c[7] + c[8] * c[8]) +
              36.0f * (c[6] * c[6] + c[9] * c[9] + c[11] * c[11] + c[13] * c[13]) +
              576.0f * (c[10] * c[10] + c[14] * c[14]) + 16.0f * c[12] * c[12];
      const float G = 73.0f * sqrt_approx(bs[0]);
      Ds[0] = 0x1p-18f * bs[0] + E * (G + 1331.0f * E);
    }
    bs[1] = k.dW * k.dW + k.dS * k.dS;
    bs[2] = k.dE * k.dE + k.dS * k.dS;
    bs[3] = k.dE * k.dE + k.dN * k.dN;
    bs[4] = k.dW * k.dW + k.dN * k.dN;
#pragma unroll
    for (int m = 1; m < 5; ++m) Ds[m] = 0x1p-20f * bs[m];
    const float tau = 0.25f * ((fabsf(bs[0] - bs[1]) + fabsf(bs[0] - bs[2])) +
                               (fabsf(bs[0] - bs[3]) + fabsf(bs[0] - bs[4])));
    const float ut = tau * (1.0f + 0x1p-20f) + Ds[0] + 0.25f * ((Ds[1] + Ds[2]) + (Ds[3] + Ds[4]));
    const float ut2 = ut * ut;
    // every a_m small <=> small against the least lower bound of beta_m
    // (x -> x^p + eps rounds monotonically)
    float L = bs[0] - Ds[0];
#pragma unroll
    for (int m = 1; m < 5; ++m) L = fminf(L, bs[m] - Ds[m]);
    L = fmaxf(L, 0.0f);
    const float dlo = (wf.pow2 ? L * L : L) + wf.eps;
    // ut, ut^2 and dlo carry at most a few FP32 roundings (relative 2^-21
    // together), so ut2 < 2^-25 dlo puts the exact bound below 2^-24: the
    // FP64 a_m, narrowed to FP32, is then at most 2^-24 and 1 + a_m rounds to
    // 1 (to nearest, ties to even), as a_m = 0 gives
    quiet = ut2 < 0x1p-25f * dlo;
  }
  return quiet;
}

// Steps 2-3, the weights from a_m (0 where screened, else indicator64):
// w~_m = gamma_m (1 + a_m) and the normalisation in FP32 (every term
// positive: a few FP32 ulp at most), r = omega_0 / gamma_0 and om[1..4],
// materialised, so that weights from a_m = 0 read the same wherever they
// were formed.
__device__ __forceinline__ void finish2(const float* a, const WeightsT<float>& wf, float& r, float* om) {
  float e[5], sum = 0.0f;
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    e[m] = wf.g[m] * (1.0f + a[m]);
    sum += e[m];
  }
  const float inv = rcp_approx(sum);
  r = opaque((1.0f + a[0]) * inv);
#pragma unroll
  for (int m = 1; m <= 4; ++m) om[m] = opaque(e[m] * inv);
}

// Values at the three Gauss points of the face xi = +-1/2 (sgn = +1 / -1)
// of the pass frame: u, d/dxi u, d/deta u; and the face averages of the
// three (the 3-point Gauss rule is exact for these degree-4 restrictions:
// over eta in [-1/2, 1/2], eta^2 averages 1/12 and eta^4 1/80).
template <typename T>
struct FacePts { T u[3], un[3], ut[3], au, an, at; };

template <typename T>
__device__ __forceinline__ void face_points(const T* c, T sgn, FacePts<T>& o) {
  if constexpr (sizeof(T) == 8) {
    // FP64: the coefficients carry the scales sc2 (c_6, c_9 x 20; c_7, c_8,
    // c_10..c_14 x 4); A3 = 20 A3, A4 = 4 A4, B2 = 4 B2 and B3 = 4 B3 below,
    // their scales folded into the constants that read them
    const double s = 0.38729833462074168852, s2 = 0.15, s3 = s * 0.15, s4 = 0.0225;
    const double A0 = (c[0] + 0.25 * c[3] + 0.015625 * c[10]) + sgn * (0.5 * c[1] + 0.00625 * c[6]);
    const double A1 = (c[2] + 0.0625 * c[7]) + sgn * (0.5 * c[4] + 0.03125 * c[11]);
    const double A2 = (c[5] + 0.0625 * c[12]) + sgn * (0.125 * c[8]);
    const double A3 = c[9] + sgn * (2.5 * c[13]);
    const double A4 = c[14];
    const double B0 = (c[1] + 0.0375 * c[6]) + sgn * (c[3] + 0.125 * c[10]);
    const double B1 = (c[4] + 0.1875 * c[11]) + sgn * (0.25 * c[7]);
    const double B2 = c[8] + sgn * c[12];
    const double B3 = c[13];
    const double ue = A0 + A2 * s2 + A4 * (s4 / 4), uo = A1 * s + A3 * (s3 / 20);
    const double ne = B0 + B2 * (s2 / 4), no = B1 * s + B3 * (s3 / 4);
    const double te = A1 + A3 * (3 * s2 / 20), to = A2 * (2 * s) + A4 * s3;
    o.u[0] = ue - uo; o.u[1] = A0; o.u[2] = ue + uo;
    o.un[0] = ne - no; o.un[1] = B0; o.un[2] = ne + no;
    o.ut[0] = te - to; o.ut[1] = A1; o.ut[2] = te + to;
    o.au = A0 + A2 * (1.0 / 12.0) + A4 * (0.0125 / 4);
    o.an = B0 + B2 * (1.0 / 48.0);
    o.at = A1 + A3 * (0.25 / 20);
    return;
  }
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
  o.au = A0 + A2 * T(1.0 / 12.0) + A4 * T(0.0125);
  o.an = B0 + B2 * T(1.0 / 12.0);
  o.at = A1 + T(0.25) * A3;
}

// face_points (FP32) for two fields at once and both faces of each (right:
// xi = +1/2, left: xi = -1/2): the even and odd parts of every face
// coefficient once, each face from their sum or difference.
__device__ __forceinline__ void face_points_x2(const float* ca, const float* cb, FacePts<float>& ra,
                                               FacePts<float>& rb, FacePts<float>& la, FacePts<float>& lb) {
  f2 c[15];
#pragma unroll
  for (int l = 0; l < 15; ++l) c[l] = pr(ca[l], cb[l]);
  const float s = 0.38729833462074168852f, s2 = 0.15f, s3 = s * 0.15f, s4 = 0.0225f;
  const f2 eA0 = fma2(sp(0.0625f), c[10], fma2(sp(0.25f), c[3], c[0]));
  const f2 oA0 = fma2(sp(0.125f), c[6], sp(0.5f) * c[1]);
  const f2 eA1 = fma2(sp(0.25f), c[7], c[2]);
  const f2 oA1 = fma2(sp(0.125f), c[11], sp(0.5f) * c[4]);
  const f2 eA2 = fma2(sp(0.25f), c[12], c[5]);
  const f2 oA2 = sp(0.5f) * c[8];
  const f2 eB0 = fma2(sp(0.75f), c[6], c[1]);
  const f2 oB0 = fma2(sp(0.5f), c[10], c[3]);
  const f2 eB1 = fma2(sp(0.75f), c[11], c[4]);
  const f2 A4 = c[14], B3 = c[13];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const bool r = side == 0;
    const f2 A0 = r ? eA0 + oA0 : eA0 - oA0;
    const f2 A1 = r ? eA1 + oA1 : eA1 - oA1;
    const f2 A2 = r ? eA2 + oA2 : eA2 - oA2;
    const f2 A3 = fma2(sp(r ? 0.5f : -0.5f), c[13], c[9]);
    const f2 B0 = r ? eB0 + oB0 : eB0 - oB0;
    const f2 B1 = r ? eB1 + c[7] : eB1 - c[7];
    const f2 B2 = r ? c[8] + c[12] : c[8] - c[12];
    const f2 ue = fma2(A4, sp(s4), fma2(A2, sp(s2), A0)), uo = fma2(A3, sp(s3), A1 * sp(s));
    const f2 ne = fma2(B2, sp(s2), B0), no = fma2(B3, sp(s3), B1 * sp(s));
    const f2 te = fma2(A3, sp(3.0f * s2), A1), to = fma2(A4, sp(4.0f * s3), A2 * sp(2.0f * s));
    const f2 u0 = ue - uo, u2 = ue + uo, n0 = ne - no, n2 = ne + no, t0 = te - to, t2 = te + to;
    const f2 au = fma2(A4, sp(0.0125f), fma2(A2, sp(1.0f / 12.0f), A0));
    const f2 an = fma2(B2, sp(1.0f / 12.0f), B0), at = fma2(sp(0.25f), A3, A1);
    FacePts<float>& oa = r ? ra : la;
    FacePts<float>& ob = r ? rb : lb;
    oa.u[0] = u0.v.x; oa.u[1] = A0.v.x; oa.u[2] = u2.v.x;
    ob.u[0] = u0.v.y; ob.u[1] = A0.v.y; ob.u[2] = u2.v.y;
    oa.un[0] = n0.v.x; oa.un[1] = B0.v.x; oa.un[2] = n2.v.x;
    ob.un[0] = n0.v.y; ob.un[1] = B0.v.y; ob.un[2] = n2.v.y;
    oa.ut[0] = t0.v.x; oa.ut[1] = A1.v.x; oa.ut[2] = t2.v.x;
    ob.ut[0] = t0.v.y; ob.ut[1] = A1.v.y; ob.ut[2] = t2.v.y;
    oa.au = au.v.x; ob.au = au.v.y;
    oa.an = an.v.x; ob.an = an.v.y;
    oa.at = at.v.x; ob.at = at.v.y;
  }
}

}  // namespace hw
