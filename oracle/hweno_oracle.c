/*
 * hweno_oracle.c -- plain, slow, serial FP64 CPU oracle of the fifth-order
 * finite-volume derivative-based HWENO scheme with unified stencils
 * (arxiv 2607.24325).  TEST INFRASTRUCTURE ONLY: used by tests/, by
 * __graft_entry__.smoke() and by the CPU legs of bench.py, never by the
 * product path, and it shares no code with the CUDA library.
 *
 * It follows the paper step by step, in the paper's order:
 *   Sec. 2.1 Step 1   polynomials p0 (quartic), p1, p2 (linear), Eq. (rewrite)
 *   Sec. 2.1 Step 2   smoothness indicators (cheap form)
 *   Sec. 2.1 Step 3   tau, nonlinear weights, Eq. (hweno-reconstruction-1D),
 *                     limited derivative v-hat, interface values
 *   Sec. 2.1          Eq. (semi-discrete-scheme), global Lax-Friedrichs flux
 *   Sec. 2.1 Step 4   SSP-RK3 with derivative substitution
 *   Sec. 2.2          the same for two dimensions (3-point Gauss-Legendre on
 *                     faces, Eq. (2D-semi-discrete-scheme-uniform))
 *   Remark 1          characteristic-wise reconstruction for Euler.
 * The polynomial coefficient maps are NOT typed in from Appendix A: they are
 * derived here from the constraint definitions of Step 1 (exact moment
 * integrals of monomials + a dense linear solve), so that the printed
 * appendix tables can pin this code from outside.
 *
 * Readings of points the paper leaves open:
 *   - 1D beta is sum_l (l! c_l)^2 (the printed formula drops the square).
 *   - 2D p0 fits the derivative moments of the 4 face neighbours in the
 *     least-squares sense (this is exactly what Appendix A prints).
 *   - characteristic fields use the eigenvectors of the target cell's
 *     average; 2D uses an x pass (x faces, v-hat) and a y pass (y faces,
 *     w-hat).
 *   - alpha is the max spectral radius over the cell averages of u^n, held
 *     for the three stages of a step; dt = CFL dx / alpha (1D),
 *     CFL / (ax/dx + ay/dy) (2D); dx -> dx^(5/3) for order studies.
 *   - ghost cells: x sides filled for interior rows first, then y sides for
 *     all columns; periodic wraps; outflow copies the nearest interior cell
 *     (average and moments); reflective mirrors, negating the normal
 *     momentum and every moment whose sign flips under the mirror; inflow
 *     imposes a fixed state with zero moments.
 */
#include "hweno_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Flop counter: the method's arithmetic per cell and stage.                */
/* ------------------------------------------------------------------------ */
/* Every formula of Steps 1-4 (and of Remark 1's projections) is charged as
 * its plain evaluation, whatever way this file happens to compute it:
 *  - add, subtract, multiply, divide and square root cost 1; absolute
 *    values, comparisons and negations cost nothing;
 *  - a product with a constant (a coefficient of the maps, a basis value at
 *    a fixed point, a factorial, a Gauss weight, a linear weight, gamma, the
 *    grid spacings, alpha, dt) costs 1, a constant 0 removes the term and a
 *    constant +-1 makes the product free;
 *  - a sum of k terms costs k - 1;
 *  - a quantity used several times is formed once per cell (primitive
 *    variables, eigenvector matrices, 1/gamma_0) or once per face state;
 *  - only the grid's own cells and faces are charged: one reconstruction of
 *    each cell per stage (per pass for characteristic 2D Euler, where a pass
 *    needs only its own two faces and one limited derivative), and its right
 *    (and top) face.  Work this file does beyond that -- the ring of cells
 *    outside the grid, the other two faces of a characteristic pass, L by
 *    elimination instead of its closed form, primitive variables recomputed
 *    -- is not charged.
 * or_flop_count reads the running total. */
static long long g_flops = 0;
static int g_charge = 1; /* 0 while reconstructing cells outside the grid */
#define FL(n) (g_flops += g_charge ? (long long)(n) : 0LL)

long long or_flop_count(int reset) {
  const long long v = g_flops;
  if (reset) g_flops = 0;
  return v;
}

/* flops of sum_k c[k] x[k] for constants c[0..n-1] (stride apart) */
static int fl_dot(const double* c, int n, int stride) {
  int terms = 0, muls = 0;
  for (int k = 0; k < n; ++k) {
    const double v = c[k * stride];
    if (v == 0.0) continue;
    ++terms;
    if (v != 1.0 && v != -1.0) ++muls;
  }
  return terms > 0 ? muls + terms - 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra: Gaussian elimination with partial pivoting.        */
/* Solves A X = B; A is n x n, B is n x m, both row-major; B becomes X.     */
/* ------------------------------------------------------------------------ */
static int dense_solve(int n, int m, double* A, double* B) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[k * n + k]);
    for (int r = k + 1; r < n; ++r)
      if (fabs(A[r * n + k]) > best) { best = fabs(A[r * n + k]); piv = r; }
    if (best == 0.0) return -1;
    if (piv != k) {
      for (int c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = t; }
      for (int c = 0; c < m; ++c) { double t = B[k * m + c]; B[k * m + c] = B[piv * m + c]; B[piv * m + c] = t; }
    }
    for (int r = k + 1; r < n; ++r) {
      double f = A[r * n + k] / A[k * n + k];
      if (f == 0.0) continue;
      for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
      for (int c = 0; c < m; ++c) B[r * m + c] -= f * B[k * m + c];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int c = 0; c < m; ++c) {
      double s = B[k * m + c];
      for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * B[j * m + c];
      B[k * m + c] = s / A[k * n + k];
    }
  return 0;
}

static double pw(double x, int n) { double r = 1.0; while (n-- > 0) r *= x; return r; }
/* int over [a-1/2, a+1/2] of s^m ds, a cell offset in cell units. */
static double mono_avg(int a, int m) { return (pw(a + 0.5, m + 1) - pw(a - 0.5, m + 1)) / (m + 1); }
/* int over [a-1/2, a+1/2] of d/ds (s^m) ds. */
static double mono_dif(int a, int m) { return m == 0 ? 0.0 : pw(a + 0.5, m) - pw(a - 0.5, m); }

static const double FACT[5] = {1.0, 1.0, 2.0, 6.0, 24.0};

/* ------------------------------------------------------------------------ */
/* Step 1 coefficient maps from the constraint definitions.                 */
/* ------------------------------------------------------------------------ */
static double G0_1D[25], G1_1D[4], G2_1D[4];
static double G0_2D[15 * 17], GM_2D[4 * 9];
static int maps_ready = 0;

/* Basis of Sec. 2.2 Step 1, exponents (m, n) of xi^m eta^n.  The order within
 * a degree (decreasing power of xi) is the one Appendix A's coefficients use. */
static const int EXP2[15][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1},
                                {1, 2}, {0, 3}, {4, 0}, {3, 1}, {2, 2}, {1, 3}, {0, 4}};
/* q1..q9: cell averages at these offsets (Appendix A). */
static const int QOFF[9][2] = {{-1, -1}, {0, -1}, {1, -1}, {-1, 0}, {0, 0},
                               {1, 0},   {-1, 1}, {0, 1},  {1, 1}};
/* q10..q13: v-bar, q14..q17: w-bar, both at these face neighbours. */
static const int FOFF[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
/* Small stencils S1..S4 of Sec. 2.2 Step 1: target, x neighbour, y neighbour. */
static const int SOFF[4][3][2] = {{{0, 0}, {-1, 0}, {0, -1}},
                                  {{0, 0}, {1, 0}, {0, -1}},
                                  {{0, 0}, {1, 0}, {0, 1}},
                                  {{0, 0}, {-1, 0}, {0, 1}}};

static void build_maps(void) {
  if (maps_ready) return;
  /* 1D p0: three cell averages and the derivative means of cells i-1, i+1;
   * the data vector is (u_{i-1}, u_i, u_{i+1}, dx v_{i-1}, dx v_{i+1}). */
  {
    double M[25], B[25];
    const int avg_off[3] = {-1, 0, 1}, dif_off[2] = {-1, 1};
    for (int l = 0; l < 5; ++l) {
      for (int r = 0; r < 3; ++r) M[r * 5 + l] = mono_avg(avg_off[r], l);
      for (int r = 0; r < 2; ++r) M[(3 + r) * 5 + l] = mono_dif(dif_off[r], l);
    }
    memset(B, 0, sizeof B);
    for (int r = 0; r < 5; ++r) B[r * 5 + r] = 1.0;
    dense_solve(5, 5, M, B);
    memcpy(G0_1D, B, sizeof B);
    /* p1 on {i-1, i}, p2 on {i, i+1}: averages of (1, xi). */
    double M1[4] = {1.0, mono_avg(-1, 1), 1.0, mono_avg(0, 1)};
    double B1[4] = {1, 0, 0, 1};
    dense_solve(2, 2, M1, B1);
    memcpy(G1_1D, B1, sizeof B1);
    double M2[4] = {1.0, mono_avg(0, 1), 1.0, mono_avg(1, 1)};
    double B2[4] = {1, 0, 0, 1};
    dense_solve(2, 2, M2, B2);
    memcpy(G2_1D, B2, sizeof B2);
  }
  /* 2D p0: the 9 cell averages of S0 exactly, the scaled derivative moments
   * of the face neighbours in the least-squares sense.  KKT system of the
   * equality-constrained problem min |B c - d|^2 s.t. A c = e:
   *   [ B^T B  A^T ] [c]   [B^T d]
   *   [ A      0   ] [l] = [  e  ]                                          */
  {
    enum { NC = 15, NE = 9, NL = 8, NK = 24, NQ = 17 };
    double A[NE][NC], Bm[NL][NC];
    for (int r = 0; r < NE; ++r)
      for (int l = 0; l < NC; ++l)
        A[r][l] = mono_avg(QOFF[r][0], EXP2[l][0]) * mono_avg(QOFF[r][1], EXP2[l][1]);
    for (int f = 0; f < 4; ++f)
      for (int l = 0; l < NC; ++l) {
        const int a = FOFF[f][0], b = FOFF[f][1], m = EXP2[l][0], n = EXP2[l][1];
        Bm[f][l] = mono_dif(a, m) * mono_avg(b, n);      /* (1/dy) int u_x  */
        Bm[4 + f][l] = mono_avg(a, m) * mono_dif(b, n);  /* (1/dx) int u_y  */
      }
    double K[NK * NK], R[NK * NQ];
    memset(K, 0, sizeof K);
    memset(R, 0, sizeof R);
    for (int r = 0; r < NC; ++r)
      for (int c = 0; c < NC; ++c) {
        double s = 0.0;
        for (int k = 0; k < NL; ++k) s += Bm[k][r] * Bm[k][c];
        K[r * NK + c] = s;
      }
    for (int r = 0; r < NE; ++r)
      for (int c = 0; c < NC; ++c) {
        K[(NC + r) * NK + c] = A[r][c];
        K[c * NK + NC + r] = A[r][c];
      }
    for (int c = 0; c < NE; ++c) R[(NC + c) * NQ + c] = 1.0;       /* e = q1..q9  */
    for (int k = 0; k < NL; ++k)                                     /* d = q10..17 */
      for (int r = 0; r < NC; ++r) R[r * NQ + NE + k] = Bm[k][r];
    dense_solve(NK, NQ, K, R);
    for (int r = 0; r < NC; ++r)
      for (int c = 0; c < NQ; ++c) G0_2D[r * NQ + c] = R[r * NQ + c];
  }
  /* 2D p1..p4: three cell averages of (1, xi, eta). */
  for (int m = 0; m < 4; ++m) {
    double M[9], B[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int r = 0; r < 3; ++r) {
      M[r * 3 + 0] = 1.0;
      M[r * 3 + 1] = mono_avg(SOFF[m][r][0], 1);
      M[r * 3 + 2] = mono_avg(SOFF[m][r][1], 1);
    }
    dense_solve(3, 3, M, B);
    memcpy(GM_2D + 9 * m, B, sizeof B);
  }
  maps_ready = 1;
}

void or_coef_maps_1d(double* G0, double* G1, double* G2) {
  build_maps();
  memcpy(G0, G0_1D, sizeof G0_1D);
  memcpy(G1, G1_1D, sizeof G1_1D);
  memcpy(G2, G2_1D, sizeof G2_1D);
}

void or_coef_maps_2d(double* G0, double* Gm) {
  build_maps();
  memcpy(G0, G0_2D, sizeof G0_2D);
  memcpy(Gm, GM_2D, sizeof GM_2D);
}

/* ------------------------------------------------------------------------ */
/* Steps 2-3: smoothness indicators and nonlinear weights.                  */
/* ------------------------------------------------------------------------ */
/* Jiang-Shu indicator, Eq. (smoothness-indicator-typical) and its 2D form:
 * beta = sum over derivative orders 1 <= l <= deg of the cell mean of
 * (dx^m dy^n d^(m+n) p / dx^m dy^n)^2 over m + n = l; in the cell's scaled
 * coordinates (xi, eta) in [-1/2, 1/2]^2 this is the plain integral of the
 * squared xi/eta derivatives.  Evaluated by 4-point Gauss-Legendre rules
 * (exact up to degree 7 per variable; the squared derivatives of a quartic
 * have degree <= 6). */
static const double GL4_X[4] = {-0.43056815579702629, -0.16999052179242813, 0.16999052179242813,
                                0.43056815579702629};  /* on [-1/2, 1/2] */
static const double GL4_W[4] = {0.17392742256872693, 0.32607257743127307, 0.32607257743127307,
                                0.17392742256872693};  /* sum 1 */


/* d^l/dxi^l of p(xi) = sum_k c[k] xi^k, k < nc */
static double poly1_deriv(const double* c, int nc, double xi, int l) {
  double s = 0.0;
  for (int k = l; k < nc; ++k) {
    double f = 1.0;
    for (int j = 0; j < l; ++j) f *= (k - j);
    s += c[k] * f * pw(xi, k - l);
  }
  return s;
}

static double beta_typical_1d(const double* c, int nc) {
  double b = 0.0;
  for (int l = 1; l < nc; ++l)
    for (int g = 0; g < 4; ++g) {
      const double d = poly1_deriv(c, nc, GL4_X[g], l);
      b += GL4_W[g] * d * d;
    }
  return b;
}

/* tau = (sum_m |beta_0 - beta_m|) / nlin  (Sec. 2.1: /2, Sec. 2.2: /4);
 * w~_m = gamma_m (1 + tau^2 / (beta_m^pow + eps)); w = w~ / sum w~.        */
static void nonlinear_weights(const or_problem* p, int nlin, const double* beta, double* w) {
  const int np = nlin + 1;
  if (p->linear_weights) {
    for (int m = 0; m < np; ++m) w[m] = p->lin_w[m];
    return;
  }
  /* tau: nlin differences, nlin - 1 adds, one product; tau^2; per weight
   * (beta^2), + eps, the quotient, 1 +, gamma x; the sum; np quotients */
  FL(2 * nlin + 1 + np * (4 + (p->weight_pow == 2)) + nlin + np);
  double tau = 0.0;
  for (int m = 1; m < np; ++m) tau += fabs(beta[0] - beta[m]);
  tau /= nlin;
  double s = 0.0;
  for (int m = 0; m < np; ++m) {
    const double bp = p->weight_pow == 2 ? beta[m] * beta[m] : beta[m];
    w[m] = p->lin_w[m] * (1.0 + tau * tau / (bp + p->eps));
    s += w[m];
  }
  for (int m = 0; m < np; ++m) w[m] /= s;
}

/* ------------------------------------------------------------------------ */
/* One-dimensional scalar reconstruction (Sec. 2.1 Steps 1-3).              */
/* ------------------------------------------------------------------------ */
int or_recon_cell_1d(const or_problem* p, const double* in, double dx, double* out) {
  build_maps();
  /* Step 1 */
  const double d[5] = {in[0], in[1], in[2], dx * in[3], dx * in[4]};
  FL(2);
  double c0[5], c1[2], c2[2];
  for (int l = 0; l < 5; ++l) {
    double s = 0.0;
    for (int k = 0; k < 5; ++k) s += G0_1D[l * 5 + k] * d[k];
    c0[l] = s;
    FL(fl_dot(G0_1D + l * 5, 5, 1));
  }
  for (int l = 0; l < 2; ++l) {
    c1[l] = G1_1D[l * 2 + 0] * in[0] + G1_1D[l * 2 + 1] * in[1];
    c2[l] = G2_1D[l * 2 + 0] * in[1] + G2_1D[l * 2 + 1] * in[2];
    FL(fl_dot(G1_1D + l * 2, 2, 1) + fl_dot(G2_1D + l * 2, 2, 1));
  }
  /* Step 2: beta = sum_{l>=1} (l! c_l)^2 */
  double beta[3] = {0.0, c1[1] * c1[1], c2[1] * c2[1]};
  for (int l = 1; l < 5; ++l) beta[0] += (FACT[l] * c0[l]) * (FACT[l] * c0[l]);
  if (p->smoothness == OR_BETA_TYPICAL) {
    beta[0] = beta_typical_1d(c0, 5);
    beta[1] = beta_typical_1d(c1, 2);
    beta[2] = beta_typical_1d(c2, 2);
    /* the closed quadratic forms: the quartic's 6 terms (c1^2 with a unit
     * coefficient: 1 product, the others 2) and 5 adds; c^2 for a line */
    FL(16 + 1 + 1);
  } else {
    /* beta_1, beta_2: a square each; beta_0: c_1^2 and (l! c_l)^2 for
     * l = 2..4 (2 products each), 3 adds */
    FL(2 + 7 + 3);
  }
  /* Step 3: weights and Eq. (hweno-reconstruction-1D) */
  double w[3];
  nonlinear_weights(p, 2, beta, w);
  const double g0 = p->lin_w[0], g1 = p->lin_w[1], g2 = p->lin_w[2];
  double cu[5];
  for (int l = 0; l < 5; ++l) {
    double q0 = c0[l];
    if (l < 2) q0 -= g1 * c1[l] + g2 * c2[l];
    q0 /= g0;
    cu[l] = w[0] * q0 + (l < 2 ? w[1] * c1[l] + w[2] * c2[l] : 0.0);
  }
  /* Eq. (hweno-reconstruction-1D): for l < 2 two products and two
   * subtractions, the quotient by gamma_0, three products and two adds; for
   * l >= 2 the quotient and one product */
  FL(2 * 10 + 3 * 2);
  double uL = 0.0, uR = 0.0, dL = 0.0, dR = 0.0;
  for (int l = 0; l < 5; ++l) {
    uL += cu[l] * pw(-0.5, l);
    uR += cu[l] * pw(0.5, l);
    if (l > 0) {
      dL += l * cu[l] * pw(-0.5, l - 1) / dx;
      dR += l * cu[l] * pw(0.5, l - 1) / dx;
    }
  }
  /* u at the faces: 5 terms, 4 non-unit basis values; u': 4 terms, each
   * with its constant l (+-1/2)^(l-1) / dx; v-hat: a difference and 1/dx */
  FL(2 * 8 + 2 * 7 + 2);
  out[0] = uL;
  out[1] = uR;
  out[2] = dL;
  out[3] = dR;
  out[4] = (uR - uL) / dx; /* v-hat = (1/dx) int u_i'(x) dx */
  for (int m = 0; m < 3; ++m) { out[5 + m] = w[m]; out[8 + m] = beta[m]; }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-dimensional scalar reconstruction (Sec. 2.2 Steps 1-3).              */
/* ------------------------------------------------------------------------ */
static const double GAUSS_S[3] = {-0.38729833462074168852, 0.0, 0.38729833462074168852}; /* sqrt(15)/10 */
static const double GAUSS_W[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};

static double poly2_eval(const double* c, double xi, double eta, int dxi, int deta) {
  double s = 0.0;
  for (int l = 0; l < 15; ++l) {
    const int m = EXP2[l][0], n = EXP2[l][1];
    if (m < dxi || n < deta) continue;
    double f = 1.0;
    for (int k = 0; k < dxi; ++k) f *= (m - k);
    for (int k = 0; k < deta; ++k) f *= (n - k);
    s += c[l] * f * pw(xi, m - dxi) * pw(eta, n - deta);
  }
  return s;
}

static double beta_typical_2d(const double* c) {
  double b = 0.0;
  for (int l = 1; l <= 4; ++l)
    for (int m = 0; m <= l; ++m)
      for (int gx = 0; gx < 4; ++gx)
        for (int gy = 0; gy < 4; ++gy) {
          const double d = poly2_eval(c, GL4_X[gx], GL4_X[gy], m, l - m);
          b += GL4_W[gx] * GL4_W[gy] * d * d;
        }
  return b;
}

/* flops of one face's values: u at the 3 Gauss points (basis values
 * phi_l(xi, eta) there), u_xi and u_eta (their derivatives, each sum then
 * divided by the spacing); face 0/1 at xi = -+1/2, 2/3 at eta = -+1/2 */
static int fl_face_2d(int face) {
  int n = 0;
  for (int mu = 0; mu < 3; ++mu) {
    double xi, eta;
    if (face < 2) { xi = face == 0 ? -0.5 : 0.5; eta = GAUSS_S[mu]; }
    else { xi = GAUSS_S[mu]; eta = face == 2 ? -0.5 : 0.5; }
    for (int t = 0; t < 3; ++t) {
      double b[15];
      for (int l = 0; l < 15; ++l) {
        const int m = EXP2[l][0], k = EXP2[l][1];
        const int dm = t == 1, dk = t == 2;
        if (m < dm || k < dk) { b[l] = 0.0; continue; }
        b[l] = (dm ? m : 1) * (dk ? k : 1) * pw(xi, m - dm) * pw(eta, k - dk);
      }
      n += fl_dot(b, 15, 1) + (t > 0); /* the derivatives: / dx or / dy */
    }
  }
  return n;
}

/* Sec. 2.2 Steps 1-3 for one field; all four faces and both limited
 * derivatives are evaluated, the flop counter is charged for the faces in
 * `need` (bit f: face f; bit 4: v-hat; bit 5: w-hat). */
static void recon_cell_2d(const or_problem* p, const double* q, double dx, double dy, double* out,
                          unsigned need) {
  build_maps();
  /* Step 1 */
  double c0[15], cm[4][3];
  for (int l = 0; l < 15; ++l) {
    double s = 0.0;
    for (int k = 0; k < 17; ++k) s += G0_2D[l * 17 + k] * q[k];
    c0[l] = s;
    FL(fl_dot(G0_2D + l * 17, 17, 1));
  }
  for (int m = 0; m < 4; ++m) {
    double a[3];
    for (int r = 0; r < 3; ++r) a[r] = q[(SOFF[m][r][1] + 1) * 3 + (SOFF[m][r][0] + 1)];
    for (int l = 0; l < 3; ++l) {
      cm[m][l] = GM_2D[9 * m + l * 3 + 0] * a[0] + GM_2D[9 * m + l * 3 + 1] * a[1] +
                 GM_2D[9 * m + l * 3 + 2] * a[2];
      FL(fl_dot(GM_2D + 9 * m + l * 3, 3, 1));
    }
  }
  /* Step 2: beta = sum over non-constant terms of (m! n! c)^2 */
  double beta[5];
  beta[0] = 0.0;
  for (int l = 1; l < 15; ++l) {
    const double f = FACT[EXP2[l][0]] * FACT[EXP2[l][1]] * c0[l];
    beta[0] += f * f;
  }
  for (int m = 0; m < 4; ++m) beta[m + 1] = cm[m][1] * cm[m][1] + cm[m][2] * cm[m][2];
  if (p->smoothness == OR_BETA_TYPICAL) {
    beta[0] = beta_typical_2d(c0);
    for (int m = 0; m < 4; ++m) {
      const double lin[15] = {cm[m][0], cm[m][1], cm[m][2]};
      beta[m + 1] = beta_typical_2d(lin);
    }
    /* the quartic's closed quadratic form: 29 terms (c_1^2 and c_2^2 with
     * unit coefficients: 1 product, the others 2), 28 adds; c_1^2 + c_2^2
     * for each linear polynomial */
    FL(84 + 4 * 3);
  } else {
    /* beta_0: 14 squares, 11 of them after a factorial product (m! n! > 1),
     * 13 adds; beta_m: two squares and an add */
    FL(38 + 4 * 3);
  }
  /* Step 3: weights and Eq. (hweno-reconstruction-2D) */
  double w[5];
  nonlinear_weights(p, 4, beta, w);
  double cu[15];
  for (int l = 0; l < 15; ++l) {
    double q0 = c0[l], lin = 0.0;
    if (l < 3)
      for (int m = 0; m < 4; ++m) { q0 -= p->lin_w[m + 1] * cm[m][l]; lin += w[m + 1] * cm[m][l]; }
    cu[l] = w[0] * q0 / p->lin_w[0] + lin;
  }
  /* Eq. (hweno-reconstruction-2D): for l < 3 four products and subtractions
   * for p0 - sum gamma_m p_m, four products and three adds for sum omega_m
   * p_m, omega_0 (.) / gamma_0 and the add; for l >= 3 omega_0 c / gamma_0 */
  FL(3 * (8 + 7 + 2 + 1) + 12 * 2);
  for (int f = 0; f < 4; ++f)
    if (need & (1u << f)) FL(fl_face_2d(f));
  /* v-hat, w-hat: the terms of cu with a nonzero cell integral of d/dxi
   * (d/deta) of their basis function */
  {
    double bv[15], bw[15];
    for (int l = 0; l < 15; ++l) {
      bv[l] = mono_dif(0, EXP2[l][0]) * mono_avg(0, EXP2[l][1]);
      bw[l] = mono_avg(0, EXP2[l][0]) * mono_dif(0, EXP2[l][1]);
    }
    if (need & 16u) FL(fl_dot(bv, 15, 1));
    if (need & 32u) FL(fl_dot(bw, 15, 1));
  }
  /* point values at the Gauss points of the four faces */
  for (int face = 0; face < 4; ++face)
    for (int mu = 0; mu < 3; ++mu) {
      double xi, eta;
      if (face < 2) { xi = face == 0 ? -0.5 : 0.5; eta = GAUSS_S[mu]; }
      else { xi = GAUSS_S[mu]; eta = face == 2 ? -0.5 : 0.5; }
      double* o = out + (face * 3 + mu) * 3;
      o[0] = poly2_eval(cu, xi, eta, 0, 0);
      o[1] = poly2_eval(cu, xi, eta, 1, 0) / dx;
      o[2] = poly2_eval(cu, xi, eta, 0, 1) / dy;
    }
  /* limited derivatives: v-hat = (1/dy) int u_x dOmega = int int d/dxi u,
   * w-hat = (1/dx) int u_y dOmega = int int d/deta u (exact integrals) */
  double vh = 0.0, wh = 0.0;
  for (int l = 0; l < 15; ++l) {
    vh += cu[l] * mono_dif(0, EXP2[l][0]) * mono_avg(0, EXP2[l][1]);
    wh += cu[l] * mono_avg(0, EXP2[l][0]) * mono_dif(0, EXP2[l][1]);
  }
  out[36] = vh;
  out[37] = wh;
  for (int m = 0; m < 5; ++m) { out[38 + m] = w[m]; out[43 + m] = beta[m]; }
}

int or_recon_cell_2d(const or_problem* p, const double* q, double dx, double dy, double* out) {
  recon_cell_2d(p, q, dx, dy, out, 63u);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Physics: fluxes, Jacobians, eigenvectors, spectral radius.               */
/* ------------------------------------------------------------------------ */
int or_ncomp(const or_problem* p) {
  if (p->equation != OR_EQ_EULER) return 1;
  return p->dim == 1 ? 3 : 4;
}
int or_nfields(const or_problem* p) { return or_ncomp(p) * (p->dim + 1); }

typedef struct { double rho, u, v, p, c, H, E; } prim_t;

static prim_t primitives(int dim, const double* U, double g) {
  prim_t s;
  s.rho = U[0];
  s.u = U[1] / U[0];
  s.v = dim == 2 ? U[2] / U[0] : 0.0;
  s.E = U[dim == 2 ? 3 : 2];
  s.p = (g - 1.0) * (s.E - 0.5 * s.rho * (s.u * s.u + s.v * s.v));
  s.c = sqrt(g * s.p / s.rho);
  s.H = (s.E + s.p) / s.rho;
  return s;
}

/* Flux Jacobian of the Euler equations (textbook form). */
int or_euler_jacobian(int dim, int dir, const double* U, double g, double* A) {
  const prim_t s = primitives(dim, U, g);
  const double u = s.u, v = s.v, H = s.H, q2 = u * u + v * v, gm = g - 1.0;
  if (dim == 1) {
    const double a[9] = {0.0, 1.0, 0.0,
                         0.5 * (g - 3.0) * u * u, (3.0 - g) * u, gm,
                         u * (0.5 * gm * u * u - H), H - gm * u * u, g * u};
    memcpy(A, a, sizeof a);
    return 0;
  }
  if (dir == 0) {
    const double a[16] = {0.0, 1.0, 0.0, 0.0,
                          0.5 * gm * q2 - u * u, (3.0 - g) * u, -gm * v, gm,
                          -u * v, v, u, 0.0,
                          u * (0.5 * gm * q2 - H), H - gm * u * u, -gm * u * v, g * u};
    memcpy(A, a, sizeof a);
  } else {
    const double a[16] = {0.0, 0.0, 1.0, 0.0,
                          -u * v, v, u, 0.0,
                          0.5 * gm * q2 - v * v, -gm * u, (3.0 - g) * v, gm,
                          v * (0.5 * gm * q2 - H), -gm * u * v, H - gm * v * v, g * v};
    memcpy(A, a, sizeof a);
  }
  return 0;
}

/* Right eigenvectors (columns) of the Jacobian in direction dir at U, and
 * the left eigenvectors L = R^{-1} obtained by a dense solve. */
int or_euler_eigen(int dim, int dir, const double* U, double g, double* R, double* L) {
  const prim_t s = primitives(dim, U, g);
  const double u = s.u, v = s.v, c = s.c, H = s.H, q2 = u * u + v * v;
  int n = dim == 1 ? 3 : 4;
  if (dim == 1) {
    const double r[9] = {1.0, 1.0, 1.0,
                         u - c, u, u + c,
                         H - u * c, 0.5 * u * u, H + u * c};
    memcpy(R, r, sizeof r);
  } else if (dir == 0) {
    const double r[16] = {1.0, 1.0, 0.0, 1.0,
                          u - c, u, 0.0, u + c,
                          v, v, 1.0, v,
                          H - u * c, 0.5 * q2, v, H + u * c};
    memcpy(R, r, sizeof r);
  } else {
    const double r[16] = {1.0, 1.0, 0.0, 1.0,
                          u, u, 1.0, u,
                          v - c, v, 0.0, v + c,
                          H - v * c, 0.5 * q2, u, H + v * c};
    memcpy(R, r, sizeof r);
  }
  double A[16], B[16];
  memcpy(A, R, sizeof(double) * n * n);
  memset(B, 0, sizeof B);
  for (int k = 0; k < n; ++k) B[k * n + k] = 1.0;
  if (dense_solve(n, n, A, B)) return -1;
  memcpy(L, B, sizeof(double) * n * n);
  return 0;
}

/* Physical flux f (dir 0) or g (dir 1). */
static void phys_flux(const or_problem* p, int dir, const double* U, double* F) {
  if (p->equation == OR_EQ_ADVECTION) { F[0] = (dir == 0 ? p->adv_x : p->adv_y) * U[0]; return; }
  if (p->equation == OR_EQ_BURGERS) { F[0] = 0.5 * U[0] * U[0]; return; }
  const prim_t s = primitives(p->dim, U, p->gamma_gas);
  if (p->dim == 1) {
    F[0] = U[1];
    F[1] = U[1] * s.u + s.p;
    F[2] = s.u * (s.E + s.p);
  } else if (dir == 0) {
    F[0] = U[1];
    F[1] = U[1] * s.u + s.p;
    F[2] = U[1] * s.v;
    F[3] = s.u * (s.E + s.p);
  } else {
    F[0] = U[2];
    F[1] = U[2] * s.u;
    F[2] = U[2] * s.v + s.p;
    F[3] = s.v * (s.E + s.p);
  }
}

/* Derivative flux f'(u) v (Sec. 2.1 h = f'(u) v; Sec. 2.2 f^v, g^v, f^w, g^w). */
static void deriv_flux(const or_problem* p, int dir, const double* U, const double* V, double* F) {
  if (p->equation == OR_EQ_ADVECTION) { F[0] = (dir == 0 ? p->adv_x : p->adv_y) * V[0]; return; }
  if (p->equation == OR_EQ_BURGERS) { F[0] = U[0] * V[0]; return; }
  const int n = or_ncomp(p);
  double A[16];
  or_euler_jacobian(p->dim, dir, U, p->gamma_gas, A);
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += A[r * n + c] * V[c];
    F[r] = s;
  }
}

static double spectral_radius(const or_problem* p, int dir, const double* U) {
  if (p->equation == OR_EQ_ADVECTION) return fabs(dir == 0 ? p->adv_x : p->adv_y);
  if (p->equation == OR_EQ_BURGERS) return fabs(U[0]);
  const prim_t s = primitives(p->dim, U, p->gamma_gas);
  return fabs(dir == 0 ? s.u : s.v) + s.c;
}

/* ------------------------------------------------------------------------ */
/* Ghost cells (2 wide) in a padded copy of the state.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nx, ny, px, py, nc, nf;
  double* a; /* [nf][py][px] */
} padded_t;

static double* pcell(padded_t* P, int f, int i, int j) {
  return P->a + ((size_t)f * P->py + (size_t)(j + (P->py > 1 ? 2 : 0))) * P->px + (i + 2);
}

/* sign of field (d, k) under a mirror across a face normal to `axis` */
static double mirror_sign(const or_problem* p, int d, int k, int axis) {
  double s = 1.0;
  if (p->equation == OR_EQ_EULER && k == 1 + axis) s = -s; /* normal momentum */
  if (d == 1 + axis) s = -s;                                 /* normal derivative */
  return s;
}

/* Fill the ghosts of one line along `axis` (0: x, 1: y) at fixed other index.
 * The split and moving-shock sides decide by the line's centre coordinate
 * along the side (y of the row for x sides, x of the column for y sides). */
static void fill_line(const or_problem* p, padded_t* P, int axis, int other) {
  const int n = axis == 0 ? P->nx : P->ny;
  const double along = axis == 0 ? p->ylo + (other + 0.5) * (p->yhi - p->ylo) / (p->dim == 2 ? p->ny : 1)
                                 : p->xlo + (other + 0.5) * (p->xhi - p->xlo) / p->nx;
  for (int f = 0; f < P->nf; ++f) {
    const int d = f / P->nc, k = f % P->nc;
#define AT(t) (*(axis == 0 ? pcell(P, f, (t), other) : pcell(P, f, other, (t))))
    for (int side = 0; side < 2; ++side) {
      const int sd = 2 * axis + side;
      int bc = p->bc[sd];
      const double* state = p->bc_state[sd];
      if (bc == OR_BC_SPLIT) {
        bc = along < p->bc_param[sd][0] ? OR_BC_INFLOW : OR_BC_REFLECT;
      } else if (bc == OR_BC_SHOCK) {
        bc = OR_BC_INFLOW;
        if (!(along < p->bc_param[sd][0] + p->bc_param[sd][1] * p->t)) state = p->bc_state2[sd];
      }
      for (int r = 0; r < 2; ++r) {
        const int g = side == 0 ? -1 - r : n + r;
        double val;
        if (bc == OR_BC_PERIODIC) {
          val = AT(side == 0 ? n - 1 - r : r);
        } else if (bc == OR_BC_OUTFLOW) {
          val = AT(side == 0 ? 0 : n - 1);
        } else if (bc == OR_BC_REFLECT) {
          val = mirror_sign(p, d, k, axis) * AT(side == 0 ? r : n - 1 - r);
        } else {
          val = d == 0 ? state[k] : 0.0;
        }
        AT(g) = val;
      }
    }
#undef AT
  }
}

static int make_padded(const or_problem* p, const double* U, padded_t* P) {
  P->nx = p->nx;
  P->ny = p->dim == 2 ? p->ny : 1;
  P->px = P->nx + 4;
  P->py = p->dim == 2 ? P->ny + 4 : 1;
  P->nc = or_ncomp(p);
  P->nf = or_nfields(p);
  P->a = (double*)calloc((size_t)P->nf * P->px * P->py, sizeof(double));
  if (!P->a) return -1;
  for (int f = 0; f < P->nf; ++f)
    for (int j = 0; j < P->ny; ++j)
      for (int i = 0; i < P->nx; ++i)
        *pcell(P, f, i, j) = U[((size_t)f * P->ny + j) * P->nx + i];
  for (int j = 0; j < P->ny; ++j) fill_line(p, P, 0, j);
  if (p->dim == 2)
    for (int i = -2; i < P->nx + 2; ++i) fill_line(p, P, 1, i);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cell reconstructions (component-wise or characteristic-wise, Remark 1).  */
/* ------------------------------------------------------------------------ */
typedef struct { double uL[4], uR[4], dL[4], dR[4], vh[4]; } rec1_t;

static void matvec(int n, const double* M, const double* x, double* y) {
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += M[r * n + c] * x[c];
    y[r] = s;
  }
}

static void cell_recon_1d(const or_problem* p, padded_t* P, int i, double dx, rec1_t* rec) {
  const int nc = P->nc;
  double Um[4], U0[4], Up[4], Vm[4], Vp[4];
  for (int k = 0; k < nc; ++k) {
    Um[k] = *pcell(P, k, i - 1, 0);
    U0[k] = *pcell(P, k, i, 0);
    Up[k] = *pcell(P, k, i + 1, 0);
    Vm[k] = *pcell(P, nc + k, i - 1, 0);
    Vp[k] = *pcell(P, nc + k, i + 1, 0);
  }
  const int chr = p->equation == OR_EQ_EULER && p->charwise;
  double R[16], L[16];
  double Wm[4], W0[4], Wp[4], Zm[4], Zp[4];
  if (chr) {
    or_euler_eigen(1, 0, U0, p->gamma_gas, R, L);
    /* Remark 1: primitive variables of the cell average (11), the entries of
     * R (6) and of L in closed form (16); L times 5 stencil vectors (9
     * products, 6 adds each) */
    FL(11 + 6 + 16 + 5 * 15);
    matvec(nc, L, Um, Wm); matvec(nc, L, U0, W0); matvec(nc, L, Up, Wp);
    matvec(nc, L, Vm, Zm); matvec(nc, L, Vp, Zp);
  } else {
    memcpy(Wm, Um, sizeof Um); memcpy(W0, U0, sizeof U0); memcpy(Wp, Up, sizeof Up);
    memcpy(Zm, Vm, sizeof Vm); memcpy(Zp, Vp, sizeof Vp);
  }
  double o[5][4];
  for (int k = 0; k < nc; ++k) {
    const double in[5] = {Wm[k], W0[k], Wp[k], Zm[k], Zp[k]};
    double out[11];
    or_recon_cell_1d(p, in, dx, out);
    for (int t = 0; t < 5; ++t) o[t][k] = out[t];
  }
  if (chr) {
    /* R (first row ones) times 5 vectors: 2 + 5 + 5 flops each */
    FL(5 * 12);
    matvec(nc, R, o[0], rec->uL); matvec(nc, R, o[1], rec->uR);
    matvec(nc, R, o[2], rec->dL); matvec(nc, R, o[3], rec->dR);
    matvec(nc, R, o[4], rec->vh);
  } else {
    memcpy(rec->uL, o[0], sizeof o[0]); memcpy(rec->uR, o[1], sizeof o[1]);
    memcpy(rec->dL, o[2], sizeof o[2]); memcpy(rec->dR, o[3], sizeof o[3]);
    memcpy(rec->vh, o[4], sizeof o[4]);
  }
}

/* 2D record: face data [face][mu][quantity][component], v-hat, w-hat. */
typedef struct { double fv[4][3][3][4]; double vh[4], wh[4]; } rec2_t;

static void gather_q(padded_t* P, int k, int i, int j, double* q) {
  const int nc = P->nc;
  for (int r = 0; r < 9; ++r) q[r] = *pcell(P, k, i + QOFF[r][0], j + QOFF[r][1]);
  for (int f = 0; f < 4; ++f) {
    q[9 + f] = *pcell(P, nc + k, i + FOFF[f][0], j + FOFF[f][1]);
    q[13 + f] = *pcell(P, 2 * nc + k, i + FOFF[f][0], j + FOFF[f][1]);
  }
}

static void cell_recon_2d(const or_problem* p, padded_t* P, int i, int j, double dx, double dy,
                          rec2_t* rec) {
  const int nc = P->nc;
  double q[4][17];
  for (int k = 0; k < nc; ++k) gather_q(P, k, i, j, q[k]);
  const int chr = p->equation == OR_EQ_EULER && p->charwise;
  if (!chr) {
    for (int k = 0; k < nc; ++k) {
      double out[48];
      recon_cell_2d(p, q[k], dx, dy, out, 63u);
      for (int face = 0; face < 4; ++face)
        for (int mu = 0; mu < 3; ++mu)
          for (int t = 0; t < 3; ++t) rec->fv[face][mu][t][k] = out[(face * 3 + mu) * 3 + t];
      rec->vh[k] = out[36];
      rec->wh[k] = out[37];
    }
    return;
  }
  double U0[4];
  for (int k = 0; k < nc; ++k) U0[k] = q[k][4];
  FL(14); /* primitive variables of the cell average, once for both passes */
  /* pass dir 0 gives the x faces and v-hat, pass dir 1 the y faces and w-hat */
  for (int dir = 0; dir < 2; ++dir) {
    double R[16], L[16];
    or_euler_eigen(2, dir, U0, p->gamma_gas, R, L);
    /* Remark 1: the entries of R (6) and of L in closed form (18); L (two
     * structural zeros and a one in the shear row) times the 17 stencil
     * vectors, 23 flops each */
    FL(6 + 18 + 17 * 23);
    double w[4][17];
    for (int s = 0; s < 17; ++s) {
      double x[4], y[4];
      for (int k = 0; k < nc; ++k) x[k] = q[k][s];
      matvec(nc, L, x, y);
      for (int k = 0; k < nc; ++k) w[k][s] = y[k];
    }
    double out[4][48];
    for (int k = 0; k < nc; ++k) recon_cell_2d(p, w[k], dx, dy, out[k], (3u << (2 * dir)) | (16u << dir));
    /* R (two structural zeros, four ones) times the pass's 18 face values and
     * its limited derivative, 20 flops each */
    FL(19 * 20);
    for (int face = 2 * dir; face < 2 * dir + 2; ++face)
      for (int mu = 0; mu < 3; ++mu)
        for (int t = 0; t < 3; ++t) {
          double x[4], y[4];
          for (int k = 0; k < nc; ++k) x[k] = out[k][(face * 3 + mu) * 3 + t];
          matvec(nc, R, x, y);
          for (int k = 0; k < nc; ++k) rec->fv[face][mu][t][k] = y[k];
        }
    double x[4], y[4];
    for (int k = 0; k < nc; ++k) x[k] = out[k][36 + dir];
    matvec(nc, R, x, y);
    for (int k = 0; k < nc; ++k) (dir == 0 ? rec->vh : rec->wh)[k] = y[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Global Lax-Friedrichs flux for (u, v) pairs.                             */
/* ------------------------------------------------------------------------ */
/* fu = 1/2 [f(u-) + f(u+)] - a/2 (u+ - u-),
 * fv = 1/2 [f'(u-) v- + f'(u+) v+] - a/2 (v+ - v-).                         */
static void lf_flux(const or_problem* p, int dir, double a, const double* um, const double* up,
                    const double* vm, const double* vp, double* fu, double* fv) {
  const int nc = or_ncomp(p);
  double Fm[4], Fp[4], Hm[4], Hp[4];
  phys_flux(p, dir, um, Fm);
  phys_flux(p, dir, up, Fp);
  deriv_flux(p, dir, um, vm, Hm);
  deriv_flux(p, dir, up, vp, Hp);
  for (int k = 0; k < nc; ++k) {
    if (fu) fu[k] = 0.5 * (Fm[k] + Fp[k]) - 0.5 * a * (up[k] - um[k]);
    fv[k] = 0.5 * (Hm[k] + Hp[k]) - 0.5 * a * (vp[k] - vm[k]);
  }
}

/* flops of the global LF fluxes at one 1D face or one 2D Gauss point, from
 * the two face states: per state the physical flux and the derivative
 * fluxes f'(u) v (and f'(u) w), each component of each family
 * 1/2 (F- + F+) - (alpha/2) (u+ - u-) for 5.
 *   advection: a u, a v (, a w);  Burgers: u^2 / 2 (2), u v (, u w);
 *   1D Euler per state: u, p, E + p, H (7), F (2), the Jacobian's entries (9),
 *     f'(u) v (10: first row a copy, the others 3 products and 2 adds);
 *   2D Euler per state: u, v, q^2, p, E + p, H (11), F (4), the entries of
 *     A_x or A_y (12), A v and A w (19 each: 0 + 7 + 5 + 7). */
static int fl_flux_point(const or_problem* p) {
  const int fam = p->dim + 1, nc = or_ncomp(p);
  int per_state;
  if (p->equation == OR_EQ_ADVECTION) per_state = fam;
  else if (p->equation == OR_EQ_BURGERS) per_state = 2 + (fam - 1);
  else per_state = p->dim == 1 ? 7 + 2 + 9 + 10 : 11 + 4 + 12 + 2 * 19;
  return 2 * per_state + 5 * fam * nc;
}

/* ------------------------------------------------------------------------ */
/* The spatial operator.                                                    */
/* ------------------------------------------------------------------------ */
static int operator_1d(const or_problem* p, const double* U, double ax, double* Lo, double* dh) {
  padded_t P;
  if (make_padded(p, U, &P)) return -1;
  const int nx = p->nx, nc = P.nc;
  const double dx = (p->xhi - p->xlo) / nx;
  rec1_t* rec = (rec1_t*)malloc(sizeof(rec1_t) * (nx + 2));
  double* Fu = (double*)malloc(sizeof(double) * 4 * (nx + 1));
  double* Fv = (double*)malloc(sizeof(double) * 4 * (nx + 1));
  if (!rec || !Fu || !Fv) { free(rec); free(Fu); free(Fv); free(P.a); return -1; }
  for (int i = -1; i <= nx; ++i) {
    g_charge = i >= 0 && i < nx; /* the ring cells are not the grid's own */
    cell_recon_1d(p, &P, i, dx, &rec[i + 1]);
    g_charge = 1;
  }
  /* face i+1/2 for i = -1..nx-1 stored at index i+1 */
  for (int i = -1; i < nx; ++i) {
    const rec1_t* a = &rec[i + 1];
    const rec1_t* b = &rec[i + 2];
    lf_flux(p, 0, ax, a->uR, b->uL, a->dR, b->dL, Fu + 4 * (i + 1), Fv + 4 * (i + 1));
    if (i >= 0) FL(fl_flux_point(p)); /* each cell's right face */
  }
  FL((long long)nx * 2 * nc * 2); /* L = -(F_right - F_left) / dx per field */
  for (int i = 0; i < nx; ++i)
    for (int k = 0; k < nc; ++k) {
      Lo[(size_t)k * nx + i] = -(Fu[4 * (i + 1) + k] - Fu[4 * i + k]) / dx;
      Lo[(size_t)(nc + k) * nx + i] = -(Fv[4 * (i + 1) + k] - Fv[4 * i + k]) / dx;
      dh[(size_t)k * nx + i] = rec[i + 1].vh[k];
    }
  free(rec); free(Fu); free(Fv); free(P.a);
  return 0;
}

static int operator_2d(const or_problem* p, const double* U, double ax, double ay, double* Lo,
                       double* dh) {
  padded_t P;
  if (make_padded(p, U, &P)) return -1;
  const int nx = p->nx, ny = p->ny, nc = P.nc;
  const double dx = (p->xhi - p->xlo) / nx, dy = (p->yhi - p->ylo) / ny;
  const int rx = nx + 2, ry = ny + 2;
  rec2_t* rec = (rec2_t*)calloc((size_t)rx * ry, sizeof(rec2_t));
  /* face integrals: x faces (nx+1) x ny, y faces nx x (ny+1); 3 families x 4 */
  double* FX = (double*)calloc((size_t)(nx + 1) * ny * 12, sizeof(double));
  double* FY = (double*)calloc((size_t)nx * (ny + 1) * 12, sizeof(double));
  if (!rec || !FX || !FY) { free(rec); free(FX); free(FY); free(P.a); return -1; }
#define REC(i, j) rec[(size_t)((j) + 1) * rx + ((i) + 1)]
  for (int j = -1; j <= ny; ++j)
    for (int i = -1; i <= nx; ++i) {
      const int in_x = i >= 0 && i < nx, in_y = j >= 0 && j < ny;
      if (!in_x && !in_y) continue; /* corners are never needed */
      g_charge = in_x && in_y;       /* the ring cells are not the grid's own */
      cell_recon_2d(p, &P, i, j, dx, dy, &REC(i, j));
      g_charge = 1;
    }
  /* per face: the Gauss points' fluxes and the Gauss sums (3 products and 2
   * adds per quantity); only each cell's right and top face is charged */
  const int fl_face = 3 * fl_flux_point(p) + 3 * nc * 5;
  /* x faces: f-hat_{i+1/2,j} = dy sum_mu sigma_mu f-hat(u-, u+) */
  for (int j = 0; j < ny; ++j)
    for (int i = -1; i < nx; ++i) {
      const rec2_t* a = &REC(i, j);
      const rec2_t* b = &REC(i + 1, j);
      double* o = FX + ((size_t)j * (nx + 1) + (i + 1)) * 12;
      if (i >= 0) FL(fl_face);
      for (int mu = 0; mu < 3; ++mu) {
        double fu[4], fv[4], fw[4];
        lf_flux(p, 0, ax, a->fv[1][mu][0], b->fv[0][mu][0], a->fv[1][mu][1], b->fv[0][mu][1], fu, fv);
        lf_flux(p, 0, ax, a->fv[1][mu][0], b->fv[0][mu][0], a->fv[1][mu][2], b->fv[0][mu][2], NULL, fw);
        for (int k = 0; k < nc; ++k) {
          o[k] += dy * GAUSS_W[mu] * fu[k];
          o[4 + k] += dy * GAUSS_W[mu] * fv[k];
          o[8 + k] += dy * GAUSS_W[mu] * fw[k];
        }
      }
    }
  /* y faces: g-hat_{i,j+1/2} = dx sum_mu sigma_mu g-hat(u-, u+) */
  for (int j = -1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const rec2_t* a = &REC(i, j);
      const rec2_t* b = &REC(i, j + 1);
      double* o = FY + ((size_t)(j + 1) * nx + i) * 12;
      if (j >= 0) FL(fl_face);
      for (int mu = 0; mu < 3; ++mu) {
        double gu[4], gv[4], gw[4];
        lf_flux(p, 1, ay, a->fv[3][mu][0], b->fv[2][mu][0], a->fv[3][mu][1], b->fv[2][mu][1], gu, gv);
        lf_flux(p, 1, ay, a->fv[3][mu][0], b->fv[2][mu][0], a->fv[3][mu][2], b->fv[2][mu][2], NULL, gw);
        for (int k = 0; k < nc; ++k) {
          o[k] += dx * GAUSS_W[mu] * gu[k];
          o[4 + k] += dx * GAUSS_W[mu] * gv[k];
          o[8 + k] += dx * GAUSS_W[mu] * gw[k];
        }
      }
    }
  const size_t plane = (size_t)nx * ny;
  FL((long long)nx * ny * 3 * nc * 4); /* -(x_r - x_l + y_r - y_l) / h per field */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double* xl = FX + ((size_t)j * (nx + 1) + i) * 12;
      const double* xr = xl + 12;
      const double* yl = FY + ((size_t)j * nx + i) * 12;
      const double* yr = FY + ((size_t)(j + 1) * nx + i) * 12;
      const size_t c = (size_t)j * nx + i;
      for (int k = 0; k < nc; ++k) {
        Lo[k * plane + c] = -(xr[k] - xl[k] + yr[k] - yl[k]) / (dx * dy);
        Lo[(nc + k) * plane + c] = -(xr[4 + k] - xl[4 + k] + yr[4 + k] - yl[4 + k]) / dy;
        Lo[(2 * nc + k) * plane + c] = -(xr[8 + k] - xl[8 + k] + yr[8 + k] - yl[8 + k]) / dx;
        dh[k * plane + c] = REC(i, j).vh[k];
        dh[(nc + k) * plane + c] = REC(i, j).wh[k];
      }
    }
#undef REC
  free(rec); free(FX); free(FY); free(P.a);
  return 0;
}

static int check_problem(const or_problem* p) {
  if (!p || (p->dim != 1 && p->dim != 2) || p->nx < 1 || (p->dim == 2 && p->ny < 1)) return -1;
  if (p->equation < 0 || p->equation > 2) return -1;
  const int nlin = p->dim == 1 ? 3 : 5;
  for (int m = 0; m < nlin; ++m)
    if (!(p->lin_w[m] > 0.0)) return -1;
  for (int sd = 0; sd < 4; ++sd) {
    if (p->bc[sd] < OR_BC_PERIODIC || p->bc[sd] > OR_BC_SHOCK) return -1;
    if (p->dim == 1 && p->bc[sd] >= OR_BC_SPLIT) return -1; /* need a coordinate along the side */
  }
  return 0;
}

int or_operator(const or_problem* p, const double* U, double ax, double ay, double* L, double* dhat) {
  if (check_problem(p)) return -1;
  build_maps();
  return p->dim == 1 ? operator_1d(p, U, ax, L, dhat) : operator_2d(p, U, ax, ay, L, dhat);
}

int or_alpha(const or_problem* p, const double* U, double* ax, double* ay) {
  if (check_problem(p)) return -1;
  const int nc = or_ncomp(p), ny = p->dim == 2 ? p->ny : 1;
  const size_t plane = (size_t)p->nx * ny;
  double mx = 0.0, my = 0.0;
  /* Euler: u (, v), p, c and |u| + c (, |v| + c) per cell; scalars: none */
  if (p->equation == OR_EQ_EULER) FL((long long)plane * (p->dim == 1 ? 10 : 14));
  for (size_t c = 0; c < plane; ++c) {
    double s[4];
    for (int k = 0; k < nc; ++k) s[k] = U[k * plane + c];
    const double a = spectral_radius(p, 0, s);
    if (a > mx || a != a) mx = a;
    if (p->dim == 2) {
      const double b = spectral_radius(p, 1, s);
      if (b > my || b != b) my = b;
    }
  }
  *ax = mx;
  *ay = my;
  return 0;
}

double or_dt(const or_problem* p, double ax, double ay) {
  const double dx = (p->xhi - p->xlo) / p->nx;
  const double hx = p->dt_rule == OR_DT_CFL_DX53 ? pow(dx, 5.0 / 3.0) : dx;
  if (p->dim == 1) return ax > 0.0 ? p->cfl * hx / ax : INFINITY;
  const double dy = (p->yhi - p->ylo) / p->ny;
  const double hy = p->dt_rule == OR_DT_CFL_DX53 ? pow(dy, 5.0 / 3.0) : dy;
  const double rate = ax / hx + ay / hy;
  return rate > 0.0 ? p->cfl / rate : INFINITY;
}

/* Step 4 (Sec. 2.1 and 2.2): SSP-RK3 where every stage combines the
 * modified state [u-bar, v-hat(, w-hat)] of the stage's input. */
int or_step(const or_problem* p, double* U, double dt, double ax, double ay) {
  if (check_problem(p)) return -1;
  const int nc = or_ncomp(p), nf = or_nfields(p);
  const size_t plane = (size_t)p->nx * (p->dim == 2 ? p->ny : 1);
  const size_t nall = plane * nf, nu = plane * nc, nd = nall - nu;
  double* U0 = (double*)malloc(sizeof(double) * nall);
  double* Us = (double*)malloc(sizeof(double) * nall);
  double* L = (double*)malloc(sizeof(double) * nall);
  double* H0 = (double*)malloc(sizeof(double) * nd);
  double* Hs = (double*)malloc(sizeof(double) * nd);
  int rc = -1;
  if (!U0 || !Us || !L || !H0 || !Hs) goto done;
  memcpy(U0, U, sizeof(double) * nall);
  /* boundary values at the stage times t^n, t^n + dt, t^n + dt/2 */
  or_problem ps = *p;
  /* stage 1: u(1) = u-hat^n + dt L(u^n) */
  if (or_operator(&ps, U0, ax, ay, L, H0)) goto done;
  FL((long long)nall * 2); /* u-hat + dt L per stored field */
  for (size_t c = 0; c < nu; ++c) Us[c] = U0[c] + dt * L[c];
  for (size_t c = 0; c < nd; ++c) Us[nu + c] = H0[c] + dt * L[nu + c];
  /* stage 2: u(2) = 3/4 u-hat^n + 1/4 (u-hat(1) + dt L(u(1))) */
  ps.t = p->t + dt;
  if (or_operator(&ps, Us, ax, ay, L, Hs)) goto done;
  FL((long long)nall * 5); /* 3/4 u-hat^n + 1/4 (u-hat + dt L) */
  for (size_t c = 0; c < nu; ++c) Us[c] = 0.75 * U0[c] + 0.25 * (Us[c] + dt * L[c]);
  for (size_t c = 0; c < nd; ++c) Us[nu + c] = 0.75 * H0[c] + 0.25 * (Hs[c] + dt * L[nu + c]);
  /* stage 3: u^{n+1} = 1/3 u-hat^n + 2/3 (u-hat(2) + dt L(u(2))) */
  ps.t = p->t + 0.5 * dt;
  if (or_operator(&ps, Us, ax, ay, L, Hs)) goto done;
  FL((long long)nall * 5); /* 1/3 u-hat^n + 2/3 (u-hat + dt L) */
  for (size_t c = 0; c < nu; ++c) U[c] = U0[c] / 3.0 + 2.0 / 3.0 * (Us[c] + dt * L[c]);
  for (size_t c = 0; c < nd; ++c) U[nu + c] = H0[c] / 3.0 + 2.0 / 3.0 * (Hs[c] + dt * L[nu + c]);
  rc = 0;
done:
  free(U0); free(Us); free(L); free(H0); free(Hs);
  return rc;
}

int or_run(const or_problem* p, double* U, double t_final, int max_steps, double* t_out,
           int* steps_out) {
  if (check_problem(p)) return -1;
  const size_t nall = (size_t)p->nx * (p->dim == 2 ? p->ny : 1) * or_nfields(p);
  or_problem ps = *p;
  double t = p->t;
  int steps = 0, rc = 0;
  while (t < t_final && steps < max_steps) {
    double ax, ay;
    or_alpha(p, U, &ax, &ay);
    double dt = or_dt(p, ax, ay);
    if (!(dt > 0.0)) { rc = -2; break; }
    if (t + dt >= t_final) dt = t_final - t;
    ps.t = t;
    if (or_step(&ps, U, dt, ax, ay)) { rc = -1; break; }
    ++steps;
    t = (t_final - (t + dt) <= 1e-15 * fabs(t_final)) ? t_final : t + dt;
    for (size_t c = 0; c < nall; ++c)
      if (!isfinite(U[c])) { rc = -2; break; }
    if (rc) break;
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Learned troubled-cell indicator (not part of the paper): the training     */
/* label and the padded state the features are read from.                   */
/* ------------------------------------------------------------------------ */
/* Per cell, the largest |omega_m / gamma_m - 1| of the plain scheme's
 * nonlinear weights (Sec. 2.1 / 2.2 Step 3) over every reconstructed field:
 * the components (component-wise) or the characteristic fields of both
 * passes (Remark 1).  dev has one value per cell. */
int or_weight_deviation(const or_problem* p, const double* U, double* dev) {
  if (check_problem(p)) return -1;
  build_maps();
  padded_t P;
  if (make_padded(p, U, &P)) return -1;
  const int nc = P.nc, nlin = p->dim == 1 ? 2 : 4;
  const double dx = (p->xhi - p->xlo) / p->nx;
  const double dy = p->dim == 2 ? (p->yhi - p->ylo) / p->ny : 1.0;
  const int chr = p->equation == OR_EQ_EULER && p->charwise;
  for (int j = 0; j < P.ny; ++j)
    for (int i = 0; i < P.nx; ++i) {
      double worst = 0.0;
      const int npass = chr ? p->dim : 1;
      for (int pass = 0; pass < npass; ++pass) {
        double R[16], L[16];
        double w[4][17];
        int nin = p->dim == 1 ? 5 : 17;
        double q[4][17];
        if (p->dim == 1) {
          for (int k = 0; k < nc; ++k) {
            q[k][0] = *pcell(&P, k, i - 1, 0);
            q[k][1] = *pcell(&P, k, i, 0);
            q[k][2] = *pcell(&P, k, i + 1, 0);
            q[k][3] = *pcell(&P, nc + k, i - 1, 0);
            q[k][4] = *pcell(&P, nc + k, i + 1, 0);
          }
        } else {
          for (int k = 0; k < nc; ++k) gather_q(&P, k, i, j, q[k]);
        }
        if (chr) {
          double U0[4];
          for (int k = 0; k < nc; ++k) U0[k] = q[k][p->dim == 1 ? 1 : 4];
          or_euler_eigen(p->dim, pass, U0, p->gamma_gas, R, L);
          for (int s = 0; s < nin; ++s) {
            double x[4], y[4];
            for (int k = 0; k < nc; ++k) x[k] = q[k][s];
            matvec(nc, L, x, y);
            for (int k = 0; k < nc; ++k) w[k][s] = y[k];
          }
        } else {
          for (int k = 0; k < nc; ++k)
            for (int s = 0; s < nin; ++s) w[k][s] = q[k][s];
        }
        for (int k = 0; k < nc; ++k) {
          double out[48], *om;
          if (p->dim == 1) { or_recon_cell_1d(p, w[k], dx, out); om = out + 5; }
          else { or_recon_cell_2d(p, w[k], dx, dy, out); om = out + 38; }
          for (int m = 0; m <= nlin; ++m) {
            const double d = fabs(om[m] / p->lin_w[m] - 1.0);
            if (d > worst || d != d) worst = d;
          }
        }
      }
      dev[(size_t)j * P.nx + i] = worst;
    }
  free(P.a);
  return 0;
}

/* The state with its 2 ghost layers filled (the boundary rules above):
 * out[f][ny+4][nx+4] in 2D, out[f][nx+4] in 1D. */
int or_padded_state(const or_problem* p, const double* U, double* out) {
  if (check_problem(p)) return -1;
  padded_t P;
  if (make_padded(p, U, &P)) return -1;
  memcpy(out, P.a, sizeof(double) * (size_t)P.nf * P.px * P.py);
  free(P.a);
  return 0;
}
