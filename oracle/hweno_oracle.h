/*
 * hweno_oracle.h -- plain, slow, serial FP64 CPU oracle of the fifth-order
 * finite-volume derivative-based HWENO scheme with unified stencils
 * (arxiv 2607.24325, Sec. 2.1 one-dimensional case, Sec. 2.2 two-dimensional
 * case, Remark 1 for systems, Appendix A for the coefficient tables).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library (libhweno); the
 * product path never calls it.
 *
 * State layout (all arrays FP64, x fastest, no ghost cells):
 *   U[f][j][i], f = d*nc + k, d = 0 cell average (u-bar), d = 1 x-derivative
 *   moment (v-bar), d = 2 y-derivative moment (w-bar, 2D only); k = component
 *   (nc = 1 scalar, 3 for 1D Euler (rho, rho*u, E), 4 for 2D Euler
 *   (rho, rho*u, rho*v, E)).
 *   1D v-bar is the mean of u_x over the cell (Sec. 2.1); 2D v-bar and w-bar
 *   are the scaled moments (1/dy) int u_x and (1/dx) int u_y (Sec. 2.2).
 * Operator output L has the layout of U (L^u, L^v, L^w).  dhat[(d-1)*nc+k]
 * holds the limited derivatives v-hat (d=1) and w-hat (d=2).
 * Every function returns 0 on success, a negative value on bad arguments.
 */
#ifndef HWENO_ORACLE_H
#define HWENO_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { OR_EQ_ADVECTION = 0, OR_EQ_BURGERS = 1, OR_EQ_EULER = 2 };
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1, OR_BC_REFLECT = 2, OR_BC_INFLOW = 3,
       OR_BC_SPLIT = 4, OR_BC_SHOCK = 5 };
/* OR_BC_SPLIT: ghost cells whose centre lies, along the side, below
 *   bc_param[side][0] take bc_state[side] (zero moments), the others mirror
 *   (OR_BC_REFLECT) -- the double Mach reflection wall (Sec. 3, the double
 *   Mach reflection example: post-shock state for x < 1/6, reflective after).
 * OR_BC_SHOCK: ghost cells whose centre lies, along the side, below
 *   bc_param[side][0] + bc_param[side][1] t take bc_state[side], the others
 *   bc_state2[side] (zero moments) -- a straight shock moving along the side
 *   (the same example's top boundary).  t is the time of the RK stage. */
enum { OR_DT_CFL = 0, OR_DT_CFL_DX53 = 1 };

typedef struct {
  int dim;            /* 1 or 2 */
  int equation;       /* OR_EQ_* */
  int nx, ny;         /* cells (ny = 1 in 1D) */
  double xlo, xhi, ylo, yhi;
  double adv_x, adv_y;      /* advection velocity (a_x, a_y) */
  double gamma_gas;         /* ratio of specific heats (Euler) */
  double lin_w[5];          /* linear weights gamma_0..gamma_{2|4}, positive, sum 1 */
  double eps;               /* epsilon in the nonlinear weights */
  int weight_pow;           /* power of beta in the weight denominator (1 or 2) */
  int charwise;             /* Euler: 1 characteristic-wise (Remark 1), 0 component-wise */
  int linear_weights;       /* 1: omega = gamma (no nonlinear weights) */
  int dt_rule;              /* OR_DT_* */
  int bc[4];                /* x-low, x-high, y-low, y-high: OR_BC_* */
  double bc_state[4][4];    /* conservative state used by OR_BC_INFLOW sides */
  double cfl;
  double bc_state2[4][4];   /* second state of OR_BC_SHOCK sides */
  double bc_param[4][2];    /* OR_BC_SPLIT: (split position, -); OR_BC_SHOCK: (x0, speed) */
  double t;                 /* time of the state (time-dependent boundaries) */
  int smoothness;           /* OR_BETA_MOMENT: Step 2's indicator (the paper's);
                               OR_BETA_TYPICAL: the Jiang-Shu integral indicator that
                               Step 2 replaces, Eq. (smoothness-indicator-typical[-2D]) */
} or_problem;
enum { OR_BETA_MOMENT = 0, OR_BETA_TYPICAL = 1 };

/* Number of components (1, 3 or 4) and of stored fields per cell. */
int or_ncomp(const or_problem* p);
int or_nfields(const or_problem* p);

/* Coefficient maps of the reconstructed polynomials, derived here from the
 * constraint definitions of Step 1 (Sec. 2.1 and 2.2) by exact moment
 * integrals and a dense linear solve.
 *  1D: c0 = G0 (u_{i-1}, u_i, u_{i+1}, dx v_{i-1}, dx v_{i+1}), G0 5x5 row-major;
 *      c1 = G1 (u_{i-1}, u_i), c2 = G2 (u_i, u_{i+1}), each 2x2.
 *  2D: c0 = G0 q (q1..q17 as in Appendix A), G0 15x17 row-major, basis order
 *      {1, xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta, xi eta^2, eta^3, xi^4,
 *      xi^3 eta, xi^2 eta^2, xi eta^3, eta^4};
 *      Gm[m][3][3], m = 0..3 for p_1..p_4, maps the three averages of S_m
 *      (in the order target, x-neighbour, y-neighbour) to (c1, c2, c3). */
void or_coef_maps_1d(double* G0, double* G1, double* G2);
void or_coef_maps_2d(double* G0, double* Gm);

/* One scalar reconstruction (Steps 1-3) of a cell.
 * 1D: in = (u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_{i+1}); out = (u(x_{i-1/2}),
 *     u(x_{i+1/2}), u'(x_{i-1/2}), u'(x_{i+1/2}), v-hat, omega_0..2, beta_0..2).
 * 2D: in = q1..q17; out = 36 face values [face][mu][quantity] with face
 *     0 = x_{i-1/2}, 1 = x_{i+1/2}, 2 = y_{j-1/2}, 3 = y_{j+1/2}, mu the Gauss
 *     point (ascending), quantity (u, u_x, u_y); then v-hat, w-hat,
 *     omega_0..4, beta_0..4. */
int or_recon_cell_1d(const or_problem* p, const double* in, double dx, double* out);
int or_recon_cell_2d(const or_problem* p, const double* in, double dx, double dy, double* out);

/* Euler flux Jacobian (dir 0: x, 1: y) and right/left eigenvectors at the
 * conservative state U (dim 1: 3x3, dim 2: 4x4, row-major; L = R^{-1}). */
int or_euler_jacobian(int dim, int dir, const double* U, double gamma_gas, double* A);
int or_euler_eigen(int dim, int dir, const double* U, double gamma_gas, double* R, double* L);

/* Spatial operator L(U) and the limited derivatives (Sec. 2.1 Eq.
 * semi-discrete-scheme; Sec. 2.2 Eq. 2D-semi-discrete-scheme-uniform), with
 * the global Lax-Friedrichs constants ax, ay given. */
int or_operator(const or_problem* p, const double* U, double ax, double ay,
                double* L, double* dhat);
/* Global Lax-Friedrichs constants: max spectral radius over cell averages. */
int or_alpha(const or_problem* p, const double* U, double* ax, double* ay);
/* Time step from the CFL number and the dt rule. */
double or_dt(const or_problem* p, double ax, double ay);
/* One SSP-RK3 step with derivative substitution (Step 4), in place. */
int or_step(const or_problem* p, double* U, double dt, double ax, double ay);
/* Advance to t_final (last step clipped), at most max_steps steps. */
int or_run(const or_problem* p, double* U, double t_final, int max_steps,
           double* t_out, int* steps_out);

/* Running count of the method's flops (see the counting rules at the top of
 * hweno_oracle.c): the plain evaluation of each formula, charged for the
 * grid's own cells and faces only.  reset != 0 zeroes it after reading. */
long long or_flop_count(int reset);

/* Learned troubled-cell indicator (not in the paper).  dev[cell] = the
 * largest |omega_m / gamma_m - 1| of the plain scheme's nonlinear weights
 * over every reconstructed field (both passes for 2D characteristic Euler):
 * the label source.  or_padded_state returns the state with its ghost
 * layers: out[f][ny+4][nx+4] (2D) or out[f][nx+4] (1D). */
int or_weight_deviation(const or_problem* p, const double* U, double* dev);
int or_padded_state(const or_problem* p, const double* U, double* out);

#ifdef __cplusplus
}
#endif
#endif
