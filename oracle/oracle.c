/*
 * Plain FP64 CPU oracle for the implicit electron-density / electric-potential
 * solve of the MISDC method of Esclapez, Ricchiuti, Bell and Day,
 * "A spectral deferred correction strategy for low Mach number reacting flows
 * subject to electric fields" (arXiv:1904.08510), Sec. 3.2.
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this code; the product path never does. It shares
 * no code, header or table with the CUDA library.
 *
 * What it computes (one independent 1D column at a time, uniform cells of
 * width h, cell centres x_i = (i + 1/2) h):
 *
 *   F_e,i   = -n_i + f_e,i - (dt/h) (Gam_{i+1/2} - Gam_{i-1/2})          Eq. nls (a)
 *   F_phi,i = -n_i + f_phi,i + (eps0 eps_r / e) (G_{i+1/2} - G_{i-1/2}) / h   Eq. nls (b)
 *
 * with f_e = n_e^n + dt I_Re and f_phi = sum_m nu_m n_m (Eq. nls; the printed
 * "-I_Re + n_e^n" is read as n_e^n + dt I_Re so that both terms are densities),
 * G = dphi/dx at faces, and Gam the electron flux n v - D dn/dx with electron
 * velocity v = U + mu grad(phi) (electrons drift up the potential; the paper's
 * constant mobility 0.4 m^2/(V s) of Sec. 2.2 is the magnitude mu) and the
 * Einstein diffusivity D = mu k_B T / e (Sec. 2.1). The face flux is the
 * Scharfetter-Gummel form Gam = (D/h) [B(-Pe) n_i - B(Pe) n_{i+1}],
 * Pe = v h / D, B(x) = x / (e^x - 1), which is upwind-stable for the
 * non-symmetric drift the paper warns about in Sec. 3.1 and second-order
 * consistent. Electrode faces: Dirichlet phi = V_L, V_R with the face gradient
 * of the quadratic through (face, x_0, x_1); electrons leave through an
 * electrode by drift only (absorbing) or, in the zero-gradient test mode, the
 * boundary flux is v n_edge in both directions.
 *
 * The solve is Algorithm 2 (JFNK), step by step:
 *   scaling S_X, S_F from typical values (Eq. newton_sc) taken at the plain
 *   start X^n = (n_e^n, phi^n) whatever the initial guess, one scalar per
 *   block: s_n = max(|n_e^n|, |f_phi|, 1), s_phi = max(|phi^n|, |V_L|, |V_R|, 1),
 *   s_Fe = max(|F_e(X^n)|, |f_e|), s_Fphi = max(|F_phi(X^n)|, |f_phi|) (max
 *   norms; the source terms keep the scale from collapsing when X^n is nearly
 *   a root); Newton loop on ||S_F^-1 F||_inf;
 *   restarted GMRES (Saad-Schultz) with modified Gram-Schmidt, delta_0 = 0,
 *   preconditioned on the right so that the Krylov space of delta is
 *   K_p(P^-1 J, P^-1 F) as in Algorithm 2 while the minimised and tested
 *   residual is the unpreconditioned ||J delta + F||_2 < gamma ||F||_2 of the
 *   stopping test; finite-difference Jacobian-vector products
 *   (Eq. jf_dfapprox, eps_FD = lambda (lambda + |X|/|v|), lambda = eps_mach^(1/3));
 *   the Schur-factorised preconditioner of Sec. 3.2 in either of the paper's
 *   forms: the exact factorisation (Eq. prec, P^-1 = J^-1; in 1D J is
 *   block-tridiagonal in (n_i, phi_i) and is solved by block elimination) or
 *   the recast form (Eq. prec_recast) with the approximate Schur complement
 *   S~ = L + I_e dt D_r, its blocks solved exactly by the Thomas algorithm (the
 *   paper's own 1D choice for the exact reference, Sec. 4.2) or by multigrid
 *   V-cycles to a tolerance gamma_MG (Sec. 4.2: red-black Gauss-Seidel, two
 *   relaxations down and up every level); backtracking
 *   line search with sufficient decrease ||F(X + lam dX)|| <= (1 - alpha lam
 *   (1 - gamma)) ||F(X)|| (halving; the printed condition is garbled).
 *
 * Precision: IEEE double everywhere.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_E 1.602176634e-19      /* elementary charge, C         */
#define OR_KB 1.380649e-23        /* Boltzmann constant, J/K      */
#define OR_EPS0 8.8541878128e-12  /* vacuum permittivity, F/m     */

enum { OR_OK = 0, OR_MAX_NEWTON = 1, OR_MAX_KRYLOV = 2, OR_LINESEARCH_FAIL = 3,
       OR_NONFINITE = 4, OR_BAD_INPUT = 5 };
enum { OR_BC_ABSORBING = 0, OR_BC_ZERO_GRADIENT = 1 };

typedef struct {
  double eps_F, eps_X, gamma, mobility, ls_alpha, eps_r;
  int restart_m, max_newton, max_krylov, max_linesearch;
  int bc_electron;
  int precond;          /* 1: recast Schur P~ (Eq. prec_recast); 2: exact Schur
                           (Eq. prec, P^-1 = J^-1); 0: none; 3: recast Schur P~
                           with its two blocks solved by multigrid V-cycles */
  double mg_gamma_A;    /* precond 3: V-cycle tolerance of the (dt D_f - I) block;
                           <= 0 solves that block exactly (Thomas) */
  double mg_gamma_S;    /* precond 3: V-cycle tolerance of the S~ block; <= 0: exact */
  int mg_max_cycles;    /* precond 3: V-cycles per block solve at most */
  int mg_transfer;      /* precond 3: 0 operator-dependent, 1 linear (see below) */
  /* electron transport: 0 constant mobility with Einstein D; 1 tables of mu and D
     over the progress variable c and the reduced field E/N (Sec. 2.2) */
  int transport;
  const double *tab_mu, *tab_D;   /* [tab_nc][tab_nx], row c_k = k/(nc-1), column
                                     E/N = j tab_en_max/(nx-1) Td */
  int tab_nc, tab_nx;
  double tab_en_max;              /* Td (1 Td = 1e-21 V m^2) */
  double T_in, T_max;             /* c = (T - T_in) / (T_max - T_in), clamped to [0, 1] */
  double gas_molar_mass;          /* kg/mol: N = rho N_A / W */
  double eps_E;         /* error test at the stop (see or_jfnk_col), 0 = off */
} or_params;

typedef struct {
  int status, newton_it, krylov_it, res_evals, ls_halvings, krylov_capped;
  int mg_cycles;        /* V-cycles of all multigrid block solves (precond 3) */
  double final_res, first_res;
} or_stats;

/* One column's problem data. */
typedef struct {
  int n;
  double h, dt, vl, vr, mu, eps_r;
  int bc;
  const double *fe, *fphi, *D, *U;   /* U may be NULL (no advection) */
  /* transport tables (NULL: constant mu, D per cell) and, for them, the
     progress variable and background gas density of every cell */
  const double *tab_mu, *tab_D;
  int tab_nc, tab_nx;
  double tab_en_max;
  const double *cprog, *Ngas;
} or_col;

#define OR_NA 6.02214076e23        /* Avogadro constant, 1/mol     */
#define OR_MAX_POLISH 2            /* Newton steps for the error test at most */
#define OR_ERR_MARGIN 10.0         /* a stale-factor error estimate within this factor
                                      of the bar is re-taken with factors at X^(l) */

/* Bilinear interpolation of a [nc][nx] table with nodes c_k = k/(nc-1) and
 * x_j = j en_max/(nx-1), at (c, x) clamped to the table. */
double or_tab_lookup(const double* t, int nc, int nx, double en_max, double c, double x);
static double tab_lookup(const double* t, int nc, int nx, double en_max, double c, double x) {
  return or_tab_lookup(t, nc, nx, en_max, c, x);
}
double or_tab_lookup(const double* t, int nc, int nx, double en_max, double c, double x) {
  double tc = c * (nc - 1), tx = x / en_max * (nx - 1);
  if (tc < 0.0) tc = 0.0;
  if (tc > nc - 1) tc = nc - 1;
  if (tx < 0.0) tx = 0.0;
  if (tx > nx - 1) tx = nx - 1;
  int ic = (int)floor(tc), jx = (int)floor(tx);
  if (ic > nc - 2) ic = nc - 2;
  if (jx > nx - 2) jx = nx - 2;
  double wc = tc - ic, wx = tx - jx;
  const double* r0 = t + (size_t)ic * nx;
  const double* r1 = r0 + nx;
  return (1.0 - wc) * ((1.0 - wx) * r0[jx] + wx * r0[jx + 1]) +
         wc * ((1.0 - wx) * r1[jx] + wx * r1[jx + 1]);
}

/* d/dx of the bilinear interpolant at (c, x) (per Td): the slope of the
 * table cell that tab_lookup interpolates in, zero where x is clamped. */
static double tab_slope(const double* t, int nc, int nx, double en_max, double c, double x) {
  double tx = x / en_max * (nx - 1);
  if (tx < 0.0 || tx > nx - 1) return 0.0;
  double tc = c * (nc - 1);
  if (tc < 0.0) tc = 0.0;
  if (tc > nc - 1) tc = nc - 1;
  int ic = (int)floor(tc), jx = (int)floor(tx);
  if (ic > nc - 2) ic = nc - 2;
  if (jx > nx - 2) jx = nx - 2;
  double wc = tc - ic;
  const double* r0 = t + (size_t)ic * nx;
  const double* r1 = r0 + nx;
  return ((1.0 - wc) * (r0[jx + 1] - r0[jx]) + wc * (r1[jx + 1] - r1[jx])) * (nx - 1) / en_max;
}

/* Electron mobility and diffusivity at the face between cells i and k
 * (k = i + 1; k = i for an electrode face) where the potential gradient is G:
 * constant mu and the mean of the cells' Einstein D, or the tables at the
 * face means of c and N and E/N = |G| / N (Sec. 2.2). With dmu, dD non-NULL
 * also their derivatives with respect to G (zero for constant transport). */
static void face_transport_d(const or_col* c, int i, int k, double G, double* mu, double* D,
                             double* dmu, double* dD) {
  if (!c->tab_mu) {
    *mu = c->mu;
    *D = k == i ? c->D[i] : 0.5 * (c->D[i] + c->D[k]);
    if (dmu) { *dmu = 0.0; *dD = 0.0; }
    return;
  }
  double cf = 0.5 * (c->cprog[i] + c->cprog[k]);
  double Nf = 0.5 * (c->Ngas[i] + c->Ngas[k]);
  double en = fabs(G) / Nf / 1e-21;
  *mu = tab_lookup(c->tab_mu, c->tab_nc, c->tab_nx, c->tab_en_max, cf, en);
  *D = tab_lookup(c->tab_D, c->tab_nc, c->tab_nx, c->tab_en_max, cf, en);
  if (dmu) {
    double den = (G < 0.0 ? -1.0 : 1.0) / Nf / 1e-21;      /* d(E/N)/dG in Td */
    *dmu = tab_slope(c->tab_mu, c->tab_nc, c->tab_nx, c->tab_en_max, cf, en) * den;
    *dD = tab_slope(c->tab_D, c->tab_nc, c->tab_nx, c->tab_en_max, cf, en) * den;
  }
}
static void face_transport(const or_col* c, int i, int k, double G, double* mu, double* D) {
  face_transport_d(c, i, k, G, mu, D, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Bernoulli function B(x) = x / (e^x - 1) and its derivative.              */
/* ------------------------------------------------------------------------ */
double or_bern(double x) {
  if (fabs(x) < 1e-3) {          /* Taylor series of x/(e^x-1) */
    double x2 = x * x;
    return 1.0 - 0.5 * x + x2 / 12.0 - x2 * x2 / 720.0;
  }
  return x / expm1(x);
}

double or_bern_deriv(double x) {
  if (fabs(x) < 1e-2) {          /* derivative of the Taylor series */
    double x2 = x * x;
    return -0.5 + x / 6.0 - x * x2 / 180.0 + x * x2 * x2 / 5040.0;
  }
  if (x > 30.0) return (1.0 - x) * exp(-x);   /* e^{-x} relative terms dropped */
  double em = expm1(x);
  return (em - x * exp(x)) / (em * em);
}

/* ------------------------------------------------------------------------ */
/* Residual F(X), Eq. nls.                                                   */
/* ------------------------------------------------------------------------ */
static double face_u(const or_col* c, int i) {   /* advective velocity at face i+1/2 */
  return c->U ? 0.5 * (c->U[i] + c->U[i + 1]) : 0.0;
}

/* The potential is carried as phi = phi_ref + psi, where phi_ref is the
 * linear profile between the electrode values, phi_ref(x) = V_L + g0 x with
 * g0 = (V_R - V_L)/L. The discrete equations are unchanged; only the stored
 * unknown is the deviation psi, whose rounding is far below that of phi when
 * |V| is large. Face gradients are therefore G = g0 + (deviation gradient). */
static double phi_ref(const or_col* c, int i) {
  return c->vl + (c->vr - c->vl) * (i + 0.5) / c->n;
}
static double grad0(const or_col* c) { return (c->vr - c->vl) / (c->n * c->h); }

/* Electrode-face gradients, quadratic through (face, x_0, x_1):
 * G_L = (-8 V_L + 9 phi_0 - phi_1) / (3h); with phi = phi_ref + psi this is
 * g0 + (9 psi_0 - psi_1) / (3h) (the quadratic fit is exact for phi_ref).   */
static double dgrad_left(const or_col* c, const double* psi) {
  return (9.0 * psi[0] - psi[1]) / (3.0 * c->h);
}
static double dgrad_right(const or_col* c, const double* psi) {
  int N = c->n;
  return (-9.0 * psi[N - 1] + psi[N - 2]) / (3.0 * c->h);
}

/* Residual in terms of (n, psi). */
void or_residual_psi(const or_col* c, const double* ne, const double* psi,
                     double* Fe, double* Fp) {
  const int N = c->n;
  const double h = c->h, dt = c->dt, g0 = grad0(c);
  const double kap = OR_EPS0 * c->eps_r / OR_E;
  double dL = dgrad_left(c, psi), dR = dgrad_right(c, psi);
  double muL, muR, Dd;
  face_transport(c, 0, 0, g0 + dL, &muL, &Dd);
  face_transport(c, N - 1, N - 1, g0 + dR, &muR, &Dd);
  double vL = (c->U ? c->U[0] : 0.0) + muL * (g0 + dL);
  double vR = (c->U ? c->U[N - 1] : 0.0) + muR * (g0 + dR);
  double GamL, GamR;
  if (c->bc == OR_BC_ZERO_GRADIENT) {
    GamL = vL * ne[0];
    GamR = vR * ne[N - 1];
  } else {
    GamL = vL < 0.0 ? vL * ne[0] : 0.0;          /* leaves to the left  */
    GamR = vR > 0.0 ? vR * ne[N - 1] : 0.0;      /* leaves to the right */
  }
  double gam_prev = GamL, d_prev = dL;
  for (int i = 0; i < N; ++i) {
    double gam_next, d_next;
    if (i == N - 1) {
      gam_next = GamR;
      d_next = dR;
    } else {
      d_next = (psi[i + 1] - psi[i]) / h;
      double muf, Df;
      face_transport(c, i, i + 1, g0 + d_next, &muf, &Df);
      double v = face_u(c, i) + muf * (g0 + d_next);
      double Pe = v * h / Df;
      gam_next = (Df / h) * (or_bern(-Pe) * ne[i] - or_bern(Pe) * ne[i + 1]);
    }
    Fe[i] = -ne[i] + c->fe[i] - (dt / h) * (gam_next - gam_prev);
    /* G_{i+1/2} - G_{i-1/2}: g0 cancels */
    Fp[i] = -ne[i] + c->fphi[i] + kap * (d_next - d_prev) / h;
    gam_prev = gam_next;
    d_prev = d_next;
  }
}

/* Residual F(n, phi) of Eq. nls. */
void or_residual_col(const or_col* c, const double* ne, const double* phi,
                     double* Fe, double* Fp) {
  double* psi = (double*)malloc(sizeof(double) * c->n);
  for (int i = 0; i < c->n; ++i) psi[i] = phi[i] - phi_ref(c, i);
  or_residual_psi(c, ne, psi, Fe, Fp);
  free(psi);
}

/* ------------------------------------------------------------------------ */
/* Analytic Jacobian blocks of the discrete residual (Eq. linear_nls):       */
/*   A = dF_e/dn (dt D_f - I), B = dF_e/dphi (dt D_r), C = dF_phi/dn = -I,   */
/*   L = dF_phi/dphi. Tridiagonal: sub[i] couples i-1, sup[i] couples i+1.   */
/* ------------------------------------------------------------------------ */
typedef struct { double *sub, *dia, *sup; } or_tri;

void or_jacobian_col(const or_col* c, const double* ne, const double* phi,
                     or_tri A, or_tri B, or_tri L) {
  const int N = c->n;
  const double h = c->h, dt = c->dt, r = dt / h;
  const double kap = OR_EPS0 * c->eps_r / OR_E;
  for (int i = 0; i < N; ++i) {
    A.sub[i] = A.sup[i] = B.sub[i] = B.sup[i] = L.sub[i] = L.sup[i] = 0.0;
    A.dia[i] = -1.0;
    B.dia[i] = 0.0;
    L.dia[i] = 0.0;
  }
  /* interior faces i+1/2 */
  for (int i = 0; i + 1 < N; ++i) {
    /* with transport tables mu and D depend on the face gradient G through
       E/N: the flux derivative includes mu'(G) and D'(G) (the slopes of the
       interpolant) */
    double G = (phi[i + 1] - phi[i]) / h;
    double muf, Df, dmu, dD;
    face_transport_d(c, i, i + 1, G, &muf, &Df, &dmu, &dD);
    double v = face_u(c, i) + muf * G;
    double Pe = v * h / Df;
    double dG_dn0 = (Df / h) * or_bern(-Pe);
    double dG_dn1 = -(Df / h) * or_bern(Pe);
    /* dGam/dG = (D'/h)[B(-Pe) n_i - B(Pe) n_{i+1}]
     *         + (D/h)[-B'(-Pe) n_i - B'(Pe) n_{i+1}] dPe/dG,
     * dPe/dG = h ((mu + G mu') D - v D') / D^2; dG/dphi_{i+1} = 1/h */
    double dPe = h * ((muf + G * dmu) * Df - v * dD) / (Df * Df);
    double dGam = (dD / h) * (or_bern(-Pe) * ne[i] - or_bern(Pe) * ne[i + 1]) +
                  (Df / h) * (-or_bern_deriv(-Pe) * ne[i] - or_bern_deriv(Pe) * ne[i + 1]) * dPe;
    double dG_dp1 = dGam / h;
    double dG_dp0 = -dG_dp1;
    /* row i carries -r*Gam_{i+1/2}; row i+1 carries +r*Gam_{i+1/2} */
    A.dia[i] += -r * dG_dn0;  A.sup[i] += -r * dG_dn1;
    A.sub[i + 1] += r * dG_dn0;  A.dia[i + 1] += r * dG_dn1;
    B.dia[i] += -r * dG_dp0;  B.sup[i] += -r * dG_dp1;
    B.sub[i + 1] += r * dG_dp0;  B.dia[i + 1] += r * dG_dp1;
    /* Poisson: row i has +kap*G_{i+1/2}/h, row i+1 has -kap*G_{i+1/2}/h */
    L.dia[i] += -kap / (h * h);  L.sup[i] += kap / (h * h);
    L.sub[i + 1] += kap / (h * h);  L.dia[i + 1] += -kap / (h * h);
  }
  /* left electrode face: row 0 carries +r*GamL and -kap*GL/h */
  {
    double GL = (-8.0 * c->vl + 9.0 * phi[0] - phi[1]) / (3.0 * h);
    double muL, Dd, dmuL, dDd;
    face_transport_d(c, 0, 0, GL, &muL, &Dd, &dmuL, &dDd);
    double vL = (c->U ? c->U[0] : 0.0) + muL * GL;
    double dvL = muL + GL * dmuL;                  /* dv/dG at the electrode face */
    int active = (c->bc == OR_BC_ZERO_GRADIENT) || vL < 0.0;
    if (active) {
      A.dia[0] += r * vL;
      B.dia[0] += r * ne[0] * dvL * (9.0 / (3.0 * h));
      B.sup[0] += r * ne[0] * dvL * (-1.0 / (3.0 * h));
    }
    L.dia[0] += -kap / h * (9.0 / (3.0 * h));
    L.sup[0] += -kap / h * (-1.0 / (3.0 * h));
  }
  /* right electrode face: row N-1 carries -r*GamR and +kap*GR/h */
  {
    double GR = (8.0 * c->vr - 9.0 * phi[N - 1] + phi[N - 2]) / (3.0 * h);
    double muR, Dd, dmuR, dDd;
    face_transport_d(c, N - 1, N - 1, GR, &muR, &Dd, &dmuR, &dDd);
    double vR = (c->U ? c->U[N - 1] : 0.0) + muR * GR;
    double dvR = muR + GR * dmuR;
    int active = (c->bc == OR_BC_ZERO_GRADIENT) || vR > 0.0;
    if (active) {
      A.dia[N - 1] += -r * vR;
      B.dia[N - 1] += -r * ne[N - 1] * dvR * (-9.0 / (3.0 * h));
      B.sub[N - 1] += -r * ne[N - 1] * dvR * (1.0 / (3.0 * h));
    }
    L.dia[N - 1] += kap / h * (-9.0 / (3.0 * h));
    L.sub[N - 1] += kap / h * (1.0 / (3.0 * h));
  }
}

/* ------------------------------------------------------------------------ */
/* Thomas algorithm (no pivoting): solve T x = d.                            */
/* ------------------------------------------------------------------------ */
void or_thomas(int n, const double* sub, const double* dia, const double* sup,
               const double* d, double* x, double* work /* 2n */) {
  double* cp = work;
  double* dp = work + n;
  double piv = dia[0];
  cp[0] = sup[0] / piv;
  dp[0] = d[0] / piv;
  for (int i = 1; i < n; ++i) {
    piv = dia[i] - sub[i] * cp[i - 1];
    cp[i] = sup[i] / piv;
    dp[i] = (d[i] - sub[i] * dp[i - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

static void tri_matvec(int n, or_tri T, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = T.dia[i] * x[i];
    if (i > 0) s += T.sub[i] * x[i - 1];
    if (i + 1 < n) s += T.sup[i] * x[i + 1];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Preconditioners of Sec. 3.2, unscaled (residual space -> unknown space).  */
/*                                                                          */
/* Recast Schur form P~^{-1} (Eq. prec_recast), three block solves:         */
/*   z1 = A^{-1} v1; z2 = S~^{-1} (v2 - C z1); x1 = z1 - A^{-1} B z2; x2 = z2 */
/* with C = -I and the approximate Schur complement S~ = L + C B = L - B.    */
/*                                                                          */
/* Exact Schur form (Eq. prec): P^{-1} = J^{-1}. In 1D, J is block-         */
/* tridiagonal in the cell-interleaved unknowns (n_i, phi_i), so J^{-1} v is */
/* computed by block Gaussian elimination (block Thomas) on 2x2 blocks.      */
/* ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------ */
/* Geometric multigrid for one tridiagonal block (Sec. 4.2): standard       */
/* V-cycles with two red-black Gauss-Seidel relaxations on every level going */
/* down and two going up, repeated from x = 0 until                          */
/* ||b - T x||_2 <= gamma_MG ||b||_2, a cycle cap, or a cycle that does not  */
/* lower the residual (that cycle is undone).                                */
/* The paper names these ingredients but not the grid transfers; readings:   */
/*  - coarse unknown I sits on fine unknown 2I+1, n_c = floor(n_f / 2); the  */
/*    even ("red", relaxed first) unknowns are the fine-only ones;           */
/*  - transfer OR_MG_OPERATOR (default): operator-dependent interpolation    */
/*    and restriction of black-box multigrid (Dendy): a fine-only unknown i  */
/*    takes -T[i][k] / T[i][i] of its coarse neighbour on fine k (P), and    */
/*    passes -T[k][i] / T[i][i] of its residual to it (R, from T^T);         */
/*    coarse unknowns are injected both ways. The electron block is an       */
/*    upwind-dominated M-matrix (cell Peclet numbers up to ~20, drift CFL    */
/*    in the thousands), on which linear transfers give coarse operators of  */
/*    the wrong sign pattern and the V-cycle diverges; these transfers keep  */
/*    the coarse operator the Schur complement onto the coarse unknowns;     */
/*  - transfer OR_MG_LINEAR: the textbook linear interpolation (mean of the  */
/*    two coarse neighbours, half of the one neighbour at an end) and        */
/*    R = P^T;                                                               */
/*  - coarse operator R T P (Galerkin; tridiagonal again);                   */
/*  - coarsening stops at OR_MG_COARSE unknowns or fewer, solved by Thomas.  */
/* ------------------------------------------------------------------------ */
#define OR_MG_COARSE 8
#define OR_MG_MAXLEV 40
enum { OR_MG_OPERATOR = 0, OR_MG_LINEAR = 1 };

typedef struct { int n; double *sub, *dia, *sup, *x, *b, *r; } or_mg_level;
typedef struct {
  int nlev, transfer;
  or_mg_level lev[OR_MG_MAXLEV];
  double* mem;
  double* xp;        /* iterate before the current cycle */
  double work[2 * OR_MG_COARSE];
} or_mg;

static double tri_at(const or_mg_level* L, int i, int k) {
  if (i < 0 || i >= L->n || k < 0 || k >= L->n) return 0.0;
  if (k == i - 1) return L->sub[i];
  if (k == i) return L->dia[i];
  if (k == i + 1) return L->sup[i];
  return 0.0;
}

/* fine unknown of coarse unknown J */
static int fine_of(int J) { return 2 * J + 1; }

/* P[i][J]: prolongation from level F (n_c = F->n / 2 coarse unknowns) */
static double mg_p(const or_mg_level* F, int transfer, int i, int J) {
  int nc = F->n / 2;
  if (i < 0 || i >= F->n || J < 0 || J >= nc) return 0.0;
  if (i & 1) return J == (i - 1) / 2 ? 1.0 : 0.0;
  int k = fine_of(J);
  if (k != i - 1 && k != i + 1) return 0.0;
  return transfer == OR_MG_LINEAR ? 0.5 : -tri_at(F, i, k) / F->dia[i];
}

/* R[J][i]: restriction to level F's coarse unknowns */
static double mg_r(const or_mg_level* F, int transfer, int J, int i) {
  int nc = F->n / 2;
  if (i < 0 || i >= F->n || J < 0 || J >= nc) return 0.0;
  if (i & 1) return J == (i - 1) / 2 ? 1.0 : 0.0;
  int k = fine_of(J);
  if (k != i - 1 && k != i + 1) return 0.0;
  return transfer == OR_MG_LINEAR ? 0.5 : -tri_at(F, k, i) / F->dia[i];
}

/* (R T P)[I][J] = sum_i sum_k R[I][i] T[i][k] P[k][J]; R[I][i] vanishes
 * outside i = 2I .. 2I+2 and T[i][k] outside k = i-1 .. i+1. */
static double galerkin_entry(const or_mg_level* F, int transfer, int I, int J) {
  double s = 0.0;
  for (int i = 2 * I; i <= 2 * I + 2; ++i) {
    double r = mg_r(F, transfer, I, i);
    if (r == 0.0) continue;
    for (int k = i - 1; k <= i + 1; ++k) {
      double p = mg_p(F, transfer, k, J);
      if (p == 0.0) continue;
      s += r * tri_at(F, i, k) * p;
    }
  }
  return s;
}

static void or_mg_init(or_mg* M, int n, int transfer) {
  int tot = 0;
  for (int m = n;; m /= 2) { tot += m; if (m <= OR_MG_COARSE) break; }
  M->mem = (double*)malloc(sizeof(double) * (6 * (size_t)tot + n));
  M->nlev = 0;
  M->transfer = transfer;
  double* p = M->mem;
  for (int m = n;; m /= 2) {
    or_mg_level* L = &M->lev[M->nlev++];
    L->n = m;
    L->sub = p; L->dia = p + m; L->sup = p + 2 * m; L->x = p + 3 * m; L->b = p + 4 * m;
    L->r = p + 5 * m;
    p += 6 * m;
    if (m <= OR_MG_COARSE) break;
  }
  M->xp = p;
}

static void or_mg_free(or_mg* M) { free(M->mem); M->mem = NULL; }

/* Level 0 = T; level l+1 = R T_l P. */
static void or_mg_setup(or_mg* M, const double* sub, const double* dia, const double* sup) {
  or_mg_level* L0 = &M->lev[0];
  memcpy(L0->sub, sub, sizeof(double) * L0->n);
  memcpy(L0->dia, dia, sizeof(double) * L0->n);
  memcpy(L0->sup, sup, sizeof(double) * L0->n);
  L0->sub[0] = 0.0;
  L0->sup[L0->n - 1] = 0.0;
  for (int l = 0; l + 1 < M->nlev; ++l) {
    const or_mg_level* F = &M->lev[l];
    or_mg_level* Cg = &M->lev[l + 1];
    for (int I = 0; I < Cg->n; ++I) {
      Cg->sub[I] = I > 0 ? galerkin_entry(F, M->transfer, I, I - 1) : 0.0;
      Cg->dia[I] = galerkin_entry(F, M->transfer, I, I);
      Cg->sup[I] = I + 1 < Cg->n ? galerkin_entry(F, M->transfer, I, I + 1) : 0.0;
    }
  }
}

/* One red-black Gauss-Seidel relaxation of T x = b. */
static void rbgs(const or_mg_level* L, double* x, const double* b) {
  for (int colour = 0; colour < 2; ++colour)
    for (int i = colour; i < L->n; i += 2) {
      double s = b[i];
      if (i > 0) s -= L->sub[i] * x[i - 1];
      if (i + 1 < L->n) s -= L->sup[i] * x[i + 1];
      x[i] = s / L->dia[i];
    }
}

static void tri_residual(const or_mg_level* L, const double* x, const double* b, double* r) {
  for (int i = 0; i < L->n; ++i) {
    double s = L->dia[i] * x[i];
    if (i > 0) s += L->sub[i] * x[i - 1];
    if (i + 1 < L->n) s += L->sup[i] * x[i + 1];
    r[i] = b[i] - s;
  }
}

/* One V-cycle on level l: improves lev[l].x for the right-hand side lev[l].b. */
static void vcycle(or_mg* M, int l) {
  or_mg_level* F = &M->lev[l];
  if (l == M->nlev - 1) {
    or_thomas(F->n, F->sub, F->dia, F->sup, F->b, F->x, M->work);
    return;
  }
  or_mg_level* Cg = &M->lev[l + 1];
  rbgs(F, F->x, F->b);
  rbgs(F, F->x, F->b);
  tri_residual(F, F->x, F->b, F->r);
  for (int I = 0; I < Cg->n; ++I) {             /* b_c = R r */
    double s = 0.0;
    for (int i = 2 * I; i <= 2 * I + 2 && i < F->n; ++i) s += mg_r(F, M->transfer, I, i) * F->r[i];
    Cg->b[I] = s;
    Cg->x[I] = 0.0;
  }
  vcycle(M, l + 1);
  for (int i = 0; i < F->n; ++i) {              /* x += P x_c */
    double s = 0.0;
    for (int J = i / 2 - 1; J <= i / 2; ++J)
      if (J >= 0 && J < Cg->n) s += mg_p(F, M->transfer, i, J) * Cg->x[J];
    F->x[i] += s;
  }
  rbgs(F, F->x, F->b);
  rbgs(F, F->x, F->b);
}

/* x = T^{-1} b by V-cycles; returns the cycles run. */
static int or_mg_solve(or_mg* M, const double* b, double* x, double gamma, int max_cycles) {
  or_mg_level* L = &M->lev[0];
  const int n = L->n;
  double nb = 0.0;
  for (int i = 0; i < n; ++i) { L->b[i] = b[i]; L->x[i] = 0.0; nb += b[i] * b[i]; }
  nb = sqrt(nb);
  double prev = nb;
  int k = 0;
  while (nb > 0.0 && k < max_cycles) {
    memcpy(M->xp, L->x, sizeof(double) * n);
    vcycle(M, 0);
    ++k;
    tri_residual(L, L->x, L->b, L->r);
    double rr = 0.0;
    for (int i = 0; i < n; ++i) rr += L->r[i] * L->r[i];
    rr = sqrt(rr);
    if (!(rr < prev)) {                  /* no progress (rounding floor or divergence) */
      memcpy(L->x, M->xp, sizeof(double) * n);
      break;
    }
    prev = rr;
    if (rr <= gamma * nb) break;
  }
  memcpy(x, L->x, sizeof(double) * n);
  return k;
}

/* Stand-alone multigrid solve of one tridiagonal system (tests). */
int or_mg_solve_tri(int n, const double* sub, const double* dia, const double* sup,
                    const double* b, double* x, double gamma, int max_cycles, int transfer) {
  or_mg M;
  or_mg_init(&M, n, transfer);
  or_mg_setup(&M, sub, dia, sup);
  int k = or_mg_solve(&M, b, x, gamma, max_cycles);
  or_mg_free(&M);
  return k;
}

/* The level hierarchy of one tridiagonal matrix: number of levels, and each
 * level's size and three diagonals packed back to back into out (tests). */
int or_mg_hierarchy(int n, const double* sub, const double* dia, const double* sup,
                    int transfer, int* sizes, double* out) {
  or_mg M;
  or_mg_init(&M, n, transfer);
  or_mg_setup(&M, sub, dia, sup);
  size_t o = 0;
  for (int l = 0; l < M.nlev; ++l) {
    const or_mg_level* L = &M.lev[l];
    sizes[l] = L->n;
    memcpy(out + o, L->sub, sizeof(double) * L->n); o += L->n;
    memcpy(out + o, L->dia, sizeof(double) * L->n); o += L->n;
    memcpy(out + o, L->sup, sizeof(double) * L->n); o += L->n;
  }
  int nl = M.nlev;
  or_mg_free(&M);
  return nl;
}

/* Dense P (nf x nf/2) and R (nf/2 x nf) of the finest transfer of T (tests). */
void or_mg_transfers(int n, const double* sub, const double* dia, const double* sup,
                     int transfer, double* P, double* R) {
  or_mg_level F = {n, (double*)sub, (double*)dia, (double*)sup, NULL, NULL, NULL};
  int nc = n / 2;
  for (int i = 0; i < n; ++i)
    for (int J = 0; J < nc; ++J) {
      P[(size_t)i * nc + J] = mg_p(&F, transfer, i, J);
      R[(size_t)J * n + i] = mg_r(&F, transfer, J, i);
    }
}

typedef struct {
  int n, mode;       /* mode 1: recast, 2: exact, 3: recast with multigrid blocks */
  or_tri A, B, L, S;
  double* work;      /* 4n (recast) or 12n (exact) */
  or_mg *mgA, *mgS;  /* mode 3: hierarchies of A and S~ (NULL: that block exact) */
  double gA, gS;
  int max_cycles;
  int* cycles;       /* mode 3: V-cycle counter */
} or_prec;

/* x = A^{-1} v (blk 0) or S~^{-1} v (blk 1): Thomas, or V-cycles in mode 3. */
static void blk_solve(const or_prec* P, int blk, const double* v, double* x, double* tw) {
  or_mg* M = blk == 0 ? P->mgA : P->mgS;
  if (P->mode == 3 && M) {
    int k = or_mg_solve(M, v, x, blk == 0 ? P->gA : P->gS, P->max_cycles);
    if (P->cycles) *P->cycles += k;
    return;
  }
  const or_tri* T = blk == 0 ? &P->A : &P->S;
  or_thomas(P->n, T->sub, T->dia, T->sup, v, x, tw);
}

void or_prec_recast_apply(const or_prec* P, const double* v1, const double* v2,
                          double* x1, double* x2) {
  int n = P->n;
  double* z1 = P->work;
  double* t = P->work + n;
  double* tw = P->work + 2 * n;
  blk_solve(P, 0, v1, z1, tw);
  for (int i = 0; i < n; ++i) t[i] = v2[i] + z1[i];            /* v2 - C z1 */
  blk_solve(P, 1, t, x2, tw);                                  /* z2 */
  tri_matvec(n, P->B, x2, t);                                  /* B z2 */
  blk_solve(P, 0, t, x1, tw);                                  /* A^{-1} B z2 */
  for (int i = 0; i < n; ++i) x1[i] = z1[i] - x1[i];
}

/* 2x2 helpers, row-major m = {m00, m01, m10, m11}. */
static void m2_inv(const double* m, double* r) {
  double det = m[0] * m[3] - m[1] * m[2];
  r[0] = m[3] / det; r[1] = -m[1] / det; r[2] = -m[2] / det; r[3] = m[0] / det;
}
static void m2_mul(const double* a, const double* b, double* r) {
  double r0 = a[0] * b[0] + a[1] * b[2], r1 = a[0] * b[1] + a[1] * b[3];
  double r2 = a[2] * b[0] + a[3] * b[2], r3 = a[2] * b[1] + a[3] * b[3];
  r[0] = r0; r[1] = r1; r[2] = r2; r[3] = r3;
}
static void m2_vec(const double* a, const double* x, double* y) {
  double y0 = a[0] * x[0] + a[1] * x[1], y1 = a[2] * x[0] + a[3] * x[1];
  y[0] = y0; y[1] = y1;
}

/* Block i of J in interleaved order: sub (couples cell i-1), dia, sup (i+1). */
static void j_blocks(const or_prec* P, int i, double* sub, double* dia, double* sup) {
  sub[0] = P->A.sub[i]; sub[1] = P->B.sub[i]; sub[2] = 0.0;  sub[3] = P->L.sub[i];
  dia[0] = P->A.dia[i]; dia[1] = P->B.dia[i]; dia[2] = -1.0; dia[3] = P->L.dia[i];
  sup[0] = P->A.sup[i]; sup[1] = P->B.sup[i]; sup[2] = 0.0;  sup[3] = P->L.sup[i];
}

void or_prec_exact_apply(const or_prec* P, const double* v1, const double* v2,
                         double* x1, double* x2) {
  int n = P->n;
  double* Cp = P->work;          /* 4n: modified super-diagonal blocks */
  double* dp = P->work + 4 * n;  /* 2n: modified right-hand sides      */
  double sub[4], dia[4], sup[4], W[4], Wi[4], t[4], r[2], s[2];
  for (int i = 0; i < n; ++i) {
    j_blocks(P, i, sub, dia, sup);
    r[0] = v1[i];
    r[1] = v2[i];
    if (i == 0) {
      memcpy(W, dia, sizeof(W));
    } else {
      m2_mul(sub, Cp + 4 * (i - 1), t);
      for (int k = 0; k < 4; ++k) W[k] = dia[k] - t[k];
      m2_vec(sub, dp + 2 * (i - 1), s);
      r[0] -= s[0];
      r[1] -= s[1];
    }
    m2_inv(W, Wi);
    m2_mul(Wi, sup, Cp + 4 * i);
    m2_vec(Wi, r, dp + 2 * i);
  }
  x1[n - 1] = dp[2 * (n - 1)];
  x2[n - 1] = dp[2 * (n - 1) + 1];
  for (int i = n - 2; i >= 0; --i) {
    double xn[2] = {x1[i + 1], x2[i + 1]};
    m2_vec(Cp + 4 * i, xn, s);
    x1[i] = dp[2 * i] - s[0];
    x2[i] = dp[2 * i + 1] - s[1];
  }
}

void or_prec_apply(const or_prec* P, const double* v1, const double* v2, double* x1,
                   double* x2) {
  if (P->mode == 2) or_prec_exact_apply(P, v1, v2, x1, x2);
  else or_prec_recast_apply(P, v1, v2, x1, x2);
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES(m), modified Gram-Schmidt, Givens rotations (Saad-Schultz). */
/* Solves op(x) = b from x = 0; stops when the residual estimate falls below  */
/* tol * ||b|| or after maxit operator applications.                          */
/* ------------------------------------------------------------------------ */
typedef void (*or_op_fn)(void* ctx, const double* v, double* w);

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int or_gmres(int n, or_op_fn op, void* ctx, const double* b, double* x,
             int m, double tol, int maxit, int* iters, double* res_est) {
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * m);
  double* sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* y = (double*)malloc(sizeof(double) * m);
  double* r = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  int total = 0, converged = 0;
  for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
  double beta0 = sqrt(dot(n, b, b));
  double beta = beta0;
  double est = beta0;
  if (beta0 == 0.0) converged = 1;
  while (!converged && total < maxit) {
    for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = V + (size_t)j * n;
      op(ctx, vj, w);
      ++total;
      for (int i = 0; i <= j; ++i) {          /* modified Gram-Schmidt */
        double* vi = V + (size_t)i * n;
        double hij = dot(n, w, vi);
        H[i * m + j] = hij;
        for (int q = 0; q < n; ++q) w[q] -= hij * vi[q];
      }
      double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {           /* previous rotations */
        double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double rho = hypot(a, bb);
      cs[j] = rho == 0.0 ? 1.0 : a / rho;
      sn[j] = rho == 0.0 ? 0.0 : bb / rho;
      H[j * m + j] = rho;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      est = fabs(g[j + 1]);
      if (est <= tol * beta0 || hn == 0.0) { converged = 1; break; }
      double* vn = V + (size_t)(j + 1) * n;
      for (int q = 0; q < n; ++q) vn[q] = w[q] / hn;
    }
    /* back substitution of the k x k triangle, x += V y */
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[i * m + q] * y[q];
      y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < k; ++i) {
      const double* vi = V + (size_t)i * n;
      for (int q = 0; q < n; ++q) x[q] += y[i] * vi[q];
    }
    if (converged || total >= maxit) break;
    /* restart from the true residual r = b - op(x) */
    op(ctx, x, w);
    ++total;
    for (int q = 0; q < n; ++q) r[q] = b[q] - w[q];
    beta = sqrt(dot(n, r, r));
    est = beta;
    if (beta <= tol * beta0) { converged = 1; break; }
  }
  if (iters) *iters = total;
  if (res_est) *res_est = beta0 > 0.0 ? est / beta0 : 0.0;
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(r); free(w);
  return converged;
}

/* Flexible GMRES (Saad 1993) for J x = b with a right preconditioner M^{-1}
 * that may differ between applications (the multigrid block solves of
 * precond 3 stop at a tolerance, so M^{-1} is not a fixed linear map): each
 * z_j = M^{-1} v_j is kept and x = Z y, so the residual the Givens estimate
 * tracks is that of the returned x. Restarts from the true residual b - J x.
 * For a fixed M^{-1} it produces the iterates of or_gmres on J M^{-1}. */
int or_fgmres(int n, or_op_fn jop, or_op_fn prec, void* ctx, const double* b, double* x,
              int m, double tol, int maxit, int* iters, double* res_est) {
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* Z = (double*)malloc(sizeof(double) * (size_t)n * m);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * m);
  double* sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* y = (double*)malloc(sizeof(double) * m);
  double* r = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  int total = 0, converged = 0;
  for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
  double beta0 = sqrt(dot(n, b, b));
  double beta = beta0;
  double est = beta0;
  if (beta0 == 0.0) converged = 1;
  while (!converged && total < maxit) {
    for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      prec(ctx, vj, zj);
      jop(ctx, zj, w);
      ++total;
      for (int i = 0; i <= j; ++i) {          /* modified Gram-Schmidt */
        double* vi = V + (size_t)i * n;
        double hij = dot(n, w, vi);
        H[i * m + j] = hij;
        for (int q = 0; q < n; ++q) w[q] -= hij * vi[q];
      }
      double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double rho = hypot(a, bb);
      cs[j] = rho == 0.0 ? 1.0 : a / rho;
      sn[j] = rho == 0.0 ? 0.0 : bb / rho;
      H[j * m + j] = rho;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      est = fabs(g[j + 1]);
      if (est <= tol * beta0 || hn == 0.0) { converged = 1; break; }
      double* vn = V + (size_t)(j + 1) * n;
      for (int q = 0; q < n; ++q) vn[q] = w[q] / hn;
    }
    /* back substitution of the k x k triangle, x += Z y */
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[i * m + q] * y[q];
      y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < k; ++i) {
      const double* zi = Z + (size_t)i * n;
      for (int q = 0; q < n; ++q) x[q] += y[i] * zi[q];
    }
    if (converged || total >= maxit) break;
    /* restart from the true residual r = b - J x */
    jop(ctx, x, w);
    ++total;
    for (int q = 0; q < n; ++q) r[q] = b[q] - w[q];
    beta = sqrt(dot(n, r, r));
    est = beta;
    if (beta <= tol * beta0) { converged = 1; break; }
  }
  if (iters) *iters = total;
  if (res_est) *res_est = beta0 > 0.0 ? est / beta0 : 0.0;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(r); free(w);
  return converged;
}

/* Dense-operator GMRES (test hook: pins GMRES against dense linear algebra). */
typedef struct { int n; const double* M; } dense_ctx;
static void dense_op(void* ctx, const double* v, double* w) {
  dense_ctx* d = (dense_ctx*)ctx;
  for (int i = 0; i < d->n; ++i) w[i] = dot(d->n, d->M + (size_t)i * d->n, v);
}
int or_gmres_dense(int n, const double* M, const double* b, double* x, int m,
                   double tol, int maxit, int* iters, double* res_est) {
  dense_ctx d = {n, M};
  return or_gmres(n, dense_op, &d, b, x, m, tol, maxit, iters, res_est);
}

/* ------------------------------------------------------------------------ */
/* JFNK (Algorithm 2) for one column. The Newton iterate is (n, psi), the   */
/* potential being phi = phi_ref + psi.                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  const or_col* c;
  const or_params* P;
  int n;
  double sn, sp, sFe, sFp;      /* S_X = diag(sn, sp), S_F = diag(sFe, sFp) */
  const double *ne, *psi;       /* current Newton iterate X^(l) */
  const double *Fe, *Fp;        /* F(X^(l)) */
  double xnorm;                 /* ||S_X^{-1} X^(l)||_2 with X = (n, phi) */
  or_prec prec;
  double *tn, *tp, *tFe, *tFp;  /* scratch: perturbed state and residual */
  double *u1, *u2, *t2;         /* scratch */
  int* res_evals;
} jf_ctx;

static int finite_vec(int n, const double* a) {
  for (int i = 0; i < n; ++i) if (!isfinite(a[i])) return 0;
  return 1;
}

/* Scaled Jacobian-vector product by finite differences (Eq. jf_dfapprox):
 * Jhat v = S_F^{-1} [F(X + eps S_X v) - F(X)] / eps,
 * eps = lambda (lambda + ||S_X^{-1} X||_2 / ||v||_2), lambda = eps_mach^(1/3). */
static void jf_jvp(jf_ctx* j, const double* v, double* out) {
  int n = j->n;
  double vn = sqrt(dot(2 * n, v, v));
  if (vn == 0.0) { for (int i = 0; i < 2 * n; ++i) out[i] = 0.0; return; }
  double lam = cbrt(DBL_EPSILON);
  double eps = lam * (lam + j->xnorm / vn);
  for (int i = 0; i < n; ++i) {
    j->tn[i] = j->ne[i] + eps * j->sn * v[i];
    j->tp[i] = j->psi[i] + eps * j->sp * v[n + i];
  }
  or_residual_psi(j->c, j->tn, j->tp, j->tFe, j->tFp);
  ++*j->res_evals;
  for (int i = 0; i < n; ++i) {
    out[i] = (j->tFe[i] - j->Fe[i]) / eps / j->sFe;
    out[n + i] = (j->tFp[i] - j->Fp[i]) / eps / j->sFp;
  }
}

/* Scaled preconditioner Mhat^{-1} r = S_X^{-1} P^{-1} S_F r. */
static void jf_prec(jf_ctx* j, const double* r, double* out) {
  int n = j->n;
  if (j->P->precond == 0) { memcpy(out, r, sizeof(double) * 2 * n); return; }
  for (int i = 0; i < n; ++i) { j->u1[i] = r[i] * j->sFe; j->u2[i] = r[n + i] * j->sFp; }
  or_prec_apply(&j->prec, j->u1, j->u2, out, out + n);
  for (int i = 0; i < n; ++i) { out[i] /= j->sn; out[n + i] /= j->sp; }
}

static void jf_jvp_op(void* ctx, const double* v, double* w) { jf_jvp((jf_ctx*)ctx, v, w); }
static void jf_prec_op(void* ctx, const double* v, double* w) { jf_prec((jf_ctx*)ctx, v, w); }

/* Right-preconditioned operator y -> Jhat Mhat^{-1} y. */
static void jf_op(void* ctx, const double* v, double* w) {
  jf_ctx* j = (jf_ctx*)ctx;
  jf_prec(j, v, j->t2);
  jf_jvp(j, j->t2, w);
}

static double scaled_norms(int n, const double* Fe, const double* Fp, double sFe,
                           double sFp, double* two) {
  double mx = 0.0, s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = fabs(Fe[i] / sFe), b = fabs(Fp[i] / sFp);
    if (a > mx) mx = a;
    if (b > mx) mx = b;
    s2 += a * a + b * b;
  }
  if (two) *two = sqrt(s2);
  if (!isfinite(s2)) mx = INFINITY;
  return mx;
}

static double maxabs(int n, const double* a) {
  double m = 0.0;
  for (int i = 0; i < n; ++i) if (fabs(a[i]) > m) m = fabs(a[i]);
  return m;
}

/* Preconditioner blocks of Eq. linear_nls at the iterate (ne, phi_ref + psi):
 * A, B, L from the analytic Jacobian, S~ = L + C B = L - B (C = -I), and the
 * multigrid hierarchies where the blocks are solved by V-cycles. phin is
 * scratch for phi. */
static void build_prec(const or_col* c, or_prec* pr, const double* ne, const double* psi,
                       double* phin) {
  const int n = c->n;
  for (int i = 0; i < n; ++i) phin[i] = phi_ref(c, i) + psi[i];
  or_jacobian_col(c, ne, phin, pr->A, pr->B, pr->L);
  for (int i = 0; i < n; ++i) {
    pr->S.sub[i] = pr->L.sub[i] - pr->B.sub[i];
    pr->S.dia[i] = pr->L.dia[i] - pr->B.dia[i];
    pr->S.sup[i] = pr->L.sup[i] - pr->B.sup[i];
  }
  if (pr->mgA) or_mg_setup(pr->mgA, pr->A.sub, pr->A.dia, pr->A.sup);
  if (pr->mgS) or_mg_setup(pr->mgS, pr->S.sub, pr->S.dia, pr->S.sup);
}

void or_jfnk_col(const or_params* P, const or_col* c, const double* ne_old,
                 const double* phi_old, const double* ne0, const double* phi0,
                 double* ne, double* phi, or_stats* st) {
  const int n = c->n;
  memset(st, 0, sizeof(*st));
  memcpy(ne, ne0 ? ne0 : ne_old, sizeof(double) * n);
  memcpy(phi, phi0 ? phi0 : phi_old, sizeof(double) * n);
  if (n < 2 || !(c->h > 0.0) || !(c->dt > 0.0) || !finite_vec(n, ne_old) ||
      !finite_vec(n, phi_old) || !finite_vec(n, c->fe) || !finite_vec(n, c->fphi) ||
      !finite_vec(n, ne) || !finite_vec(n, phi) || !isfinite(c->vl) || !isfinite(c->vr)) {
    st->status = OR_BAD_INPUT;
    return;
  }
  for (int i = 0; i < n; ++i)
    if (!(c->D[i] > 0.0) || !isfinite(c->D[i])) { st->status = OR_BAD_INPUT; return; }

  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 52);
  double* Fe = buf;             double* Fp = buf + n;
  double* tn = buf + 2 * n;     double* tp = buf + 3 * n;
  double* tFe = buf + 4 * n;    double* tFp = buf + 5 * n;
  double* u1 = buf + 6 * n;     double* u2 = buf + 7 * n;
  double* rhs = buf + 8 * n;    /* 2n */
  double* dX = buf + 10 * n;    /* 2n */
  double* tri = buf + 12 * n;   /* 9n: A, B, L */
  double* Sd = buf + 21 * n;    /* 3n: S~ */
  double* pw = buf + 24 * n;    /* 12n: preconditioner scratch */
  double* psi = buf + 36 * n;
  double* trial_n = buf + 37 * n; double* trial_p = buf + 38 * n;
  double* trial_Fe = buf + 39 * n; double* trial_Fp = buf + 40 * n;
  double* y = buf + 41 * n;     /* 2n */
  double* t2 = buf + 43 * n;    /* 2n */
  double* phin = buf + 45 * n;

  for (int i = 0; i < n; ++i) psi[i] = phi[i] - phi_ref(c, i);

  /* typical values at the plain start X^n (Eq. newton_sc, Algorithm 2 first line) */
  double sn = fmax(fmax(maxabs(n, ne_old), maxabs(n, c->fphi)), 1.0);
  double sp = fmax(fmax(maxabs(n, phi_old), fmax(fabs(c->vl), fabs(c->vr))), 1.0);
  for (int i = 0; i < n; ++i) tp[i] = phi_old[i] - phi_ref(c, i);
  or_residual_psi(c, ne_old, tp, Fe, Fp);
  st->res_evals++;
  double sFe = fmax(fmax(maxabs(n, Fe), maxabs(n, c->fe)), 1e-12 * sn);
  double sFp = fmax(fmax(maxabs(n, Fp), maxabs(n, c->fphi)), 1e-12 * sn);
  if (ne0 || phi0) { or_residual_psi(c, ne, psi, Fe, Fp); st->res_evals++; }

  jf_ctx J;
  J.c = c; J.P = P; J.n = n; J.sn = sn; J.sp = sp; J.sFe = sFe; J.sFp = sFp;
  J.ne = ne; J.psi = psi; J.Fe = Fe; J.Fp = Fp;
  J.tn = tn; J.tp = tp; J.tFe = tFe; J.tFp = tFp; J.u1 = u1; J.u2 = u2; J.t2 = t2;
  J.res_evals = &st->res_evals;
  or_tri A = {tri, tri + n, tri + 2 * n}, B = {tri + 3 * n, tri + 4 * n, tri + 5 * n},
         L = {tri + 6 * n, tri + 7 * n, tri + 8 * n}, S = {Sd, Sd + n, Sd + 2 * n};
  J.prec.n = n; J.prec.mode = P->precond; J.prec.A = A; J.prec.B = B; J.prec.L = L;
  J.prec.S = S; J.prec.work = pw;
  or_mg mgA, mgS;
  J.prec.mgA = J.prec.mgS = NULL;
  J.prec.gA = P->mg_gamma_A; J.prec.gS = P->mg_gamma_S;
  J.prec.max_cycles = P->mg_max_cycles;
  J.prec.cycles = &st->mg_cycles;
  if (P->precond == 3) {
    if (P->mg_gamma_A > 0.0) { or_mg_init(&mgA, n, P->mg_transfer); J.prec.mgA = &mgA; }
    if (P->mg_gamma_S > 0.0) { or_mg_init(&mgS, n, P->mg_transfer); J.prec.mgS = &mgS; }
  }

  double fn2;
  double fninf = scaled_norms(n, Fe, Fp, sFe, sFp, &fn2);
  st->first_res = fninf;
  st->status = OR_MAX_NEWTON;
  int have_prec = 0;   /* preconditioner blocks built at an earlier iterate */
  int prec_cur = 0;    /* ... and those blocks were built at the current iterate */
  const int from_guess = ne0 != NULL || phi0 != NULL;   /* a supplied start */
  int polished = 0;    /* Newton steps taken for the error test */
  for (int l = 0;; ++l) {
    if (!isfinite(fninf)) { st->status = OR_NONFINITE; break; }
    int polish = 0;    /* the residual test holds; this step serves the error test */
    if (fninf < P->eps_F) {
      /* Error test (eps_E > 0). Sec. 3.2 asks that the tolerances keep the
       * nonlinear solution error small; the residual test bounds the error only
       * through the conditioning of S_F^-1 J S_X, which is large for columns
       * whose potential scale (a few volts) is small beside their space-charge
       * scale. The Newton correction e = P^-1 F(X^(l)), with the preconditioner
       * of the last Newton step (built at X^(l) if there was none; with the
       * exact Schur form P = J), estimates the error of X^(l). The column stops
       * when max|e_n| <= eps_E max|n| and max|e_phi| <= eps_E max|phi|;
       * otherwise it takes one more Newton step. Blocks built at the previous
       * iterate misjudge the error by the change of J over the last step; from
       * the plain start the last step is small and the estimate matches the
       * true error, but a supplied (learned) start can end with a large step:
       * there an estimate that passes within a factor OR_ERR_MARGIN of the bar
       * is taken again with blocks built at X^(l). */
      if (!(P->eps_E > 0.0) || l >= P->max_newton || polished >= OR_MAX_POLISH) {
        st->status = OR_OK;
        break;
      }
      if (!have_prec) {
        build_prec(c, &J.prec, ne, psi, phin);
        have_prec = 1;
        prec_cur = 1;
      }
      double nmax = maxabs(n, ne), pmax = 0.0;
      for (int i = 0; i < n; ++i) pmax = fmax(pmax, fabs(phi_ref(c, i) + psi[i]));
      double en = 0.0, ep = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < n; ++i) { rhs[i] = Fe[i] / sFe; rhs[n + i] = Fp[i] / sFp; }
        jf_prec(&J, rhs, dX);
        en = sn * maxabs(n, dX);
        ep = sp * maxabs(n, dX + n);
        const int marginal = en > P->eps_E / OR_ERR_MARGIN * nmax ||
                             ep > P->eps_E / OR_ERR_MARGIN * pmax;
        if (!from_guess || prec_cur || !marginal ||
            !(en <= P->eps_E * nmax && ep <= P->eps_E * pmax))
          break;
        build_prec(c, &J.prec, ne, psi, phin);
        prec_cur = 1;
      }
      if (en <= P->eps_E * nmax && ep <= P->eps_E * pmax) { st->status = OR_OK; break; }
      polish = 1;
    }
    if (l >= P->max_newton) { st->status = OR_MAX_NEWTON; break; }
    /* build the preconditioner blocks at X^(l) */
    build_prec(c, &J.prec, ne, psi, phin);
    double xs = 0.0;
    for (int i = 0; i < n; ++i) xs += (ne[i] / sn) * (ne[i] / sn) + (phin[i] / sp) * (phin[i] / sp);
    J.xnorm = sqrt(xs);
    /* GMRES on Jhat Mhat^{-1} y = -Fhat from y = 0; delta = Mhat^{-1} y. The search
     * space Mhat^{-1} K_p(Jhat Mhat^{-1}, Fhat) equals K_p(Mhat^{-1} Jhat, Mhat^{-1} Fhat),
     * the Krylov space of Algorithm 2, and the minimised residual is the
     * unpreconditioned ||Jhat delta + Fhat||_2 that Algorithm 2 tests against gamma. */
    for (int i = 0; i < n; ++i) { rhs[i] = -Fe[i] / sFe; rhs[n + i] = -Fp[i] / sFp; }
    int its = 0;
    double est = 0.0;
    int conv;
    if (P->precond == 3) {
      /* multigrid block solves to a tolerance: a varying preconditioner */
      conv = or_fgmres(2 * n, jf_jvp_op, jf_prec_op, &J, rhs, dX, P->restart_m, P->gamma,
                       P->max_krylov, &its, &est);
    } else {
      conv = or_gmres(2 * n, jf_op, &J, rhs, y, P->restart_m, P->gamma, P->max_krylov,
                      &its, &est);
      jf_prec(&J, y, dX);
    }
    st->krylov_it += its;
    if (!conv) st->krylov_capped++;
    have_prec = 1;
    /* backtracking line search. A step taken for the error test tries lam = 1
     * only and is also accepted if the new iterate still passes the residual
     * test: near the rounding floor of F the sufficient decrease of the scaled
     * 2-norm (dominated by the Poisson block's floor) can fail while the step
     * still removes the error. If neither holds, the column keeps X^(l), which
     * passed the residual test. */
    double lam = 1.0;
    int accepted = 0;
    double tr2 = 0.0, trinf = 0.0;
    const int max_ls = polish ? 0 : P->max_linesearch;
    for (int t = 0; t <= max_ls; ++t) {
      for (int i = 0; i < n; ++i) {
        trial_n[i] = ne[i] + lam * sn * dX[i];
        trial_p[i] = psi[i] + lam * sp * dX[n + i];
      }
      or_residual_psi(c, trial_n, trial_p, trial_Fe, trial_Fp);
      st->res_evals++;
      trinf = scaled_norms(n, trial_Fe, trial_Fp, sFe, sFp, &tr2);
      if (isfinite(tr2) && (tr2 <= (1.0 - P->ls_alpha * lam * (1.0 - P->gamma)) * fn2 ||
                            (polish && trinf < P->eps_F))) {
        accepted = 1;
        break;
      }
      if (t < max_ls) { lam *= 0.5; st->ls_halvings++; }
    }
    if (!accepted && polish) { st->status = OR_OK; break; }
    if (!accepted) { st->status = conv ? OR_LINESEARCH_FAIL : OR_MAX_KRYLOV; break; }
    memcpy(ne, trial_n, sizeof(double) * n);
    memcpy(psi, trial_p, sizeof(double) * n);
    memcpy(Fe, trial_Fe, sizeof(double) * n);
    memcpy(Fp, trial_Fp, sizeof(double) * n);
    fn2 = tr2;
    fninf = trinf;
    st->newton_it++;
    polished += polish;
    prec_cur = 0;
    if (P->eps_X > 0.0) {
      double st_inf = lam * maxabs(2 * n, dX);
      if (st_inf < P->eps_X && fninf >= P->eps_F) { st->status = OR_OK; break; }
    }
  }
  for (int i = 0; i < n; ++i) phi[i] = phi_ref(c, i) + psi[i];
  st->final_res = fninf;
  if (J.prec.mgA) or_mg_free(J.prec.mgA);
  if (J.prec.mgS) or_mg_free(J.prec.mgS);
  free(buf);
}

/* ------------------------------------------------------------------------ */
/* Batch entry points (SoA layout, columns packed back to back).            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t ncol;
  const int64_t* col_off;
  const double *length, *dt, *v_left, *v_right;
  const double *ne_old, *phi_old;
  int n_species;
  const int* valence;
  const double* n_ion;          /* [n_species][cells] */
  const double *T, *u_adv, *i_re;
  const double* rho;            /* [cells] gas density (transport tables only) */
} or_batch;

/* Per-column derived inputs: f_e, f_phi and D (Einstein relation). */
static void build_col(const or_params* P, const or_batch* b, int64_t c, or_col* col,
                      double* buf /* 5 n */) {
  double *fe = buf, *fphi = buf + (b->col_off[c + 1] - b->col_off[c]);
  double* D = fphi + (b->col_off[c + 1] - b->col_off[c]);
  double* cprog = D + (b->col_off[c + 1] - b->col_off[c]);
  double* Ngas = cprog + (b->col_off[c + 1] - b->col_off[c]);
  int64_t a = b->col_off[c], e = b->col_off[c + 1];
  int n = (int)(e - a);
  int64_t ncells = b->col_off[b->ncol];
  col->n = n;
  col->h = b->length[c] / n;
  col->dt = b->dt[c];
  col->vl = b->v_left[c];
  col->vr = b->v_right[c];
  col->mu = P->mobility;
  col->eps_r = P->eps_r;
  col->bc = P->bc_electron;
  for (int i = 0; i < n; ++i) {
    fe[i] = b->ne_old[a + i] + (b->i_re ? col->dt * b->i_re[a + i] : 0.0);
    double q = 0.0;
    for (int s = 0; s < b->n_species; ++s) q += b->valence[s] * b->n_ion[s * ncells + a + i];
    fphi[i] = q;
    D[i] = P->mobility * OR_KB * b->T[a + i] / OR_E;
  }
  col->fe = fe;
  col->fphi = fphi;
  col->D = D;
  col->U = b->u_adv ? b->u_adv + a : NULL;
  col->tab_mu = col->tab_D = NULL;
  col->cprog = col->Ngas = NULL;
  if (P->transport == 1) {
    for (int i = 0; i < n; ++i) {
      double cp = (b->T[a + i] - P->T_in) / (P->T_max - P->T_in);
      cprog[i] = cp < 0.0 ? 0.0 : (cp > 1.0 ? 1.0 : cp);
      Ngas[i] = b->rho[a + i] * OR_NA / P->gas_molar_mass;
    }
    col->tab_mu = P->tab_mu;
    col->tab_D = P->tab_D;
    col->tab_nc = P->tab_nc;
    col->tab_nx = P->tab_nx;
    col->tab_en_max = P->tab_en_max;
    col->cprog = cprog;
    col->Ngas = Ngas;
  }
}

void or_residual_batch(const or_params* P, const or_batch* b, const double* ne,
                       const double* phi, double* Fe, double* Fp) {
  for (int64_t c = 0; c < b->ncol; ++c) {
    int n = (int)(b->col_off[c + 1] - b->col_off[c]);
    if (n < 2) continue;
    double* tmp = (double*)malloc(sizeof(double) * 5 * n);
    or_col col;
    build_col(P, b, c, &col, tmp);
    int64_t a = b->col_off[c];
    or_residual_col(&col, ne + a, phi + a, Fe + a, Fp + a);
    free(tmp);
  }
}

void or_jacobian_batch(const or_params* P, const or_batch* b, const double* ne,
                       const double* phi, double* A3, double* B3, double* L3) {
  /* A3/B3/L3: [3][cells] as (sub, dia, sup) planes */
  int64_t ncells = b->col_off[b->ncol];
  for (int64_t c = 0; c < b->ncol; ++c) {
    int n = (int)(b->col_off[c + 1] - b->col_off[c]);
    if (n < 2) continue;
    double* tmp = (double*)malloc(sizeof(double) * 5 * n);
    or_col col;
    build_col(P, b, c, &col, tmp);
    int64_t a = b->col_off[c];
    or_tri A = {A3 + a, A3 + ncells + a, A3 + 2 * ncells + a};
    or_tri B = {B3 + a, B3 + ncells + a, B3 + 2 * ncells + a};
    or_tri L = {L3 + a, L3 + ncells + a, L3 + 2 * ncells + a};
    or_jacobian_col(&col, ne + a, phi + a, A, B, L);
    free(tmp);
  }
}

/* Apply the preconditioner (P->precond) of one column built at (ne, phi). */
void or_prec_apply_col(const or_params* P, const or_batch* b, int64_t c, const double* ne,
                       const double* phi, const double* v1, const double* v2, double* x1,
                       double* x2, int* cycles /* precond 3: V-cycles used, or NULL */) {
  int n = (int)(b->col_off[c + 1] - b->col_off[c]);
  double* tmp = (double*)malloc(sizeof(double) * 21 * n);
  or_col col;
  build_col(P, b, c, &col, tmp);
  int64_t a = b->col_off[c];
  double* t = tmp + 5 * n;
  or_tri A = {t, t + n, t + 2 * n}, B = {t + 3 * n, t + 4 * n, t + 5 * n},
         L = {t + 6 * n, t + 7 * n, t + 8 * n}, S = {t + 9 * n, t + 10 * n, t + 11 * n};
  or_jacobian_col(&col, ne + a, phi + a, A, B, L);
  for (int i = 0; i < n; ++i) {
    S.sub[i] = L.sub[i] - B.sub[i];
    S.dia[i] = L.dia[i] - B.dia[i];
    S.sup[i] = L.sup[i] - B.sup[i];
  }
  double* w = (double*)malloc(sizeof(double) * 12 * n);
  or_prec pr = {n, P->precond == 2 ? 2 : (P->precond == 3 ? 3 : 1), A, B, L, S, w,
                NULL, NULL, P->mg_gamma_A, P->mg_gamma_S, P->mg_max_cycles, cycles};
  or_mg mgA, mgS;
  if (pr.mode == 3 && P->mg_gamma_A > 0.0) {
    or_mg_init(&mgA, n, P->mg_transfer); or_mg_setup(&mgA, A.sub, A.dia, A.sup); pr.mgA = &mgA;
  }
  if (pr.mode == 3 && P->mg_gamma_S > 0.0) {
    or_mg_init(&mgS, n, P->mg_transfer); or_mg_setup(&mgS, S.sub, S.dia, S.sup); pr.mgS = &mgS;
  }
  if (cycles) *cycles = 0;
  or_prec_apply(&pr, v1, v2, x1, x2);
  if (pr.mgA) or_mg_free(&mgA);
  if (pr.mgS) or_mg_free(&mgS);
  free(w);
  free(tmp);
}

void or_solve_batch(const or_params* P, const or_batch* b, const double* ne_guess,
                    const double* phi_guess, double* ne_out, double* phi_out, int* status,
                    int* newton_it, int* krylov_it, int* res_evals, double* final_res,
                    int* mg_cycles, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t c = 0; c < b->ncol; ++c) {
    int64_t a = b->col_off[c];
    int n = (int)(b->col_off[c + 1] - a);
    or_stats st;
    memset(&st, 0, sizeof(st));
    if (n < 2) {
      st.status = OR_BAD_INPUT;
      for (int i = 0; i < n; ++i) { ne_out[a + i] = b->ne_old[a + i]; phi_out[a + i] = b->phi_old[a + i]; }
    } else {
      double* tmp = (double*)malloc(sizeof(double) * 5 * n);
      or_col col;
      build_col(P, b, c, &col, tmp);
      or_jfnk_col(P, &col, b->ne_old + a, b->phi_old + a,
                  ne_guess ? ne_guess + a : NULL, phi_guess ? phi_guess + a : NULL,
                  ne_out + a, phi_out + a, &st);
      free(tmp);
    }
    if (status) status[c] = st.status;
    if (newton_it) newton_it[c] = st.newton_it;
    if (krylov_it) krylov_it[c] = st.krylov_it;
    if (res_evals) res_evals[c] = st.res_evals;
    if (final_res) final_res[c] = st.final_res;
    if (mg_cycles) mg_cycles[c] = st.mg_cycles;
  }
}

/* ------------------------------------------------------------------------ */
/* Provisional charged species between SDC iterations (Algorithm 1 calls the */
/* electric solve with provisional ion fields; only their electric drift is  */
/* modelled here): explicit first-order upwind update of each species,       */
/*   n~_i = n_i - (dt/h) (Phi_{i+1/2} - Phi_{i-1/2}),                         */
/*   Phi = w n_upwind, w = nu kappa_ion E_face (Eq. for U_ef,m with U = 0),   */
/* E_face = -dphi/dx at interior faces and from the quadratic electrode      */
/* stencil at the electrodes, which absorb outgoing ions and emit none.      */
/* ------------------------------------------------------------------------ */
void or_ion_update_batch(const or_batch* b, const double* phi, double kappa_ion,
                         double* n_out) {
  int64_t ncells = b->col_off[b->ncol];
  for (int64_t c = 0; c < b->ncol; ++c) {
    int64_t a = b->col_off[c];
    int n = (int)(b->col_off[c + 1] - a);
    if (n < 2) continue;
    double h = b->length[c] / n, dt = b->dt[c];
    const double* p = phi + a;
    double GL = (-8.0 * b->v_left[c] + 9.0 * p[0] - p[1]) / (3.0 * h);
    double GR = (8.0 * b->v_right[c] - 9.0 * p[n - 1] + p[n - 2]) / (3.0 * h);
    for (int s = 0; s < b->n_species; ++s) {
      const double* ni = b->n_ion + s * ncells + a;
      double* no = n_out + s * ncells + a;
      double nu = (double)b->valence[s];
      double wl = -nu * kappa_ion * GL;          /* drift velocity at x = 0 */
      double flux_prev = wl < 0.0 ? wl * ni[0] : 0.0;
      for (int i = 0; i < n; ++i) {
        double flux_next;
        if (i == n - 1) {
          double wr = -nu * kappa_ion * GR;
          flux_next = wr > 0.0 ? wr * ni[n - 1] : 0.0;
        } else {
          double w = -nu * kappa_ion * (p[i + 1] - p[i]) / h;
          flux_next = w * (w > 0.0 ? ni[i] : ni[i + 1]);
        }
        no[i] = ni[i] - (dt / h) * (flux_next - flux_prev);
        flux_prev = flux_next;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Provisional charged species of an SDC iteration with the transport of     */
/* Sec. 3.1 and Algorithm 1: for each species m                               */
/*   n~ = n^n + dt [A^{n+1/2} + (D n^n - D n^(k)) / 2 + D n~],                */
/* i.e. one implicit diffusion solve                                          */
/*   (I - dt D) n~ = n^n + dt A^{n+1/2} + (dt / 2)(D n^n - D n^(k)),          */
/* n^(k) the previous SDC iterate (n^n at the first iteration, where the      */
/* correction vanishes); no reactions (the columns carry no chemistry).       */
/*  A: advection with the effective velocity w = U_f + nu kappa E_f          */
/*     (E = -dphi/dx of the current potential), by a second-order Godunov     */
/*     (MUSCL) scheme: the face state is the upwind cell value extrapolated   */
/*     to the face and to t^{n+1/2} along the characteristic,                 */
/*       n_{i+1/2} = n_i + (1 - w dt/h) s_i / 2        (w >= 0)               */
/*                 = n_{i+1} - (1 + w dt/h) s_{i+1} / 2 (w < 0),              */
/*     s the monotonized-central limited difference of n^n (0 in the end      */
/*     cells); electrodes pass the outgoing drift of the edge cell only.      */
/*  D: (D n)_i = [D_{i+1/2}(n_{i+1} - n_i) - D_{i-1/2}(n_i - n_{i-1})] / h^2,  */
/*     D = kappa k_B T_f / (|nu| e) (Einstein, T_f the face mean), no         */
/*     diffusive flux through the electrodes.                                 */
/* ------------------------------------------------------------------------ */
static double mc_slope(double dm, double dp) {
  if (dm * dp <= 0.0) return 0.0;
  double a = fabs(dm), b = fabs(dp), c = 0.5 * fabs(dm + dp);
  double m = 2.0 * a < 2.0 * b ? 2.0 * a : 2.0 * b;
  if (c < m) m = c;
  return dm > 0.0 ? m : -m;
}

void or_ion_provisional_batch(const or_batch* b, const double* phi, const double* n_prev,
                              double kappa_ion, double* n_out) {
  int64_t ncells = b->col_off[b->ncol];
  for (int64_t c = 0; c < b->ncol; ++c) {
    int64_t a = b->col_off[c];
    int n = (int)(b->col_off[c + 1] - a);
    if (n < 2) {
      for (int s = 0; s < b->n_species; ++s)
        for (int i = 0; i < n; ++i) n_out[s * ncells + a + i] = b->n_ion[s * ncells + a + i];
      continue;
    }
    double h = b->length[c] / n, dt = b->dt[c];
    const double* p = phi + a;
    const double* T = b->T + a;
    const double* U = b->u_adv ? b->u_adv + a : NULL;
    double GL = (-8.0 * b->v_left[c] + 9.0 * p[0] - p[1]) / (3.0 * h);
    double GR = (8.0 * b->v_right[c] - 9.0 * p[n - 1] + p[n - 2]) / (3.0 * h);
    double* F = (double*)malloc(sizeof(double) * (n + 1));      /* advective face fluxes */
    double* Df = (double*)malloc(sizeof(double) * (n + 1));     /* face diffusivities    */
    double* sl = (double*)malloc(sizeof(double) * n);
    double* rhs = (double*)malloc(sizeof(double) * n);
    double* sub = (double*)malloc(sizeof(double) * n);
    double* dia = (double*)malloc(sizeof(double) * n);
    double* sup = (double*)malloc(sizeof(double) * n);
    double* work = (double*)malloc(sizeof(double) * 2 * n);
    for (int s = 0; s < b->n_species; ++s) {
      const double* n0 = b->n_ion + s * ncells + a;
      const double* nk = n_prev ? n_prev + s * ncells + a : n0;
      double* no = n_out + s * ncells + a;
      double nu = (double)b->valence[s];
      double Dc = nu != 0.0 ? kappa_ion * OR_KB / (fabs(nu) * OR_E) : 0.0;
      for (int i = 0; i < n; ++i)
        sl[i] = (i == 0 || i == n - 1) ? 0.0 : mc_slope(n0[i] - n0[i - 1], n0[i + 1] - n0[i]);
      for (int f = 0; f <= n; ++f) {
        if (f == 0 || f == n) {
          double w = (U ? U[f == 0 ? 0 : n - 1] : 0.0) + nu * kappa_ion * (f == 0 ? -GL : -GR);
          int out = f == 0 ? w < 0.0 : w > 0.0;
          F[f] = out ? w * (f == 0 ? n0[0] : n0[n - 1]) : 0.0;
          Df[f] = 0.0;
        } else {
          int i = f - 1;
          double w = (U ? 0.5 * (U[i] + U[i + 1]) : 0.0) - nu * kappa_ion * (p[i + 1] - p[i]) / h;
          double cfl = w * dt / h;
          double nf = w >= 0.0 ? n0[i] + 0.5 * (1.0 - cfl) * sl[i]
                               : n0[i + 1] - 0.5 * (1.0 + cfl) * sl[i + 1];
          F[f] = w * nf;
          Df[f] = Dc * 0.5 * (T[i] + T[i + 1]);
        }
      }
      for (int i = 0; i < n; ++i) {
        double dn0 = (Df[i + 1] * ((i + 1 < n ? n0[i + 1] : n0[i]) - n0[i]) -
                      Df[i] * (n0[i] - (i > 0 ? n0[i - 1] : n0[i]))) / (h * h);
        double dnk = (Df[i + 1] * ((i + 1 < n ? nk[i + 1] : nk[i]) - nk[i]) -
                      Df[i] * (nk[i] - (i > 0 ? nk[i - 1] : nk[i]))) / (h * h);
        rhs[i] = n0[i] - (dt / h) * (F[i + 1] - F[i]) + 0.5 * dt * (dn0 - dnk);
        sub[i] = -dt * Df[i] / (h * h);
        sup[i] = -dt * Df[i + 1] / (h * h);
        dia[i] = 1.0 - sub[i] - sup[i];
      }
      or_thomas(n, sub, dia, sup, rhs, no, work);
    }
    free(F); free(Df); free(sl); free(rhs); free(sub); free(dia); free(sup); free(work);
  }
}

/* ------------------------------------------------------------------------ */
/* Charge flux through every face (Sec. 4.4, i-V curves): J_m = nu_m e       */
/* Gamma_m with Gamma_m the number flux of species m, J+ the sum over the    */
/* positive ions, J- over the negative ions and the electrons, J = J+ + J-.  */
/*   electrons: the Scharfetter-Gummel flux of the residual (Eq. nls), the    */
/*     electrode faces by the column's electron boundary condition;          */
/*   ions: drift with the effective velocity U_ef,m = U + nu_m kappa E        */
/*     (E = -dphi/dx) carrying the upwind cell value, plus diffusion          */
/*     -D_m dn_m/dx with D_m = kappa k_B T / (|nu_m| e) (Einstein), the face  */
/*     value the mean of the two cells; at an electrode only an outgoing     */
/*     drift flux (absorbing, as in the provisional update).                 */
/* Faces of column c: [col_off[c] + c, col_off[c+1] + c], N + 1 of them,     */
/* face 0 on the left electrode.                                              */
/* ------------------------------------------------------------------------ */
void or_current_batch(const or_params* P, const or_batch* b, const double* ne,
                      const double* phi, double kappa_ion, double* j_pos, double* j_neg) {
  int64_t ncells = b->col_off[b->ncol];
  for (int64_t c = 0; c < b->ncol; ++c) {
    int64_t a = b->col_off[c];
    int n = (int)(b->col_off[c + 1] - a);
    int64_t f0 = a + c;
    for (int f = 0; f <= n; ++f) { j_pos[f0 + f] = 0.0; j_neg[f0 + f] = 0.0; }
    if (n < 2) continue;
    double* tmp = (double*)malloc(sizeof(double) * 5 * n);
    or_col col;
    build_col(P, b, c, &col, tmp);
    const double h = col.h;
    const double* p = phi + a;
    const double* x = ne + a;
    const double* U = col.U;
    double GL = (-8.0 * col.vl + 9.0 * p[0] - p[1]) / (3.0 * h);
    double GR = (8.0 * col.vr - 9.0 * p[n - 1] + p[n - 2]) / (3.0 * h);
    /* electrons */
    for (int f = 0; f <= n; ++f) {
      double gam;
      if (f == 0 || f == n) {
        double mub, Db;
        face_transport(&col, f == 0 ? 0 : n - 1, f == 0 ? 0 : n - 1, f == 0 ? GL : GR, &mub, &Db);
        double v = f == 0 ? (U ? U[0] : 0.0) + mub * GL : (U ? U[n - 1] : 0.0) + mub * GR;
        double ned = f == 0 ? x[0] : x[n - 1];
        int out = f == 0 ? v < 0.0 : v > 0.0;
        gam = (col.bc == OR_BC_ZERO_GRADIENT || out) ? v * ned : 0.0;
      } else {
        int i = f - 1;
        double muf, Df;
        face_transport(&col, i, i + 1, (p[i + 1] - p[i]) / h, &muf, &Df);
        double v = face_u(&col, i) + muf * (p[i + 1] - p[i]) / h;
        double Pe = v * h / Df;
        gam = (Df / h) * (or_bern(-Pe) * x[i] - or_bern(Pe) * x[i + 1]);
      }
      j_neg[f0 + f] += -OR_E * gam;
    }
    /* ions */
    for (int s = 0; s < b->n_species; ++s) {
      const double* ni = b->n_ion + s * ncells + a;
      double nu = (double)b->valence[s];
      if (nu == 0.0) continue;
      double* J = nu > 0.0 ? j_pos : j_neg;
      for (int f = 0; f <= n; ++f) {
        double gam;
        if (f == 0 || f == n) {
          double E = f == 0 ? -GL : -GR;
          double w = (f == 0 ? (U ? U[0] : 0.0) : (U ? U[n - 1] : 0.0)) + nu * kappa_ion * E;
          int out = f == 0 ? w < 0.0 : w > 0.0;
          gam = out ? w * (f == 0 ? ni[0] : ni[n - 1]) : 0.0;
        } else {
          int i = f - 1;
          double E = -(p[i + 1] - p[i]) / h;
          double w = face_u(&col, i) + nu * kappa_ion * E;
          double Di = 0.5 * (b->T[a + i] + b->T[a + i + 1]) * kappa_ion * OR_KB / (fabs(nu) * OR_E);
          gam = w * (w > 0.0 ? ni[i] : ni[i + 1]) - Di * (ni[i + 1] - ni[i]) / h;
        }
        J[f0 + f] += nu * OR_E * gam;
      }
    }
    free(tmp);
  }
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
