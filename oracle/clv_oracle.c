/*
 * clv_oracle.c -- plain, slow, FP64 CPU oracle for the CLVisc hydro step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * GPU path is compared against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library; the two only see the same seeded
 * inputs.
 *
 * What it computes (Pang, Petersen, Wang, "Pseudorapidity distribution and
 * decorrelation of anisotropic flow within CLVisc hydrodynamics"):
 *   - state in the tilde variables of Sec. 2 (T~^{tau mu}, pi~^{mu nu}, u~),
 *   - conservative tilde equations Eqs. (Ttilde), (pitilde) with the sources
 *     S_T, S_pi and I^{mu nu} of Sec. 2 (Eq. Ipi),
 *   - Kurganov-Tadmor central fluxes, Eqs. (kt) and (flux_out), Sec. 3,
 *   - the two-stage Runge-Kutta (Heun) update of Sec. 3 with the velocity
 *     extrapolation u* = 2u^n - u^{n-1} and the ideal first step,
 *   - primitive recovery T_ideal = T - pi -> (eps, u) by a root solve,
 *   - the vacuum cutoff eps < 1e-7 GeV/fm^3 -> eps = 0 (Sec. 5, Riemann test).
 *
 * Readings where the paper is silent, garbled or inconsistent (each one is
 * pinned by a test where a pin exists):
 *   R1  S_T carries a minus sign: S_T = -(T~^{eta eta}/tau, 0, 0, T~^{tau eta}/tau).
 *       Derived from nabla_mu T^{mu nu} = 0 with the Christoffel symbols of
 *       Eq. (christoffel); the printed plus sign contradicts Eq. (bjorken).
 *   R2  The pi~ u~^tau / tau term of S_pi enters with a minus sign.
 *   R3  I^{mu nu} enters S_pi with a minus sign (magnitudes as printed;
 *       I^{xx} = I^{xy} = I^{yy} = 0).
 *   R4  Slope limiter: minmod of backward and forward differences.
 *   R5  With one root solve per cell, interface states are built by the same
 *       limited reconstruction of T~^{tau mu}, pi~^{mu nu}, u~^tau, the axis
 *       velocity v^a = u~^a/u~^tau and P; Q_pi = u~^tau pi~ at each side.
 *       Flux of T~: v^a T~^{tau mu} + tau [P (v^a g~^{tau mu} - g~^{a mu})
 *       + pi~^{a mu} - v^a pi~^{tau mu}]; flux of Q_pi: v^a Q_pi.
 *   R6  Local speed: c = max over the two sides of (|v^a| + c_s)/(1 + |v^a| c_s),
 *       c_s of the cell on that side.
 *   R7  Spatial derivatives in sigma, theta, Du: central differences.  Time
 *       derivative: (u_late - u^n)/h, u_late = u* in stage 1, u' in stage 2.
 *   R8  First step: u^{-1} := 2u^0 - u^1_ideal, where u^1_ideal comes from one
 *       pi-free Heun step, so that u* = u^1_ideal.
 *   R9  lambda_1..3 = 0; bulk and net-baryon parts off unless asked for (the
 *       paper sets them to 0; R19, R20).
 *   R10 tau_pi = 5 eta_v/(eps + P) = 5 (eta/s) hbar c / T.
 *   R11 Conformal EOS: P = eps/3, eps = 3 g pi^2 T^4 / (90 (hbar c)^3), g = 47.5.
 *   R12 Tabulated EOS: nodes uniform in ln eps; P, T, c_s^2 linear in ln eps;
 *       below the first node P, c_s^2 of the first node scaled as described in
 *       eos_eval; above the last node conformal continuation.
 *   R13 Root solve on v in [0, M/E]: f(v) = v - M/(E + P(E - M v)).  E below the
 *       cutoff -> vacuum.  M > (1 - 1e-3) E -> M rescaled to (1 - 1e-3) E,
 *       which bounds the flow's Lorentz factor near 22.  The bound only acts
 *       in the dilute, ultra-relativistic fringe of an expanding event (the
 *       paper's analytic flows stay far below it).  There E/eps grows as
 *       gamma^2, so the rest-frame density eps = E - M v is ill-conditioned
 *       in the stored T~; a looser bound (1 - 1e-6, gamma up to ~700) let
 *       rounding-level differences of T~ grow into percent-level differences
 *       of eps near 1e-3 GeV/fm^3 after a few hundred steps.
 *   R14 Vacuum cells (eps < cutoff): eps = 0, u~ = (1, 0, 0, 0), pi~ = 0.
 *   R15 pi~ stage update: Q* = u~^{tau,n} pi~^n + h S1, pi~' = Q* / u~*^tau;
 *       Q^{n+1} = (u~^{tau,n} pi~^n + u~*^tau pi~' + h S2)/2,
 *       pi~^{n+1} = Q^{n+1}/u~'^tau.
 *   R16 sigma~ = grad^mu u^nu + grad^nu u^mu - u^mu Du^nu - u^nu Du^mu
 *       - (2/3) Delta^{mu nu} theta with finite-difference gradients.
 *   R17 Boundaries: two ghost cells per side, copies of the edge cell
 *       (zero gradient) or periodic wrap.
 *   R18 Shear regulator (the paper is silent; without one the dilute,
 *       ultra-relativistic edge of a viscous event runs away): after each
 *       stage update and before the root solve, with eps and P of the
 *       stage's input state of the cell,
 *         - pi~ is scaled by the ramp r(eps) = min(max(eps/eps_0 - 1, 0), 1)
 *           with eps_0 = 1e-3 GeV/fm^3: zero below eps_0 (ideal flow far
 *           below freeze-out densities), full above 2 eps_0, linear in
 *           between.  The ramp is continuous, so a rounding-level change of
 *           eps changes pi~ at the rounding level (a step at eps_0 switched
 *           a cell's whole pi~ on or off);
 *         - then pi~ is scaled by rho_max / rho wherever
 *           rho = sqrt(|pi~_{mu nu} pi~^{mu nu}|) / sqrt(eps^2 + 3 P^2)
 *           exceeds rho_max = 1.
 *   R19 Net charge (Eq. Ntilde with S_N = 0; the paper sets n = 0, so this
 *       is off unless an initial n is given): N~^tau = tau n u^tau (1 in
 *       place of tau in Cartesian mode) is conserved with the flux
 *       v^a N~^tau along each axis, through the same limited reconstruction
 *       of N~^tau and v^a and the same local speed as the other fields;
 *       the diffusion current d^mu is 0 (ideal charge transport).  Vacuum
 *       cells keep their charge.  n = N~^tau / (tau u^tau).
 *   R20 Bulk pressure (Eqs. Pi, Pitilde; the paper sets zeta = 0, so this is
 *       off unless zeta/s > 0, and runs with the shear machinery, eta/s > 0):
 *       Q_Pi = u~^tau Pi is carried with the flux v^a Q_Pi (the same limited
 *       reconstruction of u~^tau and Pi as for Q_pi), and Pi adds to the
 *       pressure everywhere T^{mu nu} appears: the T~ fluxes, S_T and the
 *       root solve (P(eps) + Pi).  Source, from Eq. (Pi) and the conservative
 *       form of Eq. (Pitilde):
 *         S_Pi = -(Pi + zeta theta~)/tau_Pi - Pi theta~/3 - Pi u~^tau/tau,
 *       theta~ = d~_mu u~^mu + u~^tau/tau; the printed -(Pi - zeta theta~)
 *       contradicts Eq. (Pi), and the Pi u~^tau/tau term follows from
 *       nabla_mu (Pi u^mu) as for pi~ (R2).  tau_Pi = 5 zeta/(T s) with
 *       constant zeta/s, so zeta/tau_Pi = (eps + P)/5.  Update as R15 for pi~.
 *       Regulator (as R18): Pi is scaled by the ramp r(eps) of the stage's
 *       input eps, then |Pi| <= P of that eps.  Vacuum cells: Pi = 0.  The pressure of T^{mu nu} is
 *       max(P + Pi, 0): the bound uses P of the stage's input, and where eps
 *       then falls P(eps) + Pi can dip below 0, which leaves the root
 *       function f(v) of the solve with two roots or none in [0, M/E]; with
 *       the floor (and d(P + Pi)/d eps = 0 on it) f is increasing and its
 *       root unique.  A negative total pressure is outside the validity of
 *       the second-order equations anyway.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 * Parity: bit-level determinism across thread counts (each cell is computed
 * independently; reductions are serial).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Planted mistakes, compiled in only by the pin meta-test (tests build a
 * separate copy with -DPLANT=<n>) to show that some pin fails for each. */
#ifndef PLANT
#define PLANT 0
#endif

#define HBARC 0.1973269804
#define DOF_CONF 47.5
#define NPI 10

/* pi~ component order: tt tx ty te xx xy xe yy ye ee (t = tau, e = eta_s) */
static const int PI_IDX[4][4] = {
    {0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
/* tilde metric g~ = diag(1, -1, -1, -1) (Sec. 2) */
static const double GT[4] = {1.0, -1.0, -1.0, -1.0};

typedef struct {
  int nx, ny, neta;
  double dx, dy, deta;
  double tau0, dtau;
  double eta_over_s;
  int eos_kind;     /* 0 conformal, 1 table */
  int eos_n;
  double eos_lne0;  /* ln(eps) of node 0 */
  double eos_dlne;  /* node spacing in ln(eps) */
  const double *eos_P, *eos_T, *eos_cs2;
  int cartesian;    /* 1: Christoffel terms off, tau factors 1 */
  int periodic;     /* 1: periodic ghosts, 0: zero-gradient ghosts */
  double eps_cut;
  int nthreads;
  double taupi_coef;   /* b in tau_pi = b eta_v / (eps + P); 0 -> 5 (reading R10) */
  double lambda1_hat;  /* lambda_1 = lambda1_hat / eps (conformal scaling); 0 -> no lambda_1 term */
  double zeta_over_s;  /* bulk viscosity over entropy (R20); 0 -> no bulk pressure */
} orc_config;

typedef struct {
  double *T[4];   /* T~^{tau mu} */
  double *pi[NPI];
  double *ed;     /* eps */
  double *u[3];   /* u~^x, u~^y, u~^eta */
  double *N;      /* N~^tau (R19) */
  double *Pi;     /* bulk pressure (R20) */
} orc_fields;

typedef struct {
  orc_config c;
  double *eosP, *eosT, *eosC;
  int NX, NY, NE;   /* padded extents */
  size_t NG;        /* padded cell count */
  orc_fields s;     /* state at step n */
  orc_fields s1;    /* stage-1 result */
  double *up[3];    /* u~ spatial at step n-1 */
  double tau;
  long step;
  int viscous;
  int charge;       /* 1: net charge transported (R19) */
  int bulk;         /* 1: bulk pressure evolved (R20) */
  long n_rescaled, n_rootfail;
  double stats[8];
} orc_t;

/* ------------------------------------------------------------------ */
static size_t IX(const orc_t* h, int i, int j, int k) {
  return ((size_t)(i + 2) * h->NY + (size_t)(j + 2)) * h->NE + (size_t)(k + 2);
}

static double tau_scale(const orc_t* h, double tau) { return h->c.cartesian ? 1.0 : tau; }
/* 1/tau wherever a Christoffel symbol contributes; 0 in Cartesian mode. */
static double geo(const orc_t* h, double tau) { return h->c.cartesian ? 0.0 : 1.0 / tau; }

/* ---------------------------- EOS (Sec. 3, Fig. eos) ----------------- */
static void eos_eval(const orc_t* h, double e, double* P, double* T, double* cs2) {
  if (h->c.eos_kind == 0) {
    *P = e / 3.0;
    *cs2 = 1.0 / 3.0;
    *T = (e > 0.0) ? pow(((PLANT == 29) ? 90.0 : 30.0) * HBARC * HBARC * HBARC * e / (DOF_CONF * M_PI * M_PI), 0.25)
                   : 0.0;
    return;
  }
  if (!(e > 0.0)) { *P = 0.0; *T = 0.0; *cs2 = h->eosC[0]; return; }
  int n = h->c.eos_n;
  double x = (log(e) - h->c.eos_lne0) / h->c.eos_dlne;
  if (x < 0.0) {
    /* below the first node: P proportional to eps, T to eps^(1/4) */
    double e0 = exp(h->c.eos_lne0);
    *P = h->eosP[0] * (e / e0);
    *T = h->eosT[0] * pow(e / e0, 0.25);
    *cs2 = h->eosC[0];
    return;
  }
  if (x >= (double)(n - 1)) {
    /* above the last node: conformal continuation */
    double etop = exp(h->c.eos_lne0 + (n - 1) * h->c.eos_dlne);
    *P = h->eosP[n - 1] + (e - etop) / 3.0;
    *T = h->eosT[n - 1] * pow(e / etop, 0.25);
    *cs2 = 1.0 / 3.0;
    return;
  }
  int k = (int)floor(x);
  if (k > n - 2) k = n - 2;
  double w = x - (double)k;
  *P = (PLANT == 28) ? w * h->eosP[k] + (1.0 - w) * h->eosP[k + 1] : (1.0 - w) * h->eosP[k] + w * h->eosP[k + 1];
  *T = (1.0 - w) * h->eosT[k] + w * h->eosT[k + 1];
  *cs2 = (1.0 - w) * h->eosC[k] + w * h->eosC[k + 1];
}

/* ------------------- primitive recovery (Sec. 3, R13) ---------------- */
/* Given E = T_ideal^{tau tau}, M = T_ideal^{tau i} (tilde components), find
 * eps and u~.  Returns number of iterations, -1 on iteration cap. */
static int prim_solve(const orc_t* h, double E, double Mx, double My, double Me, double Pshift,
                      double* eps, double u[4], int* rescaled) {
  *rescaled = 0;
  u[0] = 1.0; u[1] = u[2] = u[3] = 0.0;
  if (!(E >= h->c.eps_cut)) { *eps = 0.0; return 0; }
  double M = sqrt(Mx * Mx + My * My + Me * Me);
  double Mmax = (1.0 - 1e-3) * E;
  if (M > Mmax) {
    double s = Mmax / M;
    Mx *= s; My *= s; Me *= s;
    M = Mmax;
    *rescaled = 1;
  }
  if (M == 0.0) {
    *eps = E;
    if (*eps < h->c.eps_cut) *eps = 0.0;
    return 0;
  }
  double lo = 0.0, hi = M / E;
  double P, T, cs2;
  eos_eval(h, E, &P, &T, &cs2);
  P += Pshift;   /* bulk pressure, total floored at 0 (R20) */
  if (P < 0.0) P = 0.0;
  double v = M / (E + P);
  int it, ok = 0;
  for (it = 1; it <= 100; ++it) {
    double e = (PLANT == 8) ? E : E - M * v;
    eos_eval(h, e, &P, &T, &cs2);
    P += Pshift;
    if (P < 0.0) { P = 0.0; cs2 = 0.0; }
    double f = v - M / (E + P);
    if (f > 0.0) hi = v; else lo = v;
    double df = 1.0 - M * M * cs2 / ((E + P) * (E + P));
    double step = -f / df;
    /* a Newton step below the tolerance ends the solve; otherwise keep the
       iterate strictly inside the bracket (bisection when it leaves it) */
    if (fabs(step) <= 1e-15) { v += step; ok = 1; break; }
    double vn = v + step;
    if (!(vn > lo && vn < hi)) vn = 0.5 * (lo + hi);
    v = vn;
    if (hi - lo <= 1e-15) { ok = 1; break; }
  }
  double e = E - M * v;
  if (e < h->c.eps_cut) { *eps = 0.0; return ok ? it : -1; }
  *eps = e;
  double g = 1.0 / sqrt(1.0 - v * v);
  u[0] = g;
  u[1] = g * v * Mx / M;
  u[2] = g * v * My / M;
  u[3] = g * v * Me / M;
  return ok ? it : -1;
}

/* T~^{tau mu} from (eps, u~, pi~): tau_s [ (eps+P) u^tau u^mu - P g~^{tau mu} + pi~^{tau mu} ] */
static void T_from_prim(double taus, double e, double P, const double u[4], const double* pi,
                        double T[4]) {
  for (int m = 0; m < 4; ++m) {
    double v = (e + P) * u[0] * u[m] + (pi ? pi[PI_IDX[0][m]] : 0.0);
    if (m == 0) v -= P;
    T[m] = taus * v;
  }
}

/* ---------------- viscous source S_pi (Sec. 2, R2, R3, R16) ---------- */
/* du[a*4+b] = d~_a u~^b (a: tau, x, y, eta; tilde derivative d~_eta = d_eta/tau). */
static void source_pi(double g, const double u[4], const double du[16], const double pi[NPI],
                      double e, double P, double T, double eta_over_s, double taupi_coef,
                      double lambda1_hat, double S[NPI]) {
  double cov[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) cov[a][b] = du[a * 4 + b];
  /* corrected tilde covariant derivatives, Eq. (dtuz) */
  cov[3][0] += g * u[3];
  if (PLANT != 6) cov[3][3] += g * u[0];
  double theta = cov[0][0] + cov[1][1] + cov[2][2] + cov[3][3];
  double Du[4];
  for (int b = 0; b < 4; ++b) {
    Du[b] = 0.0;
    for (int a = 0; a < 4; ++a) Du[b] += u[a] * cov[a][b];
  }
  /* tau_pi = b eta_v / (eps + P) = b (eta/s) hbar c / T, so eta_v / tau_pi = (eps + P) / b */
  double b = (taupi_coef > 0.0) ? taupi_coef : 5.0;
  double inv_taupi = (eta_over_s > 0.0) ? T / (b * eta_over_s * HBARC) : 0.0;
  /* lambda_1 pi^<mu_lambda pi^nu>lambda of Eq. (pimn), in tilde components
     (the tilde metric contracts them like orthonormal ones): Y = pi g~ pi,
     X = Delta^mu_a Delta^nu_b Y^ab - Delta^mu nu (Delta_ab Y^ab) / 3 */
  double X[4][4] = {{0}};
  if (lambda1_hat != 0.0 && e > 0.0) {
    double Y[4][4], Dm[4][4];
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        double y = 0.0;
        for (int d = 0; d < 4; ++d) y += pi[PI_IDX[a][d]] * GT[d] * pi[PI_IDX[d][c]];
        Y[a][c] = y;
        Dm[a][c] = (a == c ? 1.0 : 0.0) - u[a] * GT[c] * u[c];   /* Delta^a_c */
      }
    double tr = 0.0;   /* Delta_ab Y^ab */
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) tr += ((a == c ? GT[a] : 0.0) - GT[a] * u[a] * GT[c] * u[c]) * Y[a][c];
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        double x = 0.0;
        for (int a = 0; a < 4; ++a)
          for (int c = 0; c < 4; ++c) x += Dm[m][a] * Dm[n][c] * Y[a][c];
        X[m][n] = x - ((m == n ? GT[m] : 0.0) - u[m] * u[n]) * tr / 3.0;
      }
  }
  const double l1 = (e > 0.0) ? lambda1_hat / e : 0.0;   /* lambda_1 */
  for (int m = 0; m < 4; ++m)
    for (int n = m; n < 4; ++n) {
      int id = PI_IDX[m][n];
      double grad_mn = GT[m] * cov[m][n];   /* grad^m u^n = g~^{mm} nabla_m u^n */
      double grad_nm = (PLANT == 5) ? GT[m] * cov[m][n] : GT[n] * cov[n][m];
      double Delta = (m == n ? GT[m] : 0.0) - u[m] * u[n];
      double sigma = grad_mn + grad_nm - u[m] * Du[n] - u[n] * Du[m] - (2.0 / 3.0) * Delta * theta;
      double s = -pi[id] * inv_taupi + (e + P) * sigma / b;
      s -= pi[id] * theta / 3.0;
      s -= l1 * inv_taupi * X[m][n];
      double acc = 0.0;
      for (int b = 0; b < 4; ++b)
        acc += GT[b] * (u[m] * pi[PI_IDX[n][b]] + u[n] * pi[PI_IDX[m][b]]) * Du[b];
      s -= acc;
      s -= ((PLANT == 2) ? -1.0 : 1.0) * g * u[0] * pi[id];
      S[id] = s;
    }
  /* Christoffel terms I^{mu nu}, Eq. (Ipi), entering with a minus sign (R3) */
  double ue = (PLANT == 1) ? -u[3] : u[3];
  S[0] -= 2.0 * g * ue * pi[3];
  S[1] -= g * ue * pi[6];
  S[2] -= g * ue * pi[8];
  S[3] -= g * ue * (pi[0] + pi[9]);
  S[6] -= g * ue * pi[1];
  S[8] -= g * ue * pi[2];
  S[9] -= 2.0 * g * ue * pi[3];
}

/* Shear regulator R18: pi scaled by the ramp r(eps) (0 below VISC_EPS_MIN,
 * 1 above twice it, linear between), then
 * |pi_{mu nu} pi^{mu nu}| <= rho_max^2 (eps^2 + 3 P^2). */
#define RHO_MAX 1.0
#define VISC_EPS_MIN 1e-3
static double visc_ramp(double e) {
  double r = e / VISC_EPS_MIN - ((PLANT == 27) ? 0.0 : 1.0);
  return r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
}
static void regulate_pi(const orc_t* h, double e, double* pi) {
  double r = visc_ramp(e);
  for (int q = 0; q < NPI; ++q) pi[q] *= r;
  if (r == 0.0) return;
  double P, T, cs2;
  eos_eval(h, e, &P, &T, &cs2);
  double pp = 0.0;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      double v = pi[PI_IDX[m][n]];
      pp += GT[m] * GT[n] * v * v;
    }
  double bound2 = RHO_MAX * RHO_MAX * (e * e + ((PLANT == 26) ? 0.0 : 3.0) * P * P);
  double a = fabs(pp);
  if (a > bound2) {
    double f = (bound2 > 0.0) ? sqrt(bound2 / a) : 0.0;
    for (int q = 0; q < NPI; ++q) pi[q] *= f;
  }
}

/* ------------------------- KT (Eqs. kt, flux_out) -------------------- */
#define NR 19 /* reconstructed: T(4) pi(10) u^tau v^a P(+Pi) N~^tau Pi */

/* bulk regulator (R20) with eps and P of the stage's input state */
static double regulate_Pi(const orc_t* h, double e, double Pb) {
  Pb *= visc_ramp(e);
  if (Pb == 0.0) return 0.0;
  double P, T, cs2;
  eos_eval(h, e, &P, &T, &cs2);
  if (Pb > P) return P;
  if (Pb < -P) return -P;
  return Pb;
}

static double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

typedef struct {
  const orc_t* h;
  const orc_fields* f;
  int viscous;
} view_t;

/* Cell quantities on axis a: R[17] and c_s. */
static void cell_R(const view_t* vw, size_t id, int axis, double R[NR], double* cs) {
  const orc_fields* f = vw->f;
  double u[4];
  u[1] = f->u[0][id]; u[2] = f->u[1][id]; u[3] = f->u[2][id];
  u[0] = sqrt(1.0 + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
  double P, T, cs2;
  eos_eval(vw->h, f->ed[id], &P, &T, &cs2);
  for (int m = 0; m < 4; ++m) R[m] = f->T[m][id];
  for (int q = 0; q < NPI; ++q) R[4 + q] = vw->viscous ? f->pi[q][id] : 0.0;
  R[14] = u[0];
  R[15] = u[axis] / u[0];
  R[18] = (vw->viscous && vw->h->bulk) ? f->Pi[id] : 0.0;
  R[16] = P + ((PLANT == 21) ? 0.0 : R[18]);   /* the pressure of T^{mu nu} (R20) */
  if (R[16] < 0.0) R[16] = 0.0;
  R[17] = f->N[id];
  *cs = sqrt(cs2);
}

/* Flux H at the interface between cells b and c on axis a, from cells a,b,c,d
 * (= i-1, i, i+1, i+2).  Q = (T~^{tau mu}, Q_pi = u~^tau pi~). */
static void kt_interface(const view_t* vw, int axis, double taus, size_t ia, size_t ib, size_t ic,
                         size_t id, double H[4 + NPI], double* HN, double* HPi) {
  double Ra[NR], Rb[NR], Rc[NR], Rd[NR], csa, csb, csc, csd;
  cell_R(vw, ia, axis, Ra, &csa);
  cell_R(vw, ib, axis, Rb, &csb);
  cell_R(vw, ic, axis, Rc, &csc);
  cell_R(vw, id, axis, Rd, &csd);
  double L[NR], Rr[NR];
  for (int q = 0; q < NR; ++q) {
    L[q] = Rb[q] + 0.5 * minmod(Rb[q] - Ra[q], Rc[q] - Rb[q]);
    Rr[q] = Rc[q] - ((PLANT == 24) ? -0.5 : 0.5) * minmod(Rc[q] - Rb[q], Rd[q] - Rc[q]);
  }
  double vl = L[15], vr = Rr[15];
  double lam_l = (fabs(vl) + csb) / (1.0 + fabs(vl) * csb);
  double lam_r = (fabs(vr) + ((PLANT == 25) ? csb : csc)) / (1.0 + fabs(vr) * ((PLANT == 25) ? csb : csc));
  double cmax = lam_l > lam_r ? lam_l : lam_r;
  double Fl[4 + NPI], Fr[4 + NPI], Ql[4 + NPI], Qr[4 + NPI];
  for (int side = 0; side < 2; ++side) {
    const double* S = side ? Rr : L;
    double* F = side ? Fr : Fl;
    double* Q = side ? Qr : Ql;
    double v = S[15], P = S[16];
    const double* pi = S + 4;
    for (int m = 0; m < 4; ++m) {
      /* v^a T~^{tau m} + tau [ P (v^a g~^{tau m} - g~^{a m}) + pi~^{a m} - v^a pi~^{tau m} ] */
      double gtm = (m == 0) ? 1.0 : 0.0;
      double gam = (m == axis) ? GT[m] : 0.0;
      F[m] = v * S[m] + taus * (P * (v * gtm - gam) + pi[PI_IDX[axis][m]] - v * pi[PI_IDX[0][m]]);
      Q[m] = S[m];
    }
    for (int q = 0; q < NPI; ++q) {
      Q[4 + q] = S[14] * pi[q];
      F[4 + q] = v * Q[4 + q];
    }
  }
  for (int q = 0; q < 4 + NPI; ++q)
    H[q] = 0.5 * (Fl[q] + Fr[q]) - 0.5 * cmax * (Qr[q] - Ql[q]);
  /* net charge (R19): flux v^a N~^tau */
  *HN = 0.5 * (vl * L[17] + vr * Rr[17]) - ((PLANT == 16) ? -0.5 : 0.5) * cmax * (Rr[17] - L[17]);
  /* bulk (R20): Q_Pi = u~^tau Pi on each side, flux v^a Q_Pi */
  double QPl = L[14] * L[18], QPr = Rr[14] * Rr[18];
  *HPi = 0.5 * (vl * QPl + vr * QPr) - 0.5 * cmax * (QPr - QPl);
}

/* -------------------------- ghost cells (R17) ------------------------ */
static int wrap(int i, int n, int periodic) {
  if (periodic) return ((i % n) + n) % n;
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

static void fill_ghosts_array(const orc_t* h, double* a) {
  int nx = h->c.nx, ny = h->c.ny, ne = h->c.neta, p = h->c.periodic;
  for (int i = -2; i < nx + 2; ++i)
    for (int j = -2; j < ny + 2; ++j)
      for (int k = -2; k < ne + 2; ++k) {
        if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < ne) continue;
        a[IX(h, i, j, k)] = a[IX(h, wrap(i, nx, p), wrap(j, ny, p), wrap(k, ne, p))];
      }
}

static void fill_ghosts(const orc_t* h, orc_fields* f) {
  if (h->charge) fill_ghosts_array(h, f->N);
  if (h->bulk) fill_ghosts_array(h, f->Pi);
  for (int m = 0; m < 4; ++m) fill_ghosts_array(h, f->T[m]);
  for (int q = 0; q < NPI; ++q) fill_ghosts_array(h, f->pi[q]);
  fill_ghosts_array(h, f->ed);
  for (int m = 0; m < 3; ++m) fill_ghosts_array(h, f->u[m]);
}

/* ---------------------------- one Heun stage ------------------------- */
/* Total source S_tot = S_KT + S_T (+ S_pi) at cell (i,j,k) of fields f at
 * time tau_s.  ulate: the late velocity for the time derivative (u* or u'),
 * un: velocity at step n (spatial components). */
static void stage_source(const orc_t* h, const orc_fields* f, int viscous, double tau_s, int i,
                         int j, int k, const double ulate[4], const double un[4],
                         double S[4 + NPI], double* SN, double* SPi) {
  view_t vw = {h, f, viscous};
  double taus = tau_scale(h, tau_s);
  double g = geo(h, tau_s);
  double hstep = h->c.dtau;
  for (int q = 0; q < 4 + NPI; ++q) S[q] = 0.0;
  *SN = 0.0;
  *SPi = 0.0;
  /* KT flux differences along x, y, eta_s (Eq. kt) */
  double dl[3] = {h->c.dx, h->c.dy, ((PLANT == 4) ? 1.0 : taus) * h->c.deta};
  for (int ax = 1; ax <= 3; ++ax) {
    int di = (ax == 1), dj = (ax == 2), dk = (ax == 3);
    size_t m2 = IX(h, i - 2 * di, j - 2 * dj, k - 2 * dk);
    size_t m1 = IX(h, i - di, j - dj, k - dk);
    size_t c0 = IX(h, i, j, k);
    size_t p1 = IX(h, i + di, j + dj, k + dk);
    size_t p2 = IX(h, i + 2 * di, j + 2 * dj, k + 2 * dk);
    double Hm[4 + NPI], Hp[4 + NPI], HNm, HNp, HPm, HPp;
    kt_interface(&vw, ax, taus, m2, m1, c0, p1, Hm, &HNm, &HPm);
    kt_interface(&vw, ax, taus, m1, c0, p1, p2, Hp, &HNp, &HPp);
    int nq = viscous ? 4 + NPI : 4;
    for (int q = 0; q < nq; ++q) S[q] -= (Hp[q] - Hm[q]) / dl[ax - 1];
    *SN -= (HNp - HNm) / dl[ax - 1];
    *SPi -= (HPp - HPm) / dl[ax - 1];
  }
  /* geometric source S_T (R1) */
  size_t c0 = IX(h, i, j, k);
  double u[4];
  u[1] = f->u[0][c0]; u[2] = f->u[1][c0]; u[3] = f->u[2][c0];
  u[0] = sqrt(1.0 + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
  double e = f->ed[c0], P, T, cs2;
  eos_eval(h, e, &P, &T, &cs2);
  double piee = viscous ? f->pi[9][c0] : 0.0;
  double Pb = (viscous && h->bulk) ? f->Pi[c0] : 0.0;   /* R20: the pressure of T^{mu nu} is P + Pi */
  double Pt = P + Pb;
  if (Pt < 0.0) Pt = 0.0;
  double Tee_over_tau = e * u[3] * u[3] + Pt * (1.0 + u[3] * u[3]) + piee;
  S[0] -= ((PLANT == 3) ? -1.0 : 1.0) * (h->c.cartesian ? 0.0 : 1.0) * Tee_over_tau;
  if (PLANT != 7) S[3] -= g * f->T[3][c0];
  if (!viscous) return;
  /* viscous source S_pi */
  double du[16];
  for (int b = 0; b < 4; ++b) du[0 * 4 + b] = (ulate[b] - un[b]) / hstep;
  for (int ax = 1; ax <= 3; ++ax) {
    int di = (ax == 1), dj = (ax == 2), dk = (ax == 3);
    size_t p1 = IX(h, i + di, j + dj, k + dk), m1 = IX(h, i - di, j - dj, k - dk);
    double up[4], um[4];
    up[1] = f->u[0][p1]; up[2] = f->u[1][p1]; up[3] = f->u[2][p1];
    um[1] = f->u[0][m1]; um[2] = f->u[1][m1]; um[3] = f->u[2][m1];
    up[0] = sqrt(1.0 + up[1] * up[1] + up[2] * up[2] + up[3] * up[3]);
    um[0] = sqrt(1.0 + um[1] * um[1] + um[2] * um[2] + um[3] * um[3]);
    double d = 2.0 * dl[ax - 1];
    for (int b = 0; b < 4; ++b) du[ax * 4 + b] = (up[b] - um[b]) / d;
  }
  double pi[NPI], Spi[NPI];
  for (int q = 0; q < NPI; ++q) pi[q] = f->pi[q][c0];
  source_pi(g, u, du, pi, e, P, T, h->c.eta_over_s, h->c.taupi_coef, h->c.lambda1_hat, Spi);
  for (int q = 0; q < NPI; ++q) S[4 + q] += Spi[q];
  if (h->bulk) {
    /* R20: theta~ = d~_mu u~^mu + u~^tau/tau; 1/tau_Pi = T / (5 (zeta/s) hbar c),
       zeta / tau_Pi = (eps + P)/5 */
    double theta = du[0] + du[5] + du[10] + du[15] + g * u[0];
    double inv_tauPi = T / (5.0 * h->c.zeta_over_s * HBARC);
    *SPi += -Pb * inv_tauPi - ((PLANT == 19) ? -1.0 : 1.0) * (e + P) * theta / 5.0 - Pb * theta / 3.0
            - ((PLANT == 18) ? 0.0 : 1.0) * g * u[0] * Pb;
  }
}

static void recover(orc_t* h, double tau_new, size_t c, orc_fields* out, int viscous,
                    long* nres, long* nfail) {
  double taus = tau_scale(h, tau_new);
  double pitt = viscous ? out->pi[0][c] : 0.0;
  double E = out->T[0][c] / taus - pitt;
  double Mx = out->T[1][c] / taus - (viscous ? out->pi[1][c] : 0.0);
  double My = out->T[2][c] / taus - (viscous ? out->pi[2][c] : 0.0);
  double Me = out->T[3][c] / taus - (viscous ? out->pi[3][c] : 0.0);
  double e, u[4];
  int resc;
  double Pb = (viscous && h->bulk && PLANT != 20) ? out->Pi[c] : 0.0;
  int it = prim_solve(h, E, Mx, My, Me, Pb, &e, u, &resc);
  if (it < 0) (*nfail)++;
  if (resc) (*nres)++;
  out->ed[c] = e;
  out->u[0][c] = u[1]; out->u[1][c] = u[2]; out->u[2][c] = u[3];
  if (viscous && e == 0.0) {
    for (int q = 0; q < NPI; ++q) out->pi[q][c] = 0.0;
    if (h->bulk) out->Pi[c] = 0.0;
  }
}

static void heun_step(orc_t* h, int viscous) {
  int nx = h->c.nx, ny = h->c.ny, ne = h->c.neta;
  double hs = h->c.dtau, tn = h->tau, tn1 = h->tau + hs;
  long nres = 0, nfail = 0;
  orc_fields* s = &h->s;
  orc_fields* s1 = &h->s1;
  /* ---- stage 1 ---- */
  fill_ghosts(h, s);
#pragma omp parallel for schedule(static) reduction(+ : nres, nfail)
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < ne; ++k) {
        size_t c = IX(h, i, j, k);
        double un[4], us[4];
        un[1] = s->u[0][c]; un[2] = s->u[1][c]; un[3] = s->u[2][c];
        un[0] = sqrt(1.0 + un[1] * un[1] + un[2] * un[2] + un[3] * un[3]);
        for (int b = 1; b < 4; ++b) us[b] = viscous ? 2.0 * un[b] - h->up[b - 1][c] : un[b];
        us[0] = sqrt(1.0 + us[1] * us[1] + us[2] * us[2] + us[3] * us[3]);
        double S[4 + NPI], SN, SPi;
        stage_source(h, s, viscous, tn, i, j, k, us, un, S, &SN, &SPi);
        for (int m = 0; m < 4; ++m) s1->T[m][c] = s->T[m][c] + hs * S[m];
        if (h->charge) s1->N[c] = s->N[c] + hs * SN;
        if (viscous) {
          double pv[NPI];
          for (int q = 0; q < NPI; ++q) pv[q] = (un[0] * s->pi[q][c] + hs * S[4 + q]) / us[0];
          regulate_pi(h, s->ed[c], pv);
          for (int q = 0; q < NPI; ++q) s1->pi[q][c] = pv[q];
          if (h->bulk) s1->Pi[c] = regulate_Pi(h, s->ed[c], (un[0] * s->Pi[c] + hs * SPi) / us[0]);
        }
        recover(h, tn1, c, s1, viscous, &nres, &nfail);
      }
  /* ---- stage 2 ---- */
  fill_ghosts(h, s1);
#pragma omp parallel for schedule(static) reduction(+ : nres, nfail)
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < ne; ++k) {
        size_t c = IX(h, i, j, k);
        double un[4], us[4], u1[4];
        un[1] = s->u[0][c]; un[2] = s->u[1][c]; un[3] = s->u[2][c];
        un[0] = sqrt(1.0 + un[1] * un[1] + un[2] * un[2] + un[3] * un[3]);
        for (int b = 1; b < 4; ++b) us[b] = viscous ? 2.0 * un[b] - h->up[b - 1][c] : un[b];
        us[0] = sqrt(1.0 + us[1] * us[1] + us[2] * us[2] + us[3] * us[3]);
        u1[1] = s1->u[0][c]; u1[2] = s1->u[1][c]; u1[3] = s1->u[2][c];
        u1[0] = sqrt(1.0 + u1[1] * u1[1] + u1[2] * u1[2] + u1[3] * u1[3]);
        double S[4 + NPI], SN, SPi;
        stage_source(h, s1, viscous, tn1, i, j, k, u1, un, S, &SN, &SPi);
        for (int m = 0; m < 4; ++m) s->T[m][c] = 0.5 * (s->T[m][c] + s1->T[m][c] + hs * S[m]);
        if (h->charge) s->N[c] = 0.5 * (s->N[c] + s1->N[c] + hs * SN);
        if (viscous) {
          double pv[NPI];
          for (int q = 0; q < NPI; ++q)
            pv[q] = 0.5 * (un[0] * s->pi[q][c] + us[0] * s1->pi[q][c] + hs * S[4 + q]) / u1[0];
          regulate_pi(h, s1->ed[c], pv);
          for (int q = 0; q < NPI; ++q) s->pi[q][c] = pv[q];
          if (h->bulk)
            s->Pi[c] = regulate_Pi(h, s1->ed[c], 0.5 * (un[0] * s->Pi[c] + us[0] * s1->Pi[c] + hs * SPi) / u1[0]);
        }
        /* keep u^n as u^{n-1} for the next step */
        if (PLANT != 23) { h->up[0][c] = un[1]; h->up[1][c] = un[2]; h->up[2][c] = un[3]; }
        recover(h, tn1, c, s, viscous, &nres, &nfail);
      }
  h->tau = tn1;
  h->step += 1;
  h->n_rescaled += nres;
  h->n_rootfail += nfail;
}

static void compute_stats(orc_t* h) {
  double emax = 0.0, Tmax = 0.0, Etot = 0.0;
  for (int i = 0; i < h->c.nx; ++i)
    for (int j = 0; j < h->c.ny; ++j)
      for (int k = 0; k < h->c.neta; ++k) {
        size_t c = IX(h, i, j, k);
        double e = h->s.ed[c], P, T, cs2;
        if (e > emax) emax = e;
        eos_eval(h, e, &P, &T, &cs2);
        if (T > Tmax) Tmax = T;
        Etot += h->s.T[0][c];
      }
  h->stats[0] = h->tau;
  h->stats[1] = (double)h->step;
  h->stats[2] = emax;
  h->stats[3] = Tmax;
  h->stats[4] = Etot * h->c.dx * h->c.dy * h->c.deta;
  h->stats[5] = (double)h->n_rescaled;
  h->stats[6] = (double)h->n_rootfail;
  h->stats[7] = 0.0;
}

/* ============================ public API ============================= */
static double* zalloc(size_t n) { return (double*)calloc(n, sizeof(double)); }

static void fields_alloc(orc_fields* f, size_t n) {
  for (int m = 0; m < 4; ++m) f->T[m] = zalloc(n);
  for (int q = 0; q < NPI; ++q) f->pi[q] = zalloc(n);
  f->ed = zalloc(n);
  for (int m = 0; m < 3; ++m) f->u[m] = zalloc(n);
  f->N = zalloc(n);
  f->Pi = zalloc(n);
}
static void fields_free(orc_fields* f) {
  for (int m = 0; m < 4; ++m) free(f->T[m]);
  for (int q = 0; q < NPI; ++q) free(f->pi[q]);
  free(f->ed);
  for (int m = 0; m < 3; ++m) free(f->u[m]);
  free(f->N);
  free(f->Pi);
}
static void fields_copy(orc_fields* d, const orc_fields* s, size_t n) {
  for (int m = 0; m < 4; ++m) memcpy(d->T[m], s->T[m], n * sizeof(double));
  for (int q = 0; q < NPI; ++q) memcpy(d->pi[q], s->pi[q], n * sizeof(double));
  memcpy(d->ed, s->ed, n * sizeof(double));
  for (int m = 0; m < 3; ++m) memcpy(d->u[m], s->u[m], n * sizeof(double));
  memcpy(d->N, s->N, n * sizeof(double));
  memcpy(d->Pi, s->Pi, n * sizeof(double));
}

orc_t* orc_create(const orc_config* c) {
  if (!c || c->nx < 1 || c->ny < 1 || c->neta < 1) return NULL;
  if (!(c->dx > 0 && c->dy > 0 && c->deta > 0 && c->dtau > 0)) return NULL;
  if (!c->cartesian && !(c->tau0 > 0)) return NULL;
  if (!(c->zeta_over_s >= 0.0) || (c->zeta_over_s > 0.0 && !(c->eta_over_s > 0.0))) return NULL; /* R20 */
  if (c->eos_kind == 1 && (c->eos_n < 2 || !c->eos_P || !c->eos_T || !c->eos_cs2)) return NULL;
  orc_t* h = (orc_t*)calloc(1, sizeof(orc_t));
  h->c = *c;
  if (c->eos_kind == 1) {
    h->eosP = zalloc(c->eos_n); h->eosT = zalloc(c->eos_n); h->eosC = zalloc(c->eos_n);
    memcpy(h->eosP, c->eos_P, c->eos_n * sizeof(double));
    memcpy(h->eosT, c->eos_T, c->eos_n * sizeof(double));
    memcpy(h->eosC, c->eos_cs2, c->eos_n * sizeof(double));
  }
  h->c.eos_P = h->c.eos_T = h->c.eos_cs2 = NULL;
  h->NX = c->nx + 4; h->NY = c->ny + 4; h->NE = c->neta + 4;
  h->NG = (size_t)h->NX * h->NY * h->NE;
  fields_alloc(&h->s, h->NG);
  fields_alloc(&h->s1, h->NG);
  for (int m = 0; m < 3; ++m) h->up[m] = zalloc(h->NG);
  h->tau = c->tau0;
  h->viscous = c->eta_over_s > 0.0;
  h->bulk = h->viscous && c->zeta_over_s > 0.0;
#ifdef _OPENMP
  if (c->nthreads > 0) omp_set_num_threads(c->nthreads);
#endif
  return h;
}

void orc_destroy(orc_t* h) {
  if (!h) return;
  fields_free(&h->s); fields_free(&h->s1);
  for (int m = 0; m < 3; ++m) free(h->up[m]);
  free(h->eosP); free(h->eosT); free(h->eosC);
  free(h);
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Load the state from primitives (eps, u~^x, u~^y, u~^eta, optional pi~ as
 * 10 consecutive blocks of N).  Arrays are (nx, ny, neta), eta fastest. */
int orc_set_initial(orc_t* h, const double* eps, const double* ux, const double* uy,
                    const double* ue, const double* pi) {
  int nx = h->c.nx, ny = h->c.ny, ne = h->c.neta;
  size_t N = (size_t)nx * ny * ne;
  double taus = tau_scale(h, h->c.tau0);
  h->tau = h->c.tau0;
  h->step = 0;
  h->n_rescaled = h->n_rootfail = 0;
  h->charge = 0;
  memset(h->s.N, 0, h->NG * sizeof(double));
  memset(h->s1.N, 0, h->NG * sizeof(double));
  memset(h->s.Pi, 0, h->NG * sizeof(double));   /* Pi = 0 at tau0 (R20) */
  memset(h->s1.Pi, 0, h->NG * sizeof(double));
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < ne; ++k) {
        size_t l = ((size_t)i * ny + j) * ne + k, c = IX(h, i, j, k);
        double e = eps[l];
        double u[4] = {0, ux[l], uy[l], ue[l]};
        double pv[NPI];
        for (int q = 0; q < NPI; ++q) pv[q] = (pi && h->viscous) ? pi[q * N + l] : 0.0;
        if (!(e >= h->c.eps_cut)) {
          e = 0.0;
          u[1] = u[2] = u[3] = 0.0;
          for (int q = 0; q < NPI; ++q) pv[q] = 0.0;
        }
        u[0] = sqrt(1.0 + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
        double P, T, cs2, Tt[4];
        eos_eval(h, e, &P, &T, &cs2);
        T_from_prim(taus, e, P, u, pv, Tt);
        for (int m = 0; m < 4; ++m) h->s.T[m][c] = Tt[m];
        for (int q = 0; q < NPI; ++q) h->s.pi[q][c] = pv[q];
        h->s.ed[c] = e;
        h->s.u[0][c] = u[1]; h->s.u[1][c] = u[2]; h->s.u[2][c] = u[3];
        h->up[0][c] = u[1]; h->up[1][c] = u[2]; h->up[2][c] = u[3];
      }
  if (h->viscous && PLANT != 22) {
    /* R8: one pi-free Heun step gives u^1_ideal; u^{-1} = 2 u^0 - u^1_ideal */
    orc_fields save;
    fields_alloc(&save, h->NG);
    fields_copy(&save, &h->s, h->NG);
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j)
        for (int k = 0; k < ne; ++k) {
          size_t c = IX(h, i, j, k);
          double e = h->s.ed[c], P, T, cs2, Tt[4];
          double u[4] = {0, h->s.u[0][c], h->s.u[1][c], h->s.u[2][c]};
          u[0] = sqrt(1.0 + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
          eos_eval(h, e, &P, &T, &cs2);
          T_from_prim(taus, e, P, u, NULL, Tt);
          for (int m = 0; m < 4; ++m) h->s.T[m][c] = Tt[m];
        }
    heun_step(h, 0);
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j)
        for (int k = 0; k < ne; ++k) {
          size_t c = IX(h, i, j, k);
          for (int m = 0; m < 3; ++m) h->up[m][c] = 2.0 * save.u[m][c] - h->s.u[m][c];
        }
    fields_copy(&h->s, &save, h->NG);
    fields_free(&save);
    h->tau = h->c.tau0;
    h->step = 0;
    h->n_rescaled = h->n_rootfail = 0;
  }
  compute_stats(h);
  return 0;
}

/* Initial state from T^{tau mu} with pi = 0 (the mini-jet initial flow of
 * the large-event workload).  T holds 4 x N values T^{tau tau}, T^{tau x},
 * T^{tau y} and the orthonormal tau T^{tau eta} (all GeV/fm^3).  With pi = 0
 * these are T_ideal^{tau mu}, and the primitives are the root of the
 * recovery problem of Sec. 3 (E = T^{tau tau}, M = T^{tau i}); the state then
 * follows from (eps, u~) as in orc_set_initial.  Returns -1 if a root solve
 * hit its cap. */
int orc_set_initial_T(orc_t* h, const double* T) {
  size_t N = (size_t)h->c.nx * h->c.ny * h->c.neta;
  double* a = (double*)malloc(4 * N * sizeof(double));
  if (!a) return -1;
  int fail = 0;
  for (size_t l = 0; l < N; ++l) {
    double e, u[4];
    int resc;
    const double Mx = T[((PLANT == 30) ? 2 : 1) * N + l], My = T[((PLANT == 30) ? 1 : 2) * N + l];
    if (prim_solve(h, T[l], Mx, My, T[3 * N + l], 0.0, &e, u, &resc) < 0) fail = 1;
    a[l] = e;
    a[N + l] = u[1];
    a[2 * N + l] = u[2];
    a[3 * N + l] = u[3];
  }
  int r = fail ? -1 : orc_set_initial(h, a, a + N, a + 2 * N, a + 3 * N, NULL);
  free(a);
  return r;
}

/* Net charge density n at tau0 (R19), after orc_set_initial: N~^tau =
 * tau0 n u~^tau from the initial velocities. */
int orc_set_initial_n(orc_t* h, const double* n) {
  int nx = h->c.nx, ny = h->c.ny, ne = h->c.neta;
  double taus = tau_scale(h, h->tau);
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < ne; ++k) {
        size_t l = ((size_t)i * ny + j) * ne + k, c = IX(h, i, j, k);
        double ux = h->s.u[0][c], uy = h->s.u[1][c], ue = h->s.u[2][c];
        double ut = sqrt(1.0 + ux * ux + uy * uy + ue * ue);
        h->s.N[c] = ((PLANT == 17) ? 1.0 : taus) * n[l] * ut;
      }
  h->charge = 1;
  return 0;
}

int orc_step(orc_t* h, int n) {
  for (int s = 0; s < n; ++s) heun_step(h, h->viscous);
  compute_stats(h);
  return h->n_rootfail ? 4 : 0;
}

/* which: 0 eps, 1..3 u~^x,y,eta, 4..7 T~^{tau mu}, 8..17 pi~, 18..20 u~^{n-1},
 * 21 N~^tau, 22 n, 23 Pi */
int orc_get(const orc_t* h, int which, double* out) {
  int nx = h->c.nx, ny = h->c.ny, ne = h->c.neta;
  const double* a;
  if (which == 0) a = h->s.ed;
  else if (which <= 3) a = h->s.u[which - 1];
  else if (which <= 7) a = h->s.T[which - 4];
  else if (which <= 17) a = h->s.pi[which - 8];
  else if (which <= 20) a = h->up[which - 18];
  else if (which == 21) a = h->s.N;
  else if (which == 23) a = h->s.Pi;
  else if (which == 22) {
    /* n = N~^tau / (tau u^tau) (R19) */
    double taus = tau_scale(h, h->tau);
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j)
        for (int k = 0; k < ne; ++k) {
          size_t c = IX(h, i, j, k);
          double ux = h->s.u[0][c], uy = h->s.u[1][c], ue = h->s.u[2][c];
          out[((size_t)i * ny + j) * ne + k] = h->s.N[c] / (taus * sqrt(1.0 + ux * ux + uy * uy + ue * ue));
        }
    return 0;
  }
  else return 1;
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < ne; ++k) out[((size_t)i * ny + j) * ne + k] = a[IX(h, i, j, k)];
  return 0;
}

void orc_stats(const orc_t* h, double out[8]) { memcpy(out, h->stats, sizeof(h->stats)); }

/* ---- per-cell entry points used by the unit pins ---- */
void orc_eos(const orc_t* h, double e, double out[3]) { eos_eval(h, e, &out[0], &out[1], &out[2]); }

int orc_prim(const orc_t* h, double E, double Mx, double My, double Me, double out[6]) {
  double e, u[4];
  int resc;
  int it = prim_solve(h, E, Mx, My, Me, 0.0, &e, u, &resc);
  out[0] = e; out[1] = u[0]; out[2] = u[1]; out[3] = u[2]; out[4] = u[3]; out[5] = it;
  return it;
}

/* The root solve with a bulk pressure Pi added to P (total floored at 0, R20). */
int orc_prim_bulk(const orc_t* h, double E, double Mx, double My, double Me, double Pi, double out[6]) {
  double e, u[4];
  int resc;
  int it = prim_solve(h, E, Mx, My, Me, Pi, &e, u, &resc);
  out[0] = e; out[1] = u[0]; out[2] = u[1]; out[3] = u[2]; out[4] = u[3]; out[5] = it;
  return it;
}

/* S_pi at one cell with the tilde-derivative matrix du[a*4+b] = d~_a u~^b given. */
void orc_source_pi(const orc_t* h, double tau, const double u[4], const double du[16],
                   const double pi[NPI], double e, double out[NPI]) {
  double P, T, cs2;
  eos_eval(h, e, &P, &T, &cs2);
  source_pi(geo(h, tau), u, du, pi, e, P, T, h->c.eta_over_s, h->c.taupi_coef, h->c.lambda1_hat, out);
}

/* Geometric source S_T at one cell: needs eps, u~, pi~^{eta eta} and T~^{tau eta}. */
void orc_source_T(const orc_t* h, double tau, const double u[4], double e, double piee,
                  double Tte, double out[4]) {
  double P, T, cs2;
  eos_eval(h, e, &P, &T, &cs2);
  out[0] = -(h->c.cartesian ? 0.0 : 1.0) * (e * u[3] * u[3] + P * (1.0 + u[3] * u[3]) + piee);
  out[1] = 0.0;
  out[2] = 0.0;
  out[3] = -geo(h, tau) * Tte;
}
