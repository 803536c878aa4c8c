// clv_kernels.cuh -- kernels of one Heun step of (3+1)D viscous hydro in
// Milne coordinates (CLVisc method).  Storage is structure-of-arrays, one
// array per field of nx*ny*neta values, eta_s fastest.
#pragma once
#include "clv_device.cuh"
#include "clv_mlp.cuh"

namespace clv {

constexpr int kBlock = 256;

template <typename R> struct Ptr10 {
  R* p[10];
};

// Primitive set: eps, u~^x, u~^y, u~^eta, P(eps), c_s(eps).
template <typename R> struct Prim {
  R* e;
  R* u[3];
  R* P;
  R* cs;
};

// Israel-Stewart coefficients: tau_pi = b eta_v / (eps + P) = b (eta/s) hbar c
// / T (b = 5 by default), and lambda_1 = lambda1_hat / eps (0: no term).
template <typename R> struct IsCoef {
  R inv_b_etas_hbarc;   // 1/(b (eta/s) hbar c): 1/tau_pi = T * this
  R inv_b;              // 1/b: eta_v / tau_pi = (eps + P) / b
  R lambda1_hat;
};

// T~^{tau mu} keeps ~48 significant bits on the FP32 path: a float-float pair
// T~ = T + Tl (high parts T, low parts Tl, both float arrays).  It is the
// conserved energy-momentum that every stage accumulates into; in the dilute,
// fast-moving edge of an event the rest-frame density eps = E - M v is a
// small difference of its components (E/eps ~ gamma^2), so plain FP32
// storage of T~ turned its rounding into percent-level errors of eps there
// after a few hundred steps.  The stencil reads the high parts (fluxes and
// sources stay FP32); the update adds the FP32 increment to the pair exactly,
// and the recovery forms E and M from the pair.  The FP64 path stores T~ in
// T and leaves Tl unused.
template <typename R> struct StageParams {
  // fields of the stage being differentiated (stage 1: step n, stage 2: stage-1 result)
  const R* T[4];
  const R* Tl[4];
  const R* pi[10];
  Prim<R> pr;
  // own-cell inputs: T~ and pi~ at step n, u~ at n and n-1
  const R* Tn[4];
  const R* Tnl[4];
  const R* pin[10];
  const R* un[3];
  const R* up[3];
  // outputs (stage 2 writes T and pi in place over Tn/pin, prim over the n-1 set)
  R* Tout[4];
  R* Toutl[4];
  R* piout[10];
  Prim<R> prout;
  EosView<R> eos;
  int nx, ny, ne, periodic;
  int nep;     // eta pitch of the layout (ne rounded up to a multiple of 4)
  int xhalo;   // 1: x planes -2, -1, nx, nx + 1 are stored halo planes (an x-slab); no clamping in x
  long long N;
  // tau of the step lives on the device (advanced by a kernel after every
  // step), so the launches of a step do not depend on it and a captured step
  // replays unchanged; tau_scalars() forms the stage's tau factors from it
  const double* tau_dev;
  const float* itau;   // FP32 path: 1/tau at the end of the step (Cartesian: 1) as a float-float pair
  double dtau_d;
  int cartesian;
  // scalars in the working precision
  R h, inv_h;  // time step and its inverse
  R inv_dl[2]; // 1/dx, 1/dy
  R st_tau;    // 1 in Milne (S_T^tau active), 0 in Cartesian
  R eps_cut;
  IsCoef<R> is;       // Israel-Stewart coefficients (tau_pi, lambda_1)
  R polish_E, polish_v;   // FP32: FP64 Newton where the FP32 eps < polish_E or M > polish_v E
  double eps_cut_d;
  double deta_d;   // d eta_s in FP64 (1/(tau deta) is formed in the kernels, per event in a batch)
  // reductions and error reporting
  double* block_sum;             // per block: sum of new T~^{tau tau} (stats launches only)
  unsigned long long* emax_bits; // max eps as the bits of a non-negative double
  unsigned long long* counters;  // [0] rescaled, [1] root cap, [2] polished, [3] FP32 not converged
  unsigned int* err;             // error word
  unsigned long long* fail_cell; // first failing cell + 1 (0: none)
  double* fail_EM;               // E and |M| of that cell
  const void* mlp;               // tensor-core copy of the guess network (BF16 W1|W2|W3, FP32 biases)
  // bulk pressure Pi of the stage's output (written before the stage by the
  // bulk kernel; the recovery solves with P + Pi, stores P + Pi as the cell's
  // pressure and sets Pi = 0 in vacuum cells); nullptr without bulk
  R* Pib;
};

// kGuessMlp: the network seeds the cells that were vacuum in the stage's
// input (no velocity to start from), the stage velocity every other cell;
// kGuessMlpAll: the network seeds every cell.
enum GuessMode { kGuessPrevious = 0, kGuessCold = 1, kGuessMlp = 2, kGuessMlpAll = 3 };

__device__ __forceinline__ int wrap_index(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

template <typename R> __device__ __forceinline__ R ldg(const R* p) { return __ldg(p); }

template <typename R> struct SolveTraits;
template <> struct SolveTraits<float> {
  static constexpr float tol = 5e-7f;
  static constexpr int maxit = 40;
};
template <> struct SolveTraits<double> {
  static constexpr double tol = 1e-15;
  static constexpr int maxit = 100;
};

// Reconstructed interface quantities (KT, Eq. flux_out): T~^{tau mu} (4),
// pi~ (10), u~^tau, v^a = u~^a/u~^tau, P.
// The tau factors of a stage, rounded to R exactly as a host computation in
// FP64 would be: tau_s = tau at the stage (stage 1: tau_n, stage 2:
// tau_n + dtau), or 1 in Cartesian coordinates.
template <typename R> struct TauS {
  double taus_d;   // tau_s in FP64
  R taus;          // tau_s
  R geo;           // 1/tau_s (Milne) or 0 (Cartesian)
  R taus_new;      // tau scale at the end of the step (primitive recovery)
};
template <typename R>
__device__ __forceinline__ TauS<R> tau_scalars(const StageParams<R>& p, int stage) {
  const double tn = *p.tau_dev;
  const double tn1 = tn + p.dtau_d;
  const double tst = stage == 1 ? tn : tn1;
  TauS<R> t;
  t.taus_d = p.cartesian ? 1.0 : tst;
  t.taus = (R)t.taus_d;
  t.geo = (R)(p.cartesian ? 0.0 : 1.0 / tst);
  t.taus_new = (R)(p.cartesian ? 1.0 : tn1);
  return t;
}

template <bool VISC> struct NRec { static constexpr int n = VISC ? 17 : 7; };

template <typename R, bool VISC>
__device__ __forceinline__ void interface_flux(const R* L, const R* Rr, R csl, R csr, int axis,
                                               R taus, R* H) {
  constexpr int NQ = VISC ? 14 : 4;
  constexpr int IU = VISC ? 14 : 4, IV = IU + 1, IP = IU + 2;
  const R vl = L[IV], vr = Rr[IV];
  const R al = fabs(vl), ar = fabs(vr);
  const R lam = fmax((al + csl) / (R(1) + al * csl), (ar + csr) / (R(1) + ar * csr));
  // H = (F_l + F_r)/2 - lam (Q_r - Q_l)/2 with F = v Q + tau X regrouped as
  // wl Q_l + wr Q_r + tau (X_l + X_r)/2, wl = (v_l + lam)/2, wr = (v_r - lam)/2
  const R wl = R(0.5) * (vl + lam), wr = R(0.5) * (vr - lam);
  const R ht = R(0.5) * taus;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    // X of T~^{tau m} along a: P (v d_{m tau} + d_{m a}) + pi~^{a m} - v pi~^{tau m}
    R gl = (m == 0 ? vl : R(0)) + (m == axis ? R(1) : R(0));
    R gr = (m == 0 ? vr : R(0)) + (m == axis ? R(1) : R(0));
    R xl = L[IP] * gl, xr = Rr[IP] * gr;
    if constexpr (VISC) {
      xl += L[4 + sym_index(axis, m)] - vl * L[4 + sym_index(0, m)];
      xr += Rr[4 + sym_index(axis, m)] - vr * Rr[4 + sym_index(0, m)];
    }
    H[m] = wl * L[m] + wr * Rr[m] + ht * (xl + xr);
  }
  if constexpr (VISC) {
    // Q_pi = u~^tau pi~ on each side, flux v Q_pi
    const R al2 = wl * L[IU], ar2 = wr * Rr[IU];
#pragma unroll
    for (int q = 0; q < 10; ++q) H[4 + q] = al2 * L[4 + q] + ar2 * Rr[4 + q];
  }
  (void)NQ;
}

// Shear regulator (the paper is silent; without a bound the dilute,
// ultra-relativistic edge of a viscous event runs away).  With eps and P of
// the stage's input state of the cell: pi~ is scaled by the ramp
// r(eps) = clamp(eps/kViscEpsMin - 1, 0, 1) (zero below kViscEpsMin, ideal
// flow far below freeze-out densities; continuous, so that rounding-level
// changes of eps change pi~ at the rounding level), then so that
// |pi_{mu nu} pi^{mu nu}| <= kRhoMax^2 (eps^2 + 3 P^2).
constexpr double kRhoMax = 1.0;
constexpr double kViscEpsMin = 1e-3;   // GeV/fm^3
template <typename R> __device__ __forceinline__ R visc_ramp(R e) {
  return fmin(fmax(e * R(1.0 / kViscEpsMin) - R(1), R(0)), R(1));
}
// FP64 refinement of the FP32 root solve (E - M v, the Newton step and gamma
// in FP64 around the FP32 table lookup).  A converged FP32 root starts
// kPolishSteps FP64 Newton steps (it lies in the quadratic basin; the FP32
// interpolation of P sets the noise floor beyond which more steps gain
// nothing); an unconverged one gets a full bracketed FP64 solve.  Returns the
// iterations taken, -1 if the full solve hit its cap.
constexpr int kPolishSteps = 2;
// Below this fraction of eps_cut an FP32 eps is vacuum for certain (no refinement).
constexpr double kVacuumSure = 0.999;
// E and M come in FP64 (formed from the FP64 T~), so the refined root sees
// no FP32 rounding of its inputs.
template <typename R>
__device__ __forceinline__ int polish_root(const StageParams<R>& p, double E, double Mx, double My, double Me, R v32,
                                           bool converged, R& en, R& ux, R& uy, R& ue, R Pb) {
  double dv = converged ? (double)v32 : -1.0, de, dux, duy, due;
  RootResult r2;
  if (converged)
    r2 = solve_primitive<double, R, float, true>(p.eos, p.eps_cut_d, E, Mx, My, Me, 1e-13, kPolishSteps, de, dux, duy,
                                                 due, &dv, nullptr, (double)Pb);
  else
    r2 = solve_primitive<double, R, float>(p.eos, p.eps_cut_d, E, Mx, My, Me, 1e-13, 100, de, dux, duy, due, &dv,
                                           nullptr, (double)Pb);
  en = R(de); ux = R(dux); uy = R(duy); ue = R(due);
  return r2.iters;
}

// Ideal part of the stage's T~ for the root solve (Sec. 3): E = T~^{tau tau}/tau
// - pi~^{tau tau}, M^i = T~^{tau i}/tau - pi~^{tau i}.  FP32 path: from the
// float-floats T~ and 1/tau as float-float pairs (E, M unrounded for the
// correction step, their high parts for the FP32 solve); FP64 path: in R.
template <typename R, bool VISC> struct IdealPart {
  ff E, M[3];     // FP32 path
  R e, m[3];      // rounded to R (the FP64 path's values)
};
template <typename R, bool VISC>
__device__ __forceinline__ IdealPart<R, VISC> ideal_part(const StageParams<R>& p, const R Tv[4], const R Tlv[4],
                                                        const R pi4[4], R tn) {
  IdealPart<R, VISC> a;
  if constexpr (sizeof(R) == 4) {
    const ff itn{p.itau[0], p.itau[1]};
    a.E = ff_mul(ff{Tv[0], Tlv[0]}, itn);
    if constexpr (VISC) a.E = ff_add(a.E, -pi4[0]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a.M[i] = ff_mul(ff{Tv[1 + i], Tlv[1 + i]}, itn);
      if constexpr (VISC) a.M[i] = ff_add(a.M[i], -pi4[1 + i]);
    }
    a.e = a.E.hi;
#pragma unroll
    for (int i = 0; i < 3; ++i) a.m[i] = a.M[i].hi;
  } else {
    const R itn = R(1) / tn;
    a.e = Tv[0] * itn;
#pragma unroll
    for (int i = 0; i < 3; ++i) a.m[i] = Tv[1 + i] * itn;
    if constexpr (VISC) {
      a.e -= pi4[0];
#pragma unroll
      for (int i = 0; i < 3; ++i) a.m[i] -= pi4[1 + i];
    }
  }
  return a;
}

// One Newton step of the root solve from a converged FP32 root in
// float-float arithmetic (FP32 path; cells below the FP64 refinement's
// velocity threshold, so M < (1 - kMaxMoverE) E and no rescaling applies).
// In the FP32 solve E, M and the residual v (E + P) - M carry FP32 rounding,
// which leaves eps = E - M v with a relative error of ~1e-7 E/eps (E/eps
// grows as gamma^2).  Here E and M come unrounded from the float-float T~,
// eps = E - M v and the residual are formed in float-float around the FP32
// table lookup, and only the correction itself is divided in FP32.  Returns
// false (outputs untouched) if the corrected eps falls below the cut, which
// the refinement window near the cut would have caught first.
__device__ __forceinline__ bool correct_root(const EosView<float>& eos, const ff& E, const ff Mc[3], float v32,
                                             float Pb, float eps_cut, float& en, float& ux, float& uy, float& ue,
                                             EosAtRoot<float>& at) {
  const ff M2 = ff_add(ff_add(ff_mul(Mc[0], Mc[0]), ff_mul(Mc[1], Mc[1])), ff_mul(Mc[2], Mc[2]));
  const ff M = ff_sqrt(M2);
  const ff e0 = ff_add(E, ff_neg(ff_mul(M, v32)));
  float P, T, cs2;
  eos_eval<float, float>(eos, e0.hi, P, T, cs2);
  float dPde = cs2;
  P += Pb;
  if (P < 0.f) { P = 0.f; dPde = 0.f; }
  const ff den = ff_add(E, P);
  const ff g = ff_add(ff_mul(den, v32), ff_neg(M));
  const float dv = -(den.hi * g.hi) / (den.hi * den.hi - dPde * M2.hi);
  const ff v = ff_fast_two_sum(v32, dv);
  const ff e = ff_add(E, ff_neg(ff_mul(M, v)));
  const float ef = __fadd_rn(e.hi, e.lo);
  if (!(ef >= eps_cut)) return false;
  const ff w = ff_add(ff_neg(ff_mul(v, v)), 1.f);   // 1 - v^2
  const float s = v.hi / (sqrtf(__fadd_rn(w.hi, w.lo)) * M.hi);   // gamma v / M
  en = ef;
  ux = s * Mc[0].hi;
  uy = s * Mc[1].hi;
  ue = s * Mc[2].hi;
  at.valid = true;
  at.P = P + dPde * ff_add(e, ff_neg(e0)).hi;
  at.cs2 = cs2;
  return true;
}

template <typename R>
__device__ __forceinline__ void regulate_shear(R e, R P, R* pi) {
  const R r = visc_ramp(e);
#pragma unroll
  for (int q = 0; q < 10; ++q) pi[q] *= r;
  if (r == R(0)) return;
  const R pp = pi[0] * pi[0] - R(2) * (pi[1] * pi[1] + pi[2] * pi[2] + pi[3] * pi[3]) + pi[4] * pi[4] +
               pi[7] * pi[7] + pi[9] * pi[9] + R(2) * (pi[5] * pi[5] + pi[6] * pi[6] + pi[8] * pi[8]);
  const R bound2 = R(kRhoMax * kRhoMax) * (e * e + R(3) * P * P);
  const R a = fabs(pp);
  if (a > bound2) {
    const R f = bound2 > R(0) ? sqrt(bound2 / a) : R(0);
#pragma unroll
    for (int q = 0; q < 10; ++q) pi[q] *= f;
  }
}

// Israel-Stewart source (Sec. 2, Eq. pimn with lambda_2 = lambda_3 = 0):
// du[a][b] = d~_a u~^b.
template <typename R>
__device__ __forceinline__ void shear_source(R geo, const R u[4], R du[4][4], const R pi[10], R e,
                                             R P, R inv_taupi, const IsCoef<R>& is, R* S) {
  // corrected tilde covariant derivatives (Eq. dtuz)
  du[3][0] += geo * u[3];
  du[3][3] += geo * u[0];
  const R theta = du[0][0] + du[1][1] + du[2][2] + du[3][3];
  R Du[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) Du[b] = u[0] * du[0][b] + u[1] * du[1][b] + u[2] * du[2][b] + u[3] * du[3][b];
  // w^m = g~_{bb} pi~^{m b} Du^b
  R w[4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
    w[m] = pi[sym_index(m, 0)] * Du[0] - pi[sym_index(m, 1)] * Du[1] - pi[sym_index(m, 2)] * Du[2] -
           pi[sym_index(m, 3)] * Du[3];
  const R ep5 = (e + P) * is.inv_b;
  const R decay = inv_taupi + theta * R(1.0 / 3.0) + geo * u[0];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int n = m; n < 4; ++n) {
      const int q = sym_index(m, n);
      const R sm = R(metric_sign(m)), sn = R(metric_sign(n));
      R sigma = sm * du[m][n] + sn * du[n][m] - u[m] * Du[n] - u[n] * Du[m] -
                R(2.0 / 3.0) * ((m == n ? sm : R(0)) - u[m] * u[n]) * theta;
      S[q] = ep5 * sigma - decay * pi[q] - (u[m] * w[n] + u[n] * w[m]);
    }
  // -(lambda_1 / tau_pi) pi^<mu_l pi^nu>l in tilde components: Y = pi g~ pi,
  // X = Delta^m_a Delta^n_c Y^ac - Delta^mn (Delta_ac Y^ac) / 3
  if (is.lambda1_hat != R(0) && e > R(0)) {
    R Y[10];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = a; c < 4; ++c)
        Y[sym_index(a, c)] = pi[sym_index(a, 0)] * pi[sym_index(0, c)] - pi[sym_index(a, 1)] * pi[sym_index(1, c)] -
                             pi[sym_index(a, 2)] * pi[sym_index(2, c)] - pi[sym_index(a, 3)] * pi[sym_index(3, c)];
    const R ul[4] = {u[0], -u[1], -u[2], -u[3]};   // u~_a
    // Z^m_c = Delta^m_a Y^ac = Y^mc - u^m (u_a Y^ac)
    R uY[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      uY[c] = ul[0] * Y[sym_index(0, c)] + ul[1] * Y[sym_index(1, c)] + ul[2] * Y[sym_index(2, c)] +
              ul[3] * Y[sym_index(3, c)];
    const R uYu = ul[0] * uY[0] + ul[1] * uY[1] + ul[2] * uY[2] + ul[3] * uY[3];
    // Delta_ac Y^ac = g~_ac Y^ac - u_a Y^ac u_c
    const R tr = Y[0] - Y[4] - Y[7] - Y[9] - uYu;
    const R f = -is.lambda1_hat / e * inv_taupi;
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int n = m; n < 4; ++n) {
        // Delta^m_a Delta^n_c Y^ac = Y^mn - u^m uY^n - u^n uY^m + u^m u^n uYu
        const R x = Y[sym_index(m, n)] - u[m] * uY[n] - u[n] * uY[m] + u[m] * u[n] * uYu -
                    ((m == n ? R(metric_sign(m)) : R(0)) - u[m] * u[n]) * tr * R(1.0 / 3.0);
        S[sym_index(m, n)] += f * x;
      }
  }
  // Christoffel terms I^{mu nu} (Eq. Ipi), with a minus sign in S_pi
  const R gu = geo * u[3];
  S[0] -= R(2) * gu * pi[3];
  S[1] -= gu * pi[6];
  S[2] -= gu * pi[8];
  S[3] -= gu * (pi[0] + pi[9]);
  S[6] -= gu * pi[1];
  S[8] -= gu * pi[2];
  S[9] -= R(2) * gu * pi[3];
}

template <typename R, int STAGE, bool VISC, bool STATS>
__global__ void __launch_bounds__(kBlock) stage_kernel(const StageParams<R> p) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = c < p.N && (int)(c % p.nep) < p.ne;   // padding slots of the eta rows do no work
  double my_T0 = 0.0;
  double my_e = 0.0;
  bool f_rescaled = false, f_fail = false, f_polished = false, f_nonfinite = false, f_nonconv = false;
  if (active) {
    const int k = (int)(c % p.nep);
    const long long t = c / p.nep;
    const int j = (int)(t % p.ny);
    const int i = (int)(t / p.ny);
    constexpr int NR = NRec<VISC>::n;
    constexpr int NQ = VISC ? 14 : 4;
    constexpr int IU = VISC ? 14 : 4, IV = IU + 1;
    const TauS<R> ts = tau_scalars(p, STAGE);
    const R taus = ts.taus;
    const R inv_dl[3] = {p.inv_dl[0], p.inv_dl[1], (R)(1.0 / (ts.taus_d * p.deta_d))};
    R S[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) S[q] = R(0);
    // velocities of the stage at +-1 neighbours (for the shear source)
    R unb[3][2][4];
    // ---------------- KT flux differences along x, y, eta_s (Eq. kt) ----------------
#pragma unroll
    for (int ax = 1; ax <= 3; ++ax) {
      long long id[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        const int o = d - 2;
        const int ii = ax == 1 ? (p.xhalo ? i + o : wrap_index(i + o, p.nx, p.periodic)) : i;
        const int jj = ax == 2 ? wrap_index(j + o, p.ny, p.periodic) : j;
        const int kk = ax == 3 ? wrap_index(k + o, p.ne, p.periodic) : k;
        id[d] = ((long long)ii * p.ny + jj) * p.nep + kk;
      }
      R ut[5], va[5], cs[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        const R ux = ldg(p.pr.u[0] + id[d]), uy = ldg(p.pr.u[1] + id[d]), ue = ldg(p.pr.u[2] + id[d]);
        ut[d] = sqrt(R(1) + ux * ux + uy * uy + ue * ue);
        const R ua = ax == 1 ? ux : (ax == 2 ? uy : ue);
        va[d] = ua / ut[d];
        cs[d] = ldg(p.pr.cs + id[d]);
        if (d == 1 || d == 3) {
          const int side = d == 3 ? 1 : 0;
          unb[ax - 1][side][0] = ut[d];
          unb[ax - 1][side][1] = ux;
          unb[ax - 1][side][2] = uy;
          unb[ax - 1][side][3] = ue;
        }
      }
      // reconstructed states: interface i-1/2 (Lm | Rm) and i+1/2 (Lp | Rp)
      R Lm[NR], Rm[NR], Lp[NR], Rp[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        R v[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          if (q < 4) v[d] = ldg(p.T[q] + id[d]);
          else if (VISC && q < 14) v[d] = ldg(p.pi[q - 4] + id[d]);
          else if (q == IU) v[d] = ut[d];
          else if (q == IV) v[d] = va[d];
          else v[d] = ldg(p.pr.P + id[d]);
        }
        const R s1 = minmod(v[1] - v[0], v[2] - v[1]);
        const R s2 = minmod(v[2] - v[1], v[3] - v[2]);
        const R s3 = minmod(v[3] - v[2], v[4] - v[3]);
        Lm[q] = v[1] + R(0.5) * s1;
        Rm[q] = v[2] - R(0.5) * s2;
        Lp[q] = v[2] + R(0.5) * s2;
        Rp[q] = v[3] - R(0.5) * s3;
      }
      R Hm[NQ], Hp[NQ];
      interface_flux<R, VISC>(Lm, Rm, cs[1], cs[2], ax, taus, Hm);
      interface_flux<R, VISC>(Lp, Rp, cs[2], cs[3], ax, taus, Hp);
      const R inv = inv_dl[ax - 1];
#pragma unroll
      for (int q = 0; q < NQ; ++q) S[q] -= (Hp[q] - Hm[q]) * inv;
    }
    // ---------------- own-cell state ----------------
    const R e = p.pr.e[c];
    const R Pc = p.pr.P[c];   // the pressure of T^{mu nu}: P(eps) + Pi
    R Pe = Pc;                // the EOS pressure P(eps) (shear source and regulator)
    R u[4];
    u[1] = p.pr.u[0][c]; u[2] = p.pr.u[1][c]; u[3] = p.pr.u[2][c];
    u[0] = sqrt(R(1) + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
    R pic[10];
    if constexpr (VISC) {
#pragma unroll
      for (int q = 0; q < 10; ++q) pic[q] = p.pi[q][c];
    }
    // geometric source S_T = -(T~^{ee}/tau, 0, 0, T~^{te}/tau)
    {
      R Tee = e * u[3] * u[3] + Pc * (R(1) + u[3] * u[3]);
      if constexpr (VISC) Tee += pic[9];
      S[0] -= p.st_tau * Tee;
      S[3] -= ts.geo * p.T[3][c];
    }
    // u~ at step n and the late velocity (u* in stage 1, u' in stage 2)
    R un[4], ul[4];
    if constexpr (STAGE == 1) {
#pragma unroll
      for (int b = 0; b < 4; ++b) un[b] = u[b];
    } else {
      un[1] = p.un[0][c]; un[2] = p.un[1][c]; un[3] = p.un[2][c];
      un[0] = sqrt(R(1) + un[1] * un[1] + un[2] * un[2] + un[3] * un[3]);
    }
    R ustar0 = un[0];
    if constexpr (VISC) {
      R us1 = R(2) * un[1] - p.up[0][c];
      R us2 = R(2) * un[2] - p.up[1][c];
      R us3 = R(2) * un[3] - p.up[2][c];
      ustar0 = sqrt(R(1) + us1 * us1 + us2 * us2 + us3 * us3);
      if constexpr (STAGE == 1) {
        ul[0] = ustar0; ul[1] = us1; ul[2] = us2; ul[3] = us3;
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) ul[b] = u[b];
      }
      // d~_a u~^b: time difference and central differences
      R du[4][4];
      const R invh = p.inv_h;
#pragma unroll
      for (int b = 0; b < 4; ++b) du[0][b] = (ul[b] - un[b]) * invh;
#pragma unroll
      for (int a = 1; a <= 3; ++a) {
        const R half_inv = R(0.5) * inv_dl[a - 1];
#pragma unroll
        for (int b = 0; b < 4; ++b) du[a][b] = (unb[a - 1][1][b] - unb[a - 1][0][b]) * half_inv;
      }
      R Tc, c2dummy;
      eos_eval<R, R>(p.eos, e, Pe, Tc, c2dummy);
      const R inv_taupi = Tc * p.is.inv_b_etas_hbarc;
      R Spi[10];
      shear_source<R>(ts.geo, u, du, pic, e, Pe, inv_taupi, p.is, Spi);
#pragma unroll
      for (int q = 0; q < 10; ++q) S[4 + q] += Spi[q];
    }
    // ---------------- stage update (Sec. 3) ----------------
    // FP32 path: the increment h S added exactly to the float-float T~
    // (Tnl: the new low parts)
    const R h = p.h;
    R Tnew[4], Tnl[4], pinew[10];
    if constexpr (STAGE == 1) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if constexpr (sizeof(R) == 4) {
          const ff s = ff_add(ff{p.T[m][c], p.Tl[m][c]}, mul_rn(h, S[m]));
          Tnew[m] = s.hi;
          Tnl[m] = s.lo;
        } else {
          Tnew[m] = p.T[m][c] + h * S[m];
        }
      }
      if constexpr (VISC) {
        const R inv = R(1) / ustar0;
#pragma unroll
        for (int q = 0; q < 10; ++q) pinew[q] = (un[0] * pic[q] + h * S[4 + q]) * inv;
        regulate_shear<R>(e, Pe, pinew);
      }
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if constexpr (sizeof(R) == 4) {
          const ff s = ff_add(ff_add(ff{p.Tn[m][c], p.Tnl[m][c]}, ff{p.T[m][c], p.Tl[m][c]}), mul_rn(h, S[m]));
          Tnew[m] = 0.5f * s.hi;
          Tnl[m] = 0.5f * s.lo;
        } else {
          Tnew[m] = R(0.5) * (p.Tn[m][c] + p.T[m][c] + h * S[m]);
        }
      }
      if constexpr (VISC) {
        const R inv = R(0.5) / u[0];
#pragma unroll
        for (int q = 0; q < 10; ++q) pinew[q] = (un[0] * p.pin[q][c] + ustar0 * pic[q] + h * S[4 + q]) * inv;
        regulate_shear<R>(e, Pe, pinew);
      }
    }
    // ---------------- primitive recovery from T_ideal = T - pi ----------------
    R pi4[4] = {R(0), R(0), R(0), R(0)};
    if constexpr (VISC) {
#pragma unroll
      for (int m = 0; m < 4; ++m) pi4[m] = pinew[m];
    }
    const IdealPart<R, VISC> ip = ideal_part<R, VISC>(p, Tnew, Tnl, pi4, tau_scalars(p, 1).taus_new);
    const R E = ip.e, Mx = ip.m[0], My = ip.m[1], Me = ip.m[2];
    R en = R(0), ux = R(0), uy = R(0), ue = R(0);
    R Pb = p.Pib ? p.Pib[c] : R(0);   // bulk pressure of the stage's output
    if (!(isfinite(E) && isfinite(Mx) && isfinite(My) && isfinite(Me))) {
      f_nonfinite = true;
    } else {
      R vg = R(-1);
      RootResult rr = solve_primitive<R, R>(p.eos, p.eps_cut, E, Mx, My, Me, SolveTraits<R>::tol,
                                            SolveTraits<R>::maxit, en, ux, uy, ue, &vg, nullptr, Pb);
      f_rescaled = rr.rescaled;
      if constexpr (sizeof(R) == 4) {
        // FP64 Newton near the vacuum, at high velocity, and wherever the
        // FP32 solve did not converge (near_cut: see recover_kernel)
        const R M = sqrt(Mx * Mx + My * My + Me * Me);
        f_nonconv = rr.iters < 0;
        const R eraw = E - M * vg;   // the FP32 eps before the vacuum decision
        const bool near_cut = eraw < p.polish_E && eraw > R(kVacuumSure) * p.eps_cut;
        if (E >= p.eps_cut && M > R(0) && (near_cut || M > p.polish_v * E || rr.iters < 0)) {
          rr.iters = polish_root<R>(p, ff_to_double(ip.E), ff_to_double(ip.M[0]), ff_to_double(ip.M[1]),
                                    ff_to_double(ip.M[2]), vg, rr.iters >= 0, en, ux, uy, ue, Pb);
          f_polished = true;
        } else if (en > R(0) && M > R(0)) {   // every other moving cell: one float-float Newton step
          EosAtRoot<R> unused{false, R(0), R(0)};
          correct_root(p.eos, ip.E, ip.M, vg, Pb, p.eps_cut, en, ux, uy, ue, unused);
        }
      }
      f_fail = rr.iters < 0;
      if (f_fail && atomicCAS(p.fail_cell, 0ull, (unsigned long long)c + 1ull) == 0ull) {
        p.fail_EM[0] = (double)E;
        p.fail_EM[1] = (double)sqrt(Mx * Mx + My * My + Me * Me);
      }
    }
    R Pn, Tn_, c2n;
    eos_eval<R, R>(p.eos, en, Pn, Tn_, c2n);
#pragma unroll
    for (int m = 0; m < 4; ++m) p.Tout[m][c] = Tnew[m];
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int m = 0; m < 4; ++m) p.Toutl[m][c] = Tnl[m];
    }
    if constexpr (VISC) {
      const bool vac = !(en > R(0));
#pragma unroll
      for (int q = 0; q < 10; ++q) p.piout[q][c] = vac ? R(0) : pinew[q];
      if (p.Pib && vac) { Pb = R(0); p.Pib[c] = R(0); }
    }
    Pn += Pb;
    if (Pn < R(0)) Pn = R(0);   // the pressure of T^{mu nu}, floored at 0
    p.prout.e[c] = en;
    p.prout.u[0][c] = ux;
    p.prout.u[1][c] = uy;
    p.prout.u[2][c] = ue;
    p.prout.P[c] = Pn;
    p.prout.cs[c] = sqrt(c2n);
    my_T0 = (double)Tnew[0] + (sizeof(R) == 4 ? (double)Tnl[0] : 0.0);
    my_e = (double)en;
  }
  // ---------------- counters and reductions ----------------
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned b_res = __ballot_sync(full, f_rescaled);
  const unsigned b_fail = __ballot_sync(full, f_fail);
  const unsigned b_pol = __ballot_sync(full, f_polished);
  const unsigned b_nf = __ballot_sync(full, f_nonfinite);
  const unsigned b_nc = __ballot_sync(full, f_nonconv);
  if (lane == 0) {
    if (b_res) atomicAdd(p.counters + 0, (unsigned long long)__popc(b_res));
    if (b_fail) { atomicAdd(p.counters + 1, (unsigned long long)__popc(b_fail)); atomicOr(p.err, 1u); }
    if (b_pol) atomicAdd(p.counters + 2, (unsigned long long)__popc(b_pol));
    if (b_nc) atomicAdd(p.counters + 3, (unsigned long long)__popc(b_nc));
    if (b_nf) atomicOr(p.err, 2u);
  }
  if constexpr (STATS) {
    __shared__ double s_sum[kBlock / 32];
    __shared__ double s_max[kBlock / 32];
    double sm = my_T0, mx = my_e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sm += __shfl_down_sync(full, sm, o);
      mx = fmax(mx, __shfl_down_sync(full, mx, o));
    }
    const int wid = threadIdx.x >> 5;
    if (lane == 0) { s_sum[wid] = sm; s_max[wid] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) { a += s_sum[w]; b = fmax(b, s_max[w]); }
      p.block_sum[blockIdx.x] = a;
      if (b > 0.0) atomicMax(p.emax_bits, (unsigned long long)__double_as_longlong(b));
    }
  }
}

// Primitive recovery of one stage (used after the tiled stage kernel): reads
// the new T~^{tau mu} and pi~^{tau mu}, solves for (eps, u~) warm-started
// from the stage velocity, writes P and c_s, zeroes pi~ in vacuum cells, and
// (STATS) reduces sum T~^{tau tau} and max eps.
// at least four 256-thread blocks per SM in FP32 (at most 64 registers): the
// dependent table lookups of the root solve need the occupancy
template <typename R>
struct RecoverMinBlocks {
  static constexpr int value = sizeof(R) == 4 ? 4 : 3;
};

template <typename R, bool VISC, bool STATS, int GUESS = kGuessPrevious>
__global__ void __launch_bounds__(kBlock, RecoverMinBlocks<R>::value) recover_kernel(const StageParams<R> p) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = c < p.N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double my_T0 = 0.0, my_e = 0.0;
  int my_iters = 0, my_solved = 0, my_polish_iters = 0;
  bool f_rescaled = false, f_fail = false, f_polished = false, f_nonfinite = false, f_nonconv = false;
  const R tn = tau_scalars(p, 1).taus_new;
  // the ideal part E, M of the new T~ (FP32 path: unrounded float-floats for
  // the correction step, their high parts for the FP32 solve)
  double T0v = 0.0;
  IdealPart<R, VISC> ip{};
  if (active) {
    R Tv[4], Tlv[4] = {R(0), R(0), R(0), R(0)}, pi4[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
    for (int m = 0; m < 4; ++m) Tv[m] = p.Tout[m][c];
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int m = 0; m < 4; ++m) Tlv[m] = p.Toutl[m][c];
    }
    if constexpr (VISC) {
#pragma unroll
      for (int m = 0; m < 4; ++m) pi4[m] = p.piout[m][c];
    }
    T0v = (double)Tv[0] + (double)Tlv[0];
    ip = ideal_part<R, VISC>(p, Tv, Tlv, pi4, tn);
  }
  const R E = ip.e, Mx = ip.m[0], My = ip.m[1], Me = ip.m[2];
  // initial guess for |v|
  R vg = R(-1);
  if constexpr ((GUESS == kGuessMlp || GUESS == kGuessMlpAll) && sizeof(R) == 4) {
    // learned guess: features -> BF16 tensor-core MLP, 32 cells per warp.
    // kGuessMlp runs it only for warps holding a moving cell whose stage
    // velocity is exactly 0 -- a cell leaving vacuum (vacuum cells store
    // u~ = 0), whose root at the fast edge of the flow is far from 0 -- and
    // only blocks holding such a warp load the weights; every other cell
    // starts from its stage velocity, which is closer to the root than the
    // network's guess
    bool want = active;
    if constexpr (GUESS == kGuessMlp) {
      if (active) {
        const R a = p.pr.u[0][c], b = p.pr.u[1][c], d = p.pr.u[2][c];
        const R w2 = a * a + b * b + d * d;
        vg = sqrt(w2 / (R(1) + w2));
        want = E >= p.eps_cut && w2 == R(0) && (Mx != R(0) || My != R(0) || Me != R(0));
      }
    }
    if (__syncthreads_or(want)) {
      __shared__ __align__(16) __nv_bfloat16 s_w[kMlpSmemW];
      __shared__ float s_b[kMlpBiasElems];
      __shared__ __align__(16) __nv_bfloat16 s_x[kBlock / 32][32][kMlpSX];
      __shared__ float s_y[kBlock / 32][32][4];
      mlp_load_smem(p.mlp, s_w, s_b);
      float x[kMlpIn];
      R pij[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
      if constexpr (VISC) {
        if (active) {
          pij[0] = p.piout[4][c]; pij[1] = p.piout[5][c]; pij[2] = p.piout[6][c];
          pij[3] = p.piout[7][c]; pij[4] = p.piout[8][c]; pij[5] = p.piout[9][c];
        }
      }
      mlp_features<R>(active && E > R(0) ? E : R(1), Mx, My, Me, pij, x);
#pragma unroll
      for (int k = 0; k < 16; k += 2)
        *reinterpret_cast<unsigned*>(&s_x[wid][lane][k]) = pack_bf16(k < kMlpIn ? x[k] : 0.f, k + 1 < kMlpIn ? x[k + 1] : 0.f);
      __syncthreads();
      if (__any_sync(0xffffffffu, want)) {   // warp-uniform: the MMA takes the whole warp
        mlp_tile16(&s_x[wid][0][0], s_w, s_b, &s_y[wid][0][0], lane);
        mlp_tile16(&s_x[wid][16][0], s_w, s_b, &s_y[wid][16][0], lane);
        __syncwarp();
        if (want) {
          const float vx = s_y[wid][lane][1], vy = s_y[wid][lane][2], ve = s_y[wid][lane][3];
          vg = R(sqrtf(vx * vx + vy * vy + ve * ve));
        }
      }
    }
  } else if constexpr (GUESS == kGuessPrevious) {
    if (active) {
      const R a = p.pr.u[0][c], b = p.pr.u[1][c], d = p.pr.u[2][c];
      const R w2 = a * a + b * b + d * d;
      vg = sqrt(w2 / (R(1) + w2));   // |v| of the stage velocity
    }
  }
  if (active) {
    R en = R(0), ux = R(0), uy = R(0), ue = R(0);
    R Pb = p.Pib ? p.Pib[c] : R(0);   // bulk pressure of the stage's output
    EosAtRoot<R> at_root{false, R(0), R(0)};
    if (!(isfinite(E) && isfinite(Mx) && isfinite(My) && isfinite(Me))) {
      f_nonfinite = true;
    } else {
      RootResult rr = solve_primitive<R, R>(p.eos, p.eps_cut, E, Mx, My, Me, SolveTraits<R>::tol,
                                            SolveTraits<R>::maxit, en, ux, uy, ue, &vg, &at_root, Pb);
      f_rescaled = rr.rescaled;
      my_iters = rr.iters > 0 ? rr.iters : 0;
      my_solved = rr.iters > 0 ? 1 : 0;
      if constexpr (sizeof(R) == 4) {
        // FP64 refinement of the cancellation-prone arithmetic (E - M v, Newton
        // step, gamma) at high velocity, near the vacuum decision, and wherever
        // the FP32 solve did not converge (inline: a separate pass over a
        // compacted list measured slower, its extra launch and latency-bound
        // tail outweighing the divergence it removes)
        const R M = sqrt(Mx * Mx + My * My + Me * Me);
        f_nonconv = rr.iters < 0;
        // near the cut: the FP32 eps = E - M v before the vacuum decision lies
        // in [kVacuumSure, polish_E/eps_cut) x eps_cut.  With M <= polish_v E
        // (faster cells are refined anyway) its relative error is below 3e-5,
        // so under kVacuumSure eps_cut the cell is vacuum in FP64 too and the
        // refinement could not change it (eps = 0, u = 0)
        const R eraw = E - M * vg;
        const bool near_cut = eraw < p.polish_E && eraw > R(kVacuumSure) * p.eps_cut;
        if (E >= p.eps_cut && M > R(0) && (near_cut || M > p.polish_v * E || rr.iters < 0)) {
          rr.iters = polish_root<R>(p, ff_to_double(ip.E), ff_to_double(ip.M[0]), ff_to_double(ip.M[1]),
                                    ff_to_double(ip.M[2]), vg, rr.iters >= 0, en, ux, uy, ue, Pb);
          my_polish_iters = rr.iters > 0 ? rr.iters : 0;
          f_polished = true;
          at_root.valid = false;   // the refined root: evaluate the table afresh
        } else if (en > R(0) && M > R(0)) {   // every other moving cell: one float-float Newton step
          correct_root(p.eos, ip.E, ip.M, vg, Pb, p.eps_cut, en, ux, uy, ue, at_root);
        }
      }
      f_fail = rr.iters < 0;
      if (f_fail && atomicCAS(p.fail_cell, 0ull, (unsigned long long)c + 1ull) == 0ull) {
        p.fail_EM[0] = (double)E;
        p.fail_EM[1] = (double)sqrt(Mx * Mx + My * My + Me * Me);
      }
    }
    R Pn, c2n;
    if (p.Pib && !(en > R(0))) { Pb = R(0); p.Pib[c] = R(0); }   // vacuum: no bulk pressure
    if (at_root.valid && en > R(0)) {
      // the last Newton iteration looked the table up within the tolerance of
      // the root: move its P (P + Pi with bulk) to the root to first order
      // instead of a new lookup
      Pn = at_root.P;
      c2n = at_root.cs2;
    } else {
      R Tn_;
      eos_eval<R, R>(p.eos, en, Pn, Tn_, c2n);
      Pn += Pb;
      if (Pn < R(0)) Pn = R(0);   // the pressure of T^{mu nu}, floored at 0
    }
    p.prout.e[c] = en;
    p.prout.u[0][c] = ux;
    p.prout.u[1][c] = uy;
    p.prout.u[2][c] = ue;
    p.prout.P[c] = Pn;
    p.prout.cs[c] = sqrt(c2n);
    if constexpr (VISC) {
      if (!(en > R(0))) {
#pragma unroll
        for (int q = 0; q < 10; ++q) p.piout[q][c] = R(0);
      }
    }
    my_T0 = T0v;
    my_e = (double)en;
  }
  const unsigned full = 0xffffffffu;
  const unsigned b_res = __ballot_sync(full, f_rescaled);
  const unsigned b_fail = __ballot_sync(full, f_fail);
  const unsigned b_pol = __ballot_sync(full, f_polished);
  const unsigned b_nf = __ballot_sync(full, f_nonfinite);
  const unsigned b_nc = __ballot_sync(full, f_nonconv);
  const int w_iters = __reduce_add_sync(full, my_iters);
  const int w_solved = __reduce_add_sync(full, my_solved);
  const int w_piters = __reduce_add_sync(full, my_polish_iters);
  const unsigned w_maxit = __reduce_max_sync(full, (unsigned)my_iters);   // a warp runs as long as its slowest lane
  // counters summed per block in shared memory, then one global atomic per
  // counter and block (per-warp global atomics on one cache line queue up
  // in a single L2 slice)
  __shared__ unsigned s_cnt[kBlock / 32][9];
  if (lane == 0) {
    s_cnt[wid][0] = __popc(b_res);
    s_cnt[wid][1] = __popc(b_fail);
    s_cnt[wid][2] = __popc(b_pol);
    s_cnt[wid][3] = __popc(b_nc);
    s_cnt[wid][4] = (unsigned)w_iters;
    s_cnt[wid][5] = (unsigned)w_solved;
    s_cnt[wid][6] = (unsigned)w_piters;
    s_cnt[wid][7] = w_maxit;
    s_cnt[wid][8] = w_maxit ? 1u : 0u;
    if (b_fail) atomicOr(p.err, 1u);
    if (b_nf) atomicOr(p.err, 2u);
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) t += s_cnt[w][threadIdx.x];
    if (t) atomicAdd(p.counters + threadIdx.x, t);
  }
  if constexpr (STATS) {
    __shared__ double s_sum[kBlock / 32];
    __shared__ double s_max[kBlock / 32];
    double sm = my_T0, mx = my_e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sm += __shfl_down_sync(full, sm, o);
      mx = fmax(mx, __shfl_down_sync(full, mx, o));
    }
    if (lane == 0) { s_sum[wid] = sm; s_max[wid] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) { a += s_sum[w]; b = fmax(b, s_max[w]); }
      p.block_sum[blockIdx.x] = a;
      if (b > 0.0) atomicMax(p.emax_bits, (unsigned long long)__double_as_longlong(b));
    }
  }
}

// Training samples of the current state: features of (E, M, pi~^{ij}) as in
// mlp_features and targets (eps/E, v) of every non-vacuum cell, written
// compacted in cell order.  WRITE = false counts the rows of each block into
// counts[blockIdx]; WRITE = true writes them from the exclusive offsets.
template <typename R> struct SampleIn {
  Ptr10<R> T4;    // T~ (FP32 path: high parts)
  const R* T4l[4];   // FP32 path: low parts of T~ (nullptr in FP64)
  Ptr10<R> pi;
  Prim<R> pr;
  bool viscous;
  R taus, eps_cut;
  long long N;
};

template <typename R>
__device__ __forceinline__ bool sample_of(const SampleIn<R>& a, long long c, float* x, float* y) {
  R Tv[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) Tv[m] = a.T4.p[m][c] + (a.T4l[m] ? a.T4l[m][c] : R(0));
  R E = Tv[0] / a.taus, Mx = Tv[1] / a.taus, My = Tv[2] / a.taus, Me = Tv[3] / a.taus;
  R pij[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  if (a.viscous) {
    E -= a.pi.p[0][c]; Mx -= a.pi.p[1][c]; My -= a.pi.p[2][c]; Me -= a.pi.p[3][c];
#pragma unroll
    for (int k = 0; k < 6; ++k) pij[k] = a.pi.p[4 + k][c];
  }
  const R e = a.pr.e[c];
  if (!(E >= a.eps_cut) || !(e > R(0)) || !isfinite(E)) return false;
  mlp_features<R>(E, Mx, My, Me, pij, x);
  const R u1 = a.pr.u[0][c], u2 = a.pr.u[1][c], u3 = a.pr.u[2][c];
  const R iut = R(1) / sqrt(R(1) + u1 * u1 + u2 * u2 + u3 * u3);
  y[0] = float(e / E);
  y[1] = float(u1 * iut);
  y[2] = float(u2 * iut);
  y[3] = float(u3 * iut);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) ok = ok && isfinite(x[k]);
  return ok;
}

template <typename R, bool WRITE>
__global__ void __launch_bounds__(kBlock) mlp_samples_kernel(const SampleIn<R> a, unsigned* counts,
                                                             const unsigned long long* offsets, float* X, float* Y) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float x[kMlpIn], y[kMlpOut];
  const bool ok = c < a.N && sample_of(a, c, x, y);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, ok);
  __shared__ unsigned s_w[kBlock / 32];
  if (lane == 0) s_w[wid] = __popc(b);
  __syncthreads();
  if (!WRITE) {
    if (threadIdx.x == 0) {
      unsigned t = 0;
      for (int w = 0; w < kBlock / 32; ++w) t += s_w[w];
      counts[blockIdx.x] = t;
    }
    return;
  }
  if (!ok) return;
  unsigned before = 0;
  for (int w = 0; w < wid; ++w) before += s_w[w];
  const long long row = (long long)offsets[blockIdx.x] + before + __popc(b & ((1u << lane) - 1u));
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) X[row * kMlpIn + k] = x[k];
#pragma unroll
  for (int k = 0; k < kMlpOut; ++k) Y[row * kMlpOut + k] = y[k];
}

// Exclusive scan of n block counts (one block of kBlock threads; each thread
// scans a contiguous chunk), total into *total.
static __global__ void __launch_bounds__(kBlock) scan_counts_kernel(const unsigned* counts, int n,
                                                             unsigned long long* offsets, long long* total) {
  __shared__ unsigned long long s_part[kBlock];
  const int per = (n + kBlock - 1) / kBlock;
  const int lo = threadIdx.x * per, hi = min(n, lo + per);
  unsigned long long t = 0;
  for (int i = lo; i < hi; ++i) t += counts[i];
  s_part[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int w = 0; w < kBlock; ++w) { const unsigned long long v = s_part[w]; s_part[w] = run; run += v; }
    *total = (long long)run;
  }
  __syncthreads();
  unsigned long long run = s_part[threadIdx.x];
  for (int i = lo; i < hi; ++i) { offsets[i] = run; run += counts[i]; }
}

// T~^{tau mu} = tau [(e + P) u^tau u^mu - P g~^{tau mu} + pi~^{tau mu}], in
// FP64 from the stored primitives; written as R, and (FP32 path, lo != null)
// as float-float pairs: high parts T, low parts lo
template <typename R>
__global__ void __launch_bounds__(kBlock) tilde_T_kernel(Prim<R> pr, Ptr10<R> pi, bool with_pi, Ptr10<R> T,
                                                         Ptr10<R> lo, bool with_lo, double taus, long long N) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const double e = pr.e[c], P = pr.P[c];
  const double u1 = pr.u[0][c], u2 = pr.u[1][c], u3 = pr.u[2][c];
  const double u0 = sqrt(1.0 + u1 * u1 + u2 * u2 + u3 * u3);
  const double w = (e + P) * u0;
  double a0 = w * u0 - P, a1 = w * u1, a2 = w * u2, a3 = w * u3;
  if (with_pi) { a0 += (double)pi.p[0][c]; a1 += (double)pi.p[1][c]; a2 += (double)pi.p[2][c]; a3 += (double)pi.p[3][c]; }
  const double v[4] = {taus * a0, taus * a1, taus * a2, taus * a3};
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const R hi = (R)v[m];
    T.p[m][c] = hi;
    if (with_lo) lo.p[m][c] = (R)(v[m] - (double)hi);
  }
}

// Initial primitives (already converted to R in pr.e and pr.u): vacuum below
// eps_cut (eps = 0, u = 0, pi = 0), P and c_s from the EOS, copy to the n-1 set.
template <typename R>
__global__ void __launch_bounds__(kBlock) init_primitives_kernel(Prim<R> pr, Prim<R> prev, Ptr10<R> pi,
                                                                 bool with_pi, EosView<R> eos,
                                                                 double eps_cut, long long N) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  R e = pr.e[c];
  R a = pr.u[0][c], b = pr.u[1][c], d = pr.u[2][c];
  const bool vac = !(e >= R(eps_cut));
  if (vac) {
    e = R(0); a = R(0); b = R(0); d = R(0);
    if (with_pi) {
#pragma unroll
      for (int q = 0; q < 10; ++q) pi.p[q][c] = R(0);
    }
  }
  R P, T, c2;
  eos_eval<R, R>(eos, e, P, T, c2);
  const R cs = sqrt(c2);
  pr.e[c] = e; pr.u[0][c] = a; pr.u[1][c] = b; pr.u[2][c] = d; pr.P[c] = P; pr.cs[c] = cs;
  prev.e[c] = e; prev.u[0][c] = a; prev.u[1][c] = b; prev.u[2][c] = d; prev.P[c] = P; prev.cs[c] = cs;
}

// u~^{-1} = 2 u~^0 - u~^1_ideal, written over the ideal-step result.
template <typename R>
__global__ void __launch_bounds__(kBlock) extrapolate_prev_kernel(Prim<R> cur, Prim<R> prev, long long N) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
#pragma unroll
  for (int m = 0; m < 3; ++m) prev.u[m][c] = R(2) * cur.u[m][c] - prev.u[m][c];
}

// Cell c of the compact order (nx, ny, neta) <-> its slot in the padded
// layout, whose eta rows have a pitch nep >= neta (a multiple of 4).
__device__ __forceinline__ long long padded_index(long long c, int ne, int nep) {
  return (c / ne) * nep + c % ne;
}

template <typename R>
__global__ void __launch_bounds__(kBlock) export_kernel(const R* src, double* dst, long long N, int ne, int nep) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) dst[c] = (double)src[padded_index(c, ne, nep)];
}

// a float-float field (high and low parts) as compact doubles
template <typename R>
__global__ void __launch_bounds__(kBlock) export_pair_kernel(const R* hi, const R* lo, double* dst, long long N, int ne,
                                                             int nep) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) {
    const long long k = padded_index(c, ne, nep);
    dst[c] = (double)hi[k] + (double)lo[k];
  }
}

// Deterministic final sum of the per-block partials (one block).
static __global__ void __launch_bounds__(1024) finalize_sum_kernel(const double* partial, int n, double* out) {
  __shared__ double s[1024];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += partial[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

}  // namespace clv
