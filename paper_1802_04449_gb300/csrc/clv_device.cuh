// clv_device.cuh -- device-side building blocks of the viscous Milne hydro
// step (CLVisc method: Pang, Petersen, Wang).  Templated on the storage /
// arithmetic type R (float or double).
//
// Notation: tilde variables of Sec. 2 of the paper, g~ = diag(1,-1,-1,-1).
// Symmetric shear components are numbered
//     0 tt  1 tx  2 ty  3 te  4 xx  5 xy  6 xe  7 yy  8 ye  9 ee
// (t = tau, e = eta_s).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace clv {

constexpr double kHbarC = 0.1973269804;  // GeV fm
constexpr double kDofConformal = 47.5;   // u, d, s quarks + gluons

// Slot of the symmetric component (m, n) in the packed order tt, tx, ty, te,
// xx, xy, xe, yy, ye, ee.  Written without recursion: a recursive form is not
// always folded and then costs a call with a stack frame inside the flux loops.
__host__ __device__ constexpr int sym_index(int m, int n) {
  return (m < n ? m : n) == 0 ? (m < n ? n : m)
         : (m < n ? m : n) == 1 ? 3 + (m < n ? n : m)
         : (m < n ? m : n) == 2 ? 5 + (m < n ? n : m)
                                : 9;
}
__host__ __device__ constexpr double metric_sign(int m) { return m == 0 ? 1.0 : -1.0; }

template <typename R> struct Fast;
template <> struct Fast<float> {
  static __device__ __forceinline__ float log(float x) { return __logf(x); }
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
};
template <> struct Fast<double> {
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};

// ---------------------------------------------------------------------------
// Equation of state.  Conformal: P = e/3, c_s^2 = 1/3, T = (e/(3a))^{1/4}
// with a = g pi^2/(90 (hbar c)^3).  Table: P, T, c_s^2 at nodes uniform in
// ln e, linear in ln e between nodes; below node 0 P and T scale as e and
// e^{1/4}; above the last node a conformal continuation.
// ---------------------------------------------------------------------------
template <typename R> struct EosView {
  int kind;        // 0 conformal, 1 table
  int n;
  R lne0, inv_dlne;
  R e0, e_top;             // eps of node 0 and of the last node
  R t_coef;                // conformal: T^4 = t_coef * e
  R top;                   // n - 1 as R
  const R* node;           // table nodes packed as (P, T, c_s^2, Plo), 4 values per node (Node)
  // FP32 table lookups: for e = m 2^ex (frexp, m in [0.5, 1)), entry ex + 125
  // holds (ex ln 2 - lne0)/dlne, formed in FP64 on the host and split into its
  // integer part and its fraction (ex in [-125, 128]: every positive normal float)
  const float2* xk;
};

// Node k: P, T, c_s^2 and, in the FP32 table, Plo = P - (float)P (the rest of
// the FP64 pressure, so that the interpolated P carries no rounding of the
// node values: P enters every flux and the root solve); 0 in FP64.
template <typename R> struct Node { R P, T, c2, Plo; };
__device__ __forceinline__ Node<float> load_node(const float* base, int k) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(base) + k);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Node<double> load_node(const double* base, int k) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(base) + 2 * k);
  const double2 b = __ldg(reinterpret_cast<const double2*>(base) + 2 * k + 1);
  return {a.x, a.y, b.x, 0.0};
}

// Evaluate in arithmetic type C (C may be wider than the table type R).
template <typename C, typename R>
__device__ __forceinline__ void eos_eval(const EosView<R>& q, C e, C& P, C& T, C& cs2) {
  if (q.kind == 0) {
    P = e * C(1.0 / 3.0);
    cs2 = C(1.0 / 3.0);
    T = (e > C(0)) ? sqrt(sqrt(C(q.t_coef) * e)) : C(0);
    return;
  }
  if (!(e > C(0))) {
    P = C(0);
    T = C(0);
    cs2 = C(load_node(q.node, 0).c2);
    return;
  }
  int k;
  C w;
  if constexpr (sizeof(C) == 4 && sizeof(R) == 4) {
    // The table position x = (ln e - lne0)/dlne runs up to n - 1 (4095), where
    // an FP32 x keeps only ~2e-4 of a node interval: P would carry ~1e-6
    // relative noise from the lookup alone.  So x is never formed as one
    // float: x = xk[ex] + ln(m)/dlne with ln(m) in (-0.7, 0] to ~1e-7, and the
    // fraction of the sum is exact to ~1e-5 of a node interval.
    int ex;
    const float m = frexpf(e, &ex);
    if (ex < -125) {
      k = -1;
      w = C(0);
    } else if (ex > 128) {
      k = q.n;
      w = C(0);
    } else {
      const float2 tk = __ldg(q.xk + (ex + 125));
      const float s = tk.y + logf(m) * q.inv_dlne;
      const float fs = floorf(s);
      k = (int)tk.x + (int)fs;
      w = s - fs;
    }
  } else {
    const C x = (Fast<C>::log(e) - C(q.lne0)) * C(q.inv_dlne);
    k = x < C(0) ? -1 : (int)x;
    w = x - C(k);
  }
  if (k < 0) {
    const Node<R> a = load_node(q.node, 0);
    C r = e / C(q.e0);
    P = C(a.P) * r;
    T = C(a.T) * sqrt(sqrt(r));
    cs2 = C(a.c2);
    return;
  }
  if (k >= q.n - 1) {
    const Node<R> a = load_node(q.node, q.n - 1);
    P = C(a.P) + (e - C(q.e_top)) * C(1.0 / 3.0);
    T = C(a.T) * sqrt(sqrt(e / C(q.e_top)));
    cs2 = C(1.0 / 3.0);
    return;
  }
  const Node<R> a = load_node(q.node, k), b = load_node(q.node, k + 1);
  P = C(a.P) + w * (C(b.P) - C(a.P));
  if constexpr (sizeof(R) == 4) P += C(a.Plo) + w * (C(b.Plo) - C(a.Plo));
  T = C(a.T) + w * (C(b.T) - C(a.T));
  cs2 = C(a.c2) + w * (C(b.c2) - C(a.c2));
}

// ---------------------------------------------------------------------------
// Primitive recovery: T_ideal^{tau mu} = (E, M) -> (eps, u~).  Root of
// f(v) = v - M/(E + P(E - M v)) on [0, M/E] by Newton steps kept inside a
// shrinking bracket (bisection when a step leaves it).
// ---------------------------------------------------------------------------
// M above (1 - kMaxMoverE) E is rescaled onto that bound before the solve, so
// the flow's Lorentz factor stays below ~22.  The bound only acts in the
// dilute, ultra-relativistic fringe of an expanding event, where E/eps grows
// as gamma^2 and eps = E - M v is ill-conditioned.
constexpr double kMaxMoverE = 1e-3;

struct RootResult {
  int iters;      // -1: cap reached
  int rescaled;   // |M| > (1 - kMaxMoverE) E was rescaled
};

// Division and square root for the FP64 refinement of the FP32 path: an FP32
// seed refined by Newton steps in FP64 (fused multiply-adds only; relative
// error ~1e-15), instead of the long FP64 division / square-root sequences.
__device__ __forceinline__ double refine_rcp(double b) {
  double r = (double)__frcp_rn((float)b);
  r = r * fma(-b, r, 2.0);
  r = r * fma(-b, r, 2.0);
  return r;
}
__device__ __forceinline__ double refine_sqrt(double x) {
  if (!(x > 0.0)) return 0.0;
  double y = (double)rsqrtf((float)x);  // ~ 1/sqrt(x)
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  return x * y;
}
__device__ __forceinline__ double refine_rsqrt(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  return y;
}
template <typename C, typename CE> struct SolveOps {
  static __device__ __forceinline__ C div(C a, C b) { return a / b; }
  static __device__ __forceinline__ C sqrt_(C x) { return sqrt(x); }
  static __device__ __forceinline__ C rsqrt_(C x) { return C(1) / sqrt(x); }
};
template <> struct SolveOps<float, float> {
  static __device__ __forceinline__ float div(float a, float b) { return a / b; }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
};
template <> struct SolveOps<double, float> {
  static __device__ __forceinline__ double div(double a, double b) { return a * refine_rcp(b); }
  static __device__ __forceinline__ double sqrt_(double x) { return refine_sqrt(x); }
  static __device__ __forceinline__ double rsqrt_(double x) { return refine_rsqrt(x); }
};

// C: arithmetic of the solve (E - M v, f, Newton step, gamma); CE: arithmetic
// of the EOS lookup (CE may be narrower than C: the FP32 path refines in FP64
// around an FP32 table lookup).
// FIXED: from a usable guess, run at most maxit Newton steps and accept the
// last iterate (the FP64 refinement of an FP32 root, which starts inside
// Newton's quadratic basin and whose FP32 table lookup leaves a noise floor
// above tol); without one, solve in full (up to 100 steps).
// P and c_s^2 at the root, from the last iteration's table lookup (at
// e_last) moved to the final eps to first order: P + c_s^2 (eps - e_last).
// valid = false when no iteration ran (vacuum, M = 0).
// Pshift is added to the table's P wherever the solve uses the pressure: the
// bulk pressure Pi, for which T^{mu nu} carries P + Pi floored at 0 (0
// without bulk, where P >= 0 leaves the floor inactive).  On the floor dP/de
// is 0, f(v) stays increasing and its root on [0, M/E] unique.
template <typename C> struct EosAtRoot {
  bool valid;
  C P, cs2;
};

template <typename C, typename R, typename CE = C, bool FIXED = false>
__device__ __forceinline__ RootResult solve_primitive(const EosView<R>& q, C eps_cut, C E, C Mx,
                                                      C My, C Me, C tol, int maxit, C& eps,
                                                      C& ux, C& uy, C& ue, C* vguess = nullptr,
                                                      EosAtRoot<C>* at_root = nullptr, C Pshift = C(0)) {
  if (at_root) at_root->valid = false;
  using Ops = SolveOps<C, CE>;
  RootResult rr{0, 0};
  eps = C(0);
  ux = uy = ue = C(0);
  if (!(E >= eps_cut)) return rr;
  C M2 = Mx * Mx + My * My + Me * Me;
  C M = Ops::sqrt_(M2);
  C Mcap = C(1.0 - kMaxMoverE) * E;
  if (M > Mcap) {
    C s = Ops::div(Mcap, M);
    Mx *= s; My *= s; Me *= s;
    M = Mcap;
    rr.rescaled = 1;
  }
  if (M == C(0)) {
    eps = (E >= eps_cut) ? E : C(0);
    return rr;
  }
  C lo = C(0), hi = Ops::div(M, E);
  C P, cs2, dPde;   // dPde: d(P + Pshift)/d eps, 0 on the floor (cs2 keeps the table's value)
  C v;
  bool fixed = FIXED;
  if (vguess && *vguess > lo && *vguess < hi) {
    v = *vguess;
  } else {
    if (FIXED) { fixed = false; maxit = 100; }  // no usable start: solve in full
    CE Pe, Te, ce;
    eos_eval<CE, R>(q, CE(E), Pe, Te, ce);
    P = C(Pe) + Pshift;
    if (P < C(0)) P = C(0);
    v = Ops::div(M, E + P);
  }
  int it = 1;
  bool ok = false;
  C e_last = C(0);
  for (; it <= maxit; ++it) {
    C e = E - M * v;
    e_last = e;
    {
      CE Pe, Te, ce;
      eos_eval<CE, R>(q, CE(e), Pe, Te, ce);
      P = C(Pe) + Pshift;
      cs2 = C(ce);
      dPde = cs2;
      if (P < C(0)) { P = C(0); dPde = C(0); }
    }
    // Newton step on f(v) = v - M/den, den = E + P: with g = v den - M
    // (the sign of f, den > 0) the step -f/f' is -den g / (den^2 - c_s^2 M^2),
    // one division
    const C den = E + P;
    const C g = v * den - M;
    if (g > C(0)) hi = v; else lo = v;
    const C dv = -Ops::div(den * g, den * den - dPde * (M * M));
    // converged when the Newton step is below tol; otherwise keep the iterate
    // strictly inside the shrinking bracket
    if (fabs(dv) <= tol) { v += dv; ok = true; break; }
    C vn = v + dv;
    if (!(vn > lo && vn < hi)) vn = C(0.5) * (lo + hi);
    v = vn;
    if (hi - lo <= tol) { ok = true; break; }
  }
  if (fixed && !ok) { ok = true; it = maxit; }
  rr.iters = ok ? it : -1;
  if (vguess) *vguess = v;
  C e = E - M * v;
  if (e < eps_cut) return rr;
  eps = e;
  if (at_root) {
    at_root->valid = true;
    at_root->P = P + dPde * (e - e_last);
    at_root->cs2 = cs2;
  }
  C gam = Ops::rsqrt_(C(1) - v * v);
  C s = Ops::div(gam * v, M);
  ux = s * Mx;
  uy = s * My;
  ue = s * Me;
  return rr;
}

// ---------------------------------------------------------------------------
// Float-float ("double-single") arithmetic: a value held as hi + lo with
// |lo| <= ulp(hi)/2, about 48 significant bits, computed on the FP32 pipes
// (GB300's FP64 rate is a small fraction of its FP32 rate).  Error-free
// transformations: Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|) and
// the FMA-based exact product.  Sums and products are written so that the
// compiler cannot fuse them (explicit fmaf and __fmul_rn where it matters).
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// (a.hi + a.lo) + b
__device__ __forceinline__ ff ff_add(ff a, float b) {
  ff s = ff_two_sum(a.hi, b);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float s = sqrtf(a.hi);
  // one Newton correction: s + (a - s^2)/(2 s), the residual exact by FMA
  const float r = __fadd_rn(fmaf(-s, s, a.hi), a.lo);
  return ff_fast_two_sum(s, r / (2.f * s));
}
__device__ __forceinline__ ff ff_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes per element).
__device__ __forceinline__ void cp_async_elem(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// this thread's groups complete in commit order: wait for all but the most
// recently committed one
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Product rounded on its own (never fused into a neighbouring add), so that
// differences of equal products cancel exactly.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// minmod(a, b): 0 unless a and b share a sign, else the one of smaller
// magnitude (the value is a, b or 0 exactly).  FP32: b clamped to the
// interval between 0 and a, four min/max operations on the ALU pipe.  FP64:
// min/max and comparisons would run on GB300's narrow FP64 pipe, so the
// choice is made on the bit patterns with integer operations: for finite
// IEEE values the magnitudes order like their bits without the sign; equal
// magnitudes give a.
__device__ __forceinline__ float minmod(float a, float b) {
  return fminf(fmaxf(b, fminf(a, 0.0f)), fmaxf(a, 0.0f));
}
__device__ __forceinline__ double minmod(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned long long mag = 0x7fffffffffffffffull;
  const bool same = ((ua ^ ub) >> 63) == 0ull;
  const unsigned long long pick = (ub & mag) < (ua & mag) ? ub : ua;
  return __longlong_as_double((long long)(same ? pick : 0ull));
}

}  // namespace clv
