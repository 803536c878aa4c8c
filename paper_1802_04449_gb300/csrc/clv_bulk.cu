// clv_bulk.cu -- bulk viscous pressure of a single-event handle (clv_config
// zeta_over_s > 0): Eq. (Pi) in the conservative form of Eq. (Pitilde),
//   d~_tau (u~^tau Pi) + d~_i (u~^i Pi) = S_Pi,
//   S_Pi = -(Pi + zeta theta~)/tau_Pi - Pi theta~/3 - Pi u~^tau/tau,
// theta~ = d~_mu u~^mu + u~^tau/tau (the Milne divergence nabla_mu u^mu),
// tau_Pi = 5 zeta/(T s) with constant zeta/s, so zeta/tau_Pi = (eps + P)/5
// and 1/tau_Pi = T / (5 (zeta/s) hbar c).  The -Pi u~^tau/tau term is the
// Christoffel part of nabla_mu (Pi u^mu); the sign of zeta theta follows
// Eq. (Pi) (Navier-Stokes limit Pi = -zeta theta).
//
// One launch per Heun stage, before the stage kernel (it reads only the
// stage's input: primitives, Pi, u~ at steps n and n-1), writing the stage's
// Pi, which the root solve of the same stage then adds to the pressure:
//   - per axis, Kurganov-Tadmor fluxes at the cell's two interfaces from the
//     minmod-limited reconstructions of u~^tau, v^a and Pi on each side,
//     flux v^a u~^tau Pi, with the local speed of the T~ fluxes;
//   - d~_a u~^a by central differences, d~_tau u~^tau = (u_late - u^n)/h with
//     u_late = u* = 2 u^n - u^{n-1} in stage 1 and the stage-1 velocity in
//     stage 2 (the time difference of the shear source);
//   - stage 1: Pi' = (u~^tau_n Pi^n + h S) / u*^tau;
//     stage 2: Pi^{n+1} = (u~^tau_n Pi^n + u*^tau Pi' + h S) / (2 u'^tau);
//   - regulator with eps and P(eps) of the stage's input: Pi = 0 where
//     eps < 1e-3 GeV/fm^3, else |Pi| <= P.
// Boundary cells are clamped (zero gradient) or wrapped (periodic).
#include <cuda_runtime.h>

#include "clv_kernels.cuh"

namespace clv {

constexpr double kHbarcBulk = 0.1973269804;   // GeV fm

template <typename R>
struct BulkCell {
  R ut, v, Pi, cs, ua;   // u~^tau, v^a, Pi, c_s, u~^a along the axis
};

template <typename R>
__device__ __forceinline__ BulkCell<R> bulk_cell(const StageParams<R>& p, const R* __restrict__ Pin, long long s,
                                                 int axis) {
  const R ux = p.pr.u[0][s], uy = p.pr.u[1][s], ue = p.pr.u[2][s];
  const R ut = sqrt(R(1) + ux * ux + uy * uy + ue * ue);
  const R ua = axis == 0 ? ux : (axis == 1 ? uy : ue);
  return BulkCell<R>{ut, ua / ut, Pin[s], p.pr.cs[s], ua};
}

// flux v^a u~^tau Pi at the interface between cells b and c from cells a, b, c, d
template <typename R>
__device__ __forceinline__ R bulk_flux(const BulkCell<R>& a, const BulkCell<R>& b, const BulkCell<R>& c,
                                       const BulkCell<R>& d) {
  const R utL = b.ut + R(0.5) * minmod(b.ut - a.ut, c.ut - b.ut);
  const R utR = c.ut - R(0.5) * minmod(c.ut - b.ut, d.ut - c.ut);
  const R vL = b.v + R(0.5) * minmod(b.v - a.v, c.v - b.v);
  const R vR = c.v - R(0.5) * minmod(c.v - b.v, d.v - c.v);
  const R PL = b.Pi + R(0.5) * minmod(b.Pi - a.Pi, c.Pi - b.Pi);
  const R PR = c.Pi - R(0.5) * minmod(c.Pi - b.Pi, d.Pi - c.Pi);
  const R lL = (fabs(vL) + b.cs) / (R(1) + fabs(vL) * b.cs);
  const R lR = (fabs(vR) + c.cs) / (R(1) + fabs(vR) * c.cs);
  const R lam = lL > lR ? lL : lR;
  const R QL = utL * PL, QR = utR * PR;
  return R(0.5) * (vL * QL + vR * QR) - R(0.5) * lam * (QR - QL);
}

template <typename R, int STAGE>
__global__ void __launch_bounds__(kBlock) bulk_stage_kernel(const StageParams<R> p, const R* __restrict__ Pin,
                                                            const R* Pn, R* Pout,   // Pn == Pout in stage 2
                                                            const R inv_5zs_hbarc) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const int k = (int)(c % p.nep);
  if (k >= p.ne) return;   // padding slot of the eta pitch
  const long long row = c / p.nep;
  const int j = (int)(row % p.ny), i = (int)(row / p.ny);
  const TauS<R> ts = tau_scalars(p, STAGE);
  const R inv_dl[3] = {p.inv_dl[0], p.inv_dl[1], (R)(1.0 / (ts.taus_d * p.deta_d))};
  R S = R(0), div = R(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    BulkCell<R> q[5];
    // interior cells: neighbours at a fixed stride; within two cells of an
    // edge: clamped (zero gradient) or wrapped (periodic) indices
    const int pos = ax == 0 ? i : (ax == 1 ? j : k), n = ax == 0 ? p.nx : (ax == 1 ? p.ny : p.ne);
    const long long stride = ax == 0 ? (long long)p.ny * p.nep : (ax == 1 ? (long long)p.nep : 1ll);
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      long long s = c + o * stride;
      if (pos < 2 || pos >= n - 2) s = c + (long long)(wrap_index(pos + o, n, p.periodic) - pos) * stride;
      q[o + 2] = bulk_cell(p, Pin, s, ax);
    }
    const R Hm = bulk_flux(q[0], q[1], q[2], q[3]);
    const R Hp = bulk_flux(q[1], q[2], q[3], q[4]);
    S -= (Hp - Hm) * inv_dl[ax];
    div += (q[3].ua - q[1].ua) * (R(0.5) * inv_dl[ax]);   // d~_a u~^a
  }
  // own cell: the stage's input state and the velocities of steps n and n-1
  const R e = p.pr.e[c];
  const R ux = p.pr.u[0][c], uy = p.pr.u[1][c], ue = p.pr.u[2][c];
  const R ut = sqrt(R(1) + ux * ux + uy * uy + ue * ue);
  const R un1 = p.un[0][c], un2 = p.un[1][c], un3 = p.un[2][c];
  const R utn = sqrt(R(1) + un1 * un1 + un2 * un2 + un3 * un3);
  const R us1 = R(2) * un1 - p.up[0][c], us2 = R(2) * un2 - p.up[1][c], us3 = R(2) * un3 - p.up[2][c];
  const R uts = sqrt(R(1) + us1 * us1 + us2 * us2 + us3 * us3);
  const R ut_late = STAGE == 1 ? uts : ut;
  const R theta = (ut_late - utn) * p.inv_h + div + ts.geo * ut;
  R P, T, cs2;
  eos_eval<R, R>(p.eos, e, P, T, cs2);
  const R Pc = Pin[c];
  S += -Pc * (T * inv_5zs_hbarc) - (e + P) * theta * R(0.2) - Pc * theta * (R(1) / R(3)) - ts.geo * ut * Pc;
  R Pnew = STAGE == 1 ? (utn * Pn[c] + p.h * S) / uts : R(0.5) * (utn * Pn[c] + uts * Pc + p.h * S) / ut;
  // regulator (eps and P of the stage's input): the ramp of the shear
  // regulator, then |Pi| <= P
  Pnew *= visc_ramp(e);
  if (Pnew > P) Pnew = P;
  else if (Pnew < -P) Pnew = -P;
  Pout[c] = Pnew;
}

template <typename R>
void launch_bulk_stage(const StageParams<R>& p, int stage, const void* Pin, const void* Pn, void* Pout,
                       double zeta_over_s, cudaStream_t st) {
  const unsigned g = (unsigned)((p.N + kBlock - 1) / kBlock);
  const R coef = (R)(1.0 / (5.0 * zeta_over_s * kHbarcBulk));
  if (stage == 1)
    bulk_stage_kernel<R, 1><<<g, kBlock, 0, st>>>(p, (const R*)Pin, (const R*)Pn, (R*)Pout, coef);
  else
    bulk_stage_kernel<R, 2><<<g, kBlock, 0, st>>>(p, (const R*)Pin, (const R*)Pn, (R*)Pout, coef);
}

template void launch_bulk_stage<float>(const StageParams<float>&, int, const void*, const void*, void*, double,
                                       cudaStream_t);
template void launch_bulk_stage<double>(const StageParams<double>&, int, const void*, const void*, void*, double,
                                        cudaStream_t);

}  // namespace clv
