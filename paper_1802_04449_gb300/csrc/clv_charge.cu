// clv_charge.cu -- net charge transport of a single-event handle (clv_config
// charge = 1): the conserved N~^tau = tau n u~^tau of Eq. (Ntilde) with
// S_N = 0 and no diffusion current (ideal charge; the paper runs with n = 0).
//
// One launch per Heun stage, after the stage kernel and the root solve,
// reading the stage's input primitives (the velocities the T~ fluxes used):
//   - per axis, Kurganov-Tadmor fluxes at the cell's two interfaces from the
//     minmod-limited reconstruction of N~^tau and of v^a = u~^a / u~^tau on
//     each side, with the local speed max over the sides of
//     (|v^a| + c_s)/(1 + |v^a| c_s) (c_s of the cell on that side);
//   - divisors dx, dy, tau_s deta;
//   - stage 1: N' = N^n + h S;  stage 2: N^{n+1} = (N^n + N' + h S(N')) / 2.
// Boundary cells are clamped (zero gradient) or wrapped (periodic).  Vacuum
// cells keep their charge.
#include <cuda_runtime.h>

#include "clv_kernels.cuh"

namespace clv {

template <typename R>
struct ChargeCell {
  R N, v, cs;
};

template <typename R>
__device__ __forceinline__ ChargeCell<R> charge_cell(const StageParams<R>& p, const R* __restrict__ Nin, long long s,
                                                     int axis) {
  const R ux = p.pr.u[0][s], uy = p.pr.u[1][s], ue = p.pr.u[2][s];
  const R ut = sqrt(R(1) + ux * ux + uy * uy + ue * ue);
  const R ua = axis == 0 ? ux : (axis == 1 ? uy : ue);
  return ChargeCell<R>{Nin[s], ua / ut, p.pr.cs[s]};
}

// flux at the interface between cells b and c from cells a, b, c, d
template <typename R>
__device__ __forceinline__ R charge_flux(const ChargeCell<R>& a, const ChargeCell<R>& b, const ChargeCell<R>& c,
                                         const ChargeCell<R>& d) {
  const R NL = b.N + R(0.5) * minmod(b.N - a.N, c.N - b.N);
  const R NR = c.N - R(0.5) * minmod(c.N - b.N, d.N - c.N);
  const R vL = b.v + R(0.5) * minmod(b.v - a.v, c.v - b.v);
  const R vR = c.v - R(0.5) * minmod(c.v - b.v, d.v - c.v);
  const R lL = (fabs(vL) + b.cs) / (R(1) + fabs(vL) * b.cs);
  const R lR = (fabs(vR) + c.cs) / (R(1) + fabs(vR) * c.cs);
  const R lam = lL > lR ? lL : lR;
  return R(0.5) * (vL * NL + vR * NR) - R(0.5) * lam * (NR - NL);
}

template <typename R, int STAGE>
__global__ void __launch_bounds__(kBlock) charge_stage_kernel(const StageParams<R> p, const R* __restrict__ Nin,
                                                              const R* Nn, R* Nout) {   // Nn == Nout in stage 2
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const int k = (int)(c % p.nep);
  if (k >= p.ne) return;   // padding slot of the eta pitch
  const long long row = c / p.nep;
  const int j = (int)(row % p.ny), i = (int)(row / p.ny);
  const TauS<R> ts = tau_scalars(p, STAGE);
  const R inv_dl[3] = {p.inv_dl[0], p.inv_dl[1], (R)(1.0 / (ts.taus_d * p.deta_d))};
  R S = R(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    ChargeCell<R> q[5];
    // interior cells: neighbours at a fixed stride; within two cells of an
    // edge: clamped (zero gradient) or wrapped (periodic) indices
    const int pos = ax == 0 ? i : (ax == 1 ? j : k), n = ax == 0 ? p.nx : (ax == 1 ? p.ny : p.ne);
    const long long stride = ax == 0 ? (long long)p.ny * p.nep : (ax == 1 ? (long long)p.nep : 1ll);
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      long long s = c + o * stride;
      if (pos < 2 || pos >= n - 2) s = c + (long long)(wrap_index(pos + o, n, p.periodic) - pos) * stride;
      q[o + 2] = charge_cell(p, Nin, s, ax);
    }
    const R Hm = charge_flux(q[0], q[1], q[2], q[3]);
    const R Hp = charge_flux(q[1], q[2], q[3], q[4]);
    S -= (Hp - Hm) * inv_dl[ax];
  }
  if (STAGE == 1) Nout[c] = Nin[c] + p.h * S;
  else Nout[c] = R(0.5) * (Nn[c] + Nin[c] + p.h * S);
}

// N~^tau = tau0 n u~^tau from compact doubles n and the current primitives
template <typename R>
__global__ void __launch_bounds__(kBlock) charge_init_kernel(const double* __restrict__ n, Prim<R> pr, double taus,
                                                             R* __restrict__ N, long long nc, int ne, int nep) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const long long s = padded_index(c, ne, nep);
  const double ux = pr.u[0][s], uy = pr.u[1][s], ue = pr.u[2][s];
  N[s] = (R)(taus * n[c] * sqrt(1.0 + ux * ux + uy * uy + ue * ue));
}

// n = N~^tau / (tau u~^tau) as compact doubles
template <typename R>
__global__ void __launch_bounds__(kBlock) charge_density_kernel(const R* __restrict__ N, Prim<R> pr, double taus,
                                                                double* __restrict__ out, long long nc, int ne,
                                                                int nep) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const long long s = padded_index(c, ne, nep);
  const double ux = pr.u[0][s], uy = pr.u[1][s], ue = pr.u[2][s];
  out[c] = (double)N[s] / (taus * sqrt(1.0 + ux * ux + uy * uy + ue * ue));
}

template <typename R>
void launch_charge_stage(const StageParams<R>& p, int stage, const void* Nin, const void* Nn, void* Nout,
                         cudaStream_t st) {
  const unsigned g = (unsigned)((p.N + kBlock - 1) / kBlock);
  if (stage == 1)
    charge_stage_kernel<R, 1><<<g, kBlock, 0, st>>>(p, (const R*)Nin, (const R*)Nn, (R*)Nout);
  else
    charge_stage_kernel<R, 2><<<g, kBlock, 0, st>>>(p, (const R*)Nin, (const R*)Nn, (R*)Nout);
}

template <typename R>
void launch_charge_init(const double* n, const Prim<R>& pr, double taus, void* N, long long nc, int ne, int nep,
                        cudaStream_t st) {
  const unsigned g = (unsigned)((nc + kBlock - 1) / kBlock);
  charge_init_kernel<R><<<g, kBlock, 0, st>>>(n, pr, taus, (R*)N, nc, ne, nep);
}

template <typename R>
void launch_charge_density(const void* N, const Prim<R>& pr, double taus, double* out, long long nc, int ne, int nep,
                           cudaStream_t st) {
  const unsigned g = (unsigned)((nc + kBlock - 1) / kBlock);
  charge_density_kernel<R><<<g, kBlock, 0, st>>>((const R*)N, pr, taus, out, nc, ne, nep);
}

template void launch_charge_stage<float>(const StageParams<float>&, int, const void*, const void*, void*, cudaStream_t);
template void launch_charge_stage<double>(const StageParams<double>&, int, const void*, const void*, void*,
                                          cudaStream_t);
template void launch_charge_init<float>(const double*, const Prim<float>&, double, void*, long long, int, int,
                                        cudaStream_t);
template void launch_charge_init<double>(const double*, const Prim<double>&, double, void*, long long, int, int,
                                         cudaStream_t);
template void launch_charge_density<float>(const void*, const Prim<float>&, double, double*, long long, int, int,
                                           cudaStream_t);
template void launch_charge_density<double>(const void*, const Prim<double>&, double, double*, long long, int, int,
                                            cudaStream_t);

}  // namespace clv
