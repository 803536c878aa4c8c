// clv_cooperfrye.cu -- smooth Cooper-Frye spectra of include/clv.h
// (clv_cf_spectra): dN/(dY pT dpT dphi) of hadron species on a (Y, pT, phi)
// grid from freeze-out surface elements, Sec. 4, Eqs. (cooper_frye) and
// (feq), with the shear correction delta f.
//
// Three launches on the caller's stream:
//   prep     one thread per element: the per-element constants of the sum
//            (e^eta_s and e^-eta_s, dSigma with dSigma_eta / tau, u~, pi~
//            scaled by 1/(2 T^2 (eps + P)) with the off-diagonal factor 2),
//            24 values, 16-byte aligned;
//   sum      grid (momentum tiles, element chunks, species): the elements
//            present (the device count when given) split in whole tiles over
//            the chunks; each thread owns
//            one (Y, pT) and kPhi (8) consecutive phi points; the CTA stages tiles
//            of prepared elements in shared memory (every thread reads the
//            same element: broadcast) and each thread accumulates its points
//            over the tile, then adds the tile sum to FP64 accumulators; the
//            chunk's partial sums go to scratch;
//   reduce   one thread per (species, point): the sum over chunks in a fixed
//            order (deterministic), times g / (2 pi hbar c)^3.
// The paper shares the elements of a work group across many momenta in the
// same way (appendix on the smooth spectra); here the momentum points of a
// thread also share the Y and pT parts of every product.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "clv.h"

void clv_set_global_error(const char* msg);

namespace {

constexpr int kPrep = 24;          // prepared values per element
constexpr int kThreads = 128;      // sum CTA
constexpr int kPhi = 8;            // phi points per thread
constexpr int kTile = 128;         // elements per shared-memory tile
constexpr double kHbarc = 0.1973269804;

constexpr int kMaxSpecies = CLV_CF_MAX_SPECIES;

struct SpeciesDev {
  double mass, g, mu;
  int stat;
};

struct SpeciesSet {
  SpeciesDev s[kMaxSpecies];
};

// element count: the device count when given (a finder's output), capped by n
__device__ __forceinline__ long long element_count(long long n, const int64_t* d_n) {
  if (!d_n) return n;
  const long long m = (long long)*d_n;
  return m < n ? m : n;
}

// prepared element: 0 e^eta, 1 e^-eta, 2-5 dSigma_tau, dSigma_x, dSigma_y,
// dSigma_eta/tau, 6-9 u~, 10-19 scaled pi~ (tt, tx, ty, te, xx, xy, xe, yy,
// ye, ee), 20-23 padding
template <typename R>
__global__ void cf_prep_kernel(const R* __restrict__ rec, long long cap, const int64_t* __restrict__ d_nel,
                               R pi_scale, int viscous, R* __restrict__ prep) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= element_count(cap, d_nel)) return;
  const R* r = rec + e * CLV_FO_NREC;
  R* o = prep + e * kPrep;
  const R eta = r[7], tau = r[4];
  o[0] = exp(eta);
  o[1] = exp(-eta);
  o[2] = r[0];
  o[3] = r[1];
  o[4] = r[2];
  o[5] = r[3] / tau;
#pragma unroll
  for (int m = 0; m < 4; ++m) o[6 + m] = r[8 + m];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    const bool diag = q == 0 || q == 4 || q == 7 || q == 9;
    o[10 + q] = viscous ? r[12 + q] * pi_scale * (diag ? R(1) : R(2)) : R(0);
  }
#pragma unroll
  for (int m = 20; m < kPrep; ++m) o[m] = R(0);
}

template <typename R, bool VISC>
__global__ void __launch_bounds__(kThreads) cf_sum_kernel(const R* __restrict__ prep, long long cap,
                                                          const int64_t* __restrict__ d_nel,
                                                          const double* __restrict__ Y, int nY,
                                                          const double* __restrict__ pT, int npt,
                                                          const double* __restrict__ phi, int nphi,
                                                          const SpeciesSet species, double inv_T,
                                                          double* __restrict__ partial) {
  __shared__ __align__(16) R tile[kTile * kPrep];
  const SpeciesDev sp = species.s[blockIdx.z];
  const long long nel = element_count(cap, d_nel);
  const int cgroups = (nphi + kPhi - 1) / kPhi;
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long nthr = (long long)nY * npt * cgroups;
  const bool active = t < nthr;
  int a = 0, b = 0, c0 = 0;
  if (active) {
    const long long ab = t / cgroups;
    c0 = (int)(t % cgroups) * kPhi;
    a = (int)(ab / npt);
    b = (int)(ab % npt);
  }
  // per-thread momentum constants
  const R y = active ? (R)Y[a] : R(0);
  const R eY = exp(y), emY = exp(-y);
  const R pt_ = active ? (R)pT[b] : R(0);
  const R mT = sqrt(pt_ * pt_ + (R)(sp.mass * sp.mass));
  R px[kPhi], py[kPhi];
#pragma unroll
  for (int j = 0; j < kPhi; ++j) {
    const int c = c0 + j;
    const R ph = (active && c < nphi) ? (R)phi[c] : R(0);
    px[j] = pt_ * cos(ph);
    py[j] = pt_ * sin(ph);
  }
  // exponent in base 2: (p.u - mu)/T log2(e)
  const R k2 = (R)(inv_T * 1.4426950408889634);
  const R mu2 = (R)(sp.mu * inv_T * 1.4426950408889634);
  const R s = (R)sp.stat;
  double acc[kPhi];
#pragma unroll
  for (int j = 0; j < kPhi; ++j) acc[j] = 0.0;
  // the elements split evenly (in whole tiles) over the gridDim.y chunks,
  // by the count actually present
  const long long tiles = (nel + kTile - 1) / kTile;
  const long long chunk = (tiles + gridDim.y - 1) / gridDim.y * kTile;
  const long long e_begin = (long long)blockIdx.y * chunk;
  long long e_end = e_begin + chunk;
  if (e_end > nel) e_end = nel;
  for (long long e0 = e_begin; e0 < e_end; e0 += kTile) {
    const int n = (int)((e_end - e0) < kTile ? (e_end - e0) : kTile);
    __syncthreads();
    // stage n prepared elements (16-byte vectors)
    {
      const int4* src = reinterpret_cast<const int4*>(prep + e0 * kPrep);
      int4* dst = reinterpret_cast<int4*>(tile);
      const int nvec = n * kPrep * (int)sizeof(R) / 16;
      for (int v = threadIdx.x; v < nvec; v += kThreads) dst[v] = src[v];
    }
    __syncthreads();
    R part[kPhi];
#pragma unroll
    for (int j = 0; j < kPhi; ++j) part[j] = R(0);
    for (int i = 0; i < n; ++i) {
      const R* el = tile + i * kPrep;
      // e^(Y - eta) and e^(eta - Y) as products (the addition theorem for
      // cosh(Y - eta) cancels catastrophically in single precision at large
      // |Y| and |eta|)
      const R ep = eY * el[1], em = emY * el[0];
      const R ch = R(0.5) * (ep + em);          // cosh(Y - eta)
      const R sh = R(0.5) * (ep - em);          // sinh(Y - eta)
      const R ptau = mT * ch, peta = mT * sh;
      const R base_dS = ptau * el[2] + peta * el[5];
      const R base_u = ptau * el[6] - peta * el[9];
      // p~_mu p~_nu pi^{mu nu} with p~_mu = (ptau, -px, -py, -peta): the
      // phi-independent part and the coefficients of px and py
      R qt = R(0), a1 = R(0), a2 = R(0);
      if (VISC) {
        qt = ptau * (ptau * el[10] - peta * el[13]) + peta * peta * el[19];
        a1 = peta * el[16] - ptau * el[11];
        a2 = peta * el[18] - ptau * el[12];
      }
      if constexpr (sizeof(R) == 4) {
        // FP32: two phi points per packed FP32x2 instruction (the same
        // IEEE roundings per lane as the scalar path)
        const float2 b_dS = make_float2(base_dS, base_dS), b_u = make_float2(base_u, base_u);
        const float2 e3 = make_float2(el[3], el[3]), e4 = make_float2(el[4], el[4]);
        const float2 e7 = make_float2(-el[7], -el[7]), e8 = make_float2(-el[8], -el[8]);
        const float2 k2v = make_float2(k2, k2), mu2v = make_float2(-mu2, -mu2), sv = make_float2(s, s);
        const float2 one = make_float2(1.f, 1.f), msv = make_float2(-s, -s);
        float2 e14, e15, e17, a1v, a2v, qtv;
        if (VISC) {
          e14 = make_float2(el[14], el[14]);
          e15 = make_float2(el[15], el[15]);
          e17 = make_float2(el[17], el[17]);
          a1v = make_float2(a1, a1);
          a2v = make_float2(a2, a2);
          qtv = make_float2(qt, qt);
        }
#pragma unroll
        for (int j = 0; j < kPhi; j += 2) {
          const float2 X = make_float2(px[j], px[j + 1]), Yv = make_float2(py[j], py[j + 1]);
          const float2 pdS = __ffma2_rn(Yv, e4, __ffma2_rn(X, e3, b_dS));
          const float2 pu = __ffma2_rn(Yv, e8, __ffma2_rn(X, e7, b_u));
          const float2 arg = __ffma2_rn(pu, k2v, mu2v);
          const float2 den = __fadd2_rn(make_float2(exp2f(arg.x), exp2f(arg.y)), sv);
          const float2 f = make_float2(1.f / den.x, 1.f / den.y);
          float2 term = __fmul2_rn(pdS, f);
          if (VISC) {
            const float2 qx = __ffma2_rn(X, __ffma2_rn(Yv, e15, __ffma2_rn(X, e14, a1v)), qtv);
            const float2 q = __ffma2_rn(Yv, __ffma2_rn(Yv, e17, a2v), qx);
            term = __fmul2_rn(term, __ffma2_rn(__ffma2_rn(msv, f, one), q, one));
          }
          part[j] += term.x;
          part[j + 1] += term.y;
        }
      } else {   // FP64
#pragma unroll
        for (int j = 0; j < kPhi; ++j) {
          const R pdS = base_dS + px[j] * el[3] + py[j] * el[4];
          const R pu = base_u - px[j] * el[7] - py[j] * el[8];
          const R f = R(1) / (exp2(pu * k2 - mu2) + s);
          R term = pdS * f;
          if (VISC) {
            const R q = qt + px[j] * (px[j] * el[14] + py[j] * el[15] + a1) + py[j] * (py[j] * el[17] + a2);
            term = term * (R(1) + (R(1) - s * f) * q);
          }
          part[j] += term;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kPhi; ++j) acc[j] += (double)part[j];
  }
  if (active) {
    const long long npts = (long long)nY * npt * nphi;
    double* out = partial + ((long long)blockIdx.y * gridDim.z + blockIdx.z) * npts;
#pragma unroll
    for (int j = 0; j < kPhi; ++j) {
      const int c = c0 + j;
      if (c < nphi) out[((long long)a * npt + b) * nphi + c] = acc[j];
    }
  }
}

__global__ void cf_reduce_kernel(const double* __restrict__ partial, int nchunk, int nsp, long long npts,
                                 const SpeciesSet species, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nsp * npts) return;
  const int z = (int)(i / npts);
  const long long q = i % npts;
  double s = 0.0;
  for (int k = 0; k < nchunk; ++k) s += partial[((long long)k * nsp + z) * npts + q];
  const double norm = species.s[z].g / ((2.0 * M_PI * kHbarc) * (2.0 * M_PI * kHbarc) * (2.0 * M_PI * kHbarc));
  out[i] = norm * s;
}

// ---- host side

constexpr int kTargetCtas = 1216;   // momentum tiles x element chunks x species, about 8 per SM

struct Plan {
  long long npts, nthr;
  int gx, nchunk;
  long long chunk;
  size_t prep_off, partial_off, bytes;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

Plan make_plan(long long nel, int nsp, int nY, int npt, int nphi, size_t rs) {
  Plan P{};
  P.npts = (long long)nY * npt * nphi;
  P.nthr = (long long)nY * npt * ((nphi + kPhi - 1) / kPhi);
  P.gx = (int)((P.nthr + kThreads - 1) / kThreads);
  const long long tiles = (nel + kTile - 1) / kTile;
  long long want = (kTargetCtas + (long long)P.gx * nsp - 1) / ((long long)P.gx * nsp);
  if (want < 1) want = 1;
  if (want > tiles) want = tiles;
  if (want > 65535) want = 65535;
  const long long tiles_per_chunk = want > 0 ? (tiles + want - 1) / want : 0;
  P.chunk = tiles_per_chunk * kTile;
  P.nchunk = P.chunk > 0 ? (int)((nel + P.chunk - 1) / P.chunk) : 0;
  P.prep_off = 0;
  P.partial_off = align256((size_t)nel * kPrep * rs);
  P.bytes = P.partial_off + align256((size_t)P.nchunk * nsp * P.npts * sizeof(double));
  if (P.bytes == 0) P.bytes = 256;
  return P;
}

clv_status bad(const std::string& msg) {
  clv_set_global_error(("clv_cf: " + msg).c_str());
  return CLV_EINVAL;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

clv_status check_sizes(const clv_cf_params* p, int64_t nel, int nsp, int nY, int npt, int nphi) {
  if (!p) return bad("params is NULL");
  if (!(p->Tf > 0)) return bad("Tf must be > 0");
  if (p->viscous && !(p->ePf > 0)) return bad("ePf must be > 0 with viscous");
  if (p->precision != CLV_FP64 && p->precision != CLV_FP32) return bad("precision must be CLV_FP64 or CLV_FP32");
  if (nsp < 1 || nsp > kMaxSpecies) return bad("nsp must be in [1, CLV_CF_MAX_SPECIES]");
  if (nY < 1 || npt < 1 || nphi < 1) return bad("nY, npt, nphi must be >= 1");
  if (nel < 0) return bad("nel < 0");
  if ((long long)nY * npt * nphi >= (1ll << 31)) return bad("more than 2^31 - 1 momentum points");
  return CLV_OK;
}

template <typename R>
clv_status cf_run(const clv_cf_params* p, const clv_cf_species* species, int nsp, const void* d_rec, int64_t nel,
                  const int64_t* d_nel, const double* d_Y, int nY, const double* d_pT, int npt, const double* d_phi,
                  int nphi, double* d_out, void* d_scratch, cudaStream_t st) {
  const Plan P = make_plan(nel, nsp, nY, npt, nphi, sizeof(R));
  SpeciesSet set{};
  for (int z = 0; z < nsp; ++z) {
    set.s[z].mass = species[z].mass;
    set.s[z].g = species[z].g;
    set.s[z].mu = species[z].mu;
    set.s[z].stat = species[z].stat;
  }
  char* sc = static_cast<char*>(d_scratch);
  R* prep = reinterpret_cast<R*>(sc + P.prep_off);
  double* partial = reinterpret_cast<double*>(sc + P.partial_off);
  if (P.nchunk > 0) {
    const double pi_scale = p->viscous ? 1.0 / (2.0 * p->Tf * p->Tf * p->ePf) : 0.0;
    cf_prep_kernel<R><<<(unsigned)((nel + 255) / 256), 256, 0, st>>>(static_cast<const R*>(d_rec), nel, d_nel,
                                                                     (R)pi_scale, p->viscous != 0, prep);
    const dim3 grid((unsigned)P.gx, (unsigned)P.nchunk, (unsigned)nsp);
    if (p->viscous)
      cf_sum_kernel<R, true><<<grid, kThreads, 0, st>>>(prep, nel, d_nel, d_Y, nY, d_pT, npt, d_phi, nphi, set,
                                                        1.0 / p->Tf, partial);
    else
      cf_sum_kernel<R, false><<<grid, kThreads, 0, st>>>(prep, nel, d_nel, d_Y, nY, d_pT, npt, d_phi, nphi, set,
                                                         1.0 / p->Tf, partial);
  }
  const long long nout = (long long)nsp * P.npts;
  cf_reduce_kernel<<<(unsigned)((nout + 255) / 256), 256, 0, st>>>(partial, P.nchunk, nsp, P.npts, set, d_out);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    clv_set_global_error((std::string("clv_cf_spectra: ") + cudaGetErrorString(err)).c_str());
    return CLV_ECUDA;
  }
  return CLV_OK;
}

}  // namespace

extern "C" {

clv_status clv_cf_scratch_bytes(const clv_cf_params* p, int64_t nel, int nsp, int nY, int npt, int nphi,
                                size_t* bytes) {
  const clv_status s = check_sizes(p, nel, nsp, nY, npt, nphi);
  if (s != CLV_OK) return s;
  if (!bytes) return bad("bytes is NULL");
  *bytes = make_plan(nel, nsp, nY, npt, nphi, p->precision == CLV_FP64 ? 8 : 4).bytes;
  return CLV_OK;
}

clv_status clv_cf_spectra(const clv_cf_params* p, const clv_cf_species* species, int nsp, const void* d_rec,
                          int64_t nel, const int64_t* d_nel, const double* d_Y, int nY, const double* d_pT, int npt,
                          const double* d_phi, int nphi, double* d_out, void* d_scratch, void* cuda_stream) {
  const clv_status s = check_sizes(p, nel, nsp, nY, npt, nphi);
  if (s != CLV_OK) return s;
  if (!species) return bad("species is NULL");
  for (int z = 0; z < nsp; ++z) {
    if (!(species[z].mass >= 0) || !(species[z].g > 0)) return bad("species mass must be >= 0 and g > 0");
    if (species[z].stat < -1 || species[z].stat > 1) return bad("species stat must be -1, 0 or +1");
    if (!(species[z].mu == species[z].mu)) return bad("species mu is NaN");
  }
  const size_t rs = p->precision == CLV_FP64 ? 8 : 4;
  if (nel > 0 && (!d_rec || !aligned(d_rec, rs))) return bad("d_rec is NULL or misaligned");
  if (d_nel && !aligned(d_nel, 8)) return bad("d_nel is misaligned");
  if (!d_Y || !d_pT || !d_phi || !aligned(d_Y, 8) || !aligned(d_pT, 8) || !aligned(d_phi, 8))
    return bad("momentum grids are NULL or misaligned");
  if (!d_out || !aligned(d_out, 8)) return bad("d_out is NULL or misaligned");
  if (!d_scratch || !aligned(d_scratch, 256)) return bad("d_scratch is NULL or not 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return p->precision == CLV_FP64
             ? cf_run<double>(p, species, nsp, d_rec, nel, d_nel, d_Y, nY, d_pT, npt, d_phi, nphi, d_out, d_scratch, st)
             : cf_run<float>(p, species, nsp, d_rec, nel, d_nel, d_Y, nY, d_pT, npt, d_phi, nphi, d_out, d_scratch, st);
}

}  // extern "C"
