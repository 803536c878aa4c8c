// clv_freezeout.cu -- the freeze-out surface finder of include/clv.h
// (clv_fo_find): surface elements dSigma_mu of eps = eps_f between two time
// slices, the input of the Cooper-Frye integral of Sec. 4, Eq.
// (cooper_frye), from the piecewise-linear interpolant over the Freudenthal
// triangulation of each space-time hypercube.
//
// Four launches on the caller's stream:
//   classify  one thread per hypercube: crossed or not (16 corner loads, eta
//             fastest across the warp); a flag byte and a count per CTA;
//   scan      one CTA: exclusive prefix of the CTA counts -> CTA offsets and
//             the element count;
//   compact   one thread per hypercube: the crossed hypercubes' indices in
//             increasing order (CTA offset + rank in the CTA);
//   elements  persistent, one warp per element: lane s < 24 takes simplex s
//             of the hypercube, the warp sums the pieces by shuffles, lanes
//             0..12 interpolate the fields and lanes 0..21 store the record.
// The element order and values do not depend on the launch geometry.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "clv.h"

// defined in clv_api.cu: message returned by clv_last_error(NULL)
void clv_set_global_error(const char* msg);

namespace {

constexpr int kThreads = 256;      // classify / compact CTAs
constexpr int kScanThreads = 1024;
constexpr int kElemThreads = 256;  // 8 warps per CTA
constexpr int kNF = 13;            // interpolated fields: u~ (3), pi~ (10)
constexpr unsigned kFull = 0xffffffffu;

template <typename R>
struct FoArgs {
  const R* e[2];           // eps of slice 0 (tau0) and slice 1 (tau1)
  const R* f[2][kNF];      // u~^x, u~^y, u~^eta, pi~ tt..ee (pi entries null when pi = 0)
  int ny, pitch;
  int cy, ce;              // hypercubes along y and eta: ny - 1, neta - 1
  long long ncube;
  R ef;
  R h[4];                  // tau1 - tau0, dx, dy, deta
  R x0[4];                 // tau0 and the coordinates of cell (0, 0, 0)
  R cof[4];                // h0 h1 h2 h3 / h_mu: the 3-volume covector of local edges -> physical
  int cartesian;
  int has_pi;
};

template <typename R>
__device__ __forceinline__ long long corner_offset(const FoArgs<R>& a, int i, int j, int k, int q) {
  return ((long long)(i + (q >> 1 & 1)) * a.ny + (j + (q >> 2 & 1))) * a.pitch + (k + (q >> 3 & 1));
}

__device__ __forceinline__ void decode_cube(long long c, int cy, int ce, int& i, int& j, int& k) {
  k = (int)(c % ce);
  const long long t = c / ce;
  j = (int)(t % cy);
  i = (int)(t / cy);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) fo_classify_kernel(FoArgs<R> a, unsigned char* __restrict__ flags,
                                                               int* __restrict__ counts) {
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  int crossed = 0;
  if (c < a.ncube) {
    int i, j, k;
    decode_cube(c, a.cy, a.ce, i, j, k);
    int nin = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) nin += a.e[q & 1][corner_offset(a, i, j, k, q)] >= a.ef;
    crossed = nin > 0 && nin < 16;
    flags[c] = (unsigned char)crossed;
  }
  const int n = __syncthreads_count(crossed);
  if (threadIdx.x == 0) counts[blockIdx.x] = n;
}

__global__ void __launch_bounds__(kScanThreads) fo_scan_kernel(const int* __restrict__ counts, int nblk,
                                                               long long* __restrict__ offsets,
                                                               long long* __restrict__ total,
                                                               int64_t* __restrict__ d_count) {
  __shared__ long long warp_sum[kScanThreads / 32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += kScanThreads) {
    const int b = base + threadIdx.x;
    const long long v = b < nblk ? counts[b] : 0;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(kFull, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long w = warp_sum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(kFull, w, d);
        if (lane >= d) w += y;
      }
      warp_sum[lane] = w;
    }
    __syncthreads();
    const long long excl = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
    if (b < nblk) offsets[b] = excl;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry;
    *d_count = (int64_t)carry;
  }
}

__global__ void __launch_bounds__(kThreads) fo_compact_kernel(const unsigned char* __restrict__ flags,
                                                              long long ncube,
                                                              const long long* __restrict__ offsets,
                                                              int* __restrict__ list) {
  __shared__ int warp_cnt[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  const int f = c < ncube ? flags[c] : 0;
  const unsigned b = __ballot_sync(kFull, f);
  if (lane == 0) warp_cnt[warp] = __popc(b);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += warp_cnt[w];
  if (f) list[offsets[blockIdx.x] + before + __popc(b & ((1u << lane) - 1u))] = (int)c;
}

// value of a 5-array at a runtime index, by selects (no local memory)
template <typename T>
__device__ __forceinline__ T sel5(const T (&x)[5], int m) {
  return m == 0 ? x[0] : m == 1 ? x[1] : m == 2 ? x[2] : m == 3 ? x[3] : x[4];
}

// level-set point on the simplex edge from inside vertex vi (value fi >= 0)
// to outside vertex vo (fo < 0), in local coordinates of the hypercube
template <typename R>
__device__ __forceinline__ void edge_point(int vi, int vo, R fi, R fo, R p[4]) {
  const R t = fi / (fi - fo);
#pragma unroll
  for (int ax = 0; ax < 4; ++ax) {
    const R bi = (R)(vi >> ax & 1), bo = (R)(vo >> ax & 1);
    p[ax] = bi + t * (bo - bi);
  }
}

template <typename R>
struct Piece {
  R dS[4], A, Ac[4];
};

// one tetrahedron of a piece: physical 3-volume from the local edge minors
// scaled by the cofactors of the diagonal local -> physical map
template <typename R>
__device__ __forceinline__ void add_tet(const FoArgs<R>& a, const R* p0, const R* p1, const R* p2, const R* p3,
                                        const R nhat[4], Piece<R>& pc) {
  R e1[4], e2[4], e3[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    e1[m] = p1[m] - p0[m];
    e2[m] = p2[m] - p0[m];
    e3[m] = p3[m] - p0[m];
  }
  R n2 = 0;
#pragma unroll
  for (int skip = 0; skip < 4; ++skip) {
    const int c0 = skip == 0 ? 1 : 0;
    const int c1 = skip <= 1 ? 2 : 1;
    const int c2 = skip <= 2 ? 3 : 2;
    const R det = e1[c0] * (e2[c1] * e3[c2] - e2[c2] * e3[c1]) - e1[c1] * (e2[c0] * e3[c2] - e2[c2] * e3[c0]) +
                  e1[c2] * (e2[c0] * e3[c1] - e2[c1] * e3[c0]);
    const R n = det * a.cof[skip];
    n2 += n * n;
  }
  const R A = sqrt(n2) / R(6);
  R c[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) c[m] = R(0.25) * (p0[m] + p1[m] + p2[m] + p3[m]);
  const R w = a.cartesian ? R(1) : a.x0[0] + a.h[0] * c[0];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    pc.dS[m] += nhat[m] * A * w;
    pc.Ac[m] += A * c[m];
  }
  pc.A += A;
}

// the piece of the level set in the simplex with vertex corners v[5] and
// values f[5] (f = eps - eps_f)
template <typename R>
__device__ void simplex_piece(const FoArgs<R>& a, const int (&v)[5], const R (&f)[5], const int (&perm)[4],
                              Piece<R>& pc) {
  unsigned inmask = 0;
#pragma unroll
  for (int m = 0; m < 5; ++m) inmask |= (f[m] >= R(0) ? 1u : 0u) << m;
  const int nin = __popc(inmask);
  if (nin == 0 || nin == 5) return;
  R grad[4];
#pragma unroll
  for (int ax = 0; ax < 4; ++ax) {
    R d = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (perm[m] == ax) d = f[m + 1] - f[m];
    grad[ax] = d / a.h[ax];
  }
  const R gn = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2] + grad[3] * grad[3]);
  if (!(gn > R(0))) return;  // only when the differences underflow: no piece
  R nhat[4];
#pragma unroll
  for (int ax = 0; ax < 4; ++ax) nhat[ax] = -grad[ax] / gn;
  // minority side (one or two vertices) against the majority, each in
  // increasing vertex order
  const bool min_in = nin <= 2;
  unsigned mm = min_in ? inmask : (~inmask & 31u);
  unsigned MM = ~mm & 31u;
  int mi[2], Mi[4];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    mi[r] = mm ? __ffs(mm) - 1 : 0;
    mm &= mm - 1u;
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    Mi[s] = MM ? __ffs(MM) - 1 : 0;
    MM &= MM - 1u;
  }
  const int nmin = min_in ? nin : 5 - nin;
  auto point = [&](int r, int s, R p[4]) {
    const int vm = mi[r], vM = Mi[s];
    if (min_in) edge_point<R>(sel5(v, vm), sel5(v, vM), sel5(f, vm), sel5(f, vM), p);
    else edge_point<R>(sel5(v, vM), sel5(v, vm), sel5(f, vM), sel5(f, vm), p);
  };
  if (nmin == 1) {
    R q0[4], q1[4], q2[4], q3[4];
    point(0, 0, q0);
    point(0, 1, q1);
    point(0, 2, q2);
    point(0, 3, q3);
    add_tet<R>(a, q0, q1, q2, q3, nhat, pc);
  } else {
    // prism: triangles (0, s) and (1, s), lateral edges (0, s) - (1, s)
    R q00[4], q01[4], q02[4], q10[4], q11[4], q12[4];
    point(0, 0, q00);
    point(0, 1, q01);
    point(0, 2, q02);
    point(1, 0, q10);
    point(1, 1, q11);
    point(1, 2, q12);
    add_tet<R>(a, q00, q01, q02, q10, nhat, pc);
    add_tet<R>(a, q01, q02, q10, q11, nhat, pc);
    add_tet<R>(a, q02, q10, q11, q12, nhat, pc);
  }
}

template <typename R>
__device__ __forceinline__ R warp_sum(R x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
  return x;
}

// At least four CTAs per SM (at most 64 registers, a 4-byte spill in FP32):
// the warps are latency-bound, and 32 resident warps per SM instead of 24
// (78 registers) made a find 5% faster.
template <typename R>
__global__ void __launch_bounds__(kElemThreads, 4) fo_elements_kernel(FoArgs<R> a, const int* __restrict__ list,
                                                                   const long long* __restrict__ total,
                                                                   long long capacity, R* __restrict__ rec,
                                                                   int64_t* __restrict__ cube_out) {
  const int lane = threadIdx.x & 31;
  // the ordering of the axes of this lane's simplex: lexicographic rank s
  const int s = lane < 24 ? lane : lane - 24;
  int perm[4];
  {
    int avail = 0x3210;  // remaining axes, 4 bits each, increasing
    const int digit[3] = {s / 6, (s / 2) % 3, s % 2};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int sh = 4 * digit[m];
      perm[m] = (avail >> sh) & 15;
      const int low = avail & ((1 << sh) - 1);
      avail = low | ((avail >> (sh + 4)) << sh);
    }
    perm[3] = avail & 15;
  }
  int v[5];
  v[0] = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) v[m + 1] = v[m] | (1 << perm[m]);

  long long n = *total;
  if (n > capacity) n = capacity;
  const long long nwarps = (long long)gridDim.x * (kElemThreads / 32);
  for (long long e = (long long)blockIdx.x * (kElemThreads / 32) + (threadIdx.x >> 5); e < n; e += nwarps) {
    const int c = list[e];
    int i, j, k;
    decode_cube(c, a.cy, a.ce, i, j, k);
    R fq = 0;
    if (lane < 16) fq = a.e[lane & 1][corner_offset(a, i, j, k, lane)] - a.ef;
    R f[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) f[m] = __shfl_sync(kFull, fq, v[m]);
    Piece<R> pc;
#pragma unroll
    for (int m = 0; m < 4; ++m) pc.dS[m] = pc.Ac[m] = 0;
    pc.A = 0;
    if (lane < 24) simplex_piece<R>(a, v, f, perm, pc);
    R dS[4], Ac[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      dS[m] = warp_sum(pc.dS[m]);
      Ac[m] = warp_sum(pc.Ac[m]);
    }
    const R A = warp_sum(pc.A);
    // position (local coordinates) and the simplex that holds it
    R sv[4];
    int so[4];
#pragma unroll
    for (int ax = 0; ax < 4; ++ax) {
      R t = A > R(0) ? Ac[ax] / A : R(0.5);
      sv[ax] = t < R(0) ? R(0) : (t > R(1) ? R(1) : t);
      so[ax] = ax;
    }
    const R pos_tau = a.x0[0] + a.h[0] * sv[0];
    const R pos_x = a.x0[1] + ((R)i + sv[1]) * a.h[1];
    const R pos_y = a.x0[2] + ((R)j + sv[2]) * a.h[2];
    const R pos_e = a.x0[3] + ((R)k + sv[3]) * a.h[3];
#pragma unroll
    for (int p = 1; p < 4; ++p)
#pragma unroll
      for (int b = p; b > 0; --b) {
        const bool sw = sv[b] > sv[b - 1];
        const R tv = sv[b];
        const int to = so[b];
        sv[b] = sw ? sv[b - 1] : tv;
        so[b] = sw ? so[b - 1] : to;
        sv[b - 1] = sw ? tv : sv[b - 1];
        so[b - 1] = sw ? to : so[b - 1];
      }
    R w[5];
    int vq[5];
    w[0] = R(1) - sv[0];
    w[1] = sv[0] - sv[1];
    w[2] = sv[1] - sv[2];
    w[3] = sv[2] - sv[3];
    w[4] = sv[3];
    vq[0] = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) vq[m + 1] = vq[m] | (1 << so[m]);
    R F = 0;
    if (lane < kNF && (lane < 3 || a.has_pi)) {
#pragma unroll
      for (int m = 0; m < 5; ++m) F += w[m] * a.f[vq[m] & 1][lane][corner_offset(a, i, j, k, vq[m])];
    }
    const R ux = __shfl_sync(kFull, F, 0), uy = __shfl_sync(kFull, F, 1), ue = __shfl_sync(kFull, F, 2);
    const R Fr = __shfl_sync(kFull, F, (lane >= 9 && lane < 22) ? lane - 9 : 0);
    if (lane < CLV_FO_NREC) {
      R val;
      switch (lane) {
        case 0: val = dS[0]; break;
        case 1: val = dS[1]; break;
        case 2: val = dS[2]; break;
        case 3: val = dS[3]; break;
        case 4: val = pos_tau; break;
        case 5: val = pos_x; break;
        case 6: val = pos_y; break;
        case 7: val = pos_e; break;
        case 8: val = sqrt(R(1) + ux * ux + uy * uy + ue * ue); break;
        default: val = Fr; break;
      }
      rec[e * CLV_FO_NREC + lane] = val;
    }
    if (lane == 0 && cube_out) cube_out[e] = c;
  }
}

struct ScratchLayout {
  size_t total, counts, offsets, flags, list, bytes;
  long long ncube;
  int nblk;
};

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

ScratchLayout scratch_layout(const clv_fo_grid* g) {
  ScratchLayout L{};
  L.ncube = (long long)(g->nx - 1) * (g->ny - 1) * (g->neta - 1);
  L.nblk = (int)((L.ncube + kThreads - 1) / kThreads);
  size_t o = 0;
  L.total = o;
  o = align16(o + 8);
  L.counts = o;
  o = align16(o + (size_t)L.nblk * 4);
  L.offsets = o;
  o = align16(o + (size_t)L.nblk * 8);
  L.flags = o;
  o = align16(o + (size_t)L.ncube);
  L.list = o;
  o = align16(o + (size_t)L.ncube * 4);
  L.bytes = o;
  return L;
}

clv_status bad(const std::string& msg) {
  clv_set_global_error(("clv_fo: " + msg).c_str());
  return CLV_EINVAL;
}

clv_status check_grid(const clv_fo_grid* g) {
  if (!g) return bad("grid is NULL");
  if (g->nx < 2 || g->ny < 2 || g->neta < 2) return bad("nx, ny, neta must be >= 2");
  if (g->eta_pitch != 0 && g->eta_pitch < g->neta) return bad("eta_pitch < neta");
  if (!(g->dx > 0 && g->dy > 0 && g->deta > 0)) return bad("spacings must be > 0");
  if (g->precision != CLV_FP64 && g->precision != CLV_FP32) return bad("precision must be CLV_FP64 or CLV_FP32");
  const long long ncube = (long long)(g->nx - 1) * (g->ny - 1) * (g->neta - 1);
  if (ncube >= (1ll << 31)) return bad("more than 2^31 - 1 hypercubes");
  return CLV_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename R>
clv_status fo_run(const clv_fo_grid* g, const clv_fo_slice* s0, const clv_fo_slice* s1, double eps_f, void* d_rec,
                  int64_t* d_cube, int64_t capacity, int64_t* d_count, void* d_scratch, cudaStream_t st) {
  const clv_fo_slice* sl[2] = {s0, s1};
  FoArgs<R> a{};
  int npi[2] = {0, 0};
  for (int t = 0; t < 2; ++t) {
    if (!sl[t]->eps || !aligned(sl[t]->eps, sizeof(R))) return bad("slice eps is NULL or misaligned");
    a.e[t] = static_cast<const R*>(sl[t]->eps);
    for (int m = 0; m < 3; ++m) {
      if (!sl[t]->u[m] || !aligned(sl[t]->u[m], sizeof(R))) return bad("slice u is NULL or misaligned");
      a.f[t][m] = static_cast<const R*>(sl[t]->u[m]);
    }
    for (int q = 0; q < 10; ++q) {
      if (sl[t]->pi[q] && !aligned(sl[t]->pi[q], sizeof(R))) return bad("slice pi is misaligned");
      npi[t] += sl[t]->pi[q] != nullptr;
      a.f[t][3 + q] = static_cast<const R*>(sl[t]->pi[q]);
    }
  }
  if ((npi[0] != 0 && npi[0] != 10) || npi[1] != npi[0])
    return bad("pi must be given for all ten components of both slices, or for none");
  a.has_pi = npi[0] == 10;
  const ScratchLayout L = scratch_layout(g);
  a.ny = g->ny;
  a.pitch = g->eta_pitch ? g->eta_pitch : g->neta;
  a.cy = g->ny - 1;
  a.ce = g->neta - 1;
  a.ncube = L.ncube;
  a.ef = (R)eps_f;
  const double h[4] = {s1->tau - s0->tau, g->dx, g->dy, g->deta};
  const double x0[4] = {s0->tau, -0.5 * (g->nx - 1) * g->dx, -0.5 * (g->ny - 1) * g->dy,
                        -0.5 * (g->neta - 1) * g->deta};
  const double vol = h[0] * h[1] * h[2] * h[3];
  for (int m = 0; m < 4; ++m) {
    a.h[m] = (R)h[m];
    a.x0[m] = (R)x0[m];
    a.cof[m] = (R)(vol / h[m]);
  }
  a.cartesian = g->cartesian != 0;
  char* sc = static_cast<char*>(d_scratch);
  long long* total = reinterpret_cast<long long*>(sc + L.total);
  int* counts = reinterpret_cast<int*>(sc + L.counts);
  long long* offsets = reinterpret_cast<long long*>(sc + L.offsets);
  unsigned char* flags = reinterpret_cast<unsigned char*>(sc + L.flags);
  int* list = reinterpret_cast<int*>(sc + L.list);
  fo_classify_kernel<R><<<L.nblk, kThreads, 0, st>>>(a, flags, counts);
  fo_scan_kernel<<<1, kScanThreads, 0, st>>>(counts, L.nblk, offsets, total, d_count);
  fo_compact_kernel<<<L.nblk, kThreads, 0, st>>>(flags, L.ncube, offsets, list);
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fo_elements_kernel<R>, kElemThreads, 0);
  const long long need = (L.ncube + kElemThreads / 32 - 1) / (kElemThreads / 32);
  long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > need) blocks = need;
  fo_elements_kernel<R><<<(unsigned)blocks, kElemThreads, 0, st>>>(a, list, total, (long long)capacity,
                                                                   static_cast<R*>(d_rec), d_cube);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    clv_set_global_error((std::string("clv_fo_find: ") + cudaGetErrorString(err)).c_str());
    return CLV_ECUDA;
  }
  return CLV_OK;
}

}  // namespace

extern "C" {

clv_status clv_fo_scratch_bytes(const clv_fo_grid* g, size_t* bytes) {
  const clv_status s = check_grid(g);
  if (s != CLV_OK) return s;
  if (!bytes) return bad("bytes is NULL");
  *bytes = scratch_layout(g).bytes;
  return CLV_OK;
}

clv_status clv_fo_find(const clv_fo_grid* g, const clv_fo_slice* s0, const clv_fo_slice* s1, double eps_f,
                       void* d_rec, int64_t* d_cube, int64_t capacity, int64_t* d_count, void* d_scratch,
                       void* cuda_stream) {
  const clv_status s = check_grid(g);
  if (s != CLV_OK) return s;
  if (!s0 || !s1) return bad("slice is NULL");
  if (!(s1->tau > s0->tau)) return bad("s1->tau must exceed s0->tau");
  if (!g->cartesian && !(s0->tau > 0)) return bad("tau must be > 0 in Milne coordinates");
  if (!(eps_f == eps_f)) return bad("eps_f is NaN");
  if (capacity < 0) return bad("capacity < 0");
  const size_t rs = g->precision == CLV_FP64 ? 8 : 4;
  if (capacity > 0 && (!d_rec || !aligned(d_rec, rs))) return bad("d_rec is NULL or misaligned");
  if (d_cube && !aligned(d_cube, 8)) return bad("d_cube is misaligned");
  if (!d_count || !aligned(d_count, 8)) return bad("d_count is NULL or misaligned");
  if (!d_scratch || !aligned(d_scratch, 16)) return bad("d_scratch is NULL or not 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return g->precision == CLV_FP64 ? fo_run<double>(g, s0, s1, eps_f, d_rec, d_cube, capacity, d_count, d_scratch, st)
                                  : fo_run<float>(g, s0, s1, eps_f, d_rec, d_cube, capacity, d_count, d_scratch, st);
}

}  // extern "C"
