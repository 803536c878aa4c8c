// clv_api.cu -- host implementation of the C ABI declared in include/clv.h.
// Owns the device layout, buffer rotation and kernel launches of the Heun
// step (two stage kernels per step); all arithmetic of the method runs in
// the kernels of clv_kernels.cuh.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "clv.h"
#include "clv_kernels.cuh"
#include "clv_tile.cuh"

using namespace clv;

// clv_charge.cu: the net-charge kernels
namespace clv {
template <typename R>
void launch_charge_stage(const StageParams<R>& p, int stage, const void* Nin, const void* Nn, void* Nout,
                         cudaStream_t st);
template <typename R>
void launch_charge_init(const double* n, const Prim<R>& pr, double taus, void* N, long long nc, int ne, int nep,
                        cudaStream_t st);
template <typename R>
void launch_charge_density(const void* N, const Prim<R>& pr, double taus, double* out, long long nc, int ne, int nep,
                           cudaStream_t st);
// clv_bulk.cu: the bulk-pressure kernel
template <typename R>
void launch_bulk_stage(const StageParams<R>& p, int stage, const void* Pin, const void* Pn, void* Pout,
                       double zeta_over_s, cudaStream_t st);
}  // namespace clv

namespace {

std::string g_create_error;

constexpr int kNumPrimSets = 3;
constexpr int kEosXkEntries = 254;   // frexp exponents -125..128 of positive normal floats
constexpr int kPrimFields = 6;  // e, ux, uy, ueta, P, cs

struct DevStats {
  double esum;
  double T_at_emax;
  unsigned long long emax_bits;
  unsigned long long counters[9];  // rescaled, root cap, polished, FP32 not converged, Newton iterations,
                                   // solved cells, FP64 refinement iterations, sum over warps of the
                                   // warp's largest iteration count, warps with a solve
  unsigned int err;
  unsigned int pad;
  unsigned long long fail_cell;  // first cell (+1) whose root solve hit the cap
  double fail_EM[2];
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct clv_handle {
  clv_config cfg;
  cudaStream_t stream = nullptr;
  bool own_ws = false;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  long long N = 0;                // cells of the padded layout (eta rows of pitch nep)
  long long Nc = 0;               // cells of the grid (compact order of the host arrays)
  int nep = 1;                    // eta pitch: neta rounded up to a multiple of 4
  int rsize = 8;
  bool viscous = false;
  int nblocks = 0;
  // device arrays (typed at use)
  void* T0[4];                    // T~ (FP32 path: high parts of the float-float pairs)
  void* PI0[10];
  void* T1[4];
  void* PI1[10];
  void* TL0[4] = {nullptr, nullptr, nullptr, nullptr};   // FP32 path: low parts of T~ (state)
  void* TL1[4] = {nullptr, nullptr, nullptr, nullptr};   // and of the stage-1 result
  void* PR[kNumPrimSets][kPrimFields];
  void* NC[2] = {nullptr, nullptr};   // charge = 1: N~^tau of the state and of the stage
  bool charge_on = false;             // clv_set_initial_n since the last initial state
  void* PB[2] = {nullptr, nullptr};   // zeta_over_s > 0: Pi of the state and of the stage
  int cur = 0, prev = 1;
  void* eos[3];
  void* mlp = nullptr;            // tensor-core copy of the guess network
  bool mlp_loaded = false;
  int guess = 0;                  // GuessMode
  double* staging = nullptr;      // N doubles
  double* block_sum = nullptr;    // nblocks doubles
  DevStats* dstats = nullptr;
  int sms = 148;                  // multiprocessors of the device
  double* tau_dev = nullptr;      // tau of the step on the device (the kernels read it)
  float* itau_dev = nullptr;      // 1/tau at the end of the step as a float-float pair (FP32 recovery)
  double tau = 0.0;               // host copy, advanced by the same additions
  long long step = 0;
  bool initialized = false;
  bool predictor_pending = false;   // x-slab: the first-step predictor is driven by clv_slab_predictor
  std::string last_error;
  // kernel timing (instrumentation)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<cudaEvent_t> ev_pending;  // five per step: around the four kernel launches
  double t_ms[4] = {0.0, 0.0, 0.0, 0.0};
  long long t_launches[4] = {0, 0, 0, 0};
  // tiled stage kernel geometry
  TileArgs tile{};
  int tile_threads = 0;
  unsigned tile_blocks = 0;
  size_t tile_smem = 0;
  int stat_blocks = 0;  // block partials written by the last stats launch
  // batch of events stored back to back (clv_create_batch; empty otherwise)
  struct Event {
    clv_config cfg;
    long long off = 0, N = 0, Nc = 0;   // padded offset and cells, compact cells
    int nep = 1;
    TileArgs tile{};
    bool viscous = false, set = false;
  };
  std::vector<Event> batch;
  // replay of captured step pairs (the primitive sets alternate with period 2)
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};   // two steps starting from cur = 0 / cur = 1
  void* batch_geom = nullptr;       // EventGeom<R>[events]
  TileArgs* batch_tiles = nullptr;  // TileArgs[events]
  int2* batch_items = nullptr;      // (event, tile-chunk), most expensive first
  int* batch_ctr = nullptr;         // work counters of the two stage launches
  int batch_nitems = 0, batch_threads = 0;
  unsigned batch_blocks = 0;
  size_t batch_smem = 0;
  int batch_maxthr = 0, batch_chunk = 0;   // tiling policy of the batch (thread cap per CTA, x chunk)
};

namespace {

clv_status fail(clv_handle* h, clv_status s, const std::string& msg) {
  if (h) h->last_error = msg; else g_create_error = msg;
  return s;
}

#define CLV_CUDA(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((h), CLV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

int device_sms(size_t* smem_optin) {
  int sms = 148, dev = 0, sm = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  if (smem_optin) *smem_optin = (size_t)sm;
  return sms;
}

clv_status validate(const clv_config* c) {
  if (!c) return fail(nullptr, CLV_EINVAL, "config is NULL");
  if (c->nx < 1 || c->ny < 1 || c->neta < 1) return fail(nullptr, CLV_EINVAL, "grid dims must be >= 1");
  if (!(c->dx > 0 && c->dy > 0 && c->deta > 0 && c->dtau > 0))
    return fail(nullptr, CLV_EINVAL, "spacings and dtau must be > 0");
  if (!c->cartesian && !(c->tau0 > 0)) return fail(nullptr, CLV_EINVAL, "tau0 must be > 0 in Milne coordinates");
  if (!(c->eta_over_s >= 0)) return fail(nullptr, CLV_EINVAL, "eta_over_s must be >= 0");
  if (c->precision != CLV_FP64 && c->precision != CLV_FP32) return fail(nullptr, CLV_EINVAL, "unknown precision");
  if (c->eos_kind == CLV_EOS_TABLE) {
    if (c->eos_n < 2 || !c->eos_P || !c->eos_T || !c->eos_cs2 || !(c->eos_dlne > 0))
      return fail(nullptr, CLV_EINVAL, "EOS table needs eos_n >= 2, eos_dlne > 0 and P, T, cs2 arrays");
  } else if (c->eos_kind != CLV_EOS_CONFORMAL) {
    return fail(nullptr, CLV_EINVAL, "unknown eos_kind");
  }
  if (!(c->eps_cut >= 0)) return fail(nullptr, CLV_EINVAL, "eps_cut must be >= 0");
  if (c->kernel != 0 && c->kernel != 1) return fail(nullptr, CLV_EINVAL, "unknown kernel variant");
  if (c->halo_x != 0 && c->halo_x != 2) return fail(nullptr, CLV_EINVAL, "halo_x must be 0 or 2");
  if (c->halo_x && (c->nx < 2 || c->kernel != 0)) return fail(nullptr, CLV_EINVAL, "an x-slab needs nx >= 2 and kernel 0");
  if (c->charge != 0 && c->charge != 1) return fail(nullptr, CLV_EINVAL, "charge must be 0 or 1");
  if (c->charge && c->halo_x) return fail(nullptr, CLV_EINVAL, "charge transport runs on single events, not x-slabs");
  if (!(c->zeta_over_s >= 0) || !std::isfinite(c->zeta_over_s))
    return fail(nullptr, CLV_EINVAL, "zeta_over_s must be finite and >= 0");
  if (c->zeta_over_s > 0 && !(c->eta_over_s > 0))
    return fail(nullptr, CLV_EINVAL, "bulk pressure (zeta_over_s > 0) needs eta_over_s > 0");
  if (c->zeta_over_s > 0 && c->halo_x)
    return fail(nullptr, CLV_EINVAL, "bulk pressure runs on single events, not x-slabs");
  if (!(c->taupi_coef >= 0) || !std::isfinite(c->lambda1_hat))
    return fail(nullptr, CLV_EINVAL, "taupi_coef must be >= 0 and lambda1_hat finite");
  long long N = (long long)c->nx * c->ny * c->neta;
  if (N > (1LL << 34)) return fail(nullptr, CLV_EINVAL, "grid too large");
  return CLV_OK;
}

// shared memory a block may opt in to on sm_100 / sm_103 (227 KiB)
constexpr size_t kSmemOptinMax = 232448;

struct TileGeom {
  TileArgs t;
  int threads;
  unsigned blocks;
  size_t smem;
};

// CTAs of a stage kernel resident on one SM at `threads` threads and `smem`
// bytes of dynamic shared memory, from the device's occupancy calculator
// (registers, shared memory and warps); 1 when it cannot tell.
int kernel_occupancy(const void* f, int threads, size_t smem) {
  int n = 0;
  if (smem > kSmemOptinMax) return 1;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemOptinMax) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();   // a failed query leaves no error behind
    return 1;
  }
  return std::max(1, n);
}

int tile_occupancy(const clv_config* c, int threads, size_t smem) {
  const bool visc = c->eta_over_s > 0.0;
  if (c->precision == CLV_FP64)
    return kernel_occupancy(visc ? (const void*)stage_tile_kernel<double, 2, true> : (const void*)stage_tile_kernel<double, 2, false>,
                            threads, smem);
  return kernel_occupancy(visc ? (const void*)stage_tile_kernel<float, 2, true> : (const void*)stage_tile_kernel<float, 2, false>,
                          threads, smem);
}

// x chunking of a tile grid: the number of chunks that minimises waves x
// (planes per chunk + the 4 halo planes each chunk also stages), with `slots`
// CTAs resident on the device at a time
int chunk_planes(int nx, long long tiles, long long slots) {
  long long best_nch = 1;
  double best = 1e300;
  for (long long nch = 1; nch <= std::min<long long>(nx, 8LL * slots); ++nch) {
    const long long cx = (nx + nch - 1) / nch;
    const long long used = (nx + cx - 1) / cx;
    const long long waves = (tiles * used + slots - 1) / slots;
    const double cost = (double)waves * (double)(cx + 4);
    if (cost < best - 1e-9) { best = cost; best_nch = used; }
  }
  return (int)((nx + best_nch - 1) / best_nch);
}

TileGeom tile_geometry_of(const clv_config* c, int sms, int TJ, int TK, int cx);

// Tile shape: TK columns fit neta in ceil(neta/32) tiles; the block has
// (TJ+1) x (TK+1) threads, at most CLV_TILE_MAX_THREADS (FP32) or 128 (FP64),
// and fewer rows while its shared memory exceeds the opt-in limit of a block;
// x is cut into chunks of CX planes by the makespan rule of chunk_planes.
TileGeom tile_geometry(const clv_config* c, int sms) {
  const int rsize = c->precision == CLV_FP64 ? 8 : 4;
  const int maxthr = rsize == 4 ? CLV_TILE_MAX_THREADS : std::min(CLV_TILE_MAX_THREADS, kBlock / 2);
  const int nk = (c->neta + 31) / 32;
  const int TK = (c->neta + nk - 1) / nk;
  const bool visc = c->eta_over_s > 0.0;
  int TJ = std::max(1, std::min(c->ny, maxthr / (TK + 1) - 1));
  auto smem_of = [&](int tj) {
    return visc ? tile_smem_bytes<true>(tj, TK, rsize) : tile_smem_bytes<false>(tj, TK, rsize);
  };
  while (TJ > 1 && smem_of(TJ) > kSmemOptinMax) --TJ;
  return tile_geometry_of(c, sms, TJ, TK, 0);
}

// Geometry of an explicit (TJ, TK) tile shape; CX from the makespan rule of
// chunk_planes when cx <= 0, with as many CTAs per SM as the device keeps
// resident at this shape.
TileGeom tile_geometry_of(const clv_config* c, int sms, int TJ, int TK, int cx) {
  const int rsize = c->precision == CLV_FP64 ? 8 : 4;
  TileGeom g;
  TileArgs& t = g.t;
  t.TJ = TJ;
  t.TK = TK;
  t.ntj = (c->ny + TJ - 1) / TJ;
  t.ntk = (c->neta + TK - 1) / TK;
  const bool visc = c->eta_over_s > 0.0;
  g.threads = (TJ + 1) * (TK + 1);
  g.smem = visc ? tile_smem_bytes<true>(TJ, TK, rsize) : tile_smem_bytes<false>(TJ, TK, rsize);
  const long long tiles = (long long)t.ntj * t.ntk;
  if (cx <= 0) cx = chunk_planes(c->nx, tiles, (long long)sms * tile_occupancy(c, g.threads, g.smem));
  t.CX = cx;
  const long long nch = (c->nx + t.CX - 1) / t.CX;
  g.blocks = (unsigned)(tiles * nch);
  return g;
}

inline int tile_max_threads(const clv_config* c) {
  return c->precision == CLV_FP64 ? std::min(CLV_TILE_MAX_THREADS, kBlock / 2) : CLV_TILE_MAX_THREADS;
}

// Candidate tile shapes for the autotuner, best modelled makespan first:
// eta_s split into 1..4 columns of tiles, y tiles from the largest that fits
// the thread limit down to a third of it, the x chunking of each by the
// makespan rule.  Model: waves x (planes + 4 halo planes) x staged box cells
// x CTAs sharing an SM, over the SM's issue efficiency (resident warps, up to
// 16, over 16).
std::vector<TileGeom> tile_candidates(const clv_config* c, int sms, size_t smem_max) {
  std::vector<std::pair<double, TileGeom>> v;
  const int maxthr = tile_max_threads(c);
  int last_tk = -1;
  for (int nk = 1; nk <= 4; ++nk) {
    const int TK = (c->neta + nk - 1) / nk;
    if (TK == last_tk || TK < 1) continue;
    last_tk = TK;
    const int maxTJ = std::min(c->ny, maxthr / (TK + 1) - 1);
    if (maxTJ < 1) continue;
    for (int TJ = maxTJ; TJ >= std::max(1, maxTJ / 3); --TJ) {
      TileGeom g = tile_geometry_of(c, sms, TJ, TK, 0);
      if (g.smem > smem_max) continue;
      const int occ = tile_occupancy(c, g.threads, g.smem);
      const long long slots = (long long)sms * occ;
      const long long waves = ((long long)g.blocks + slots - 1) / slots;
      const double eff = std::min(1.0, occ * ((g.threads + 31) / 32) / 16.0);
      const double cost = (double)waves * (g.t.CX + 4) * (double)((TJ + 4) * (TK + 4)) * occ / eff;
      v.push_back({cost, g});
    }
  }
  std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<TileGeom> out;
  for (auto& x : v) out.push_back(x.second);
  return out;
}

inline int eta_pitch(int neta) { return (neta + 3) & ~3; }

size_t layout(const clv_config* c, clv_handle* h) {
  // eta rows are padded to a multiple of 4 cells (16-byte aligned rows for
  // vector copies); the padding slots hold vacuum and are never updated
  const int nep = eta_pitch(c->neta);
  const long long N = (long long)c->nx * c->ny * nep;
  const size_t rs = c->precision == CLV_FP64 ? 8 : 4;
  // per-cell fields hold halo_x extra planes on each x side (an x-slab); the
  // field pointers below point at plane 0, so [0, N) is the interior
  const size_t hoff = (size_t)c->halo_x * c->ny * nep * rs;
  const size_t fb = align_up((size_t)N * rs + 2 * hoff, 256);
  // FP32 path: T~ as float-float pairs (StageParams), the low parts in 2 x 4 more arrays
  const bool ffT = c->precision != CLV_FP64;
  // block partials of the stats reduction: enough for the direct grid and for
  // the tiled grid on any device (at most 1024 SMs)
  const int nblocks = (int)std::max<long long>((N + kBlock - 1) / kBlock, tile_geometry(c, 1024).blocks);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes, 256); return o; };
  size_t oT0[4], oPI0[10], oT1[4], oPI1[10], oPR[kNumPrimSets][kPrimFields], oE[3];
  for (int m = 0; m < 4; ++m) oT0[m] = take(fb);
  for (int q = 0; q < 10; ++q) oPI0[q] = take(fb);
  for (int m = 0; m < 4; ++m) oT1[m] = take(fb);
  for (int q = 0; q < 10; ++q) oPI1[q] = take(fb);
  for (int s = 0; s < kNumPrimSets; ++s)
    for (int f = 0; f < kPrimFields; ++f) oPR[s][f] = take(fb);
  size_t oTL0[4] = {0, 0, 0, 0}, oTL1[4] = {0, 0, 0, 0};
  if (ffT)
    for (int m = 0; m < 4; ++m) { oTL0[m] = take(fb); oTL1[m] = take(fb); }
  size_t oNC[2] = {0, 0}, oPB[2] = {0, 0};
  if (c->charge)
    for (int t = 0; t < 2; ++t) oNC[t] = take(fb);
  const bool bulk = c->zeta_over_s > 0;
  if (bulk)
    for (int t = 0; t < 2; ++t) oPB[t] = take(fb);
  const int ne = c->eos_kind == CLV_EOS_TABLE ? c->eos_n : 1;
  oE[0] = take((size_t)4 * ne * rs + kEosXkEntries * sizeof(float2));  // nodes packed as (P, T, c_s^2, Plo), then xk
  oE[1] = oE[2] = oE[0];
  size_t oMlp = take(kMlpDeviceBytes);
  size_t oStage = take(std::max((size_t)N * 8, (size_t)256));  // also scratch of clv_mlp_samples
  size_t oBlock = take((size_t)nblocks * 8);
  size_t oStats = take(sizeof(DevStats));
  size_t oTau = take(4 * sizeof(double));   // tau (double), then 1/tau as two floats
  if (h) {
    char* b = h->ws;
    for (int m = 0; m < 4; ++m) { h->T0[m] = b + oT0[m] + hoff; h->T1[m] = b + oT1[m] + hoff; }
    for (int m = 0; m < 4; ++m) {
      h->TL0[m] = ffT ? b + oTL0[m] + hoff : nullptr;
      h->TL1[m] = ffT ? b + oTL1[m] + hoff : nullptr;
    }
    for (int q = 0; q < 10; ++q) { h->PI0[q] = b + oPI0[q] + hoff; h->PI1[q] = b + oPI1[q] + hoff; }
    for (int s = 0; s < kNumPrimSets; ++s)
      for (int f = 0; f < kPrimFields; ++f) h->PR[s][f] = b + oPR[s][f] + hoff;
    for (int t = 0; t < 2; ++t) h->NC[t] = c->charge ? b + oNC[t] + hoff : nullptr;
    for (int t = 0; t < 2; ++t) h->PB[t] = bulk ? b + oPB[t] + hoff : nullptr;
    for (int t = 0; t < 3; ++t) h->eos[t] = b + oE[t];
    h->mlp = b + oMlp;
    h->staging = (double*)(b + oStage);
    h->block_sum = (double*)(b + oBlock);
    h->dstats = (DevStats*)(b + oStats);
    h->tau_dev = (double*)(b + oTau);
    h->itau_dev = (float*)(b + oTau + 2 * sizeof(double));
    h->nblocks = nblocks;
    h->N = N;
    h->Nc = (long long)c->nx * c->ny * c->neta;
    h->nep = nep;
    h->rsize = (int)rs;
  }
  return off;
}

// four T~ arrays (or their low parts; nullptr stays nullptr) as a Ptr10
template <typename R> Ptr10<R> t_arrays(void* const a[4]) {
  Ptr10<R> t{};
  for (int m = 0; m < 4; ++m) t.p[m] = (R*)a[m];
  return t;
}

template <typename R> Prim<R> prim_set(clv_handle* h, int s) {
  Prim<R> p;
  p.e = (R*)h->PR[s][0];
  for (int m = 0; m < 3; ++m) p.u[m] = (R*)h->PR[s][1 + m];
  p.P = (R*)h->PR[s][4];
  p.cs = (R*)h->PR[s][5];
  return p;
}

template <typename R> EosView<R> eos_view(const clv_handle* h) {
  const clv_config& c = h->cfg;
  EosView<R> v;
  v.kind = c.eos_kind;
  v.n = c.eos_kind == CLV_EOS_TABLE ? c.eos_n : 1;
  v.lne0 = (R)c.eos_lne0;
  v.inv_dlne = (R)(c.eos_kind == CLV_EOS_TABLE ? 1.0 / c.eos_dlne : 0.0);
  v.e0 = (R)std::exp(c.eos_lne0);
  v.e_top = (R)std::exp(c.eos_lne0 + (v.n - 1) * c.eos_dlne);
  v.top = (R)(v.n - 1);
  const double pi = 3.14159265358979323846;
  v.t_coef = (R)(30.0 * kHbarC * kHbarC * kHbarC / (kDofConformal * pi * pi));
  v.node = (const R*)h->eos[0];
  v.xk = (const float2*)((const char*)h->eos[0] + (size_t)4 * v.n * sizeof(R));
  return v;
}

inline unsigned grid_of(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }

template <typename R> IsCoef<R> is_coef(const clv_config& c) {
  const double b = c.taupi_coef > 0 ? c.taupi_coef : 5.0;
  return IsCoef<R>{(R)(c.eta_over_s > 0 ? 1.0 / (b * c.eta_over_s * kHbarC) : 0.0), (R)(1.0 / b), (R)c.lambda1_hat};
}

template <typename R>
StageParams<R> stage_params(clv_handle* h, int stage) {
  const clv_config& c = h->cfg;
  StageParams<R> p;
  const int st = 3 - h->cur - h->prev;
  const Prim<R> pcur = prim_set<R>(h, h->cur), pprev = prim_set<R>(h, h->prev), pst = prim_set<R>(h, st);
  const bool s1 = stage == 1;
  for (int m = 0; m < 4; ++m) {
    p.T[m] = (const R*)(s1 ? h->T0[m] : h->T1[m]);
    p.Tn[m] = (const R*)h->T0[m];
    p.Tout[m] = (R*)(s1 ? h->T1[m] : h->T0[m]);
    p.Tl[m] = (const R*)(s1 ? h->TL0[m] : h->TL1[m]);
    p.Tnl[m] = (const R*)h->TL0[m];
    p.Toutl[m] = (R*)(s1 ? h->TL1[m] : h->TL0[m]);
  }
  for (int q = 0; q < 10; ++q) {
    p.pi[q] = (const R*)(s1 ? h->PI0[q] : h->PI1[q]);
    p.pin[q] = (const R*)h->PI0[q];
    p.piout[q] = (R*)(s1 ? h->PI1[q] : h->PI0[q]);
  }
  p.pr = s1 ? pcur : pst;
  for (int m = 0; m < 3; ++m) { p.un[m] = pcur.u[m]; p.up[m] = pprev.u[m]; }
  p.prout = s1 ? pst : pprev;
  p.eos = eos_view<R>(h);
  p.nx = c.nx; p.ny = c.ny; p.ne = c.neta; p.periodic = c.periodic;
  p.nep = h->nep;
  p.xhalo = c.halo_x > 0 ? 1 : 0;
  p.N = h->N;
  p.tau_dev = h->tau_dev;
  p.itau = h->itau_dev;
  p.dtau_d = c.dtau;
  p.cartesian = c.cartesian;
  p.h = (R)c.dtau;
  p.inv_h = (R)(1.0 / c.dtau);
  p.inv_dl[0] = (R)(1.0 / c.dx);
  p.inv_dl[1] = (R)(1.0 / c.dy);
  p.st_tau = (R)(c.cartesian ? 0.0 : 1.0);
  p.eps_cut = (R)c.eps_cut;
  p.eps_cut_d = c.eps_cut;
  p.deta_d = c.deta;
  p.is = is_coef<R>(c);
  p.polish_E = (R)(1.01 * c.eps_cut);
  p.polish_v = (R)0.99;   // gamma above ~7: E/eps > ~65, the FP32 eps = E - M v loses digits
  p.block_sum = h->block_sum;
  p.emax_bits = &h->dstats->emax_bits;
  p.counters = h->dstats->counters;
  p.err = &h->dstats->err;
  p.fail_cell = &h->dstats->fail_cell;
  p.fail_EM = h->dstats->fail_EM;
  p.mlp = h->mlp;
  p.Pib = nullptr;   // set by launch_half for viscous stages with bulk pressure
  return p;
}

constexpr size_t kMaxTimedSteps = 8192;
constexpr size_t kEventsPerStep = 5;

cudaEvent_t timing_event(clv_handle* h) {
  cudaEvent_t e = nullptr;
  if (!h->ev_pool.empty()) {
    e = h->ev_pool.back();
    h->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(e, h->stream);
  h->ev_pending.push_back(e);
  return e;
}

void choose_tile(clv_handle* h) {
  int sms = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TileGeom g = tile_geometry(&h->cfg, sms);
  h->tile = g.t;
  h->tile_threads = g.threads;
  h->tile_blocks = g.blocks;
  h->tile_smem = g.smem;
}

template <typename R, bool VISC> cudaError_t tile_attributes(size_t smem) {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  };
  set((const void*)stage_tile_kernel<R, 1, VISC>);
  set((const void*)stage_tile_kernel<R, 2, VISC>);
  return e;
}

template <typename R, bool VISC, bool STATS> void launch_recover(clv_handle* h, const StageParams<R>& p) {
  const unsigned g = grid_of(h->N);
  if (sizeof(R) == 4 && h->guess == kGuessMlp)
    recover_kernel<R, VISC, STATS, sizeof(R) == 4 ? kGuessMlp : kGuessPrevious><<<g, kBlock, 0, h->stream>>>(p);
  else if (sizeof(R) == 4 && h->guess == kGuessMlpAll)
    recover_kernel<R, VISC, STATS, sizeof(R) == 4 ? kGuessMlpAll : kGuessPrevious><<<g, kBlock, 0, h->stream>>>(p);
  else if (h->guess == kGuessCold) recover_kernel<R, VISC, STATS, kGuessCold><<<g, kBlock, 0, h->stream>>>(p);
  else recover_kernel<R, VISC, STATS, kGuessPrevious><<<g, kBlock, 0, h->stream>>>(p);
}

// One stage: the stage kernel, then the root solve (the direct kernel does
// both).  With timing on, an event follows each of the two.
template <typename R, bool VISC, int STAGE, bool STATS>
void launch_stage(clv_handle* h, const StageParams<R>& p, bool timed) {
  if (!h->batch.empty()) {
    cudaMemsetAsync(h->batch_ctr + (STAGE - 1), 0, sizeof(int), h->stream);
    stage_batch_kernel<R, STAGE, VISC><<<h->batch_blocks, h->batch_threads, h->batch_smem, h->stream>>>(
        p, (const EventGeom<R>*)h->batch_geom, h->batch_tiles, h->batch_items, h->batch_nitems,
        h->batch_ctr + (STAGE - 1));
    if (timed) timing_event(h);
    launch_recover<R, VISC, STATS>(h, p);
  } else if (h->cfg.kernel == 1) {
    stage_kernel<R, STAGE, VISC, STATS><<<grid_of(h->N), kBlock, 0, h->stream>>>(p);
    if (timed) timing_event(h);   // empty recovery slot
  } else {
    stage_tile_kernel<R, STAGE, VISC><<<h->tile_blocks, h->tile_threads, h->tile_smem, h->stream>>>(p, h->tile);
    if (timed) timing_event(h);
    launch_recover<R, VISC, STATS>(h, p);
  }
  if (timed) timing_event(h);
}

// tau of the step, and 1/tau of the end of the step (tau + dtau; 1 in
// Cartesian mode) as a float-float pair for the FP32 recovery
__device__ __forceinline__ void store_itau(float* itau, double tau, double dtau, int cartesian) {
  const double x = cartesian ? 1.0 : 1.0 / (tau + dtau);
  const float hi = (float)x;
  itau[0] = hi;
  itau[1] = (float)(x - (double)hi);
}
__global__ void set_tau_kernel(double* tau_dev, float* itau, double tau, double dtau, int cartesian) {
  *tau_dev = tau;
  store_itau(itau, tau, dtau, cartesian);
}
__global__ void advance_tau_kernel(double* tau_dev, float* itau, double dtau, int cartesian) {
  const double t = *tau_dev + dtau;
  *tau_dev = t;
  store_itau(itau, t, dtau, cartesian);
}

void set_tau(clv_handle* h, double tau) {
  h->tau = tau;
  set_tau_kernel<<<1, 1, 0, h->stream>>>(h->tau_dev, h->itau_dev, tau, h->cfg.dtau, h->cfg.cartesian);
}

// Half of a Heun step: stage 1, or stage 2 with the end-of-step bookkeeping
// (tau advance, rotation of the primitive sets).
template <typename R, bool VISC>
void launch_half(clv_handle* h, int stage, bool stats, bool timed) {
  if (stage == 1) {
    StageParams<R> p1 = stage_params<R>(h, 1);
    if (VISC && h->PB[0]) {   // bulk: Pi' from Pi^n before the stage (its root solve adds Pi' to P)
      p1.Pib = (R*)h->PB[1];
      launch_bulk_stage<R>(p1, 1, h->PB[0], h->PB[0], h->PB[1], h->cfg.zeta_over_s, h->stream);
    }
    launch_stage<R, VISC, 1, false>(h, p1, timed);
    // net charge: stage 1 from N^n into the stage buffer, with the stage's input velocities
    if (h->charge_on) launch_charge_stage<R>(p1, 1, h->NC[0], h->NC[0], h->NC[1], h->stream);
    return;
  }
  StageParams<R> p2 = stage_params<R>(h, 2);
  if (VISC && h->PB[0]) {   // bulk: Pi^{n+1} from Pi' and Pi^n, in place over Pi^n
    p2.Pib = (R*)h->PB[0];
    launch_bulk_stage<R>(p2, 2, h->PB[1], h->PB[0], h->PB[0], h->cfg.zeta_over_s, h->stream);
  }
  if (stats) {
    launch_stage<R, VISC, 2, true>(h, p2, timed);
    h->stat_blocks = (int)grid_of(h->N);
  } else {
    launch_stage<R, VISC, 2, false>(h, p2, timed);
  }
  if (h->charge_on) launch_charge_stage<R>(p2, 2, h->NC[1], h->NC[0], h->NC[0], h->stream);
  advance_tau_kernel<<<1, 1, 0, h->stream>>>(h->tau_dev, h->itau_dev, h->cfg.dtau, h->cfg.cartesian);
  std::swap(h->cur, h->prev);
  h->tau = h->tau + h->cfg.dtau;
  h->step += 1;
}

template <typename R, bool VISC>
void launch_step(clv_handle* h, bool stats) {
  // events: [0] stage-1 kernel [1] stage-1 recovery [2] stage-2 kernel [3] stage-2 recovery [4]
  // (with kernel = 1 the recovery slots collapse: two events are recorded back to back)
  const bool timed = h->timing && h->ev_pending.size() < kEventsPerStep * kMaxTimedSteps;
  if (timed) timing_event(h);
  launch_half<R, VISC>(h, 1, false, timed);
  launch_half<R, VISC>(h, 2, stats, timed);
}

void invalidate_graphs(clv_handle* h) {
  for (auto& g : h->step_graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

void launch_one_step(clv_handle* h, bool stats) {
  if (h->rsize == 8) {
    if (h->viscous) launch_step<double, true>(h, stats); else launch_step<double, false>(h, stats);
  } else {
    if (h->viscous) launch_step<float, true>(h, stats); else launch_step<float, false>(h, stats);
  }
}

// The executable graph of two plain steps from the current buffer parity,
// captured once on a private stream (capture issues no work) and replayed on
// the handle's stream.  nullptr (and graphs off for the handle) if capture is
// not possible.
cudaGraphExec_t step_pair_graph(clv_handle* h) {
  const int key = h->cur;
  if (h->step_graph[key]) return h->step_graph[key];
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->graphs = false;
    return nullptr;
  }
  const cudaStream_t user = h->stream;
  const double tau = h->tau;
  const long long step = h->step;
  const int cur = h->cur, prev = h->prev;
  h->stream = h->cap_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    launch_one_step(h, false);
    launch_one_step(h, false);
    e = cudaStreamEndCapture(h->cap_stream, &graph);
  }
  h->stream = user;
  h->tau = tau;
  h->step = step;
  h->cur = cur;
  h->prev = prev;
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->graphs = false;
    return nullptr;
  }
  h->step_graph[key] = ex;
  return ex;
}

// T0l: the low parts of the float-float T~ (FP32 path) or nullptr
template <typename R> __global__ void stats_scan_kernel(const R* e, const R* T0, const R* T0l, long long N,
                                                        double* block_sum, unsigned long long* emax_bits) {
  __shared__ double s_sum[kBlock / 32], s_max[kBlock / 32];
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0;
  if (c < N) { a = (double)T0[c] + (T0l ? (double)T0l[c] : 0.0); b = (double)e[c]; }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) { s_sum[threadIdx.x >> 5] = a; s_max[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) { x += s_sum[w]; y = fmax(y, s_max[w]); }
    block_sum[blockIdx.x] = x;
    if (y > 0.0) atomicMax(emax_bits, (unsigned long long)__double_as_longlong(y));
  }
}

template <typename R> __global__ void finalize_stats_kernel(DevStats* ds, EosView<R> eos) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const R e = (R)__longlong_as_double((long long)ds->emax_bits);
    R P, T, c2;
    eos_eval<R, R>(eos, e, P, T, c2);
    ds->T_at_emax = (double)T;
  }
}

template <typename R> clv_status reduce_stats(clv_handle* h, bool scan, clv_stats* out) {
  // the fused stage-2 launch (scan == false) already wrote block_sum and emax
  if (scan) {
    CLV_CUDA(h, cudaMemsetAsync(&h->dstats->emax_bits, 0, sizeof(unsigned long long), h->stream));
    stats_scan_kernel<R><<<grid_of(h->N), kBlock, 0, h->stream>>>(
        (const R*)h->PR[h->cur][0], (const R*)h->T0[0], (const R*)h->TL0[0], h->N, h->block_sum,
        &h->dstats->emax_bits);
    h->stat_blocks = (int)grid_of(h->N);
  }
  finalize_sum_kernel<<<1, 1024, 0, h->stream>>>(h->block_sum, h->stat_blocks, &h->dstats->esum);
  finalize_stats_kernel<R><<<1, 32, 0, h->stream>>>(h->dstats, eos_view<R>(h));
  CLV_CUDA(h, cudaGetLastError());
  DevStats ds;
  CLV_CUDA(h, cudaMemcpyAsync(&ds, h->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream));
  CLV_CUDA(h, cudaStreamSynchronize(h->stream));
  const clv_config& c = h->cfg;
  out->tau = h->tau;
  out->step = h->step;
  std::memcpy(&out->eps_max, &ds.emax_bits, sizeof(double));
  out->T_max = ds.T_at_emax;
  out->E_tot = h->batch.empty() ? ds.esum * c.dx * c.dy * c.deta : 0.0;  // batch: per event (clv_batch_event_stats)
  out->n_rescaled = (int64_t)ds.counters[0];
  out->n_rootfail = (int64_t)ds.counters[1];
  out->n_polished = (int64_t)ds.counters[2];
  out->n_fp32_nonconverged = (int64_t)ds.counters[3];
  out->n_newton_iters = (int64_t)ds.counters[4];
  out->n_newton_cells = (int64_t)ds.counters[5];
  out->n_polish_iters = (int64_t)ds.counters[6];
  out->n_newton_warp_max = (int64_t)ds.counters[7];
  out->n_newton_warps = (int64_t)ds.counters[8];
  out->error_word = ds.err;
  out->_pad = 0;
  if (ds.err & 2u) return fail(h, CLV_ENONFINITE, "non-finite value in the state");
  if (ds.err & 1u) {
    char msg[256];
    const long long cell = (long long)ds.fail_cell - 1;
    std::snprintf(msg, sizeof msg,
                  "primitive root solve hit its iteration cap (%lld cells; first: cell %lld, E=%.17g, |M|=%.17g)",
                  (long long)ds.counters[1], cell, ds.fail_EM[0], ds.fail_EM[1]);
    return fail(h, CLV_EROOT, msg);
  }
  if (ds.err & 4u) return fail(h, CLV_ETIMEOUT, "a bounded device wait gave up");
  return CLV_OK;
}

// compact doubles -> the padded layout in R
template <typename R> __global__ void convert_kernel(const double* s, R* d, long long N, int ne, int nep) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) d[padded_index(c, ne, nep)] = (R)s[c];
}

template <typename R> Prim<R> prim_at(Prim<R> p, long long off) {
  p.e += off;
  for (int m = 0; m < 3; ++m) p.u[m] += off;
  p.P += off;
  p.cs += off;
  return p;
}

// Primitives (and pi~) of one grid from compact doubles (host arrays go
// through the staging buffer): nc = nx ny neta input cells, stored at
// padded slots [off, off + npad) with eta pitch nep (padding slots: vacuum);
// vacuum below the cutoff, P and c_s from the EOS, copied to the
// previous-step set.
template <typename R>
clv_status load_initial_range(clv_handle* h, long long off, long long npad, long long nc, int ne, int nep, bool visc,
                              const double* const in[4], const double* pi, bool host) {
  const unsigned gc = grid_of(nc), gp = grid_of(npad);
  const clv_config& c = h->cfg;
  Prim<R> pc = prim_at(prim_set<R>(h, h->cur), off), pp = prim_at(prim_set<R>(h, h->prev), off);
  R* dst_prim[4] = {pc.e, pc.u[0], pc.u[1], pc.u[2]};
  for (int f = 0; f < 4; ++f) {
    const double* src = in[f];
    if (host) {
      CLV_CUDA(h, cudaMemcpyAsync(h->staging, src, (size_t)nc * 8, cudaMemcpyHostToDevice, h->stream));
      src = h->staging;
    }
    if (nep != ne) CLV_CUDA(h, cudaMemsetAsync(dst_prim[f], 0, (size_t)npad * sizeof(R), h->stream));
    convert_kernel<R><<<gc, kBlock, 0, h->stream>>>(src, dst_prim[f], nc, ne, nep);
  }
  Ptr10<R> pi0;
  for (int q = 0; q < 10; ++q) pi0.p[q] = (R*)h->PI0[q] + off;
  for (int q = 0; q < 10; ++q) {
    CLV_CUDA(h, cudaMemsetAsync(pi0.p[q], 0, (size_t)npad * sizeof(R), h->stream));
    if (pi && visc) {
      const double* src = pi + (size_t)q * nc;
      if (host) {
        CLV_CUDA(h, cudaMemcpyAsync(h->staging, src, (size_t)nc * 8, cudaMemcpyHostToDevice, h->stream));
        src = h->staging;
      }
      convert_kernel<R><<<gc, kBlock, 0, h->stream>>>(src, pi0.p[q], nc, ne, nep);
    }
  }
  init_primitives_kernel<R><<<gp, kBlock, 0, h->stream>>>(pc, pp, pi0, visc, eos_view<R>(h), c.eps_cut, npad);
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

// The rest of the initial state, over all cells: tau reset and T~ from the
// primitives -- the ideal T~ that the first-step predictor of Sec. 3 starts
// from in viscous runs (initial_end completes those after the predictor).
template <typename R> clv_status initial_begin(clv_handle* h) {
  const long long N = h->N;
  const unsigned g = grid_of(N);
  const clv_config& c = h->cfg;
  Prim<R> pc = prim_set<R>(h, h->cur);
  Ptr10<R> pi0;
  for (int q = 0; q < 10; ++q) pi0.p[q] = (R*)h->PI0[q];
  if (!h->batch.empty())   // ideal events of a batch keep pi~ = 0 in the stage buffers too
    for (int q = 0; q < 10; ++q) CLV_CUDA(h, cudaMemsetAsync(h->PI1[q], 0, (size_t)N * sizeof(R), h->stream));
  const double taus0 = c.cartesian ? 1.0 : c.tau0;
  set_tau(h, c.tau0);
  h->step = 0;
  tilde_T_kernel<R><<<g, kBlock, 0, h->stream>>>(pc, pi0, false, t_arrays<R>(h->T0), t_arrays<R>(h->TL0),
                                                 h->TL0[0] != nullptr, taus0, N);
  if (!h->viscous) {
    CLV_CUDA(h, cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream));
    h->initialized = true;
  }
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

// After the first-step predictor (one pi-free Heun step, Sec. 3): u~^{-1} =
// 2 u~^0 - u~^1_ideal, tau and T~ (now with pi~) of the initial state again.
template <typename R> clv_status initial_end(clv_handle* h) {
  const long long N = h->N;
  const unsigned g = grid_of(N);
  const clv_config& c = h->cfg;
  Ptr10<R> pi0;
  for (int q = 0; q < 10; ++q) pi0.p[q] = (R*)h->PI0[q];
  std::swap(h->cur, h->prev);  // undo the rotation: cur = u^0, prev = u^1_ideal
  extrapolate_prev_kernel<R><<<g, kBlock, 0, h->stream>>>(prim_set<R>(h, h->cur), prim_set<R>(h, h->prev), N);
  set_tau(h, c.tau0);
  h->step = 0;
  tilde_T_kernel<R><<<g, kBlock, 0, h->stream>>>(prim_set<R>(h, h->cur), pi0, true, t_arrays<R>(h->T0),
                                                 t_arrays<R>(h->TL0), h->TL0[0] != nullptr,
                                                 c.cartesian ? 1.0 : c.tau0, N);
  CLV_CUDA(h, cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream));
  CLV_CUDA(h, cudaGetLastError());
  h->predictor_pending = false;
  h->initialized = true;
  return CLV_OK;
}

template <typename R> clv_status finish_initial(clv_handle* h) {
  if (h->cfg.charge) {   // a new initial state carries no charge until clv_set_initial_n
    if (h->charge_on) invalidate_graphs(h);
    h->charge_on = false;
    for (int t = 0; t < 2; ++t)
      CLV_CUDA(h, cudaMemsetAsync(h->NC[t], 0, (size_t)h->N * h->rsize, h->stream));
  }
  if (h->PB[0])   // Pi = 0 at tau0
    for (int t = 0; t < 2; ++t)
      CLV_CUDA(h, cudaMemsetAsync(h->PB[t], 0, (size_t)h->N * h->rsize, h->stream));
  clv_status s = initial_begin<R>(h);
  if (s != CLV_OK || !h->viscous) return s;
  if (h->cfg.halo_x) {   // an x-slab: the caller drives the predictor with halo exchanges
    h->predictor_pending = true;
    return CLV_OK;
  }
  launch_half<R, false>(h, 1, false, false);
  launch_half<R, false>(h, 2, false, false);
  return initial_end<R>(h);
}

template <typename R>
clv_status set_initial_impl(clv_handle* h, const double* const in[4], const double* pi, bool host) {
  clv_status s = load_initial_range<R>(h, 0, h->N, h->Nc, h->cfg.neta, h->nep, h->viscous, in, pi, host);
  return s != CLV_OK ? s : finish_initial<R>(h);
}

// field `which` of the grid at padded offset off (n compact cells, eta rows
// ne of pitch nep) as compact doubles
template <typename R>
clv_status export_field(clv_handle* h, int which, double* dst, long long off, long long n, int ne, int nep) {
  if (which == 22) {   // n = N~^tau / (tau u~^tau)
    launch_charge_density<R>(h->NC[0], prim_set<R>(h, h->cur), h->cfg.cartesian ? 1.0 : h->tau, dst, n, ne, nep,
                             h->stream);
    CLV_CUDA(h, cudaGetLastError());
    return CLV_OK;
  }
  const void* src = nullptr;
  if (which <= 3) src = h->PR[h->cur][which];
  else if (which <= 7) src = h->T0[which - 4];
  else if (which <= 17) src = h->PI0[which - 8];
  else if (which <= 20) src = h->PR[h->prev][1 + (which - 18)];
  else if (which == 23) src = h->PB[0];
  else src = h->NC[0];
  if (which >= 4 && which <= 7 && h->TL0[0])   // FP32 path: T~ = high + low parts
    export_pair_kernel<R><<<grid_of(n), kBlock, 0, h->stream>>>((const R*)src + off,
                                                                (const R*)h->TL0[which - 4] + off, dst, n, ne, nep);
  else
    export_kernel<R><<<grid_of(n), kBlock, 0, h->stream>>>((const R*)src + off, dst, n, ne, nep);
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

clv_status create_common(const clv_config* cfg, void* stream, void* ws, size_t ws_bytes, clv_handle** out) {
  if (!out) return fail(nullptr, CLV_EINVAL, "out is NULL");
  *out = nullptr;
  clv_status s = validate(cfg);
  if (s != CLV_OK) return s;
  clv_handle* h = new clv_handle();
  h->cfg = *cfg;
  h->cfg.eos_P = h->cfg.eos_T = h->cfg.eos_cs2 = nullptr;
  h->stream = (cudaStream_t)stream;
  h->viscous = cfg->eta_over_s > 0.0;
  const size_t need = layout(cfg, nullptr);
  if (ws) {
    if (ws_bytes < need || ((uintptr_t)ws & 255u)) {
      delete h;
      return fail(nullptr, CLV_ENOMEM, "workspace too small or not 256-byte aligned");
    }
    h->ws = (char*)ws;
    h->own_ws = false;
  } else {
    cudaError_t e = cudaMalloc((void**)&h->ws, need);
    if (e != cudaSuccess) {
      delete h;
      return fail(nullptr, CLV_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->own_ws = true;
  }
  h->ws_bytes = need;
  layout(cfg, h);
  {
    // padding slots of the eta rows (and every field before its first use) hold zeros: vacuum
    cudaError_t e = cudaMemsetAsync(h->ws, 0, need, h->stream);
    if (e != cudaSuccess) {
      if (h->own_ws) cudaFree(h->ws);
      delete h;
      return fail(nullptr, CLV_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    }
  }
  h->sms = device_sms(nullptr);
  h->tau = cfg->tau0;
  choose_tile(h);
  {
    // the ideal first step of viscous runs uses the ideal tile kernels with the viscous tile shape
    cudaError_t e = h->rsize == 8 ? tile_attributes<double, false>(h->tile_smem) : tile_attributes<float, false>(h->tile_smem);
    if (e == cudaSuccess && h->viscous)
      e = h->rsize == 8 ? tile_attributes<double, true>(h->tile_smem) : tile_attributes<float, true>(h->tile_smem);
    if (e != cudaSuccess) {
      clv_destroy(h);
      return fail(nullptr, CLV_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
  }
  // EOS table in the working precision, nodes packed as (P, T, c_s^2, Plo); Plo = 0 in FP64
  if (cfg->eos_kind == CLV_EOS_TABLE) {
    const int n = cfg->eos_n;
    cudaError_t e;
    if (h->rsize == 8) {
      std::vector<double> pk((size_t)4 * n);
      for (int i = 0; i < n; ++i) {
        pk[4 * i] = cfg->eos_P[i]; pk[4 * i + 1] = cfg->eos_T[i]; pk[4 * i + 2] = cfg->eos_cs2[i]; pk[4 * i + 3] = 0.0;
      }
      e = cudaMemcpy(h->eos[0], pk.data(), pk.size() * 8, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> pk((size_t)4 * n);
      for (int i = 0; i < n; ++i) {
        pk[4 * i] = (float)cfg->eos_P[i]; pk[4 * i + 1] = (float)cfg->eos_T[i];
        pk[4 * i + 2] = (float)cfg->eos_cs2[i];
        pk[4 * i + 3] = (float)(cfg->eos_P[i] - (double)pk[4 * i]);   // the rest of P (EosView)
      }
      e = cudaMemcpy(h->eos[0], pk.data(), pk.size() * 4, cudaMemcpyHostToDevice);
    }
    // table positions of the powers of two for the FP32 lookups (EosView::xk)
    if (e == cudaSuccess) {
      std::vector<float2> xk(kEosXkEntries);
      for (int i = 0; i < kEosXkEntries; ++i) {
        const double x = ((i - 125) * std::log(2.0) - cfg->eos_lne0) / cfg->eos_dlne;
        const double ip = std::floor(x);
        xk[i] = make_float2((float)ip, (float)(x - ip));
      }
      e = cudaMemcpy((char*)h->eos[0] + (size_t)4 * n * h->rsize, xk.data(), xk.size() * sizeof(float2),
                     cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) { clv_destroy(h); return fail(nullptr, CLV_ECUDA, cudaGetErrorString(e)); }
  }
  cudaError_t e = cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { clv_destroy(h); return fail(nullptr, CLV_ECUDA, cudaGetErrorString(e)); }
  *out = h;
  return CLV_OK;
}

}  // namespace

// Message for clv_last_error(NULL) from calls that have no handle.
void clv_set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }

// ============================== C ABI =====================================
extern "C" {

clv_status clv_workspace_bytes(const clv_config* cfg, size_t* bytes) {
  clv_status s = validate(cfg);
  if (s != CLV_OK) return s;
  if (!bytes) return fail(nullptr, CLV_EINVAL, "bytes is NULL");
  *bytes = layout(cfg, nullptr);
  return CLV_OK;
}

clv_status clv_create(const clv_config* cfg, void* cuda_stream, clv_handle** out) {
  return create_common(cfg, cuda_stream, nullptr, 0, out);
}

clv_status clv_create_ws(const clv_config* cfg, void* cuda_stream, void* device_ws, size_t ws_bytes,
                         clv_handle** out) {
  if (!device_ws) return fail(nullptr, CLV_EINVAL, "device_ws is NULL");
  return create_common(cfg, cuda_stream, device_ws, ws_bytes, out);
}

}  // extern "C"

// Primitives of an initial T^{tau mu} with pi = 0 (T_ideal = T): the FP64
// root solve of Sec. 3 on the handle's EOS table, in place (a[0..3] hold
// T^{tau tau}, T^{tau x}, T^{tau y}, tau T^{tau eta} on entry and eps, u~^x,
// u~^y, u~^eta on exit).
template <typename R>
__global__ void __launch_bounds__(kBlock) prims_from_T_kernel(double* a0, double* a1, double* a2, double* a3,
                                                              EosView<R> eos, double eps_cut, long long N,
                                                              unsigned long long* counters, unsigned* err) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double e, ux, uy, ue;
  const double E = a0[c], Mx = a1[c], My = a2[c], Me = a3[c];
  if (!(isfinite(E) && isfinite(Mx) && isfinite(My) && isfinite(Me))) {
    atomicOr(err, 2u);
    e = ux = uy = ue = 0.0;
  } else {
    const RootResult rr = solve_primitive<double, R, R>(eos, eps_cut, E, Mx, My, Me, 1e-15, 200, e, ux, uy, ue);
    if (rr.rescaled) atomicAdd(counters + 0, 1ull);
    if (rr.iters < 0) { atomicAdd(counters + 1, 1ull); atomicOr(err, 1u); }
  }
  a0[c] = e; a1[c] = ux; a2[c] = uy; a3[c] = ue;
}

extern "C" {

static clv_status set_initial_T_any(clv_handle* h, const double* T, bool host) {
  if (!h) return CLV_EINVAL;
  if (!h->batch.empty()) return fail(h, CLV_EINVAL, "a batch takes its events' states by clv_batch_set_initial");
  if (!T) return fail(h, CLV_EINVAL, "T is required");
  const long long N = h->Nc;   // compact input cells
  // scratch: the stage-2 shear buffers (>= 4 N doubles in either precision),
  // which the initial state does not use
  double* a = reinterpret_cast<double*>(h->PI1[0]);
  CLV_CUDA(h, cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream));
  for (int m = 0; m < 4; ++m)
    CLV_CUDA(h, cudaMemcpyAsync(a + (size_t)m * N, T + (size_t)m * N, (size_t)N * 8,
                                host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
  const unsigned g = grid_of(N);
  if (h->rsize == 8)
    prims_from_T_kernel<double><<<g, kBlock, 0, h->stream>>>(a, a + N, a + 2 * N, a + 3 * N, eos_view<double>(h),
                                                             h->cfg.eps_cut, N, h->dstats->counters,
                                                             &h->dstats->err);
  else
    prims_from_T_kernel<float><<<g, kBlock, 0, h->stream>>>(a, a + N, a + 2 * N, a + 3 * N, eos_view<float>(h),
                                                            h->cfg.eps_cut, N, h->dstats->counters,
                                                            &h->dstats->err);
  CLV_CUDA(h, cudaGetLastError());
  unsigned err = 0;
  CLV_CUDA(h, cudaMemcpyAsync(&err, &h->dstats->err, 4, cudaMemcpyDeviceToHost, h->stream));
  CLV_CUDA(h, cudaStreamSynchronize(h->stream));
  if (err & 2u) return fail(h, CLV_ENONFINITE, "non-finite T^{tau mu} in the initial state");
  if (err & 1u) return fail(h, CLV_EROOT, "root solve of the initial state hit its iteration cap");
  const double* in[4] = {a, a + N, a + 2 * N, a + 3 * N};
  h->cur = 0;
  h->prev = 1;
  clv_status st =
      h->rsize == 8 ? set_initial_impl<double>(h, in, nullptr, false) : set_initial_impl<float>(h, in, nullptr, false);
  if (st != CLV_OK) return st;
  // the scratch is consumed (stream order): the stage buffers return to zeros, as the
  // padding slots of the eta rows, which the stages never write, must stay vacuum
  for (int q = 0; q < 10; ++q)
    CLV_CUDA(h, cudaMemsetAsync((char*)h->PI1[q] - (size_t)h->cfg.halo_x * h->cfg.ny * h->nep * h->rsize, 0,
                                ((size_t)h->N + 2 * (size_t)h->cfg.halo_x * h->cfg.ny * h->nep) * h->rsize,
                                h->stream));
  return CLV_OK;
}

static clv_status set_initial_any(clv_handle* h, const double* eps, const double* ux, const double* uy,
                                  const double* ueta, const double* pi, bool host) {
  if (!h) return CLV_EINVAL;
  if (!h->batch.empty()) return fail(h, CLV_EINVAL, "a batch takes its events' states by clv_batch_set_initial");
  if (!eps || !ux || !uy || !ueta) return fail(h, CLV_EINVAL, "eps, ux, uy and ueta are required");
  const double* in[4] = {eps, ux, uy, ueta};
  h->cur = 0;
  h->prev = 1;
  return h->rsize == 8 ? set_initial_impl<double>(h, in, pi, host) : set_initial_impl<float>(h, in, pi, host);
}

clv_status clv_set_initial(clv_handle* h, const double* eps, const double* ux, const double* uy,
                           const double* ueta, const double* pi) {
  return set_initial_any(h, eps, ux, uy, ueta, pi, true);
}

clv_status clv_set_initial_T(clv_handle* h, const double* T) { return set_initial_T_any(h, T, true); }

clv_status clv_set_initial_T_device(clv_handle* h, const double* d_T) { return set_initial_T_any(h, d_T, false); }

clv_status clv_set_initial_device(clv_handle* h, const double* d_eps, const double* d_ux, const double* d_uy,
                                  const double* d_ueta, const double* d_pi) {
  return set_initial_any(h, d_eps, d_ux, d_uy, d_ueta, d_pi, false);
}

static clv_status set_initial_n_any(clv_handle* h, const double* n, bool host) {
  if (!h || !n) return CLV_EINVAL;
  if (!h->cfg.charge) return fail(h, CLV_EINVAL, "the handle was created without charge = 1");
  if (!h->batch.empty()) return fail(h, CLV_EINVAL, "charge transport runs on single events, not a batch");
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  const double* src = n;
  if (host) {
    CLV_CUDA(h, cudaMemcpyAsync(h->staging, n, (size_t)h->Nc * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    src = h->staging;
  }
  const double taus = h->cfg.cartesian ? 1.0 : h->tau;
  if (h->rsize == 8)
    launch_charge_init<double>(src, prim_set<double>(h, h->cur), taus, h->NC[0], h->Nc, h->cfg.neta, h->nep, h->stream);
  else
    launch_charge_init<float>(src, prim_set<float>(h, h->cur), taus, h->NC[0], h->Nc, h->cfg.neta, h->nep, h->stream);
  CLV_CUDA(h, cudaGetLastError());
  if (host) CLV_CUDA(h, cudaStreamSynchronize(h->stream));   // the staging buffer is reused
  if (!h->charge_on) invalidate_graphs(h);
  h->charge_on = true;
  return CLV_OK;
}

clv_status clv_set_initial_n(clv_handle* h, const double* n) { return set_initial_n_any(h, n, true); }
clv_status clv_set_initial_n_device(clv_handle* h, const double* d_n) { return set_initial_n_any(h, d_n, false); }

clv_status clv_step(clv_handle* h, int nsteps, clv_stats* stats) {
  if (!h) return CLV_EINVAL;
  if (h->cfg.halo_x) return fail(h, CLV_EINVAL, "an x-slab steps by clv_stage with halo exchanges in between");
  if (!h->initialized && !h->batch.empty()) {
    for (const auto& ev : h->batch)
      if (!ev.set) return fail(h, CLV_EINVAL, "clv_batch_set_initial was not called for every event");
    clv_status s = h->rsize == 8 ? finish_initial<double>(h) : finish_initial<float>(h);
    if (s != CLV_OK) return s;
  }
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  if (nsteps < 0) return fail(h, CLV_EINVAL, "nsteps must be >= 0");
  if (stats && nsteps > 0) CLV_CUDA(h, cudaMemsetAsync(&h->dstats->emax_bits, 0, 8, h->stream));
  for (int s = 0; s < nsteps;) {
    const bool last = stats && s == nsteps - 1;
    const int plain_left = nsteps - s - (stats ? 1 : 0);   // steps before the one that reduces stats
    if (h->graphs && !h->timing && plain_left >= 2) {
      cudaGraphExec_t g = step_pair_graph(h);
      if (g) {
        CLV_CUDA(h, cudaGraphLaunch(g, h->stream));
        for (int k = 0; k < 2; ++k) h->tau = h->tau + h->cfg.dtau;   // the device's additions
        h->step += 2;
        s += 2;
        continue;
      }
    }
    launch_one_step(h, last);
    ++s;
  }
  CLV_CUDA(h, cudaGetLastError());
  if (!stats) return CLV_OK;
  const bool scan = nsteps == 0;
  return h->rsize == 8 ? reduce_stats<double>(h, scan, stats) : reduce_stats<float>(h, scan, stats);
}

clv_status clv_get_stats(clv_handle* h, clv_stats* stats) {
  if (!h || !stats) return CLV_EINVAL;
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  return h->rsize == 8 ? reduce_stats<double>(h, true, stats) : reduce_stats<float>(h, true, stats);
}

static clv_status get_fields_range(clv_handle* h, uint32_t mask, double* out, bool host, long long off,
                                   long long n, int ne, int nep) {
  if (!h || !out) return CLV_EINVAL;
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  if (mask >> 24) return fail(h, CLV_EINVAL, "mask selects fields beyond index 23");
  if ((mask >> 21 & 3u) && !h->cfg.charge) return fail(h, CLV_EINVAL, "fields 21 and 22 need charge = 1");
  if ((mask >> 23 & 1u) && !h->PB[0]) return fail(h, CLV_EINVAL, "field 23 needs zeta_over_s > 0");
  size_t slot = 0;
  for (int f = 0; f < 24; ++f) {
    if (!(mask >> f & 1u)) continue;
    double* dst = host ? h->staging : out + slot * (size_t)n;
    clv_status s = h->rsize == 8 ? export_field<double>(h, f, dst, off, n, ne, nep)
                                 : export_field<float>(h, f, dst, off, n, ne, nep);
    if (s != CLV_OK) return s;
    if (host) {
      CLV_CUDA(h, cudaMemcpyAsync(out + slot * (size_t)n, h->staging, (size_t)n * 8,
                                  cudaMemcpyDeviceToHost, h->stream));
      CLV_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    ++slot;
  }
  return CLV_OK;
}

static clv_status get_fields_any(clv_handle* h, uint32_t mask, double* out, bool host) {
  if (!h) return CLV_EINVAL;
  return get_fields_range(h, mask, out, host, 0, h->Nc, h->cfg.neta, h->nep);
}

clv_status clv_get_fields(clv_handle* h, uint32_t mask, double* host_out) {
  return get_fields_any(h, mask, host_out, true);
}

clv_status clv_get_fields_device(clv_handle* h, uint32_t mask, double* device_out) {
  return get_fields_any(h, mask, device_out, false);
}

clv_status clv_get_time(const clv_handle* h, double* tau, int64_t* step) {
  if (!h) return CLV_EINVAL;
  if (tau) *tau = h->tau;
  if (step) *step = h->step;
  return CLV_OK;
}

clv_status clv_set_guess(clv_handle* h, int mode) {
  if (!h) return CLV_EINVAL;
  if (mode < kGuessPrevious || mode > kGuessMlpAll) return fail(h, CLV_EINVAL, "unknown guess mode");
  const bool net = mode == kGuessMlp || mode == kGuessMlpAll;
  if (net && !h->mlp_loaded) return fail(h, CLV_EINVAL, "no network loaded (clv_set_mlp)");
  if (net && h->rsize != 4) return fail(h, CLV_EINVAL, "the learned guess runs on the FP32 path");
  if (h->guess != mode) invalidate_graphs(h);
  h->guess = mode;
  return CLV_OK;
}

static uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);  // NaN stays NaN
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;                                                          // round to nearest even
  return (uint16_t)(u >> 16);
}

clv_status clv_set_mlp(clv_handle* h, const float* params) {
  if (!h || !params) return CLV_EINVAL;
  std::vector<uint16_t> w(kMlpBf16Elems, 0);
  std::vector<float> b(kMlpBiasElems, 0.f);
  for (int i = 0; i < kMlpHid; ++i)
    for (int k = 0; k < kMlpIn; ++k) w[i * 16 + k] = to_bf16(params[kOffW1 + i * kMlpIn + k]);
  for (int i = 0; i < kMlpHid; ++i)
    for (int k = 0; k < kMlpHid; ++k) w[kMlpW1e + i * 64 + k] = to_bf16(params[kOffW2 + i * kMlpHid + k]);
  for (int o = 0; o < kMlpOut; ++o)
    for (int k = 0; k < kMlpHid; ++k) w[kMlpW1e + kMlpW2e + o * 64 + k] = to_bf16(params[kOffW3 + o * kMlpHid + k]);
  for (int i = 0; i < kMlpHid; ++i) { b[i] = params[kOffB1 + i]; b[64 + i] = params[kOffB2 + i]; }
  for (int o = 0; o < kMlpOut; ++o) b[128 + o] = params[kOffB3 + o];
  char* dst = (char*)h->mlp;
  CLV_CUDA(h, cudaMemcpyAsync(dst, w.data(), w.size() * 2, cudaMemcpyHostToDevice, h->stream));
  CLV_CUDA(h, cudaMemcpyAsync(dst + w.size() * 2, b.data(), b.size() * 4, cudaMemcpyHostToDevice, h->stream));
  CLV_CUDA(h, cudaStreamSynchronize(h->stream));
  h->mlp_loaded = true;
  return CLV_OK;
}

}  // extern "C"

template <typename R> static clv_status mlp_samples_impl(clv_handle* h, float* X, float* Y, int64_t* count) {
  SampleIn<R> a;
  for (int m = 0; m < 4; ++m) { a.T4.p[m] = (R*)h->T0[m]; a.T4l[m] = (const R*)h->TL0[m]; }
  for (int q = 0; q < 10; ++q) a.pi.p[q] = (R*)h->PI0[q];
  a.pr = prim_set<R>(h, h->cur);
  a.viscous = h->viscous;
  a.taus = (R)(h->cfg.cartesian ? 1.0 : h->tau);
  a.eps_cut = (R)h->cfg.eps_cut;
  a.N = h->N;
  // scratch in the staging buffer: block counts, then their offsets
  const unsigned nb = grid_of(h->N);
  unsigned* counts = reinterpret_cast<unsigned*>(h->staging);
  unsigned long long* offsets = reinterpret_cast<unsigned long long*>(h->staging + (nb + 1) / 2 + 1);
  mlp_samples_kernel<R, false><<<nb, kBlock, 0, h->stream>>>(a, counts, nullptr, nullptr, nullptr);
  scan_counts_kernel<<<1, kBlock, 0, h->stream>>>(counts, (int)nb, offsets, reinterpret_cast<long long*>(count));
  mlp_samples_kernel<R, true><<<nb, kBlock, 0, h->stream>>>(a, nullptr, offsets, X, Y);
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

extern "C" {

clv_status clv_mlp_samples(clv_handle* h, float* d_X, float* d_Y, int64_t* d_count) {
  if (!h || !d_X || !d_Y || !d_count) return CLV_EINVAL;
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  return h->rsize == 8 ? mlp_samples_impl<double>(h, d_X, d_Y, d_count)
                       : mlp_samples_impl<float>(h, d_X, d_Y, d_count);
}

}  // extern "C"

__global__ void __launch_bounds__(kBlock) mlp_forward_kernel(const void* mlp, const float* X, long long n, float* Y) {
  __shared__ __align__(16) __nv_bfloat16 s_w[kMlpSmemW];
  __shared__ float s_b[kMlpBiasElems];
  __shared__ __align__(16) __nv_bfloat16 s_x[kBlock / 32][32][kMlpSX];
  __shared__ float s_y[kBlock / 32][32][4];
  mlp_load_smem(mlp, s_w, s_b);
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 16; k += 2) {
    const float lo = (c < n && k < kMlpIn) ? X[c * kMlpIn + k] : 0.f;
    const float hi = (c < n && k + 1 < kMlpIn) ? X[c * kMlpIn + k + 1] : 0.f;
    *reinterpret_cast<unsigned*>(&s_x[wid][lane][k]) = pack_bf16(lo, hi);
  }
  __syncthreads();
  mlp_tile16(&s_x[wid][0][0], s_w, s_b, &s_y[wid][0][0], lane);
  mlp_tile16(&s_x[wid][16][0], s_w, s_b, &s_y[wid][16][0], lane);
  __syncwarp();
  if (c < n)
    for (int o = 0; o < kMlpOut; ++o) Y[c * kMlpOut + o] = s_y[wid][lane][o];
}

extern "C" {

clv_status clv_mlp_forward(clv_handle* h, const float* d_X, int64_t n, float* d_Y) {
  if (!h || n < 0) return CLV_EINVAL;
  if (!h->mlp_loaded) return fail(h, CLV_EINVAL, "no network loaded (clv_set_mlp)");
  if (n == 0) return CLV_OK;
  if (!d_X || !d_Y) return fail(h, CLV_EINVAL, "null feature or output array");
  mlp_forward_kernel<<<grid_of(n), kBlock, 0, h->stream>>>(h->mlp, d_X, n, d_Y);
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

static clv_status mlp_grad_attr() {
  static bool done = false;
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute((const void*)mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mlp_grad_smem_bytes());
    if (e != cudaSuccess) return fail(nullptr, CLV_ECUDA, cudaGetErrorString(e));
    done = true;
  }
  return CLV_OK;
}

// blocks of a deterministic gradient launch over `batch` samples
static int mlp_grad_blocks(long long batch) {
  return (int)std::min<long long>(kMlpGradBlocks, (batch + kMlpTrainBlock - 1) / kMlpTrainBlock);
}

clv_status clv_mlp_loss_grad(const float* d_params, const float* d_X, const float* d_Y, int64_t n, void* stream,
                             float* d_grad, float* d_loss, float* d_work) {
  if (!d_params || !d_X || !d_Y || !d_grad || !d_loss || !d_work || n < 1)
    return fail(nullptr, CLV_EINVAL, "bad arguments");
  clv_status s = mlp_grad_attr();
  if (s != CLV_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = mlp_grad_blocks(n);
  mlp_grad_kernel<<<blocks, kMlpTrainBlock, mlp_grad_smem_bytes(), st>>>(d_params, d_X, d_Y, n, n, 0ull, 0, d_work);
  mlp_reduce_kernel<<<(kMlpPartialRow + 255) / 256, 256, 0, st>>>(d_work, blocks, d_grad, d_loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CLV_OK : fail(nullptr, CLV_ECUDA, cudaGetErrorString(e));
}

clv_status clv_mlp_train(float* d_params, float* d_work, const float* d_X, const float* d_Y, int64_t n, int iters,
                         int batch, float lr, uint64_t seed, int step0, void* stream, float* d_loss) {
  if (!d_params || !d_work || !d_X || !d_Y || !d_loss || n < 1 || iters < 0 || batch < 1 || step0 < 0 || seed == 0)
    return fail(nullptr, CLV_EINVAL, "bad arguments (seed must be nonzero)");
  clv_status s = mlp_grad_attr();
  if (s != CLV_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  float* m = d_work;
  float* v = d_work + kMlpParams;
  float* g = d_work + 2 * kMlpParams;
  float* partial = d_work + 3 * kMlpParams;
  const int blocks = mlp_grad_blocks(batch);
  for (int it = 0; it < iters; ++it) {
    mlp_grad_kernel<<<blocks, kMlpTrainBlock, mlp_grad_smem_bytes(), st>>>(d_params, d_X, d_Y, n, batch, seed,
                                                                          step0 + it, partial);
    mlp_reduce_kernel<<<(kMlpPartialRow + 255) / 256, 256, 0, st>>>(partial, blocks, g, d_loss + it);
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(d_params, m, v, g, step0 + it + 1, lr);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CLV_OK : fail(nullptr, CLV_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"

static void tile_info(const clv_handle* h, double ms, clv_tile_info* out) {
  if (!h->batch.empty()) {   // a batch: its tiling policy (thread cap, x chunk) and launch shape
    out->TJ = h->batch_maxthr;
    out->TK = 0;
    out->CX = h->batch_chunk;
    out->threads = h->batch_threads;
    out->blocks = (int)h->batch_blocks;
    out->smem_bytes = (int)h->batch_smem;
    out->ms = ms;
    return;
  }
  out->TJ = h->tile.TJ;
  out->TK = h->tile.TK;
  out->CX = h->tile.CX;
  out->threads = h->tile_threads;
  out->blocks = (int)h->tile_blocks;
  out->smem_bytes = (int)h->tile_smem;
  out->ms = ms;
}

static cudaError_t apply_tile(clv_handle* h, const TileGeom& g) {
  cudaError_t e = h->rsize == 8 ? tile_attributes<double, false>(g.smem) : tile_attributes<float, false>(g.smem);
  if (e == cudaSuccess && h->viscous)
    e = h->rsize == 8 ? tile_attributes<double, true>(g.smem) : tile_attributes<float, true>(g.smem);
  if (e != cudaSuccess) return e;
  invalidate_graphs(h);
  h->tile = g.t;
  h->tile_threads = g.threads;
  h->tile_blocks = g.blocks;
  h->tile_smem = g.smem;
  return cudaSuccess;
}

// Mean time of `reps` stage-1 tile launches on the current state (stage 1
// reads the state and writes only the stage buffers, so repeating it leaves
// the evolution unchanged).
static cudaError_t batch_schedule(clv_handle* h, int maxthr, int chunk, int sms, size_t smem_max);

template <typename R, bool VISC>
static cudaError_t time_stage1_batch(clv_handle* h, int reps, cudaEvent_t e0, cudaEvent_t e1, double* ms) {
  const StageParams<R> p = stage_params<R>(h, 1);
  auto launch = [&]() {
    cudaMemsetAsync(h->batch_ctr, 0, sizeof(int), h->stream);
    stage_batch_kernel<R, 1, VISC><<<h->batch_blocks, h->batch_threads, h->batch_smem, h->stream>>>(
        p, (const EventGeom<R>*)h->batch_geom, h->batch_tiles, h->batch_items, h->batch_nitems, h->batch_ctr);
  };
  launch();
  cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, h->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  *ms = (double)t / reps;
  return e;
}

template <typename R, bool VISC>
static cudaError_t time_stage1(clv_handle* h, int reps, cudaEvent_t e0, cudaEvent_t e1, double* ms) {
  const StageParams<R> p = stage_params<R>(h, 1);
  stage_tile_kernel<R, 1, VISC><<<h->tile_blocks, h->tile_threads, h->tile_smem, h->stream>>>(p, h->tile);
  cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps; ++r)
    stage_tile_kernel<R, 1, VISC><<<h->tile_blocks, h->tile_threads, h->tile_smem, h->stream>>>(p, h->tile);
  cudaEventRecord(e1, h->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  *ms = (double)t / reps;
  return e;
}


extern "C" {

// ---------------- checkpoint ----------------
struct StateHeader {
  uint32_t magic, version;
  int32_t nx, ny, neta, precision, viscous, pad;
  double tau, dx, dy, deta, dtau, eta_over_s;
  int64_t step;
};
constexpr uint32_t kStateMagic = 0x53564c43u;  // "CLVS"
constexpr uint32_t kStateVersion = 2u;          // 2: the FP32 path's T~ as float-float pairs
constexpr int kStateFieldsMax = 4 + 4 + 10 + 2 * kPrimFields;

// fields of the checkpoint (FP32 path: the low parts of T~ follow T~)
static int state_fields(const clv_handle* h) { return kStateFieldsMax - (h->TL0[0] ? 0 : 4); }

static size_t state_bytes(const clv_handle* h) {
  return sizeof(StateHeader) + (size_t)(state_fields(h) + (h->cfg.charge ? 1 : 0) + (h->PB[0] ? 1 : 0)) *
                                   (size_t)h->N * h->rsize;
}

// device arrays of the state in checkpoint order: T~ (4; FP32 path: then its
// low parts, 4), pi~ (10), the primitives of the current step (6) and of the
// previous step (6)
static void state_arrays(clv_handle* h, void* a[kStateFieldsMax]) {
  int k = 0;
  for (int m = 0; m < 4; ++m) a[k++] = h->T0[m];
  if (h->TL0[0])
    for (int m = 0; m < 4; ++m) a[k++] = h->TL0[m];
  for (int q = 0; q < 10; ++q) a[k++] = h->PI0[q];
  for (int f = 0; f < kPrimFields; ++f) a[k++] = h->PR[h->cur][f];
  for (int f = 0; f < kPrimFields; ++f) a[k++] = h->PR[h->prev][f];
}

clv_status clv_state_bytes(const clv_handle* h, size_t* bytes) {
  if (!h || !bytes) return CLV_EINVAL;
  *bytes = state_bytes(h);
  return CLV_OK;
}

clv_status clv_get_state(clv_handle* h, void* buf, size_t bytes) {
  if (!h || !buf) return CLV_EINVAL;
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  if (bytes < state_bytes(h)) return fail(h, CLV_EINVAL, "state buffer too small (clv_state_bytes)");
  const clv_config& c = h->cfg;
  // pad: bit 0 = the net charge is being transported (its field follows the others),
  // bit 1 = the state carries the bulk pressure (its field comes last)
  StateHeader hd{kStateMagic, kStateVersion, c.nx, c.ny, c.neta, c.precision, h->viscous ? 1 : 0,
                 (h->charge_on ? 1 : 0) | (h->PB[0] ? 2 : 0),
                 h->tau, c.dx, c.dy, c.deta, c.dtau, c.eta_over_s, h->step};
  std::memcpy(buf, &hd, sizeof(hd));
  void* a[kStateFieldsMax];
  state_arrays(h, a);
  char* dst = static_cast<char*>(buf) + sizeof(hd);
  const size_t fb = (size_t)h->N * h->rsize;
  for (int k = 0; k < state_fields(h); ++k) {
    CLV_CUDA(h, cudaMemcpyAsync(dst, a[k], fb, cudaMemcpyDeviceToHost, h->stream));
    dst += fb;
  }
  if (c.charge) {
    CLV_CUDA(h, cudaMemcpyAsync(dst, h->NC[0], fb, cudaMemcpyDeviceToHost, h->stream));
    dst += fb;
  }
  if (h->PB[0])   // the bulk pressure follows (after the charge field, if any)
    CLV_CUDA(h, cudaMemcpyAsync(dst, h->PB[0], fb, cudaMemcpyDeviceToHost, h->stream));
  CLV_CUDA(h, cudaStreamSynchronize(h->stream));
  return CLV_OK;
}

clv_status clv_set_state(clv_handle* h, const void* buf, size_t bytes) {
  if (!h || !buf) return CLV_EINVAL;
  if (bytes < sizeof(StateHeader)) return fail(h, CLV_EINVAL, "state buffer too small");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  const clv_config& c = h->cfg;
  if (hd.magic != kStateMagic || hd.version != kStateVersion)
    return fail(h, CLV_EINVAL, "not a checkpoint of this library version");
  if (hd.nx != c.nx || hd.ny != c.ny || hd.neta != c.neta || hd.precision != c.precision ||
      hd.viscous != (h->viscous ? 1 : 0) || hd.dx != c.dx || hd.dy != c.dy || hd.deta != c.deta ||
      hd.dtau != c.dtau || hd.eta_over_s != c.eta_over_s || ((hd.pad >> 1) & 1) != (h->PB[0] ? 1 : 0))
    return fail(h, CLV_EINVAL, "checkpoint of a different configuration");
  if (bytes < state_bytes(h)) return fail(h, CLV_EINVAL, "state buffer too small (clv_state_bytes)");
  h->cur = 0;
  h->prev = 1;
  void* a[kStateFieldsMax];
  state_arrays(h, a);
  const char* src = static_cast<const char*>(buf) + sizeof(hd);
  const size_t fb = (size_t)h->N * h->rsize;
  for (int k = 0; k < state_fields(h); ++k) {
    CLV_CUDA(h, cudaMemcpyAsync(a[k], src, fb, cudaMemcpyHostToDevice, h->stream));
    src += fb;
  }
  if (c.charge) {
    const bool on = (hd.pad & 1) != 0;
    if (on != h->charge_on) invalidate_graphs(h);
    h->charge_on = on;
    CLV_CUDA(h, cudaMemcpyAsync(h->NC[0], src, fb, cudaMemcpyHostToDevice, h->stream));
    src += fb;
  }
  if (h->PB[0]) CLV_CUDA(h, cudaMemcpyAsync(h->PB[0], src, fb, cudaMemcpyHostToDevice, h->stream));
  CLV_CUDA(h, cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream));
  set_tau(h, hd.tau);
  CLV_CUDA(h, cudaStreamSynchronize(h->stream));
  h->step = hd.step;
  h->initialized = true;
  return CLV_OK;
}

// ---------------- x-slab: halo planes and stage-level stepping ----------------
}  // extern "C"

template <typename R> struct Ptr23 { R* p[23]; };

// mode 0: pack planes src, src + 1 of every field into buf [field][2][plane];
// mode 1: unpack buf into planes dst, dst + 1; mode 2: copy plane src into
// planes dst, dst + 1 (zero-gradient edge).
template <typename R>
__global__ void __launch_bounds__(kBlock) slab_planes_kernel(Ptr23<R> f, int nf, long long plane, long long src,
                                                             long long dst, R* buf, int mode) {
  const long long per = 2 * plane;
  const long long total = per * nf;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int fi = (int)(i / per);
    const long long r = i - fi * per;
    const long long pp = r / plane, cell = r - pp * plane;
    R* a = f.p[fi];
    if (mode == 0) buf[i] = a[(src + pp) * plane + cell];
    else if (mode == 1) a[(dst + pp) * plane + cell] = buf[i];
    else a[(dst + pp) * plane + cell] = a[src * plane + cell];
  }
}

// The fields a stage reads from its x-neighbours: set 1 (stage 1) T~ (FP32
// path: high and low parts), pi~ and the current primitives u~, P, c_s; set 2
// (stage 2) the stage-1 results.
static int slab_nfields(const clv_handle* h) {
  return 4 + (h->TL0[0] ? 4 : 0) + (h->viscous ? 10 : 0) + (kPrimFields - 1);
}
template <typename R> static int slab_fields(clv_handle* h, int set, Ptr23<R>& f) {
  int n = 0;
  const int st = 3 - h->cur - h->prev;
  for (int m = 0; m < 4; ++m) f.p[n++] = (R*)(set == 1 ? h->T0[m] : h->T1[m]);
  if (h->TL0[0])
    for (int m = 0; m < 4; ++m) f.p[n++] = (R*)(set == 1 ? h->TL0[m] : h->TL1[m]);
  if (h->viscous)
    for (int q = 0; q < 10; ++q) f.p[n++] = (R*)(set == 1 ? h->PI0[q] : h->PI1[q]);
  const int ps = set == 1 ? h->cur : st;
  for (int k = 1; k < kPrimFields; ++k) f.p[n++] = (R*)h->PR[ps][k];   // u~ (3), P, c_s
  return n;
}

template <typename R> static clv_status slab_op(clv_handle* h, int set, int side, R* buf, int mode) {
  Ptr23<R> f;
  const int nf = slab_fields<R>(h, set, f);
  const long long plane = (long long)h->cfg.ny * h->nep;
  const long long nx = h->cfg.nx;
  long long src = 0, dst = 0;
  if (mode == 0) src = side == 0 ? 0 : nx - 2;
  if (mode == 1) dst = side == 0 ? -2 : nx;
  if (mode == 2) { src = side == 0 ? 0 : nx - 1; dst = side == 0 ? -2 : nx; }
  const long long total = 2 * plane * nf;
  const unsigned g = (unsigned)std::min<long long>((total + kBlock - 1) / kBlock, (long long)h->sms * 8);
  slab_planes_kernel<R><<<g, kBlock, 0, h->stream>>>(f, nf, plane, src, dst, buf, mode);
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

static clv_status slab_check(clv_handle* h, int set, int side) {
  if (!h) return CLV_EINVAL;
  if (!h->cfg.halo_x) return fail(h, CLV_EINVAL, "not an x-slab (halo_x = 0)");
  if ((set != 1 && set != 2) || (side != 0 && side != 1)) return fail(h, CLV_EINVAL, "set must be 1 or 2, side 0 or 1");
  return CLV_OK;
}

extern "C" {

clv_status clv_slab_halo_bytes(const clv_handle* h, size_t* bytes) {
  if (!h || !bytes) return CLV_EINVAL;
  *bytes = (size_t)2 * h->cfg.ny * h->nep * slab_nfields(h) * h->rsize;
  return CLV_OK;
}

clv_status clv_slab_pack(clv_handle* h, int set, int side, void* d_buf) {
  clv_status s = slab_check(h, set, side);
  if (s != CLV_OK) return s;
  if (!d_buf) return fail(h, CLV_EINVAL, "buffer is NULL");
  return h->rsize == 8 ? slab_op<double>(h, set, side, (double*)d_buf, 0) : slab_op<float>(h, set, side, (float*)d_buf, 0);
}

clv_status clv_slab_unpack(clv_handle* h, int set, int side, const void* d_buf) {
  clv_status s = slab_check(h, set, side);
  if (s != CLV_OK) return s;
  if (!d_buf) return fail(h, CLV_EINVAL, "buffer is NULL");
  return h->rsize == 8 ? slab_op<double>(h, set, side, (double*)d_buf, 1) : slab_op<float>(h, set, side, (float*)d_buf, 1);
}

clv_status clv_slab_fill_edge(clv_handle* h, int set, int side) {
  clv_status s = slab_check(h, set, side);
  if (s != CLV_OK) return s;
  return h->rsize == 8 ? slab_op<double>(h, set, side, nullptr, 2) : slab_op<float>(h, set, side, nullptr, 2);
}

clv_status clv_slab_predictor(clv_handle* h, int stage) {
  if (!h) return CLV_EINVAL;
  if (!h->predictor_pending) return fail(h, CLV_EINVAL, "no first-step predictor pending");
  if (stage != 1 && stage != 2) return fail(h, CLV_EINVAL, "stage must be 1 or 2");
  if (h->rsize == 8) {
    launch_half<double, false>(h, stage, false, false);
    if (stage == 2) return initial_end<double>(h);
  } else {
    launch_half<float, false>(h, stage, false, false);
    if (stage == 2) return initial_end<float>(h);
  }
  CLV_CUDA(h, cudaGetLastError());
  return CLV_OK;
}

clv_status clv_stage(clv_handle* h, int stage, clv_stats* stats) {
  if (!h) return CLV_EINVAL;
  if (!h->initialized) return fail(h, CLV_EINVAL, "the initial state (and, for an x-slab, its predictor) is not complete");
  if (stage != 1 && stage != 2) return fail(h, CLV_EINVAL, "stage must be 1 or 2");
  const bool st = stats && stage == 2;
  if (st) CLV_CUDA(h, cudaMemsetAsync(&h->dstats->emax_bits, 0, 8, h->stream));
  if (h->rsize == 8) {
    if (h->viscous) launch_half<double, true>(h, stage, st, false); else launch_half<double, false>(h, stage, st, false);
  } else {
    if (h->viscous) launch_half<float, true>(h, stage, st, false); else launch_half<float, false>(h, stage, st, false);
  }
  CLV_CUDA(h, cudaGetLastError());
  if (!st) return CLV_OK;
  return h->rsize == 8 ? reduce_stats<double>(h, false, stats) : reduce_stats<float>(h, false, stats);
}

clv_status clv_set_graphs(clv_handle* h, int enable) {
  if (!h) return CLV_EINVAL;
  h->graphs = enable != 0;
  if (!h->graphs) invalidate_graphs(h);
  return CLV_OK;
}

clv_status clv_get_tile(clv_handle* h, clv_tile_info* out) {
  if (!h || !out) return CLV_EINVAL;
  tile_info(h, 0.0, out);
  return CLV_OK;
}

clv_status clv_set_tile(clv_handle* h, int TJ, int TK, int CX) {
  if (!h) return CLV_EINVAL;
  if (!h->batch.empty()) return fail(h, CLV_EINVAL, "a batch sets its tiles per event");
  const clv_config& c = h->cfg;
  if (TJ < 1 || TJ > c.ny || TK < 1 || TK > c.neta || CX < 0 || CX > c.nx)
    return fail(h, CLV_EINVAL, "tile shape out of range");
  if ((TJ + 1) * (TK + 1) > tile_max_threads(&c)) return fail(h, CLV_EINVAL, "tile needs too many threads");
  size_t smem_max = 0;
  const int sms = device_sms(&smem_max);
  const TileGeom g = tile_geometry_of(&c, sms, TJ, TK, CX);
  if (g.smem > smem_max) return fail(h, CLV_EINVAL, "tile needs more shared memory than a block may have");
  CLV_CUDA(h, apply_tile(h, g));
  return CLV_OK;
}

static clv_status autotune_batch(clv_handle* h, int max_candidates, int reps, clv_tile_info* best) {
  if (!h->initialized) return fail(h, CLV_EINVAL, "the batch is initialised by its first clv_step; autotune after it");
  size_t smem_max = 0;
  const int sms = device_sms(&smem_max);
  // candidate policies: thread cap per CTA x planes per x chunk, the current first
  const int tmax = h->rsize == 8 ? std::min(CLV_TILE_MAX_THREADS, kBlock / 2) : CLV_TILE_MAX_THREADS;
  std::vector<std::pair<int, int>> cand = {{h->batch_maxthr, h->batch_chunk}};
  for (int thr : {tmax, tmax * 3 / 4, tmax / 2})
    for (int chunk : {32, 16, 24, 48, 64})
      if (std::make_pair(thr, chunk) != cand[0] && (int)cand.size() <= max_candidates) cand.push_back({thr, chunk});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CLV_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(h, CLV_ECUDA, "cudaEventCreate"); }
  double best_ms = 1e300, cur_ms = 1e300;
  size_t best_i = 0;
  cudaError_t err = cudaSuccess;
  for (size_t i = 0; i < cand.size() && err == cudaSuccess; ++i) {
    cudaError_t es = batch_schedule(h, cand[i].first, cand[i].second, sms, smem_max);
    if (es == cudaErrorInvalidValue) continue;   // beyond the shared memory of a CTA: not a candidate
    err = es;
    double ms = 0.0;
    if (err == cudaSuccess) {
      if (h->rsize == 8)
        err = h->viscous ? time_stage1_batch<double, true>(h, reps, e0, e1, &ms)
                         : time_stage1_batch<double, false>(h, reps, e0, e1, &ms);
      else
        err = h->viscous ? time_stage1_batch<float, true>(h, reps, e0, e1, &ms)
                         : time_stage1_batch<float, false>(h, reps, e0, e1, &ms);
    }
    if (err == cudaSuccess && i == 0) cur_ms = ms;
    if (err == cudaSuccess && ms < best_ms) { best_ms = ms; best_i = i; }
  }
  // keep the current policy unless a candidate is clearly (2%) faster
  if (best_i != 0 && best_ms > 0.98 * cur_ms) { best_i = 0; best_ms = cur_ms; }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(h, CLV_ECUDA, std::string("autotune: ") + cudaGetErrorString(err));
  CLV_CUDA(h, batch_schedule(h, cand[best_i].first, cand[best_i].second, sms, smem_max));
  if (best) tile_info(h, best_ms, best);
  return CLV_OK;
}

clv_status clv_autotune(clv_handle* h, int max_candidates, int reps, clv_tile_info* best) {
  if (!h || max_candidates < 1 || reps < 1) return CLV_EINVAL;
  if (!h->batch.empty()) return autotune_batch(h, max_candidates, reps, best);
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  if (h->cfg.kernel != 0) return fail(h, CLV_EINVAL, "the autotuner tunes the tiled stage kernel");
  size_t smem_max = 0;
  const int sms = device_sms(&smem_max);
  std::vector<TileGeom> cand = tile_candidates(&h->cfg, sms, smem_max);
  if ((int)cand.size() > max_candidates) cand.resize(max_candidates);
  // the current shape competes too
  TileGeom cur;
  cur.t = h->tile; cur.threads = h->tile_threads; cur.blocks = h->tile_blocks; cur.smem = h->tile_smem;
  cand.insert(cand.begin(), cur);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CLV_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(h, CLV_ECUDA, "cudaEventCreate"); }
  double best_ms = 1e300, cur_ms = 0.0;
  size_t best_i = 0;
  cudaError_t err = cudaSuccess;
  for (size_t i = 0; i < cand.size() && err == cudaSuccess; ++i) {
    err = apply_tile(h, cand[i]);
    double ms = 0.0;
    if (err == cudaSuccess) {
      if (h->rsize == 8)
        err = h->viscous ? time_stage1<double, true>(h, reps, e0, e1, &ms) : time_stage1<double, false>(h, reps, e0, e1, &ms);
      else
        err = h->viscous ? time_stage1<float, true>(h, reps, e0, e1, &ms) : time_stage1<float, false>(h, reps, e0, e1, &ms);
    }
    if (err == cudaSuccess && i == 0) cur_ms = ms;
    if (err == cudaSuccess && ms < best_ms) { best_ms = ms; best_i = i; }
  }
  // keep the current shape unless a candidate is clearly (2%) faster: the
  // timings of near-equal shapes differ by run-to-run noise
  if (best_i != 0 && best_ms > 0.98 * cur_ms) { best_i = 0; best_ms = cur_ms; }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(h, CLV_ECUDA, std::string("autotune: ") + cudaGetErrorString(err));
  CLV_CUDA(h, apply_tile(h, cand[best_i]));
  if (best) tile_info(h, best_ms, best);
  return CLV_OK;
}

// ---------------- batch of events ----------------
}  // extern "C"

// Tile of one event of a batch under a tiling policy: TK from the eta_s
// extent (at most 32 columns), TJ as large as the thread cap allows (at most
// maxthr threads per CTA), x chunks of about `chunk` planes.
static TileArgs batch_tile(const clv_config& c, int maxthr_cap, int chunk) {
  TileArgs t;
  const int maxthr = std::min(tile_max_threads(&c), maxthr_cap);
  const int nk = (c.neta + 31) / 32;
  t.TK = (c.neta + nk - 1) / nk;
  t.TJ = std::max(1, std::min(c.ny, maxthr / (t.TK + 1) - 1));
  const size_t rsize = c.precision == CLV_FP64 ? 8 : 4;
  auto smem_of = [&](int TJ) {
    return c.eta_over_s > 0 ? tile_smem_bytes<true>(TJ, t.TK, rsize) : tile_smem_bytes<false>(TJ, t.TK, rsize);
  };
  while (t.TJ > 1 && smem_of(t.TJ) > kSmemOptinMax) --t.TJ;
  const int nch = (c.nx + chunk - 1) / chunk;
  t.CX = (c.nx + nch - 1) / nch;
  t.ntj = (c.ny + t.TJ - 1) / t.TJ;
  t.ntk = (c.neta + t.TK - 1) / t.TK;
  return t;
}

template <typename R> static cudaError_t batch_upload(clv_handle* h) {
  const size_t ne = h->batch.size();
  std::vector<EventGeom<R>> g(ne);
  std::vector<TileArgs> t(ne);
  for (size_t e = 0; e < ne; ++e) {
    const auto& ev = h->batch[e];
    const clv_config& c = ev.cfg;
    g[e] = EventGeom<R>{ev.off, c.nx, c.ny, c.neta, ev.nep, (R)(1.0 / c.dx), (R)(1.0 / c.dy), is_coef<R>(c), c.deta,
                        ev.viscous ? 1 : 0};
    t[e] = ev.tile;
  }
  cudaError_t err = cudaMalloc(&h->batch_geom, ne * sizeof(EventGeom<R>));
  if (err == cudaSuccess) err = cudaMemcpy(h->batch_geom, g.data(), ne * sizeof(EventGeom<R>), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc((void**)&h->batch_tiles, ne * sizeof(TileArgs));
  (void)t;
  return err;
}

template <typename R> static cudaError_t batch_attributes(size_t smem) {
  cudaError_t err = cudaSuccess;
  auto attr = [&](const void* f) {
    if (err == cudaSuccess) err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  };
  attr((const void*)stage_batch_kernel<R, 1, false>);
  attr((const void*)stage_batch_kernel<R, 2, false>);
  attr((const void*)stage_batch_kernel<R, 1, true>);
  attr((const void*)stage_batch_kernel<R, 2, true>);
  return err;
}

// (Re)builds the events' tiles and the work-item list (event, tile-chunk),
// most expensive first, for one tiling policy, and uploads them on the
// handle's stream.  Nothing changes (and cudaErrorInvalidValue is returned)
// if a tile would exceed the shared memory of a CTA.
static cudaError_t batch_schedule(clv_handle* h, int maxthr, int chunk, int sms, size_t smem_max) {
  maxthr = std::min(maxthr, h->rsize == 8 ? std::min(CLV_TILE_MAX_THREADS, kBlock / 2) : CLV_TILE_MAX_THREADS);
  const size_t ne = h->batch.size();
  std::vector<TileArgs> tiles(ne);
  std::vector<std::pair<double, int2>> items;
  size_t smem = 0;
  int thr = 0;
  for (size_t e = 0; e < ne; ++e) {
    const auto& ev = h->batch[e];
    const TileArgs t = batch_tile(ev.cfg, maxthr, chunk);
    tiles[e] = t;
    const size_t sm = ev.viscous ? tile_smem_bytes<true>(t.TJ, t.TK, h->rsize) : tile_smem_bytes<false>(t.TJ, t.TK, h->rsize);
    smem = std::max(smem, sm);
    thr = std::max(thr, (t.TJ + 1) * (t.TK + 1));
    const int nch = (ev.cfg.nx + t.CX - 1) / t.CX;
    const int nb = t.ntj * t.ntk * nch;
    for (int b = 0; b < nb; ++b) {
      const int ch = b / (t.ntj * t.ntk);
      const int planes = std::min(t.CX, ev.cfg.nx - ch * t.CX);
      const double cost = (planes + 4.0) * (t.TJ + 4.0) * (t.TK + 4.0) * (ev.viscous ? 2.0 : 1.0);
      items.push_back({cost, make_int2((int)e, b)});
    }
  }
  if (smem > smem_max) return cudaErrorInvalidValue;
  std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<int2> it(items.size());
  for (size_t i = 0; i < items.size(); ++i) it[i] = items[i].second;
  cudaError_t err = cudaStreamSynchronize(h->stream);   // no launch of the old schedule is in flight
  if (err == cudaSuccess) err = h->rsize == 8 ? batch_attributes<double>(smem) : batch_attributes<float>(smem);
  if (err == cudaSuccess && it.size() > (size_t)h->batch_nitems) {
    cudaFree(h->batch_items);
    h->batch_items = nullptr;
    err = cudaMalloc((void**)&h->batch_items, it.size() * sizeof(int2));
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(h->batch_items, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(h->batch_tiles, tiles.data(), ne * sizeof(TileArgs), cudaMemcpyHostToDevice, h->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);   // host vectors die here
  if (err != cudaSuccess) return err;
  for (size_t e = 0; e < ne; ++e) h->batch[e].tile = tiles[e];
  h->batch_smem = smem;
  h->batch_threads = thr;
  h->batch_nitems = (int)it.size();
  const void* bk = h->rsize == 8 ? (const void*)stage_batch_kernel<double, 2, true> : (const void*)stage_batch_kernel<float, 2, true>;
  h->batch_blocks = (unsigned)std::min<long long>((long long)sms * kernel_occupancy(bk, thr, smem), h->batch_nitems);
  h->batch_maxthr = maxthr;
  h->batch_chunk = chunk;
  invalidate_graphs(h);   // captured steps hold the old launch shape and item list
  return cudaSuccess;
}

extern "C" {

clv_status clv_create_batch(const clv_config* cfgs, int nevents, void* cuda_stream, clv_handle** out) {
  if (!out || !cfgs || nevents < 1) return fail(nullptr, CLV_EINVAL, "bad arguments");
  *out = nullptr;
  const clv_config& c0 = cfgs[0];
  long long N = 0;
  double eta_max = 0.0;
  for (int e = 0; e < nevents; ++e) {
    const clv_config& c = cfgs[e];
    clv_status st = validate(&c);
    if (st != CLV_OK) return st;
    const bool same_eos =
        c.eos_kind == c0.eos_kind &&
        (c.eos_kind != CLV_EOS_TABLE ||
         (c.eos_n == c0.eos_n && c.eos_lne0 == c0.eos_lne0 && c.eos_dlne == c0.eos_dlne &&
          std::equal(c.eos_P, c.eos_P + c.eos_n, c0.eos_P) && std::equal(c.eos_T, c.eos_T + c.eos_n, c0.eos_T) &&
          std::equal(c.eos_cs2, c.eos_cs2 + c.eos_n, c0.eos_cs2)));
    if (c.charge) return fail(nullptr, CLV_EINVAL, "charge transport runs on single events, not a batch");
    if (c.zeta_over_s > 0) return fail(nullptr, CLV_EINVAL, "bulk pressure runs on single events, not a batch");
    if (c.tau0 != c0.tau0 || c.dtau != c0.dtau || c.precision != c0.precision || c.cartesian != c0.cartesian ||
        c.periodic != c0.periodic || c.eps_cut != c0.eps_cut || c.kernel != 0 || !same_eos)
      return fail(nullptr, CLV_EINVAL,
                  "batch events must share tau0, dtau, precision, EOS, eps_cut, coordinates and boundaries "
                  "(kernel 0)");
    N += (long long)c.nx * c.ny * eta_pitch(c.neta);
    eta_max = std::max(eta_max, c.eta_over_s);
  }
  if (N > (1LL << 31) - 1) return fail(nullptr, CLV_EINVAL, "batch too large (at most 2^31 - 1 cells)");
  // the batch as one flat grid of N cells (layout, recovery, stats): N / 4
  // rows of 4 (every event's padded size is a multiple of 4)
  clv_config bc = c0;
  bc.nx = (int)(N / 4);
  bc.ny = 1;
  bc.neta = 4;
  bc.eta_over_s = eta_max;
  clv_status st = create_common(&bc, cuda_stream, nullptr, 0, out);
  if (st != CLV_OK) return st;
  clv_handle* h = *out;
  size_t smem_max = 0;
  const int sms = device_sms(&smem_max);
  long long off = 0;
  h->batch.resize(nevents);
  for (int e = 0; e < nevents; ++e) {
    auto& ev = h->batch[e];
    ev.cfg = cfgs[e];
    ev.cfg.eos_P = ev.cfg.eos_T = ev.cfg.eos_cs2 = nullptr;
    ev.off = off;
    ev.nep = eta_pitch(ev.cfg.neta);
    ev.N = (long long)ev.cfg.nx * ev.cfg.ny * ev.nep;
    ev.Nc = (long long)ev.cfg.nx * ev.cfg.ny * ev.cfg.neta;
    ev.viscous = ev.cfg.eta_over_s > 0.0;
    off += ev.N;
  }
  // default policy: the largest tiles the thread limit allows, x chunks of about 32 planes
  cudaError_t err = h->rsize == 8 ? batch_upload<double>(h) : batch_upload<float>(h);
  if (err == cudaSuccess) err = batch_schedule(h, CLV_TILE_MAX_THREADS, 32, sms, smem_max);
  if (err == cudaSuccess) err = cudaMalloc((void**)&h->batch_ctr, 2 * sizeof(int));
  if (err != cudaSuccess) {
    clv_destroy(h);
    *out = nullptr;
    return fail(nullptr, CLV_ECUDA, std::string("batch setup: ") + cudaGetErrorString(err));
  }
  return CLV_OK;
}

clv_status clv_batch_size(const clv_handle* h, int* nevents, int64_t* cells) {
  if (!h) return CLV_EINVAL;
  if (nevents) *nevents = (int)h->batch.size();
  if (cells) {
    long long nc = 0;
    for (const auto& ev : h->batch) nc += ev.Nc;
    *cells = h->batch.empty() ? h->Nc : nc;
  }
  return CLV_OK;
}

clv_status clv_batch_set_initial(clv_handle* h, int event, const double* eps, const double* ux, const double* uy,
                                 const double* ueta, const double* pi) {
  if (!h) return CLV_EINVAL;
  if (h->batch.empty()) return fail(h, CLV_EINVAL, "not a batch (clv_create_batch)");
  if (event < 0 || event >= (int)h->batch.size()) return fail(h, CLV_EINVAL, "event index out of range");
  if (h->initialized) return fail(h, CLV_EINVAL, "the batch has started; create a new one");
  if (!eps || !ux || !uy || !ueta) return fail(h, CLV_EINVAL, "eps, ux, uy and ueta are required");
  auto& ev = h->batch[event];
  const double* in[4] = {eps, ux, uy, ueta};
  clv_status s =
      h->rsize == 8 ? load_initial_range<double>(h, ev.off, ev.N, ev.Nc, ev.cfg.neta, ev.nep, ev.viscous, in, pi, true)
                    : load_initial_range<float>(h, ev.off, ev.N, ev.Nc, ev.cfg.neta, ev.nep, ev.viscous, in, pi, true);
  if (s == CLV_OK) ev.set = true;
  return s;
}

clv_status clv_batch_get_fields(clv_handle* h, int event, uint32_t mask, double* host_out) {
  if (!h) return CLV_EINVAL;
  if (h->batch.empty()) return fail(h, CLV_EINVAL, "not a batch (clv_create_batch)");
  if (event < 0 || event >= (int)h->batch.size()) return fail(h, CLV_EINVAL, "event index out of range");
  const auto& ev = h->batch[event];
  return get_fields_range(h, mask, host_out, true, ev.off, ev.Nc, ev.cfg.neta, ev.nep);
}

clv_status clv_batch_set_schedule(clv_handle* h, int max_threads, int chunk) {
  if (!h) return CLV_EINVAL;
  if (h->batch.empty()) return fail(h, CLV_EINVAL, "not a batch (clv_create_batch)");
  if (max_threads < 32 || max_threads > CLV_TILE_MAX_THREADS || chunk < 1 || chunk > 4096)
    return fail(h, CLV_EINVAL, "max_threads must be in [32, 256] and chunk in [1, 4096]");
  size_t smem_max = 0;
  const int sms = device_sms(&smem_max);
  const cudaError_t e = batch_schedule(h, max_threads, chunk, sms, smem_max);
  if (e == cudaErrorInvalidValue) return fail(h, CLV_EINVAL, "a tile of this policy exceeds the shared memory of a CTA");
  CLV_CUDA(h, e);
  return CLV_OK;
}

clv_status clv_batch_event_stats(clv_handle* h, int event, clv_stats* out) {
  if (!h || !out) return CLV_EINVAL;
  if (h->batch.empty()) return fail(h, CLV_EINVAL, "not a batch (clv_create_batch)");
  if (event < 0 || event >= (int)h->batch.size()) return fail(h, CLV_EINVAL, "event index out of range");
  if (!h->initialized) return fail(h, CLV_EINVAL, "the batch has not started (clv_step)");
  const auto& ev = h->batch[event];
  const unsigned g = grid_of(ev.N);
  CLV_CUDA(h, cudaMemsetAsync(&h->dstats->emax_bits, 0, sizeof(unsigned long long), h->stream));
  if (h->rsize == 8) {
    stats_scan_kernel<double><<<g, kBlock, 0, h->stream>>>((const double*)h->PR[h->cur][0] + ev.off,
                                                           (const double*)h->T0[0] + ev.off, nullptr, ev.N,
                                                           h->block_sum, &h->dstats->emax_bits);
  } else {
    stats_scan_kernel<float><<<g, kBlock, 0, h->stream>>>((const float*)h->PR[h->cur][0] + ev.off,
                                                          (const float*)h->T0[0] + ev.off,
                                                          (const float*)h->TL0[0] + ev.off, ev.N, h->block_sum,
                                                          &h->dstats->emax_bits);
  }
  h->stat_blocks = (int)g;
  clv_status s = h->rsize == 8 ? reduce_stats<double>(h, false, out) : reduce_stats<float>(h, false, out);
  double esum = 0.0;
  cudaMemcpy(&esum, &h->dstats->esum, sizeof(double), cudaMemcpyDeviceToHost);
  out->E_tot = esum * ev.cfg.dx * ev.cfg.dy * ev.cfg.deta;
  return s;
}

clv_status clv_enable_kernel_timing(clv_handle* h, int enable) {
  if (!h) return CLV_EINVAL;
  h->timing = enable != 0;
  return CLV_OK;
}

clv_status clv_get_kernel_times(clv_handle* h, double ms[4], int64_t launches[4]) {
  if (!h || !ms || !launches) return CLV_EINVAL;
  CLV_CUDA(h, cudaStreamSynchronize(h->stream));
  const bool direct = h->cfg.kernel == 1;
  for (size_t i = 0; i + kEventsPerStep - 1 < h->ev_pending.size(); i += kEventsPerStep) {
    for (int k = 0; k < 4; ++k) {
      float a = 0.f;
      CLV_CUDA(h, cudaEventElapsedTime(&a, h->ev_pending[i + k], h->ev_pending[i + k + 1]));
      h->t_ms[k] += a;
      if (!(direct && (k & 1))) h->t_launches[k] += 1;
    }
  }
  for (cudaEvent_t e : h->ev_pending) h->ev_pool.push_back(e);
  h->ev_pending.clear();
  for (int i = 0; i < 4; ++i) {
    ms[i] = h->t_ms[i];
    launches[i] = h->t_launches[i];
    h->t_ms[i] = 0.0;
    h->t_launches[i] = 0;
  }
  return CLV_OK;
}

// ---- freeze-out surface: the handle's state as slices (clv_fo_find is in clv_freezeout.cu)

clv_status clv_fo_grid_of(clv_handle* h, clv_fo_grid* out) {
  if (!h || !out) return fail(h, CLV_EINVAL, "handle or out is NULL");
  if (!h->batch.empty() || h->cfg.halo_x)
    return fail(h, CLV_EINVAL, "freeze-out slices: single-event handles only (not a batch or an x-slab)");
  if (h->cfg.nx < 2 || h->cfg.ny < 2 || h->cfg.neta < 2)
    return fail(h, CLV_EINVAL, "freeze-out slices need nx, ny, neta >= 2");
  out->nx = h->cfg.nx;
  out->ny = h->cfg.ny;
  out->neta = h->cfg.neta;
  out->eta_pitch = h->nep;
  out->dx = h->cfg.dx;
  out->dy = h->cfg.dy;
  out->deta = h->cfg.deta;
  out->precision = h->cfg.precision;
  out->cartesian = h->cfg.cartesian;
  return CLV_OK;
}

clv_status clv_fo_current(clv_handle* h, clv_fo_slice* out) {
  clv_fo_grid g;
  clv_status s = clv_fo_grid_of(h, &g);
  if (s != CLV_OK) return s;
  if (!h->initialized) return fail(h, CLV_EINVAL, "clv_set_initial was not called");
  out->tau = h->tau;
  out->eps = h->PR[h->cur][0];
  for (int m = 0; m < 3; ++m) out->u[m] = h->PR[h->cur][1 + m];
  for (int q = 0; q < 10; ++q) out->pi[q] = h->viscous ? h->PI0[q] : nullptr;
  return CLV_OK;
}

clv_status clv_fo_slice_bytes(clv_handle* h, size_t* bytes) {
  clv_fo_grid g;
  clv_status s = clv_fo_grid_of(h, &g);
  if (s != CLV_OK) return s;
  if (!bytes) return fail(h, CLV_EINVAL, "bytes is NULL");
  *bytes = 14 * align_up((size_t)h->N * h->rsize, 256);
  return CLV_OK;
}

clv_status clv_fo_snapshot(clv_handle* h, void* d_buf, clv_fo_slice* out) {
  clv_fo_slice cur;
  clv_status s = clv_fo_current(h, &cur);
  if (s != CLV_OK) return s;
  if (!d_buf || (reinterpret_cast<uintptr_t>(d_buf) & 255)) return fail(h, CLV_EINVAL, "d_buf is NULL or not 256-byte aligned");
  if (!out) return fail(h, CLV_EINVAL, "out is NULL");
  const size_t fb = align_up((size_t)h->N * h->rsize, 256), n = (size_t)h->N * h->rsize;
  char* b = static_cast<char*>(d_buf);
  const void* src[14] = {cur.eps, cur.u[0], cur.u[1], cur.u[2]};
  for (int q = 0; q < 10; ++q) src[4 + q] = cur.pi[q];
  const int nf = h->viscous ? 14 : 4;
  for (int f = 0; f < nf; ++f) CLV_CUDA(h, cudaMemcpyAsync(b + f * fb, src[f], n, cudaMemcpyDeviceToDevice, h->stream));
  out->tau = cur.tau;
  out->eps = b;
  for (int m = 0; m < 3; ++m) out->u[m] = b + (1 + m) * fb;
  for (int q = 0; q < 10; ++q) out->pi[q] = h->viscous ? b + (4 + q) * fb : nullptr;
  return CLV_OK;
}

void clv_destroy(clv_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  for (cudaEvent_t e : h->ev_pending) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  invalidate_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaFree(h->batch_geom);
  cudaFree(h->batch_tiles);
  cudaFree(h->batch_items);
  cudaFree(h->batch_ctr);
  delete h;
}

const char* clv_last_error(const clv_handle* h) {
  return h ? h->last_error.c_str() : g_create_error.c_str();
}

const char* clv_version(void) { return "clv-gb300 0.1 (sm_103a)"; }

}  // extern "C"
