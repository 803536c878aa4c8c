// clv_tile.cuh -- tiled stage kernel.
//
// A CTA owns a (y, eta_s) tile of TJ x TK cells and marches along x over a
// chunk of CX planes.  Per plane:
//   1. the tile plus a two-cell halo in y and eta_s is staged once in shared
//      memory as the per-cell reconstruction fields (T~, pi~, u~^tau, v, P, c_s),
//      by cp.async one plane ahead, together with the per-cell inputs of the
//      cell that plane's iteration outputs;
//   2. every y- and eta_s-interface flux of the tile is computed once: the
//      block has (TJ+1) x (TK+1) threads, thread (a, b) computes the
//      y-interface below row a of column b and the eta_s-interface left of
//      column b of row a, so each thread does at most one interface per axis;
//   3. each cell thread forms its y/eta_s flux differences and the y/eta_s
//      derivatives of u~, which wait in shared memory for two planes.
// The x-direction stencil lives in a register window over the thread's own
// column: every x-interface is computed once, when the plane two cells to its
// right arrives.
#pragma once
#include "clv_kernels.cuh"

namespace clv {

template <bool VISC> struct Box {
  static constexpr int UT = VISC ? 14 : 4;  // u~^tau
  static constexpr int V = UT + 1;          // v^x, v^y, v^eta
  static constexpr int P = UT + 4;
  static constexpr int CS = UT + 5;
  static constexpr int NF = UT + 6;         // staged fields per cell
  static constexpr int NQ = VISC ? 14 : 4;  // conserved components
  static constexpr int NR = NRec<VISC>::n;  // reconstructed per interface
  static constexpr int NDU = VISC ? 8 : 0;  // d~_y u~^b, d~_eta u~^b
  static constexpr int NPEND = NQ + NDU;
};

struct TileArgs {
  int TJ, TK, CX;     // tile rows (y), tile columns (eta), planes per chunk (x)
  int ntj, ntk;       // tiles per plane
};

// Grid of one event: its cells start at `off` in every field array (one
// event: off = 0; a batch stores its events back to back).
template <typename R> struct EventGeom {
  long long off;
  int nx, ny, ne;
  int nep;            // eta pitch (ne rounded up to a multiple of 4)
  R inv_dx, inv_dy;
  IsCoef<R> is;
  double deta;
  int viscous;        // batch: 1 if the event has eta/s > 0
};

// Per-cell inputs of the output cell that are not staged with the planes
// (eps, u~^{n-1}; in stage 2 also u~^n, T~^n, pi~^n), prefetched one plane
// ahead into a per-thread slot: the copies for the next output cell are
// issued right after this thread has consumed the slot for the current one.  FF (the FP32 path, whose T~ is a
// float-float pair): also the low parts of the stage's input T~ and, in stage
// 2, of T~^n (the staged planes carry the high parts only).
template <int STAGE, bool VISC, bool FF> struct CellIn {
  static constexpr int E = 0;
  static constexpr int UP = 1;                       // u~^{n-1} (VISC)
  static constexpr int UN = VISC ? 4 : 1;            // u~^n (stage 2)
  static constexpr int TN = UN + 3;                  // T~^n (stage 2; FF: high parts)
  static constexpr int PIN = TN + 4;                 // pi~^n (stage 2, VISC)
  static constexpr int TL = STAGE == 1 ? (VISC ? 4 : 1) : (VISC ? PIN + 10 : TN + 4);   // FF: low parts of T~
  static constexpr int TNL = TL + 4;                 // FF, stage 2: low parts of T~^n
  static constexpr int n = TL + (FF ? (STAGE == 1 ? 4 : 8) : 0);
};

// Row width of the staged box (in cells): the tile's TK columns with a
// two-cell halo on each side, widened so that the box starts at a multiple of
// 4 columns (rows of the layout are 16-byte aligned) and holds whole
// 4-cell vectors: round_up(TK + 7, 4).
__host__ __device__ constexpr int box_width(int TK) { return (TK + 10) & ~3; }

// shared memory of one CTA, in bytes (sized for stage 2, which prefetches the
// most per-cell inputs): two plane buffers, the y/eta interface fluxes, the
// pending y/eta flux differences, the per-cell prefetch (one slot per cell)
// and the vector table
template <bool VISC> inline size_t tile_smem_bytes(int TJ, int TK, size_t rsize) {
  using L = Box<VISC>;
  const size_t NB = (size_t)(TJ + 4) * box_width(TK);
  const size_t ncell = (size_t)TJ * TK;
  const size_t nin = rsize == 4 ? CellIn<2, VISC, true>::n : CellIn<2, VISC, false>::n;
  const size_t elems = 2 * L::NF * NB + (size_t)L::NQ * ((TJ + 1) * TK + TJ * (TK + 1)) + 2 * (size_t)L::NPEND * ncell +
                       nin * ncell;
  return elems * rsize + 16 + NB * sizeof(int);   // vector table (NB / 4 int4) after up to 15 bytes of alignment
}

// Asynchronous copy of one 4-cell vector (16 bytes per 4 floats, two 16-byte
// copies per 4 doubles): both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async_vec4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_vec4(double* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa + 16u), "l"(gmem + 2) : "memory");
}

// Issue the asynchronous copies of the plane at offset poff (event offset +
// plane index x ny x nep) of the tile's box into a box buffer of NB cells per
// field: T~, pi~, P, c_s to their slots, u~ into the v slots (the conversion
// pass turns them into u~^tau and v once the copies land).  The box is made
// of 4-cell vectors (vector w = box cells 4w .. 4w + 3); voff[w] holds the
// in-plane offset of a vector inside the grid's eta range (.y < 0: one
// vector copy) or the four offsets, clamped or wrapped at the boundary, of a
// vector that crosses it.  Thread tid handles vectors w = tid, tid + nthr,
// ... < nvec; the caller commits the group.
template <typename R, bool VISC>
__device__ __forceinline__ void stage_plane_async(const StageParams<R>& p, R* box, int nvec, long long poff,
                                                  const int4* voff, int tid, int nthr, int NB) {
  using L = Box<VISC>;
  for (int w = tid; w < nvec; w += nthr) {
    const int4 o = voff[w];
    R* d = box + 4 * w;
    auto copy = [&](R* dst, const R* src) {
      if (o.y < 0) {
        cp_async_vec4(dst, src + poff + o.x);
      } else {
        cp_async_elem(dst, src + poff + o.x);
        cp_async_elem(dst + 1, src + poff + o.y);
        cp_async_elem(dst + 2, src + poff + o.z);
        cp_async_elem(dst + 3, src + poff + o.w);
      }
    };
#pragma unroll
    for (int m = 0; m < 4; ++m) copy(d + m * NB, p.T[m]);
    if constexpr (VISC) {
#pragma unroll
      for (int r = 0; r < 10; ++r) copy(d + (4 + r) * NB, p.pi[r]);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) copy(d + (L::V + m) * NB, p.pr.u[m]);
    copy(d + L::P * NB, p.pr.P);
    copy(d + L::CS * NB, p.pr.cs);
  }
}

// Prefetch of the per-cell inputs of global cell gc into slot cb (stride ncell).
template <typename R, int STAGE, bool VISC>
__device__ __forceinline__ void prefetch_cell(const StageParams<R>& p, R* cb, int ncell, long long gc) {
  using C = CellIn<STAGE, VISC, sizeof(R) == 4>;
  cp_async_elem(cb + C::E * ncell, p.pr.e + gc);
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int m = 0; m < 4; ++m) cp_async_elem(cb + (C::TL + m) * ncell, p.Tl[m] + gc);
    if constexpr (STAGE == 2) {
#pragma unroll
      for (int m = 0; m < 4; ++m) cp_async_elem(cb + (C::TNL + m) * ncell, p.Tnl[m] + gc);
    }
  }
  if constexpr (VISC) {
#pragma unroll
    for (int m = 0; m < 3; ++m) cp_async_elem(cb + (C::UP + m) * ncell, p.up[m] + gc);
  }
  if constexpr (STAGE == 2) {
#pragma unroll
    for (int m = 0; m < 3; ++m) cp_async_elem(cb + (C::UN + m) * ncell, p.un[m] + gc);
#pragma unroll
    for (int m = 0; m < 4; ++m) cp_async_elem(cb + (C::TN + m) * ncell, p.Tn[m] + gc);
    if constexpr (VISC) {
#pragma unroll
      for (int r = 0; r < 10; ++r) cp_async_elem(cb + (C::PIN + r) * ncell, p.pin[r] + gc);
    }
  }
}

// component q of the reconstruction vector along axis a from staged fields
template <bool VISC, typename R>
__device__ __forceinline__ R rec_comp(const R* f, int q, int a) {
  using L = Box<VISC>;
  constexpr int IU = L::UT;
  if (q < IU) return f[q];
  if (q == IU) return f[L::UT];
  if (q == IU + 1) return f[L::V + a - 1];
  return f[L::P];
}

// Interface flux between box cells c - stride and c, reading cells
// c - 2 stride .. c + stride (minmod slopes at both sides).
template <typename R, bool VISC>
__device__ __forceinline__ void box_interface(const R* box, int NB, int c, int stride, int ax, R taus,
                                              R* H) {
  using L = Box<VISC>;
  constexpr int NR = L::NR;
  R Ls[NR], Rs[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int f = q < L::UT ? q : (q == L::UT ? L::UT : (q == L::UT + 1 ? L::V + ax - 1 : L::P));
    const R* col = box + f * NB + c;
    const R v0 = col[-2 * stride], v1 = col[-stride], v2 = col[0], v3 = col[stride];
    Ls[q] = v1 + R(0.5) * minmod(v1 - v0, v2 - v1);
    Rs[q] = v2 - R(0.5) * minmod(v2 - v1, v3 - v2);
  }
  const R* cs = box + L::CS * NB + c;
  interface_flux<R, VISC>(Ls, Rs, cs[-stride], cs[0], ax, taus, H);
}

// Thread cap of a stage-kernel CTA.  FP32: 384 threads (12 warps) fit the
// register file at the 168 registers that bound allows; a CTA of at most 192
// threads then leaves room for a second one on the SM, when its shared
// memory fits too.  FP64: 128 threads (255 registers).
#ifndef CLV_TILE_MAX_THREADS
#define CLV_TILE_MAX_THREADS 384
#endif
template <typename R> struct TileBound {
  static constexpr int threads = sizeof(R) == 4 ? CLV_TILE_MAX_THREADS : (CLV_TILE_MAX_THREADS < 128 ? CLV_TILE_MAX_THREADS : 128);
};

// One tile-chunk (index bidx within its event) of a stage; every thread of
// the block calls it (threads beyond the tile's (TJ+1)(TK+1) only take part
// in the barriers).
template <typename R, int STAGE, bool VISC>
__device__ __forceinline__ void stage_tile_body(const StageParams<R>& p, const EventGeom<R>& ev, const TileArgs& t,
                                                int bidx, unsigned char* smem_raw) {
  using L = Box<VISC>;
  constexpr int NF = L::NF, NQ = L::NQ, NR = L::NR, NPEND = L::NPEND;
  const int BW = box_width(t.TK), NB = BW * (t.TJ + 4), NV = NB / 4;
  const int NHY = (t.TJ + 1) * t.TK, NHK = t.TJ * (t.TK + 1);
  const int ncell = t.TJ * t.TK;
  R* boxbuf = reinterpret_cast<R*>(smem_raw);   // two plane buffers [2][NF][NB]
  R* Hy = boxbuf + 2 * NF * NB;  // [NQ][TJ+1][TK]
  R* Hk = Hy + NQ * NHY;       // [NQ][TJ][TK+1]
  R* pend = Hk + NQ * NHK;     // [2][NPEND][ncell]
  using CI = CellIn<STAGE, VISC, sizeof(R) == 4>;
  R* cellbuf = pend + 2 * NPEND * ncell;             // [CI::n][ncell]
  // [NV] vector table, 16-byte aligned (int4 accesses)
  int4* voff = reinterpret_cast<int4*>(
      (reinterpret_cast<uintptr_t>(cellbuf + CellIn<2, VISC, sizeof(R) == 4>::n * ncell) + 15) &
      ~static_cast<uintptr_t>(15));

  const int nthr = (t.TJ + 1) * (t.TK + 1);
  const bool worker = threadIdx.x < nthr;
  // threads beyond the tile act as a copy of thread 0 that skips every
  // shared-memory write and every output (only the barriers need them)
  const int tid = worker ? (int)threadIdx.x : 0;
  const int ta = tid / (t.TK + 1), tb = tid - ta * (t.TK + 1);
  const int tkt = bidx % t.ntk;
  bidx /= t.ntk;
  const int tjt = bidx % t.ntj;
  const int ch = bidx / t.ntj;
  const int j0 = tjt * t.TJ, k0 = tkt * t.TK, x0 = ch * t.CX;
  const int kb0 = ((k0 - 2) >> 2) << 2;   // first box column: k0 - 2 rounded down to a multiple of 4
  const int coff = k0 - kb0;              // box column of the tile's first column (2..5)
  const int x1 = min(x0 + t.CX, ev.nx);
  const bool is_cell = worker && ta < t.TJ && tb < t.TK;
  const int j = j0 + ta, k = k0 + tb;
  const bool active = is_cell && j < ev.ny && k < ev.ne;
  const int cid = ta * t.TK + tb;                  // cell slot (valid when is_cell)
  const int center = (ta + 2) * BW + (tb + coff);  // box cell of (ta, tb)
  const TauS<R> ts = tau_scalars(p, STAGE);
  const R taus = ts.taus;
  const R inv_dx = ev.inv_dx;
  const R inv_dy = ev.inv_dy;
  const R inv_de = (R)(1.0 / (ts.taus_d * ev.deta));   // 1/(tau deta)

  R W0[NF], W1[NF];      // staged fields of the own column at planes pl-2, pl-1
  R S0[NR];              // x-slope at plane pl-2
  R Hprev[NQ];           // x-interface flux at c - 1/2
  R ucm1[4];             // u~ at plane c - 1
#pragma unroll
  for (int f = 0; f < NF; ++f) { W0[f] = R(0); W1[f] = R(0); }
#pragma unroll
  for (int q = 0; q < NR; ++q) S0[q] = R(0);
#pragma unroll
  for (int q = 0; q < NQ; ++q) Hprev[q] = R(0);
#pragma unroll
  for (int m = 0; m < 4; ++m) ucm1[m] = R(0);


  // in-plane offsets of this thread's box vectors (only this thread uses them)
  const int vend = worker ? NV : 0;   // vectors this thread stages: w = tid, tid + nthr, ... < vend
  for (int w = tid; w < vend; w += nthr) {
    const int bj = (4 * w) / BW, c0 = kb0 + 4 * w - bj * BW;
    const int row = wrap_index(j0 + bj - 2, ev.ny, p.periodic) * ev.nep;
    if (c0 >= 0 && c0 + 3 < ev.ne)
      voff[w] = make_int4(row + c0, -1, 0, 0);
    else
      voff[w] = make_int4(row + wrap_index(c0, ev.ne, p.periodic), row + wrap_index(c0 + 1, ev.ne, p.periodic),
                          row + wrap_index(c0 + 2, ev.ne, p.periodic), row + wrap_index(c0 + 3, ev.ne, p.periodic));
  }
  const long long plane = (long long)ev.ny * ev.nep;
  // x planes beyond the grid: clamped or wrapped, or (an x-slab) the stored halo planes
  auto xplane = [&](int x) { return p.xhalo ? x : wrap_index(x, ev.nx, p.periodic); };
  // Copy groups of a thread alternate: a plane group, then a cell group
  // (the per-cell inputs of its next output cell), each possibly empty, so
  // that waiting for all but the newest group lands exactly the one needed.
  stage_plane_async<R, VISC>(p, boxbuf + ((x0 - 2) & 1) * NF * NB, vend, ev.off + xplane(x0 - 2) * plane, voff, tid,
                             nthr, NB);
  cp_async_commit();
  cp_async_commit();   // no cell group before the first plane
  for (int pl = x0 - 2; pl <= x1 + 1; ++pl) {
    const bool out_plane = pl >= x0 && pl < x1;
    R* box = boxbuf + (pl & 1) * NF * NB;
    // ---- 1. this thread's copies of plane pl have landed (the cell group
    // committed after them may still be in flight): its u~ -> (u~^tau, v) in
    // place, then one barrier makes the whole plane visible
    cp_async_wait_prior();
    for (int w = tid; w < vend; w += nthr) {   // the cells of its vectors
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = 4 * w + i;
        const R ux = box[L::V * NB + q], uy = box[(L::V + 1) * NB + q], ue = box[(L::V + 2) * NB + q];
        const R ut = sqrt(R(1) + ux * ux + uy * uy + ue * ue);
        const R iu = R(1) / ut;
        box[L::UT * NB + q] = ut;
        box[L::V * NB + q] = ux * iu;
        box[(L::V + 1) * NB + q] = uy * iu;
        box[(L::V + 2) * NB + q] = ue * iu;
      }
    }
    __syncthreads();
    // prefetch the next plane into the other buffer while this one is used
    if (pl + 1 <= x1 + 1)
      stage_plane_async<R, VISC>(p, boxbuf + ((pl + 1) & 1) * NF * NB, vend,
                                 ev.off + xplane(pl + 1) * plane, voff, tid, nthr, NB);
    cp_async_commit();
    // ---- 2. every y- and eta-interface of an output plane, once
    if (out_plane) {
      R H[NQ];
      if (worker && tb < t.TK) {   // y-interface between rows ta-1 and ta of column tb
        box_interface<R, VISC>(box, NB, (ta + 2) * BW + tb + coff, BW, 2, taus, H);
#pragma unroll
        for (int q = 0; q < NQ; ++q) Hy[q * NHY + ta * t.TK + tb] = H[q];
      }
      if (worker && ta < t.TJ) {   // eta-interface between columns tb-1 and tb of row ta
        box_interface<R, VISC>(box, NB, (ta + 2) * BW + tb + coff, 1, 3, taus, H);
#pragma unroll
        for (int q = 0; q < NQ; ++q) Hk[q * NHK + ta * (t.TK + 1) + tb] = H[q];
      }
      __syncthreads();
    }
    if (is_cell) {
      R Wn[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) Wn[f] = box[f * NB + center];
      const int it = pl - (x0 - 2);
      if (it >= 2) {
        // x-slope at plane pl-1
        R S1[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const R a = rec_comp<VISC>(W0, q, 1), m = rec_comp<VISC>(W1, q, 1), c = rec_comp<VISC>(Wn, q, 1);
          S1[q] = minmod(m - a, c - m);
        }
        if (it >= 3) {
          // x-interface between planes pl-2 and pl-1
          R Ls[NR], Rs[NR], H[NQ];
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            Ls[q] = rec_comp<VISC>(W0, q, 1) + R(0.5) * S0[q];
            Rs[q] = rec_comp<VISC>(W1, q, 1) - R(0.5) * S1[q];
          }
          interface_flux<R, VISC>(Ls, Rs, W0[L::CS], W1[L::CS], 1, taus, H);
          if (it >= 4 && active) {
            // ============ output cell c = pl - 2 (own fields: W0) ============
            const int c = pl - 2;
            const long long gc = ev.off + ((long long)c * ev.ny + j) * ev.nep + k;
            const R* pd = pend + (size_t)(c & 1) * NPEND * ncell;
            cp_async_wait_prior();   // the cell group, older than the plane group just committed
            const R* cb = cellbuf + cid;
            R S[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) S[q] = pd[q * ncell + cid] - (H[q] - Hprev[q]) * inv_dx;
            const R e = cb[CI::E * ncell];
            const R Pc = W0[L::P];   // the pressure of T^{mu nu}: P(eps) + Pi
            R Pe = Pc;               // the EOS pressure P(eps) (shear source and regulator)
            R u[4];
            u[0] = W0[L::UT];
            u[1] = mul_rn(u[0], W0[L::V]);
            u[2] = mul_rn(u[0], W0[L::V + 1]);
            u[3] = mul_rn(u[0], W0[L::V + 2]);
            {
              R Tee = e * u[3] * u[3] + Pc * (R(1) + u[3] * u[3]);
              if constexpr (VISC) Tee += W0[4 + 9];
              S[0] -= p.st_tau * Tee;
              S[3] -= ts.geo * W0[3];
            }
            R un[4];
            if constexpr (STAGE == 1) {
#pragma unroll
              for (int b2 = 0; b2 < 4; ++b2) un[b2] = u[b2];
            } else {
              un[1] = cb[CI::UN * ncell]; un[2] = cb[(CI::UN + 1) * ncell]; un[3] = cb[(CI::UN + 2) * ncell];
              un[0] = sqrt(R(1) + un[1] * un[1] + un[2] * un[2] + un[3] * un[3]);
            }
            R ustar0 = un[0];
            if constexpr (VISC) {
              const R us1 = R(2) * un[1] - cb[CI::UP * ncell];
              const R us2 = R(2) * un[2] - cb[(CI::UP + 1) * ncell];
              const R us3 = R(2) * un[3] - cb[(CI::UP + 2) * ncell];
              ustar0 = sqrt(R(1) + us1 * us1 + us2 * us2 + us3 * us3);
              R ul[4];
              if constexpr (STAGE == 1) {
                ul[0] = ustar0; ul[1] = us1; ul[2] = us2; ul[3] = us3;
              } else {
#pragma unroll
                for (int b2 = 0; b2 < 4; ++b2) ul[b2] = u[b2];
              }
              R du[4][4];
              const R invh = p.inv_h;
              const R half_dx = R(0.5) * inv_dx;
              R up1[4];
              up1[0] = W1[L::UT];
              up1[1] = mul_rn(up1[0], W1[L::V]);
              up1[2] = mul_rn(up1[0], W1[L::V + 1]);
              up1[3] = mul_rn(up1[0], W1[L::V + 2]);
#pragma unroll
              for (int b2 = 0; b2 < 4; ++b2) {
                du[0][b2] = (ul[b2] - un[b2]) * invh;
                du[1][b2] = (up1[b2] - ucm1[b2]) * half_dx;
                du[2][b2] = pd[(NQ + b2) * ncell + cid];
                du[3][b2] = pd[(NQ + 4 + b2) * ncell + cid];
              }
              R Tc, c2d;
              eos_eval<R, R>(p.eos, e, Pe, Tc, c2d);
              const R inv_taupi = Tc * ev.is.inv_b_etas_hbarc;
              R pic[10], Spi[10];
#pragma unroll
              for (int r = 0; r < 10; ++r) pic[r] = W0[4 + r];
              shear_source<R>(ts.geo, u, du, pic, e, Pe, inv_taupi, ev.is, Spi);
#pragma unroll
              for (int r = 0; r < 10; ++r) S[4 + r] += Spi[r];
            }
            // ---- stage update (Sec. 3).  FP32 path: T~ is a float-float
            // pair (high part staged in W0, low part prefetched) and the
            // increment h S is added to it exactly (Tnl: the new low parts)
            const R hh = p.h;
            R Tnew[4], Tnl[4], pinew[10];
            if constexpr (STAGE == 1) {
#pragma unroll
              for (int m = 0; m < 4; ++m) {
                if constexpr (sizeof(R) == 4) {
                  const ff s = ff_add(ff{W0[m], cb[(CI::TL + m) * ncell]}, mul_rn(hh, S[m]));
                  Tnew[m] = s.hi;
                  Tnl[m] = s.lo;
                } else {
                  Tnew[m] = W0[m] + hh * S[m];
                }
              }
              if constexpr (VISC) {
                const R inv = R(1) / ustar0;
#pragma unroll
                for (int r = 0; r < 10; ++r) pinew[r] = (un[0] * W0[4 + r] + hh * S[4 + r]) * inv;
                regulate_shear<R>(e, Pe, pinew);
              }
            } else {
#pragma unroll
              for (int m = 0; m < 4; ++m) {
                if constexpr (sizeof(R) == 4) {
                  const ff s = ff_add(ff_add(ff{cb[(CI::TN + m) * ncell], cb[(CI::TNL + m) * ncell]},
                                             ff{W0[m], cb[(CI::TL + m) * ncell]}),
                                      mul_rn(hh, S[m]));
                  Tnew[m] = 0.5f * s.hi;   // halving is exact
                  Tnl[m] = 0.5f * s.lo;
                } else {
                  Tnew[m] = R(0.5) * (cb[(CI::TN + m) * ncell] + W0[m] + hh * S[m]);
                }
              }
              if constexpr (VISC) {
                const R inv = R(0.5) / u[0];
#pragma unroll
                for (int r = 0; r < 10; ++r)
                  pinew[r] = (un[0] * cb[(CI::PIN + r) * ncell] + ustar0 * W0[4 + r] + hh * S[4 + r]) * inv;
                regulate_shear<R>(e, Pe, pinew);
              }
            }
            // conserved quantities of the stage; the primitive recovery runs in
            // recover_kernel (high occupancy hides its dependent table lookups)
#pragma unroll
            for (int m = 0; m < 4; ++m) p.Tout[m][gc] = Tnew[m];
            if constexpr (sizeof(R) == 4) {
#pragma unroll
              for (int m = 0; m < 4; ++m) p.Toutl[m][gc] = Tnl[m];
            }
            if constexpr (VISC) {
#pragma unroll
              for (int r = 0; r < 10; ++r) p.piout[r][gc] = pinew[r];
            }
          }
#pragma unroll
          for (int q = 0; q < NQ; ++q) Hprev[q] = H[q];
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) S0[q] = S1[q];
      }
      // shift the window; keep u~ of plane pl-2 as u(c-1) for the next output
      if constexpr (VISC) {
        ucm1[0] = W0[L::UT];
        ucm1[1] = mul_rn(W0[L::UT], W0[L::V]);
        ucm1[2] = mul_rn(W0[L::UT], W0[L::V + 1]);
        ucm1[3] = mul_rn(W0[L::UT], W0[L::V + 2]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) { W0[f] = W1[f]; W1[f] = Wn[f]; }
      // the per-cell inputs of the next output cell (pl - 1), into the slot
      // the output above has consumed (committed below); they have the next
      // iteration's interface phase to land
      if (active && pl - 1 >= x0 && pl - 1 < x1)
        prefetch_cell<R, STAGE, VISC>(p, cellbuf + cid, ncell, ev.off + ((long long)(pl - 1) * ev.ny + j) * ev.nep + k);
      // ---- 3. y and eta_s flux differences of plane pl, consumed two planes later
      if (out_plane && active) {
        R* pd = pend + (size_t)(pl & 1) * NPEND * ncell;
        const R iy = inv_dy, ie = inv_de;
        const int hy = ta * t.TK + tb, hk = ta * (t.TK + 1) + tb;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          pd[q * ncell + cid] = -(Hy[q * NHY + hy + t.TK] - Hy[q * NHY + hy]) * iy -
                                (Hk[q * NHK + hk + 1] - Hk[q * NHK + hk]) * ie;
        if constexpr (VISC) {
          // central differences d~_y u~^b and d~_eta u~^b
#pragma unroll
          for (int ax = 2; ax <= 3; ++ax) {
            const int stride = ax == 2 ? BW : 1;
            const R hinv = R(0.5) * (ax == 2 ? inv_dy : inv_de);
            const R utp = box[L::UT * NB + center + stride], utm = box[L::UT * NB + center - stride];
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) {
              const R up_ = b2 == 0 ? utp : mul_rn(utp, box[(L::V + b2 - 1) * NB + center + stride]);
              const R um_ = b2 == 0 ? utm : mul_rn(utm, box[(L::V + b2 - 1) * NB + center - stride]);
              pd[(NQ + (ax - 2) * 4 + b2) * ncell + cid] = (up_ - um_) * hinv;
            }
          }
        }
      }
    }
    cp_async_commit();   // the cell group (empty without a next output cell)
  }
}

template <typename R, int STAGE, bool VISC>
__global__ void __launch_bounds__(TileBound<R>::threads, 1)
    stage_tile_kernel(const StageParams<R> p, const TileArgs t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EventGeom<R> ev{0, p.nx, p.ny, p.ne, p.nep, p.inv_dl[0], p.inv_dl[1], p.is, p.deta_d, VISC ? 1 : 0};
  stage_tile_body<R, STAGE, VISC>(p, ev, t, blockIdx.x, smem_raw);
}

// A batch of events stored back to back: one persistent launch (a CTA per
// SM) takes work items (event, tile-chunk index), most expensive first, from
// an atomic counter until none is left.  ANY_VISC: viscous events run the
// viscous body, the others the ideal one (false: all ideal, the first-step
// predictor).  Counters only grow; no CTA waits for another.
template <typename R, int STAGE, bool ANY_VISC>
__global__ void __launch_bounds__(TileBound<R>::threads, 1)
    stage_batch_kernel(const StageParams<R> p, const EventGeom<R>* __restrict__ evs,
                       const TileArgs* __restrict__ tiles, const int2* __restrict__ items, int nitems, int* next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();   // the previous item is done with shared memory and s_item
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) return;
    const int2 w = items[it];
    const EventGeom<R> ev = evs[w.x];
    const TileArgs t = tiles[w.x];
    if (ANY_VISC && ev.viscous) stage_tile_body<R, STAGE, true>(p, ev, t, w.y, smem_raw);
    else stage_tile_body<R, STAGE, false>(p, ev, t, w.y, smem_raw);
  }
}

}  // namespace clv
