// clv_mlp.cuh -- learned initial guess for the primitive root solve.
//
// Not part of the paper: a 10 -> 64 -> 64 -> 4 SiLU network maps features of
// a cell's ideal part (E, M) and its spatial shear components to
// (eps/E, v^x, v^y, v^eta); |v| seeds the Newton solve.  Inference runs on the
// tensor cores (BF16 mma.sync m16n8k16, FP32 accumulate) inside the recovery
// kernel; training runs in FP32 with the kernels below.
//
// Features of a cell (the same definition is used for the training samples):
//   x0 = (ln E - kLnEShift) / kLnEScale,  x1..3 = M^{x,y,eta} / E,
//   x4..9 = pi~^{xx, xy, x eta, yy, y eta, eta eta} / E, clamped to [-4, 4].
// Parameters are packed W1 (64x10) | b1 | W2 (64x64) | b2 | W3 (4x64) | b3.
#pragma once
#include <cuda_bf16.h>

#include "clv_device.cuh"

namespace clv {

constexpr int kMlpIn = 10, kMlpHid = 64, kMlpOut = 4;
constexpr int kMlpParams = kMlpHid * kMlpIn + kMlpHid + kMlpHid * kMlpHid + kMlpHid + kMlpOut * kMlpHid + kMlpOut;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpHid * kMlpIn, kOffW2 = kOffB1 + kMlpHid,
              kOffB2 = kOffW2 + kMlpHid * kMlpHid, kOffW3 = kOffB2 + kMlpHid, kOffB3 = kOffW3 + kMlpOut * kMlpHid;
constexpr float kLnEShift = -5.0f, kLnEScale = 5.0f, kFeatClamp = 4.0f;

// Tensor-core copy of the network: BF16 weights padded to the mma tiles
// (W1 64x16, W2 64x64, W3 8x64) and FP32 biases (64, 64, 8).
constexpr int kMlpW1e = 64 * 16, kMlpW2e = 64 * 64, kMlpW3e = 8 * 64;
constexpr int kMlpBf16Elems = kMlpW1e + kMlpW2e + kMlpW3e;      // 5632
constexpr int kMlpBiasElems = 64 + 64 + 8;                       // 136
constexpr size_t kMlpDeviceBytes = kMlpBf16Elems * 2 + kMlpBiasElems * 4;

// Shared-memory copy: rows padded by 8 BF16 (16 bytes) so that the eight rows
// a fragment load touches fall in distinct banks.
constexpr int kMlpS1 = 16 + 8, kMlpS2 = 64 + 8, kMlpSX = 16 + 8;   // row strides (BF16)
constexpr int kMlpSW1 = 64 * kMlpS1, kMlpSW2 = 64 * kMlpS2, kMlpSW3 = 8 * kMlpS2;
constexpr int kMlpSmemW = kMlpSW1 + kMlpSW2 + kMlpSW3;             // BF16 elements

// Cooperative copy of the network from global (compact) to shared (padded).
__device__ __forceinline__ void mlp_load_smem(const void* mlp, __nv_bfloat16* s_w, float* s_b) {
  const unsigned* gw = reinterpret_cast<const unsigned*>(mlp);   // BF16 pairs
  const float* gb = reinterpret_cast<const float*>(reinterpret_cast<const __nv_bfloat16*>(mlp) + kMlpBf16Elems);
  unsigned* sw = reinterpret_cast<unsigned*>(s_w);
  for (int i = threadIdx.x; i < kMlpBf16Elems / 2; i += blockDim.x) {
    int d;
    if (i < kMlpW1e / 2) d = (i >> 3) * (kMlpS1 / 2) + (i & 7);
    else if (i < (kMlpW1e + kMlpW2e) / 2) { const int j = i - kMlpW1e / 2; d = kMlpSW1 / 2 + (j >> 5) * (kMlpS2 / 2) + (j & 31); }
    else { const int j = i - (kMlpW1e + kMlpW2e) / 2; d = (kMlpSW1 + kMlpSW2) / 2 + (j >> 5) * (kMlpS2 / 2) + (j & 31); }
    sw[d] = gw[i];
  }
  for (int i = threadIdx.x; i < kMlpBiasElems; i += blockDim.x) s_b[i] = gb[i];
}

// silu(z) = z sigmoid(z) = z (1 + tanh(z / 2)) / 2: one hardware tanh
// (tanh.approx.f32, max relative error ~2^-11) instead of an exponential and
// a reciprocal.
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu(float z) {
  const float hz = 0.5f * z;
  return fmaf(hz, tanh_approx(hz), hz);
}

template <typename R>
__device__ __forceinline__ void mlp_features(R E, R Mx, R My, R Me, const R* pij, float* x) {
  const float iE = 1.0f / float(E);
  x[0] = (__logf(float(E)) - kLnEShift) * (1.0f / kLnEScale);
  x[1] = float(Mx) * iE;
  x[2] = float(My) * iE;
  x[3] = float(Me) * iE;
#pragma unroll
  for (int k = 0; k < 6; ++k) x[4 + k] = fminf(kFeatClamp, fmaxf(-kFeatClamp, float(pij[k]) * iE));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Four 8x8 BF16 matrices from shared memory: lane l gives the row address of
// row l & 7 of matrix l >> 3 (16 bytes, 16-byte aligned); register j of lane
// l receives elements (l >> 2, 2 (l & 3) .. + 1) of matrix j.
__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* row_addr) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(row_addr);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Forward pass of 16 cells (rows of xs, bf16 [16][kMlpSX] in shared memory)
// on one warp; writes the 4 outputs of each row to ys ([16][4] floats).
// s_w: the padded shared copy (mlp_load_smem); bias: b1[64] b2[64] b3[8].
// Fragments come from ldmatrix: the B fragments (b0, b1) of n-tile n and k
// tile kk are the 8x8 blocks (rows n*8.., columns kk*16 and kk*16 + 8) of the
// row-major [out][in] weights.
__device__ __forceinline__ void mlp_tile16(const __nv_bfloat16* xs, const __nv_bfloat16* s_w, const float* bias,
                                           float* ys, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int mi = lane >> 3, mr = lane & 7;   // matrix and row this lane addresses
  const __nv_bfloat16* w1 = s_w;
  const __nv_bfloat16* w2 = s_w + kMlpSW1;
  const __nv_bfloat16* w3 = s_w + kMlpSW1 + kMlpSW2;
  // A: rows 0-7 / 8-15 x columns 0-7 / 8-15 -> a0 (r0-7,c0-7) a1 (r8-15,c0-7) a2 (r0-7,c8-15) a3 (r8-15,c8-15)
  unsigned a[4];
  ldmatrix_x4(a, xs + (mr + 8 * (mi & 1)) * kMlpSX + 8 * (mi >> 1));
  // layer 1: 16x16 . 16x64; n-tiles in pairs: matrices (nt, c0-7) (nt, c8-15) (nt+1, c0-7) (nt+1, c8-15)
  float h[8][4];
#pragma unroll
  for (int np = 0; np < 4; ++np) {
    unsigned b[4];
    ldmatrix_x4(b, w1 + ((2 * np + (mi >> 1)) * 8 + mr) * kMlpS1 + 8 * (mi & 1));
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int nt = 2 * np + u;
      const float bl = bias[nt * 8 + 2 * t], bh = bias[nt * 8 + 2 * t + 1];
      h[nt][0] = bl; h[nt][1] = bh; h[nt][2] = bl; h[nt][3] = bh;
      mma_bf16(h[nt], a[0], a[1], a[2], a[3], b[2 * u], b[2 * u + 1]);
#pragma unroll
      for (int r = 0; r < 4; ++r) h[nt][r] = silu(h[nt][r]);
    }
  }
  // layer 2: 16x64 . 64x64 (accumulators of two n-tiles form one k-tile of A)
  float h2[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = bias[64 + nt * 8 + 2 * t], bh = bias[64 + nt * 8 + 2 * t + 1];
    h2[nt][0] = bl; h2[nt][1] = bh; h2[nt][2] = bl; h2[nt][3] = bh;
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const unsigned a0 = pack_bf16(h[2 * kk][0], h[2 * kk][1]), a1 = pack_bf16(h[2 * kk][2], h[2 * kk][3]);
    const unsigned a2 = pack_bf16(h[2 * kk + 1][0], h[2 * kk + 1][1]), a3 = pack_bf16(h[2 * kk + 1][2], h[2 * kk + 1][3]);
#pragma unroll
    for (int np = 0; np < 4; ++np) {
      unsigned b[4];
      ldmatrix_x4(b, w2 + ((2 * np + (mi >> 1)) * 8 + mr) * kMlpS2 + kk * 16 + 8 * (mi & 1));
      mma_bf16(h2[2 * np], a0, a1, a2, a3, b[0], b[1]);
      mma_bf16(h2[2 * np + 1], a0, a1, a2, a3, b[2], b[3]);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int r = 0; r < 4; ++r) h2[nt][r] = silu(h2[nt][r]);
  // layer 3: 16x64 . 64x8 (outputs 4..7 are padding); k-tiles in pairs:
  // matrices (kk, c0-7) (kk, c8-15) (kk+1, c0-7) (kk+1, c8-15) of W3's 8 rows
  float y[4];
  {
    const float bl = bias[128 + 2 * t], bh = bias[128 + 2 * t + 1];
    y[0] = bl; y[1] = bh; y[2] = bl; y[3] = bh;
  }
#pragma unroll
  for (int kp = 0; kp < 2; ++kp) {
    unsigned b[4];
    ldmatrix_x4(b, w3 + mr * kMlpS2 + (2 * kp + (mi >> 1)) * 16 + 8 * (mi & 1));
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int kk = 2 * kp + u;
      const unsigned a0 = pack_bf16(h2[2 * kk][0], h2[2 * kk][1]), a1 = pack_bf16(h2[2 * kk][2], h2[2 * kk][3]);
      const unsigned a2 = pack_bf16(h2[2 * kk + 1][0], h2[2 * kk + 1][1]),
                     a3 = pack_bf16(h2[2 * kk + 1][2], h2[2 * kk + 1][3]);
      mma_bf16(y, a0, a1, a2, a3, b[2 * u], b[2 * u + 1]);
    }
  }
  if (t < 2) {
    ys[g * 4 + 2 * t] = y[0];
    ys[g * 4 + 2 * t + 1] = y[1];
    ys[(g + 8) * 4 + 2 * t] = y[2];
    ys[(g + 8) * 4 + 2 * t + 1] = y[3];
  }
}

// ---------------------------------------------------------------------------
// Training (FP32).  One block of kMlpTrainBlock samples: every thread runs
// the forward and backward pass of one sample, keeping the activations and
// their gradients in shared memory; the parameter gradients are then formed
// as block-level products (each thread owns a slice of the 5124 parameters)
// and added to the global gradient.
// ---------------------------------------------------------------------------
constexpr int kMlpTrainBlock = 128;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// sample index of slot j of a batch: uniform in [0, n) from (seed, iter, j);
// seed = 0 selects the identity (slot j -> sample j) for full-batch gradients
__device__ __forceinline__ long long batch_index(unsigned long long seed, int iter, long long j, long long n) {
  if (seed == 0) return j;
  return (long long)(mix64(seed ^ ((unsigned long long)iter << 32) ^ (unsigned long long)j) % (unsigned long long)n);
}

// Gradient of the loss over a batch, deterministically: the launch has a
// fixed number of blocks (at most kMlpGradBlocks); block b takes the chunks
// of kMlpTrainBlock samples b, b + gridDim.x, ... in order and sums their
// parameter gradients and loss into its own row of `partial`
// ([gridDim.x][kMlpParams + 1], loss last), which mlp_reduce_kernel adds up
// in block order.  No atomics: the same inputs give the same bits.
constexpr int kMlpGradBlocks = 256;
constexpr int kMlpPartialRow = kMlpParams + 1;

static __global__ void __launch_bounds__(kMlpTrainBlock) mlp_grad_kernel(const float* __restrict__ params,
                                                                  const float* __restrict__ X,
                                                                  const float* __restrict__ Y, long long n,
                                                                  long long batch, unsigned long long seed, int iter,
                                                                  float* partial) {
  extern __shared__ float sm[];
  float* P = sm;                                   // kMlpParams
  float* sX = P + kMlpParams;                      // [10][B]
  float* sH1 = sX + kMlpIn * kMlpTrainBlock;       // [64][B]
  float* sH2 = sH1 + kMlpHid * kMlpTrainBlock;     // [64][B]
  float* sD1 = sH2 + kMlpHid * kMlpTrainBlock;     // [64][B]
  float* sD2 = sD1 + kMlpHid * kMlpTrainBlock;     // [64][B]
  float* sDY = sD2 + kMlpHid * kMlpTrainBlock;     // [4][B]
  __shared__ float s_loss[kMlpTrainBlock / 32];
  const int tid = threadIdx.x;
  for (int i = tid; i < kMlpParams; i += kMlpTrainBlock) P[i] = params[i];
  float* row = partial + (size_t)blockIdx.x * kMlpPartialRow;
  for (int i = tid; i < kMlpPartialRow; i += kMlpTrainBlock) row[i] = 0.0f;
  __syncthreads();
  for (long long chunk = blockIdx.x; chunk * kMlpTrainBlock < batch; chunk += gridDim.x) {
  const long long j = chunk * kMlpTrainBlock + tid;
  const bool valid = j < batch;
  float l = 0.0f;
  {
    float x[kMlpIn], z1[kMlpHid], z2[kMlpHid];
    float yt[kMlpOut];
    if (valid) {
      const long long s = batch_index(seed, iter, j, n);
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) x[k] = X[s * kMlpIn + k];
#pragma unroll
      for (int k = 0; k < kMlpOut; ++k) yt[k] = Y[s * kMlpOut + k];
    } else {
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) x[k] = 0.0f;
#pragma unroll
      for (int k = 0; k < kMlpOut; ++k) yt[k] = 0.0f;
    }
    for (int i = 0; i < kMlpHid; ++i) {
      float a = P[kOffB1 + i];
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) a = fmaf(P[kOffW1 + i * kMlpIn + k], x[k], a);
      z1[i] = a;
      sH1[i * kMlpTrainBlock + tid] = a / (1.0f + expf(-a));
    }
    for (int i = 0; i < kMlpHid; ++i) {
      float a = P[kOffB2 + i];
      for (int k = 0; k < kMlpHid; ++k) a = fmaf(P[kOffW2 + i * kMlpHid + k], sH1[k * kMlpTrainBlock + tid], a);
      z2[i] = a;
      sH2[i * kMlpTrainBlock + tid] = a / (1.0f + expf(-a));
    }
    const float inv_b = 1.0f / (float)batch;
    float dy[kMlpOut];
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
      float a = P[kOffB3 + o];
      for (int k = 0; k < kMlpHid; ++k) a = fmaf(P[kOffW3 + o * kMlpHid + k], sH2[k * kMlpTrainBlock + tid], a);
      const float r = valid ? a - yt[o] : 0.0f;
      l += r * r;
      dy[o] = 2.0f * r * inv_b;
      sDY[o * kMlpTrainBlock + tid] = dy[o];
    }
    for (int i = 0; i < kMlpHid; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int o = 0; o < kMlpOut; ++o) a = fmaf(P[kOffW3 + o * kMlpHid + i], dy[o], a);
      const float sg = 1.0f / (1.0f + expf(-z2[i]));
      sD2[i * kMlpTrainBlock + tid] = a * sg * (1.0f + z2[i] * (1.0f - sg));
    }
    for (int i = 0; i < kMlpHid; ++i) {
      float a = 0.0f;
      for (int k = 0; k < kMlpHid; ++k) a = fmaf(P[kOffW2 + k * kMlpHid + i], sD2[k * kMlpTrainBlock + tid], a);
      const float sg = 1.0f / (1.0f + expf(-z1[i]));
      sD1[i * kMlpTrainBlock + tid] = a * sg * (1.0f + z1[i] * (1.0f - sg));
    }
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) sX[k * kMlpTrainBlock + tid] = x[k];
  }
  // per-block loss
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((tid & 31) == 0) s_loss[tid >> 5] = l;
  __syncthreads();
  if (tid == 0) {
    float a = 0.0f;
    for (int w = 0; w < kMlpTrainBlock / 32; ++w) a += s_loss[w];
    row[kMlpParams] += a / (float)batch;
  }
  // parameter gradients: sums over the chunk's samples, added to the block's
  // row (each entry belongs to one thread)
  const int nb = (int)min((long long)kMlpTrainBlock, batch - chunk * kMlpTrainBlock);
  for (int pidx = tid; pidx < kMlpParams; pidx += kMlpTrainBlock) {
    const float *u, *v;
    if (pidx < kOffB1) { u = sD1 + (pidx / kMlpIn) * kMlpTrainBlock; v = sX + (pidx % kMlpIn) * kMlpTrainBlock; }
    else if (pidx < kOffW2) { u = sD1 + (pidx - kOffB1) * kMlpTrainBlock; v = nullptr; }
    else if (pidx < kOffB2) { const int q = pidx - kOffW2; u = sD2 + (q / kMlpHid) * kMlpTrainBlock; v = sH1 + (q % kMlpHid) * kMlpTrainBlock; }
    else if (pidx < kOffW3) { u = sD2 + (pidx - kOffB2) * kMlpTrainBlock; v = nullptr; }
    else if (pidx < kOffB3) { const int q = pidx - kOffW3; u = sDY + (q / kMlpHid) * kMlpTrainBlock; v = sH2 + (q % kMlpHid) * kMlpTrainBlock; }
    else { u = sDY + (pidx - kOffB3) * kMlpTrainBlock; v = nullptr; }
    float a = 0.0f;
    if (v) { for (int s = 0; s < nb; ++s) a = fmaf(u[s], v[s], a); }
    else { for (int s = 0; s < nb; ++s) a += u[s]; }
    row[pidx] += a;
  }
  __syncthreads();   // the next chunk overwrites the activations
  }
}

// grad = sum of the partial rows in block order (loss likewise)
static __global__ void mlp_reduce_kernel(const float* __restrict__ partial, int nblocks, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpPartialRow) return;
  float a = 0.0f;
  for (int b = 0; b < nblocks; ++b) a += partial[(size_t)b * kMlpPartialRow + p];
  if (p < kMlpParams) grad[p] = a;
  else *loss = a;
}

constexpr size_t mlp_grad_smem_bytes() {
  return (size_t)(kMlpParams + (kMlpIn + 4 * kMlpHid + kMlpOut) * kMlpTrainBlock) * sizeof(float);
}

// Adam step (Kingma & Ba 2015) on all parameters.
static __global__ void mlp_adam_kernel(float* params, float* m, float* v, float* grad, int step, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.0f - powf(b1, (float)step));
  const float vh = vi / (1.0f - powf(b2, (float)step));
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace clv
