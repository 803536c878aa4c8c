// clv_measure.cu -- clv_fma_rate: the fused multiply-add rate of the current
// device in FP64 or FP32, the denominator of the ALU rooflines of the FP64
// path and of the Cooper-Frye sum.  No counterpart in the paper.
//
// Every thread runs kChains independent chains a <- a * b + c for `iters`
// rounds (no chain waits on another, so the pipe stays full), on a grid of
// 8 CTAs of 256 threads per SM; one FMA counts as two flops.
#include <cuda_runtime.h>

#include <string>

#include "clv.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T> __global__ void __launch_bounds__(kThreads) fma_chain_kernel(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + 1) * T(1e-3) + T(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T> cudaError_t time_chain(int blocks, int iters, double* ms) {
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc((void**)&out, (size_t)blocks * kThreads * sizeof(T));
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 1e30f;
  // b close to 1 and c small keep the values finite and normal over any
  // number of rounds; the first launch warms the clocks up and is not kept
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, 0);
    fma_chain_kernel<T><<<blocks, kThreads>>>(out, iters, T(0.999999), T(1e-6));
    cudaEventRecord(e1, 0);
    err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    if (err == cudaSuccess && rep > 0 && t < best) best = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  *ms = best;
  return err;
}

}  // namespace

extern "C" {

clv_status clv_fma_rate(int precision, double* tflops) {
  if (!tflops || (precision != CLV_FP64 && precision != CLV_FP32)) return CLV_EINVAL;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CLV_ECUDA;
  const int blocks = 8 * sms;
  // about 10-40 ms per launch on a GB300 at either precision
  const int iters = precision == CLV_FP64 ? 2000 : 100000;
  double ms = 0.0;
  const cudaError_t err = precision == CLV_FP64 ? time_chain<double>(blocks, iters, &ms) : time_chain<float>(blocks, iters, &ms);
  if (err != cudaSuccess || !(ms > 0.0)) return CLV_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return CLV_OK;
}

}  // extern "C"
