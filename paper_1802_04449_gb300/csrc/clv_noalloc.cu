// clv_noalloc.cu -- statistics reduction that allocates nothing.
//
// Some callers cannot allocate device memory: code that runs under a fixed
// device-memory budget owned by another framework's pool, or in a loop whose
// contract forbids allocation between its timing points.  For them this file
// provides clv_field_stats_noalloc: the same reduction as the statistics of
// clv_get_stats (sum of T~^{tau tau} times the cell volume, maximum eps), over
// caller-owned device arrays, with its scratch (per-block partial sums and the
// running maximum) in a file-scope device array instead of a workspace.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; each call clears the slot that must start at zero before
// using it.  Calls that overlap on the GPU (different streams, or different
// host threads, on the same device) race on the scratch array and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "clv.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxPartials = 32768;                 // one per block of kBlock cells
constexpr long long kMaxCells = (long long)kMaxPartials * kBlock;  // 8,388,608 cells
constexpr int kMaxDevices = 64;

// Scratch: kMaxPartials partial sums, then the maximum as the bits of a
// non-negative double (256 KiB + 8 bytes per device that loads the library).
static __device__ __align__(256) double g_noalloc_scratch[kMaxPartials + 1];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void noalloc_clear_kernel(double* scratch) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    reinterpret_cast<unsigned long long*>(scratch)[kMaxPartials] = 0ull;
}

__global__ void __launch_bounds__(kBlock) noalloc_partials_kernel(const double* eps, const double* Ttt,
                                                                   long long n, double* scratch) {
  __shared__ double s_sum[kBlock / 32], s_max[kBlock / 32];
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0;
  if (c < n) {
    a = Ttt[c];
    b = eps[c] > 0.0 ? eps[c] : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_sum[threadIdx.x >> 5] = a;
    s_max[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) {
      x += s_sum[w];
      y = fmax(y, s_max[w]);
    }
    scratch[blockIdx.x] = x;
    if (y > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(scratch) + kMaxPartials,
                (unsigned long long)__double_as_longlong(y));
  }
}

__global__ void __launch_bounds__(1024) noalloc_final_kernel(const double* scratch, int nparts, double volume,
                                                             double* out) {
  __shared__ double s[1024];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += scratch[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[0] * volume;
    out[1] = __longlong_as_double(
        (long long)reinterpret_cast<const unsigned long long*>(scratch)[kMaxPartials]);
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code).
// The cached address belongs to the device's primary context: after
// cudaDeviceReset the module is loaded anew and the address may change, so
// a process that resets a device must not call this entry point on it again.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

// defined in clv_api.cu: message returned by clv_last_error(NULL)
void clv_set_global_error(const char* msg);

static clv_status noalloc_fail(clv_status s, const char* msg) {
  clv_set_global_error(msg);
  return s;
}

extern "C" {

clv_status clv_field_stats_noalloc(const double* d_eps, const double* d_Ttt, int64_t n, double cell_volume,
                                   void* cuda_stream, double* d_out) {
  if (!d_eps || !d_Ttt || !d_out) return noalloc_fail(CLV_EINVAL, "d_eps, d_Ttt and d_out are required");
  if (n < 1) return noalloc_fail(CLV_EINVAL, "n must be >= 1");
  if (n > kMaxCells)
    return noalloc_fail(CLV_EINVAL, "n exceeds the no-allocation limit of 8388608 cells (32768 blocks x 256)");
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return noalloc_fail(CLV_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nparts = (int)((n + kBlock - 1) / kBlock);
  // an error left pending by earlier, unrelated work is not this call's: it
  // is reported as such and left pending (cudaPeekAtLastError does not clear it)
  e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return noalloc_fail(CLV_ECUDA, (std::string("error pending before the call: ") + cudaGetErrorString(e)).c_str());
  // each launch checked on its own (a launch error is this call's and is cleared)
  noalloc_clear_kernel<<<1, 32, 0, st>>>(scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(CLV_ECUDA, cudaGetErrorString(e));
  noalloc_partials_kernel<<<nparts, kBlock, 0, st>>>(d_eps, d_Ttt, (long long)n, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(CLV_ECUDA, cudaGetErrorString(e));
  noalloc_final_kernel<<<1, 1024, 0, st>>>(scratch, nparts, cell_volume, d_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(CLV_ECUDA, cudaGetErrorString(e));
  return CLV_OK;
}

}  // extern "C"
