// Error norms without any memory allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// result: their framework's memory pool may already hold (nearly) all of the
// device, so a cudaMalloc would fail or force the pool to release memory; or
// they run under a policy or in a callback (for example inside an allocator
// hook) where calling the allocator is not allowed.  elmfb_error_norms()
// allocates staging and scratch buffers per call; this variant takes device
// inputs as they are and keeps its scratch -- the per-block partial sums of
// the two reduction passes -- in a file-scope __device__ array of fixed size.
//
// The array exists once per device that loads this library and lives until
// the process exits.  Every call shares it and it keeps the previous call's
// contents; each pass writes every slot it later reads, so nothing needs
// clearing.  Calls whose kernels overlap on the GPU (different streams, no
// ordering) race on the array.  Its device address is looked up once per
// device and cached; a cudaDeviceReset() reloads the module at another
// address, so the cache does not survive a reset of that device.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "elmfb_internal.cuh"

namespace {

constexpr int kNaBlocks = 256;   // partial-sum slots of each pass
constexpr int kNaThreads = 256;
constexpr int kNaSlots = kNaBlocks * 5 + kNaBlocks;

// pass 1: [block][0..4] = sum u, sum |d|, sum d^2, sum u^2, max |d|
// pass 2: [5*kNaBlocks + block] = sum (u - mean)^2
static __device__ __align__(256) double g_noalloc_scratch[kNaSlots];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

__global__ void k_na_pass1(const double* __restrict__ uh, const double* __restrict__ ur, int64_t n,
                           double* __restrict__ part) {
  __shared__ double sh[5][kNaThreads / 32];
  double su = 0, sad = 0, sd2 = 0, su2 = 0, mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = uh[i] - ur[i];
    su += ur[i];
    sad += fabs(d);
    sd2 += d * d;
    su2 += ur[i] * ur[i];
    mx = fmax(mx, fabs(d));
  }
  double v[5] = {su, sad, sd2, su2, mx};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 5; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, t, o);
      t = k == 4 ? fmax(t, y) : t + y;
    }
    if (lane == 0) sh[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = k == 4 ? fmax(t, sh[k][w]) : t + sh[k][w];
      part[blockIdx.x * 5 + k] = t;
    }
  }
}

__global__ void k_na_pass2(const double* __restrict__ ur, int64_t n, double* __restrict__ part,
                           int nb) {
  __shared__ double sh[kNaThreads / 32];
  double su = 0.0;
  for (int b = 0; b < nb; ++b) su += part[b * 5 + 0];
  const double mean = su / (double)n;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = ur[i] - mean;
    acc += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[kNaBlocks * 5 + blockIdx.x] = t;
  }
}

// Device memory of device `dev` (the kernels read it in place, so memory of
// another GPU is refused: without peer access it is not addressable here), or
// managed memory.
bool is_device_pointer(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // the lookup's own error, raised just now
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev;
  return a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int elmfb_error_norms_noalloc(const double* u_hat, const double* u_ref, int64_t n,
                                         double* out3, void* cuda_stream) {
  if (n < 1 || !u_hat || !u_ref || !out3) return ELMFB_ERR_INVALID_ARG;
  if (n > ELMFB_NOALLOC_MAX_POINTS) return ELMFB_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ELMFB_ERR_CUDA;
  // an error left pending by earlier runtime calls is reported, not consumed
  if (cudaPeekAtLastError() != cudaSuccess) return ELMFB_ERR_CUDA;
  if (!is_device_pointer(u_hat, dev) || !is_device_pointer(u_ref, dev)) return ELMFB_ERR_INVALID_ARG;
  double* scratch = nullptr;
  {
    // one-time set-up per device, with that device current
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();   // the lookup's own error (none was pending before it)
        return ELMFB_ERR_CUDA;
      }
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nb = (int)std::min<int64_t>((n + kNaThreads - 1) / kNaThreads, kNaBlocks);
  k_na_pass1<<<nb, kNaThreads, 0, st>>>(u_hat, u_ref, n, scratch);
  if (cudaPeekAtLastError() != cudaSuccess) return ELMFB_ERR_CUDA;
  k_na_pass2<<<nb, kNaThreads, 0, st>>>(u_ref, n, scratch, nb);
  if (cudaPeekAtLastError() != cudaSuccess) return ELMFB_ERR_CUDA;
  double part[kNaSlots];
  if (cudaMemcpyAsync(part, scratch, sizeof(part), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ELMFB_ERR_CUDA;
  double sad = 0, sd2 = 0, su2 = 0, mx = 0, var = 0;
  for (int b = 0; b < nb; ++b) {
    sad += part[b * 5 + 1];
    sd2 += part[b * 5 + 2];
    su2 += part[b * 5 + 3];
    mx = std::max(mx, part[b * 5 + 4]);
    var += part[kNaBlocks * 5 + b];
  }
  const double sd = std::sqrt(var / (double)n);
  out3[0] = su2 > 0.0 ? std::sqrt(sd2 / su2) : NAN;
  out3[1] = sd > 0.0 ? sad / ((double)n * sd) : NAN;
  out3[2] = mx;
  return ELMFB_OK;
}
