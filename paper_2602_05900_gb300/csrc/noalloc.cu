// Allocation-free variant of the max-norm rescale (hotrg_rescale_noalloc).
//
// Some callers cannot call cudaMalloc: frameworks that hand all device memory to
// their own pool and forbid other allocators, processes whose device-memory
// quota is already taken by such a pool, and latency-critical loops where
// cudaMalloc's implicit device synchronisation is not acceptable.  This entry
// point lets them normalise a tensor they own by its max-norm and accumulate
// the log of the norm without the library allocating anything: its only
// scratch is the file-scope device array below, which every GPU that loads the
// library holds until the process exits.
#include <math.h>

#include <mutex>

#include "../../include/hotrg.h"

namespace {

constexpr int kNoAllocBlocks = 1024;        // partial maxima (one per block)
constexpr int kNoAllocThreads = 256;
constexpr long long kNoAllocMaxCount = 1LL << 26;   // 64 Mi doubles (512 MiB) per call
constexpr int kMaxDevices = 64;

// Scratch: kNoAllocBlocks partial maxima followed by the status word of the
// last call (8 KiB + 256 bytes).  Shared by every call on a device.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks + 32];

// Device address of g_noalloc_scratch, resolved once per device.
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__global__ void k_noalloc_partial_max(const double *T, long long count, double *partial) {
  double v = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(T[e]);
    v = (a != a) ? INFINITY : fmax(v, a);   // NaN poisons the norm
  }
  __shared__ double part[kNoAllocThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) m = fmax(m, part[w]);
    partial[blockIdx.x] = m;   // every slot in [0, gridDim.x) is written each call
  }
}

// Every block reduces the partials itself (at most 1024 values), so no second
// pass over global memory is needed; block 0 updates the log-sum and status.
__global__ void k_noalloc_scale(double *T, long long count, const double *partial, int nparts,
                                double weight, double *logsum, double *status) {
  __shared__ double s_c;
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) m = fmax(m, partial[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) s_c = m;
  }
  __syncthreads();
  const double c = s_c;
  const bool ok = (c > 0.0) && isfinite(c);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *status = ok ? 0.0 : 1.0;                // written on every call
    if (ok) *logsum += log(c) * weight;
  }
  if (!ok) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    T[e] = T[e] / c;
}

}  // namespace

extern "C" hotrg_status hotrg_rescale_noalloc(double *T, long long count, double weight,
                                              double *logsum, void *stream) {
  if (!T || !logsum || count < 1 || !isfinite(weight)) return HOTRG_EINVAL;
  if (count > kNoAllocMaxCount) return HOTRG_EINVAL;   // beyond the scratch design limit
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HOTRG_ECUDA;
  double *scratch;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HOTRG_ECUDA;
      g_scratch_addr[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long blocks = (count + kNoAllocThreads - 1) / kNoAllocThreads;
  if (blocks > kNoAllocBlocks) blocks = kNoAllocBlocks;
  const int nb = (int)blocks;
  double *partial = scratch;
  double *status = scratch + kNoAllocBlocks;
  k_noalloc_partial_max<<<nb, kNoAllocThreads, 0, s>>>(T, count, partial);
  k_noalloc_scale<<<nb, kNoAllocThreads, 0, s>>>(T, count, partial, nb, weight, logsum, status);
  if (cudaGetLastError() != cudaSuccess) return HOTRG_ECUDA;
  double h = 0.0;
  if (cudaMemcpyAsync(&h, status, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HOTRG_ECUDA;
  return h == 0.0 ? HOTRG_OK : HOTRG_ENONFINITE;
}
