// hotrg_dgemm_emu: the exact-slice tensor-core GEMM (tc_exact.cuh) as a
// stand-alone FP64 GEMM entry point (declared in include/hotrg.h).
#include <string.h>

#include <vector>

#include "../../include/hotrg.h"
#include "tc_exact.cuh"

using namespace hotrg;

namespace {

struct Scratch {
  std::vector<void *> ptrs;
  ~Scratch() {
    for (void *p : ptrs) cudaFree(p);
  }
  void *get(size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes + 256) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return p;
  }
};

hotrg_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return HOTRG_OK;
  return e == cudaErrorMemoryAllocation ? HOTRG_ENOMEM
                                        : (e == cudaErrorInvalidValue ? HOTRG_EINVAL : HOTRG_ECUDA);
}

}  // namespace

extern "C" hotrg_status hotrg_dgemm_emu(int M, int N, int K, const double *A, long long lda,
                                        const double *B, long long ldb, double *C, long long ldc,
                                        int slices, void *stream) {
  if (M < 0 || N < 0 || K < 1 || !A || !B || !C || lda < K || ldb < K || ldc < N || slices < 4 ||
      slices > 8 || M > (1 << 24) || N > (1 << 24))
    return HOTRG_EINVAL;
  if (M == 0 || N == 0) return HOTRG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc;
  const int pitch = xs_pitch(K);
  XsOperand a{sc.get(sizeof(short) * xs_elems(M, K, slices)), nullptr, M, K, pitch, slices, 1, 0, 0};
  XsOperand b{sc.get(sizeof(short) * xs_elems(N, K, slices)), nullptr, N, K, pitch, slices, 1, 0, 0};
  a.scale = static_cast<double *>(sc.get(sizeof(double) * M));
  b.scale = static_cast<double *>(sc.get(sizeof(double) * N));
  int *err = static_cast<int *>(sc.get(sizeof(int)));
  const int ksplit = xs_min_split(K);
  double *parts = ksplit > 1 ? static_cast<double *>(sc.get(sizeof(double) * ksplit * (size_t)M * N))
                             : nullptr;
  if (!a.slices || !b.slices || !a.scale || !b.scale || !err || (ksplit > 1 && !parts))
    return HOTRG_ENOMEM;
  cudaError_t e;
  PSet pa{const_cast<double *>(A), const_cast<double *>(A), 0};
  PSet pb{const_cast<double *>(B), const_cast<double *>(B), 0};
  if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) ||
      (e = xs_split(pa, map1(lda), map1(1), a, s)) || (e = xs_split(pb, map1(ldb), map1(1), b, s)))
    return from_cuda(e);
  if (ksplit == 1) {
    e = xs_gemm(a, b, M, N, K, C, map1(ldc), map1(1), 0, 1, 0, err, s);
  } else {
    e = xs_gemm(a, b, M, N, K, parts, map1(N), map1(1), 0, ksplit, (long long)M * N, err, s);
    if (e == cudaSuccess) e = xs_sum_parts(parts, ksplit, (long long)M * N, M, N, C, ldc, s);
  }
  if (e != cudaSuccess) return from_cuda(e);
  int herr = 0;
  if ((e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return from_cuda(e);
  return herr ? HOTRG_ETIMEOUT : HOTRG_OK;
}
