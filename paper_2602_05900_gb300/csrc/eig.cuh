// Thin owner of the cuSOLVER handle and workspaces used for the FP64
// environment eigendecompositions.
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <vector>

namespace hotrg {

class Eig {
 public:
  ~Eig();
  // 0 on success, 1 library error, 2 allocation failure.
  int init(cudaStream_t s);
  // The m largest eigenpairs of the symmetric n x n matrix A (column-major,
  // lower triangle read): ascending values in w[0..m), vectors overwrite the
  // first m columns of A.  Returns 0, 1 (library error), 2 (allocation), 3
  // (wrong eigenpair count).  cusolver's per-call status goes to info(slot).
  int top(double *A, int n, int m, double *w, int slot);
  // All eigenvalues (ascending) of A; A is destroyed.
  int values(double *A, int n, double *w, int slot);
  int *d_info() { return d_info_; }

 private:
  int reserve(size_t dev_bytes, size_t host_bytes);
  cusolverDnHandle_t handle_ = nullptr;
  cusolverDnParams_t params_ = nullptr;
  void *d_work_ = nullptr;
  size_t dev_bytes_ = 0;
  std::vector<char> h_work_;
  int *d_info_ = nullptr;
};

}  // namespace hotrg
