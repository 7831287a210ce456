// FP64 eigendecomposition of the symmetric environment matrices through
// cuSOLVER's 64-bit syevd/syevdx entry points (the library eigensolver of the
// step; the truncation is taken from the leading eigenvectors, Sec. II.A and
// the Hermitian case of Eq. 5).
#include <cusolverDn.h>

#include <vector>

#include "eig.cuh"

namespace hotrg {

Eig::~Eig() {
  if (d_work_) cudaFree(d_work_);
  if (d_info_) cudaFree(d_info_);
  if (params_) cusolverDnDestroyParams(params_);
  if (handle_) cusolverDnDestroy(handle_);
}

int Eig::init(cudaStream_t s) {
  if (cusolverDnCreate(&handle_) != CUSOLVER_STATUS_SUCCESS) return 1;
  if (cusolverDnSetStream(handle_, s) != CUSOLVER_STATUS_SUCCESS) return 1;
  if (cusolverDnCreateParams(&params_) != CUSOLVER_STATUS_SUCCESS) return 1;
  if (cudaMalloc(&d_info_, 2 * sizeof(int)) != cudaSuccess) return 2;
  if (cudaMemsetAsync(d_info_, 0, 2 * sizeof(int), s) != cudaSuccess) return 1;
  return 0;
}

int Eig::reserve(size_t dev_bytes, size_t host_bytes) {
  if (dev_bytes > dev_bytes_) {
    if (d_work_) cudaFree(d_work_);
    d_work_ = nullptr;
    if (cudaMalloc(&d_work_, dev_bytes) != cudaSuccess) { dev_bytes_ = 0; return 2; }
    dev_bytes_ = dev_bytes;
  }
  if (host_bytes > h_work_.size()) h_work_.resize(host_bytes);
  return 0;
}

int Eig::top(double *A, int n, int m, double *w, int slot) {
  int64_t meig = 0;
  const int64_t il = (int64_t)n - m + 1, iu = n;
  double vl = 0.0, vu = 0.0;
  size_t db = 0, hb = 0;
  if (cusolverDnXsyevdx_bufferSize(handle_, params_, CUSOLVER_EIG_MODE_VECTOR,
                                   CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A,
                                   n, &vl, &vu, il, iu, &meig, CUDA_R_64F, w, CUDA_R_64F, &db,
                                   &hb) != CUSOLVER_STATUS_SUCCESS)
    return 1;
  if (int r = reserve(db, hb)) return r;
  if (cusolverDnXsyevdx(handle_, params_, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                        CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n, &vl, &vu, il, iu, &meig,
                        CUDA_R_64F, w, CUDA_R_64F, d_work_, dev_bytes_,
                        h_work_.empty() ? nullptr : h_work_.data(), h_work_.size(),
                        d_info_ + slot) != CUSOLVER_STATUS_SUCCESS)
    return 1;
  if (meig != m) return 3;
  return 0;
}

int Eig::values(double *A, int n, double *w, int slot) {
  size_t db = 0, hb = 0;
  if (cusolverDnXsyevd_bufferSize(handle_, params_, CUSOLVER_EIG_MODE_NOVECTOR,
                                  CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n, CUDA_R_64F, w,
                                  CUDA_R_64F, &db, &hb) != CUSOLVER_STATUS_SUCCESS)
    return 1;
  if (int r = reserve(db, hb)) return r;
  if (cusolverDnXsyevd(handle_, params_, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                       CUDA_R_64F, A, n, CUDA_R_64F, w, CUDA_R_64F, d_work_, dev_bytes_,
                       h_work_.empty() ? nullptr : h_work_.data(), h_work_.size(),
                       d_info_ + slot) != CUSOLVER_STATUS_SUCCESS)
    return 1;
  return 0;
}

}  // namespace hotrg
