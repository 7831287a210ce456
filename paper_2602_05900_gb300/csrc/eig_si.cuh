// Batched FP64 eigensolver for the leading eigenpairs of symmetric positive
// semi-definite environment matrices: block subspace iteration with
// Rayleigh-Ritz, where the small projected problem is diagonalised by a
// parallel-ordered two-sided Jacobi method (Sec. II.B, Eqs. 5-6: rotations of
// 2x2 blocks, all disjoint pairs of a round at once, pairs rotated between
// rounds so that every pair meets once per sweep).
#pragma once

#include <cuda_runtime.h>

namespace hotrg {

constexpr int kSiMaxBatch = 8;     // problems per call (the two environments of a step)
constexpr int kSiMaxBlock = 96;    // largest Rayleigh-Ritz block / direct-Jacobi size

struct SiBatch {
  int P;                           // number of problems
  int n;                           // matrix size (same for all problems)
  int k;                           // wanted leading eigenpairs
  int m;                           // block size (k <= m <= min(n, kSiMaxBlock))
  const double *G[kSiMaxBatch];    // symmetric n x n (row- or column-major)
  double *X[kSiMaxBatch];          // in/out: n x m column-major; on return the leading
                                   // columns hold the Ritz vectors, descending
  double *theta[kSiMaxBatch];      // out: m Ritz values, descending
  const double *warm[kSiMaxBatch]; // optional n x kw column-major start vectors (or null)
  int kw;                          // number of warm-start columns
};

// Workspace (doubles) needed for a batch of P problems of size n with block m.
long long si_workspace_doubles(int P, int n, int m);

struct SiResult {
  int iterations;       // subspace iterations performed
  int rr;               // Rayleigh-Ritz solves performed
  double residual;      // max over problems and i < k of ||G x_i - theta_i x_i|| / theta_0
  bool converged;
};

class StageHook;

// Runs the solver on stream s (synchronises it once per convergence check).
// `tol` is the residual target relative to the largest Ritz value.  Returns a
// CUDA error code; `res` reports convergence (the caller decides on fallback).
// `launches` is incremented by the number of kernels launched.
cudaError_t si_solve(const SiBatch &b, double *work, double tol, int max_iter, cudaStream_t s,
                     SiResult *res, long long *launches);

// Direct two-sided Jacobi on whole small matrices (n <= kSiMaxBlock): G_p is
// copied, diagonalised, and X_p / theta_p receive all n eigenpairs, descending.
cudaError_t jacobi_full(const SiBatch &b, double *work, cudaStream_t s, long long *launches);

}  // namespace hotrg
