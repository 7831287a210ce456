// Batched FP64 eigensolver for the leading eigenpairs of symmetric positive
// semi-definite environment matrices: block subspace iteration with
// Rayleigh-Ritz, where the small projected problem is diagonalised by a
// parallel-ordered two-sided Jacobi method (Sec. II.B, Eqs. 5-6: rotations of
// 2x2 blocks, all disjoint pairs of a round at once, rows exchanged between
// rounds so that every pair meets once per sweep).
//
// A batch is P problems of the same size n (the two environments of each of
// G instances are problems 2i and 2i + 1).  All per-problem buffers live in one
// workspace at a fixed stride, so a batch of any size costs the same launches.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hotrg {

constexpr int kSiMaxBlock = 96;    // largest Rayleigh-Ritz block / direct-Jacobi size
constexpr int kSiSlices = 8;       // exact-slice digits of the products G X

struct SiBatch {
  int P;                 // number of problems
  int n;                 // matrix size (same for all problems)
  int k;                 // wanted leading eigenpairs
  int m;                 // block size (k <= m <= min(n, kSiMaxBlock), even)
  PSet G;                // symmetric n x n matrix of problem z
  PSet warm;             // optional n x kw column-major start vectors of problem z
  bool has_warm;
  int kw;
  bool xs;               // G X on the tensor cores (exact slices) instead of FP64 SIMT
  int *err;              // device flag set to 2 if a tensor-core wait runs out (xs only)
  PSet trace;            // Tr G of problem z at trace.at(z)[0] (iteration shift)
  bool has_trace;
  double shift_rel;      // initial shift / Tr G
  int first_check;       // expected convergence iteration (first Rayleigh-Ritz step of small batches)
  double floor_tol;      // residual accepted once it stops decreasing (0: the FP64 default, 1e-10)
};

// Where a solve leaves its results inside the workspace: Ritz vectors of
// problem z at X.at(z) (n x m column-major, leading columns descending) and Ritz
// values at theta.at(z) (m values, descending).
struct SiOut {
  PSet X, theta;
};
SiOut si_outputs(double *work, int P, int n, int m);

// Workspace (doubles) for P problems of size n with block m.
long long si_workspace_doubles(int P, int n, int m);

struct SiResult {
  int iterations;       // subspace iterations performed
  int rr;               // Rayleigh-Ritz solves performed
  double residual;      // max over problems and i < k of ||G x_i - theta_i x_i|| / theta_0
  bool converged;
  int breakdown;        // 0, 1 (a Cholesky factorisation broke down) or 2 (a Jacobi sweep limit)
  int sweeps64;         // most FP64 Jacobi sweeps of one Rayleigh-Ritz solve
  int sweeps32;         // most FP32 Jacobi sweeps of one Rayleigh-Ritz solve
};

// Runs the solver on stream s (synchronises it once per convergence check).
// `tol` is the residual target relative to the largest Ritz value.  Returns a
// CUDA error code; `res` reports convergence (the caller decides on fallback).
// `launches` is incremented by the number of kernels launched.
cudaError_t si_solve(const SiBatch &b, double *work, double tol, int max_iter, cudaStream_t s,
                     SiResult *res, long long *launches);

// Direct two-sided Jacobi on whole small matrices (n <= kSiMaxBlock): G is
// copied (zero-padded to the even size jacobi_block(n)), diagonalised, and the
// k leading eigenpairs land in si_outputs(work, P, n, jacobi_block(n)).
int jacobi_block(int n);
cudaError_t jacobi_full(const SiBatch &b, double *work, cudaStream_t s, long long *launches);

}  // namespace hotrg
