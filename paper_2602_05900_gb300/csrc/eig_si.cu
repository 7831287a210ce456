// Batched FP64 subspace-iteration eigensolver for the environments (see
// eig_si.cuh).  GB300's FP64 rate is a few flops per clock per SM, so the
// work is arranged for the whole GPU: the products with G, the Gram matrices
// and the basis rotations are tall-skinny FP64 GEMMs spread over all SMs (the
// two environments of a step run in the same launches), and only the small
// m x m factorisations run on one CTA per problem.
//
// The iteration runs on G + sigma I with sigma = 2^-40 Tr G (same
// eigenvectors; the Ritz values are shifted back at the end).  The shift keeps
// the columns of G X that belong to the numerical null space of G at least
// sigma long and along their own direction when the products are nearly
// exact (HOTRG fixed points far from criticality have numerically rank
// deficient G).  Where columns still become nearly dependent (G from
// reduced-precision contractions is indefinite at their rounding level, and a
// Ritz value can sit at zero), the FP32 CholeskyQR pass restarts with a shift
// instead of breaking down.
//
// One iteration:  Y = G X  ->  X = orth(Y): CholeskyQR with FP32 Cholesky
// factors and FP64 rotations -- two passes while the block may be ill
// conditioned (or shifted CholeskyQR3 in FP64 for large batches), one pass once
// its columns are close to eigenvectors, two FP64 passes where the block holds
// numerically null directions.  A Rayleigh-Ritz step works with C0 = X^T X:
// W = C0^(-1/2) (Newton-Schulz on the m x m side, or a shifted FP64 Cholesky
// where C0 is far from I), H = W^T (X^T Y) W, H diagonalised by the parallel
// two-sided Jacobi method (FP32, then an FP64 finish), and X, Y rotated onto
// the Ritz vectors.  The iteration stops when ||G x_i - theta_i x_i|| <= tol *
// theta_0 for i < k (or at the accuracy floor of G); the next check is
// scheduled from the observed Ritz-value ratio theta_m / theta_k.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include <cooperative_groups.h>

#include "eig_si.cuh"
#include "tc_exact.cuh"

namespace cg = cooperative_groups;

namespace hotrg {
namespace {

constexpr int kSplitMax = 8;     // split-K partials of G X
constexpr int kChunkMax = 256;   // row chunks of the Gram reduction
constexpr int kRowsPerChunk = 16;
constexpr int kCluster = 8;      // CTAs per Jacobi problem (one thread-block cluster)
constexpr int kJacobiMaxSweeps = 40;
constexpr int kCholThreads = 256;
constexpr int kCholPanel = 8;      // columns per panel of the blocked FP32 Cholesky
constexpr double kXsSmallWork = 32.0 * 1024 * 1024;   // FP64 FMAs of one n x m x m product batch
constexpr int kSiSmallBatch = 8;      // problems up to which the solve is latency bound
constexpr double kSiFloorTol = 1e-10;  // residuals accepted once they stop decreasing
constexpr int kSiSlowIters = 24;       // iterations after which a residual below the floor is accepted
constexpr float kChol32Retry = 0x1.0p-12f;   // diagonal shift of a retried FP32 CholeskyQR pass


// splitmix64 finaliser (Steele, Lea, Flood 2014) -> uniform double in [-1, 1)
__device__ inline double hash_uniform(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return static_cast<double>(x >> 11) * 0x1.0p-52 - 1.0;
}

// GB300 executes FP64 square roots and divisions as long dependent instruction
// sequences; on the latency-bound paths below they are replaced by an FP32
// estimate refined with FP64 fused multiply-adds (Newton's method), which is
// accurate to FP64 rounding after two steps.

// 2^-e scaling factor with e the binary exponent of x (exact, x > 0 finite)
__device__ inline double pow2_inv_of(double x) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF) - 1023;
  return __longlong_as_double((long long)(1023 - e) << 52);
}

// 1/sqrt(x) for x > 0 to FP64 accuracy: FP32 seed on a power-of-two scaled
// argument, two Newton steps y <- y (3 - x y^2) / 2 in FP64.
__device__ inline double rsqrt_fp64(double x) {
  const double s = pow2_inv_of(x);                  // x s in [1, 2)
  const double xs = x * s;
  double y = (double)rsqrtf((float)xs);
  y = y * fma(-0.5 * xs, y * y, 1.5);
  y = y * fma(-0.5 * xs, y * y, 1.5);
  // 1/sqrt(x) = (1/sqrt(x s)) sqrt(s); s is a power of two
  const long long sb = __double_as_longlong(s);
  const int es = (int)((sb >> 52) & 0x7FF) - 1023;
  double root_s = (es & 1) ? 1.4142135623730951 : 1.0;
  root_s *= __longlong_as_double((long long)(1023 + (es >> 1)) << 52);
  return y * root_s;
}

__global__ void k_si_init(PSet X, PSet warm, int has_warm, int kw, int n, int m) {
  const int z = blockIdx.z;
  const long long total = (long long)n * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n);
    double v;
    if (has_warm && j < kw) v = warm.at(z)[e];
    else v = hash_uniform(((unsigned long long)z << 56) ^ ((unsigned long long)j << 32) ^ (unsigned long long)(e % n));
    X.at(z)[e] = v;
  }
}

// Out_s = G[rows i0.., cols in split s] . X[those rows, :]  (X, Out column-major n x m)
__global__ void __launch_bounds__(256) k_si_gemm(PSet G, PSet X, PSet Out, int n, int m, int chunk) {
  __shared__ double Gs[16][65];
  __shared__ double Xs[16][kSiMaxBlock];
  const int z = blockIdx.z;
  const double *g = G.at(z);
  const double *x = X.at(z);
  double *out = Out.at(z) + (size_t)blockIdx.y * n * m;
  const int i0 = blockIdx.x * 64;
  const int k0 = blockIdx.y * chunk;
  const int k1 = min(n, k0 + chunk);
  const int t = threadIdx.x, r = t & 63, cg = t >> 6;
  double acc[kSiMaxBlock / 4];
#pragma unroll
  for (int c = 0; c < kSiMaxBlock / 4; ++c) acc[c] = 0.0;
  for (int kk = k0; kk < k1; kk += 16) {
    for (int e = t; e < 64 * 16; e += 256) {
      const int row = e >> 4, col = e & 15;
      const int gi = i0 + row, gk = kk + col;
      Gs[col][row] = (gi < n && gk < k1) ? g[(size_t)gi * n + gk] : 0.0;
    }
    for (int e = t; e < 16 * m; e += 256) {
      const int j = e >> 4, col = e & 15;
      const int gk = kk + col;
      Xs[col][j] = (gk < k1) ? x[(size_t)j * n + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const double gv = Gs[l][r];
#pragma unroll
      for (int c = 0; c < kSiMaxBlock / 4; ++c) {
        const int j = cg + 4 * c;
        if (j < m) acc[c] = fma(gv, Xs[l][j], acc[c]);
      }
    }
    __syncthreads();
  }
  const int i = i0 + r;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < kSiMaxBlock / 4; ++c) {
      const int j = cg + 4 * c;
      if (j < m) out[(size_t)j * n + i] = acc[c];
    }
  }
}

// Shift of the iteration (see si_solve): sig[0] is the shift of the current
// Y = (G + sig[0] I) X, sig[1] the shift of the next product (equal to it in
// this solver; kept apart so that a shift change can never mix the two).
__global__ void k_si_sigma_init(PSet sig, PSet trace, double factor) {
  const int z = blockIdx.z;
  if (threadIdx.x == 0) {
    const double t = trace.at(z)[0];
    const double v = (t > 0.0 && isfinite(t)) ? factor * t : 0.0;
    sig.at(z)[0] = v;
    sig.at(z)[1] = v;
  }
}

// Y += sig[1] X; block (0, 0, z) records sig[0] = sig[1] (the shift now in Y)
__global__ void k_si_shift_add(PSet Y, PSet X, PSet sig, long long nm) {
  const int z = blockIdx.z;
  const double sg = sig.at(z)[1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nm;
       e += (long long)gridDim.x * blockDim.x)
    Y.at(z)[e] = fma(sg, X.at(z)[e], Y.at(z)[e]);
  if (blockIdx.x == 0 && threadIdx.x == 0) sig.at(z)[0] = sg;
}

// theta_z[i] -= sig[0] for i < m (the shift of the last Rayleigh-Ritz step)
__global__ void k_si_unshift(PSet theta, PSet sig, int m) {
  const int z = blockIdx.z;
  const double sg = sig.at(z)[0];
  for (int i = threadIdx.x; i < m; i += blockDim.x) theta.at(z)[i] -= sg;
}

// ks[j] = power of two within a factor 2 of 1 / sqrt(C_jj) (1 if C_jj is not
// positive and finite): the column scales of a CholeskyQR basis change
__global__ void k_si_colscale(PSet C, PSet ks, int m) {
  const int z = blockIdx.z;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double c = C.at(z)[(size_t)j * m + j];
    int e = 0;
    if (c > 0.0 && isfinite(c)) (void)frexp(c, &e);
    ks.at(z)[j] = ldexp(1.0, -(e / 2));
  }
}

// out = sum of the S K-parts; with shift, + sig[1] X as well (the iteration's
// shift, the same fma as k_si_shift_add) and sig[0] = sig[1]
__global__ void k_si_sum_split(PSet part, PSet out, int S, long long nm, PSet X, PSet sig, int shift) {
  const int z = blockIdx.z;
  const double sg = shift ? sig.at(z)[1] : 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nm;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += part.at(z)[s * nm + e];
    if (shift) v = fma(sg, X.at(z)[e], v);
    out.at(z)[e] = v;
  }
  if (shift && blockIdx.x == 0 && threadIdx.x == 0) sig.at(z)[0] = sg;
}

// Cp[c] = A[rows of chunk c]^T B[same rows]   (m x m, row-major a*m + b)
template <typename Acc>
__global__ void __launch_bounds__(256) k_si_gram(PSet A, PSet B, PSet Cp, int n, int m, int sym) {
  __shared__ Acc As[16][kSiMaxBlock + 1];
  __shared__ Acc Bs[16][kSiMaxBlock + 1];
  const int z = blockIdx.z, c = blockIdx.x;
  const double *a = A.at(z);
  const double *b = B.at(z);
  const int r0 = c * kRowsPerChunk, r1 = min(n, r0 + kRowsPerChunk);
  const int ta = threadIdx.x >> 4, tb = threadIdx.x & 15;
  constexpr int U = kSiMaxBlock / 16;   // 6 x 6 outputs per thread
  // A^T A is symmetric: only the tiles on or above the diagonal are computed
  const bool skip = sym && (ta > tb);
  Acc acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = Acc(0);
  for (int rr = r0; rr < r1; rr += 16) {
    for (int e = threadIdx.x; e < 16 * m; e += 256) {
      const int j = e >> 4, ii = e & 15;
      const int row = rr + ii;
      As[ii][j] = (row < r1) ? (Acc)a[(size_t)j * n + row] : Acc(0);
      Bs[ii][j] = (row < r1) ? (Acc)b[(size_t)j * n + row] : Acc(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 16 && !skip; ++ii) {
      Acc av[U], bv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) av[u] = As[ii][ta * U + u];
#pragma unroll
      for (int v = 0; v < U; ++v) bv[v] = Bs[ii][tb * U + v];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  double *out = Cp.at(z) + (size_t)c * m * m;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int ia = ta * U + u, ib = tb * U + v;
      if (ia < m && ib < m && !skip) out[ia * m + ib] = (double)acc[u][v];
    }
}

// C = sum over row chunks of the Gram partials (fixed order), symmetrised.
// sym: the partials hold only the upper tiles (A^T A).  ns: write instead the
// Newton-Schulz polish W = (3 I - C) / 2 (column-major, = row-major by symmetry).
__global__ void k_si_gram_reduce(PSet Cp, PSet C, int nchunks, int m, int sym, int ns) {
  const int z = blockIdx.z;
  const long long mm = (long long)m * m;
  constexpr int U = kSiMaxBlock / 16;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int a = e / m, b = e % m;
    if (b < a) continue;
    const double *src = Cp.at(z);
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    double sv;
    if (sym) {
      // (a, b) lives in tile (a / U, b / U); a tile below the diagonal was skipped.
      // Eight independent partial sums keep eight loads in flight (the chunk
      // sums are load-latency bound), combined in a fixed order.
      const bool upper = (a / U) <= (b / U);
      const long long off = upper ? (long long)a * m + b : (long long)b * m + a;
      double v4 = 0.0, v5 = 0.0, v6 = 0.0, v7 = 0.0;
      int c = 0;
      for (; c + 8 <= nchunks; c += 8) {
        v0 += src[c * mm + off];
        v1 += src[(c + 1) * mm + off];
        v2 += src[(c + 2) * mm + off];
        v3 += src[(c + 3) * mm + off];
        v4 += src[(c + 4) * mm + off];
        v5 += src[(c + 5) * mm + off];
        v6 += src[(c + 6) * mm + off];
        v7 += src[(c + 7) * mm + off];
      }
      for (; c < nchunks; ++c) v0 += src[c * mm + off];
      sv = ((v0 + v1) + (v2 + v3)) + ((v4 + v5) + (v6 + v7));
    } else {
      double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
      int c = 0;
      for (; c + 4 <= nchunks; c += 4) {
        v0 += src[c * mm + a * m + b];
        w0 += src[c * mm + b * m + a];
        v1 += src[(c + 1) * mm + a * m + b];
        w1 += src[(c + 1) * mm + b * m + a];
        v2 += src[(c + 2) * mm + a * m + b];
        w2 += src[(c + 2) * mm + b * m + a];
        v3 += src[(c + 3) * mm + a * m + b];
        w3 += src[(c + 3) * mm + b * m + a];
      }
      for (; c < nchunks; ++c) {
        v0 += src[c * mm + a * m + b];
        w0 += src[c * mm + b * m + a];
      }
      sv = 0.5 * (((v0 + v1) + (v2 + v3)) + ((w0 + w1) + (w2 + w3)));
    }
    if (ns) sv = (a == b ? 1.5 : 0.0) - 0.5 * sv;
    C.at(z)[a * m + b] = sv;
    C.at(z)[b * m + a] = sv;
  }
}

// Shifted, column-scaled Cholesky in FP32 of a block's Gram matrix C and the
// rotation W = diag(d) R^-1 (column-major, stored in FP64) such that Y W is
// orthonormal up to FP32 accuracy: C_hat = diag(d) C diag(d) + shift I = R^T R,
// d_j = 1 / sqrt(C_jj).  Used for the iterations between Rayleigh-Ritz steps,
// where an approximately orthonormal basis is all the power iteration needs.
__global__ void __launch_bounds__(kCholThreads) k_si_chol32(PSet Cin, int m, float shift, PSet Wout,
                                                            int *flag) {
  extern __shared__ float shf[];
  const int ld = m + 1;
  float *C = shf;                 // m x ld: C_hat, updated in place (rows below the step)
  float *R = shf + m * ld;        // m x ld: the factor R (upper triangle)
  float *d = R + m * ld;          // m
  const int z = blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double cjj = Cin.at(z)[(size_t)j * m + j];
    d[j] = (cjj > 0.0 && isfinite(cjj)) ? (float)rsqrt_fp64(cjj) : 1.0f;
  }
  __shared__ int bad;
  // A nearly dependent set of columns breaks the unshifted factorisation; the
  // second attempt adds kChol32Retry to the unit diagonal, which always
  // succeeds and leaves a basis with condition number below about
  // kChol32Retry^-1/2 for the next pass to finish.
  for (int attempt = 0; attempt < 2; ++attempt) {
    const float sh = attempt == 0 ? shift : fmaxf(shift, kChol32Retry);
    __syncthreads();
    // coalesced reads, four in flight per thread
    for (int e0 = threadIdx.x; e0 < m * m; e0 += 4 * blockDim.x) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = e < m * m ? Cin.at(z)[e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < m * m) {
          const int a = e / m, b = e % m;
          C[a * ld + b] = (float)v[u] * (d[a] * d[b]) + (a == b ? sh : 0.0f);
        }
      }
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    // Blocked right-looking factorisation, panels of kCholPanel columns and two
    // barriers per panel: (a) the threads of the first three warps (the ones
    // that need it: m <= 96) factor the panel's diagonal block U^T U = C_jj
    // redundantly in registers (identical inputs, identical results); (b) the
    // panel's rows of R right of the block, U^T R_j,rest = C_j,rest, by forward
    // substitution, one column per thread; (c) after the barrier, a failed pivot
    // (published by thread 0) stops every thread, else the trailing update
    // C_rest -= R_j,rest^T R_j,rest.
    const bool factor = threadIdx.x < 96;
    for (int j0 = 0; j0 < m; j0 += kCholPanel) {
      const int w = min(kCholPanel, m - j0);
      float U[kCholPanel][kCholPanel];
      float uinv[kCholPanel];
      bool ok = factor;
      if (factor) {
        // the block's upper triangle into registers first (rows past w: identity),
        // then the dependent chain; 1 / u_ii by rsqrtf (an FP32 factor is all
        // the pass needs: the FP64 rotation preserves the span whatever W is)
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i)
#pragma unroll
          for (int b = i; b < kCholPanel; ++b)
            U[i][b] = (i < w && b < w) ? C[(j0 + i) * ld + j0 + b] : (i == b ? 1.0f : 0.0f);
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i) {
          float dd = U[i][i];
#pragma unroll
          for (int k = 0; k < i; ++k) dd = fmaf(-U[k][i], U[k][i], dd);
          ok = ok && dd > 0.0f && isfinite(dd);
          const float r = rsqrtf(dd);
          uinv[i] = r;
          U[i][i] = dd * r;
#pragma unroll
          for (int b = i + 1; b < kCholPanel; ++b) {
            float v = U[i][b];
#pragma unroll
            for (int k = 0; k < i; ++k) v = fmaf(-U[k][i], U[k][b], v);
            U[i][b] = v * r;
          }
        }
      }
      if (factor && !ok && threadIdx.x == 0) bad = 1;
      if (ok && threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i)
#pragma unroll
          for (int b = i; b < kCholPanel; ++b)
            if (b < w) R[(j0 + i) * ld + j0 + b] = U[i][b];
      }
      for (int l = j0 + w + threadIdx.x; ok && l < m; l += blockDim.x) {
        // a panel with columns past it is a full one (w = kCholPanel)
        float cv[kCholPanel], y[kCholPanel];
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i) cv[i] = C[(j0 + i) * ld + l];
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i) {
          float v = cv[i];
#pragma unroll
          for (int k = 0; k < i; ++k) v = fmaf(-U[k][i], y[k], v);
          y[i] = v * uinv[i];
        }
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i) R[(j0 + i) * ld + l] = y[i];
      }
      __syncthreads();
      if (bad) break;
      // a panel with a trailing part is a full one (w = kCholPanel); the
      // thread's column a of the panel rows stays in registers
      for (int a = j0 + w + ty; a < m; a += 16) {
        float ra[kCholPanel];
#pragma unroll
        for (int i = 0; i < kCholPanel; ++i) ra[i] = R[(j0 + i) * ld + a];
        for (int b = a + tx; b < m; b += 16) {
          float v = C[a * ld + b];
#pragma unroll
          for (int i = 0; i < kCholPanel; ++i) v = fmaf(-ra[i], R[(j0 + i) * ld + b], v);
          C[a * ld + b] = v;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!bad) break;
  }
  if (bad) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  // W = diag(d) R^-1.  Z = R^-1 (upper triangular, in the now free C storage)
  // by 8 x 8 blocks: (1) every diagonal block Z_II = R_II^-1 by back
  // substitution, one thread per column; (2) the off-diagonal blocks by
  // distance d = J - I, all blocks of one distance at once:
  // Z_IJ = -Z_II sum_{K = I+1..J} R_IK Z_KJ (the blocks Z_KJ, K > I, have
  // smaller distances).  Two barriers per distance: the dependent chains are
  // at most 8 d long instead of m.
  constexpr int BS = kCholPanel;
  const int nb = (m + BS - 1) / BS;
  float *Z = C;
  float *Tt = d + m;                      // nb BS x BS scratch blocks: the sums of one distance
  for (int e = threadIdx.x; e < m * ld; e += blockDim.x) Z[e] = 0.0f;
  __syncthreads();
  for (int t = threadIdx.x; t < nb * BS; t += blockDim.x) {
    const int I = t / BS, cl = t % BS, i0 = I * BS, w = min(BS, m - i0);
    if (cl < w) {
      const int c = i0 + cl;
      float zc[BS];
#pragma unroll
      for (int ii = BS - 1; ii >= 0; --ii) {
        float v = 0.0f;
        if (ii <= cl) {
          const int i = i0 + ii;
          v = (ii == cl) ? 1.0f : 0.0f;
#pragma unroll
          for (int kk = ii + 1; kk < BS; ++kk)
            if (kk <= cl) v = fmaf(-R[i * ld + i0 + kk], zc[kk], v);
          v /= R[i * ld + i];
        }
        zc[ii] = v;
      }
#pragma unroll
      for (int ii = 0; ii < BS; ++ii)
        if (ii <= cl) Z[(i0 + ii) * ld + c] = zc[ii];
    }
  }
  __syncthreads();
  for (int dist = 1; dist < nb; ++dist) {
    const int nblk = nb - dist;
    // T_IJ[i][j] = sum_{k in blocks I+1..J} R[i][k] Z[k][j]
    for (int t = threadIdx.x; t < nblk * BS * BS; t += blockDim.x) {
      const int I = t / (BS * BS), ij = t % (BS * BS), ii = ij / BS, jj = ij % BS;
      const int J = I + dist, i = I * BS + ii, j = J * BS + jj;
      float v = 0.0f;
      if (i < m && j < m) {
        const int k1 = min(m, J * BS + BS);
        for (int k = (I + 1) * BS; k < k1; ++k) v = fmaf(R[i * ld + k], Z[k * ld + j], v);
      }
      Tt[t] = v;
    }
    __syncthreads();
    // Z_IJ = -Z_II T_IJ
    for (int t = threadIdx.x; t < nblk * BS * BS; t += blockDim.x) {
      const int I = t / (BS * BS), ij = t % (BS * BS), ii = ij / BS, jj = ij % BS;
      const int J = I + dist, i0 = I * BS, i = i0 + ii, j = J * BS + jj;
      if (i < m && j < m) {
        float v = 0.0f;
        for (int l = ii; l < BS && i0 + l < m; ++l) v = fmaf(Z[i * ld + i0 + l], Tt[I * BS * BS + l * BS + jj], v);
        Z[i * ld + j] = -v;
      }
    }
    __syncthreads();
  }
  double *W = Wout.at(z);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int c = e / m, j = e % m;           // W[j + c m]
    W[e] = (j <= c) ? (double)Z[j * ld + c] * (double)d[j] : 0.0;
  }
}

// Shifted, column-scaled Cholesky of a block's Gram matrix C and the rotation
// W = diag(d) R^-1 (column-major) such that Y W is orthonormal:
//   C_hat = diag(d) C diag(d) + shift I = R^T R,  d_j = 1 / sqrt(C_jj).
__global__ void __launch_bounds__(kCholThreads) k_si_chol(PSet Cin, int m, double shift, PSet Wout,
                                                          int *flag, PSet only_if) {
  // only_if (optional): run for problem z only if only_if.at(z)[2] != 0
  if (only_if.b0 && only_if.at(blockIdx.z)[2] == 0.0) return;
  extern __shared__ double sh[];
  const int ld = m + 1;
  double *C = sh;                 // m x ld, upper triangle -> R
  double *Z = sh + m * ld;        // m x ld, R^-1 (upper)
  double *d = Z + m * ld;         // m
  double *rinv = d + m;           // m: 1 / R_jj
  const int z = blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) C[(e / m) * ld + e % m] = Cin.at(z)[e];
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double cjj = C[j * ld + j];
    d[j] = (cjj > 0.0 && isfinite(cjj)) ? rsqrt_fp64(cjj) : 1.0;   // 1 / column norm
  }
  __syncthreads();
  __shared__ int bad;
  // Nearly dependent columns break the factorisation: later attempts add a
  // larger diagonal shift (2^-26, then 2^-12 of the unit diagonal), which
  // always succeeds and leaves a basis the next pass finishes.
  for (int attempt = 0; attempt < 3; ++attempt) {
  const double shv = attempt == 0 ? shift : fmax(shift, attempt == 1 ? 0x1.0p-26 : 0x1.0p-12);
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) C[(e / m) * ld + e % m] = Cin.at(z)[e];
  __syncthreads();
  for (int a = ty; a < m; a += 16)
    for (int b = tx; b < m; b += 16) C[a * ld + b] = C[a * ld + b] * (d[a] * d[b]) + (a == b ? shv : 0.0);
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // right-looking Cholesky on the upper triangle
  for (int j = 0; j < m; ++j) {
    const double piv = C[j * ld + j];
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (threadIdx.x == 0) bad = 1;
      break;
    }
    const double ri = rsqrt_fp64(piv);          // 1 / R_jj
    __syncthreads();
    for (int l = j + 1 + threadIdx.x; l < m; l += blockDim.x) C[j * ld + l] *= ri;
    __syncthreads();
    if (threadIdx.x == 0) {
      C[j * ld + j] = piv * ri;
      rinv[j] = ri;
    }
    for (int a = j + 1 + ty; a < m; a += 16)
      for (int b = a + tx; b < m; b += 16) C[a * ld + b] -= C[j * ld + a] * C[j * ld + b];
    __syncthreads();
  }
  __syncthreads();
  if (!bad) break;
  }
  if (bad) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  // R^-1 by right-looking back substitution: Z = I, then for i = m-1 .. 0 scale
  // row i by 1/R_ii and eliminate it from the rows above (depth m, not m^2)
  for (int a = ty; a < m; a += 16)
    for (int b = tx; b < m; b += 16) Z[a * ld + b] = (a == b) ? 1.0 : 0.0;
  __syncthreads();
  for (int i = m - 1; i >= 0; --i) {
    for (int b = i + threadIdx.x; b < m; b += blockDim.x) Z[i * ld + b] *= rinv[i];
    __syncthreads();
    for (int a = ty; a < i; a += 16)
      for (int b = i + tx; b < m; b += 16) Z[a * ld + b] = fma(-C[a * ld + i], Z[i * ld + b], Z[a * ld + b]);
    __syncthreads();
  }
  double *W = Wout.at(z);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int c = e / m, j = e % m;           // W[j + c m]
    W[e] = (j <= c) ? Z[j * ld + c] * d[j] : 0.0;
  }
}

// Parallel two-sided Jacobi on a symmetric m x m matrix (m even) by a cluster
// of kCluster CTAs, laid out as the systolic scheme of Sec. II.B / Fig. 3.
// The m/2 index pairs of a round are "slots"; slot I holds two whole rows of
// the matrix (its top and bottom index) and belongs to one CTA (contiguous
// slots per CTA).  A round: (1) every CTA computes the rotations of all slots
// from a replicated table of their 2x2 diagonal blocks; (2) one thread per 2x2
// block of the CTA's rows applies both rotations at once,
// M'_{IJ} = J_I^T M_{IJ} J_J (Eq. 6: the quad tile as the unit of work), and
// (3) writes the four results to the slots their rows move to (tops one slot
// down, bottoms one slot up, turning at both ends: the round-robin order in
// which every pair meets once per sweep); each moved row also writes its
// entries of the next round's 2x2 blocks into every CTA's table.  One cluster
// barrier per round, split into arrive / wait so that each CTA rotates its
// share of the rows of V while the others finish; since all CTAs see the same
// table, the sweep decision needs no exchange.  Sweeps stop when no pair needs rotating (an off-diagonal entry is
// rotated when it is above 2^-56 of the largest diagonal entry and not tiny
// against its own diagonal pair), or after a sweep whose rotated entries were
// all below 1e-8 relative (quadratic convergence).
__device__ inline void jacobi_angle(double hpp, double hqq, double hpq, double &c, double &s) {
  // solve h_pq t^2 + (h_qq - h_pp) t - h_pq = 0 for the smaller root (Golub &
  // Van Loan's symmetric Schur decomposition) on a power-of-two scaled copy:
  // FP32 estimate, then two Newton steps whose residual is evaluated in FP64
  const double sc = pow2_inv_of(fmax(fabs(hpq), fmax(fabs(hpp), fabs(hqq))));
  const double a = hpp * sc, b = hqq * sc, g = hpq * sc, diff = b - a;
  const float fg = (float)g, fd = (float)diff;
  float t32;
  if (fabsf(fd) > 1e6f * fabsf(fg)) {
    t32 = fg / fd;                                  // 1/(2 tau), tau = diff / (2 g)
  } else {
    const float tau = fd / (2.0f * fg);
    t32 = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
  }
  double t = (double)t32;
  // seed of c = (1 + t^2)^(-1/2) from the FP32 root, computed while t is refined
  const float c32 = rsqrtf(fmaf(t32, t32, 1.0f));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double F = fma(fma(g, t, diff), t, -g);   // g t^2 + diff t - g
    const double dF = fma(2.0 * g, t, diff);
    t -= F * (double)__frcp_rn((float)dF);
  }
  // |t| <= 1 (the smaller root), so x = 1 + t^2 lies in [1, 2] and needs no
  // power-of-two scaling: two Newton steps y <- y (3 - x y^2) / 2 in FP64
  const double x = fma(t, t, 1.0);
  double y = (double)c32;
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  c = y;
  s = t * c;
}

__global__ void __launch_bounds__(512, 2) k_si_jacobi(PSet Cin, int m, PSet Wout, PSet theta, int *flag,
                                                   int *sweeps, int floor_exp, int sig_exp) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.z;
  extern __shared__ double sh[];
  const int half = m / 2;
  const int spc = (half + kCluster - 1) / kCluster;          // slots per CTA
  const int s0 = rank * spc, s1 = min(half, s0 + spc);      // own slots [s0, s1)
  const int vrows = (m + kCluster - 1) / kCluster;
  const int v0 = rank * vrows, v1 = min(m, v0 + vrows);     // own rows of V
  // rows[buf][slot - s0][0 = top, 1 = bottom][m]
  double *rowsb = sh;
  auto ROW = [&](int buf, int slot, int tb) { return rowsb + (((size_t)buf * spc + (slot - s0)) * 2 + tb) * m; };
  double *V = rowsb + (size_t)2 * spc * 2 * m;              // vrows x m
  double *ac = V + (size_t)vrows * m;                       // c of every slot, [round parity][slot]
  double *as = ac + 2 * half;                               // s of every slot, same
  // angle inputs of every slot, replicated in every CTA, double-buffered by
  // round parity: [buf][slot][0 = h of the top row's index, 1 = h of the
  // bottom row's index, 2 = h_pq from the row of the smaller index]
  double *nd = as + 2 * half;
  double *diag = nd + 2 * 3 * half;                         // m diagonal entries
  int *ap = reinterpret_cast<int *>(diag + m);              // p of every slot, [parity][slot]
  int *aq = ap + 2 * half;                                  // q of every slot, same
  __shared__ int rotated;
  __shared__ unsigned int maxrel_bits;
  __shared__ double s_floor, s_sig;
  __shared__ int s_more, s_any[2];     // post-sweep test: this CTA's rows / the cluster's
  auto top_index = [&](int sl, int rr) { return (sl == 0) ? 0 : 1 + (sl - 1 + rr) % (m - 1); };
  auto bot_index = [&](int sl, int rr) { return 1 + (m - 2 - sl + rr) % (m - 1); };

  // round 0 layout: position j holds index j; slot I = positions (I, m-1-I).
  // The symmetric part of the input: the rotations assume h_pq = h_qp, and a
  // stored asymmetry above the stop thresholds would never be rotated away.
  for (int e = threadIdx.x; e < (s1 - s0) * 2 * m; e += blockDim.x) {
    const int sl = s0 + e / (2 * m), tb = (e / m) & 1, c = e % m;
    const int idx = tb == 0 ? sl : m - 1 - sl;
    const double *C = Cin.at(z);
    ROW(0, sl, tb)[c] = 0.5 * (C[(size_t)idx * m + c] + C[(size_t)c * m + idx]);
  }
  for (int e = threadIdx.x; e < (v1 - v0) * m; e += blockDim.x) {
    const int rl = e / m, c = e % m;
    V[rl * m + c] = (v0 + rl == c) ? 1.0 : 0.0;
  }
  for (int sl = threadIdx.x; sl < half; sl += blockDim.x) {
    const int u = top_index(sl, 0), v = bot_index(sl, 0);
    const double *C = Cin.at(z);
    nd[sl * 3 + 0] = C[(size_t)u * m + u];
    nd[sl * 3 + 1] = C[(size_t)v * m + v];
    nd[sl * 3 + 2] = 0.5 * (C[(size_t)u * m + v] + C[(size_t)v * m + u]);
  }
  // absolute floor of the rotations: entries below 2^-56 of the largest diagonal
  // entry (a quarter ulp of the matrix norm) are rounding noise; rotating them
  // changes no eigenpair beyond that level, while the relative test below would
  // keep rotating noise between near-null diagonal entries (measured: 12 -> 9.7
  // sweeps per Rayleigh-Ritz solve on D = 32-48 environments)
  if (threadIdx.x == 0) s_any[0] = s_any[1] = 0;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < m; i += 32) v = fmax(v, fabs(Cin.at(z)[(size_t)i * m + i]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      s_floor = ldexp(v, -floor_exp);
      // rotations below 2^-sig_exp of the largest diagonal entry do not hold
      // the sweeps back (their entries are absolutely negligible, whatever
      // their size against their own diagonal pair)
      s_sig = ldexp(v, -sig_exp);
    }
  }
  __syncthreads();
  // the round-0 inputs are read locally; remote writes only target buffer 1
  // before the first cluster barrier, so no barrier is needed here

  int cur = 0, sweep = 0, r_global = 0;
  bool stop = false;
  for (; sweep < kJacobiMaxSweeps && !stop; ++sweep) {
    if (threadIdx.x == 0) {
      rotated = 0;
      maxrel_bits = 0u;
    }
    __syncthreads();
    for (int r = 0; r < m - 1; ++r, ++r_global) {
      const int rr = r_global % (m - 1), rn = (r_global + 1) % (m - 1);
      const double *ndc = nd + (r_global & 1) * 3 * half;
      double *ndn_local = nd + ((r_global + 1) & 1) * 3 * half;
      // this round's angle arrays (double-buffered by round parity: a thread may
      // still rotate V with this round's angles while others start the next round)
      double *acr = ac + (r_global & 1) * half, *asr = as + (r_global & 1) * half;
      int *apr = ap + (r_global & 1) * half, *aqr = aq + (r_global & 1) * half;
      // (1) every CTA computes the angles of every slot from the replicated inputs
      for (int sl = threadIdx.x; sl < half; sl += blockDim.x) {
        const int u = top_index(sl, rr), v = bot_index(sl, rr);
        const int p = min(u, v), q = max(u, v);
        const double hpp = (u < v) ? ndc[sl * 3 + 0] : ndc[sl * 3 + 1];
        const double hqq = (u < v) ? ndc[sl * 3 + 1] : ndc[sl * 3 + 0];
        const double hpq = ndc[sl * 3 + 2];
        double c = 1.0, sv = 0.0;
        if (fabs(hpq) > s_floor && hpq * hpq > 1e-30 * fabs(hpp * hqq) && fabs(hpq) > 1e-300) {
          const float den = fabsf((float)hpp * (float)hqq);
          const float rel2 = den > 0.0f ? fminf(1.0f, (float)hpq * (float)hpq / den) : 1.0f;
          if (fabs(hpq) > s_sig) atomicMax(&maxrel_bits, __float_as_uint(rel2));
          jacobi_angle(hpp, hqq, hpq, c, sv);
          rotated = 1;
        }
        acr[sl] = c;
        asr[sl] = sv;
        apr[sl] = p;
        aqr[sl] = q;
      }
      __syncthreads();
      // (2) the two-sided rotation of every 2x2 block held by this CTA, Eq. 6:
      // M'_{IJ} = J_I^T M_{IJ} J_J for the row pair I of an own slot and every
      // column pair J, in one pass; (3) the four results go straight to the slots
      // their rows move to (tops one slot down, bottoms one slot up, slot 0's top
      // fixed), and a row that lands in a slot also publishes that slot's
      // next-round angle inputs (its diagonal entry, and h_pq if it holds the
      // smaller index) into every CTA's table.  Remote addresses are mapped at
      // each store (one mapa each) rather than held in registers.
      for (int e = threadIdx.x; e < (s1 - s0) * half; e += blockDim.x) {
        const int sl = s0 + e / half, J = e % half;
        const double *top = ROW(cur, sl, 0), *bot = ROW(cur, sl, 1);
        const bool top_is_p = (top_index(sl, rr) == apr[sl]);
        const double *rp = top_is_p ? top : bot, *rq = top_is_p ? bot : top;
        const int pc = apr[J], qc = aqr[J];
        const double cJ = acr[J], sJ = asr[J], c = acr[sl], sv = asr[sl];
        // right factor J_J on the two rows
        const double xp = rp[pc], yp = rp[qc], xq = rq[pc], yq = rq[qc];
        const double p_pc = cJ * xp - sJ * yp, p_qc = sJ * xp + cJ * yp;
        const double q_pc = cJ * xq - sJ * yq, q_qc = sJ * xq + cJ * yq;
        // left factor J_I^T
        double np_pc = c * p_pc - sv * q_pc, np_qc = c * p_qc - sv * q_qc;
        double nq_pc = sv * p_pc + c * q_pc, nq_qc = sv * p_qc + c * q_qc;
        if (J == sl) {          // the rotated pair's own block is diagonal to rounding
          np_qc = 0.0;
          nq_pc = 0.0;
        }
        int dsl[2], dtb[2];
        if (sl == 0) { dsl[0] = 0; dtb[0] = 0; }          // slot 0's top is fixed
        else if (sl == 1) { dsl[0] = 0; dtb[0] = 1; }     // -> slot 0 bottom
        else { dsl[0] = sl - 1; dtb[0] = 0; }
        if (sl == half - 1) { dsl[1] = sl; dtb[1] = 0; } else { dsl[1] = sl + 1; dtb[1] = 1; }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = h == 0 ? pc : qc;
          const double np = h == 0 ? np_pc : np_qc, nq = h == 0 ? nq_pc : nq_qc;
          const double vals[2] = {top_is_p ? np : nq, top_is_p ? nq : np};   // new top, new bottom
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const int own = dsl[w] / spc;
            double *base = cluster.map_shared_rank(rowsb, own) +
                           ((((size_t)1 - cur) * spc + (dsl[w] - own * spc)) * 2 + dtb[w]) * m;
            base[col] = vals[w];
            const int nu = top_index(dsl[w], rn), nv = bot_index(dsl[w], rn);
            const int idx = dtb[w] == 0 ? nu : nv, partner = dtb[w] == 0 ? nv : nu;
            if (col == idx) {
              for (int k = 0; k < kCluster; ++k)
                cluster.map_shared_rank(ndn_local, k)[dsl[w] * 3 + dtb[w]] = vals[w];
            } else if (col == partner && idx < partner) {
              for (int k = 0; k < kCluster; ++k) cluster.map_shared_rank(ndn_local, k)[dsl[w] * 3 + 2] = vals[w];
            }
          }
        }
      }
      // the rows are in place once every CTA has arrived; meanwhile V <- V J on the
      // rows of V this CTA holds (local, needs only the angles)
      asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      for (int e = threadIdx.x; e < (v1 - v0) * half; e += blockDim.x) {
        const int rl = e / half, J = e % half;
        const int pj = apr[J], qj = aqr[J];
        const double x = V[rl * m + pj], y = V[rl * m + qj];
        V[rl * m + pj] = acr[J] * x - asr[J] * y;
        V[rl * m + qj] = asr[J] * x + acr[J] * y;
      }
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
      cur ^= 1;
    }
    // every CTA saw the same angles: the sweep decision needs no exchange.
    // Quadratic convergence: once every rotated entry was below 1e-8 relative,
    // what remains after this sweep is at rounding level.
    __syncthreads();
    stop = (rotated == 0) || __uint_as_float(maxrel_bits) < 1e-16f;
    __syncthreads();
    if (!stop) {
      // Would the next sweep rotate anything?  Every CTA applies the rotation
      // test to the entries of its own rows (diagonal entries from the
      // replicated table of the next round, gathered into `diag`, which is
      // free until the end), the answers are OR-ed across the cluster, and a
      // sweep that would rotate nothing is not run.
      const int rr = r_global % (m - 1);
      const double *ndc = nd + (r_global & 1) * 3 * half;
      for (int sl = threadIdx.x; sl < half; sl += blockDim.x) {
        diag[top_index(sl, rr)] = ndc[sl * 3 + 0];
        diag[bot_index(sl, rr)] = ndc[sl * 3 + 1];
      }
      if (threadIdx.x == 0) s_more = 0;
      __syncthreads();
      for (int e = threadIdx.x; e < (s1 - s0) * 2 * m; e += blockDim.x) {
        const int sl = s0 + e / (2 * m), tb = (e / m) & 1, c = e % m;
        const int idx = tb == 0 ? top_index(sl, rr) : bot_index(sl, rr);
        if (c != idx) {
          const double h = ROW(cur, sl, tb)[c];
          if (fabs(h) > s_floor && h * h > 1e-30 * fabs(diag[idx] * diag[c]) && fabs(h) > 1e-300)
            s_more = 1;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && s_more)
        for (int k = 0; k < kCluster; ++k) atomicExch(cluster.map_shared_rank(&s_any[sweep & 1], k), 1);
      cluster.sync();
      stop = s_any[sweep & 1] == 0;
      __syncthreads();
      if (threadIdx.x == 0) s_any[sweep & 1] = 0;   // reused two sweeps on, after this CTA's next barriers
    }
  }
  // diagonal: each CTA knows the index of every row it holds; gather all m values
  {
    const int rr = r_global % (m - 1);
    for (int e = threadIdx.x; e < (s1 - s0) * 2; e += blockDim.x) {
      const int sl = s0 + (e >> 1), tb = e & 1;
      const int idx = tb == 0 ? top_index(sl, rr) : bot_index(sl, rr);
      const double dv = ROW(cur, sl, tb)[idx];
      for (int k = 0; k < kCluster; ++k) cluster.map_shared_rank(diag, k)[idx] = dv;
    }
  }
  cluster.sync();
  if (threadIdx.x == 0 && rank == 0) {
    if (!stop) atomicExch(flag, 2);
    atomicMax(sweeps, sweep);
  }
  // sort descending (rank of each diagonal entry, ties by index)
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ti = diag[i];
    int rk = 0;
    for (int j = 0; j < m; ++j) {
      const double tj = diag[j];
      rk += (tj > ti) || (tj == ti && j < i);
    }
    if (rank == 0) theta.at(z)[rk] = ti;
    for (int row = v0; row < v1; ++row) Wout.at(z)[(size_t)rk * m + row] = V[(row - v0) * m + i];
  }
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

// ---- Rayleigh-Ritz eigensolver of the small projected matrix H (m x m) ----
//
// GB300 runs FP64 at a few flops per clock per SM, so the two-sided Jacobi
// sweeps from a general H are done first in FP32 (one CTA per problem, all
// disjoint pairs of a round at once, Eq. 6 per 2 x 2 block of the rotated
// rows and columns), which leaves V with V^T H V diagonal to FP32 accuracy.
// V is then made orthonormal to FP64 accuracy by two Newton-Schulz steps,
// H' = V^T H V is formed in FP64, and the FP64 cluster Jacobi finishes on H',
// whose off-diagonal entries are already at FP32 level: quadratic
// convergence takes about two sweeps instead of the ten a general H needs.
// The eigenvectors of H are V W' (W' those of H').

constexpr int kJ32Threads = 1024;
constexpr int kJ32MaxSweeps = 30;

size_t j32_smem(int m) {
  return (size_t)(2 * m * (m + 1) + 2 * (m / 2)) * sizeof(float) + (size_t)(2 * (m / 2)) * sizeof(int);
}

// FP32 cyclic Jacobi on the symmetric m x m matrix C of problem z (m even),
// round-robin pair order (every pair meets once per sweep).  Vout (FP64,
// column-major) receives the accumulated rotation V (columns in the order of
// the final diagonal, unsorted).  A pair is rotated while |h_pq| exceeds both
// 2^-30 of the largest diagonal entry and 1e-6 of sqrt|h_pp h_qq|: entries
// between two small diagonal entries are resolved to FP32 relative accuracy
// (once the couplings to the large ones are small, the rounding noise the
// rotations leave in them is relative to their own size), so that the FP64
// stage starts in its quadratic regime.  The sweeps stop when none was rotated; the count goes to *sweeps
// (maximum over problems).
__global__ void __launch_bounds__(kJ32Threads, 1) k_rr_jacobi32(PSet Cin, int m, PSet Vout, int *sweeps) {
  extern __shared__ float jsh[];
  const int ld = m + 1, half = m / 2;
  float *A = jsh;
  float *V = A + m * ld;
  float *cs = V + m * ld;
  float *sn = cs + half;
  int *pp = reinterpret_cast<int *>(sn + half);
  int *qq = pp + half;
  __shared__ double s_scale;
  __shared__ int s_rot;
  const int z = blockIdx.z;
  const double *C = Cin.at(z);
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < m; i += 32) v = fmax(v, fabs(C[(size_t)i * m + i]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) s_scale = (v > 0.0 && isfinite(v)) ? pow2_inv_of(v) : 1.0;
  }
  __syncthreads();
  const double sc = s_scale;
  // H is symmetric by definition; its stored copy is not where W amplifies
  // rounding (nearly dependent basis columns), and the two-sided rotations of
  // an unsymmetric matrix do not settle: read the symmetric part
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int a = e / m, b = e % m;
    A[a * ld + b] = (float)(0.5 * (C[e] + C[(size_t)b * m + a]) * sc);
    V[a * ld + b] = (a == b) ? 1.0f : 0.0f;
  }
  auto top_index = [&](int sl, int rr) { return (sl == 0) ? 0 : 1 + (sl - 1 + rr) % (m - 1); };
  auto bot_index = [&](int sl, int rr) { return 1 + (m - 2 - sl + rr) % (m - 1); };
  const float floor_abs = 0x1.0p-30f;      // the scaled largest diagonal entry lies in [1, 2)
  int sweep = 0;
  for (; sweep < kJ32MaxSweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        const int u = top_index(k, r), v = bot_index(k, r);
        const int p = min(u, v), q = max(u, v);
        const float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
        float c = 1.0f, sv = 0.0f;
        if (fabsf(apq) > floor_abs && apq * apq > 1e-12f * fabsf(app * aqq)) {
          const float tau = (aqq - app) / (2.0f * apq);
          const float t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
          c = rsqrtf(fmaf(t, t, 1.0f));
          sv = t * c;
          s_rot = 1;
        }
        cs[k] = c;
        sn[k] = sv;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // M'_IJ = J_I^T M_IJ J_J for every 2 x 2 block (the blocks are disjoint)
      for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
        const int I = e / half, J = e % half;
        const int pI = pp[I], qI = qq[I], pJ = pp[J], qJ = qq[J];
        const float cI = cs[I], sI = sn[I], cJ = cs[J], sJ = sn[J];
        const float a00 = A[pI * ld + pJ], a01 = A[pI * ld + qJ];
        const float a10 = A[qI * ld + pJ], a11 = A[qI * ld + qJ];
        const float b00 = cJ * a00 - sJ * a01, b01 = sJ * a00 + cJ * a01;
        const float b10 = cJ * a10 - sJ * a11, b11 = sJ * a10 + cJ * a11;
        float n00 = cI * b00 - sI * b10, n01 = cI * b01 - sI * b11;
        float n10 = sI * b00 + cI * b10, n11 = sI * b01 + cI * b11;
        if (I == J) n01 = n10 = 0.0f;
        A[pI * ld + pJ] = n00;
        A[pI * ld + qJ] = n01;
        A[qI * ld + pJ] = n10;
        A[qI * ld + qJ] = n11;
      }
      // V <- V J
      for (int e = threadIdx.x; e < m * half; e += blockDim.x) {
        const int row = e / half, J = e % half;
        const int pJ = pp[J], qJ = qq[J];
        const float x = V[row * ld + pJ], y = V[row * ld + qJ];
        V[row * ld + pJ] = cs[J] * x - sn[J] * y;
        V[row * ld + qJ] = sn[J] * x + cs[J] * y;
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
    // The sweep that would find nothing to rotate is not run: the rotation
    // test of every off-diagonal entry, once, decides it (m^2 / 2 tests
    // against the m - 1 rounds of a sweep).
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int p = e / m, q = e % m;
      if (q > p) {
        const float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
        if (fabsf(apq) > floor_abs && apq * apq > 1e-12f * fabsf(app * aqq)) s_rot = 1;
      }
    }
    __syncthreads();
    const int more = s_rot;
    __syncthreads();
    if (!more) break;
  }
  if (threadIdx.x == 0) atomicMax(sweeps, sweep + 1);
  double *out = Vout.at(z);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int c = e / m, j = e % m;            // out[j + c m] = V[j][c]
    out[e] = (double)V[j * ld + c];
  }
}

// ---- FP64 finish of the Rayleigh-Ritz eigensolver --------------------------
//
// After the FP32 stage, H' = V^T H V is diagonal to FP32 accuracy: its
// off-diagonal entries e_ij are ~1e-7 of their diagonal pair.  Two steps of a
// simultaneous first-order correction remove them for every pair whose
// diagonal entries are well separated: with A_ij = e_ij / (d_j - d_i) (skew
// symmetric), Q = orth(I + A + A^2 / 2) (one Newton-Schulz step) and
// H' <- Q^T H' Q, the remaining coupling of such a pair is of order
// e_ij^2 / (d_j - d_i); the second step takes it to rounding level.  These are
// dense m x m FP64 products spread over many CTAs (k_rr_mm).  Pairs inside a
// cluster of near-equal diagonal entries (|d_j - d_i| <= kSfsCluster |e_ij|)
// are left out of A and resolved afterwards by exact 2 x 2 rotations
// (Eq. 6) of the sparse Jacobi below, which only rotates the pairs that still
// need it -- instead of full sweeps of (m - 1) rounds over all pairs, which
// a nearly diagonal H' mostly does not need.
constexpr double kSfsCluster = 1e3;

__global__ void k_rr_sfs_build(PSet Hp, int m, PSet Aout) {
  const int z = blockIdx.z;
  const double *h = Hp.at(z);
  double *a = Aout.at(z);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;                      // column-major: a[i + j m]
    double v = 0.0;
    if (i != j) {
      const double eij = 0.5 * (h[(size_t)j * m + i] + h[(size_t)i * m + j]);
      const double gap = h[(size_t)j * m + j] - h[(size_t)i * m + i];
      if (eij != 0.0 && fabs(gap) > kSfsCluster * fabs(eij)) v = eij / gap;
    }
    a[e] = v;
  }
}

// Classical-order ("largest first") two-sided Jacobi on the nearly diagonal
// symmetric m x m matrix Hin (one CTA per problem): each round, every row
// finds the partner with the largest entry that needs rotating (the rotation
// test of k_si_jacobi: above 2^-44 of the largest diagonal entry and not
// negligible against its own diagonal pair), the mutually largest pairs --
// disjoint by construction, and always including the largest entry of the
// matrix -- are rotated at once (Eq. 6), and the accumulated rotation W (in:
// Win, m x m column-major) follows.  Stops when nothing needs rotating;
// *rounds receives the round count (maximum over problems), flag is set to 2
// if kSparseRounds * m rounds do not suffice.  Output as k_si_jacobi: Ritz
// values descending in theta, Wout columns in the same order.
constexpr int kSparseRounds = 16;
constexpr int kSparseThreads = 1024;

size_t sparse_smem(int m) {
  return (size_t)2 * m * (m + 1) * sizeof(double) + (size_t)m * (sizeof(int) + sizeof(double)) +
         (size_t)(m / 2 + 1) * (2 * sizeof(int) + 2 * sizeof(double)) + 64;
}

__global__ void __launch_bounds__(kSparseThreads, 1)
    k_rr_sparse_jacobi(PSet Hin, int m, PSet Win, PSet Wout, PSet theta, int *flag, int *rounds_out) {
  extern __shared__ double ssh[];
  const int ld = m + 1, maxsel = m / 2 + 1;
  double *H = ssh;                                  // row-major, symmetric part of Hin
  double *W = H + (size_t)m * ld;                   // W[r * ld + c] = Win(r, c)
  double *sc = W + (size_t)m * ld;                  // rotation c of selected pair k
  double *ss = sc + maxsel;                         // rotation s
  int *best = reinterpret_cast<int *>(ss + maxsel); // per row: partner with the largest entry, -1
  int *selp = best + m, *selq = selp + maxsel;
  __shared__ int nsel;
  __shared__ double s_floor;
  const int z = blockIdx.z;
  const double *hin = Hin.at(z), *win = Win.at(z);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;                 // column-major inputs: coalesced reads
    H[r * ld + c] = 0.5 * (hin[(size_t)c * m + r] + hin[(size_t)r * m + c]);
    W[r * ld + c] = win[(size_t)c * m + r];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < m; i += 32) v = fmax(v, fabs(H[i * ld + i]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) s_floor = ldexp(v, -44);
  }
  __syncthreads();
  const double fl = s_floor;
  auto needs = [&](double hpp, double hqq, double hpq) {
    return fabs(hpq) > fl && hpq * hpq > 1e-30 * fabs(hpp * hqq) && fabs(hpq) > 1e-300;
  };
  int round = 0;
  bool done = false;
  for (; round < kSparseRounds * m; ++round) {
    // (1) each row's best partner (one warp per row)
    for (int p = warp; p < m; p += nwarps) {
      double bv = 0.0;
      int bq = -1;
      const double hpp = H[p * ld + p];
      for (int q = lane; q < m; q += 32) {
        // the symmetric value: rows p and q must agree on it for the pair to be mutual
        const double h = 0.5 * (H[p * ld + q] + H[q * ld + p]);
        if (q != p && needs(hpp, H[q * ld + q], h) && fabs(h) > bv) {
          bv = fabs(h);
          bq = q;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
        if (ov > bv || (ov == bv && oq > bq)) {
          bv = ov;
          bq = oq;
        }
      }
      if (lane == 0) best[p] = bq;
    }
    if (threadIdx.x == 0) nsel = 0;
    __syncthreads();
    // (2) mutually best pairs, their angles
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const int q = best[p];
      if (q > p && best[q] == p) {
        const int k = atomicAdd(&nsel, 1);
        double c, sv;
        jacobi_angle(H[p * ld + p], H[q * ld + q], 0.5 * (H[p * ld + q] + H[q * ld + p]), c, sv);
        selp[k] = p;
        selq[k] = q;
        sc[k] = c;
        ss[k] = sv;
      }
    }
    __syncthreads();
    const int ns = nsel;
    if (ns == 0) {
      done = true;
      break;
    }
    // (3) right factor: columns p, q of H and W
    for (int e = threadIdx.x; e < ns * m; e += blockDim.x) {
      const int k = e / m, r = e % m, p = selp[k], q = selq[k];
      const double c = sc[k], sv = ss[k];
      const double x = H[r * ld + p], y = H[r * ld + q];
      H[r * ld + p] = c * x - sv * y;
      H[r * ld + q] = sv * x + c * y;
      const double wx = W[r * ld + p], wy = W[r * ld + q];
      W[r * ld + p] = c * wx - sv * wy;
      W[r * ld + q] = sv * wx + c * wy;
    }
    __syncthreads();
    // (4) left factor: rows p, q; the rotated pair's own entries are zero
    for (int e = threadIdx.x; e < ns * m; e += blockDim.x) {
      const int k = e / m, col = e % m, p = selp[k], q = selq[k];
      const double c = sc[k], sv = ss[k];
      const double x = H[p * ld + col], y = H[q * ld + col];
      H[p * ld + col] = (col == q) ? 0.0 : c * x - sv * y;
      H[q * ld + col] = (col == p) ? 0.0 : sv * x + c * y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!done) atomicExch(flag, 2);
    atomicMax(rounds_out, round);
  }
  // sort descending (rank of each diagonal entry, ties by index); best[] now
  // holds the column of each rank
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ti = H[i * ld + i];
    int rk = 0;
    for (int j = 0; j < m; ++j) {
      const double tj = H[j * ld + j];
      rk += (tj > ti) || (tj == ti && j < i);
    }
    theta.at(z)[rk] = ti;
    best[rk] = i;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int row = e % m, rk = e / m;
    Wout.at(z)[e] = W[row * ld + best[rk]];
  }
}

// flags.at(z)[2] = 1 if max |C_ij - delta_ij| > 1/4 (the Newton-Schulz
// iteration for C^-1/2 from I is then not to be trusted), else 0.
__global__ void k_rr_far_from_identity(PSet C, int m, PSet flags) {
  const int z = blockIdx.z;
  double v = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const double d = C.at(z)[e] - ((e % m == e / m) ? 1.0 : 0.0);
    v = fmax(v, (d == d) ? fabs(d) : INFINITY);
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) w = fmax(w, part[i]);
    flags.at(z)[2] = (w > 0.25) ? 1.0 : 0.0;
  }
}

// Out = a A + b I for m x m matrices of every problem z.
__global__ void k_rr_axpi(PSet A, double a, double b, PSet Out, int m) {
  const int z = blockIdx.z;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x)
    Out.at(z)[e] = a * A.at(z)[e] + ((e % m == e / m) ? b : 0.0);
}

// Out = op(A) (bs B + bd I) for m x m column-major FP64 matrices of every
// problem z (op(A) = A^T if ta).  One CTA per 8 x 8 output tile; the sum over
// k is split four ways across the CTA's threads and combined in a fixed order.
__global__ void __launch_bounds__(256) k_rr_mm(PSet A, int ta, PSet B, double bs, double bd,
                                               PSet Out, int m) {
  __shared__ double As[8][kSiMaxBlock + 1];   // op(A) rows i0..i0+7, all k
  __shared__ double Bs[8][kSiMaxBlock + 1];   // B columns j0..j0+7, all k
  __shared__ double part[4][8][9];
  const int z = blockIdx.z;
  const int i0 = blockIdx.x * 8, j0 = blockIdx.y * 8;
  const double *a = A.at(z), *b = B.at(z);
  for (int e = threadIdx.x; e < 8 * m; e += blockDim.x) {
    const int r = e / m, k = e % m;
    const int i = i0 + r, j = j0 + r;
    // op(A)(i, k): A[i + k m] or (transposed) A[k + i m]
    As[r][k] = (i < m) ? (ta ? a[(size_t)i * m + k] : a[(size_t)k * m + i]) : 0.0;
    Bs[r][k] = (j < m) ? bs * b[(size_t)j * m + k] + (k == j ? bd : 0.0) : 0.0;
  }
  __syncthreads();
  const int ti = threadIdx.x & 7, tj = (threadIdx.x >> 3) & 7, ks = threadIdx.x >> 6;
  double acc = 0.0;
  for (int k = ks; k < m; k += 4) acc = fma(As[ti][k], Bs[tj][k], acc);
  part[ks][ti][tj] = acc;
  __syncthreads();
  if (threadIdx.x < 64) {
    const int i = i0 + ti, j = j0 + tj;
    if (i < m && j < m)
      Out.at(z)[(size_t)j * m + i] = (part[0][ti][tj] + part[1][ti][tj]) + (part[2][ti][tj] + part[3][ti][tj]);
  }
}

// Out = A . W  (A, Out n x m column-major; W m x m column-major: W[j + c m])
// tri: W is upper triangular (W[j, c] = 0 for j > c), so j-blocks past the tile's last column are skipped
__global__ void __launch_bounds__(256) k_si_rotate(PSet A, PSet W, PSet Out, int n, int m, int tri) {
  __shared__ double As[32][33];
  __shared__ double Ws[32][33];
  const int z = blockIdx.z;
  const double *a = A.at(z);
  const double *w = W.at(z);
  const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int jend = tri ? min(m, c0 + 32) : m;
  // skip the zero-padded tail of the last j-chunk and the groups of 8 columns
  // that start past m (uniform per block; their loads are zero-filled, so only
  // work is skipped; at m = 72 the padding was 44 % of the FMAs)
  const int ugroups = min(4, (m - c0 + 7) / 8);
  for (int j0 = 0; j0 < jend; j0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int jj = e >> 5, ii = e & 31;
      const int row = i0 + ii, j = j0 + jj;
      As[jj][ii] = (row < n && j < m) ? a[(size_t)j * n + row] : 0.0;
      const int cc = c0 + jj;          // Ws[j][c]: load W[j + cc m] along j
      const int jw = j0 + ii;
      Ws[ii][jj] = (jw < m && cc < m) ? w[(size_t)cc * m + jw] : 0.0;
    }
    __syncthreads();
    const int jn = min(32, jend - j0);
#pragma unroll 8
    for (int jj = 0; jj < jn; ++jj) {
      const double av = As[jj][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < ugroups) acc[u] = fma(av, Ws[jj][ty + 8 * u], acc[u]);
    }
    __syncthreads();
  }
  const int i = i0 + tx;
  if (i < n) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + ty + 8 * u;
      if (c < m) Out.at(z)[(size_t)c * n + i] = acc[u];
    }
  }
}

// res[i] = ||Y_i - theta_i X_i|| / |theta_0|, i < k
// res_i = ||y_i - theta_i x_i|| / theta_0, or 0 for a pair whose unshifted
// value lies below half the shift (2^-41 Tr G: inside the band where G's own
// rounding makes the eigenpairs arbitrary; any orthonormal completion there
// is as good as another)
__global__ void k_si_residual(PSet X, PSet Y, PSet theta, PSet res, PSet sig, int use_sig, int n,
                              int k) {
  const int z = blockIdx.z, i = blockIdx.x;
  const double th = theta.at(z)[i];
  if (use_sig && th - sig.at(z)[0] <= 0.5 * sig.at(z)[1] && i > 0) {
    if (threadIdx.x == 0) res.at(z)[i] = 0.0;
    return;
  }
  const double *x = X.at(z) + (size_t)i * n;
  const double *y = Y.at(z) + (size_t)i * n;
  double v = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double d = y[r] - th * x[r];
    v = fma(d, d, v);
  }
  __shared__ double part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    res.at(z)[i] = sqrt(s) / fabs(theta.at(z)[0]);
  }
}

// G (n x n) into an m x m zero-padded square (m = n or n + 1) for the direct Jacobi path.
__global__ void k_si_copy_square(PSet G, PSet out, int n, int m) {
  const int z = blockIdx.z;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int a = e / m, b = e % m;
    out.at(z)[e] = (a < n && b < n) ? G.at(z)[a * n + b] : 0.0;
  }
}

// X[:, c] = first n rows of W[:, c] for c < k
__global__ void k_si_take(PSet W, PSet X, int n, int m, int k) {
  const int z = blockIdx.z;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += gridDim.x * blockDim.x) {
    const int c = e / n, r = e % n;
    X.at(z)[(size_t)c * n + r] = W.at(z)[(size_t)c * m + r];
  }
}

// Copy of problem z's n x m block from src to dst (final placement of Ritz vectors).
__global__ void k_si_copy(PSet src, PSet dst, long long nm) {
  const int z = blockIdx.z;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nm;
       e += (long long)gridDim.x * blockDim.x)
    dst.at(z)[e] = src.at(z)[e];
}

// ---- host helpers ----

struct Layout {
  int S, NC, m;
  long long nm, mm;
  long long per;   // doubles per problem
  // slot offsets (doubles) inside a problem's workspace
  long long oY, oZ, oX, oYp, oCp, oC, oW, oRes, oTh, oSig;
  // exact-slice operands (BF16 slices and row scales): G, and two general
  // slots for the n x m / m x n / m x m operands of the other products
  int xsp;
  long long oGs, oGsc, oSa, oSasc, oSb, oSbsc, oKs;
};

Layout layout(int P, int n, int m) {
  Layout L;
  L.nm = (long long)n * m;
  L.mm = (long long)m * m;
  L.m = m;
  const int tiles = (n + 63) / 64;
  L.S = std::max(1, std::min(kSplitMax, (2 * 152 + tiles * P - 1) / std::max(1, tiles * P)));
  while (L.S > 1 && (n + L.S - 1) / L.S < 64) --L.S;
  L.NC = std::min(kChunkMax, (n + kRowsPerChunk - 1) / kRowsPerChunk);
  auto up = [](long long v) { return (v + 31) / 32 * 32; };   // 256-byte aligned slots
  long long o = 0;
  L.oY = o; o += up(L.nm);
  L.oZ = o; o += up(L.nm);
  L.oX = o; o += up(L.nm);
  L.oYp = o; o += up(kSplitMax * L.nm);
  L.oCp = o; o += up(kChunkMax * L.mm);
  L.oC = o; o += up(L.mm);
  L.oW = o; o += up(L.mm);
  L.oRes = o; o += up(m);
  L.oTh = o; o += up(m);
  L.oSig = o; o += up(2);
  L.xsp = xs_pitch(n);
  const long long sa = std::max(xs_elems(n, m, kSiSlices), xs_elems(m, n, kSiSlices));
  const long long sb = std::max(xs_elems(m, n, kSiSlices), xs_elems(m, m, kSiSlices));
  L.oGs = o; o += up((xs_elems(n, n, kSiSlices) + 3) / 4);
  L.oGsc = o; o += up(n);
  L.oSa = o; o += up((sa + 3) / 4);
  L.oSasc = o; o += up(std::max(n, m));
  L.oSb = o; o += up((sb + 3) / 4);
  L.oSbsc = o; o += up(std::max(n, m));
  L.oKs = o; o += up(m);
  L.per = o;
  return L;
}

struct Bufs {
  PSet Y, Z, X, Yp, Cp, C, W, res, th, sig;
  int *flag, *sweeps;
};

Bufs carve(double *work, int P, const Layout &L) {
  Bufs B;
  B.Y = pset_linear(work + L.oY, L.per);
  B.Z = pset_linear(work + L.oZ, L.per);
  B.X = pset_linear(work + L.oX, L.per);
  B.Yp = pset_linear(work + L.oYp, L.per);
  B.Cp = pset_linear(work + L.oCp, L.per);
  B.C = pset_linear(work + L.oC, L.per);
  B.W = pset_linear(work + L.oW, L.per);
  B.res = pset_linear(work + L.oRes, L.per);
  B.th = pset_linear(work + L.oTh, L.per);
  B.sig = pset_linear(work + L.oSig, L.per);
  B.flag = reinterpret_cast<int *>(work + (long long)P * L.per);
  B.sweeps = B.flag + 2;
  return B;
}

bool same(const PSet &a, const PSet &b) { return a.b0 == b.b0 && a.b1 == b.b1 && a.stride == b.stride; }

size_t jacobi_smem(int m) {
  const int half = m / 2;
  const int spc = (half + kCluster - 1) / kCluster, vrows = (m + kCluster - 1) / kCluster;
  return ((size_t)2 * spc * 2 * m + (size_t)vrows * m + 4 * half + 6 * half + m) * sizeof(double) +
         (size_t)(4 * half) * sizeof(int) + 64;
}
size_t chol_smem(int m) { return (size_t)(2 * m * (m + 1) + 2 * m) * sizeof(double); }
size_t chol32_smem(int m) {
  const int nb = (m + kCholPanel - 1) / kCholPanel;
  return (size_t)(2 * m * (m + 1) + m + nb * kCholPanel * kCholPanel) * sizeof(float);
}

cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e;
  const int big = 200 * 1024;
  if ((e = cudaFuncSetAttribute(k_si_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) ||
      (e = cudaFuncSetAttribute(k_si_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) ||
      (e = cudaFuncSetAttribute(k_si_chol32, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) ||
      (e = cudaFuncSetAttribute(k_rr_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) ||
      (e = cudaFuncSetAttribute(k_rr_sparse_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))
    return e;
  done = true;
  return cudaSuccess;
}

int grid_1d(long long count, int P) {
  long long b = (count + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(b, (152 * 4 + P - 1) / P));
}

cudaError_t launch_jacobi(PSet C, int m, PSet W, PSet theta, int *flag, int *sweeps, int P,
                          cudaStream_t s, int floor_exp = 56, int sig_exp = 2000) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(kCluster, 1, P);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = jacobi_smem(m);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_si_jacobi, C, m, W, theta, flag, sweeps, floor_exp, sig_exp);
}

}  // namespace

long long si_workspace_doubles(int P, int n, int m) {
  return layout(P, n, m).per * P + 64;
}

int jacobi_block(int n) {
  const int m = n + (n & 1);
  return m < 4 ? 4 : m;
}

SiOut si_outputs(double *work, int P, int n, int m) {
  const Layout L = layout(P, n, m);
  Bufs B = carve(work, P, L);
  return SiOut{B.X, B.th};
}

cudaError_t jacobi_full(const SiBatch &b, double *work, cudaStream_t s, long long *launches) {
  cudaError_t e = set_attrs();
  if (e) return e;
  const int n = b.n, P = b.P;
  int m = n + (n & 1);              // the round-robin pairing needs an even size
  if (m < 4) m = 4;                 // and at least two pairs
  if (m > kSiMaxBlock || b.k > n || P > 65535) return cudaErrorInvalidValue;
  const Layout L = layout(P, n, m);
  Bufs B = carve(work, P, L);
  if ((e = cudaMemsetAsync(B.flag, 0, 4 * sizeof(int), s))) return e;
  k_si_copy_square<<<dim3(grid_1d((long long)m * m, P), 1, P), 256, 0, s>>>(b.G, B.C, n, m);
  if ((e = launch_jacobi(B.C, m, B.W, B.th, B.flag, B.sweeps, P, s))) return e;
  k_si_take<<<dim3(grid_1d((long long)n * b.k, P), 1, P), 256, 0, s>>>(B.W, B.X, n, m, b.k);
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t si_solve(const SiBatch &b, double *work, double tol, int max_iter, cudaStream_t s,
                     SiResult *res, long long *launches) {
  cudaError_t e = set_attrs();
  if (e) return e;
  const int P = b.P, n = b.n, m = b.m, k = b.k;
  if (P < 1 || P > 65535 || m > kSiMaxBlock || m > n || k > m || (m & 1))
    return cudaErrorInvalidValue;
  const Layout L = layout(P, n, m);
  Bufs B = carve(work, P, L);
  PSet X = B.X, Y = B.Y, Z = B.Z;
  const dim3 gz(1, 1, P);
  const dim3 grot((n + 31) / 32, (m + 31) / 32, P);
  const int chunk = ((n + L.S - 1) / L.S + 15) / 16 * 16;
  const double shift = 11.0 * ((double)n * m + (double)m * (m + 1)) * 1.1102230246251565e-16;
  long long nl = 0;

  // Products over the long dimension n (G X, the basis rotations X W and the
  // Gram matrices X^T Y) run as exact-slice tensor-core GEMMs (FP64-grade, see
  // tc_exact.cuh) unless the caller asked for the FP64 SIMT kernels.  The
  // n x m x m rotations and Gram matrices go to the tensor cores only when the
  // batch makes them FP64-throughput bound (P n m^2 >= kXsSmallWork); below
  // that the single SIMT launch beats the slice-and-multiply sequence.
  const bool xs = b.xs;
  const bool xs_small = xs && (double)P * n * m * m >= kXsSmallWork;
  XsOperand gs{};
  int xsplit = 1, gsplit = 1;
  // slices of a row-major (rows x K) view of problem z's buffer at src
  auto xs_slot = [&](long long off, long long scoff, int rows, int K) {
    return XsOperand{work + off, work + scoff, rows, K, xs_pitch(K), kSiSlices, P, L.per * 4, L.per};
  };
  if (xs) {
    gs = XsOperand{work + L.oGs, work + L.oGsc, n, n, L.xsp, kSiSlices, P, L.per * 4, L.per};
    const int tiles = ((n + 127) / 128) * ((m + 95) / 96) * P;
    xsplit = std::max(xs_min_split(n), std::min(kSplitMax, (2 * 152 + tiles - 1) / tiles));
    while (xsplit > xs_min_split(n) && (n + xsplit - 1) / xsplit < 128) --xsplit;
    const int gtiles = ((m + 79) / 80) * P;
    gsplit = std::max(xs_min_split(n), std::min(std::min(kChunkMax, n / 64), (2 * 152 + gtiles - 1) / gtiles));
    if ((e = xs_split(b.G, map1(n), map1(1), gs, s))) return e;
    nl += 1;
  }
  auto add_shift = [&](PSet src, PSet dst) -> cudaError_t {
    if (!b.has_trace) return cudaSuccess;
    k_si_shift_add<<<dim3(grid_1d(L.nm, P), 1, P), 256, 0, s>>>(dst, src, B.sig, L.nm);
    nl += 1;
    return cudaGetLastError();
  };
  // dst = G src; where the K parts are summed by a separate pass, that pass
  // also adds the shift (shifted = true)
  bool shifted = false;
  auto product = [&](PSet src, PSet dst) -> cudaError_t {
    shifted = false;
    const int sh = b.has_trace ? 1 : 0;
    if (xs) {
      const XsOperand xsl = xs_slot(L.oSb, L.oSbsc, m, n);     // rows of X^T
      cudaError_t r = xs_split(src, map1(n), map1(1), xsl, s);
      if (r) return r;
      if (xsplit == 1) {
        r = xs_gemm(gs, xsl, n, m, n, dst.b0, map1(1), map1(n), L.per, 1, 0, b.err, s);
        nl += 2;
      } else {
        r = xs_gemm(gs, xsl, n, m, n, B.Yp.b0, map1(1), map1(n), L.per, xsplit, L.nm, b.err, s);
        if (r) return r;
        k_si_sum_split<<<dim3(grid_1d(L.nm, P), 1, P), 256, 0, s>>>(B.Yp, dst, xsplit, L.nm, src, B.sig, sh);
        shifted = true;
        nl += 3;
      }
      return r ? r : cudaGetLastError();
    }
    if (L.S == 1) {
      k_si_gemm<<<dim3((n + 63) / 64, 1, P), 256, 0, s>>>(b.G, src, dst, n, m, chunk);
      nl += 1;
    } else {
      k_si_gemm<<<dim3((n + 63) / 64, L.S, P), 256, 0, s>>>(b.G, src, B.Yp, n, m, chunk);
      k_si_sum_split<<<dim3(grid_1d(L.nm, P), 1, P), 256, 0, s>>>(B.Yp, dst, L.S, L.nm, src, B.sig, sh);
      shifted = true;
      nl += 2;
    }
    return cudaGetLastError();
  };
  auto gemm = [&](PSet src, PSet dst) -> cudaError_t {
    cudaError_t r0 = product(src, dst);
    return r0 ? r0 : (shifted ? cudaSuccess : add_shift(src, dst));
  };
  // dst = src W (n x m times m x m, W column-major; tri: W upper triangular).
  // A CholeskyQR basis change (tri) normalises columns whose lengths can differ
  // by many orders of magnitude: the exact-slice product then scales column j
  // of src by a power of two near 1 / |src_j| (and row j of W inversely), so
  // that the row slicing of src keeps every column's relative accuracy.
  auto rot = [&](PSet src, PSet W, PSet dst, int tri) -> cudaError_t {
    if (xs_small) {
      const XsOperand a = xs_slot(L.oSa, L.oSasc, n, m);       // rows of X
      const XsOperand w = xs_slot(L.oSb, L.oSbsc, m, m);       // columns of W
      const PSet ks = pset_linear(work + L.oKs, L.per);
      cudaError_t r;
      if (tri) {
        k_si_colscale<<<dim3(1, 1, P), 128, 0, s>>>(B.C, ks, m);
        nl += 1;
      }
      if ((r = xs_split_scaled(src, map1(1), map1(n), ks, tri ? 1 : 0, a, s)) ||
          (r = xs_split_scaled(W, map1(m), map1(1), ks, tri ? 2 : 0, w, s)) ||
          (r = xs_gemm(a, w, n, m, m, dst.b0, map1(1), map1(n), L.per, 1, 0, b.err, s)))
        return r;
      nl += 3;
      return cudaSuccess;
    }
    k_si_rotate<<<grot, 256, 0, s>>>(src, W, dst, n, m, tri);
    nl += 1;
    return cudaGetLastError();
  };
  // C = A^T B (m x m), symmetrised; ns: write the Newton-Schulz polish (3I - C)/2 instead
  auto gram = [&](PSet A, PSet Bm, bool sym, bool f32, bool ns, PSet out) -> cudaError_t {
    if (xs_small) {
      const XsOperand a = xs_slot(L.oSa, L.oSasc, m, n);       // columns of A
      const XsOperand bb = xs_slot(L.oSb, L.oSbsc, m, n);      // columns of B
      cudaError_t r;
      if ((r = xs_split(A, map1(n), map1(1), a, s))) return r;
      const bool one = same(A, Bm);
      if (!one && (r = xs_split(Bm, map1(n), map1(1), bb, s))) return r;
      if ((r = xs_gemm(a, one ? a : bb, m, m, n, B.Cp.b0, map1(m), map1(1), L.per, gsplit, L.mm,
                       b.err, s)))
        return r;
      k_si_gram_reduce<<<dim3(grid_1d(L.mm, P), 1, P), 256, 0, s>>>(B.Cp, out, gsplit, m, 0, ns);
      nl += one ? 3 : 4;
      return cudaGetLastError();
    }
    if (f32)
      k_si_gram<float><<<dim3(L.NC, 1, P), 256, 0, s>>>(A, Bm, B.Cp, n, m, sym);
    else
      k_si_gram<double><<<dim3(L.NC, 1, P), 256, 0, s>>>(A, Bm, B.Cp, n, m, sym);
    k_si_gram_reduce<<<dim3(grid_1d(L.mm, P), 1, P), 256, 0, s>>>(B.Cp, out, L.NC, m, sym, ns);
    nl += 2;
    return cudaGetLastError();
  };
  // Eigenpairs of the projected matrix H (in B.C) into B.W (columns, descending)
  // and B.th: FP32 Jacobi -> FP64 Newton-Schulz orthonormalisation -> FP64
  // cluster Jacobi on H' = V^T H V -> W = V W'.  Scratch: three m x m slots in
  // the (then unused) Gram-partial region.
  auto small_eig = [&]() -> cudaError_t {
    auto slot = [&](int i) { return PSet{B.Cp.b0 + i * L.mm, B.Cp.b1 + i * L.mm, B.Cp.stride}; };
    const PSet V1 = slot(0), V2 = slot(1), T1 = slot(2);
    const dim3 gmm((m + 7) / 8, (m + 7) / 8, P);
    k_rr_jacobi32<<<gz, kJ32Threads, j32_smem(m), s>>>(B.C, m, V1, B.flag + 3);
    k_rr_mm<<<gmm, 256, 0, s>>>(V1, 1, V1, 1.0, 0.0, T1, m);      // T1 = V1^T V1
    k_rr_mm<<<gmm, 256, 0, s>>>(V1, 0, T1, -0.5, 1.5, V2, m);     // V2 = V1 (3I - T1) / 2
    k_rr_mm<<<gmm, 256, 0, s>>>(V2, 1, V2, 1.0, 0.0, T1, m);
    k_rr_mm<<<gmm, 256, 0, s>>>(V2, 0, T1, -0.5, 1.5, V1, m);     // V1 orthonormal (FP64)
    k_rr_mm<<<gmm, 256, 0, s>>>(B.C, 0, V1, 1.0, 0.0, T1, m);     // T1 = H V1
    k_rr_mm<<<gmm, 256, 0, s>>>(V1, 1, T1, 1.0, 0.0, V2, m);      // V2 = V1^T H V1
    nl += 7;
    cudaError_t r;
    if ((r = cudaGetLastError())) return r;
    // FP64 finish: two first-order correction steps (k_rr_sfs_build above),
    // W' = Q1 Q2, then the sparse Jacobi on what still needs rotating.  H'
    // comes from two FP64 products: its entries carry rounding noise of about
    // m u ||H|| (2^-46 at m = 72), so entries below 2^-44 of its largest
    // diagonal entry are left alone (their effect on a residual is below
    // 1e-13 of the largest eigenvalue).
    const PSet Am = slot(4), Q0 = slot(5), Tq = slot(6), Qm = slot(7), Tt = slot(8);
    const dim3 g1(grid_1d(L.mm, P), 1, P);
    for (int step = 0; step < 2; ++step) {
      k_rr_sfs_build<<<g1, 256, 0, s>>>(V2, m, Am);
      k_rr_mm<<<gmm, 256, 0, s>>>(Am, 0, Am, 0.5, 1.0, Q0, m);       // A + A^2 / 2
      k_rr_axpi<<<g1, 256, 0, s>>>(Q0, 1.0, 1.0, Q0, m);              // + I
      k_rr_mm<<<gmm, 256, 0, s>>>(Q0, 1, Q0, 1.0, 0.0, Tq, m);        // Q0^T Q0
      k_rr_mm<<<gmm, 256, 0, s>>>(Q0, 0, Tq, -0.5, 1.5, Qm, m);       // Q = Q0 (3I - Q0^T Q0) / 2
      k_rr_mm<<<gmm, 256, 0, s>>>(V2, 0, Qm, 1.0, 0.0, Tt, m);        // H' Q
      k_rr_mm<<<gmm, 256, 0, s>>>(Qm, 1, Tt, 1.0, 0.0, V2, m);        // H' <- Q^T H' Q
      if (step == 0) {
        k_si_copy<<<g1, 256, 0, s>>>(Qm, T1, L.mm);                    // W' = Q1
        nl += 8;
      } else {
        k_rr_mm<<<gmm, 256, 0, s>>>(T1, 0, Qm, 1.0, 0.0, Tt, m);      // W' Q2
        k_si_copy<<<g1, 256, 0, s>>>(Tt, T1, L.mm);
        nl += 9;
      }
    }
    k_rr_sparse_jacobi<<<gz, kSparseThreads, sparse_smem(m), s>>>(V2, m, T1, T1, B.th, B.flag, B.sweeps);
    nl += 1;
    if ((r = cudaGetLastError())) return r;
    k_rr_mm<<<gmm, 256, 0, s>>>(V1, 0, T1, 1.0, 0.0, B.W, m);     // W = V1 W'
    nl += 2;
    return cudaGetLastError();
  };
  // one CholeskyQR pass with an FP32 factorisation: dst = src W
  auto cholqr32 = [&](PSet src, PSet dst, float sh) -> cudaError_t {
    cudaError_t r = gram(src, src, true, true, false, B.C);
    if (r) return r;
    k_si_chol32<<<gz, kCholThreads, chol32_smem(m), s>>>(B.C, m, sh, B.W, B.flag);
    nl += 1;
    return rot(src, B.W, dst, 1);
  };
  // one CholeskyQR pass in FP64 (robust for any conditioning with the shift)
  auto cholqr64 = [&](PSet src, PSet dst, double sh) -> cudaError_t {
    cudaError_t r = gram(src, src, true, false, false, B.C);
    if (r) return r;
    k_si_chol<<<gz, kCholThreads, chol_smem(m), s>>>(B.C, m, sh, B.W, B.flag, PSet{nullptr, nullptr, 0});
    nl += 1;
    return rot(src, B.W, dst, 1);
  };
  // dst = orth(src) through tmp (src is overwritten).  After the first
  // Rayleigh-Ritz step the basis holds Ritz vectors, G X is X Theta up to the
  // residual, its column-scaled Gram matrix is close to I, and one CholeskyQR
  // pass with an FP32 factorisation suffices for the power iteration.  Before
  // it the block can be ill conditioned.  Small batches (latency bound: the
  // single-CTA FP64 factorisation costs more than its iterations save) use the
  // same two FP32 passes, the first of which retries with a diagonal shift
  // where the columns are nearly dependent; large batches use shifted
  // CholeskyQR3 in FP64, which keeps more of the ill-conditioned directions and
  // saves iterations on their hardest problems.
  //
  // A block that holds numerically null directions of G (Ritz values below
  // 1e-9 of the largest: rank-deficient environments at fixed points and in
  // limits such as the classical Ising chain) cannot be orthogonalised in FP32:
  // each FP32 pass leaves about 1e-7 of the dominant directions in the null
  // columns, and the next product amplifies it by theta_0 / sigma (~1e12), so
  // the basis collapses.  Once a Rayleigh-Ritz step sees such directions, the
  // rest of the solve orthogonalises with two FP64 CholeskyQR passes.
  const bool fp64_start = P > kSiSmallBatch;
  bool orth64 = false;
  int n_orth = 0;
  auto orth = [&](PSet src, PSet tmp, PSet dst, bool after_rr) -> cudaError_t {
    cudaError_t r;
    ++n_orth;
    if (orth64) {
      if ((r = cholqr64(src, tmp, shift))) return r;
      return cholqr64(tmp, dst, 0.0);
    }
    // One FP32 pass once the columns are close to eigenvectors (after a
    // Rayleigh-Ritz step, or from the third iteration of a warm start): the
    // column-scaled Gram matrix of G X is then close to I and one pass leaves
    // X orthonormal to about FP32 accuracy, which is all the power iteration
    // needs -- the Rayleigh-Ritz step works with C0 = X^T X and does not
    // assume an orthonormal basis (measured at D = 32: 8.5 iterations per
    // step either way, 0.6 ms less per step).
    if (after_rr || (b.has_warm && n_orth >= 3)) return cholqr32(src, dst, 0.0f);
    if (!fp64_start) {
      if ((r = cholqr32(src, tmp, 0.0f))) return r;
      return cholqr32(tmp, dst, 0.0f);
    }
    if ((r = cholqr64(src, tmp, shift)) || (r = cholqr64(tmp, src, 0.0))) return r;
    return cholqr64(src, dst, 0.0);
  };

  if ((e = cudaMemsetAsync(B.flag, 0, 4 * sizeof(int), s))) return e;
  if (b.has_trace) {
    k_si_sigma_init<<<dim3(1, 1, P), 32, 0, s>>>(B.sig, b.trace, b.shift_rel);
    nl += 1;
  }
  k_si_init<<<dim3(grid_1d(L.nm, P), 1, P), 256, 0, s>>>(X, b.warm, b.has_warm ? 1 : 0, b.kw, n, m);
  nl += 1;
  // a random or partly warm start is orthogonalised (well conditioned); a start
  // from all m Ritz vectors of the previous solve is orthonormal to FP64 accuracy
  // already (the final rotation of a Rayleigh-Ritz step)
  if (!(b.has_warm && b.kw >= m)) {
    if ((e = cholqr32(X, Z, 0.0f)) || (e = cholqr32(Z, Y, 0.0f))) return e;
    std::swap(X, Y);
  }

  res->converged = false;
  res->breakdown = 0;
  res->sweeps64 = 0;
  res->sweeps32 = 0;
  res->rr = 0;
  res->residual = INFINITY;
  int it = 0;
  // With the FP32 start-up a Rayleigh-Ritz step costs several iterations:
  // the first one goes where the caller expects convergence.
  int next_check = fp64_start ? 3 : std::max(3, b.first_check);
  std::vector<double> hres((size_t)P * k), hth((size_t)P * m);
  // HOTRG_TRACE_EIG=1 (or 2, with every residual and Ritz value) prints each
  // convergence check of the solve to stderr
  static const int trace = getenv("HOTRG_TRACE_EIG") ? atoi(getenv("HOTRG_TRACE_EIG")) : 0;
  double prev_worst = INFINITY;
  while (it < max_iter) {
    const bool check = (it + 1 >= next_check) || (it + 1 == max_iter);
    if ((e = gemm(X, Y))) return e;  // Y = G X
    ++it;
    if (check) {
      // Rayleigh-Ritz on the span of X, whose columns the FP32 CholeskyQR left
      // orthonormal only to about its own accuracy: with C0 = X^T X and
      // W = C0^(-1/2) (Newton-Schulz on the m x m side, from C0 ~ I), X W is
      // orthonormal to FP64 accuracy, G X W = Y W, and the projected matrix
      // is H = W^T (X^T Y) W.  Its eigenvectors Z give the Ritz vectors X (W Z)
      // and G X (W Z) = Y (W Z) with one rotation each.
      auto slot = [&](int i) { return PSet{B.Cp.b0 + i * L.mm, B.Cp.b1 + i * L.mm, B.Cp.stride}; };
      const PSet Wn = slot(3), Tn = slot(4), Ck = slot(5), Rr = slot(6);
      const dim3 gmm((m + 7) / 8, (m + 7) / 8, P), g1(grid_1d(L.mm, P), 1, P);
      if ((e = gram(X, X, true, false, false, B.W))) return e;   // C0 (B.W until small_eig)
      if ((e = gram(X, Y, false, false, false, B.C))) return e;  // X^T Y
      k_rr_axpi<<<g1, 256, 0, s>>>(B.W, -0.5, 1.5, Wn, m);       // W1 = (3I - C0) / 2
      nl += 1;
      for (int ns = 0; ns < 3; ++ns) {                              // W <- W (3I - W^T C0 W) / 2
        k_rr_mm<<<gmm, 256, 0, s>>>(B.W, 0, Wn, 1.0, 0.0, Tn, m);   // C0 W
        k_rr_mm<<<gmm, 256, 0, s>>>(Wn, 1, Tn, 1.0, 0.0, Ck, m);    // W^T C0 W
        k_rr_mm<<<gmm, 256, 0, s>>>(Wn, 0, Ck, -0.5, 1.5, Tn, m);   // next W
        k_si_copy<<<g1, 256, 0, s>>>(Tn, Wn, L.mm);
        nl += 4;
      }
      // where X is far from orthonormal (nearly dependent columns at a first
      // check), W comes instead from a shifted FP64 Cholesky of C0 (X W is
      // then orthonormal for any conditioning the shift allows)
      k_rr_far_from_identity<<<gz, 256, 0, s>>>(B.W, m, B.sig);
      k_si_chol<<<gz, kCholThreads, chol_smem(m), s>>>(B.W, m, shift, Wn, B.flag, B.sig);
      nl += 2;
      k_rr_mm<<<gmm, 256, 0, s>>>(B.C, 0, Wn, 1.0, 0.0, Tn, m);     // (X^T Y) W
      k_rr_mm<<<gmm, 256, 0, s>>>(Wn, 1, Tn, 1.0, 0.0, Ck, m);      // H = W^T X^T Y W
      k_si_copy<<<g1, 256, 0, s>>>(Ck, B.C, L.mm);
      nl += 3;
      if ((e = cudaGetLastError())) return e;
      if ((e = small_eig())) return e;                              // H = Z Theta Z^T (Z in B.W)
      k_rr_mm<<<gmm, 256, 0, s>>>(Wn, 0, B.W, 1.0, 0.0, Rr, m);     // R = W Z
      nl += 1;
      if ((e = rot(X, Rr, Z, 0))) return e;
      std::swap(X, Z);
      if ((e = rot(Y, Rr, Z, 0))) return e;
      std::swap(Y, Z);
      k_si_residual<<<dim3(k, 1, P), 256, 0, s>>>(X, Y, B.th, B.res, B.sig, b.has_trace ? 1 : 0, n, k);
      nl += 2;
      ++res->rr;
      if ((e = cudaMemcpy2DAsync(hres.data(), sizeof(double) * k, B.res.at(0), sizeof(double) * L.per,
                                 sizeof(double) * k, P, cudaMemcpyDeviceToHost, s)))
        return e;
      if ((e = cudaMemcpy2DAsync(hth.data(), sizeof(double) * m, B.th.at(0), sizeof(double) * L.per,
                                 sizeof(double) * m, P, cudaMemcpyDeviceToHost, s)))
        return e;
      int hflag[4];
      if ((e = cudaMemcpyAsync(hflag, B.flag, sizeof(hflag), cudaMemcpyDeviceToHost, s))) return e;
      if ((e = cudaStreamSynchronize(s))) return e;
      double worst = 0.0;
      int wp = 0, wi = 0;
      for (int q = 0; q < P * k; ++q) {
        const double v = std::isfinite(hres[q]) ? hres[q] : INFINITY;
        if (v > worst) {
          worst = v;
          wp = q / k;
          wi = q % k;
        }
      }
      res->residual = worst;
      if (trace) {
        const double *th = hth.data() + (size_t)wp * m;
        fprintf(stderr,
                "[hotrg eig] n %d m %d k %d P %d it %d rr %d worst %.3e at problem %d pair %d: "
                "theta_i/theta_0 %.6e theta_k/theta_0 %.6e theta_m/theta_0 %.6e sweeps %d/%d flag %d\n",
                n, m, k, P, it, res->rr, worst, wp, wi, th[wi] / th[0], th[k - 1] / th[0],
                th[m - 1] / th[0], hflag[3], hflag[2], hflag[0]);
        if (trace > 1) {
          fprintf(stderr, "[hotrg eig]   residuals:");
          for (int i = 0; i < k; ++i) fprintf(stderr, " %.1e", hres[(size_t)wp * k + i]);
          fprintf(stderr, "\n[hotrg eig]   theta/theta_0:");
          for (int i = 0; i < m; ++i) fprintf(stderr, " %.4e", th[i] / th[0]);
          fprintf(stderr, "\n");
        }
      }
      res->breakdown = hflag[0];
      res->sweeps64 = hflag[2];
      res->sweeps32 = hflag[3];
      if (hflag[0]) break;          // breakdown: reported to the caller
      // Converged at the bound, or at the accuracy floor of G: a residual
      // below the floor that no longer halves between two Rayleigh-Ritz
      // steps cannot be improved by more iterations (the exact-slice products
      // reach about 1e-12 relative at n = 4096; an environment built with
      // reduced-precision products carries a noise floor of eigenvalues whose
      // vectors are not determined beyond that noise).
      const double floor_tol = b.floor_tol > 0.0 ? b.floor_tol : kSiFloorTol;
      const bool stalled = worst <= floor_tol && res->rr >= 2 && worst > 0.5 * prev_worst;
      // In a flat tail of noise-level eigenvalues (reduced-precision G) the
      // wanted pairs converge at a rate near 1: after kSiSlowIters iterations
      // a residual below the accuracy floor of G is accepted.
      const bool slow = b.floor_tol > 0.0 && worst <= floor_tol && it >= kSiSlowIters;
      if (worst <= tol || stalled || slow) {
        res->converged = true;
        break;
      }
      prev_worst = worst;
      // A Ritz value well below zero is as telling where G is accurate to FP64
      // (G + sigma I is positive definite): the FP32 passes have let the block
      // collapse onto nearly dependent columns.
      for (int p = 0; p < P && !orth64; ++p) {
        const double t0 = hth[(size_t)p * m], tm = hth[(size_t)p * m + m - 1];
        if (!(fabs(tm) > 1e-9 * fabs(t0))) orth64 = true;
        if (b.floor_tol == 0.0 && tm < -1e-9 * fabs(t0)) orth64 = true;
      }
      // Errors in the wanted Ritz pairs shrink by about theta_m / theta_k per
      // iteration: schedule the next check where that predicts convergence.
      double rho = 0.0;
      for (int p = 0; p < P; ++p) {
        const double tk = fabs(hth[(size_t)p * m + k - 1]), tm = fabs(hth[(size_t)p * m + m - 1]);
        rho = std::max(rho, tk > 0.0 ? tm / tk : 1.0);
      }
      int need = 2;
      if (rho > 0.0 && rho < 0.9 && std::isfinite(worst) && worst > 0.0)
        need = (int)std::ceil(std::log(tol / worst) / std::log(rho)) + 1;
      next_check = it + std::max(1, std::min(need, 8));
    }
    if ((e = orth(Y, Z, X, res->rr > 0))) return e;   // X = orth(G X)
  }
  res->iterations = it;
  if (b.has_trace) {
    k_si_unshift<<<dim3(1, 1, P), 128, 0, s>>>(B.th, B.sig, m);
    nl += 1;
  }
  // the Ritz vectors end in the workspace's X slot
  if (!same(X, B.X)) {
    k_si_copy<<<dim3(grid_1d(L.nm, P), 1, P), 256, 0, s>>>(X, B.X, L.nm);
    nl += 1;
  }
  *launches += nl;
  return cudaGetLastError();
}

}  // namespace hotrg
