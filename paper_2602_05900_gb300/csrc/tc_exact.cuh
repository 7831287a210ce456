// Exact-slice GEMM: FP64-grade products on the BF16 tensor cores (sm_103a).
//
// GB300 executes FP64 at a few flops per clock per SM, BF16 tensor-core MMAs at
// thousands.  An FP64 operand row is written as 2^e (a_1 2^-6 + a_2 2^-12 + ...
// + a_S 2^-6S) with integers |a_1| <= 64, |a_s| <= 32 (round-to-nearest
// digits of the row scaled below 1); each digit times its power of two is an
// exact BF16 value (a "slice").  The product of two rows is then the sum over
// slice pairs (s, t) of exact BF16 x BF16 products; pairs with s + t <= S + 1
// are kept (the rest lie below 2^-6(S+1) of the leading term).  Pairs with the
// same s + t = d share one FP32 accumulator in tensor memory; for d <= 6 every
// partial sum is an integer multiple of 2^-6d below 2^24 of that unit as long as
// K <= kXsMaxK (the d = 6 sum has five terms of at most 2^11, 2^10, 2^10,
// 2^10, 2^11 per k), so those accumulators are exact whatever the order of
// summation, and all d >= 7 pairs share one more, inexact but 2^-30 smaller,
// accumulator (the tensor cores' FP32 accumulation truncates, so its error
// grows with K; one level lower it set the error floor near 2^-44).  The
// epilogue combines the exact accumulators in 64-bit integer arithmetic, adds
// the small one and the row and column scales in FP64.  With
// S slices the result is within about 2^-(6S-1) of max|A_i.| max|B_j.| per
// term; the eigensolver's products G X use S = 8 (about 2^-47: FP64-grade).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hotrg {

constexpr int kXsBits = 6;        // bits per slice digit
constexpr int kXsExactDiagonals = 5;  // digit sums d = 2..6 accumulate exactly
constexpr int kXsMaxK = 2336;     // largest K (multiple of 32) with 7 2^10 K < 2^24
constexpr int kXsMaxSlices = 8;
constexpr int kXsStagedK = 128;  // strided-K operands up to this K are sliced through shared memory

// Sliced operand: S planes of rows x pitch BF16 values (plane stride
// rows * pitch elements, K contiguous) and one power-of-two scale per row, for
// `batch` instances at fixed strides.
struct XsOperand {
  void *slices;        // __nv_bfloat16
  double *scale;
  int rows, K, pitch, S;
  int batch;
  long long bstride;   // BF16 elements between instances
  long long sstride;   // doubles between instances' scales
};

// Row pitch (elements) with a 16-byte multiple byte pitch.
inline int xs_pitch(int K) { return (K + 7) / 8 * 8; }
// BF16 elements of one instance's slices.
inline long long xs_elems(int rows, int K, int S) { return (long long)S * rows * xs_pitch(K); }

// Slices row r of instance z, whose element k is src.at(z)[rm(r) + km(k)].
cudaError_t xs_split(PSet src, IdxMap rm, IdxMap km, const XsOperand &dst, cudaStream_t s);

// The same with element k multiplied (kmode 1) or divided (kmode 2) by
// kscale.at(z)[k], a power of two (exact).  A product A B^T with A's columns
// and B's columns scaled inversely is unchanged, but the row slicing then
// sees balanced rows: used where the columns of A differ by many orders of
// magnitude (a column-normalising basis change).
cudaError_t xs_split_scaled(PSet src, IdxMap rm, IdxMap km, PSet kscale, int kmode,
                            const XsOperand &dst, cudaStream_t s);

// C(m, n) = sum_k A(m, k) B(n, k) in FP64 for every instance z, written to
// C + z * cstride + cm(m) + cn(n).  The K range is cut into `ksplit` equal
// parts (each <= kXsMaxK); part p is written at C + p * pstride (the caller
// sums the parts).  A.S == B.S, A.batch == B.batch.  err_flag receives 2 if a
// bounded wait runs out.
cudaError_t xs_gemm(const XsOperand &A, const XsOperand &B, int M, int N, int K, double *C,
                    IdxMap cm, IdxMap cn, long long cstride, int ksplit, long long pstride,
                    int *err_flag, cudaStream_t s);

// C[m * ldc + n] = sum_p parts[p * pstride + m * N + n] (row-major parts).
cudaError_t xs_sum_parts(const double *parts, int nparts, long long pstride, int M, int N,
                         double *C, long long ldc, cudaStream_t s);

// Smallest number of K parts with each part <= kXsMaxK.
inline int xs_min_split(int K) { return (K + kXsMaxK - 1) / kXsMaxK; }

}  // namespace hotrg

namespace hotrg {

// Scratch of gemm_xs: slices and row scales of both operands (for all
// instances of a batch) and the FP64 partial products of a split K.
struct XsWork {
  void *sa, *sb;              // BF16 slices
  double *sca, *scb;          // row scales
  double *parts;              // K-part results (dense [part][instance][M][N])
  long long cap_a, cap_b;     // BF16 elements
  long long cap_sa, cap_sb;   // doubles
  long long cap_parts;        // doubles
};

// Elements gemm_xs needs for one GEMM (A slices, B slices, A scales, B
// scales, parts), for `batch` instances.
void xs_gemm_needs(int M, int N, int K, int S, int batch, long long need[5]);

// The mapped GEMM of `g` (C(m, n) = sum_k A(m, k) B(n, k) through index maps,
// batched) as an exact-slice tensor-core GEMM with S digits: the operands are
// gathered and sliced, K is split into exact parts, the result is written in
// FP64 through g's output maps.
cudaError_t gemm_xs(const MappedGemm &g, int S, const XsWork &w, int *err_flag, cudaStream_t s);

}  // namespace hotrg
