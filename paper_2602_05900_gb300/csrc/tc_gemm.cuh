// tcgen05 / TMA GEMM for sm_103a: C = sum over products of A_p . B_q^T with
// K-major operands in shared memory (128-byte swizzle), FP32 accumulation in
// tensor memory, and an epilogue that writes through an (IdxMap, IdxMap) pair
// into FP32, FP64 or split-BF16 planes.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace hotrg {

// Operand arithmetic of a tensor-core GEMM.
enum class TcMode : int {
  TF32 = 0,     // one FP32 plane (pre-rounded to TF32), kind::tf32
  BF16X3 = 1,   // two BF16 planes (hi, lo), products hh + hl + lh, kind::f16
  BF16X6 = 2,   // three BF16 planes, products with plane-index sum <= 2 (0-based)
};

inline int tc_planes(TcMode m) { return m == TcMode::TF32 ? 1 : (m == TcMode::BF16X3 ? 2 : 3); }
inline int tc_elem_bytes(TcMode m) { return m == TcMode::TF32 ? 4 : 2; }

// Output format of the epilogue.
enum class OutKind : int { F32 = 0, F64 = 1, BF16P = 2 };

// A dense operand in global memory: `planes` planes of `rows` x `pitch`
// elements (K contiguous), plane stride rows * pitch, for `batch` instances
// `bstride` elements apart.  Only the first K columns are read (the rest of
// each row is padding).
struct TcOperand {
  const void *base;
  int rows, K, pitch;
  int batch;
  long long bstride;
};

struct TcEpilogue {
  OutKind kind;
  void *C;
  long long plane_stride;  // elements between output planes (BF16P)
  int planes;              // output planes (BF16P): 1, 2 or 3
  bool round_tf32;         // F32 output feeds a TF32 operand: round to nearest TF32
  IdxMap cm, cn;
  long long bstride;       // elements between the outputs of consecutive instances
  bool transpose;          // set by tc_gemm: stage through shared memory so that a warp
                           // stores 32 consecutive columns of one row (unit-stride cn)
  long long cap;           // elements of C from its base, all instances and planes (0 =
                           // unknown): bounds of the checked build
  bool vec4;               // set by tc_gemm: transposed F32 / F64 stores of 4 consecutive
                           // columns at once (unit-stride, 4-aligned column map)
};

// Launches C(M x N) = A(M x K) . B(N x K)^T for every instance of the batch
// (A.batch == B.batch; the tiles of all instances form one persistent
// schedule); returns a CUDA error code (cudaErrorInvalidValue for unsupported
// shapes).
cudaError_t tc_gemm(TcMode mode, const TcOperand &A, const TcOperand &B, int M, int N, int K,
                    const TcEpilogue &epi, int *err_flag, cudaStream_t s);

// Tile-width autotuning of tc_gemm (process-wide, on by default): the first
// GEMM of each shape times every tile width and keeps the fastest.
void tc_set_autotune(bool on);

// Number of padded columns an operand row needs so that its byte pitch is a
// multiple of 16 (the TMA stride rule).
inline int tc_pitch(int K, TcMode m) {
  const int q = 16 / tc_elem_bytes(m);
  return ((K + q - 1) / q) * q;
}

}  // namespace hotrg
