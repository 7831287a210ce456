// Shared declarations of libhotrg's CUDA sources.
//
// Every kernel works on a uniform batch of instances (same shapes, buffers at a
// fixed per-instance stride); a single HOTRG instance is a batch of one.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hotrg {

// Maps a flat index i in [0, extent) to an element offset through a mixed-radix
// split i = (i2 * n1 + i1) * n0 + i0 (i0 < n0, i1 < n1):
//   offset(i) = i0 * s0 + i1 * s1 + i2 * s2.
// A contraction whose operands are permuted views of a tensor is a GEMM whose
// row, column and reduction indices each go through one such map; this is how
// every permute/reshape of the step is folded into addressing instead of being
// materialised (the layout idea of Sec. II.B, Eq. 3).
struct IdxMap {
  int n0, n1;
  long long s0, s1, s2;
};

inline IdxMap map1(long long s) { return IdxMap{1 << 30, 1, s, 0, 0}; }
inline IdxMap map2(int n0, long long s0, long long s1) { return IdxMap{n0, 1 << 30, s0, s1, 0}; }
inline IdxMap map3(int n0, int n1, long long s0, long long s1, long long s2) {
  return IdxMap{n0, n1, s0, s1, s2};
}

__host__ __device__ inline long long map_off(const IdxMap &m, long long i) {
  long long i0 = i % m.n0;
  long long r = i / m.n0;
  long long i1 = r % m.n1;
  long long i2 = r / m.n1;
  return i0 * m.s0 + i1 * m.s1 + i2 * m.s2;
}

// A family of buffers indexed by problem z: even z -> b0, odd z -> b1, plus
// (z / 2) * stride.  The two environments of instance i are problems 2i (left)
// and 2i + 1 (right); pset_linear(base, s) is simply "problem z at base + z s".
struct PSet {
  double *b0, *b1;
  long long stride;
  __host__ __device__ double *at(int z) const {
    return ((z & 1) ? b1 : b0) + (long long)(z >> 1) * stride;
  }
};
inline PSet pset_pairs(double *left, double *right, long long inst_stride) {
  return PSet{left, right, inst_stride};
}
inline PSet pset_linear(double *base, long long stride) {
  return PSet{base, base + stride, 2 * stride};
}

// Stage boundaries and launch counts reported to the context's profiler.
struct StageHook {
  virtual void begin(int stage) = 0;
  virtual void end(int stage) = 0;
  virtual void launched(int stage, int n) = 0;
  virtual ~StageHook() {}
};

// Bounds-checked build (-DHOTRG_CHECKED=1, the stand-in for memory sanitizers):
// every mapped access of the GEMM, gather and epilogue kernels is compared
// with the capacity of its buffer; an access outside it is skipped and
// recorded in the context's device error flag as 3 (reported as
// HOTRG_EBOUNDS).  A capacity of 0 means "not known" (no check).  The normal
// build compiles the checks away.
#ifdef HOTRG_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool checked_ok(long long off, long long cap, int *err) {
  if constexpr (kChecked) {
    if (cap > 0 && (off < 0 || off >= cap)) {
      if (err) atomicMax(err, 3);
      return false;
    }
  }
  return true;
}

// C(m, n) = sum_k A(m, k) * B(n, k) over mapped operands, for `batch`
// instances whose operands lie bA, bB, bC elements apart.  capA, capB, capC:
// elements of each buffer from its base (all instances; 0 = unknown), used by
// the checked build, which records violations in *err.
struct MappedGemm {
  int M, N, K;
  const double *A;
  IdxMap am, ak;
  const double *B;
  IdxMap bn, bk;
  double *C;
  IdxMap cm, cn;
  int batch;
  long long bA, bB, bC;
  long long capA = 0, capB = 0, capC = 0;
  int *err = nullptr;
};

// gemm_f64.cu
cudaError_t gemm_f64(const MappedGemm &g, cudaStream_t s);

// elementwise.cu  (all batched over `batch` instances with the given strides)
// G = (G + G^T) / 2 and its trace for `batch` problems sG apart: trace of
// problem z at trace_out[z sTr], or with per_side > 0 (problems
// side * per_side + i, the two sides of per_side instances) at
// trace_out[i sTr + side].
cudaError_t symmetrize_trace(double *G, int n, long long sG, double *trace_out, long long sTr,
                             int batch, cudaStream_t s, int per_side = 0);
cudaError_t identity_isometry(double *U, int n, long long sU, int batch, cudaStream_t s);
// T /= max|T| per instance, logsum += ln(max) * inv_two_pow_n, ln_c_out (may be null)
// receives ln(max); scratch holds one word per instance (stride sScratch doubles).
cudaError_t maxabs_scale_log(double *T, long long count, long long sT, double *scratch,
                             long long sScratch, double *logsum, long long sLog,
                             double inv_two_pow_n, double *ln_c_out, long long sLnc, int *err_flag,
                             int batch, cudaStream_t s);
cudaError_t periodic_trace(const double *T, int Dx, int Dy, long long sT, double *out,
                           long long sOut, int batch, cudaStream_t s);
// Tx[x][x'] = sum_y T[x][x'][y][y] (Tx and T distinct buffers, same stride sT).
cudaError_t trace_y(const double *T, double *Tx, int Dx, int Dy, long long sT, int batch,
                    cudaStream_t s);

// Device-side choice of the environment side and assembly of U (sign-fixed
// leading eigenvectors) plus the step record, for every instance i: its left
// environment is eigen-problem 2i, its right one 2i + 1.
struct SelectArgs {
  int n, Dn, m;               // matrix size, kept count, eigenpairs available per side
  int desc;                   // 1: values/vectors in descending order, 0: ascending
  PSet w;                     // eigenvalues of problem z: w.at(z)[0..m)
  PSet v;                     // eigenvectors of problem z: column-major n x m at v.at(z)
  const double *tr;           // traces: tr + i * sTr + {0: G_L, 1: G_R}
  long long sTr;
  double *U;                  // out: U + i * sU, n x Dn column-major
  long long sU;
  double *record;             // out: record + i * sRec: [side, eps_L, eps_R, cut_gap, trace_G]
  long long sRec;
  double *spectrum;           // out: spectrum + i * sSpec
  long long sSpec;
  int batch;
};
cudaError_t select_isometry(const SelectArgs &a, cudaStream_t s);
// no cut: record + spectrum of the left environment only (eigen-problem i of w)
cudaError_t spectrum_no_cut(PSet w, int n, int desc, const double *tr, long long sTr,
                            double *record, long long sRec, double *spectrum, long long sSpec,
                            int batch, cudaStream_t s);

}  // namespace hotrg
