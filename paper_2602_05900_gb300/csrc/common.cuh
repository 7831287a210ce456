// Shared declarations of libhotrg's CUDA sources.
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

// Stage boundaries and launch counts reported to the context's profiler.
struct StageHook {
  virtual void begin(int stage) = 0;
  virtual void end(int stage) = 0;
  virtual void launched(int stage, int n) = 0;
  virtual ~StageHook() {}
};

// C(m, n) = sum_k A(m, k) * B(n, k) over mapped operands.
struct MappedGemm {
  int M, N, K;
  const double *A;
  IdxMap am, ak;
  const double *B;
  IdxMap bn, bk;
  double *C;
  IdxMap cm, cn;
};

// gemm_f64.cu
cudaError_t gemm_f64(const MappedGemm &g, cudaStream_t s);

// elementwise.cu
cudaError_t symmetrize_trace(double *G, int n, double *trace_out, cudaStream_t s);
cudaError_t identity_isometry(double *U, int n, cudaStream_t s);
cudaError_t maxabs_scale_log(double *T, long long count, double *scratch_max, double *logsum,
                             double inv_two_pow_n, double *ln_c_out, int *err_flag, cudaStream_t s);
cudaError_t periodic_trace(const double *T, int Dx, int Dy, double *out, cudaStream_t s);
cudaError_t scale_initial(double *T, long long count, double *scratch_max, double *logsum,
                          int *err_flag, cudaStream_t s);

// Device-side choice of the environment side and assembly of U (descending
// eigenvectors, sign-fixed) plus the step record.  eig_L / eig_R hold `m`
// ascending eigenpairs (values wL/wR, column-major vectors with leading dim n)
// of the top of each spectrum.
struct SelectArgs {
  int n, Dn, m;               // matrix size, kept count, eigenpairs computed per side
  int desc;                   // 1: values/vectors in descending order, 0: ascending
  const double *wL, *wR;      // eigenvalues (m)
  const double *vL, *vR;      // eigenvectors, column-major n x m
  const double *trL, *trR;    // traces of G_L, G_R
  double *U;                  // out: n x Dn column-major
  double *record;             // out: [side, eps_L, eps_R, cut_gap, trace_G]
  double *spectrum;           // out: normalised spectrum, Dn (+1 if cut) values
};
cudaError_t select_isometry(const SelectArgs &a, cudaStream_t s);
cudaError_t spectrum_no_cut(const double *w, int n, int desc, const double *trL, double *record,
                            double *spectrum, cudaStream_t s);

}  // namespace hotrg
