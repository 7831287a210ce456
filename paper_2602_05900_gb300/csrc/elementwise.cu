// Small FP64 kernels of the step: Gram symmetrisation and trace, the choice of
// the truncating isometry, max-norm rescale with the log-sum update, and the
// periodic trace used by the free energy.
#include <math.h>

#include "common.cuh"

namespace hotrg {
namespace {

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum over 1024 threads max; result valid in thread 0.
__device__ double block_sum(double v) {
  __shared__ double part[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? part[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

__global__ void k_symmetrize(double *G, int n) {
  long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (j > i) {
      double a = G[(long long)i * n + j], b = G[(long long)j * n + i];
      double v = 0.5 * (a + b);
      G[(long long)i * n + j] = v;
      G[(long long)j * n + i] = v;
    }
  }
}

__global__ void k_trace_diag(const double *G, int n, double *out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += G[(long long)i * n + i];
  v = block_sum(v);
  if (threadIdx.x == 0) *out = v;
}

__global__ void k_identity(double *U, int n) {
  long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    U[e] = (e % n == e / n) ? 1.0 : 0.0;
}

// Max |T| by a grid-stride reduction; non-negative doubles order like their
// bit patterns, so the grid-level combine is an integer atomicMax.
__global__ void k_maxabs(const double *T, long long count, unsigned long long *out) {
  double v = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double a = fabs(T[e]);
    v = (a != a) ? INFINITY : fmax(v, a);   // NaN poisons the norm
  }
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_scale(double *T, long long count, const unsigned long long *maxbits,
                        double *logsum, double inv_two_pow_n, double *ln_c_out, int *err) {
  const double c = __longlong_as_double((long long)*maxbits);
  const bool ok = (c > 0.0) && isfinite(c);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (ok) {
      const double lc = log(c);
      *logsum += lc * inv_two_pow_n;
      if (ln_c_out) *ln_c_out = lc;
    } else {
      atomicExch(err, 1);
      if (ln_c_out) *ln_c_out = NAN;
    }
  }
  if (!ok) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    T[e] = T[e] / c;
}

__global__ void k_periodic_trace(const double *T, int Dx, int Dy, double *out) {
  double v = 0.0;
  const long long sx = (long long)Dx * Dy * Dy + (long long)Dy * Dy;  // step along x == x'
  const int sy = Dy + 1;                                              // step along y == y'
  for (int e = threadIdx.x; e < Dx * Dy; e += blockDim.x) {
    int x = e / Dy, y = e % Dy;
    v += T[x * sx + (long long)y * sy];
  }
  v = block_sum(v);
  if (threadIdx.x == 0) *out = v;
}

// One block per kept column a.  Every block recomputes the side choice from the
// eigenvalues (a few dozen adds) so no separate launch or host round trip is
// needed; block 0 also writes the step record and the normalised spectrum.
__global__ void k_select(SelectArgs a) {
  __shared__ int s_side;
  __shared__ int s_arg;
  const int col = blockIdx.x;
  // i-th largest eigenvalue / its vector, whatever order the solver returned
  auto val = [&](const double *w, int i) { return a.desc ? w[i] : w[a.m - 1 - i]; };
  auto vecidx = [&](int i) { return a.desc ? i : a.m - 1 - i; };
  if (threadIdx.x == 0) {
    double sumL = 0.0, sumR = 0.0;
    for (int i = 0; i < a.Dn; ++i) {
      sumL += val(a.wL, i);
      sumR += val(a.wR, i);
    }
    const double epsL = *a.trL - sumL, epsR = *a.trR - sumR;
    s_side = (epsL <= epsR) ? 0 : 1;
    if (col == 0) {
      const double *w = s_side == 0 ? a.wL : a.wR;
      const double l1 = val(w, 0);
      a.record[0] = (double)s_side;
      a.record[1] = epsL;
      a.record[2] = epsR;
      a.record[3] = (a.m > a.Dn) ? (val(w, a.Dn - 1) - val(w, a.Dn)) / l1 : INFINITY;
      a.record[4] = *a.trL;
      for (int i = 0; i < a.m; ++i) a.spectrum[i] = val(w, i) / l1;
    }
  }
  __syncthreads();
  const double *v = (s_side == 0 ? a.vL : a.vR) + (long long)vecidx(col) * a.n;
  // sign convention: the component of largest magnitude (first on ties) is positive
  double best = -1.0;
  int arg = 0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    double x = fabs(v[i]);
    if (x > best) { best = x; arg = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
  }
  __shared__ double wbest[32];
  __shared__ int warg[32];
  if ((threadIdx.x & 31) == 0) {
    wbest[threadIdx.x >> 5] = best;
    warg[threadIdx.x >> 5] = arg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int g = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (wbest[w] > b || (wbest[w] == b && warg[w] < g)) { b = wbest[w]; g = warg[w]; }
    }
    s_arg = g;
  }
  __syncthreads();
  const double sg = (v[s_arg] < 0.0) ? -1.0 : 1.0;
  double *u = a.U + (long long)col * a.n;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) u[i] = sg * v[i];
}

__global__ void k_spectrum_no_cut(const double *w, int n, int desc, const double *trL,
                                  double *record, double *spectrum) {
  if (threadIdx.x == 0) {
    const double l1 = desc ? w[0] : w[n - 1];
    record[0] = -1.0;
    record[1] = 0.0;
    record[2] = 0.0;
    record[3] = INFINITY;
    record[4] = *trL;
    for (int i = 0; i < n; ++i) spectrum[i] = (desc ? w[i] : w[n - 1 - i]) / l1;
  }
}

int grid_for(long long count, int threads) {
  long long b = (count + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t symmetrize_trace(double *G, int n, double *trace_out, cudaStream_t s) {
  const long long total = (long long)n * n;
  k_symmetrize<<<grid_for(total, 256), 256, 0, s>>>(G, n);
  k_trace_diag<<<1, 1024, 0, s>>>(G, n, trace_out);
  return cudaGetLastError();
}

cudaError_t identity_isometry(double *U, int n, cudaStream_t s) {
  k_identity<<<grid_for((long long)n * n, 256), 256, 0, s>>>(U, n);
  return cudaGetLastError();
}

cudaError_t maxabs_scale_log(double *T, long long count, double *scratch_max, double *logsum,
                             double inv_two_pow_n, double *ln_c_out, int *err_flag,
                             cudaStream_t s) {
  unsigned long long *bits = reinterpret_cast<unsigned long long *>(scratch_max);
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_maxabs<<<grid_for(count, 256), 256, 0, s>>>(T, count, bits);
  k_scale<<<grid_for(count, 256), 256, 0, s>>>(T, count, bits, logsum, inv_two_pow_n, ln_c_out,
                                                err_flag);
  return cudaGetLastError();
}

cudaError_t scale_initial(double *T, long long count, double *scratch_max, double *logsum,
                          int *err_flag, cudaStream_t s) {
  return maxabs_scale_log(T, count, scratch_max, logsum, 1.0, nullptr, err_flag, s);
}

cudaError_t periodic_trace(const double *T, int Dx, int Dy, double *out, cudaStream_t s) {
  k_periodic_trace<<<1, 1024, 0, s>>>(T, Dx, Dy, out);
  return cudaGetLastError();
}

cudaError_t select_isometry(const SelectArgs &a, cudaStream_t s) {
  k_select<<<a.Dn, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t spectrum_no_cut(const double *w, int n, int desc, const double *trL, double *record,
                            double *spectrum, cudaStream_t s) {
  k_spectrum_no_cut<<<1, 32, 0, s>>>(w, n, desc, trL, record, spectrum);
  return cudaGetLastError();
}

}  // namespace hotrg
