// Small FP64 kernels of the step, batched over instances (grid.y or grid.x):
// Gram symmetrisation and trace, the choice of the truncating isometry,
// max-norm rescale with the log-sum update, and the periodic trace used by the
// free energy.
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

// Block-wide sum over up to 1024 threads; result valid in thread 0.
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

// grid (x: chunks of the n x n matrix, y: instance)

// G = (G + G^T) / 2 by pairs of 32 x 32 tiles (I <= J, one block each,
// blockIdx.y = problem): both tiles are read and written row by row through
// shared memory, so every global access is coalesced.  Each off-diagonal pair
// (i, j) gets 0.5 (G_ij + G_ji) in both places; diagonal entries are unchanged.
__global__ void __launch_bounds__(256) k_symmetrize_tiled(double *G, int n, long long sG) {
  __shared__ double A[32][33], B[32][33];
  G += blockIdx.y * sG;
  const int T = (n + 31) / 32;
  int p = blockIdx.x, I = 0;
  while (p >= T - I) {
    p -= T - I;
    ++I;
  }
  const int J = I + p;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int i = I * 32 + r, j = J * 32 + tx;
    A[r][tx] = (i < n && j < n) ? G[(long long)i * n + j] : 0.0;
    const int i2 = J * 32 + r, j2 = I * 32 + tx;
    B[r][tx] = (i2 < n && j2 < n) ? G[(long long)i2 * n + j2] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = I * 32 + r, j = J * 32 + tx;
    const double v = 0.5 * (A[r][tx] + B[tx][r]);
    if (i < n && j < n && i != j) G[(long long)i * n + j] = v;
    A[r][tx] = v;
  }
  if (I == J) return;
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = J * 32 + r, j = I * 32 + tx;
    if (i < n && j < n) G[(long long)i * n + j] = A[tx][r];
  }
}

// one block per problem z; the trace goes to out[z sOut], or with per_side > 0
// (problems side * per_side + i) to out[i sOut + side]
__global__ void k_trace_diag(const double *G, int n, long long sG, double *out, long long sOut,
                             int per_side) {
  G += blockIdx.x * sG;
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += G[(long long)i * n + i];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    const long long o = per_side > 0 ? (long long)(blockIdx.x % per_side) * sOut + blockIdx.x / per_side
                                     : (long long)blockIdx.x * sOut;
    out[o] = v;
  }
}

__global__ void k_identity(double *U, int n, long long sU) {
  U += blockIdx.y * sU;
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    U[e] = (e % n == e / n) ? 1.0 : 0.0;
}

// Max |T| per instance by a grid-stride reduction; non-negative doubles order
// like their bit patterns, so the combine is an integer atomicMax.
__global__ void k_maxabs(const double *T, long long count, long long sT, unsigned long long *out,
                         long long sOut) {
  T += blockIdx.y * sT;
  double v = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(T[e]);
    v = (a != a) ? INFINITY : fmax(v, a);   // NaN poisons the norm
  }
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0)
    atomicMax(out + blockIdx.y * sOut, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_scale(double *T, long long count, long long sT, const unsigned long long *maxbits,
                        long long sMax, double *logsum, long long sLog, double inv_two_pow_n,
                        double *ln_c_out, long long sLnc, int *err) {
  const long long inst = blockIdx.y;
  T += inst * sT;
  const double c = __longlong_as_double((long long)maxbits[inst * sMax]);
  const bool ok = (c > 0.0) && isfinite(c);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (ok) {
      const double lc = log(c);
      logsum[inst * sLog] += lc * inv_two_pow_n;
      if (ln_c_out) ln_c_out[inst * sLnc] = lc;
    } else {
      atomicMax(err, 1);
      if (ln_c_out) ln_c_out[inst * sLnc] = NAN;
    }
  }
  if (!ok) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    T[e] = T[e] / c;
}

// one block per instance
__global__ void k_periodic_trace(const double *T, int Dx, int Dy, long long sT, double *out,
                                 long long sOut) {
  T += blockIdx.x * sT;
  double v = 0.0;
  const long long sx = (long long)Dx * Dy * Dy + (long long)Dy * Dy;  // step along x == x'
  const int sy = Dy + 1;                                              // step along y == y'
  for (int e = threadIdx.x; e < Dx * Dy; e += blockDim.x) {
    const int x = e / Dy, y = e % Dy;
    v += T[x * sx + (long long)y * sy];
  }
  v = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x * sOut] = v;
}

// Tx[x][x'] = sum_y T[x][x'][y][y]: one thread per output element of every
// instance (grid.y); the Dy summands of an element lie Dy + 1 apart.
__global__ void k_trace_y(const double *T, double *Tx, int Dx, int Dy, long long sT) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Dx * Dx) return;
  const double *t = T + blockIdx.y * sT + (long long)e * Dy * Dy;
  double v = 0.0;
  for (int y = 0; y < Dy; ++y) v += t[y * (Dy + 1)];
  Tx[blockIdx.y * sT + e] = v;
}

// grid (kept column a, instance).  Every block recomputes the side choice from
// the eigenvalues (a few dozen adds), so no separate launch or host round trip
// is needed; block (0, i) also writes instance i's record and spectrum.
__global__ void k_select(SelectArgs a) {
  __shared__ int s_side;
  __shared__ int s_arg;
  __shared__ double wbest[32];
  __shared__ int warg[32];
  const int col = blockIdx.x, inst = blockIdx.y;
  const double *wL = a.w.at(2 * inst), *wR = a.w.at(2 * inst + 1);
  const double *tr = a.tr + inst * a.sTr;
  // i-th largest eigenvalue / its vector, whatever order the solver returned
  auto val = [&](const double *w, int i) { return a.desc ? w[i] : w[a.m - 1 - i]; };
  auto vecidx = [&](int i) { return a.desc ? i : a.m - 1 - i; };
  if (threadIdx.x == 0) {
    double sumL = 0.0, sumR = 0.0;
    for (int i = 0; i < a.Dn; ++i) {
      sumL += val(wL, i);
      sumR += val(wR, i);
    }
    const double epsL = tr[0] - sumL, epsR = tr[1] - sumR;
    s_side = (epsL <= epsR) ? 0 : 1;
    if (col == 0) {
      const double *w = s_side == 0 ? wL : wR;
      const double l1 = val(w, 0);
      double *rec = a.record + inst * a.sRec;
      double *spec = a.spectrum + inst * a.sSpec;
      rec[0] = (double)s_side;
      rec[1] = epsL;
      rec[2] = epsR;
      rec[3] = (a.m > a.Dn) ? (val(w, a.Dn - 1) - val(w, a.Dn)) / l1 : INFINITY;
      rec[4] = tr[0];
      for (int i = 0; i < a.m; ++i) spec[i] = val(w, i) / l1;
    }
  }
  __syncthreads();
  const double *v = a.v.at(2 * inst + s_side) + (long long)vecidx(col) * a.n;
  // sign convention: the component of largest magnitude (first on ties) is positive
  double best = -1.0;
  int arg = 0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    const double x = fabs(v[i]);
    if (x > best) { best = x; arg = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
  }
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
  double *u = a.U + inst * a.sU + (long long)col * a.n;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) u[i] = sg * v[i];
}

// one block per instance: eigen-problem `inst` of w holds the left environment
__global__ void k_spectrum_no_cut(PSet w, int n, int desc, const double *tr, long long sTr,
                                  double *record, long long sRec, double *spectrum,
                                  long long sSpec) {
  const int inst = blockIdx.x;
  if (threadIdx.x == 0) {
    const double *wv = w.at(inst);
    double *rec = record + inst * sRec;
    double *spec = spectrum + inst * sSpec;
    const double l1 = desc ? wv[0] : wv[n - 1];
    rec[0] = -1.0;
    rec[1] = 0.0;
    rec[2] = 0.0;
    rec[3] = INFINITY;
    rec[4] = tr[inst * sTr];
    for (int i = 0; i < n; ++i) spec[i] = (desc ? wv[i] : wv[n - 1 - i]) / l1;
  }
}

int grid_for(long long count, int threads, int batch) {
  long long b = (count + threads - 1) / threads;
  const long long cap = (152LL * 16 + batch - 1) / batch;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t symmetrize_trace(double *G, int n, long long sG, double *trace_out, long long sTr,
                             int batch, cudaStream_t s, int per_side) {
  const int T = (n + 31) / 32;
  k_symmetrize_tiled<<<dim3(T * (T + 1) / 2, batch), 256, 0, s>>>(G, n, sG);
  k_trace_diag<<<batch, 1024, 0, s>>>(G, n, sG, trace_out, sTr, per_side);
  return cudaGetLastError();
}

cudaError_t identity_isometry(double *U, int n, long long sU, int batch, cudaStream_t s) {
  k_identity<<<dim3(grid_for((long long)n * n, 256, batch), batch), 256, 0, s>>>(U, n, sU);
  return cudaGetLastError();
}

cudaError_t maxabs_scale_log(double *T, long long count, long long sT, double *scratch,
                             long long sScratch, double *logsum, long long sLog,
                             double inv_two_pow_n, double *ln_c_out, long long sLnc, int *err_flag,
                             int batch, cudaStream_t s) {
  unsigned long long *bits = reinterpret_cast<unsigned long long *>(scratch);
  cudaError_t e = cudaMemset2DAsync(bits, sScratch * sizeof(double), 0, sizeof(unsigned long long),
                                    batch, s);
  if (e != cudaSuccess) return e;
  const dim3 g(grid_for(count, 256, batch), batch);
  k_maxabs<<<g, 256, 0, s>>>(T, count, sT, bits, sScratch);
  k_scale<<<g, 256, 0, s>>>(T, count, sT, bits, sScratch, logsum, sLog, inv_two_pow_n, ln_c_out,
                            sLnc, err_flag);
  return cudaGetLastError();
}

cudaError_t periodic_trace(const double *T, int Dx, int Dy, long long sT, double *out,
                           long long sOut, int batch, cudaStream_t s) {
  k_periodic_trace<<<batch, 1024, 0, s>>>(T, Dx, Dy, sT, out, sOut);
  return cudaGetLastError();
}

cudaError_t trace_y(const double *T, double *Tx, int Dx, int Dy, long long sT, int batch,
                    cudaStream_t s) {
  const int n = Dx * Dx;
  k_trace_y<<<dim3((n + 255) / 256, batch), 256, 0, s>>>(T, Tx, Dx, Dy, sT);
  return cudaGetLastError();
}

cudaError_t select_isometry(const SelectArgs &a, cudaStream_t s) {
  k_select<<<dim3(a.Dn, a.batch), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t spectrum_no_cut(PSet w, int n, int desc, const double *tr, long long sTr,
                            double *record, long long sRec, double *spectrum, long long sSpec,
                            int batch, cudaStream_t s) {
  k_spectrum_no_cut<<<batch, 32, 0, s>>>(w, n, desc, tr, sTr, record, sRec, spectrum, sSpec);
  return cudaGetLastError();
}

}  // namespace hotrg
