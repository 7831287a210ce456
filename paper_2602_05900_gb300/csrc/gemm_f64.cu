// FP64 SIMT GEMM over mapped operands: the plain FP64 path of every contraction
// of the HOTRG step (environment partials, Gram combine, projection chain).
//
// C(m, n) = sum_k A(m, k) B(n, k), where A(m, k) = A[am(m) + ak(k)] and so on
// for B and C (see IdxMap).  64 x 64 output tile per 256-thread block, 4 x 4
// outputs per thread, K staged through shared memory in chunks of 16 with a
// register prefetch of the next chunk; grid.z runs over the instances of a batch.
// GEMMs with at most 64 outputs and K >= 256 take a block-per-output dot kernel,
// GEMMs with M, N <= 128 a 16 x 16-tile kernel.
#include "common.cuh"

namespace hotrg {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool K_FAST_A, bool K_FAST_B>
__global__ void __launch_bounds__(NT) k_gemm_f64(MappedGemm g) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  __shared__ long long rowA[BM], rowB[BN];
  __shared__ long long kA[2][BK], kB[2][BK];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * BM;
  const long long n0 = (long long)blockIdx.y * BN;
  // instance of the batch
  const long long zA = blockIdx.z * g.bA, zB = blockIdx.z * g.bB, zC = blockIdx.z * g.bC;
  g.A += zA;
  g.B += zB;
  g.C += zC;

  if (tid < BM) {
    long long m = m0 + tid;
    rowA[tid] = (m < g.M) ? map_off(g.am, m) : -1;
  } else if (tid < BM + BN) {
    long long n = n0 + tid - BM;
    rowB[tid - BM] = (n < g.N) ? map_off(g.bn, n) : -1;
  }
  auto k_offsets = [&](int buf, int kc) {
    if (tid < BK) {
      int k = kc + tid;
      kA[buf][tid] = (k < g.K) ? map_off(g.ak, k) : -1;
    } else if (tid < 2 * BK) {
      int k = kc + tid - BK;
      kB[buf][tid - BK] = (k < g.K) ? map_off(g.bk, k) : -1;
    }
  };
  k_offsets(0, 0);
  __syncthreads();

  // Each thread loads 4 elements of the A tile and 4 of the B tile per chunk.
  // The thread-to-element assignment puts consecutive threads on consecutive
  // k when the k map is unit-stride, otherwise on consecutive rows.
  auto load_regs = [&](int buf, double ra[4], double rb[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + i * NT;
      int r, k;
      if (K_FAST_A) { r = e / BK; k = e % BK; } else { r = e % BM; k = e / BM; }
      long long ro = rowA[r], ko = kA[buf][k];
      ra[i] = (ro >= 0 && ko >= 0 && checked_ok(zA + ro + ko, g.capA, g.err)) ? g.A[ro + ko] : 0.0;
      if (K_FAST_B) { r = e / BK; k = e % BK; } else { r = e % BN; k = e / BN; }
      ro = rowB[r]; ko = kB[buf][k];
      rb[i] = (ro >= 0 && ko >= 0 && checked_ok(zB + ro + ko, g.capB, g.err)) ? g.B[ro + ko] : 0.0;
    }
  };
  auto store_regs = [&](int buf, const double ra[4], const double rb[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + i * NT;
      int r, k;
      if (K_FAST_A) { r = e / BK; k = e % BK; } else { r = e % BM; k = e / BM; }
      As[buf][k][r] = ra[i];
      if (K_FAST_B) { r = e / BK; k = e % BK; } else { r = e % BN; k = e / BN; }
      Bs[buf][k][r] = rb[i];
    }
  };

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  load_regs(0, ra, rb);
  store_regs(0, ra, rb);
  const int nchunks = (g.K + BK - 1) / BK;
  if (nchunks > 1) k_offsets(1, BK);
  __syncthreads();

  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    const bool has_next = (c + 1 < nchunks);
    if (has_next) load_regs(buf ^ 1, ra, rb);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (has_next) {
      store_regs(buf ^ 1, ra, rb);
      __syncthreads();
      if (c + 2 < nchunks) k_offsets(buf, (c + 2) * BK);
      __syncthreads();
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
    long long co = map_off(g.cm, m);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long n = n0 + tx + 16 * j;
      if (n < g.N) {
        const long long off = co + map_off(g.cn, n);
        if (checked_ok(zC + off, g.capC, g.err)) g.C[off] = acc[i][j];
      }
    }
  }
}

// Few outputs over a long K (e.g. the 1 x 1 environment of a step whose fused
// legs are trivial, K = E^2): one block per output element, K strided over the
// threads and combined by a fixed-order tree, so the result is deterministic.
__global__ void __launch_bounds__(NT) k_dot_f64(MappedGemm g) {
  __shared__ double red[NT];
  const long long e = blockIdx.x;
  const long long m = e / g.N, n = e % g.N;
  const long long zA = blockIdx.z * g.bA, zB = blockIdx.z * g.bB, zC = blockIdx.z * g.bC;
  g.A += zA;
  g.B += zB;
  g.C += zC;
  const long long ao = map_off(g.am, m), bo = map_off(g.bn, n);
  double v = 0.0;
  for (int k = threadIdx.x; k < g.K; k += NT) {
    const long long oa = ao + map_off(g.ak, k), ob = bo + map_off(g.bk, k);
    if (checked_ok(zA + oa, g.capA, g.err) && checked_ok(zB + ob, g.capB, g.err)) v = fma(g.A[oa], g.B[ob], v);
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const long long oc = map_off(g.cm, m) + map_off(g.cn, n);
  if (threadIdx.x == 0 && checked_ok(zC + oc, g.capC, g.err)) g.C[oc] = red[0];
}

constexpr long long kDotMaxOutputs = 64, kDotMinK = 256;

// Small GEMMs (M, N <= 128): 16 x 16 output tiles, one output per thread, K in
// chunks of 16 through shared memory.  A 64 x 64 tiling would put such a product
// on at most four SMs, and GB300's FP64 rate per SM (about 2 FMA per clock) makes
// the number of SMs, not the tile efficiency, the limit.
constexpr int ST = 16;
constexpr int kSmallMax = 128;

__global__ void __launch_bounds__(256) k_gemm_f64_small(MappedGemm g) {
  __shared__ double As[ST][ST + 1], Bs[ST][ST + 1];   // [k][row]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long m0 = (long long)blockIdx.x * ST, n0 = (long long)blockIdx.y * ST;
  const long long zA = blockIdx.z * g.bA, zB = blockIdx.z * g.bB, zC = blockIdx.z * g.bC;
  g.A += zA;
  g.B += zB;
  g.C += zC;
  // loads: thread (ty, tx) brings A(m0 + ty, k0 + tx) and B(n0 + ty, k0 + tx)
  const long long ar = (m0 + ty < g.M) ? map_off(g.am, m0 + ty) : -1;
  const long long br = (n0 + ty < g.N) ? map_off(g.bn, n0 + ty) : -1;
  double acc = 0.0;
  for (int k0 = 0; k0 < g.K; k0 += ST) {
    const int k = k0 + tx;
    const bool kv = k < g.K;
    const long long oa = ar + (kv ? map_off(g.ak, k) : 0), ob = br + (kv ? map_off(g.bk, k) : 0);
    As[tx][ty] = (ar >= 0 && kv && checked_ok(zA + oa, g.capA, g.err)) ? g.A[oa] : 0.0;
    Bs[tx][ty] = (br >= 0 && kv && checked_ok(zB + ob, g.capB, g.err)) ? g.B[ob] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ST; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
    __syncthreads();
  }
  const long long m = m0 + ty, n = n0 + tx;
  if (m < g.M && n < g.N) {
    const long long oc = map_off(g.cm, m) + map_off(g.cn, n);
    if (checked_ok(zC + oc, g.capC, g.err)) g.C[oc] = acc;
  }
}

}  // namespace

cudaError_t gemm_f64(const MappedGemm &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if ((long long)g.M * g.N <= kDotMaxOutputs && g.K >= kDotMinK) {
    if (g.batch > 65535) return cudaErrorInvalidConfiguration;
    k_dot_f64<<<dim3((unsigned)(g.M * g.N), 1, (unsigned)(g.batch < 1 ? 1 : g.batch)), NT, 0, s>>>(g);
    return cudaGetLastError();
  }
  if (g.M <= kSmallMax && g.N <= kSmallMax) {
    if (g.batch > 65535) return cudaErrorInvalidConfiguration;
    const dim3 gs((unsigned)((g.M + ST - 1) / ST), (unsigned)((g.N + ST - 1) / ST),
                  (unsigned)(g.batch < 1 ? 1 : g.batch));
    k_gemm_f64_small<<<gs, 256, 0, s>>>(g);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN),
            (unsigned)(g.batch < 1 ? 1 : g.batch));
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  const bool ka = (g.ak.s0 == 1), kb = (g.bk.s0 == 1);
  if (ka && kb) k_gemm_f64<true, true><<<grid, NT, 0, s>>>(g);
  else if (ka) k_gemm_f64<true, false><<<grid, NT, 0, s>>>(g);
  else if (kb) k_gemm_f64<false, true><<<grid, NT, 0, s>>>(g);
  else k_gemm_f64<false, false><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace hotrg
