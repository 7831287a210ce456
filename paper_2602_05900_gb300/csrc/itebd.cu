// iTEBD ground state of the spin-1/2 XXZ chain (Sec. II.A, Eq. 1) on the GPU:
// a batch of chains, each a two-site-cell matrix-product state (P, Q, lam) in
// right-canonical form, advanced by imaginary-time two-site gates
// U = exp(-tau h).  One update of every chain of the batch:
//
//   phi   = P Q                        FP64 GEMM, rows (i, a), columns (b, m)
//   phit  = g phi, theta = lam phit    k_itebd_gate
//   rho   = theta^T theta              FP64 GEMM + symmetrise: the bond's right
//                                      reduced density matrix (2D x 2D)
//   Y, w  = eig(rho)                   cluster two-sided Jacobi (Sec. II.B, Eqs. 5-6),
//                                      warm-started from the same kind of bond's
//                                      last eigenbasis V: eig(V^T rho V), Y = V W
//   lam'  = sqrt(w[:D']) / norm        k_itebd_schmidt (+ the discarded weight)
//   P'    = phit Y[:, :D'] / |s|       FP64 GEMM + k_itebd_scale (keeps the state
//                                      normalised under the non-unitary gate)
//   Q'    = Y[:, :D']^T                k_itebd_take (Y is column-major: a copy)
//
// then (P, Q, lam) <- (Q', P', lam') for the other kind of bond.  The singular
// values of theta are the square roots of rho's eigenvalues (the paper's SVD of a
// Hermitian matrix), and P' = phit Y is Gamma' lam' without dividing by any
// Schmidt value.  Every chain of a batch has the same bond dimensions after
// every update (D' depends only on the dimensions), so one launch of each kernel
// serves the whole batch (grid.y / grid.z over chains).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "eig_si.cuh"
#include "hotrg.h"
#include "xxz.cuh"

namespace hotrg {
namespace {

constexpr int kPhys = 2;                       // physical dimension of a site
constexpr int kItebdMaxD = kSiMaxBlock / 2;    // 2 D_b <= 96: the direct Jacobi's size

// phit[i][A][B][m] = sum_ab g[AB][ab] phi[i][a][b][m], theta = lam[i] phit
__global__ void k_itebd_gate(const double *phi, double *phit, double *theta, const double *gates,
                             const double *lam, int Dl, int Dr, long long sM, long long sL) {
  const long long z = blockIdx.y;
  phi += z * sM;
  phit += z * sM;
  theta += z * sM;
  lam += z * sL;
  const double *g = gates + z * 16;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Dl * Dr; e += gridDim.x * blockDim.x) {
    const int i = e / Dr, m = e % Dr;
    double v[4];
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) v[ab] = phi[((long long)(i * 2 + (ab >> 1)) * 2 + (ab & 1)) * Dr + m];
#pragma unroll
    for (int AB = 0; AB < 4; ++AB) {
      double s = 0.0;
#pragma unroll
      for (int ab = 0; ab < 4; ++ab) s = fma(g[AB * 4 + ab], v[ab], s);
      const long long o = ((long long)(i * 2 + (AB >> 1)) * 2 + (AB & 1)) * Dr + m;
      phit[o] = s;
      theta[o] = lam[i] * s;
    }
  }
}

// one block per chain: lam'[k] = sqrt(w_k) / sqrt(sum_{k < Dn} w_k) with w = max(eig, 0);
// disc = sum_{k >= Dn} w_k / sum_k w_k over the m eigenvalues (descending);
// rnorm = 1 / sqrt(sum_{k < Dn} w_k), the factor that keeps the state normalised
__global__ void k_itebd_schmidt(PSet w, int m, int Dn, double *lam, long long sL, double *disc,
                                double *rnorm, int *err) {
  const int z = blockIdx.x;
  const double *wz = w.at(z);
  __shared__ double keep;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < m; ++k) {
      const double v = fmax(wz[k], 0.0);
      b += v;
      if (k < Dn) a += v;
    }
    keep = a;
    disc[z] = b > 0.0 ? (b - a) / b : NAN;
    rnorm[z] = 1.0 / sqrt(a);
    if (!(a > 0.0) || !isfinite(b)) atomicExch(err, 1);
  }
  __syncthreads();
  const double inv = 1.0 / sqrt(keep);
  for (int k = threadIdx.x; k < Dn; k += blockDim.x) lam[z * sL + k] = sqrt(fmax(wz[k], 0.0)) * inv;
}

// P' *= rnorm of its chain
__global__ void k_itebd_scale(double *P, long long count, long long sT, const double *rnorm) {
  const long long z = blockIdx.y;
  const double r = rnorm[z];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    P[z * sT + e] *= r;
}

// Q'[j][B][m] = Y[(B m), j] for j < Dn: the first Dn columns of the column-major Y
__global__ void k_itebd_take(PSet Y, long long count, double *Q, long long sT) {
  const long long z = blockIdx.y;
  const double *y = Y.at((int)z);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    Q[z * sT + e] = y[e];
}

// one block per chain: <theta|h|theta> / <theta|theta>, theta = lam[i] phi[i][a][b][m]
__global__ void k_itebd_energy(const double *phi, const double *lam, const double *hs, int Dl, int Dr,
                               long long sM, long long sL, double *out, int slot) {
  const long long z = blockIdx.x;
  phi += z * sM;
  lam += z * sL;
  const double *h = hs + z * 16;
  double num = 0.0, den = 0.0;
  for (int e = threadIdx.x; e < Dl * Dr; e += blockDim.x) {
    const int i = e / Dr, m = e % Dr;
    double v[4];
#pragma unroll
    for (int ab = 0; ab < 4; ++ab)
      v[ab] = lam[i] * phi[((long long)(i * 2 + (ab >> 1)) * 2 + (ab & 1)) * Dr + m];
#pragma unroll
    for (int AB = 0; AB < 4; ++AB) {
      double s = 0.0;
#pragma unroll
      for (int ab = 0; ab < 4; ++ab) s = fma(h[AB * 4 + ab], v[ab], s);
      num = fma(v[AB], s, num);
      den = fma(v[AB], v[AB], den);
    }
  }
  __shared__ double rn[256], rd[256];
  rn[threadIdx.x] = num;
  rd[threadIdx.x] = den;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      rn[threadIdx.x] += rn[threadIdx.x + w];
      rd[threadIdx.x] += rd[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[z * 2 + slot] = rn[0] / rd[0];
}

}  // namespace
}  // namespace hotrg

using namespace hotrg;

struct hotrg_itebd {
  cudaStream_t stream = nullptr;
  int G = 0, Db = 0;
  int outer = 1, mid = 1;         // P is (outer, 2, mid), Q is (mid, 2, outer)
  long long nsteps = 0;
  long long sT = 0, sL = 0, sM = 0;
  double *t[4] = {};              // site tensors: P, Q and two buffers for P', Q'
  int iP = 0, iQ = 1;
  double *l[3] = {};              // Schmidt values: lam, lam_other, lam'
  int iL = 0, iO = 1;
  double *phi = nullptr, *phit = nullptr, *theta = nullptr, *rho = nullptr;
  double *gates = nullptr, *hs = nullptr, *disc = nullptr, *energy = nullptr, *trace = nullptr;
  double *rnorm = nullptr;
  // warm start: the last full eigenbasis of each kind of bond (n x n column-major,
  // n = nb[parity], -1 = none) and a buffer for the next one
  double *Vb[2] = {nullptr, nullptr}, *Vn = nullptr;
  int nb[2] = {-1, -1};
  double *si_work = nullptr;
  int *err = nullptr;
  std::vector<void *> allocs;
  hotrg_status status = HOTRG_OK;
  std::string msg;
};

namespace {

hotrg_status ifail(hotrg_itebd *c, hotrg_status s, const std::string &m) {
  if (c->status == HOTRG_OK) {
    c->status = s;
    c->msg = m;
  }
  return c->status;
}

#define ICK(c, call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return ifail((c), HOTRG_ECUDA, std::string(#call ": ") +       \
                                                              cudaGetErrorString(e_));    \
  } while (0)

template <typename T>
hotrg_status ialloc(hotrg_itebd *c, T **p, long long count) {
  void *q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (size_t)std::max(1LL, count)) != cudaSuccess) {
    (void)cudaGetLastError();
    return ifail(c, HOTRG_ENOMEM, "device allocation failed");
  }
  c->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return HOTRG_OK;
}

int grid1(long long count) {
  long long b = (count + 255) / 256;
  return (int)std::min(std::max(b, 1LL), 1024LL);
}

// one gate update of every chain (see the file comment)
hotrg_status itebd_update(hotrg_itebd *c) {
  cudaStream_t st = c->stream;
  const int G = c->G, Dl = c->outer, Dm = c->mid, Dr = c->outer;
  const int n = kPhys * Dr, Dn = std::min(c->Db, std::min(kPhys * Dl, kPhys * Dr));
  double *P = c->t[c->iP], *Q = c->t[c->iQ];
  // the two tensor buffers not holding P or Q receive P' and Q'
  int iPn = -1, iQn = -1;
  for (int k = 0; k < 4; ++k) {
    if (k == c->iP || k == c->iQ) continue;
    if (iPn < 0) iPn = k;
    else iQn = k;
  }
  double *Pn = c->t[iPn], *Qn = c->t[iQn];
  const int iN = 3 - c->iL - c->iO;
  // phi = P Q
  MappedGemm g1{kPhys * Dl, kPhys * Dr, Dm, P, map1(Dm), map1(1), Q, map1(1), map1(kPhys * Dr),
                c->phi, map1(kPhys * Dr), map1(1), G, c->sT, c->sT, c->sM};
  ICK(c, gemm_f64(g1, st));
  k_itebd_gate<<<dim3(grid1((long long)Dl * Dr), G), 256, 0, st>>>(c->phi, c->phit, c->theta, c->gates,
                                                                   c->l[c->iL], Dl, Dr, c->sM, c->sL);
  ICK(c, cudaGetLastError());
  // rho = theta^T theta, symmetrised
  MappedGemm g2{n, n, kPhys * Dl, c->theta, map1(1), map1(n), c->theta, map1(1), map1(n),
                c->rho, map1(n), map1(1), G, c->sM, c->sM, c->sM};
  ICK(c, gemm_f64(g2, st));
  ICK(c, symmetrize_trace(c->rho, n, c->sM, c->trace, 1, G, st));
  // Warm start: two updates ago the same kind of bond had eigenbasis V; near the
  // fixed point rho is nearly diagonal in it, so the Jacobi runs on
  // rho~ = V^T rho V (a few sweeps instead of ~11 from scratch) and the basis
  // becomes V W.  phi and theta are free here and hold V^T-products.
  const int par = (int)(c->nsteps & 1);
  const bool warm = c->nb[par] == n;
  double *Vold = c->Vb[par];
  if (warm) {
    // phi = rho V (row-major n x n), theta = V^T phi
    MappedGemm w1{n, n, n, c->rho, map1(n), map1(1), Vold, map1(n), map1(1), c->phi, map1(n), map1(1),
                  G, c->sM, c->sM, c->sM};
    ICK(c, gemm_f64(w1, st));
    MappedGemm w2{n, n, n, Vold, map1(n), map1(1), c->phi, map1(1), map1(n), c->theta, map1(n), map1(1),
                  G, c->sM, c->sM, c->sM};
    ICK(c, gemm_f64(w2, st));
    ICK(c, symmetrize_trace(c->theta, n, c->sM, c->trace, 1, G, st));
  }
  // all n eigenpairs (the full basis is kept for the next warm start)
  SiBatch sb{};
  sb.P = G;
  sb.n = n;
  sb.k = n;
  sb.m = jacobi_block(n);
  sb.G = pset_linear(warm ? c->theta : c->rho, c->sM);
  long long nl = 0;
  ICK(c, jacobi_full(sb, c->si_work, st, &nl));
  const SiOut o = si_outputs(c->si_work, G, n, sb.m);
  k_itebd_schmidt<<<G, 64, 0, st>>>(o.theta, sb.m, Dn, c->l[iN], c->sL, c->disc, c->rnorm, c->err);
  ICK(c, cudaGetLastError());
  // the new basis V' = V W (or W cold), column-major n x n, into Vn
  const long long ys = o.X.b1 - o.X.b0;
  if (warm) {
    MappedGemm w3{n, n, n, Vold, map1(1), map1(n), o.X.b0, map1(n), map1(1), c->Vn, map1(1), map1(n),
                  G, c->sM, ys, c->sM};
    ICK(c, gemm_f64(w3, st));
  } else {
    k_itebd_take<<<dim3(grid1((long long)n * n), G), 256, 0, st>>>(o.X, (long long)n * n, c->Vn, c->sM);
    ICK(c, cudaGetLastError());
  }
  std::swap(c->Vb[par], c->Vn);
  c->nb[par] = n;
  const PSet Y = pset_linear(c->Vb[par], c->sM);
  // P' = phit Y / |s|, Q' = Y^T (Y = the leading Dn columns of the basis)
  MappedGemm g3{kPhys * Dl, Dn, n, c->phit, map1(n), map1(1), Y.b0, map1(n), map1(1), Pn, map1(Dn),
                map1(1), G, c->sM, c->sM, c->sT};
  ICK(c, gemm_f64(g3, st));
  k_itebd_scale<<<dim3(grid1((long long)kPhys * Dl * Dn), G), 256, 0, st>>>(Pn, (long long)kPhys * Dl * Dn,
                                                                           c->sT, c->rnorm);
  ICK(c, cudaGetLastError());
  k_itebd_take<<<dim3(grid1((long long)Dn * n), G), 256, 0, st>>>(Y, (long long)Dn * n, Qn, c->sT);
  ICK(c, cudaGetLastError());
  // the next bond: (P, Q, lam) <- (Q', P', lam'); lam_other <- lam
  c->iP = iQn;
  c->iQ = iPn;
  c->iO = c->iL;
  c->iL = iN;
  c->mid = c->outer;
  c->outer = Dn;
  return HOTRG_OK;
}

hotrg_status isync(hotrg_itebd *c) {
  ICK(c, cudaStreamSynchronize(c->stream));
  int h = 0;
  ICK(c, cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) return ifail(c, HOTRG_ENONFINITE, "a bond's density matrix has no positive weight");
  return HOTRG_OK;
}

}  // namespace

extern "C" {

hotrg_status hotrg_itebd_create(int n, const double *couplings, int D_b, int D0,
                                const double *const *P0s, const double *const *Q0s,
                                const double *const *lam0s, void *stream, hotrg_itebd **out) {
  if (!out) return HOTRG_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 65535 || !couplings || D_b < 1 || D_b > kItebdMaxD || D0 < 1 || D0 > D_b)
    return HOTRG_EINVAL;
  const bool init = P0s || Q0s || lam0s;
  if (init && (!P0s || !Q0s || !lam0s)) return HOTRG_EINVAL;
  if (!init && D0 != 1) return HOTRG_EINVAL;
  for (int i = 0; i < n; ++i) {
    const double Jxy = couplings[3 * i], Jz = couplings[3 * i + 1], tau = couplings[3 * i + 2];
    if (!std::isfinite(Jxy) || !std::isfinite(Jz) || !(tau > 0.0) || !std::isfinite(tau)) return HOTRG_EINVAL;
    if (init && (!P0s[i] || !Q0s[i] || !lam0s[i])) return HOTRG_EINVAL;
  }
  auto *c = new hotrg_itebd();
  c->stream = static_cast<cudaStream_t>(stream);
  c->G = n;
  c->Db = D_b;
  c->outer = c->mid = D0;
  const long long Db = D_b, twoD = 2 * Db;
  c->sT = (Db * kPhys * Db + 31) / 32 * 32;
  c->sL = (Db + 31) / 32 * 32;
  c->sM = (twoD * twoD + 31) / 32 * 32;
  auto bail = [&](hotrg_status s) {
    for (void *p : c->allocs) cudaFree(p);
    delete c;
    return s;
  };
  hotrg_status s = HOTRG_OK;
  for (int k = 0; k < 4 && !s; ++k) s = ialloc(c, &c->t[k], c->sT * n);
  for (int k = 0; k < 3 && !s; ++k) s = ialloc(c, &c->l[k], c->sL * n);
  if (s || (s = ialloc(c, &c->phi, c->sM * n)) || (s = ialloc(c, &c->phit, c->sM * n)) ||
      (s = ialloc(c, &c->theta, c->sM * n)) || (s = ialloc(c, &c->rho, c->sM * n)) ||
      (s = ialloc(c, &c->gates, 16LL * n)) || (s = ialloc(c, &c->hs, 16LL * n)) ||
      (s = ialloc(c, &c->disc, (long long)n)) || (s = ialloc(c, &c->energy, 2LL * n)) ||
      (s = ialloc(c, &c->trace, (long long)n)) || (s = ialloc(c, &c->rnorm, (long long)n)) ||
      (s = ialloc(c, &c->Vb[0], c->sM * n)) || (s = ialloc(c, &c->Vb[1], c->sM * n)) ||
      (s = ialloc(c, &c->Vn, c->sM * n)) ||
      (s = ialloc(c, &c->si_work, si_workspace_doubles(n, (int)twoD, jacobi_block((int)twoD)))) ||
      (s = ialloc(c, &c->err, 4LL)))
    return bail(s);
  // host-side initial state and per-chain operators
  std::vector<double> hT((size_t)(c->sT * n), 0.0), hQ((size_t)(c->sT * n), 0.0);
  std::vector<double> hL((size_t)(c->sL * n), 0.0), hO((size_t)(c->sL * n), 0.0);
  std::vector<double> hg(16 * (size_t)n), hh(16 * (size_t)n);
  const long long tsz = (long long)D0 * kPhys * D0;
  for (int i = 0; i < n; ++i) {
    xxz_gate(couplings[3 * i], couplings[3 * i + 1], couplings[3 * i + 2], &hg[16 * (size_t)i]);
    xxz_bond_h(couplings[3 * i], couplings[3 * i + 1], &hh[16 * (size_t)i]);
    double *P = &hT[(size_t)(i * c->sT)], *Q = &hQ[(size_t)(i * c->sT)];
    double *L = &hL[(size_t)(i * c->sL)], *O = &hO[(size_t)(i * c->sL)];
    if (init) {
      std::copy(P0s[i], P0s[i] + tsz, P);
      std::copy(Q0s[i], Q0s[i] + tsz, Q);
      std::copy(lam0s[i], lam0s[i] + D0, L);
    } else {               // Neel state: P = |up>, Q = |down>, D = 1
      P[0] = 1.0;
      Q[1] = 1.0;
      L[0] = 1.0;
    }
    for (int k = 0; k < D0; ++k) O[k] = 1.0 / std::sqrt((double)D0);
  }
  if (cudaMemcpyAsync(c->t[0], hT.data(), sizeof(double) * hT.size(), cudaMemcpyHostToDevice, c->stream) ||
      cudaMemcpyAsync(c->t[1], hQ.data(), sizeof(double) * hQ.size(), cudaMemcpyHostToDevice, c->stream) ||
      cudaMemcpyAsync(c->l[0], hL.data(), sizeof(double) * hL.size(), cudaMemcpyHostToDevice, c->stream) ||
      cudaMemcpyAsync(c->l[1], hO.data(), sizeof(double) * hO.size(), cudaMemcpyHostToDevice, c->stream) ||
      cudaMemcpyAsync(c->gates, hg.data(), sizeof(double) * hg.size(), cudaMemcpyHostToDevice, c->stream) ||
      cudaMemcpyAsync(c->hs, hh.data(), sizeof(double) * hh.size(), cudaMemcpyHostToDevice, c->stream) ||
      cudaMemsetAsync(c->err, 0, 4 * sizeof(int), c->stream) || cudaStreamSynchronize(c->stream))
    return bail(HOTRG_ECUDA);
  *out = c;
  return HOTRG_OK;
}

hotrg_status hotrg_itebd_step(hotrg_itebd *c, int nsteps) {
  if (!c || nsteps < 0) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  for (int k = 0; k < nsteps; ++k) {
    if (hotrg_status s = itebd_update(c)) return s;
    c->nsteps += 1;
  }
  return isync(c);
}

hotrg_status hotrg_itebd_energy(hotrg_itebd *c, double *out_n) {
  if (!c || !out_n) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  cudaStream_t st = c->stream;
  const int G = c->G, o = c->outer, m = c->mid;
  double *P = c->t[c->iP], *Q = c->t[c->iQ];
  // bond (P, Q) in the environment lam (outer bond), then bond (Q, P) in lam_other
  MappedGemm g1{kPhys * o, kPhys * o, m, P, map1(m), map1(1), Q, map1(1), map1(kPhys * o), c->phi,
                map1(kPhys * o), map1(1), G, c->sT, c->sT, c->sM};
  ICK(c, gemm_f64(g1, st));
  k_itebd_energy<<<G, 256, 0, st>>>(c->phi, c->l[c->iL], c->hs, o, o, c->sM, c->sL, c->energy, 0);
  ICK(c, cudaGetLastError());
  MappedGemm g2{kPhys * m, kPhys * m, o, Q, map1(o), map1(1), P, map1(1), map1(kPhys * m), c->phi,
                map1(kPhys * m), map1(1), G, c->sT, c->sT, c->sM};
  ICK(c, gemm_f64(g2, st));
  k_itebd_energy<<<G, 256, 0, st>>>(c->phi, c->l[c->iO], c->hs, m, m, c->sM, c->sL, c->energy, 1);
  ICK(c, cudaGetLastError());
  std::vector<double> h(2 * (size_t)G);
  ICK(c, cudaMemcpyAsync(h.data(), c->energy, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  if (hotrg_status s = isync(c)) return s;
  for (int i = 0; i < G; ++i) out_n[i] = 0.5 * (h[2 * i] + h[2 * i + 1]);
  return HOTRG_OK;
}

hotrg_status hotrg_itebd_lambda(hotrg_itebd *c, int inst, double *buf, int cap, int *nout) {
  if (!c || !buf || !nout || inst < 0 || inst >= c->G) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (cap < c->outer) return HOTRG_EINVAL;
  ICK(c, cudaMemcpyAsync(buf, c->l[c->iL] + inst * c->sL, sizeof(double) * c->outer,
                         cudaMemcpyDeviceToHost, c->stream));
  if (hotrg_status s = isync(c)) return s;
  *nout = c->outer;
  return HOTRG_OK;
}

hotrg_status hotrg_itebd_discarded(hotrg_itebd *c, int inst, double *out) {
  if (!c || !out || inst < 0 || inst >= c->G) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (c->nsteps == 0) {
    *out = 0.0;
    return HOTRG_OK;
  }
  ICK(c, cudaMemcpyAsync(out, c->disc + inst, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return isync(c);
}

hotrg_status hotrg_itebd_dims(hotrg_itebd *c, int *outer, int *mid, long long *nsteps) {
  if (!c || !outer || !mid || !nsteps) return HOTRG_EINVAL;
  *outer = c->outer;
  *mid = c->mid;
  *nsteps = c->nsteps;
  return HOTRG_OK;
}

const char *hotrg_itebd_last_error(const hotrg_itebd *c) { return c ? c->msg.c_str() : "NULL context"; }

void hotrg_itebd_destroy(hotrg_itebd *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

}  // extern "C"
