// C ABI of libhotrg (declared in include/hotrg.h): context management, initial
// tensors and the step driver that chains the kernels of one HOTRG
// coarse-graining step (Sec. II.A):
//
//   environment partials  A_L, B_L, A_R, B_R   (four GEMMs, K = Dx*Dy)
//   Gram combine          G_L, G_R              (two GEMMs, K = Dy^2), FP64 symmetrise
//   eigendecomposition    top D'(+1) pairs of G_L and G_R (FP64, cuSOLVER)
//   isometry choice       smaller discarded weight, sign-fixed U   (device)
//   projection chain      P = U.T, Q = P.T, T' = Q.U               (three GEMMs)
//   rescale               c = max|T'|, T' /= c, logsum += ln(c) / 2^n (FP64)
//
// An X step runs the same chain on the strided view T[y,y',x,x'] and writes
// its result back through the transposed view; nothing is copied to switch
// directions.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/hotrg.h"
#include "common.cuh"
#include "eig.cuh"
#include "eig_si.cuh"
#include "tc_path.cuh"

using namespace hotrg;

namespace {

constexpr int kMaxSteps = 256;
constexpr int kRecord = 8;  // side, eps_L, eps_R, cut_gap, trace_G, ln_c, -, -

// Records CUDA events around each stage while enabled; the intervals are
// resolved into milliseconds once the stream has passed them.
class Profiler : public StageHook {
 public:
  cudaStream_t stream = nullptr;
  bool on = false;
  hotrg_profile_t acc{};
  long long launches_total = 0;   // own launches, whether or not profiling is on

  ~Profiler() {
    for (auto &p : pending_) {
      cudaEventDestroy(p.b);
      cudaEventDestroy(p.e);
    }
    for (cudaEvent_t e : pool_) cudaEventDestroy(e);
  }
  void reset() {
    collect(true);
    acc = hotrg_profile_t{};
  }
  void begin(int stage) override {
    if (!on) return;
    open_[stage] = get();
    if (open_[stage]) cudaEventRecord(open_[stage], stream);
  }
  void end(int stage) override {
    if (!on || !open_[stage]) return;
    cudaEvent_t e = get();
    if (!e) return;
    cudaEventRecord(e, stream);
    pending_.push_back({stage, open_[stage], e});
    open_[stage] = nullptr;
  }
  void launched(int stage, int n) override {
    launches_total += n;
    if (!on) return;
    acc.launches += n;
    acc.stage_launches[stage] += n;
  }
  void flops(int stage, double f) {
    if (on) acc.flops[stage] += f;
  }
  // Resolve finished intervals (all of them if `all`, after a stream sync).
  void collect(bool all) {
    std::vector<Interval> keep;
    for (auto &p : pending_) {
      float ms = 0.f;
      cudaError_t r = cudaEventElapsedTime(&ms, p.b, p.e);
      if (r == cudaSuccess) {
        acc.ms[p.stage] += ms;
        pool_.push_back(p.b);
        pool_.push_back(p.e);
      } else if (r == cudaErrorNotReady && !all) {
        keep.push_back(p);
      } else {
        (void)cudaGetLastError();
        pool_.push_back(p.b);
        pool_.push_back(p.e);
      }
    }
    pending_.swap(keep);
  }

 private:
  struct Interval {
    int stage;
    cudaEvent_t b, e;
  };
  cudaEvent_t get() {
    if (!pool_.empty()) {
      cudaEvent_t e = pool_.back();
      pool_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  std::vector<Interval> pending_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t open_[HOTRG_NSTAGES] = {};
};

}  // namespace

struct hotrg_ctx {
  Profiler prof;
  cudaStream_t stream = nullptr;
  Eig eig;
  TcPath tc;
  int D0 = 0, D_cut = 0, Dm = 0;
  hotrg_prec prec = HOTRG_FP64;
  int dx = 0, dy = 0, nsteps = 0;
  int last_n = 0, last_dn = 0;   // shape of U of the last step

  double *T = nullptr, *Tn = nullptr;
  double *AL = nullptr, *BL = nullptr, *AR = nullptr, *BR = nullptr;
  double *GL = nullptr, *GR = nullptr;
  double *wL = nullptr, *wR = nullptr;
  double *U = nullptr;
  double *P = nullptr, *Q = nullptr;
  double *scal = nullptr;      // [0] logsum, [1] max scratch, [2] tr G_L, [3] tr G_R, [4] trace T
  int *err = nullptr;
  double *records = nullptr;   // kMaxSteps x kRecord
  double *spectra = nullptr;   // kMaxSteps x (D_cut + 1)
  std::vector<hotrg_step_info_t> info;
  std::vector<int> spec_count;
  // own FP64 eigensolver: workspace, Ritz vectors / values of both sides, and the
  // last isometry per direction (start vectors of the next step in that direction)
  double *si_work = nullptr;
  double *XL = nullptr, *XR = nullptr, *thL = nullptr, *thR = nullptr;
  double *Uprev[2] = {nullptr, nullptr};
  int nprev[2] = {0, 0}, kprev[2] = {0, 0};

  hotrg_status status = HOTRG_OK;
  std::string msg;
  std::vector<void *> allocs;
};

namespace {

hotrg_status fail(hotrg_ctx *c, hotrg_status s, const std::string &m) {
  if (c && c->status == HOTRG_OK) {
    c->status = s;
    c->msg = m;
  }
  return s;
}

#define CK_CUDA(c, expr)                                                                 \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((c), e_ == cudaErrorMemoryAllocation ? HOTRG_ENOMEM : HOTRG_ECUDA,     \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

template <typename T>
hotrg_status dalloc(hotrg_ctx *c, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 256);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(c, HOTRG_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return HOTRG_OK;
}

// Symmetric positive definite square root of the bond matrix, closed forms:
// Ising B = [[e^b, e^-b], [e^-b, e^b]] has eigenpairs (2 cosh b, (1,1)/sqrt2) and
// (2 sinh b, (1,-1)/sqrt2); Potts B = (e^b - 1) I + J has eigenvalue e^b - 1 + q on
// the all-ones vector and e^b - 1 on its complement.
void tensor_from_sqrt(int q, const double *W, const double *w, double *T0) {
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b)
      for (int c = 0; c < q; ++c)
        for (int d = 0; d < q; ++d) {
          double v = 0.0;
          for (int s = 0; s < q; ++s) v += w[s] * W[s * q + a] * W[s * q + b] * W[s * q + c] * W[s * q + d];
          T0[((a * q + b) * q + c) * q + d] = v;
        }
}

// Reads the device error flag after a synchronisation: 1 = a max-norm was zero
// or not finite, 2 = a bounded device wait ran out.
hotrg_status check_flag(hotrg_ctx *c) {
  int herr = 0;
  if (cudaMemcpy(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, HOTRG_ECUDA, "reading the device error flag failed");
  if (herr == 1) return fail(c, HOTRG_ENONFINITE, "max-norm of a coarse-grained tensor was zero or not finite");
  if (herr) return fail(c, HOTRG_ETIMEOUT, "a tensor-core kernel's bounded wait ran out");
  return HOTRG_OK;
}

}  // namespace

extern "C" {

const char *hotrg_status_string(hotrg_status s) {
  switch (s) {
    case HOTRG_OK: return "HOTRG_OK";
    case HOTRG_EINVAL: return "HOTRG_EINVAL";
    case HOTRG_ENOMEM: return "HOTRG_ENOMEM";
    case HOTRG_ECUDA: return "HOTRG_ECUDA";
    case HOTRG_EEIG: return "HOTRG_EEIG";
    case HOTRG_ENONFINITE: return "HOTRG_ENONFINITE";
    case HOTRG_ETIMEOUT: return "HOTRG_ETIMEOUT";
    case HOTRG_ESTATE: return "HOTRG_ESTATE";
  }
  return "HOTRG_UNKNOWN";
}

const char *hotrg_last_error(const hotrg_ctx *c) { return c ? c->msg.c_str() : "NULL context"; }

hotrg_status hotrg_ising_tensor(double beta, double h, double *T0_out) {
  if (!T0_out || !(beta > 0.0) || !isfinite(beta) || !isfinite(h)) return HOTRG_EINVAL;
  const double a = sqrt(2.0 * cosh(beta)), b = sqrt(2.0 * sinh(beta));
  const double W[4] = {0.5 * (a + b), 0.5 * (a - b), 0.5 * (a - b), 0.5 * (a + b)};
  const double w[2] = {exp(beta * h), exp(-beta * h)};
  tensor_from_sqrt(2, W, w, T0_out);
  return HOTRG_OK;
}

hotrg_status hotrg_potts_tensor(int q, double beta, double *T0_out) {
  if (!T0_out || q < 2 || q > 16 || !(beta > 0.0) || !isfinite(beta)) return HOTRG_EINVAL;
  const double r0 = sqrt(expm1(beta)), r1 = sqrt(expm1(beta) + q);
  std::vector<double> W((size_t)q * q), w((size_t)q, 1.0);
  for (int s = 0; s < q; ++s)
    for (int t = 0; t < q; ++t) W[s * q + t] = (s == t ? r0 : 0.0) + (r1 - r0) / q;
  tensor_from_sqrt(q, W.data(), w.data(), T0_out);
  return HOTRG_OK;
}

void hotrg_destroy(hotrg_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

hotrg_status hotrg_create(const double *T0, int D0, int D_cut, hotrg_prec prec, void *stream,
                          hotrg_ctx **out) {
  if (!out) return HOTRG_EINVAL;
  *out = nullptr;
  if (!T0 || D0 < 1 || D0 > 64 || D_cut < 1 || D_cut > 64) return HOTRG_EINVAL;
  if (prec != HOTRG_FP64 && prec != HOTRG_TF32 && prec != HOTRG_BF16X3 && prec != HOTRG_BF16X6)
    return HOTRG_EINVAL;
  hotrg_ctx *c = new (std::nothrow) hotrg_ctx();
  if (!c) return HOTRG_ENOMEM;
  auto bail = [&](hotrg_status s) {
    hotrg_destroy(c);
    return s;
  };
  c->stream = static_cast<cudaStream_t>(stream);
  c->prof.stream = c->stream;
  c->D0 = D0;
  c->D_cut = D_cut;
  c->Dm = D0 > D_cut ? D0 : D_cut;
  c->prec = prec;
  c->dx = c->dy = D0;
  const long long Dm = c->Dm;
  const long long t4 = Dm * Dm * Dm * Dm;            // any tensor, partial or Gram matrix
  const long long p5 = (long long)D_cut * t4;        // P and Q
  const long long nmax = Dm * Dm;
  hotrg_status s;
  if ((s = dalloc(c, &c->T, t4)) || (s = dalloc(c, &c->Tn, t4)) || (s = dalloc(c, &c->AL, t4)) ||
      (s = dalloc(c, &c->BL, t4)) || (s = dalloc(c, &c->AR, t4)) || (s = dalloc(c, &c->BR, t4)) ||
      (s = dalloc(c, &c->GL, t4)) || (s = dalloc(c, &c->GR, t4)) || (s = dalloc(c, &c->wL, nmax)) ||
      (s = dalloc(c, &c->wR, nmax)) || (s = dalloc(c, &c->U, nmax * (D_cut + 1))) ||
      (s = dalloc(c, &c->scal, 8)) || (s = dalloc(c, &c->err, 4)) ||
      (s = dalloc(c, &c->records, (size_t)kMaxSteps * kRecord)) ||
      (s = dalloc(c, &c->spectra, (size_t)kMaxSteps * (D_cut + 1))))
    return bail(s);
  {
    const int nsi = (int)(nmax > kSiMaxBlock + 1 ? nmax : kSiMaxBlock + 1);
    if ((s = dalloc(c, &c->si_work, (size_t)si_workspace_doubles(2, nsi, kSiMaxBlock))) ||
        (s = dalloc(c, &c->XL, (size_t)nsi * kSiMaxBlock)) ||
        (s = dalloc(c, &c->XR, (size_t)nsi * kSiMaxBlock)) || (s = dalloc(c, &c->thL, kSiMaxBlock)) ||
        (s = dalloc(c, &c->thR, kSiMaxBlock)) || (s = dalloc(c, &c->Uprev[0], nmax * D_cut)) ||
        (s = dalloc(c, &c->Uprev[1], nmax * D_cut)))
      return bail(s);
  }
  if (prec == HOTRG_FP64) {
    if ((s = dalloc(c, &c->P, p5)) || (s = dalloc(c, &c->Q, p5))) return bail(s);
  } else {
    int r = c->tc.init(prec, D0, D_cut, c->stream, c->err);
    if (r == 2) return bail(HOTRG_ENOMEM);
    if (r) return bail(HOTRG_ECUDA);
  }
  if (int r = c->eig.init(c->stream)) return bail(r == 2 ? HOTRG_ENOMEM : HOTRG_ECUDA);
  if (cudaMemsetAsync(c->scal, 0, 8 * sizeof(double), c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->T, T0, sizeof(double) * D0 * D0 * D0 * D0, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      scale_initial(c->T, (long long)D0 * D0 * D0 * D0, c->scal + 1, c->scal, c->err,
                    c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(HOTRG_ECUDA);
  int herr = 0;
  if (cudaMemcpy(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bail(HOTRG_ECUDA);
  if (herr) return bail(HOTRG_ENONFINITE);
  *out = c;
  return HOTRG_OK;
}

hotrg_status hotrg_step(hotrg_ctx *c, hotrg_dir dir) {
  if (!c) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (dir != HOTRG_DIR_X && dir != HOTRG_DIR_Y) return HOTRG_EINVAL;
  if (c->nsteps >= kMaxSteps) return fail(c, HOTRG_ESTATE, "step limit reached");
  cudaStream_t st = c->stream;
  Profiler &pf = c->prof;

  // ---- the step's view of the stored tensor T[x,x',y,y'] (shape dx,dx,dy,dy)
  const bool ydir = (dir == HOTRG_DIR_Y);
  const int D = ydir ? c->dx : c->dy;     // fused legs
  const int E = ydir ? c->dy : c->dx;     // contracted legs
  const long long cx = (long long)c->dx * c->dy * c->dy, cxp = (long long)c->dy * c->dy,
                  cy = c->dy, cyp = 1;
  const long long sx = ydir ? cx : cy, sxp = ydir ? cxp : cyp;
  const long long sy = ydir ? cy : cx, syp = ydir ? cyp : cxp;
  const int n = D * D;
  const int Dn = n < c->D_cut ? n : c->D_cut;
  const long long DE = (long long)D * E, E2 = (long long)E * E, D2 = (long long)D * D;
  const int step = c->nsteps;
  double *rec = c->records + (size_t)step * kRecord;
  double *spec = c->spectra + (size_t)step * (c->D_cut + 1);
  const double fD = D, fE = E, fDn = Dn;
  pf.flops(HOTRG_ST_ENV, 4.0 * 2.0 * fD * fD * fD * fE * fE * fE);
  pf.flops(HOTRG_ST_GRAM, 2.0 * 2.0 * fD * fD * fD * fD * fE * fE);
  pf.flops(HOTRG_ST_PROJ_P, 2.0 * fDn * fD * fD * fD * fE * fE);
  pf.flops(HOTRG_ST_PROJ_Q, 2.0 * fDn * fD * fD * fD * fE * fE * fE);
  pf.flops(HOTRG_ST_PROJ_T, 2.0 * fDn * fDn * fD * fD * fE * fE);

  // ---- a2/a3: environments G_L, G_R ([x1][x2][u1][u2], FP64)
  const bool tc = (c->prec != HOTRG_FP64);
  if (tc) {
    if (c->tc.environment(c->T, D, E, sx, sxp, sy, syp, c->GL, c->GR, &pf))
      return fail(c, HOTRG_ECUDA, "tensor-core environment chain failed");
  } else {
    // partials written as [x][u][k][k'] for the Gram combine
    const IdxMap out_m = map2(E, E, (long long)D * E2), out_n = map2(E, 1, E2);
    struct Part { double *dst; IdxMap row, red; };
    const Part parts[4] = {
        {c->AL, map2(E, syp, sx), map2(E, sy, sxp)},    // A_L[x1,k,u1,k']: sum over (x1', y)
        {c->BL, map2(E, sy, sx), map2(E, syp, sxp)},    // B_L[x2,k,u2,k']: sum over (x2', y')
        {c->AR, map2(E, syp, sxp), map2(E, sy, sx)},    // A_R[x1',k,u1',k']: sum over (x1, y)
        {c->BR, map2(E, sy, sxp), map2(E, syp, sx)},    // B_R[x2',k,u2',k']: sum over (x2, y')
    };
    pf.begin(HOTRG_ST_ENV);
    for (const Part &p : parts) {
      MappedGemm g{(int)DE, (int)DE, (int)DE, c->T, p.row, p.red, c->T, p.row, p.red, p.dst, out_m, out_n};
      CK_CUDA(c, gemm_f64(g, st));
    }
    pf.launched(HOTRG_ST_ENV, 4);
    pf.end(HOTRG_ST_ENV);
    // G[x1,x2,u1,u2] = sum_{k,k'} A[x1,u1,k,k'] B[x2,u2,k,k']
    pf.begin(HOTRG_ST_GRAM);
    const IdxMap gm = map2(D, D, D2 * D), gn = map2(D, 1, D2);
    MappedGemm gl{(int)D2, (int)D2, (int)E2, c->AL, map1(E2), map1(1), c->BL, map1(E2), map1(1), c->GL, gm, gn};
    MappedGemm gr{(int)D2, (int)D2, (int)E2, c->AR, map1(E2), map1(1), c->BR, map1(E2), map1(1), c->GR, gm, gn};
    CK_CUDA(c, gemm_f64(gl, st));
    CK_CUDA(c, gemm_f64(gr, st));
    pf.launched(HOTRG_ST_GRAM, 2);
  }
  CK_CUDA(c, symmetrize_trace(c->GL, n, c->scal + 2, st));
  CK_CUDA(c, symmetrize_trace(c->GR, n, c->scal + 3, st));
  pf.launched(HOTRG_ST_GRAM, 4);
  pf.end(HOTRG_ST_GRAM);

  // ---- a4: FP64 eigendecomposition and choice of U
  pf.begin(HOTRG_ST_EIG);
  int spec_n;
  int eig_path = 0, eig_iters = 0;
  double eig_res = 0.0;
  if (n <= c->D_cut) {
    // nothing is cut (U = I); the spectrum of G_L is still recorded
    CK_CUDA(c, identity_isometry(c->U, n, st));
    SiBatch sb{};
    sb.P = 1;
    sb.n = n;
    sb.k = n;
    sb.G[0] = c->GL;
    sb.X[0] = c->XL;
    sb.theta[0] = c->thL;
    long long nl = 0;
    CK_CUDA(c, jacobi_full(sb, c->si_work, st, &nl));
    CK_CUDA(c, spectrum_no_cut(c->thL, n, 1, c->scal + 2, rec, spec, st));
    pf.launched(HOTRG_ST_EIG, 2 + (int)nl);
    spec_n = n;
  } else {
    // leading k = D'+1 eigenpairs of both environments (batched FP64 solver)
    const int k = Dn + 1;
    SiBatch sb{};
    sb.P = 2;
    sb.n = n;
    sb.k = k;
    sb.G[0] = c->GL;
    sb.G[1] = c->GR;
    sb.X[0] = c->XL;
    sb.X[1] = c->XR;
    sb.theta[0] = c->thL;
    sb.theta[1] = c->thR;
    long long nl = 0;
    bool ok = false;
    if (n + (n & 1) <= kSiMaxBlock) {
      CK_CUDA(c, jacobi_full(sb, c->si_work, st, &nl));
      eig_path = 1;
      ok = true;
    } else {
      int m = ((2 * k + 7) / 8) * 8;
      if (m > kSiMaxBlock) m = kSiMaxBlock;
      if (m > n) m = n & ~1;
      sb.m = m;
      const int di = ydir ? 1 : 0;
      if (c->nprev[di] == n && c->kprev[di] <= m) {
        sb.warm[0] = sb.warm[1] = c->Uprev[di];
        sb.kw = c->kprev[di];
      }
      SiResult r{};
      CK_CUDA(c, si_solve(sb, c->si_work, 1e-12, 80, st, &r, &nl));
      eig_path = 2;
      eig_iters = r.iterations;
      eig_res = r.residual;
      ok = r.converged;
    }
    pf.launched(HOTRG_ST_EIG, (int)nl);
    if (ok) {
      SelectArgs a{n, Dn, k, 1, c->thL, c->thR, c->XL, c->XR, c->scal + 2, c->scal + 3, c->U, rec, spec};
      CK_CUDA(c, select_isometry(a, st));
    } else {
      // library fallback (G_L, G_R are untouched by the own solver)
      eig_path = 3;
      if (int r = c->eig.top(c->GL, n, k, c->wL, 0))
        return fail(c, r == 2 ? HOTRG_ENOMEM : HOTRG_EEIG, "eigensolver (left) failed");
      if (int r = c->eig.top(c->GR, n, k, c->wR, 1))
        return fail(c, r == 2 ? HOTRG_ENOMEM : HOTRG_EEIG, "eigensolver (right) failed");
      SelectArgs a{n, Dn, k, 0, c->wL, c->wR, c->GL, c->GR, c->scal + 2, c->scal + 3, c->U, rec, spec};
      CK_CUDA(c, select_isometry(a, st));
    }
    pf.launched(HOTRG_ST_EIG, 1);
    const int di = ydir ? 1 : 0;
    CK_CUDA(c, cudaMemcpyAsync(c->Uprev[di], c->U, sizeof(double) * (size_t)n * Dn,
                               cudaMemcpyDeviceToDevice, st));
    c->nprev[di] = n;
    c->kprev[di] = Dn;
    spec_n = k;
  }
  pf.end(HOTRG_ST_EIG);
  int hinfo[2] = {0, 0};
  CK_CUDA(c, cudaMemcpyAsync(hinfo, c->eig.d_info(), sizeof(hinfo), cudaMemcpyDeviceToHost, st));
  CK_CUDA(c, cudaStreamSynchronize(st));
  pf.collect(false);
  if (hotrg_status fs = check_flag(c)) return fs;
  if (eig_path == 3 && (hinfo[0] != 0 || hinfo[1] != 0))
    return fail(c, HOTRG_EEIG, "eigensolver info = " + std::to_string(hinfo[0]) + ", " +
                                   std::to_string(hinfo[1]));

  // ---- a5-a7: projection chain
  // output of the step in the stored layout: Y -> T'[a][b][y][y'], X -> T'[x][x'][a][b]
  const IdxMap tm = ydir ? map3(E, E, 1, E, (long long)Dn * E2)
                         : map3(E, E, (long long)Dn * Dn, (long long)E * Dn * Dn, Dn);
  const IdxMap tn = ydir ? map1(E2) : map1(1);
  if (tc) {
    if (c->tc.project(c->T, c->U, D, E, Dn, sx, sxp, sy, syp, c->Tn, tm, tn, &pf))
      return fail(c, HOTRG_ECUDA, "tensor-core projection chain failed");
  } else {
    // a5: P[a][x1'][y][x2][k] = sum_x1 U[(x1 x2), a] T[x1,x1',y,k]
    pf.begin(HOTRG_ST_PROJ_P);
    MappedGemm g5{(int)(D * Dn), (int)(D * E2), D,
                  c->U, map2(Dn, n, 1), map1(D),
                  c->T, map3(E, E, syp, sy, sxp), map1(sx),
                  c->P, map2(Dn, D2 * E2, E), map3(E, E, 1, DE, DE * E)};
    CK_CUDA(c, gemm_f64(g5, st));
    pf.launched(HOTRG_ST_PROJ_P, 1);
    pf.end(HOTRG_ST_PROJ_P);
    // a6: Q[a][y][y'][x1'][x2'] = sum_{x2,k} P[(a,x1',y),(x2,k)] T[x2,x2',k,y']
    pf.begin(HOTRG_ST_PROJ_Q);
    MappedGemm g6{(int)(Dn * DE), (int)DE, (int)DE,
                  c->P, map1(DE), map1(1),
                  c->T, map2(D, sxp, syp), map2(E, sy, sx),
                  c->Q, map3(E, D, E * D2, D, E2 * D2), map2(D, 1, D2)};
    CK_CUDA(c, gemm_f64(g6, st));
    pf.launched(HOTRG_ST_PROJ_Q, 1);
    pf.end(HOTRG_ST_PROJ_Q);
    // a7: T'[(a,y,y'), b] = sum_{x1',x2'} Q[(a,y,y'),(x1',x2')] U[(x1' x2'), b]
    pf.begin(HOTRG_ST_PROJ_T);
    MappedGemm g7{(int)(Dn * E2), Dn, (int)D2,
                  c->Q, map1(D2), map1(1),
                  c->U, map1(n), map1(1),
                  c->Tn, tm, tn};
    CK_CUDA(c, gemm_f64(g7, st));
    pf.launched(HOTRG_ST_PROJ_T, 1);
    pf.end(HOTRG_ST_PROJ_T);
  }

  // ---- a8: rescale and FP64 log-sum
  pf.begin(HOTRG_ST_RESCALE);
  const long long count = (long long)Dn * Dn * E2;
  CK_CUDA(c, maxabs_scale_log(c->Tn, count, c->scal + 1, c->scal, ldexp(1.0, -(step + 1)),
                              rec + 5, c->err, st));
  pf.launched(HOTRG_ST_RESCALE, 2);
  pf.end(HOTRG_ST_RESCALE);
  if (pf.on) pf.acc.steps += 1;
  double *tmp = c->T;
  c->T = c->Tn;
  c->Tn = tmp;
  if (ydir) c->dx = Dn; else c->dy = Dn;
  c->last_n = n;
  c->last_dn = Dn;
  c->nsteps = step + 1;
  hotrg_step_info_t inf{};
  inf.dir = dir;
  inf.Dx = D;
  inf.Dy = E;
  inf.Dn = Dn;
  inf.eig_path = eig_path;
  inf.eig_iters = eig_iters;
  inf.eig_residual = eig_res;
  c->info.push_back(inf);
  c->spec_count.push_back(spec_n);
  return HOTRG_OK;
}

hotrg_status hotrg_profile_enable(hotrg_ctx *c, int enable) {
  if (!c) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  c->prof.reset();
  c->prof.on = enable != 0;
  return HOTRG_OK;
}

hotrg_status hotrg_profile_read(hotrg_ctx *c, hotrg_profile_t *out) {
  if (!c || !out) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  c->prof.collect(true);
  *out = c->prof.acc;
  return HOTRG_OK;
}

hotrg_status hotrg_log_z_per_site(hotrg_ctx *c, double *out) {
  if (!c || !out) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  CK_CUDA(c, periodic_trace(c->T, c->dx, c->dy, c->scal + 4, c->stream));
  double h[5];
  CK_CUDA(c, cudaMemcpyAsync(h, c->scal, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  if (hotrg_status fs = check_flag(c)) return fs;
  if (!(h[4] > 0.0) || !isfinite(h[4]))
    return fail(c, HOTRG_ENONFINITE, "periodic trace is not positive");
  *out = h[0] + log(h[4]) * ldexp(1.0, -c->nsteps);
  return HOTRG_OK;
}

hotrg_status hotrg_free_energy(hotrg_ctx *c, double beta, double *f_out) {
  if (!c || !f_out || !(beta > 0.0)) return HOTRG_EINVAL;
  double lz;
  hotrg_status s = hotrg_log_z_per_site(c, &lz);
  if (s != HOTRG_OK) return s;
  *f_out = -lz / beta;
  return HOTRG_OK;
}

hotrg_status hotrg_step_info(hotrg_ctx *c, int step, hotrg_step_info_t *out) {
  if (!c || !out) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (step < 0 || step >= c->nsteps) return HOTRG_EINVAL;
  double r[kRecord];
  CK_CUDA(c, cudaMemcpyAsync(r, c->records + (size_t)step * kRecord, sizeof(r),
                             cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = c->info[step];
  out->side = (int)r[0];
  out->eps_L = r[1];
  out->eps_R = r[2];
  out->cut_gap = r[3];
  out->trace_G = r[4];
  out->ln_c = r[5];
  return HOTRG_OK;
}

hotrg_status hotrg_spectrum(hotrg_ctx *c, int step, double *buf, int cap, int *n) {
  if (!c || !n || (cap > 0 && !buf)) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (step < 0 || step >= c->nsteps) return HOTRG_EINVAL;
  const int cnt = c->spec_count[step];
  *n = cnt;
  const int k = cnt < cap ? cnt : cap;
  if (k > 0) {
    CK_CUDA(c, cudaMemcpyAsync(buf, c->spectra + (size_t)step * (c->D_cut + 1), sizeof(double) * k,
                               cudaMemcpyDeviceToHost, c->stream));
    CK_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return HOTRG_OK;
}

hotrg_status hotrg_get_tensor(hotrg_ctx *c, double *host_out, long long cap, int dims[4]) {
  if (!c || !dims) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  dims[0] = dims[1] = c->dx;
  dims[2] = dims[3] = c->dy;
  const long long cnt = (long long)c->dx * c->dx * c->dy * c->dy;
  if (!host_out || cap < cnt) return HOTRG_EINVAL;
  CK_CUDA(c, cudaMemcpyAsync(host_out, c->T, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOTRG_OK;
}

hotrg_status hotrg_get_isometry(hotrg_ctx *c, double *host_out, long long cap, int *rows, int *cols) {
  if (!c || !rows || !cols) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (c->nsteps == 0) return HOTRG_ESTATE;
  *rows = c->last_n;
  *cols = c->last_dn;
  const long long cnt = (long long)c->last_n * c->last_dn;
  if (!host_out || cap < cnt) return HOTRG_EINVAL;
  CK_CUDA(c, cudaMemcpyAsync(host_out, c->U, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOTRG_OK;
}

hotrg_status hotrg_dims(hotrg_ctx *c, int *Dx, int *Dy, int *nsteps) {
  if (!c || !Dx || !Dy || !nsteps) return HOTRG_EINVAL;
  *Dx = c->dx;
  *Dy = c->dy;
  *nsteps = c->nsteps;
  return HOTRG_OK;
}

}  // extern "C"
