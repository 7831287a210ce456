// C ABI of libhotrg (declared in include/hotrg.h): context management, initial
// tensors and the step driver that chains the kernels of one HOTRG
// coarse-graining step (Sec. II.A):
//
//   environment partials  A_L, B_L, A_R, B_R   (four GEMMs, K = Dx*Dy)
//   Gram combine          G_L, G_R              (two GEMMs, K = Dy^2), FP64 symmetrise
//   eigendecomposition    top D'(+1) pairs of G_L and G_R (FP64)
//   isometry choice       smaller discarded weight, sign-fixed U   (device)
//   projection chain      P = U.T, Q = P.T, T' = Q.U               (three GEMMs)
//   rescale               c = max|T'|, T' /= c, logsum += ln(c) / 2^n (FP64)
//
// An X step runs the same chain on the strided view T[y,y',x,x'] and writes
// its result back through the transposed view; nothing is copied to switch
// directions.
//
// A context holds one or more instances.  Instances with the same (D0, D_cut)
// have the same bond dimensions after every step, so they form a group whose
// buffers sit at a fixed per-instance stride; every kernel of the step runs
// once per group over all of its instances (grid.z / grid.y batching), and the
// eigensolver treats the group's 2G environments as one batch.  A context made
// by hotrg_create is a single group of one instance.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hotrg.h"
#include "common.cuh"
#include "eig_si.cuh"
#include "tc_exact.cuh"
#include "tc_gemm.cuh"
#include "tc_path.cuh"
#include "tcgen05.cuh"
#include "xxz.cuh"

using namespace hotrg;

namespace {

constexpr int kMaxSteps = 256;
constexpr int kRecord = 8;       // side, eps_L, eps_R, cut_gap, trace_G, ln_c, -, -
constexpr int kScal = 8;         // logsum, max scratch, tr G_L, tr G_R, trace T, ln c of trace_y, -, -
constexpr int kMaxInstances = 4096;
constexpr int kXsDigitsMax = 8;  // digits per operand row of the exact-slice contraction mode

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

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
      if (p.graph_owned) continue;
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
    if (open_[stage]) record(open_[stage]);
  }
  // inside a capture the event must be an external record node, recorded each
  // time the graph runs (a plain record would only order the capture)
  void record(cudaEvent_t e) {
    if (capture_)
      cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal);
    else
      cudaEventRecord(e, stream);
  }
  void end(int stage) override {
    if (!on || !open_[stage]) return;
    cudaEvent_t e = get();
    if (!e) return;
    record(e);
    if (capture_) {
      captured_.push_back({stage, open_[stage], e, true});
    } else {
      pending_.push_back({stage, open_[stage], e, false});
    }
    open_[stage] = nullptr;
  }
  // While a graph is captured, the stage events become event-record nodes of
  // the graph (owned by it, never pooled); each replay queues them for timing.
  struct Interval {
    int stage;
    cudaEvent_t b, e;
    bool graph_owned;
  };
  void begin_capture() {
    capture_ = true;
    captured_.clear();
  }
  std::vector<Interval> end_capture() {
    capture_ = false;
    std::vector<Interval> v;
    v.swap(captured_);
    return v;
  }
  void replay(const std::vector<Interval> &v) {
    for (const Interval &i : v) pending_.push_back(i);
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
        if (!p.graph_owned) {
          pool_.push_back(p.b);
          pool_.push_back(p.e);
        }
      } else if (r == cudaErrorNotReady && !all) {
        keep.push_back(p);
      } else {
        (void)cudaGetLastError();
        if (!p.graph_owned) {
          pool_.push_back(p.b);
          pool_.push_back(p.e);
        }
      }
    }
    pending_.swap(keep);
  }

 private:
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
  std::vector<Interval> pending_, captured_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t open_[HOTRG_NSTAGES] = {};
  bool capture_ = false;
};

// An instantiated graph of one contraction segment, its kernel count per
// stage, and the stage events recorded inside it (when it was captured with
// the profiler on).
struct SegGraph {
  cudaGraphExec_t exec = nullptr;
  long long launches[HOTRG_NSTAGES] = {};
  std::vector<Profiler::Interval> events;
};

// Hook used while a segment is captured: stage events go into the graph,
// launches are counted for the replays.
struct CaptureHook : StageHook {
  Profiler *prof;
  long long per_stage[HOTRG_NSTAGES] = {};
  explicit CaptureHook(Profiler *p) : prof(p) {}
  void begin(int stage) override { prof->begin(stage); }
  void end(int stage) override { prof->end(stage); }
  void launched(int stage, int n) override { per_stage[stage] += n; }
};

// Per-step diagnostics that are the same for every instance of a group.
struct GroupStep {
  hotrg_step_info_t info;   // dir, Dx, Dy, Dn, eig_path, eig_iters, eig_residual
  int spec_count;
  int n, dn;                // shape of U
};

// Instances that share (D0, D_cut) and so every bond dimension.  Buffers hold
// G instances at the strides below (elements, multiples of 32 doubles).
struct Group {
  int D0 = 0, D_cut = 0, Dm = 0, G = 0;
  int dx = 0, dy = 0;
  std::vector<int> members;       // instance ids, in creation order
  long long sT = 0;               // T, Tn, partials, Gram matrices: Dm^4
  long long sU = 0;               // U: Dm^2 (D_cut + 1)
  long long sUp = 0;              // previous isometry per direction: Dm^2 D_cut
  long long sP = 0;               // FP64 P and Q: D_cut Dm^4
  long long sRec = 0, sSpec = 0;  // step records / spectra per instance
  double *T = nullptr, *Tn = nullptr;
  double *AL = nullptr, *BL = nullptr, *AR = nullptr, *BR = nullptr;
  double *GL = nullptr, *GR = nullptr;
  double *U = nullptr, *P = nullptr, *Q = nullptr;
  // tensor-core modes: FP64 partials and P, Q of the steps with D = 1 (each
  // Dm^2 per instance at stride sC1; the full-size buffers above stay unset)
  double *c1 = nullptr;
  long long sC1 = 0;
  double *scal = nullptr;         // kScal per instance
  double *records = nullptr;      // kMaxSteps x kRecord per instance
  double *spectra = nullptr;      // kMaxSteps x (D_cut + 1) per instance
  double *Uprev[2] = {nullptr, nullptr};
  int nprev[2] = {0, 0}, kprev[2] = {0, 0};
  // all m Ritz vectors of both environments of the last solve per direction
  // (problem z of the solve at Xprev + z sXp), the next solve's start block
  double *Xprev[2] = {nullptr, nullptr};
  long long sXp = 0;
  int xprev_n[2] = {0, 0}, xprev_m[2] = {0, 0};
  int iters_prev[2] = {0, 0};     // subspace iterations of the last solve per direction
  int rr_prev[2] = {0, 0};        // and its Rayleigh-Ritz steps
  TcPath tc;
  XsWork xw{};                    // exact-slice contraction mode scratch
  std::vector<GroupStep> steps;
  // CUDA graphs of the tensor-core contraction segments, keyed by (segment,
  // direction, D, E, D', address of T, profiler on): the key fixes every
  // launch's arguments, and T alternates between two buffers, so a
  // steady-state run replays two graphs per segment.
  std::map<std::array<long long, 8>, SegGraph> graphs;
  std::set<std::array<long long, 8>> seen, nograph;
  // Work of the group's steps: its own stream (the context's stream when the
  // context holds one group), stage profiler and eigensolver workspace, so
  // that the groups of a batch can step concurrently.
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Profiler prof;
  double *si_work = nullptr;
  ~Group() {
    if (own_stream && stream) {
      cudaStreamSynchronize(stream);
      cudaStreamDestroy(stream);
    }
    for (auto &kv : graphs) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      for (auto &iv : kv.second.events) {
        cudaEventDestroy(iv.b);
        cudaEventDestroy(iv.e);
      }
    }
  }
};

}  // namespace

struct hotrg_ctx {
  bool prof_on = false;                     // stage profiler enabled
  int prof_steps = 0;                       // steps taken while it was on
  std::mutex mu;                            // guards status/msg (groups step on their own threads)
  cudaStream_t stream = nullptr;
  hotrg_prec prec = HOTRG_FP64;
  int nsteps = 0;
  int n_inst = 0;
  std::vector<std::unique_ptr<Group>> groups;
  std::vector<std::pair<int, int>> where;   // instance -> (group, index in group)
  bool eig_tc = true;                       // exact-slice tensor-core products G X
  bool use_graphs = true;                   // replay contraction segments as CUDA graphs
  bool fuse_chain = false;                  // fused a6 -> a7 kernel where its shapes allow
  int xs_digits = 6;                        // digits of the exact-slice contraction mode
  int eig_max_iters = 80;                   // subspace iterations before HOTRG_EEIG
  int *err = nullptr;
  hotrg_status status = HOTRG_OK;
  std::string msg;
  std::vector<void *> allocs;
};

namespace {

hotrg_status fail(hotrg_ctx *c, hotrg_status s, const std::string &m) {
  if (!c) return s;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->status == HOTRG_OK) {
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
// or not finite, 2 = a bounded device wait ran out, 3 = an index outside its
// buffer (bounds-checked build only).
hotrg_status check_flag(hotrg_ctx *c) {
  int herr = 0;
  if (cudaMemcpy(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, HOTRG_ECUDA, "reading the device error flag failed");
  if (herr == 1) return fail(c, HOTRG_ENONFINITE, "max-norm of a coarse-grained tensor was zero or not finite");
  if (herr == 3)
    return fail(c, HOTRG_EBOUNDS, "a kernel's mapped index fell outside its buffer (bounds-checked build)");
  if (herr) return fail(c, HOTRG_ETIMEOUT, "a tensor-core kernel's bounded wait ran out");
  return HOTRG_OK;
}

// Device buffers of one group, sized for bond dimensions up to max(D0, D_cut).
hotrg_status alloc_group(hotrg_ctx *c, Group &g) {
  const long long Dm = g.Dm, t4 = Dm * Dm * Dm * Dm, nmax = Dm * Dm;
  const int G = g.G;
  g.sT = round_up(t4, 32);
  g.sU = round_up(nmax * (g.D_cut + 1), 32);
  g.sUp = round_up(nmax * g.D_cut, 32);
  g.sXp = round_up(nmax * kSiMaxBlock, 32);
  g.sP = round_up((long long)g.D_cut * t4, 32);
  g.sRec = (long long)kMaxSteps * kRecord;
  g.sSpec = round_up((long long)kMaxSteps * (g.D_cut + 1), 32);
  hotrg_status s;
  if ((s = dalloc(c, &g.T, g.sT * G)) || (s = dalloc(c, &g.Tn, g.sT * G)) ||
      (s = dalloc(c, &g.GL, 2 * g.sT * G)) ||
      (s = dalloc(c, &g.U, g.sU * G)) || (s = dalloc(c, &g.scal, (long long)kScal * G)) ||
      (s = dalloc(c, &g.records, g.sRec * G)) || (s = dalloc(c, &g.spectra, g.sSpec * G)) ||
      (s = dalloc(c, &g.Uprev[0], g.sUp * G)) || (s = dalloc(c, &g.Uprev[1], g.sUp * G)) ||
      (s = dalloc(c, &g.Xprev[0], g.sXp * 2 * G)) || (s = dalloc(c, &g.Xprev[1], g.sXp * 2 * G)))
    return s;
  // G_R follows G_L's G instances (one batched Gram combine over both sides)
  g.GR = g.GL + g.sT * G;
  if (c->prec == HOTRG_FP64 || c->prec == HOTRG_BF16XS) {
    if ((s = dalloc(c, &g.AL, g.sT * G)) || (s = dalloc(c, &g.BL, g.sT * G)) ||
        (s = dalloc(c, &g.AR, g.sT * G)) || (s = dalloc(c, &g.BR, g.sT * G)) ||
        (s = dalloc(c, &g.P, g.sP * G)) || (s = dalloc(c, &g.Q, g.sP * G)))
      return s;
    if (c->prec == HOTRG_BF16XS) {
      // largest operands of the step's GEMMs (every dimension <= Dm, D' <= D_cut)
      const int Dm2 = g.Dm * g.Dm, Dc = g.D_cut;
      const int shapes[5][3] = {{Dm2, Dm2, Dm2},                   // a2, a3
                                {g.Dm * Dc, g.Dm * Dm2, g.Dm},     // a5
                                {Dc * Dm2, Dm2, Dm2},              // a6
                                {Dc * Dm2, Dc, Dm2},               // a7
                                {Dm2, Dm2, Dm2}};
      long long cap[5] = {0, 0, 0, 0, 0};
      for (auto &sh : shapes) {
        long long need[5];
        xs_gemm_needs(sh[0], sh[1], sh[2], kXsDigitsMax, G, need);
        for (int i = 0; i < 5; ++i) cap[i] = std::max(cap[i], need[i]);
      }
      short *sa = nullptr, *sb = nullptr;
      if ((s = dalloc(c, &sa, cap[0])) || (s = dalloc(c, &sb, cap[1])) ||
          (s = dalloc(c, &g.xw.sca, cap[2])) || (s = dalloc(c, &g.xw.scb, cap[3])) ||
          (cap[4] > 0 && (s = dalloc(c, &g.xw.parts, cap[4]))))
        return s;
      g.xw.sa = sa;
      g.xw.sb = sb;
      g.xw.cap_a = cap[0];
      g.xw.cap_b = cap[1];
      g.xw.cap_sa = cap[2];
      g.xw.cap_sb = cap[3];
      g.xw.cap_parts = cap[4];
    }
  } else {
    g.sC1 = round_up(nmax, 32);
    if ((s = dalloc(c, &g.c1, 6 * g.sC1 * G))) return s;
    const int r = g.tc.init(c->prec, g.D0, g.D_cut, G, g.stream, c->err);
    if (r == 2) return fail(c, HOTRG_ENOMEM, "tensor-core operand buffers do not fit");
    if (r) return fail(c, HOTRG_ECUDA, "tensor-core path initialisation failed");
  }
  return HOTRG_OK;
}

bool valid_prec(hotrg_prec p) {
  return p == HOTRG_FP64 || p == HOTRG_TF32 || p == HOTRG_BF16X3 || p == HOTRG_BF16X6 ||
         p == HOTRG_BF16XS;
}

// Shared constructor: n instances, T0s[i] of D0s[i]^4 doubles.
hotrg_status create_ctx(int n, const double *const *T0s, const int *D0s, const int *Dcuts,
                        hotrg_prec prec, void *stream, hotrg_ctx **out) {
  if (!out) return HOTRG_EINVAL;
  *out = nullptr;
  if (n < 1 || n > kMaxInstances || !T0s || !D0s || !Dcuts || !valid_prec(prec)) return HOTRG_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!T0s[i] || D0s[i] < 1 || D0s[i] > 64 || Dcuts[i] < 1 || Dcuts[i] > 64) return HOTRG_EINVAL;
  hotrg_ctx *c = new (std::nothrow) hotrg_ctx();
  if (!c) return HOTRG_ENOMEM;
  auto bail = [&](hotrg_status s) {
    hotrg_destroy(c);
    return s;
  };
  c->stream = static_cast<cudaStream_t>(stream);
  c->prec = prec;
  c->n_inst = n;
  c->where.resize(n);
  for (int i = 0; i < n; ++i) {
    int gi = -1;
    for (int j = 0; j < (int)c->groups.size(); ++j)
      if (c->groups[j]->D0 == D0s[i] && c->groups[j]->D_cut == Dcuts[i]) gi = j;
    if (gi < 0) {
      std::unique_ptr<Group> g(new (std::nothrow) Group());
      if (!g) return bail(HOTRG_ENOMEM);
      g->D0 = D0s[i];
      g->D_cut = Dcuts[i];
      g->Dm = std::max(D0s[i], Dcuts[i]);
      g->dx = g->dy = D0s[i];
      c->groups.push_back(std::move(g));
      gi = (int)c->groups.size() - 1;
    }
    Group &g = *c->groups[gi];
    c->where[i] = {gi, (int)g.members.size()};
    g.members.push_back(i);
  }
  hotrg_status s;
  if ((s = dalloc(c, &c->err, 4))) return bail(s);
  for (auto &gp : c->groups) {
    Group &g = *gp;
    g.G = (int)g.members.size();
    if (c->groups.size() == 1) {
      g.stream = c->stream;
    } else {
      if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        return bail(HOTRG_ECUDA);
      }
      g.own_stream = true;
    }
    g.prof.stream = g.stream;
    if ((s = alloc_group(c, g))) return bail(s);
    const int nsi = std::max(g.Dm * g.Dm, kSiMaxBlock + 1);
    if ((s = dalloc(c, &g.si_work, (size_t)si_workspace_doubles(2 * g.G, nsi, kSiMaxBlock))))
      return bail(s);
  }
  if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess) return bail(HOTRG_ECUDA);
  for (auto &gp : c->groups) {
    Group &g = *gp;
    const long long cnt = (long long)g.D0 * g.D0 * g.D0 * g.D0;
    if (cudaMemsetAsync(g.scal, 0, sizeof(double) * kScal * g.G, c->stream) != cudaSuccess)
      return bail(HOTRG_ECUDA);
    for (int j = 0; j < g.G; ++j)
      if (cudaMemcpyAsync(g.T + j * g.sT, T0s[g.members[j]], sizeof(double) * cnt,
                          cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return bail(HOTRG_ECUDA);
    // c_0 = max|T0| with weight 1: the initial tensor is one site
    if (maxabs_scale_log(g.T, cnt, g.sT, g.scal + 1, kScal, g.scal, kScal, 1.0, nullptr, 0, c->err,
                         g.G, c->stream) != cudaSuccess)
      return bail(HOTRG_ECUDA);
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(HOTRG_ECUDA);
  int herr = 0;
  if (cudaMemcpy(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bail(HOTRG_ECUDA);
  if (herr) return bail(HOTRG_ENONFINITE);
  *out = c;
  return HOTRG_OK;
}

// One step of every instance of group g (see the file comment).
hotrg_status step_group(hotrg_ctx *c, Group &g, hotrg_dir dir, int step) {
  cudaStream_t st = g.stream;
  Profiler &pf = g.prof;
  const int G = g.G;

  // ---- the step's view of the stored tensor T[x,x',y,y'] (shape dx,dx,dy,dy)
  const bool ydir = (dir == HOTRG_DIR_Y);
  const int D = ydir ? g.dx : g.dy;     // fused legs
  const int E = ydir ? g.dy : g.dx;     // contracted legs
  const long long cx = (long long)g.dx * g.dy * g.dy, cxp = (long long)g.dy * g.dy,
                  cy = g.dy, cyp = 1;
  const long long sx = ydir ? cx : cy, sxp = ydir ? cxp : cyp;
  const long long sy = ydir ? cy : cx, syp = ydir ? cyp : cxp;
  const int n = D * D;
  const int Dn = n < g.D_cut ? n : g.D_cut;
  const long long DE = (long long)D * E, E2 = (long long)E * E, D2 = (long long)D * D;
  double *rec = g.records + (size_t)step * kRecord;
  double *spec = g.spectra + (size_t)step * (g.D_cut + 1);
  const double fD = D, fE = E, fDn = Dn, fG = G;
  pf.flops(HOTRG_ST_ENV, fG * 4.0 * 2.0 * fD * fD * fD * fE * fE * fE);
  pf.flops(HOTRG_ST_GRAM, fG * 2.0 * 2.0 * fD * fD * fD * fD * fE * fE);
  pf.flops(HOTRG_ST_PROJ_P, fG * 2.0 * fDn * fD * fD * fD * fE * fE);
  pf.flops(HOTRG_ST_PROJ_Q, fG * 2.0 * fDn * fD * fD * fD * fE * fE * fE);
  pf.flops(HOTRG_ST_PROJ_T, fG * 2.0 * fDn * fDn * fD * fD * fE * fE);

  // ---- a2/a3: environments G_L, G_R ([x1][x2][u1][u2], FP64)
  // A step whose fused legs are trivial (D = 1: X steps after the y legs were
  // closed by a trace) multiplies Dx x Dx column matrices, E^3 flops: it runs
  // on the FP64 SIMT GEMMs in every precision mode.
  const bool tc = D > 1 &&
                  (c->prec == HOTRG_TF32 || c->prec == HOTRG_BF16X3 || c->prec == HOTRG_BF16X6);
  // FP64 partials and projection intermediates: the full-size buffers, or in
  // the tensor-core modes (D = 1 only) the small ones
  double *AL = g.AL, *BL = g.BL, *AR = g.AR, *BR = g.BR, *P = g.P, *Q = g.Q;
  long long sPart = g.sT, sPQ = g.sP;
  if (!AL) {
    const long long b = g.sC1 * G;
    AL = g.c1, BL = g.c1 + b, AR = g.c1 + 2 * b, BR = g.c1 + 3 * b, P = g.c1 + 4 * b,
    Q = g.c1 + 5 * b;
    sPart = sPQ = g.sC1;
  }
  // FP64 SIMT or exact-slice tensor-core GEMM over the same mapped operands
  auto mgemm = [&](const MappedGemm &mg) -> cudaError_t {
    if (c->prec == HOTRG_BF16XS && D > 1) return gemm_xs(mg, c->xs_digits, g.xw, c->err, st);
    return gemm_f64(mg, st);
  };
  // A tensor-core contraction segment (its launches depend only on the key):
  // run eagerly the first time (the GEMM autotuner times its shapes then),
  // captured into a CUDA graph the second time, replayed afterwards.  With the
  // stage profiler on, the stage events are recorded inside the graph (a
  // separate graph from the unprofiled one) and timed after each replay.
  auto run_segment = [&](int seg, const std::function<int(StageHook *)> &body) -> int {
    if (!c->use_graphs || st == nullptr) return body(&pf);
    const std::array<long long, 8> key{seg, (long long)dir, D, E, Dn,
                                       (long long)reinterpret_cast<uintptr_t>(g.T), pf.on ? 1 : 0,
                                       c->fuse_chain ? 1 : 0};
    auto it = g.graphs.find(key);
    if (it != g.graphs.end()) {
      for (int k = 0; k < HOTRG_NSTAGES; ++k)
        if (it->second.launches[k]) pf.launched(k, (int)it->second.launches[k]);
      const cudaError_t e = cudaGraphLaunch(it->second.exec, st);
      if (e == cudaSuccess) pf.replay(it->second.events);
      return (int)e;
    }
    if (g.nograph.count(key) || !g.seen.count(key)) {
      g.seen.insert(key);
      return body(&pf);
    }
    CaptureHook ch(&pf);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      g.nograph.insert(key);
      return body(&pf);
    }
    pf.begin_capture();
    const int r = body(&ch);
    std::vector<Profiler::Interval> evs = pf.end_capture();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    SegGraph sg;
    if (r || ec != cudaSuccess || !graph ||
        cudaGraphInstantiate(&sg.exec, graph, 0ULL) != cudaSuccess) {
      // not capturable here: nothing of the segment ran; run it eagerly from now on
      if (graph) cudaGraphDestroy(graph);
      for (auto &iv : evs) {
        cudaEventDestroy(iv.b);
        cudaEventDestroy(iv.e);
      }
      (void)cudaGetLastError();
      g.nograph.insert(key);
      return body(&pf);
    }
    cudaGraphDestroy(graph);
    std::copy(ch.per_stage, ch.per_stage + HOTRG_NSTAGES, sg.launches);
    sg.events = std::move(evs);
    SegGraph &slot = g.graphs[key];
    slot = std::move(sg);
    for (int k = 0; k < HOTRG_NSTAGES; ++k)
      if (slot.launches[k]) pf.launched(k, (int)slot.launches[k]);
    const cudaError_t e = cudaGraphLaunch(slot.exec, st);
    if (e == cudaSuccess) pf.replay(slot.events);
    return (int)e;
  };
  if (tc) {
    if (int r = run_segment(0, [&](StageHook *hook) {
          return g.tc.environment(g.T, g.sT, D, E, sx, sxp, sy, syp, g.GL, g.GR, g.sT, hook);
        }))
      return fail(c, HOTRG_ECUDA, std::string("tensor-core environment chain failed: ") +
                                      cudaGetErrorString(static_cast<cudaError_t>(r)));
  } else {
    // partials written as [x][u][k][k'] for the Gram combine
    const IdxMap out_m = map2(E, E, (long long)D * E2), out_n = map2(E, 1, E2);
    struct Part { double *dst; IdxMap row, red; };
    const Part parts[4] = {
        {AL, map2(E, syp, sx), map2(E, sy, sxp)},    // A_L[x1,k,u1,k']: sum over (x1', y)
        {BL, map2(E, sy, sx), map2(E, syp, sxp)},    // B_L[x2,k,u2,k']: sum over (x2', y')
        {AR, map2(E, syp, sxp), map2(E, sy, sx)},    // A_R[x1',k,u1',k']: sum over (x1, y)
        {BR, map2(E, sy, sxp), map2(E, syp, sx)},    // B_R[x2',k,u2',k']: sum over (x2, y')
    };
    pf.begin(HOTRG_ST_ENV);
    for (const Part &p : parts) {
      MappedGemm m{(int)DE, (int)DE, (int)DE, g.T, p.row, p.red, g.T, p.row, p.red, p.dst, out_m,
                   out_n, G, g.sT, g.sT, sPart};
      m.capA = m.capB = g.sT * G;
      m.capC = sPart * G;
      m.err = c->err;
      CK_CUDA(c, mgemm(m));
    }
    pf.launched(HOTRG_ST_ENV, 4);
    pf.end(HOTRG_ST_ENV);
    // G[x1,x2,u1,u2] = sum_{k,k'} A[x1,u1,k,k'] B[x2,u2,k,k']
    pf.begin(HOTRG_ST_GRAM);
    const IdxMap gm = map2(D, D, D2 * D), gn = map2(D, 1, D2);
    MappedGemm gl{(int)D2, (int)D2, (int)E2, AL, map1(E2), map1(1), BL, map1(E2), map1(1),
                  g.GL, gm, gn, G, sPart, sPart, g.sT};
    MappedGemm gr{(int)D2, (int)D2, (int)E2, AR, map1(E2), map1(1), BR, map1(E2), map1(1),
                  g.GR, gm, gn, G, sPart, sPart, g.sT};
    for (MappedGemm *q : {&gl, &gr}) {
      q->capA = q->capB = sPart * G;
      q->capC = g.sT * G;
      q->err = c->err;
    }
    CK_CUDA(c, mgemm(gl));
    CK_CUDA(c, mgemm(gr));
    pf.launched(HOTRG_ST_GRAM, 2);
  }
  // the tensor-core chain closed its own Gram stage (it may run as a graph)
  if (tc) pf.begin(HOTRG_ST_GRAM);
  // both sides at once (G_R follows G_L's G instances): traces to scal + 2 + side
  CK_CUDA(c, symmetrize_trace(g.GL, n, g.sT, g.scal + 2, kScal, 2 * G, st, G));
  pf.launched(HOTRG_ST_GRAM, 2);
  pf.end(HOTRG_ST_GRAM);

  // ---- a4: FP64 eigendecomposition and choice of U
  pf.begin(HOTRG_ST_EIG);
  int spec_n;
  int eig_path = 0, eig_iters = 0;
  double eig_res = 0.0;
  SiResult r{};
  if (n <= g.D_cut) {
    // nothing is cut (U = I); the spectrum of G_L is still recorded
    CK_CUDA(c, identity_isometry(g.U, n, g.sU, G, st));
    SiBatch sb{};
    sb.P = G;
    sb.n = n;
    sb.k = n;
    sb.m = jacobi_block(n);
    sb.G = pset_linear(g.GL, g.sT);
    long long nl = 0;
    CK_CUDA(c, jacobi_full(sb, g.si_work, st, &nl));
    const SiOut o = si_outputs(g.si_work, G, n, sb.m);
    CK_CUDA(c, spectrum_no_cut(o.theta, n, 1, g.scal + 2, kScal, rec, g.sRec, spec, g.sSpec, G, st));
    pf.launched(HOTRG_ST_EIG, 2 + (int)nl);
    spec_n = n;
  } else {
    // leading k = D'+1 eigenpairs of both environments of every instance
    const int k = Dn + 1;
    SiBatch sb{};
    sb.P = 2 * G;
    sb.n = n;
    sb.k = k;
    sb.G = pset_pairs(g.GL, g.GR, g.sT);
    long long nl = 0;
    bool ok = false;
    if (n + (n & 1) <= kSiMaxBlock) {
      sb.m = jacobi_block(n);
      CK_CUDA(c, jacobi_full(sb, g.si_work, st, &nl));
      eig_path = 1;
      ok = true;
    } else {
      // Rayleigh-Ritz block: 5k/4 rounded up to a multiple of 8 (m = 48 for the
      // k = 33 pairs of D' = 32).  A smaller block costs more iterations (the
      // error of the wanted pairs shrinks by theta_m / theta_k per iteration)
      // but each of its iterations, orthogonalisations and Jacobi solves is
      // cheaper; measured at D = 32: m = 72 (2k) 243, m = 48 277-284, m = 40
      // 230-237 RG-steps/s.
      int m = ((5 * k + 3) / 4 + 7) / 8 * 8;
      if (m > kSiMaxBlock) m = kSiMaxBlock;
      if (m > n) m = n & ~1;
      sb.m = m;
      sb.xs = c->eig_tc;
      sb.err = c->err;
      sb.trace = PSet{g.scal + 2, g.scal + 3, kScal};
      sb.has_trace = true;
      sb.shift_rel = 0x1.0p-40;
      // Environments built from reduced-precision products are accurate to
      // about the operands' unit roundoff u (TF32 2^-11, two-term BF16 ~2^-17):
      // eigenvalues below that level relative to the largest are noise, with
      // eigenvectors undetermined beyond it, so a residual that stalls there is
      // accepted (2 u; FP64-grade G: 1e-10).  The three-term split represents
      // its operands to 2^-24, below the FP32 accumulation error of its
      // products over K = Dy^2 terms (residuals measured to stall at 1.2e-7 at
      // D = 48): its floor is 8 x 2^-24.
      switch (c->prec) {
        case HOTRG_TF32: sb.floor_tol = 2.0 * 0x1.0p-11; break;
        case HOTRG_BF16X3: sb.floor_tol = 2.0 * 0x1.0p-17; break;
        case HOTRG_BF16X6: sb.floor_tol = 8.0 * 0x1.0p-24; break;
        default: sb.floor_tol = 0.0; break;
      }
      // the solve of the last step in this direction took iters_prev
      // iterations; a Rayleigh-Ritz step costs several iterations, so the
      // first one is scheduled just before that count -- one iteration
      // earlier still if that solve converged at its first check (so that the
      // schedule can find a shorter solve instead of repeating the last one)
      // -- but no later than iteration 24, after which a slow solve (a flat
      // noise tail) needs its checks to see the residual stall
      const int di = ydir ? 1 : 0;
      const int back = g.rr_prev[di] == 1 ? 2 : 1;
      sb.first_check = g.iters_prev[di] > 0 ? std::min(24, std::max(3, g.iters_prev[di] - back)) : 3;
      if (g.xprev_n[di] == n && g.xprev_m[di] == m) {
        // the last solve of this direction (same sizes) starts each side's
        // iteration from all of its Ritz vectors: the trailing columns start
        // close to the next eigenvectors instead of random
        sb.warm = pset_linear(g.Xprev[di], g.sXp);
        sb.has_warm = true;
        sb.kw = m;
      } else if (g.nprev[di] == n && g.kprev[di] <= m) {
        // the last isometry of this direction starts both sides' iteration
        sb.warm = pset_pairs(g.Uprev[di], g.Uprev[di], g.sUp);
        sb.has_warm = true;
        sb.kw = g.kprev[di];
      }
      CK_CUDA(c, si_solve(sb, g.si_work, 1e-12, c->eig_max_iters, st, &r, &nl));
      eig_path = 2;
      eig_iters = r.iterations;
      g.iters_prev[di] = r.converged ? r.iterations : 0;
      g.rr_prev[di] = r.rr;
      eig_res = r.residual;
      ok = r.converged;
      if (ok) {
        const SiOut o = si_outputs(g.si_work, 2 * G, n, m);
        CK_CUDA(c, cudaMemcpy2DAsync(g.Xprev[di], sizeof(double) * g.sXp, o.X.at(0),
                                     sizeof(double) * (o.X.at(1) - o.X.at(0)), sizeof(double) * (size_t)n * m,
                                     2 * G, cudaMemcpyDeviceToDevice, st));
        g.xprev_n[di] = n;
        g.xprev_m[di] = m;
      }
    }
    pf.launched(HOTRG_ST_EIG, (int)nl);
    if (!ok) {
      char why[256];
      snprintf(why, sizeof(why),
               "eigensolver stopped without reaching its residual bound: %d of at most %d subspace "
               "iterations, %d Rayleigh-Ritz steps, residual %.3e, breakdown %d (1 Cholesky, 2 Jacobi "
               "sweep limit), FP64 finishing Jacobi rounds %d, FP32 Jacobi sweeps %d",
               r.iterations, c->eig_max_iters, r.rr, eig_res, r.breakdown, r.sweeps64, r.sweeps32);
      return fail(c, HOTRG_EEIG, why);
    }
    {
      const SiOut o = si_outputs(g.si_work, 2 * G, n, sb.m);
      SelectArgs a{n, Dn, k, 1, o.theta, o.X, g.scal + 2, kScal, g.U, g.sU,
                   rec, g.sRec, spec, g.sSpec, G};
      CK_CUDA(c, select_isometry(a, st));
    }
    pf.launched(HOTRG_ST_EIG, 1);
    const int di = ydir ? 1 : 0;
    CK_CUDA(c, cudaMemcpy2DAsync(g.Uprev[di], sizeof(double) * g.sUp, g.U, sizeof(double) * g.sU,
                                 sizeof(double) * (size_t)n * Dn, G, cudaMemcpyDeviceToDevice, st));
    g.nprev[di] = n;
    g.kprev[di] = Dn;
    spec_n = k;
  }
  pf.end(HOTRG_ST_EIG);

  // ---- a5-a7: projection chain
  // output of the step in the stored layout: Y -> T'[a][b][y][y'], X -> T'[x][x'][a][b]
  const IdxMap tm = ydir ? map3(E, E, 1, E, (long long)Dn * E2)
                         : map3(E, E, (long long)Dn * Dn, (long long)E * Dn * Dn, Dn);
  const IdxMap tn = ydir ? map1(E2) : map1(1);
  if (tc) {
    if (int r = run_segment(1, [&](StageHook *hook) {
          return g.tc.project(g.T, g.sT, g.U, g.sU, D, E, Dn, sx, sxp, sy, syp, g.Tn, g.sT, tm, tn,
                              c->fuse_chain, hook);
        }))
      return fail(c, HOTRG_ECUDA, std::string("tensor-core projection chain failed: ") +
                                      cudaGetErrorString(static_cast<cudaError_t>(r)));
  } else {
    // a5: P[a][x1'][y][x2][k] = sum_x1 U[(x1 x2), a] T[x1,x1',y,k]
    pf.begin(HOTRG_ST_PROJ_P);
    MappedGemm g5{(int)(D * Dn), (int)(D * E2), D,
                  g.U, map2(Dn, n, 1), map1(D),
                  g.T, map3(E, E, syp, sy, sxp), map1(sx),
                  P, map2(Dn, D2 * E2, E), map3(E, E, 1, DE, DE * E),
                  G, g.sU, g.sT, sPQ};
    g5.capA = g.sU * G;
    g5.capB = g.sT * G;
    g5.capC = sPQ * G;
    g5.err = c->err;
    CK_CUDA(c, mgemm(g5));
    pf.launched(HOTRG_ST_PROJ_P, 1);
    pf.end(HOTRG_ST_PROJ_P);
    // a6: Q[a][y][y'][x1'][x2'] = sum_{x2,k} P[(a,x1',y),(x2,k)] T[x2,x2',k,y']
    pf.begin(HOTRG_ST_PROJ_Q);
    MappedGemm g6{(int)(Dn * DE), (int)DE, (int)DE,
                  P, map1(DE), map1(1),
                  g.T, map2(D, sxp, syp), map2(E, sy, sx),
                  Q, map3(E, D, E * D2, D, E2 * D2), map2(D, 1, D2),
                  G, sPQ, g.sT, sPQ};
    g6.capA = sPQ * G;
    g6.capB = g.sT * G;
    g6.capC = sPQ * G;
    g6.err = c->err;
    CK_CUDA(c, mgemm(g6));
    pf.launched(HOTRG_ST_PROJ_Q, 1);
    pf.end(HOTRG_ST_PROJ_Q);
    // a7: T'[(a,y,y'), b] = sum_{x1',x2'} Q[(a,y,y'),(x1',x2')] U[(x1' x2'), b]
    pf.begin(HOTRG_ST_PROJ_T);
    MappedGemm g7{(int)(Dn * E2), Dn, (int)D2,
                  Q, map1(D2), map1(1),
                  g.U, map1(n), map1(1),
                  g.Tn, tm, tn,
                  G, sPQ, g.sU, g.sT};
    g7.capA = sPQ * G;
    g7.capB = g.sU * G;
    g7.capC = g.sT * G;
    g7.err = c->err;
    CK_CUDA(c, mgemm(g7));
    pf.launched(HOTRG_ST_PROJ_T, 1);
    pf.end(HOTRG_ST_PROJ_T);
  }

  // ---- a8: rescale and FP64 log-sum
  pf.begin(HOTRG_ST_RESCALE);
  const long long count = (long long)Dn * Dn * E2;
  CK_CUDA(c, maxabs_scale_log(g.Tn, count, g.sT, g.scal + 1, kScal, g.scal, kScal,
                              ldexp(1.0, -(step + 1)), rec + 5, g.sRec, c->err, G, st));
  pf.launched(HOTRG_ST_RESCALE, 3);
  pf.end(HOTRG_ST_RESCALE);
  std::swap(g.T, g.Tn);
  if (ydir) g.dx = Dn; else g.dy = Dn;
  GroupStep gs{};
  gs.info.dir = dir;
  gs.info.Dx = D;
  gs.info.Dy = E;
  gs.info.Dn = Dn;
  gs.info.eig_path = eig_path;
  gs.info.eig_iters = eig_iters;
  gs.info.eig_residual = eig_res;
  gs.info.eig_rr = r.rr;
  gs.info.eig_sweeps = r.sweeps64;
  gs.info.eig_sweeps32 = r.sweeps32;
  gs.spec_count = spec_n;
  gs.n = n;
  gs.dn = Dn;
  g.steps.push_back(gs);
  return HOTRG_OK;
}

hotrg_status locate(hotrg_ctx *c, int inst, Group **g, int *j) {
  if (!c || inst < 0 || inst >= c->n_inst) return HOTRG_EINVAL;
  *g = c->groups[c->where[inst].first].get();
  *j = c->where[inst].second;
  return HOTRG_OK;
}

hotrg_status step_info_of(hotrg_ctx *c, int inst, int step, hotrg_step_info_t *out) {
  Group *g;
  int j;
  if (!out || locate(c, inst, &g, &j)) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (step < 0 || step >= c->nsteps) return HOTRG_EINVAL;
  double r[kRecord];
  CK_CUDA(c, cudaMemcpyAsync(r, g->records + j * g->sRec + (size_t)step * kRecord, sizeof(r),
                             cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = g->steps[step].info;
  out->side = (int)r[0];
  out->eps_L = r[1];
  out->eps_R = r[2];
  out->cut_gap = r[3];
  out->trace_G = r[4];
  out->ln_c = r[5];
  return HOTRG_OK;
}

hotrg_status get_tensor_of(hotrg_ctx *c, int inst, double *host_out, long long cap, int dims[4]) {
  Group *g;
  int j;
  if (!dims || locate(c, inst, &g, &j)) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  dims[0] = dims[1] = g->dx;
  dims[2] = dims[3] = g->dy;
  const long long cnt = (long long)g->dx * g->dx * g->dy * g->dy;
  if (!host_out || cap < cnt) return HOTRG_EINVAL;
  CK_CUDA(c, cudaMemcpyAsync(host_out, g->T + j * g->sT, sizeof(double) * cnt,
                             cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
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
    case HOTRG_EBOUNDS: return "HOTRG_EBOUNDS";
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

hotrg_status hotrg_xxz_tensor(double Jxy, double Jz, double tau, double *T0_out) {
  if (!T0_out || !(tau > 0.0) || !isfinite(tau) || !isfinite(Jxy) || !isfinite(Jz))
    return HOTRG_EINVAL;
  double gf[16];
  xxz_gate(Jxy, Jz, tau, gf);
  const double p = gf[0], u = gf[5], v = gf[6];
  double g[4][4] = {{p, 0, 0, 0}, {0, u, v, 0}, {0, v, u, 0}, {0, 0, 0, p}};
  // g = a I(x)I + b (X(x)X + Y(x)Y) + d Z(x)Z with Y(x)Y = -E(x)E, E = [[0,1],[-1,0]]:
  // diagonal a + d = p, a - d = u; off-diagonal 2 b = v
  const double coef[4] = {0.5 * (p + u), 0.5 * v, -0.5 * v, 0.5 * (p - u)};
  static const double basis[4][2][2] = {
      {{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, 1}, {-1, 0}}, {{1, 0}, {0, -1}}};
  double A[4][2][2], B[4][2][2];
  for (int k = 0; k < 4; ++k) {
    const double r = sqrt(fabs(coef[k])), sg = coef[k] < 0.0 ? -r : r;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        A[k][i][j] = r * basis[k][i][j];
        B[k][i][j] = sg * basis[k][i][j];
      }
  }
  // T[x][x'][(e0 o0)][(e2 o2)] = sum_{e1,o1} g[(e1 o1)][(e0 o0)] B_x[e2][e1] A_x'[o2][o1]
  for (int x = 0; x < 4; ++x)
    for (int xp = 0; xp < 4; ++xp)
      for (int y = 0; y < 4; ++y)
        for (int yp = 0; yp < 4; ++yp) {
          const int e0 = y >> 1, o0 = y & 1, e2 = yp >> 1, o2 = yp & 1;
          double acc = 0.0;
          for (int e1 = 0; e1 < 2; ++e1)
            for (int o1 = 0; o1 < 2; ++o1)
              acc += g[2 * e1 + o1][2 * e0 + o0] * B[x][e2][e1] * A[xp][o2][o1];
          T0_out[((x * 4 + xp) * 4 + y) * 4 + yp] = acc;
        }
  return HOTRG_OK;
}

void hotrg_destroy(hotrg_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto &g : c->groups)
    if (g->own_stream && g->stream) cudaStreamSynchronize(g->stream);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

hotrg_status hotrg_create(const double *T0, int D0, int D_cut, hotrg_prec prec, void *stream,
                          hotrg_ctx **out) {
  return create_ctx(1, &T0, &D0, &D_cut, prec, stream, out);
}

hotrg_status hotrg_batch_create(int n, const double *const *T0s, const int *D0s, const int *Dcuts,
                                hotrg_prec prec, void *stream, hotrg_ctx **out) {
  return create_ctx(n, T0s, D0s, Dcuts, prec, stream, out);
}

hotrg_status hotrg_step(hotrg_ctx *c, hotrg_dir dir) {
  if (!c) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (dir != HOTRG_DIR_X && dir != HOTRG_DIR_Y) return HOTRG_EINVAL;
  if (c->nsteps >= kMaxSteps) return fail(c, HOTRG_ESTATE, "step limit reached");
  if (c->groups.size() == 1) {
    if (hotrg_status s = step_group(c, *c->groups[0], dir, c->nsteps)) return s;
    // one synchronisation per step: device errors of this step surface here
    CK_CUDA(c, cudaStreamSynchronize(c->stream));
  } else {
    // The cut groups of a batch step concurrently: each on its own host thread
    // and stream (their eigensolvers are latency-bound chains that leave most
    // SMs idle), ordered after the work already on the context's stream.
    cudaEvent_t start = nullptr;
    CK_CUDA(c, cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    CK_CUDA(c, cudaEventRecord(start, c->stream));
    for (auto &g : c->groups) CK_CUDA(c, cudaStreamWaitEvent(g->stream, start, 0));
    std::vector<hotrg_status> st(c->groups.size(), HOTRG_OK);
    std::vector<std::thread> th;
    th.reserve(c->groups.size());
    const int step = c->nsteps;
    for (size_t i = 0; i < c->groups.size(); ++i)
      th.emplace_back([c, &st, i, dir, step] { st[i] = step_group(c, *c->groups[i], dir, step); });
    for (auto &t : th) t.join();
    cudaEventDestroy(start);
    for (auto &g : c->groups) CK_CUDA(c, cudaStreamSynchronize(g->stream));
    for (hotrg_status s : st)
      if (s != HOTRG_OK) return c->status != HOTRG_OK ? c->status : s;
  }
  for (auto &g : c->groups) g->prof.collect(false);
  if (hotrg_status fs = check_flag(c)) return fs;
  if (c->prof_on) c->prof_steps += 1;
  c->nsteps += 1;
  return HOTRG_OK;
}

hotrg_status hotrg_batch_step(hotrg_ctx *c, hotrg_dir dir) { return hotrg_step(c, dir); }

hotrg_status hotrg_trace_y(hotrg_ctx *c) {
  if (!c) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  const double w = ldexp(1.0, -c->nsteps);
  for (auto &gp : c->groups) {
    Group &g = *gp;
    CK_CUDA(c, trace_y(g.T, g.Tn, g.dx, g.dy, g.sT, g.G, c->stream));
    CK_CUDA(c, maxabs_scale_log(g.Tn, (long long)g.dx * g.dx, g.sT, g.scal + 1, kScal, g.scal,
                                kScal, w, g.scal + 5, kScal, c->err, g.G, c->stream));
    std::swap(g.T, g.Tn);
    g.dy = 1;
  }
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_flag(c);
}

hotrg_status hotrg_set_option(hotrg_ctx *c, int option, int value) {
  if (!c) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  switch (option) {
    case HOTRG_OPT_EIG_TC_PRODUCTS:
      if (value != 0 && value != 1) return HOTRG_EINVAL;
      c->eig_tc = value != 0;
      return HOTRG_OK;
    case HOTRG_OPT_XS_DIGITS:
      if (value < 4 || value > kXsDigitsMax) return HOTRG_EINVAL;
      c->xs_digits = value;
      return HOTRG_OK;
    case HOTRG_OPT_GEMM_AUTOTUNE:
      if (value != 0 && value != 1) return HOTRG_EINVAL;
      tc_set_autotune(value != 0);
      return HOTRG_OK;
    case HOTRG_OPT_GRAPHS:
      if (value != 0 && value != 1) return HOTRG_EINVAL;
      c->use_graphs = value != 0;
      return HOTRG_OK;
    case HOTRG_OPT_EIG_MAX_ITERS:
      if (value < 1 || value > 1000) return HOTRG_EINVAL;
      c->eig_max_iters = value;
      return HOTRG_OK;
    case HOTRG_OPT_WAIT_CYCLES:
      if (value < 1) return HOTRG_EINVAL;
      tc::set_wait_limit(value);
      return HOTRG_OK;
    case HOTRG_OPT_TEST_STALL:
      if (value != 1 && value != 2) return HOTRG_EINVAL;
      tc::arm_stall(value == 1 ? tc::kStallGemm : tc::kStallChain);
      return HOTRG_OK;
    case HOTRG_OPT_FUSED_CHAIN:
      if (value != 0 && value != 1) return HOTRG_EINVAL;
      c->fuse_chain = value != 0;
      return HOTRG_OK;
  }
  return HOTRG_EINVAL;
}

hotrg_status hotrg_batch_size(hotrg_ctx *c, int *n) {
  if (!c || !n) return HOTRG_EINVAL;
  *n = c->n_inst;
  return HOTRG_OK;
}

hotrg_status hotrg_profile_enable(hotrg_ctx *c, int enable) {
  if (!c) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  for (auto &g : c->groups) {
    CK_CUDA(c, cudaStreamSynchronize(g->stream));
    g->prof.reset();
    g->prof.on = enable != 0;
  }
  c->prof_on = enable != 0;
  c->prof_steps = 0;
  return HOTRG_OK;
}

hotrg_status hotrg_profile_read(hotrg_ctx *c, hotrg_profile_t *out) {
  if (!c || !out) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  hotrg_profile_t sum{};
  for (auto &g : c->groups) {
    CK_CUDA(c, cudaStreamSynchronize(g->stream));
    g->prof.collect(true);
    const hotrg_profile_t &a = g->prof.acc;
    sum.launches += a.launches;
    for (int k = 0; k < HOTRG_NSTAGES; ++k) {
      sum.stage_launches[k] += a.stage_launches[k];
      sum.ms[k] += a.ms[k];
      sum.flops[k] += a.flops[k];
    }
  }
  sum.steps = c->prof_steps;
  *out = sum;
  return HOTRG_OK;
}

hotrg_status hotrg_batch_log_z(hotrg_ctx *c, double *out_n) {
  if (!c || !out_n) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  std::vector<std::vector<double>> h(c->groups.size());
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    Group &g = *c->groups[gi];
    CK_CUDA(c, periodic_trace(g.T, g.dx, g.dy, g.sT, g.scal + 4, kScal, g.G, c->stream));
    h[gi].resize((size_t)kScal * g.G);
    CK_CUDA(c, cudaMemcpyAsync(h[gi].data(), g.scal, sizeof(double) * kScal * g.G,
                               cudaMemcpyDeviceToHost, c->stream));
  }
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  if (hotrg_status fs = check_flag(c)) return fs;
  const double w = ldexp(1.0, -c->nsteps);
  for (int i = 0; i < c->n_inst; ++i) {
    const double *s = h[c->where[i].first].data() + (size_t)kScal * c->where[i].second;
    if (!(s[4] > 0.0) || !isfinite(s[4]))
      return fail(c, HOTRG_ENONFINITE,
                  "periodic trace of instance " + std::to_string(i) + " is not positive");
    out_n[i] = s[0] + log(s[4]) * w;
  }
  return HOTRG_OK;
}

hotrg_status hotrg_log_z_per_site(hotrg_ctx *c, double *out) {
  if (!c || !out) return HOTRG_EINVAL;
  if (c->n_inst != 1) return HOTRG_ESTATE;
  return hotrg_batch_log_z(c, out);
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
  return step_info_of(c, 0, step, out);
}

hotrg_status hotrg_batch_step_info(hotrg_ctx *c, int inst, int step, hotrg_step_info_t *out) {
  return step_info_of(c, inst, step, out);
}

hotrg_status hotrg_spectrum(hotrg_ctx *c, int step, double *buf, int cap, int *n) {
  if (!c || !n || (cap > 0 && !buf)) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (step < 0 || step >= c->nsteps) return HOTRG_EINVAL;
  const Group &g = *c->groups[c->where[0].first];
  const int j = c->where[0].second;
  const int cnt = g.steps[step].spec_count;
  *n = cnt;
  const int k = cnt < cap ? cnt : cap;
  if (k > 0) {
    CK_CUDA(c, cudaMemcpyAsync(buf, g.spectra + j * g.sSpec + (size_t)step * (g.D_cut + 1),
                               sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
    CK_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return HOTRG_OK;
}

hotrg_status hotrg_get_tensor(hotrg_ctx *c, double *host_out, long long cap, int dims[4]) {
  return get_tensor_of(c, 0, host_out, cap, dims);
}

hotrg_status hotrg_batch_get_tensor(hotrg_ctx *c, int inst, double *host_out, long long cap,
                                    int dims[4]) {
  return get_tensor_of(c, inst, host_out, cap, dims);
}

hotrg_status hotrg_get_isometry(hotrg_ctx *c, double *host_out, long long cap, int *rows, int *cols) {
  if (!c || !rows || !cols) return HOTRG_EINVAL;
  if (c->status != HOTRG_OK) return c->status;
  if (c->nsteps == 0) return HOTRG_ESTATE;
  const Group &g = *c->groups[c->where[0].first];
  const int j = c->where[0].second;
  *rows = g.steps.back().n;
  *cols = g.steps.back().dn;
  const long long cnt = (long long)*rows * *cols;
  if (!host_out || cap < cnt) return HOTRG_EINVAL;
  CK_CUDA(c, cudaMemcpyAsync(host_out, g.U + j * g.sU, sizeof(double) * cnt,
                             cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOTRG_OK;
}

hotrg_status hotrg_dims(hotrg_ctx *c, int *Dx, int *Dy, int *nsteps) {
  if (!c || !Dx || !Dy || !nsteps) return HOTRG_EINVAL;
  const Group &g = *c->groups[c->where[0].first];
  *Dx = g.dx;
  *Dy = g.dy;
  *nsteps = c->nsteps;
  return HOTRG_OK;
}

}  // extern "C"
