// Tensor-core (tcgen05) path of the step's contractions: TF32 or split-BF16
// operands, FP32 accumulation in TMEM.  The eigendecomposition, rescale and
// log-sum stay FP64 and live in the step driver.  Every call works on a batch
// of G instances whose FP64 inputs and outputs lie at fixed instance strides.
#pragma once

#include <cuda_runtime.h>

#include "../../include/hotrg.h"
#include "common.cuh"

namespace hotrg {

class TcPath {
 public:
  ~TcPath();
  // 0 on success, 1 CUDA error, 2 allocation failure.  err_flag (device int)
  // receives 2 if a kernel's bounded wait runs out.
  int init(hotrg_prec prec, int D0, int D_cut, int G, cudaStream_t s, int *err_flag);
  // Both chains return 0 or the CUDA error of the failing call.
  // a2 + a3: environments G_L, G_R (FP64, [x1,x2,u1,u2], instance stride sG) of a
  // Y step on the strided view (sx, sxp, sy, syp) of T (instance stride sT) with
  // fused dim D and contracted dim E.
  int environment(const double *T, long long sT, int D, int E, long long sx, long long sxp,
                  long long sy, long long syp, double *GL, double *GR, long long sG,
                  StageHook *hook);
  // a5 - a7: T'(m, b) = [U^T (T.T) U], written in FP64 through the maps (tm, tn)
  // at Tout + i * sTout.  fuse: a6 and a7 as one kernel (Q kept on chip) where
  // tc_chain_supported(D, E, Dn) and the mode is TF32.
  int project(const double *T, long long sT, const double *U, long long sU, int D, int E, int Dn,
              long long sx, long long sxp, long long sy, long long syp, double *Tout,
              long long sTout, IdxMap tm, IdxMap tn, bool fuse, StageHook *hook);

  struct Impl;

 private:
  Impl *impl_ = nullptr;
};

}  // namespace hotrg
