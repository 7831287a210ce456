// Fused a6 -> a7 projection (TF32, tcgen05): T'[(a,y,y')][b] from P, the a6
// view of T and U without writing Q to global memory.  Shapes: D = E in {16,
// 32}, D' <= 32 (the steady state of the D_cut = 16 and 32 runs); other shapes
// use the unfused chain.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hotrg {

struct ChainArgs {
  int D, E, Dn, batch;
  const float *P;      // rows (a, y, x1') (x1' fastest), K = (x2, k); pitch pitchP, stride sP
  int pitchP;
  long long sP;
  const float *T6;     // rows (y', x2') (x2' fastest), K = (x2, k)
  int pitchT;
  long long sT6;
  const float *U7;     // rows b < D', K = (x2', x1') (x1' fastest): U[(x1' D + x2'), b]
  int pitchU;
  long long sU7;
  double *Tout;        // T'(m = (a, y, y'), b) at Tout + i sTout + tm(m) + tn(b)
  long long sTout;
  IdxMap tm, tn;
  long long cap;       // elements of Tout (all instances) for the checked build, 0 = unknown
  int *err;            // device flag: 2 if a bounded wait runs out, 3 on a bounds violation
};

bool tc_chain_supported(int D, int E, int Dn);
cudaError_t tc_chain(const ChainArgs &a, cudaStream_t s);

}  // namespace hotrg
