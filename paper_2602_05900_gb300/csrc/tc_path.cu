// Tensor-core chain of the HOTRG step's contractions (TF32 / split BF16).
//
// Operands of every GEMM are dense K-major planes (TMA needs a unit-stride
// K axis), so the step first gathers the permuted views of T and U it needs
// into such planes (a1: small, D^4 elements each).  The GEMMs whose result
// feeds the next GEMM (environment partials -> Gram combine, P -> Q, Q -> T')
// write that result straight into the next GEMM's operand format through
// their epilogue maps, so no D^5 tensor is ever permuted or converted in a
// separate pass.
#include <cuda_bf16.h>

#include "tc_chain.cuh"
#include "tc_gemm.cuh"
#include "tc_path.cuh"

namespace hotrg {

struct TcPath::Impl {
  TcMode mode = TcMode::TF32;
  cudaStream_t s = nullptr;
  int planes = 1, eb = 4;
  int G = 1;                       // instances
  long long sTop = 0, sPop = 0;    // elements between instances: operand buffers, P / Q
  // a2 operands (permuted views of T) and a2 outputs / a3 operands ([x][u] x
  // [k][k']): four per instance, interleaved as q = (side G + g) 2 + j for
  // view i = 2 side + j of instance g, so that a2 is one batched GEMM over
  // all q and a3 one over (side, g) with A at q = 2 (side G + g), B at q + 1
  void *opT = nullptr, *part = nullptr;
  void *opU5 = nullptr, *opT5 = nullptr, *opT6 = nullptr, *opU7 = nullptr;
  void *P = nullptr, *Q = nullptr;
  int *err = nullptr;
  std::size_t capT = 0, capP = 0;  // elements per plane
  ~Impl() {
    cudaFree(opT);
    cudaFree(part);
    cudaFree(opU5);
    cudaFree(opT5);
    cudaFree(opT6);
    cudaFree(opU7);
    cudaFree(P);
    cudaFree(Q);
  }
};

namespace {

__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return __uint_as_float(u);
}

// dst[p][r][k] (pitch columns, zero beyond K) = split_p(src[rm(r) + km(k)])
template <int MODE>
__global__ void k_gather(const double *src, long long sSrc, int R, int K, int pitch, IdxMap rm,
                         IdxMap km, void *dst, long long sDst, long long plane_stride,
                         long long src_cap, int *err) {
  const long long zs = blockIdx.y * sSrc;
  src += zs;
  dst = static_cast<char *>(dst) + blockIdx.y * sDst * (MODE == 0 ? 4 : 2);
  const long long total = (long long)R * pitch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / pitch), k = (int)(e % pitch);
    const long long so = (k < K) ? map_off(rm, r) + map_off(km, k) : 0;
    const double v = (k < K && checked_ok(zs + so, src_cap, err)) ? src[so] : 0.0;
    if constexpr (MODE == 0) {
      static_cast<float *>(dst)[e] = tf32_rna(static_cast<float>(v));
    } else {
      constexpr int NP = MODE == 1 ? 2 : 3;
      __nv_bfloat16 *d = static_cast<__nv_bfloat16 *>(dst);
      double rem = v;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const __nv_bfloat16 t = __double2bfloat16(rem);
        d[e + p * plane_stride] = t;
        rem -= static_cast<double>(__bfloat162float(t));
      }
    }
  }
}

int grid_for(long long count, int batch) {
  long long b = (count + 255) / 256;
  const long long cap = (152LL * 8 + batch - 1) / batch;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

void *alloc(std::size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, bytes + 256) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}

}  // namespace

TcPath::~TcPath() { delete impl_; }

int TcPath::init(hotrg_prec prec, int D0, int D_cut, int G, cudaStream_t s, int *err_flag) {
  impl_ = new Impl();
  Impl &I = *impl_;
  I.mode = prec == HOTRG_TF32 ? TcMode::TF32 : (prec == HOTRG_BF16X3 ? TcMode::BF16X3 : TcMode::BF16X6);
  I.s = s;
  I.G = G;
  I.planes = tc_planes(I.mode);
  I.eb = tc_elem_bytes(I.mode);
  const long long Dm = D0 > D_cut ? D0 : D_cut;
  // Per-plane capacities.  Rows are padded to a 16-byte pitch (at most 7 extra
  // elements): the largest operand is the a5 view of T, D E^2 rows of pitch(D)
  // <= Dm^3 (Dm + 8) elements, and every D^5 intermediate fits D_cut Dm^2 (Dm^2 + 8).
  I.capT = (std::size_t)(Dm * Dm * Dm * (Dm + 8));
  I.capP = (std::size_t)(D_cut * Dm * Dm * (Dm * Dm + 8));
  // instance strides: all planes of an instance, rounded to 64 elements (TMA strides)
  I.sTop = ((long long)I.capT * I.planes + 63) / 64 * 64;
  I.sPop = ((long long)I.capP * I.planes + 63) / 64 * 64;
  const std::size_t bt = (std::size_t)I.sTop * G * I.eb, bp = (std::size_t)I.sPop * G * I.eb;
  if (!(I.opT = alloc(4 * bt)) || !(I.part = alloc(4 * bt))) return 2;
  if (!(I.opU5 = alloc(bt)) || !(I.opT5 = alloc(bt)) || !(I.opT6 = alloc(bt)) ||
      !(I.opU7 = alloc(bt)) || !(I.P = alloc(bp)) || !(I.Q = alloc(bp)))
    return 2;
  I.err = err_flag;
  return 0;
}

// dst: instance g's plane at dst + g sDst elements (default: the operand stride)
static cudaError_t gather(const TcPath::Impl &I, const double *src, long long sSrc, int R, int K,
                          int pitch, IdxMap rm, IdxMap km, void *dst, long long sDst = -1) {
  const long long ps = (long long)R * pitch;
  const dim3 g(grid_for(ps, I.G), I.G);
  const long long cap = sSrc * I.G;
  if (sDst < 0) sDst = I.sTop;
  switch (I.mode) {
    case TcMode::TF32: k_gather<0><<<g, 256, 0, I.s>>>(src, sSrc, R, K, pitch, rm, km, dst, sDst, ps, cap, I.err); break;
    case TcMode::BF16X3: k_gather<1><<<g, 256, 0, I.s>>>(src, sSrc, R, K, pitch, rm, km, dst, sDst, ps, cap, I.err); break;
    case TcMode::BF16X6: k_gather<2><<<g, 256, 0, I.s>>>(src, sSrc, R, K, pitch, rm, km, dst, sDst, ps, cap, I.err); break;
  }
  return cudaGetLastError();
}

// an operand of `count` instances (default: the context's batch) bstride apart
static TcOperand operand(const TcPath::Impl &I, const void *base, int rows, int K, int pitch,
                         long long bstride, int count = 0) {
  return TcOperand{base, rows, K, pitch, count > 0 ? count : I.G, bstride};
}

// Epilogue writing an operand-format result (next GEMM's A or B planes) for
// `count` instances (default: the context's batch).
static TcEpilogue operand_epilogue(const TcPath::Impl &I, void *dst, long long plane_stride,
                                   IdxMap cm, IdxMap cn, long long bstride, int count = 0) {
  TcEpilogue e{};
  if (I.mode == TcMode::TF32) {
    e.kind = OutKind::F32;
    e.round_tf32 = true;
  } else {
    e.kind = OutKind::BF16P;
    e.planes = I.planes;
  }
  e.C = dst;
  e.plane_stride = plane_stride;
  e.cm = cm;
  e.cn = cn;
  e.bstride = bstride;
  e.cap = bstride * (count > 0 ? count : I.G);
  return e;
}

static TcEpilogue f64_epilogue(const TcPath::Impl &I, double *dst, IdxMap cm, IdxMap cn,
                               long long bstride, int count = 0) {
  TcEpilogue e{};
  e.kind = OutKind::F64;
  e.C = dst;
  e.planes = 1;
  e.cm = cm;
  e.cn = cn;
  e.bstride = bstride;
  e.cap = bstride * (count > 0 ? count : I.G);
  return e;
}

int TcPath::environment(const double *T, long long sT, int D, int E, long long sx, long long sxp,
                        long long sy, long long syp, double *GL, double *GR, long long sG,
                        StageHook *hook) {
  Impl &I = *impl_;
  const int DE = D * E, E2 = E * E, D2 = D * D;
  const int p2 = tc_pitch(DE, I.mode);   // a2 operand pitch
  const int p3 = tc_pitch(E2, I.mode);   // a3 operand pitch
  if ((std::size_t)DE * p2 > I.capT || (std::size_t)D2 * p3 > I.capT) return cudaErrorInvalidValue;
  const IdxMap rows[4] = {map2(E, syp, sx), map2(E, sy, sx), map2(E, syp, sxp), map2(E, sy, sxp)};
  const IdxMap reds[4] = {map2(E, sy, sxp), map2(E, syp, sxp), map2(E, sy, sx), map2(E, syp, sx)};
  const int G = I.G;
  const std::size_t eb = (std::size_t)I.eb;
  auto q_base = [&](void *base, int i) {       // view i of instance 0; instances 2 sTop apart
    return static_cast<char *>(base) + ((std::size_t)(i / 2) * G * 2 + (i % 2)) * I.sTop * eb;
  };
  hook->begin(HOTRG_ST_PREP);
  for (int i = 0; i < 4; ++i)
    if (cudaError_t e_ = gather(I, T, sT, DE, DE, p2, rows[i], reds[i], q_base(I.opT, i), 2 * I.sTop))
      return e_;
  hook->launched(HOTRG_ST_PREP, 4);
  hook->end(HOTRG_ST_PREP);
  // a2, one GEMM over the 4 G views: part_q[(x,u)][(k,k')], rows m = (x, k),
  // cols n = (u, k')
  hook->begin(HOTRG_ST_ENV);
  {
    TcOperand op = operand(I, I.opT, DE, DE, p2, I.sTop, 4 * G);
    TcEpilogue ep = operand_epilogue(I, I.part, (long long)D2 * p3, map2(E, E, (long long)D * p3),
                                     map2(E, 1, p3), I.sTop, 4 * G);
    if (cudaError_t e_ = tc_gemm(I.mode, op, op, DE, DE, DE, ep, I.err, I.s)) return e_;
  }
  hook->launched(HOTRG_ST_ENV, 1);
  hook->end(HOTRG_ST_ENV);
  // a3: G_side = part_(2 side) . part_(2 side + 1)^T, one GEMM over (side, g)
  // when the caller's G_R follows G_L's G instances, else one per side
  hook->begin(HOTRG_ST_GRAM);
  const IdxMap gm = map2(D, D, (long long)D2 * D), gn = map2(D, 1, D2);
  if (GR == GL + (std::size_t)G * sG) {
    TcOperand a = operand(I, I.part, D2, E2, p3, 2 * I.sTop, 2 * G);
    TcOperand b = operand(I, static_cast<char *>(I.part) + I.sTop * eb, D2, E2, p3, 2 * I.sTop, 2 * G);
    if (cudaError_t e_ = tc_gemm(I.mode, a, b, D2, D2, E2, f64_epilogue(I, GL, gm, gn, sG, 2 * G), I.err, I.s))
      return e_;
    hook->launched(HOTRG_ST_GRAM, 1);
  } else {
    for (int side = 0; side < 2; ++side) {
      TcOperand a = operand(I, q_base(I.part, 2 * side), D2, E2, p3, 2 * I.sTop);
      TcOperand b = operand(I, q_base(I.part, 2 * side + 1), D2, E2, p3, 2 * I.sTop);
      if (cudaError_t e_ = tc_gemm(I.mode, a, b, D2, D2, E2, f64_epilogue(I, side ? GR : GL, gm, gn, sG),
                                   I.err, I.s))
        return e_;
    }
    hook->launched(HOTRG_ST_GRAM, 2);
  }
  hook->end(HOTRG_ST_GRAM);
  return 0;
}

int TcPath::project(const double *T, long long sT, const double *U, long long sU, int D, int E,
                    int Dn, long long sx, long long sxp, long long sy, long long syp, double *Tout,
                    long long sTout, IdxMap tm, IdxMap tn, bool fuse, StageHook *hook) {
  Impl &I = *impl_;
  fuse = fuse && I.mode == TcMode::TF32 && tc_chain_supported(D, E, Dn);
  const int n = D * D, DE = D * E, E2 = E * E;
  const int p5 = tc_pitch(D, I.mode), p6 = tc_pitch(DE, I.mode), p7 = tc_pitch(n, I.mode);
  if ((std::size_t)D * Dn * p5 > I.capT || (std::size_t)D * E2 * p5 > I.capT ||
      (std::size_t)DE * p6 > I.capT || (std::size_t)Dn * p7 > I.capT ||
      (std::size_t)Dn * DE * p6 > I.capP || (std::size_t)Dn * E2 * p7 > I.capP)
    return cudaErrorInvalidValue;
  // a1: operands of a5 (U and T views with the x1 axis as K), a6 (T view) and a7 (U^T;
  // the fused kernel reads its K axis (x1', x2') in the order x2', x1')
  hook->begin(HOTRG_ST_PREP);
  if (cudaError_t e_ = gather(I, U, sU, D * Dn, D, p5, map2(Dn, n, 1), map1(D), I.opU5)) return e_;
  if (cudaError_t e_ = gather(I, T, sT, D * E2, D, p5, map3(E, E, syp, sy, sxp), map1(sx), I.opT5))
    return e_;
  if (cudaError_t e_ = gather(I, T, sT, DE, DE, p6, map2(D, sxp, syp), map2(E, sy, sx), I.opT6))
    return e_;
  if (cudaError_t e_ = gather(I, U, sU, Dn, n, p7, map1(n), fuse ? map2(D, D, 1) : map1(1), I.opU7))
    return e_;
  hook->launched(HOTRG_ST_PREP, 4);
  hook->end(HOTRG_ST_PREP);

  // a5: P[(a,x1',y)][(x2,k)] = sum_x1 U[(x1 x2),a] T[x1,x1',y,k]; rows m = (x2,a), cols (x1',y,k).
  // The fused kernel wants P's rows in the order (a, y, x1').
  hook->begin(HOTRG_ST_PROJ_P);
  {
    TcOperand a = operand(I, I.opU5, D * Dn, D, p5, I.sTop), b = operand(I, I.opT5, D * E2, D, p5, I.sTop);
    const long long ps = (long long)Dn * DE * p6;
    const IdxMap pn = fuse ? map3(E, E, 1, (long long)D * p6, p6) : map3(E, E, 1, p6, (long long)E * p6);
    TcEpilogue ep = operand_epilogue(I, I.P, ps, map2(Dn, (long long)DE * p6, E), pn, I.sPop);
    if (cudaError_t e_ = tc_gemm(I.mode, a, b, D * Dn, D * E2, D, ep, I.err, I.s)) return e_;
  }
  hook->launched(HOTRG_ST_PROJ_P, 1);
  hook->end(HOTRG_ST_PROJ_P);
  if (fuse) {
    // a6 + a7 in one kernel (its time is reported under the a6 stage)
    hook->begin(HOTRG_ST_PROJ_Q);
    ChainArgs ca{};
    ca.D = D;
    ca.E = E;
    ca.Dn = Dn;
    ca.batch = I.G;
    ca.P = static_cast<const float *>(I.P);
    ca.pitchP = p6;
    ca.sP = I.sPop;
    ca.T6 = static_cast<const float *>(I.opT6);
    ca.pitchT = p6;
    ca.sT6 = I.sTop;
    ca.U7 = static_cast<const float *>(I.opU7);
    ca.pitchU = p7;
    ca.sU7 = I.sTop;
    ca.Tout = Tout;
    ca.sTout = sTout;
    ca.tm = tm;
    ca.tn = tn;
    ca.cap = sTout * I.G;
    ca.err = I.err;
    if (cudaError_t e_ = tc_chain(ca, I.s)) return e_;
    hook->launched(HOTRG_ST_PROJ_Q, 1);
    hook->end(HOTRG_ST_PROJ_Q);
    hook->begin(HOTRG_ST_PROJ_T);
    hook->end(HOTRG_ST_PROJ_T);
    return 0;
  }
  // a6: Q[(a,y,y')][(x1',x2')] = sum_{x2,k} P[(a,x1',y),(x2,k)] T[x2,x2',k,y']
  hook->begin(HOTRG_ST_PROJ_Q);
  {
    TcOperand a = operand(I, I.P, Dn * DE, DE, p6, I.sPop), b = operand(I, I.opT6, DE, DE, p6, I.sTop);
    const long long ps = (long long)Dn * E2 * p7;
    TcEpilogue ep = operand_epilogue(I, I.Q, ps,
                                     map3(E, D, (long long)E * p7, D, (long long)E2 * p7),
                                     map2(D, 1, p7), I.sPop);
    if (cudaError_t e_ = tc_gemm(I.mode, a, b, Dn * DE, DE, DE, ep, I.err, I.s)) return e_;
  }
  hook->launched(HOTRG_ST_PROJ_Q, 1);
  hook->end(HOTRG_ST_PROJ_Q);
  // a7: T'(m = (a,y,y'), b) = sum_{(x1',x2')} Q[m][(x1',x2')] U[(x1' x2'), b]
  hook->begin(HOTRG_ST_PROJ_T);
  {
    TcOperand a = operand(I, I.Q, Dn * E2, n, p7, I.sPop), b = operand(I, I.opU7, Dn, n, p7, I.sTop);
    if (cudaError_t e_ = tc_gemm(I.mode, a, b, Dn * E2, Dn, n, f64_epilogue(I, Tout, tm, tn, sTout),
                                 I.err, I.s))
      return e_;
  }
  hook->launched(HOTRG_ST_PROJ_T, 1);
  hook->end(HOTRG_ST_PROJ_T);
  return 0;
}

}  // namespace hotrg
