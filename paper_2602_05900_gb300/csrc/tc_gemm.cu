// tcgen05 tensor-core GEMM with TMA operand staging (sm_103a).
//
// One CTA computes a 128 x BN tile of C = sum_products A_p . B_q^T:
//   warp 0 / lane 0   TMA producer: 128-byte-swizzled K-major tiles of every
//                     operand plane into a STAGES-deep shared-memory ring;
//   warp 1 / lane 0   MMA issuer: tcgen05.mma (kind::tf32 or kind::f16) into a
//                     128 x BN FP32 accumulator in tensor memory, one commit per
//                     stage to release it back to the producer;
//   warps 0-3         epilogue: tcgen05.ld of the thread's accumulator row,
//                     stores through the output index maps.
// Every pipeline wait is bounded (wait_limit(), about a second by default); on
// timeout the kernel sets *err_flag, waits (with the default bound) for its own
// TMA copies and MMAs still in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "tc_gemm.cuh"
#include "tcgen05.cuh"

namespace hotrg {
namespace {

using namespace tc;

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ float round_tf32(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return __uint_as_float(u);
}

// Stores v at element off of instance buffer e.C; zoff is that buffer's
// offset from the base of the whole allocation (bounds of the checked build).
__device__ __forceinline__ void store_out(const TcEpilogue &e, long long off, float v, long long zoff,
                                          int *err) {
  if (!checked_ok(zoff + off, e.cap, err)) return;
  if (e.kind == OutKind::BF16P && !checked_ok(zoff + off + (e.planes - 1) * e.plane_stride, e.cap, err))
    return;
  switch (e.kind) {
    case OutKind::F32:
      static_cast<float *>(e.C)[off] = e.round_tf32 ? round_tf32(v) : v;
      break;
    case OutKind::F64:
      static_cast<double *>(e.C)[off] = static_cast<double>(v);
      break;
    case OutKind::BF16P: {
      __nv_bfloat16 *c = static_cast<__nv_bfloat16 *>(e.C);
      float r = v;
      for (int p = 0; p < e.planes; ++p) {
        __nv_bfloat16 t = __float2bfloat16_rn(r);
        c[off + p * e.plane_stride] = t;
        r -= __bfloat162float(t);
      }
      break;
    }
  }
}

// Stores 4 consecutive columns (off .. off + 3) of an F32 or F64 output at once
// (16-byte stores; tc_gemm checked the alignment when it set e.vec4).
__device__ __forceinline__ void store_out4(const TcEpilogue &e, long long off, float v0, float v1,
                                           float v2, float v3, long long zoff, int *err) {
  if (!checked_ok(zoff + off, e.cap, err) || !checked_ok(zoff + off + 3, e.cap, err)) return;
  if (e.kind == OutKind::F32) {
    if (e.round_tf32) {
      v0 = round_tf32(v0);
      v1 = round_tf32(v1);
      v2 = round_tf32(v2);
      v3 = round_tf32(v3);
    }
    *reinterpret_cast<float4 *>(static_cast<float *>(e.C) + off) = make_float4(v0, v1, v2, v3);
  } else {
    double2 *d = reinterpret_cast<double2 *>(static_cast<double *>(e.C) + off);
    d[0] = make_double2(v0, v1);
    d[1] = make_double2(v2, v3);
  }
}

template <int MODE>
struct ModeTraits;
template <>
struct ModeTraits<0> {  // TF32
  static constexpr bool kTf32 = true;
  static constexpr int kPlanes = 1, kBK = 32, kMmaK = 8, kProducts = 1;
  __device__ static void product(int, int &pa, int &pb) { pa = 0; pb = 0; }
};
template <>
struct ModeTraits<1> {  // BF16 x3: hi.hi, hi.lo, lo.hi (small terms issued first)
  static constexpr bool kTf32 = false;
  static constexpr int kPlanes = 2, kBK = 64, kMmaK = 16, kProducts = 3;
  __device__ static void product(int i, int &pa, int &pb) {
    const int a[3] = {0, 1, 0}, b[3] = {1, 0, 0};
    pa = a[i];
    pb = b[i];
  }
};
template <>
struct ModeTraits<2> {  // BF16 x6: every (p, q) with p + q <= 2, smallest first
  static constexpr bool kTf32 = false;
  static constexpr int kPlanes = 3, kBK = 64, kMmaK = 16, kProducts = 6;
  __device__ static void product(int i, int &pa, int &pb) {
    const int a[6] = {0, 1, 2, 0, 1, 0}, b[6] = {2, 1, 0, 1, 0, 0};
    pa = a[i];
    pb = b[i];
  }
};

template <int MODE, int BN>
struct Cfg {
  using Tr = ModeTraits<MODE>;
  static constexpr int BM = 128;
  static constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
  static constexpr int STAGE_BYTES = Tr::kPlanes * (A_BYTES + B_BYTES);
  static constexpr int EPI_WARPS = 8;                        // two per tensor-memory lane quadrant
  static constexpr int STAGING_BYTES = EPI_WARPS * 32 * 33 * 4;   // epilogue transpose, 32 x 33 per warp
  static constexpr int STAGES_RAW = (196 * 1024) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 6 ? 6 : STAGES_RAW;
  static constexpr int SMEM = STAGES * STAGE_BYTES + STAGING_BYTES + 1024;
  static constexpr int TMEM_COLS = 2 * BN;                   // two accumulator buffers
  static_assert(STAGES >= 2, "pipeline needs two stages");
  static_assert(TMEM_COLS <= 512, "accumulators exceed tensor memory");
};

// Persistent, warp-specialised: every CTA walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (N tiles fastest, then M tiles, then the
// instance of the batch).  Warp 0 streams the operand k-blocks of all its
// tiles through the shared-memory ring without draining it between tiles;
// warp 1 issues the MMAs of tile i into tensor-memory buffer i & 1; warps
// 4-11 drain buffer i & 1 to global memory while the MMAs of tile i + 1 proceed
// (warp w reads tensor-memory lanes 32 (w mod 4) .. + 31, the two warps of a
// quadrant take alternate 32-column chunks: the epilogue is latency bound, so
// it gets two warps per scheduler).
template <int MODE, int BN>
__global__ void __launch_bounds__(384, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              int M, int N, int K, int batch, TcEpilogue epi, int *err_flag, long long wait,
              int stall) {
  using C = Cfg<MODE, BN>;
  using Tr = typename C::Tr;
  constexpr int STAGES = C::STAGES;
  constexpr uint32_t IDESC = make_idesc(Tr::kTf32, C::BM, BN);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_fail, s_issued, s_consumed;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (K + Tr::kBK - 1) / Tr::kBK;
  const int ntn = (N + BN - 1) / BN, mtn = (M + C::BM - 1) / C::BM;
  const long long ntiles = (long long)ntn * mtn * batch;
  const int esize = epi.kind == OutKind::F64 ? 8 : (epi.kind == OutKind::F32 ? 4 : 2);

  auto a_tile = [&](int s, int p) { return smem_base + s * C::STAGE_BYTES + p * C::A_BYTES; };
  auto b_tile = [&](int s, int p) {
    return smem_base + s * C::STAGE_BYTES + Tr::kPlanes * C::A_BYTES + p * C::B_BYTES;
  };
  auto tile_coords = [&](long long t, int &n0, int &m0, int &z) {
    n0 = (int)(t % ntn) * BN;
    m0 = (int)((t / ntn) % mtn) * C::BM;
    z = (int)(t / ((long long)ntn * mtn));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), C::EPI_WARPS);   // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;
  auto failed = [&]() { return *(volatile int *)&s_fail != 0; };

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one continuous k-block stream over all own tiles
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
    int g = 0;
    bool ok = !stall;     // a stalled launch issues nothing: its consumers' waits run out
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int n0, m0, z;
      tile_coords(t, n0, m0, z);
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = g % STAGES;
        const uint32_t ph = (g / STAGES) & 1;
        if (failed() || !mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1, wait)) {
          atomicExch(&s_fail, 1);
          ok = false;
          break;
        }
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, C::STAGE_BYTES);
        for (int p = 0; p < Tr::kPlanes; ++p)
          tma_load_4d(a_tile(s, p), &ta, fb, kb * Tr::kBK, m0, p, z);
        for (int p = 0; p < Tr::kPlanes; ++p)
          tma_load_4d(b_tile(s, p), &tb, fb, kb * Tr::kBK, n0, p, z);
      }
    }
    s_issued = g;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: tile i accumulates into tensor-memory buffer i & 1
    int g = 0, i = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
      const int buf = i & 1;
      if (failed() || !mbar_wait(smem_u32(&acc_empty[buf]), ((i >> 1) & 1) ^ 1, wait)) {
        atomicExch(&s_fail, 1);
        break;
      }
      fence_after();
      const uint32_t dt = tmem + buf * BN;
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = g % STAGES;
        const uint32_t ph = (g / STAGES) & 1;
        if (failed() || !mbar_wait(smem_u32(&full_bar[s]), ph, wait)) {
          atomicExch(&s_fail, 1);
          ok = false;
          break;
        }
        s_consumed = g + 1;
        fence_after();
#pragma unroll
        for (int k = 0; k < Tr::kBK / Tr::kMmaK; ++k) {
#pragma unroll
          for (int q = 0; q < Tr::kProducts; ++q) {
            int pa, pb;
            Tr::product(q, pa, pb);
            const uint64_t ad = sw_desc<128>(a_tile(s, pa) + k * 32);
            const uint64_t bd = sw_desc<128>(b_tile(s, pb) + k * 32);
            mma_issue<Tr::kTf32>(dt, ad, bd, IDESC, (kb | k | q) != 0);
          }
        }
        mma_commit(smem_u32(&empty_bar[s]));
      }
      if (ok) mma_commit(smem_u32(&acc_full[buf]));
    }
    // tracks every MMA this thread issued: the teardown waits for it
    mma_commit(smem_u32(&drain_bar));
  } else if (warp >= 4) {
    // ---- epilogue warps: thread (warp w, lane l) owns accumulator row 32 (w mod 4) + l
    const int ew = warp - 4;
    const int quad = warp & 3, half = ew >> 2;
    float *stage = reinterpret_cast<float *>(smem_raw + (smem_base - smem_u32(smem_raw)) +
                                             STAGES * C::STAGE_BYTES) + ew * 32 * 33;
    const uint32_t trow = static_cast<uint32_t>(quad * 32) << 16;
    int i = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int buf = i & 1;
      if (failed() || !mbar_wait(smem_u32(&acc_full[buf]), (i >> 1) & 1, wait)) {
        atomicExch(&s_fail, 1);
        break;
      }
      fence_after();
      int n0, m0, z;
      tile_coords(t, n0, m0, z);
      TcEpilogue e = epi;
      e.C = static_cast<char *>(epi.C) + (long long)z * epi.bstride * esize;
      const long long zoff = (long long)z * epi.bstride;
      const int row = m0 + quad * 32 + lane;
      const bool rv = row < M;
      const long long roff = rv ? map_off(e.cm, row) : -1;
#pragma unroll 1
      for (int c = half; c < BN / 32; c += 2) {
        if (n0 + c * 32 >= N) break;
        uint32_t r[32];
        tmem_ld32(tmem + trow + buf * BN + c * 32, r);
        const int col = n0 + c * 32 + lane;
        const long long coff = (col < N) ? map_off(e.cn, col) : -1;
        if (!e.transpose) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const long long co = __shfl_sync(0xffffffffu, coff, j);
            if (rv && co >= 0) store_out(e, roff + co, __uint_as_float(r[j]), zoff, err_flag);
          }
        } else if (e.vec4 && n0 + c * 32 + 32 <= N) {
          // column-major staging (stage[col][row], conflict-free), then lane l
          // stores columns 4 (l mod 8) .. + 3 of row 4 it + l / 8: eight 16-byte
          // stores per lane and chunk instead of 32 scalar ones
#pragma unroll
          for (int j = 0; j < 32; ++j) stage[j * 33 + lane] = __uint_as_float(r[j]);
          __syncwarp();
          const int q = lane & 7;
          const long long cq = map_off(e.cn, n0 + c * 32 + 4 * q);
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int rr = it * 4 + (lane >> 3);
            const long long ro = __shfl_sync(0xffffffffu, roff, rr);
            const float v0 = stage[(4 * q) * 33 + rr], v1 = stage[(4 * q + 1) * 33 + rr];
            const float v2 = stage[(4 * q + 2) * 33 + rr], v3 = stage[(4 * q + 3) * 33 + rr];
            if (ro >= 0) store_out4(e, ro + cq, v0, v1, v2, v3, zoff, err_flag);
          }
          __syncwarp();
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
          __syncwarp();
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const long long ro = __shfl_sync(0xffffffffu, roff, rr);
            const float v = stage[rr * 33 + lane];
            if (ro >= 0 && coff >= 0) store_out(e, ro + coff, v, zoff, err_flag);
          }
          __syncwarp();
        }
      }
      // buffer drained: the MMA warp may reuse it
      fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  }
  __syncwarp();

  fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_fail) atomicMax(err_flag, 2);   // a timeout outranks the non-finite flag (1) it may cause
    // TMA copies issued but never consumed (only after a timeout): let them land
    for (int g = s_consumed; g < s_issued; ++g)
      (void)mbar_wait(smem_u32(&full_bar[g % STAGES]), (g / STAGES) & 1);
    // MMAs still running (only after a timeout) must finish before the dealloc
    (void)mbar_wait(smem_u32(&drain_bar), 0);
  }
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ---- host side ----------------------------------------------------------

bool make_map(CUtensorMap *m, TcMode mode, const TcOperand &op, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const int eb = tc_elem_bytes(mode);
  const int planes = tc_planes(mode);
  const long long bs = op.batch > 1 ? op.bstride : (long long)op.pitch * op.rows * planes;
  cuuint64_t dims[4] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)planes,
                        (cuuint64_t)(op.batch < 1 ? 1 : op.batch)};
  cuuint64_t strides[3] = {(cuuint64_t)op.pitch * eb, (cuuint64_t)op.pitch * eb * op.rows,
                           (cuuint64_t)bs * eb};
  cuuint32_t box[4] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt =
      mode == TcMode::TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = enc(m, dt, 4, const_cast<void *>(op.base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int MODE, int BN>
cudaError_t launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int batch,
                   const TcEpilogue &epi, int *err, cudaStream_t s) {
  const int stall = take_stall(kStallGemm) ? 1 : 0;
  using C = Cfg<MODE, BN>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<MODE, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 148;
  }
  const long long tiles = (long long)((N + BN - 1) / BN) * ((M + C::BM - 1) / C::BM) * batch;
  const int grid = (int)(tiles < nsm ? tiles : nsm);
  k_tc_gemm<MODE, BN><<<grid, 384, C::SMEM, s>>>(ta, tb, M, N, K, batch, epi, err, wait_limit(),
                                                  stall);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t run_bn(int bn, const TcOperand &A, const TcOperand &B, int M, int N, int K,
                   const TcEpilogue &epi, int *err, cudaStream_t s) {
  const TcMode mode = static_cast<TcMode>(MODE);
  CUtensorMap ta, tb;
  if (!make_map(&ta, mode, A, 128) || !make_map(&tb, mode, B, bn)) return cudaErrorInvalidValue;
  const int batch = A.batch < 1 ? 1 : A.batch;
  if (bn == 64) return launch<MODE, 64>(ta, tb, M, N, K, batch, epi, err, s);
  if (bn == 128) return launch<MODE, 128>(ta, tb, M, N, K, batch, epi, err, s);
  if constexpr (MODE == 0) {
    if (bn == 256) return launch<MODE, 256>(ta, tb, M, N, K, batch, epi, err, s);
  }
  return cudaErrorInvalidValue;
}

// Tile-width autotuner: the first GEMM of each shape (mode, M, N, K, batch,
// output kind and store layout) runs once with every tile width and keeps the
// fastest (CUDA events on the caller's stream; every width computes the same
// products in the same order, so the result does not depend on the choice).
// Shapes met while the stream is being captured into a graph use the cached
// choice, or the static heuristic if there is none.
struct TuneKey {
  int mode, M, N, K, batch, kind, transpose;
  bool operator<(const TuneKey &o) const {
    return std::tie(mode, M, N, K, batch, kind, transpose) <
           std::tie(o.mode, o.M, o.N, o.K, o.batch, o.kind, o.transpose);
  }
};
std::map<TuneKey, int> g_tuned;
std::mutex g_tune_mu;
std::atomic<bool> g_autotune{true};

template <int MODE>
cudaError_t dispatch_bn(const TcOperand &A, const TcOperand &B, int M, int N, int K,
                        const TcEpilogue &epi, int *err, cudaStream_t s) {
  const int heuristic = N <= 64 ? 64 : (N <= 128 || MODE != 0 ? 128 : 256);
  if (!g_autotune.load()) return run_bn<MODE>(heuristic, A, B, M, N, K, epi, err, s);
  const TuneKey key{MODE, M, N, K, A.batch < 1 ? 1 : A.batch, (int)epi.kind, epi.transpose ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return run_bn<MODE>(it->second, A, B, M, N, K, epi, err, s);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return run_bn<MODE>(heuristic, A, B, M, N, K, epi, err, s);
  }
  const int cands[3] = {64, 128, 256};
  const int ncand = MODE == 0 ? 3 : 2;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    (void)cudaGetLastError();
    if (ev[0]) cudaEventDestroy(ev[0]);
    return run_bn<MODE>(heuristic, A, B, M, N, K, epi, err, s);
  }
  int best = heuristic;
  float best_ms = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ncand && e == cudaSuccess; ++i) {
    const int bn = cands[i];
    if ((e = run_bn<MODE>(bn, A, B, M, N, K, epi, err, s))) break;     // warm-up
    if ((e = cudaEventRecord(ev[0], s)) || (e = run_bn<MODE>(bn, A, B, M, N, K, epi, err, s)) ||
        (e = cudaEventRecord(ev[1], s)) || (e = cudaEventSynchronize(ev[1])))
      break;
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, ev[0], ev[1]))) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = bn;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e) return e;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
  }
  return cudaSuccess;   // the last timed launch already wrote the result
}

}  // namespace

namespace tc {

namespace {
std::atomic<long long> g_wait_limit{kWaitCycles};
std::atomic<int> g_stall{0};
}  // namespace

void set_wait_limit(long long cycles) { g_wait_limit.store(cycles > 0 ? cycles : kWaitCycles); }
long long wait_limit() { return g_wait_limit.load(); }
void arm_stall(int kind) { g_stall.store(kind); }
bool take_stall(int kind) {
  int k = kind;
  return g_stall.compare_exchange_strong(k, 0);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace tc

void tc_set_autotune(bool on) { g_autotune.store(on); }

cudaError_t tc_gemm(TcMode mode, const TcOperand &A, const TcOperand &B, int M, int N, int K,
                    const TcEpilogue &epi, int *err_flag, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0 || A.K != K || B.K != K || A.rows < M || B.rows < N) return cudaErrorInvalidValue;
  if ((A.batch < 1 ? 1 : A.batch) != (B.batch < 1 ? 1 : B.batch)) return cudaErrorInvalidValue;
  {
    // TMA strides must be multiples of 16 bytes
    const int eb = tc_elem_bytes(mode);
    if ((A.batch > 1 && (A.bstride * eb) % 16) || (B.batch > 1 && (B.bstride * eb) % 16))
      return cudaErrorInvalidValue;
  }
  if (A.pitch != tc_pitch(A.pitch, mode) || B.pitch != tc_pitch(B.pitch, mode) || A.pitch < K ||
      B.pitch < K)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A.base) & 15) || (reinterpret_cast<uintptr_t>(B.base) & 15))
    return cudaErrorInvalidValue;
  TcEpilogue e = epi;
  // store layout: keep lane = row when the rows are unit-stride, else transpose
  e.transpose = !(epi.cm.s0 == 1 && epi.cm.n0 >= 8);
  // transposed F32 / F64 stores 4 columns at a time where every group of 4
  // consecutive columns is contiguous and 16-byte aligned: unit column stride,
  // all other strides and the instance stride multiples of 4 elements
  {
    auto m4 = [](long long v) { return (v & 3) == 0; };
    const IdxMap &cm = epi.cm, &cn = epi.cn;
    e.vec4 = e.transpose && (epi.kind == OutKind::F32 || epi.kind == OutKind::F64) && cn.s0 == 1 &&
             (cn.n0 & 3) == 0 && m4(cn.s1) && m4(cn.s2) && m4(cm.s0) && m4(cm.s1) && m4(cm.s2) &&
             m4(epi.bstride) && (reinterpret_cast<uintptr_t>(epi.C) & 15) == 0;
  }
  switch (mode) {
    case TcMode::TF32: return dispatch_bn<0>(A, B, M, N, K, e, err_flag, s);
    case TcMode::BF16X3: return dispatch_bn<1>(A, B, M, N, K, e, err_flag, s);
    case TcMode::BF16X6: return dispatch_bn<2>(A, B, M, N, K, e, err_flag, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hotrg
