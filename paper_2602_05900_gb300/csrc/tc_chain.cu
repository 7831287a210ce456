// Fused second half of the projection chain (Sec. II.B, Eq. 3: each product
// written straight into the layout its consumer reads), TF32 on tcgen05:
//
//   Q[(a,y,y')][(x1',x2')] = sum_{x2,k} P[(a,y,x1')][(x2,k)] T[(y',x2')][(x2,k)]   (a6)
//   T'[(a,y,y')][b]        = sum_{x1',x2'} Q[(a,y,y')][(x1',x2')] U[(x1',x2')][b]  (a7)
//
// One CTA computes a 128 x 128 tile of a6 whose rows are (y, x1') for 128 / D
// values of y (x1' fastest) and whose columns are (y', x2') for 128 / D values
// of y' (x2' fastest): the tile holds every (x1', x2') of NC = (128 / D)^2
// pairs (y, y'), which is all a7 needs of Q for those pairs.  The epilogue
// warps move the tile from tensor memory into shared memory as the K-major B
// operand of a7 (NC rows, K = D^2 ordered (x2', x1'), 128-byte swizzle, TF32
// rounded like the unfused chain's Q), and a second tcgen05.mma contracts it
// with U streamed through the same TMA ring (A operand: 32 rows b of U per
// k-block; the MMA's other 96 rows read whatever follows in shared memory and
// produce accumulator rows nobody reads).  Q never reaches global memory.
//
// Warp roles as in tc_gemm: warp 0 lane 0 TMA producer, warp 1 lane 0 MMA
// issuer, warp 2 tensor-memory allocation, warps 4-11 epilogue.  The MMA
// order over a CTA's units is a6(0), a6(1), a7(0), a6(2), a7(1), ...: the
// epilogue turns unit i's tile into the a7 operand while a6 of unit i + 1
// runs.  Every wait is bounded; a timeout sets *err_flag to 2, lets the
// kernel's own copies and MMAs finish, frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_chain.cuh"
#include "tcgen05.cuh"

namespace hotrg {
namespace {

using namespace tc;

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ float rna_tf32(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return __uint_as_float(u);
}

template <int D>
struct ChainCfg {
  static constexpr int BM = 128, BN = 128;
  static constexpr int NY = BM / D;             // y values of a tile
  static constexpr int NYP = BN / D;            // y' values of a tile
  static constexpr int NC = NY * NYP;           // (y, y') pairs: N of a7
  static constexpr int NKB6 = D * D / 32;       // a6 k-blocks (K = D E, E = D)
  static constexpr int NKB7 = D * D / 32;       // a7 k-blocks (K = D^2)
  static constexpr int TILE = 128 * 128;        // bytes of a 128-row k-block tile
  static constexpr int STAGE_BYTES = 2 * TILE;
  static constexpr int U7_TILE = 32 * 128;      // 32 rows of U per k-block
  static constexpr int U7_PER_STAGE = STAGE_BYTES / U7_TILE;
  static constexpr int NST7 = (NKB7 + U7_PER_STAGE - 1) / U7_PER_STAGE;
  static constexpr int STAGES = 4;
  static constexpr int B7_BYTES = NKB7 * NC * 128;
  // the A descriptor of the last U tile of the last stage spans 12 KB past
  // the ring: the a7 operand that follows covers it
  static_assert(B7_BYTES >= TILE - U7_TILE, "ring overrun of the a7 A descriptor");
  static constexpr int SMEM = STAGES * STAGE_BYTES + B7_BYTES + 1024;
  static constexpr int EPI_WARPS = 8;
  static constexpr int ACC7_COL = 2 * BN;       // tensor-memory column of the a7 accumulators
  static constexpr int TMEM_COLS = 512;
  static_assert(ACC7_COL + 2 * NC <= TMEM_COLS, "accumulators exceed tensor memory");
  static_assert(NC % 16 == 0 && NC <= 256, "a7 MMA shape");
};

template <int D>
__global__ void __launch_bounds__(384, 1)
    k_tc_chain(const __grid_constant__ CUtensorMap tp, const __grid_constant__ CUtensorMap tt,
               const __grid_constant__ CUtensorMap tu, int Dn, int batch, double *Tout,
               long long sTout, IdxMap tm, IdxMap tn, long long cap, int *err_flag, long long wait,
               int stall) {
  using C = ChainCfg<D>;
  constexpr int STAGES = C::STAGES;
  constexpr uint32_t IDESC6 = make_idesc(true, 128, C::BN);
  constexpr uint32_t IDESC7 = make_idesc(true, 128, C::NC);
  constexpr int E = D;

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc6_full[2], acc6_empty[2], acc7_full[2], acc7_empty[2];
  __shared__ __align__(8) uint64_t b7_full, b7_empty, drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_fail, s_issued, s_consumed;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t b7_base = smem_base + STAGES * C::STAGE_BYTES;
  float *b7 = reinterpret_cast<float *>(smem_raw + (smem_base - smem_u32(smem_raw)) +
                                        STAGES * C::STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = D * E / C::BN;                       // N tiles of a6 per instance
  const int mtn = Dn * D * E / C::BM;                  // M tiles of a6 per instance
  const long long nunits = (long long)ntn * mtn * batch;

  auto stage = [&](int s) { return smem_base + s * C::STAGE_BYTES; };
  auto unit_coords = [&](long long t, int &n0, int &m0, int &z) {
    n0 = (int)(t % ntn) * C::BN;
    m0 = (int)((t / ntn) % mtn) * C::BM;
    z = (int)(t / ((long long)ntn * mtn));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc6_full[b]), 1);
      mbar_init(smem_u32(&acc6_empty[b]), C::EPI_WARPS);
      mbar_init(smem_u32(&acc7_full[b]), 1);
      mbar_init(smem_u32(&acc7_empty[b]), C::EPI_WARPS);
    }
    mbar_init(smem_u32(&b7_full), C::EPI_WARPS);
    mbar_init(smem_u32(&b7_empty), 1);
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
    // ---- TMA producer: a6 k-blocks of unit i, then U for a7 of unit i - 1
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tp)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tt)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tu)) : "memory");
    int g = 0;
    bool ok = !stall;     // a stalled launch issues nothing: its consumers' waits run out
    auto acquire = [&](int &s) {
      s = g % STAGES;
      if (failed() || !mbar_wait(smem_u32(&empty_bar[s]), ((g / STAGES) & 1) ^ 1, wait)) {
        atomicExch(&s_fail, 1);
        ok = false;
      }
      return ok;
    };
    auto load7 = [&](int z) {
      for (int j = 0; j < C::NST7 && ok; ++j, ++g) {
        int s;
        if (!acquire(s)) break;
        const int cnt = min(C::U7_PER_STAGE, C::NKB7 - j * C::U7_PER_STAGE);
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, cnt * C::U7_TILE);
        for (int q = 0; q < cnt; ++q)
          tma_load_4d(stage(s) + q * C::U7_TILE, &tu, fb, (j * C::U7_PER_STAGE + q) * 32, 0, 0, z);
      }
    };
    int zprev = -1;
    for (long long t = blockIdx.x; t < nunits && ok; t += gridDim.x) {
      int n0, m0, z;
      unit_coords(t, n0, m0, z);
      for (int kb = 0; kb < C::NKB6 && ok; ++kb, ++g) {
        int s;
        if (!acquire(s)) break;
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, C::STAGE_BYTES);
        tma_load_4d(stage(s), &tp, fb, kb * 32, m0, 0, z);
        tma_load_4d(stage(s) + C::TILE, &tt, fb, kb * 32, n0, 0, z);
      }
      if (zprev >= 0 && ok) load7(zprev);
      zprev = z;
    }
    if (zprev >= 0 && ok) load7(zprev);
    s_issued = g;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer, same order as the producer
    int g = 0;
    bool ok = true;
    auto take = [&](int &s) {
      s = g % STAGES;
      if (failed() || !mbar_wait(smem_u32(&full_bar[s]), (g / STAGES) & 1, wait)) {
        atomicExch(&s_fail, 1);
        ok = false;
        return false;
      }
      s_consumed = g + 1;
      fence_after();
      return true;
    };
    auto wait_or_fail = [&](uint64_t *bar, uint32_t parity) {
      if (failed() || !mbar_wait(smem_u32(bar), parity, wait)) {
        atomicExch(&s_fail, 1);
        ok = false;
      }
      return ok;
    };
    auto phase7 = [&](int i) {
      const int buf = i & 1;
      if (!wait_or_fail(&acc7_empty[buf], ((i >> 1) & 1) ^ 1)) return;
      if (!wait_or_fail(&b7_full, i & 1)) return;
      fence_after();
      const uint32_t dt = tmem + C::ACC7_COL + buf * C::NC;
      for (int j = 0; j < C::NST7 && ok; ++j, ++g) {
        int s;
        if (!take(s)) break;
        const int cnt = min(C::U7_PER_STAGE, C::NKB7 - j * C::U7_PER_STAGE);
        for (int q = 0; q < cnt; ++q) {
          const int kb = j * C::U7_PER_STAGE + q;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t ad = sw_desc<128>(stage(s) + q * C::U7_TILE + k * 32);
            const uint64_t bd = sw_desc<128>(b7_base + kb * C::NC * 128 + k * 32);
            mma_tf32(dt, ad, bd, IDESC7, (kb | k) != 0);
          }
        }
        mma_commit(smem_u32(&empty_bar[s]));
      }
      if (ok) {
        mma_commit(smem_u32(&acc7_full[buf]));
        mma_commit(smem_u32(&b7_empty));
      }
    };
    int i = 0;
    for (long long t = blockIdx.x; t < nunits && ok; t += gridDim.x, ++i) {
      const int buf = i & 1;
      if (!wait_or_fail(&acc6_empty[buf], ((i >> 1) & 1) ^ 1)) break;
      fence_after();
      const uint32_t dt = tmem + buf * C::BN;
      for (int kb = 0; kb < C::NKB6 && ok; ++kb, ++g) {
        int s;
        if (!take(s)) break;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t ad = sw_desc<128>(stage(s) + k * 32);
          const uint64_t bd = sw_desc<128>(stage(s) + C::TILE + k * 32);
          mma_tf32(dt, ad, bd, IDESC6, (kb | k) != 0);
        }
        mma_commit(smem_u32(&empty_bar[s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&acc6_full[buf]));
      if (i > 0) phase7(i - 1);
    }
    if (ok && i > 0) phase7(i - 1);
    mma_commit(smem_u32(&drain_bar));   // tracks every MMA issued: the teardown waits for it
  } else if (warp >= 4) {
    // ---- epilogue: thread (warp w, lane l) owns accumulator row 32 (w mod 4) + l
    const int ew = warp - 4, quad = warp & 3, half = ew >> 2;
    const uint32_t trow = static_cast<uint32_t>(quad * 32) << 16;
    const int r = quad * 32 + lane;           // a6 row (y_l, x1'), x1' fastest
    const int yl = r / D, x1p = r % D;
    int i = 0;
    auto wait_or_fail = [&](uint64_t *bar, uint32_t parity) {
      if (failed() || !mbar_wait(smem_u32(bar), parity, wait)) {
        atomicExch(&s_fail, 1);
        return false;
      }
      return true;
    };
    for (long long t = blockIdx.x; t < nunits; t += gridDim.x, ++i) {
      const int buf = i & 1;
      if (!wait_or_fail(&acc6_full[buf], (i >> 1) & 1)) break;
      if (!wait_or_fail(&b7_empty, (i & 1) ^ 1)) break;   // a7 of unit i - 1 has read the operand
      fence_after();
      // (1) a6 tile -> a7 operand: element (row r, column c = (y'_l, x2')) goes to
      //     operand row n7 = y_l NYP + y'_l at k7 = x2' D + x1'
#pragma unroll 1
      for (int c = half; c < C::BN / 32; c += 2) {
        uint32_t v[32];
        tmem_ld32(tmem + trow + buf * C::BN + c * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c * 32 + j;
          const int ypl = col / D, x2p = col % D;
          const int n7 = yl * C::NYP + ypl, k7 = x2p * D + x1p;
          const int kb = k7 >> 5, w = k7 & 31;
          const int byte = kb * C::NC * 128 + n7 * 128 + ((((w >> 2) ^ (n7 & 7)) << 4) | ((w & 3) << 2));
          b7[byte >> 2] = rna_tf32(__uint_as_float(v[j]));
        }
      }
      // generic-proxy stores are read by the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      fence_before();
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc6_empty[buf])) : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&b7_full)) : "memory");
      }
      // (2) a7 accumulator (rows b < Dn) -> T'
      if (!wait_or_fail(&acc7_full[buf], (i >> 1) & 1)) break;
      fence_after();
      if (half == 0 && quad * 32 < Dn) {
        int n0, m0, z;
        unit_coords(t, n0, m0, z);
        const int a = m0 / (D * E), y0 = (m0 % (D * E)) / D, yp0 = n0 / D;
        const int b = quad * 32 + lane;
        const long long zoff = (long long)z * sTout;
        const long long boff = b < Dn ? map_off(tn, b) : 0;
        const uint32_t t7 = tmem + trow + C::ACC7_COL + buf * C::NC;
#pragma unroll 1
        for (int c0 = 0; c0 < C::NC; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(t7 + c0, v);
          if (b < Dn) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n7 = c0 + j, y = y0 + n7 / C::NYP, yp = yp0 + n7 % C::NYP;
              const long long off = map_off(tm, ((long long)a * E + y) * E + yp) + boff;
              if (checked_ok(zoff + off, cap, err_flag)) Tout[zoff + off] = (double)__uint_as_float(v[j]);
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc7_empty[buf])) : "memory");
    }
  }
  __syncwarp();

  fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_fail) atomicMax(err_flag, 2);
    for (int g = s_consumed; g < s_issued; ++g)
      (void)mbar_wait(smem_u32(&full_bar[g % STAGES]), (g / STAGES) & 1);
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

bool make_map_f32(CUtensorMap *m, const void *base, int K, int rows, int pitch, int batch,
                  long long bstride, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const long long bs = batch > 1 ? bstride : (long long)pitch * rows;
  cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, 1, (cuuint64_t)(batch < 1 ? 1 : batch)};
  cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * rows, (cuuint64_t)bs * 4};
  cuuint32_t box[4] = {32, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int D>
cudaError_t launch_chain(const ChainArgs &a, cudaStream_t s) {
  using C = ChainCfg<D>;
  CUtensorMap tp, tt, tu;
  const int DE = D * D, n = D * D;
  if (!make_map_f32(&tp, a.P, DE, a.Dn * DE, a.pitchP, a.batch, a.sP, 128) ||
      !make_map_f32(&tt, a.T6, DE, DE, a.pitchT, a.batch, a.sT6, 128) ||
      !make_map_f32(&tu, a.U7, n, a.Dn, a.pitchU, a.batch, a.sU7, 32))
    return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_chain<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
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
  const long long units = (long long)(DE / C::BN) * (a.Dn * DE / C::BM) * a.batch;
  const int grid = (int)(units < nsm ? units : nsm);
  const int stall = take_stall(kStallChain) ? 1 : 0;
  k_tc_chain<D><<<grid, 384, C::SMEM, s>>>(tp, tt, tu, a.Dn, a.batch, a.Tout, a.sTout, a.tm, a.tn,
                                            a.cap, a.err, wait_limit(), stall);
  return cudaGetLastError();
}

}  // namespace

bool tc_chain_supported(int D, int E, int Dn) {
  return D == E && (D == 16 || D == 32) && Dn >= 1 && Dn <= 32 && (Dn * D * E) % 128 == 0;
}

cudaError_t tc_chain(const ChainArgs &a, cudaStream_t s) {
  if (!tc_chain_supported(a.D, a.E, a.Dn) || a.batch < 1) return cudaErrorInvalidValue;
  const int DE = a.D * a.E;
  if (a.pitchP < DE || a.pitchT < DE || a.pitchU < a.D * a.D || (a.pitchP % 4) || (a.pitchT % 4) ||
      (a.pitchU % 4))
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(a.P) & 15) || (reinterpret_cast<uintptr_t>(a.T6) & 15) ||
      (reinterpret_cast<uintptr_t>(a.U7) & 15))
    return cudaErrorInvalidValue;
  if (a.batch > 1 && ((a.sP * 4) % 16 || (a.sT6 * 4) % 16 || (a.sU7 * 4) % 16)) return cudaErrorInvalidValue;
  return a.D == 32 ? launch_chain<32>(a, s) : launch_chain<16>(a, s);
}

}  // namespace hotrg
