// Exact-slice GEMM kernels (see tc_exact.cuh).
//
// k_xs_split   one warp per row: row max, power-of-two scale, S digits.
// k_xs_gemm    one CTA per 128 x BN output tile (and K part):
//   warp 0 / lane 0   TMA producer: S slice tiles of A and of B per 32-wide K
//                     block (64-byte swizzled rows) into a shared-memory ring;
//   warp 1 / lane 0   MMA issuer: for every kept slice pair one kind::f16
//                     tcgen05.mma per 16-wide K step into the accumulator of
//                     its diagonal (tensor memory, BN columns each);
//   warps 0-3         epilogue: exact accumulators -> int64, small one and
//                     scales in FP64, FP64 stores.
// Waits are bounded as in the other tcgen05 kernels: on timeout the kernel sets
// *err_flag, lets its own TMA copies land, frees tensor memory and returns.
#include <cuda_bf16.h>

#include "tc_exact.cuh"
#include "tcgen05.cuh"

namespace hotrg {
namespace {

using namespace tc;

// Kept slice pairs (0-based s + t <= S - 1) ordered by diagonal, with their
// accumulator (diagonals 0..4 exact, 5 and up shared) and whether they are
// the first pair of that accumulator.
template <int S>
struct XsTable {
  static constexpr int kPairs = S * (S + 1) / 2;
  static constexpr int kExact = S < kXsExactDiagonals ? S : kXsExactDiagonals;
  static constexpr int kAcc = S <= kXsExactDiagonals ? S : kXsExactDiagonals + 1;
  int a[kPairs], b[kPairs], acc[kPairs], first[kPairs];
  constexpr XsTable() : a(), b(), acc(), first() {
    int q = 0;
    for (int d = 0; d < S; ++d)
      for (int s = 0; s <= d; ++s) {
        a[q] = s;
        b[q] = d - s;
        acc[q] = d < kXsExactDiagonals ? d : kXsExactDiagonals;
        first[q] = (s == 0 && d <= kXsExactDiagonals) ? 1 : 0;
        ++q;
      }
  }
};

template <int S, int BN>
struct XsCfg {
  // K block: 32 BF16 (64-byte rows, 64-byte swizzle) while two such stages of
  // all slices fit in shared memory, else 16 BF16 (32-byte rows and swizzle)
  static constexpr int BM = 128;
  static constexpr int ROW = (2 * S * (BM + BN) * 64 <= 200 * 1024) ? 64 : 32;
  static constexpr int BK = ROW / 2;
  static constexpr int A_BYTES = BM * ROW, B_BYTES = BN * ROW;
  static constexpr int STAGE_BYTES = S * (A_BYTES + B_BYTES);
  static constexpr int STAGES_RAW = (200 * 1024) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 4 ? 4 : STAGES_RAW;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static constexpr int NACC = XsTable<S>::kAcc;
  static constexpr int COLS_RAW = NACC * BN;
  static constexpr int TMEM_COLS = COLS_RAW <= 32 ? 32 : COLS_RAW <= 64 ? 64 : COLS_RAW <= 128 ? 128
                                   : COLS_RAW <= 256 ? 256 : 512;
  static_assert(STAGES >= 2, "pipeline needs two stages");
  static_assert(COLS_RAW <= 512, "accumulators exceed tensor memory");
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "BN");
};

struct XsOut {
  double *C;
  IdxMap cm, cn;
  long long cstride, pstride;
  const double *sa, *sb;
  long long ssa, ssb;
};

// One warp per row.  The row maximum is taken on the bit patterns (|x| of a
// double orders like its bits as an unsigned integer), the scaled row is
// rounded once to a 6S-bit fixed-point integer (one FP64 multiply and one
// conversion per element: GB300's FP64 units are slow), and the digits come
// off that integer from the bottom in balanced form: d_S..d_2 in [-32, 31],
// then the top digit d_1 = what is left, |d_1| <= 64 because |row| < 2^e.
template <int S>
__global__ void __launch_bounds__(256) k_xs_split(PSet src, int R, int K, IdxMap rm, IdxMap km,
                                                  __nv_bfloat16 *dst, int pitch, long long bstride,
                                                  double *scale, long long sstride, PSet kscale,
                                                  int kmode) {
  const int z = blockIdx.z;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  const double *a = src.at(z);
  const double *ks = kmode ? kscale.at(z) : nullptr;
  const long long ro = map_off(rm, r);
  // element k (with the optional power-of-two column factor)
  auto elem = [&](int k) {
    const double v = a[ro + map_off(km, k)];
    if (kmode == 1) return v * ks[k];
    if (kmode == 2) return v / ks[k];
    return v;
  };
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  unsigned long long mb = 0;
  for (int k = lane; k < K; k += 32) {
    unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(elem(k))) & kAbs;
    if (u > kInf) u = kInf;                                   // NaN poisons the row like +inf
    mb = u > mb ? u : mb;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = t > mb ? t : mb;
  }
  const double mx = __longlong_as_double(static_cast<long long>(mb));
  int e = 0;
  const bool finite = mb < kInf;
  if (finite && mb != 0) (void)frexp(mx, &e);                // mx < 2^e
  if (lane == 0) scale[z * sstride + r] = finite ? ldexp(1.0, e) : NAN;
  const double up = ldexp(1.0, kXsBits * S - e);             // row -> 6S-bit fixed point
  __nv_bfloat16 *out = dst + z * bstride + (long long)r * pitch;
  const long long plane = (long long)R * pitch;
  for (int k = lane; k < K; k += 32) {
    long long N = finite ? __double2ll_rn(elem(k) * up) : 0;
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
      const long long d = ((N + 32) & 63) - 32;
      N = (N - d) >> kXsBits;                                 // exact: N - d is a multiple of 64
      out[p * plane + k] = __float2bfloat16_rn(ldexpf((float)d, -kXsBits * (p + 1)));
    }
    out[k] = __float2bfloat16_rn(ldexpf((float)N, -kXsBits));
  }
}

// The same slicing with one 256-thread block per row, for long rows (K >= 256):
// the warp-per-row kernel leaves most of the GPU idle when there are few rows
// (the n-long columns of a basis: 2m rows) and walks each row serially.  Same
// arithmetic per element, so the slices are identical.
template <int S>
__global__ void __launch_bounds__(256) k_xs_split_row(PSet src, int R, int K, IdxMap rm, IdxMap km,
                                                      __nv_bfloat16 *dst, int pitch, long long bstride,
                                                      double *scale, long long sstride, PSet kscale,
                                                      int kmode) {
  const int z = blockIdx.z, r = blockIdx.x;
  const double *a = src.at(z);
  const double *ks = kmode ? kscale.at(z) : nullptr;
  const long long ro = map_off(rm, r);
  auto elem = [&](int k) {
    const double v = a[ro + map_off(km, k)];
    if (kmode == 1) return v * ks[k];
    if (kmode == 2) return v / ks[k];
    return v;
  };
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  unsigned long long mb = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(elem(k))) & kAbs;
    if (u > kInf) u = kInf;
    mb = u > mb ? u : mb;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = t > mb ? t : mb;
  }
  __shared__ unsigned long long part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mb;
  __syncthreads();
  mb = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) mb = part[w] > mb ? part[w] : mb;
  const double mx = __longlong_as_double(static_cast<long long>(mb));
  int e = 0;
  const bool finite = mb < kInf;
  if (finite && mb != 0) (void)frexp(mx, &e);
  if (threadIdx.x == 0) scale[z * sstride + r] = finite ? ldexp(1.0, e) : NAN;
  const double up = ldexp(1.0, kXsBits * S - e);
  __nv_bfloat16 *out = dst + z * bstride + (long long)r * pitch;
  const long long plane = (long long)R * pitch;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    long long N = finite ? __double2ll_rn(elem(k) * up) : 0;
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
      const long long d = ((N + 32) & 63) - 32;
      N = (N - d) >> kXsBits;
      out[p * plane + k] = __float2bfloat16_rn(ldexpf((float)d, -kXsBits * (p + 1)));
    }
    out[k] = __float2bfloat16_rn(ldexpf((float)N, -kXsBits));
  }
}

// The same slicing for operands whose rows are contiguous but whose K index is
// strided (the basis of a rotation X W, column-major X as the A operand): a
// block stages 32 rows x K (K <= kXsStagedK) through shared memory with loads
// that run along the rows, then each warp slices its rows along K as above.
template <int S>
__global__ void __launch_bounds__(256) k_xs_split_staged(PSet src, int R, int K, IdxMap rm,
                                                         IdxMap km, __nv_bfloat16 *dst, int pitch,
                                                         long long bstride, double *scale,
                                                         long long sstride, PSet kscale, int kmode) {
  __shared__ double tile[32][kXsStagedK + 1];
  const int z = blockIdx.z;
  const int r0 = blockIdx.x * 32;
  const double *a = src.at(z);
  const double *ks = kmode ? kscale.at(z) : nullptr;
  // load: thread t reads row r0 + (t & 31) of column k = t / 32, + 8 per pass
  for (int e = threadIdx.x; e < 32 * K; e += blockDim.x) {
    const int rl = e & 31, k = e >> 5, r = r0 + rl;
    double v = 0.0;
    if (r < R) {
      v = a[map_off(rm, r) + map_off(km, k)];
      if (kmode == 1) v *= ks[k];
      if (kmode == 2) v /= ks[k];
    }
    tile[rl][k] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  for (int rl = threadIdx.x >> 5; rl < 32; rl += blockDim.x >> 5) {
    const int r = r0 + rl;
    if (r >= R) break;
    unsigned long long mb = 0;
    for (int k = lane; k < K; k += 32) {
      unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(tile[rl][k])) & kAbs;
      if (u > kInf) u = kInf;
      mb = u > mb ? u : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = t > mb ? t : mb;
    }
    const double mx = __longlong_as_double(static_cast<long long>(mb));
    int e = 0;
    const bool finite = mb < kInf;
    if (finite && mb != 0) (void)frexp(mx, &e);
    if (lane == 0) scale[z * sstride + r] = finite ? ldexp(1.0, e) : NAN;
    const double up = ldexp(1.0, kXsBits * S - e);
    __nv_bfloat16 *out = dst + z * bstride + (long long)r * pitch;
    const long long plane = (long long)R * pitch;
    for (int k = lane; k < K; k += 32) {
      long long N = finite ? __double2ll_rn(tile[rl][k] * up) : 0;
#pragma unroll
      for (int p = S - 1; p >= 1; --p) {
        const long long d = ((N + 32) & 63) - 32;
        N = (N - d) >> kXsBits;
        out[p * plane + k] = __float2bfloat16_rn(ldexpf((float)d, -kXsBits * (p + 1)));
      }
      out[k] = __float2bfloat16_rn(ldexpf((float)N, -kXsBits));
    }
  }
}

template <int S, int BN>
__global__ void __launch_bounds__(128, 1)
    k_xs_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              int M, int N, int K, int kb_per_part, int ntn, XsOut o, int *err_flag,
              long long wait, int stall) {
  using C = XsCfg<S, BN>;
  constexpr XsTable<S> T{};
  constexpr int STAGES = C::STAGES;
  constexpr uint32_t IDESC = make_idesc(false, C::BM, BN);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_fail, s_issued, s_consumed;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = blockIdx.x % ntn, part = blockIdx.x / ntn;
  const int m0 = blockIdx.y * C::BM, n0 = ntile * BN, z = blockIdx.z;
  const int nkb = (K + C::BK - 1) / C::BK;
  const int kb0 = part * kb_per_part;
  const int kb1 = min(nkb, kb0 + kb_per_part);
  const int nk = kb1 - kb0;

  auto a_tile = [&](int s, int p) { return smem_base + s * C::STAGE_BYTES + p * C::A_BYTES; };
  auto b_tile = [&](int s, int p) {
    return smem_base + s * C::STAGE_BYTES + S * C::A_BYTES + p * C::B_BYTES;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&acc_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  if (warp == 1) {
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

  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
    int i = 0;
    for (; i < (stall ? 0 : nk); ++i) {    // a stalled launch issues nothing
      const int s = i % STAGES;
      const uint32_t ph = (i / STAGES) & 1;
      if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1, wait)) {
        atomicExch(&s_fail, 1);
        break;
      }
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, C::STAGE_BYTES);
      const int kx = (kb0 + i) * C::BK;
#pragma unroll
      for (int p = 0; p < S; ++p) tma_load_4d(a_tile(s, p), &ta, fb, kx, m0, p, z);
#pragma unroll
      for (int p = 0; p < S; ++p) tma_load_4d(b_tile(s, p), &tb, fb, kx, n0, p, z);
    }
    s_issued = i;
  } else if (warp == 1 && lane == 0) {
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (i / STAGES) & 1;
      if (!mbar_wait(smem_u32(&full_bar[s]), ph, wait)) {
        atomicExch(&s_fail, 1);
        break;
      }
      fence_after();
      // descriptors differ only in their start-address field (address >> 4,
      // 14 bits, no carry for shared-memory addresses): base + offset >> 4
      const uint64_t adesc = sw_desc<C::ROW>(a_tile(s, 0)), bdesc = sw_desc<C::ROW>(b_tile(s, 0));
#pragma unroll 1
      for (int k = 0; k < C::BK / 16; ++k) {
#pragma unroll
        for (int q = 0; q < T.kPairs; ++q) {
          const uint64_t ad = adesc + ((T.a[q] * C::A_BYTES + k * 32) >> 4);
          const uint64_t bd = bdesc + ((T.b[q] * C::B_BYTES + k * 32) >> 4);
          const uint32_t accum = (i == 0 && k == 0 && T.first[q]) ? 0u : 1u;
          mma_bf16(tmem + T.acc[q] * BN, ad, bd, IDESC, accum);
        }
      }
      mma_commit(smem_u32(&empty_bar[s]));
    }
    s_consumed = i;
    mma_commit(smem_u32(&acc_bar));
  }
  __syncwarp();

  // ---- epilogue: thread (warp w, lane l) owns accumulator row 32 w + l
  const bool acc_ok = mbar_wait(smem_u32(&acc_bar), 0, wait);
  fence_after();
  if (!acc_ok) atomicExch(&s_fail, 1);
  const bool ok = acc_ok && nk > 0 && (*(volatile int *)&s_fail == 0);
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const bool rv = row < M;
    const long long roff = rv ? map_off(o.cm, row) : 0;
    const double sa = rv ? o.sa[z * o.ssa + row] : 0.0;
    double *Cz = o.C + z * o.cstride + part * o.pstride;
    // value = (sum_d n_d 2^(6 (kExact - 1 - d))) 2^(-6 (kExact + 1)) + small
    const double unit = ldexp(1.0, -kXsBits * (T.kExact + 1));
    const uint32_t trow = static_cast<uint32_t>(warp * 32) << 16;
#pragma unroll 1
    for (int c = 0; c < BN / 16; ++c) {
      if (n0 + c * 16 >= N) break;
      long long acc[16];
      uint32_t r[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = 0;
#pragma unroll
      for (int d = 0; d < T.kExact; ++d) {
        tmem_ld16(tmem + trow + d * BN + c * 16, r);
        // diagonal d holds integers in units of 2^-6(d+2): scale them up exactly
        const float up = ldexpf(1.0f, kXsBits * (d + 2));
#pragma unroll
        for (int j = 0; j < 16; ++j)
          acc[j] = acc[j] * 64 + __float2ll_rn(__uint_as_float(r[j]) * up);
      }
      float small[16];
      if constexpr (T.kAcc > T.kExact) {
        tmem_ld16(tmem + trow + T.kExact * BN + c * 16, r);
#pragma unroll
        for (int j = 0; j < 16; ++j) small[j] = __uint_as_float(r[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) small[j] = 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = n0 + c * 16 + j;
        if (rv && col < N) {
          const double v = fma((double)acc[j], unit, (double)small[j]);
          Cz[roff + map_off(o.cn, col)] = v * sa * o.sb[z * o.ssb + col];
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_fail) atomicMax(err_flag, 2);   // a timeout outranks the non-finite flag (1) it may cause
    for (int i = s_consumed; i < s_issued; ++i)
      (void)mbar_wait(smem_u32(&full_bar[i % STAGES]), (i / STAGES) & 1);
    // the MMAs (acc_bar tracks all of them) finish before the dealloc
    (void)mbar_wait(smem_u32(&acc_bar), 0);
  }
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ---- host side ----------------------------------------------------------

bool make_xs_map(CUtensorMap *m, const XsOperand &op, int box_rows, int row_bytes) {
  auto enc = encode_fn();
  if (!enc) return false;
  const long long bs = op.batch > 1 ? op.bstride : (long long)op.pitch * op.rows * op.S;
  cuuint64_t dims[4] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)op.S,
                        (cuuint64_t)(op.batch < 1 ? 1 : op.batch)};
  cuuint64_t strides[3] = {(cuuint64_t)op.pitch * 2, (cuuint64_t)op.pitch * 2 * op.rows,
                           (cuuint64_t)bs * 2};
  cuuint32_t box[4] = {(cuuint32_t)(row_bytes / 2), (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, op.slices, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int S, int BN>
cudaError_t launch_xs(const XsOperand &A, const XsOperand &B, int M, int N, int K,
                      const XsOut &o, int ksplit, int *err, cudaStream_t s) {
  using C = XsCfg<S, BN>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_xs_gemm<S, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap ta, tb;
  if (!make_xs_map(&ta, A, C::BM, C::ROW) || !make_xs_map(&tb, B, BN, C::ROW))
    return cudaErrorInvalidValue;
  const int nkb = (K + C::BK - 1) / C::BK;
  const int kbp = (nkb + ksplit - 1) / ksplit;
  if (kbp * C::BK > kXsMaxK) return cudaErrorInvalidValue;
  const int ntn = (N + BN - 1) / BN;
  const int batch = A.batch < 1 ? 1 : A.batch;
  dim3 grid(ntn * ksplit, (M + C::BM - 1) / C::BM, batch);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  const int stall = take_stall(kStallGemm) ? 1 : 0;
  k_xs_gemm<S, BN><<<grid, 128, C::SMEM, s>>>(ta, tb, M, N, K, kbp, ntn, o, err, wait_limit(),
                                              stall);
  return cudaGetLastError();
}

// Tile width: one tile when N fits the accumulators' share of tensor memory,
// else the widest tile that splits N into near-equal parts.
template <int S>
cudaError_t dispatch_xs(const XsOperand &A, const XsOperand &B, int M, int N, int K,
                        const XsOut &o, int ksplit, int *err, cudaStream_t s) {
  constexpr bool wide = XsTable<S>::kAcc * 96 <= 512;
  if (N <= 32) return launch_xs<S, 32>(A, B, M, N, K, o, ksplit, err, s);
  if (N <= 48) return launch_xs<S, 48>(A, B, M, N, K, o, ksplit, err, s);
  if (N <= 64) return launch_xs<S, 64>(A, B, M, N, K, o, ksplit, err, s);
  if (N <= 80) return launch_xs<S, 80>(A, B, M, N, K, o, ksplit, err, s);
  if constexpr (wide) return launch_xs<S, 96>(A, B, M, N, K, o, ksplit, err, s);
  return launch_xs<S, 48>(A, B, M, N, K, o, ksplit, err, s);
}

}  // namespace

cudaError_t xs_split(PSet src, IdxMap rm, IdxMap km, const XsOperand &d, cudaStream_t s) {
  return xs_split_scaled(src, rm, km, PSet{nullptr, nullptr, 0}, 0, d, s);
}

cudaError_t xs_split_scaled(PSet src, IdxMap rm, IdxMap km, PSet kscale, int kmode,
                            const XsOperand &d, cudaStream_t s) {
  if (d.rows <= 0 || d.K <= 0) return cudaSuccess;
  if (d.S < 1 || d.S > kXsMaxSlices || d.pitch < d.K) return cudaErrorInvalidValue;
  const dim3 g((d.rows + 7) / 8, 1, d.batch < 1 ? 1 : d.batch);
  if (g.z > 65535u) return cudaErrorInvalidConfiguration;
  __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(d.slices);
  if (rm.s0 == 1 && rm.n0 >= d.rows && km.s0 != 1 && d.K <= kXsStagedK) {
    const dim3 gs((d.rows + 31) / 32, 1, d.batch < 1 ? 1 : d.batch);
    switch (d.S) {
#define XS_STAGED_CASE(SS)                                                                    \
  case SS:                                                                                    \
    k_xs_split_staged<SS><<<gs, 256, 0, s>>>(src, d.rows, d.K, rm, km, dst, d.pitch, d.bstride, \
                                             d.scale, d.sstride, kscale, kmode);              \
    break;
      XS_STAGED_CASE(1) XS_STAGED_CASE(2) XS_STAGED_CASE(3) XS_STAGED_CASE(4)
      XS_STAGED_CASE(5) XS_STAGED_CASE(6) XS_STAGED_CASE(7) XS_STAGED_CASE(8)
#undef XS_STAGED_CASE
    }
    return cudaGetLastError();
  }
  if (d.K >= 256) {
    const dim3 gr(d.rows, 1, d.batch < 1 ? 1 : d.batch);
    switch (d.S) {
#define XS_ROW_CASE(SS)                                                                       \
  case SS:                                                                                    \
    k_xs_split_row<SS><<<gr, 256, 0, s>>>(src, d.rows, d.K, rm, km, dst, d.pitch, d.bstride,  \
                                          d.scale, d.sstride, kscale, kmode);                 \
    break;
      XS_ROW_CASE(1) XS_ROW_CASE(2) XS_ROW_CASE(3) XS_ROW_CASE(4)
      XS_ROW_CASE(5) XS_ROW_CASE(6) XS_ROW_CASE(7) XS_ROW_CASE(8)
#undef XS_ROW_CASE
    }
    return cudaGetLastError();
  }
  switch (d.S) {
#define XS_SPLIT_CASE(SS)                                                                     \
  case SS:                                                                                    \
    k_xs_split<SS><<<g, 256, 0, s>>>(src, d.rows, d.K, rm, km, dst, d.pitch, d.bstride,       \
                                     d.scale, d.sstride, kscale, kmode);                      \
    break;
    XS_SPLIT_CASE(1) XS_SPLIT_CASE(2) XS_SPLIT_CASE(3) XS_SPLIT_CASE(4)
    XS_SPLIT_CASE(5) XS_SPLIT_CASE(6) XS_SPLIT_CASE(7) XS_SPLIT_CASE(8)
#undef XS_SPLIT_CASE
  }
  return cudaGetLastError();
}

cudaError_t xs_gemm(const XsOperand &A, const XsOperand &B, int M, int N, int K, double *C,
                    IdxMap cm, IdxMap cn, long long cstride, int ksplit, long long pstride,
                    int *err_flag, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0 || A.K != K || B.K != K || A.rows < M || B.rows < N || A.S != B.S || ksplit < 1)
    return cudaErrorInvalidValue;
  if ((A.batch < 1 ? 1 : A.batch) != (B.batch < 1 ? 1 : B.batch)) return cudaErrorInvalidValue;
  if (A.pitch != xs_pitch(A.pitch) || B.pitch != xs_pitch(B.pitch) || A.pitch < K || B.pitch < K)
    return cudaErrorInvalidValue;
  if ((A.batch > 1 && (A.bstride * 2) % 16) || (B.batch > 1 && (B.bstride * 2) % 16))
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A.slices) & 15) || (reinterpret_cast<uintptr_t>(B.slices) & 15))
    return cudaErrorInvalidValue;
  XsOut o{C, cm, cn, cstride, pstride, A.scale, B.scale, A.sstride, B.sstride};
  switch (A.S) {
    case 4: return dispatch_xs<4>(A, B, M, N, K, o, ksplit, err_flag, s);
    case 5: return dispatch_xs<5>(A, B, M, N, K, o, ksplit, err_flag, s);
    case 6: return dispatch_xs<6>(A, B, M, N, K, o, ksplit, err_flag, s);
    case 7: return dispatch_xs<7>(A, B, M, N, K, o, ksplit, err_flag, s);
    case 8: return dispatch_xs<8>(A, B, M, N, K, o, ksplit, err_flag, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hotrg

namespace hotrg {
namespace {

__global__ void k_xs_sum_parts(const double *parts, int nparts, long long pstride, int M, int N,
                               double *C, long long ldc) {
  const long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int p = 0; p < nparts; ++p) v += parts[p * pstride + e];
    C[(e / N) * ldc + e % N] = v;
  }
}

}  // namespace

cudaError_t xs_sum_parts(const double *parts, int nparts, long long pstride, int M, int N,
                         double *C, long long ldc, cudaStream_t s) {
  const long long total = (long long)M * N;
  long long b = (total + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  k_xs_sum_parts<<<(int)(b < 1 ? 1 : b), 256, 0, s>>>(parts, nparts, pstride, M, N, C, ldc);
  return cudaGetLastError();
}

}  // namespace hotrg

namespace hotrg {
namespace {

// C(cm(m) + cn(n)) of instance z = sum_p parts[((p * batch + z) * M + m) * N + n]
__global__ void k_xs_scatter_parts(const double *parts, int nparts, int batch, int M, int N,
                                   double *C, IdxMap cm, IdxMap cn, long long bC) {
  const int z = blockIdx.y;
  const long long mn = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int p = 0; p < nparts; ++p) v += parts[((long long)p * batch + z) * mn + e];
    const long long m = e / N, n = e % N;
    C[z * bC + map_off(cm, m) + map_off(cn, n)] = v;
  }
}

}  // namespace

void xs_gemm_needs(int M, int N, int K, int S, int batch, long long need[5]) {
  const int ks = xs_min_split(K);
  need[0] = xs_elems(M, K, S) * batch;
  need[1] = xs_elems(N, K, S) * batch;
  need[2] = (long long)M * batch;
  need[3] = (long long)N * batch;
  need[4] = ks > 1 ? (long long)ks * batch * M * N : 0;
}

cudaError_t gemm_xs(const MappedGemm &g, int S, const XsWork &w, int *err_flag, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const int batch = g.batch < 1 ? 1 : g.batch;
  long long need[5];
  xs_gemm_needs(g.M, g.N, g.K, S, batch, need);
  if (need[0] > w.cap_a || need[1] > w.cap_b || need[2] > w.cap_sa || need[3] > w.cap_sb ||
      need[4] > w.cap_parts)
    return cudaErrorInvalidValue;
  const long long ea = xs_elems(g.M, g.K, S), eb = xs_elems(g.N, g.K, S);
  XsOperand a{w.sa, w.sca, g.M, g.K, xs_pitch(g.K), S, batch, ea, g.M};
  XsOperand b{w.sb, w.scb, g.N, g.K, xs_pitch(g.K), S, batch, eb, g.N};
  // a batch of instances at stride bA is the PSet "problem z at A + z bA"
  const PSet pa{const_cast<double *>(g.A), const_cast<double *>(g.A) + g.bA, 2 * g.bA};
  const PSet pb{const_cast<double *>(g.B), const_cast<double *>(g.B) + g.bB, 2 * g.bB};
  cudaError_t e;
  if ((e = xs_split(pa, g.am, g.ak, a, s)) || (e = xs_split(pb, g.bn, g.bk, b, s))) return e;
  const int ks = xs_min_split(g.K);
  if (ks == 1) return xs_gemm(a, b, g.M, g.N, g.K, g.C, g.cm, g.cn, g.bC, 1, 0, err_flag, s);
  const long long mn = (long long)g.M * g.N;
  if ((e = xs_gemm(a, b, g.M, g.N, g.K, w.parts, map1(g.N), map1(1), mn, ks, mn * batch,
                   err_flag, s)))
    return e;
  long long blocks = (mn + 255) / 256;
  const long long cap = (152LL * 8 + batch - 1) / batch;
  if (blocks > cap) blocks = cap;
  k_xs_scatter_parts<<<dim3((unsigned)(blocks < 1 ? 1 : blocks), batch), 256, 0, s>>>(
      w.parts, ks, batch, g.M, g.N, g.C, g.cm, g.cn, g.bC);
  return cudaGetLastError();
}

}  // namespace hotrg
