// Persistent grouped bf16 / split-bf16 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands staged by TMA), with the fused
// epilogue every Newton-Schulz product needs:
//
//   D = s * (L R) + beta * C + gamma * I
//
// which covers F = I - A G (s = -1, gamma = 1), X_{j+1} = X_j + X_j P_j
// (beta = 1, C = X_j), P_{j+1} = P_j P_j and T_c + Gamma_c X.  The epilogue
// writes the f32 master of D, its bf16 hi/lo split (the operands of the next
// product) and per-tile partial sums of D^2 (for ||F||_F).
//
// Roles (192 threads, one CTA per SM):
//   warp 0 lane 0   TMA producer: fills a ring of shared-memory stages
//   warp 1          TMEM allocator; lane 0 issues tcgen05.mma for a tile
//   warps 2..5      epilogue: TMEM -> registers -> shared-memory transpose ->
//                   fused math -> coalesced global stores (whole 128-B rows)
// The accumulator is double-buffered in TMEM (2 x BN columns), so the
// epilogue of tile i overlaps the MMAs of tile i+1.
//
// One CTA per tile: every CTA loads its own L and R tiles (no cluster, no
// shared loads); the CTA-pair kernel (gemm_tc2.cu) is the wide-tile form.
//
// Shared-memory layouts (both 128-byte swizzled, atoms of 8 rows x 128 B):
//   L tile 128 x 64 (K-major):  row r at r*128 B; MMA K-slice k at +32k B.
//   R tile 64 x BN (N-major):   BN/64 chunks of 64 K-rows x 64 N-columns,
//                               chunk j at j*8 KiB (LBO), 8-row groups at 1 KiB
//                               (SBO); MMA K-slice k at +2 KiB*k.
//
// Split products (X3): one stage holds all four operand parts of a 32-deep K
// slice -- L_hi, L_lo (128 x 32 each, 64-byte swizzle, 8-row atoms of 512 B)
// and R_hi, R_lo (32 x BN each: BN/64 chunks of 32 K-rows x 128 B at 4 KiB) --
// and issues the 6 products L_hi R_hi, L_hi R_lo, L_lo R_hi of its two K=16
// slices.  Same bytes per stage as one plain pass, 1.5x the tensor work, so
// the ring covers 1.5x more load latency and L2 is read 1/3 less per product.
#include <mutex>
#include <cstdio>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace nsgb {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kThreads = 192;

constexpr uint32_t pow2_cols(int c) { return c <= 32 ? 32u : (c <= 64 ? 64u : (c <= 128 ? 128u : (c <= 256 ? 256u : 512u))); }

template <int BN>
struct TcCfg {
  static constexpr int kABytes = kBM * kBK * 2;  // 16 KiB
  static constexpr int kBBytes = BN * kBK * 2;   // BN * 128 B
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = (196 * 1024) / kStageBytes > 8 ? 8 : (196 * 1024) / kStageBytes;
  static constexpr uint32_t kTmemCols = pow2_cols(2 * BN);
  static constexpr int kBarBytes = 256;
  // epilogue transpose buffers: 4 warps x 32 rows x 36 floats (rows padded to
  // 144 B so that the float4 writes and reads of a quarter-warp hit distinct banks)
  static constexpr int kEpiStride = 36;
  static constexpr int kEpiBytes = 4 * 32 * kEpiStride * 4;
  static constexpr int kSmem = kStages * kStageBytes + kBarBytes + kEpiBytes + 1024;
};

using tc::decode_item;

template <int BN, bool X3>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ TcParams p) {
  using Cfg = TcCfg<BN>;
  constexpr int CM = 1;
  constexpr int rank = 0;
  const int first = blockIdx.x;   // this CTA's first work item
  const int stride = gridDim.x;   // CTAs in the grid
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + Cfg::kStages * Cfg::kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + Cfg::kStages * Cfg::kBBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + Cfg::kStages;
  uint64_t* tfull = bars + 2 * Cfg::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* ebuf = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + Cfg::kBarBytes);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_barrier_init();
    fence_proxy_async_smem();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint64_t tlim = p.timeout_ns;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    for (int i = 0; p.gprob == nullptr && i < p.nprob; ++i) {
      tma_prefetch_desc(&p.prob[i].L[0]);
      tma_prefetch_desc(&p.prob[i].R[0]);
      if (p.npass > 1) {
        tma_prefetch_desc(&p.prob[i].L[1]);
        tma_prefetch_desc(&p.prob[i].R[1]);
      }
    }
    int armed[Cfg::kStages];
    for (int s = 0; s < Cfg::kStages; ++s) armed[s] = -1;
    int stage = 0;
    uint32_t phase = 0;
    int it = 0;
    bool ok = true;
    for (int w = first; w < p.total_tiles && ok; w += stride) {
      int pi, mt, nt;
      decode_item(p, w, rank, CM, pi, mt, nt);
      const TcProblem& P = p.gprob != nullptr ? p.gprob[pi] : p.prob[pi];
      if (p.gprob != nullptr && w + stride < p.total_tiles) {
        // list mode: every item may name another problem, i.e. other tensor
        // maps; warm the descriptors of this CTA's next item
        const TcProblem& Q = p.gprob[p.items[w + stride].prob];
        tma_prefetch_desc(&Q.L[0]);
        tma_prefetch_desc(&Q.R[0]);
        if (X3 || p.npass > 1) {
          tma_prefetch_desc(&Q.L[1]);
          tma_prefetch_desc(&Q.R[1]);
        }
      }
      const int m0 = mt * kBM, n0 = nt * BN;
      const int kstep = X3 ? kBK / 2 : kBK;
      const int nkb = (P.K + kstep - 1) / kstep;
      const int npass = X3 ? 1 : p.npass;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        for (int ps = 0; ps < npass; ++ps) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, tlim, abort_flag)) {
            ok = false;
            break;
          }
          if (X3 && it != p.debug_stall_iter) {
            mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
            armed[stage] = static_cast<int>(phase);
            uint8_t* a = sA + stage * Cfg::kABytes;
            uint8_t* b = sB + stage * Cfg::kBBytes;
            const int x = kb * (kBK / 2);
            tma_load_2d(a, &P.L[0], &full[stage], x, m0);
            tma_load_2d(a + 4096, &P.L[0], &full[stage], x, m0 + 64);
            tma_load_2d(a + 8192, &P.L[1], &full[stage], x, m0);
            tma_load_2d(a + 12288, &P.L[1], &full[stage], x, m0 + 64);
#pragma unroll
            for (int j = 0; j < 2 * (BN / 64); ++j) {
              const int part = j / (BN / 64), c = j % (BN / 64);
              uint8_t* dst = b + part * (BN * 64) + c * 4096;
              tma_load_2d(dst, &P.R[part], &full[stage], n0 + 64 * c, x);
            }
          } else if (!X3 && it != p.debug_stall_iter) {
            const CUtensorMap* ml = &P.L[ps == 2 ? 1 : 0];
            const CUtensorMap* mr = &P.R[ps == 1 ? 1 : 0];
            mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
            armed[stage] = static_cast<int>(phase);
            uint8_t* a = sA + stage * Cfg::kABytes;
            uint8_t* b = sB + stage * Cfg::kBBytes;
            tma_load_2d(a, ml, &full[stage], kb * kBK, m0);
            tma_load_2d(a + 8192, ml, &full[stage], kb * kBK, m0 + 64);
#pragma unroll
            for (int j = 0; j < BN / 64; ++j) tma_load_2d(b + j * 8192, mr, &full[stage], n0 + 64 * j, kb * kBK);
          }
          ++it;
          if (++stage == Cfg::kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, DEV_TIMEOUT);
      // let every load this thread issued land before the CTA exits
      volatile int never = 0;
      for (int s = 0; s < Cfg::kStages; ++s)
        if (armed[s] >= 0) mbar_wait(&full[s], static_cast<uint32_t>(armed[s]), 100000000ull, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idesc = make_idesc_bf16(kBM, BN, 0, 1);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    bool issued = false;
    for (int w = first; w < p.total_tiles && ok; w += stride) {
      int pi, mt, nt;
      decode_item(p, w, rank, CM, pi, mt, nt);
      const TcProblem& P = p.gprob != nullptr ? p.gprob[pi] : p.prob[pi];
      const int kstep = X3 ? kBK / 2 : kBK;
      const int nkb = (P.K + kstep - 1) / kstep;
      const int npass = X3 ? 1 : p.npass;
      if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, tlim, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
      uint32_t accumulate = 0;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        for (int ps = 0; ps < npass; ++ps) {
          if (!mbar_wait(&full[stage], phase, tlim, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(sA + stage * Cfg::kABytes);
          const uint32_t b_base = smem_u32(sB + stage * Cfg::kBBytes);
          if (X3) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              const uint64_t ah = make_sdesc(a_base + 32u * k, 16u, 512u, kSwz64);
              const uint64_t al = make_sdesc(a_base + 8192u + 32u * k, 16u, 512u, kSwz64);
              const uint64_t bh = make_sdesc(b_base + 2048u * k, 4096u, 1024u);
              const uint64_t bl = make_sdesc(b_base + static_cast<uint32_t>(BN * 64) + 2048u * k, 4096u, 1024u);
              tc_mma_bf16(d_tmem, ah, bh, idesc, accumulate);
              accumulate = 1;
              tc_mma_bf16(d_tmem, ah, bl, idesc, 1u);
              tc_mma_bf16(d_tmem, al, bh, idesc, 1u);
            }
          } else {
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
              const uint64_t ad = make_sdesc(a_base + 32u * k, 16u, 1024u);
              const uint64_t bd = make_sdesc(b_base + 2048u * k, 8192u, 1024u);
              tc_mma_bf16(d_tmem, ad, bd, idesc, accumulate);
              accumulate = 1;
            }
          }
          issued = true;
          tc_commit(&empty[stage]);
          if (++stage == Cfg::kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) break;
      tc_commit(&tfull[acc]);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, DEV_TIMEOUT);
      if (issued) {
        // all MMAs this thread issued must finish before TMEM is released
        volatile int never = 0;
        tc_commit(drain);
        mbar_wait(drain, 0, 100000000ull, &never);
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int w = first; w < p.total_tiles; w += stride) {
      int pi, mt, nt;
      decode_item(p, w, rank, CM, pi, mt, nt);
      const TcProblem& P = p.gprob != nullptr ? p.gprob[pi] : p.prob[pi];
      const int m0 = mt * kBM, n0 = nt * BN;
      bool ok = mbar_wait(&tfull[acc], acc_phase, tlim, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        *abort_flag = 1;
        if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
        break;
      }
      tc_fence_after();
      const float frob = tc::epilogue_tile<BN, Cfg::kEpiStride>(
          P, m0, n0, q, lane, ebuf + q * 32 * Cfg::kEpiStride,
          tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(acc * BN));
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      if (P.frob_partials != nullptr && mt < P.tiles_m) {
        double f = static_cast<double>(frob);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0) P.frob_partials[(mt * P.tiles_n + nt) * 4 + q] = f;
      }
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::kTmemCols);
  }
}

template <int BN, bool X3>
cudaError_t launch_bn(const TcParams& p, int num_sms, cudaStream_t s) {
  using Cfg = TcCfg<BN>;
  // once per instantiation, safe from several host threads
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_gemm_tc<BN, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  });
  if (attr != cudaSuccess) return attr;
  const int ctas = p.total_tiles < num_sms ? p.total_tiles : num_sms;
  if (ctas <= 0) return cudaSuccess;
  k_gemm_tc<BN, X3><<<ctas, kThreads, Cfg::kSmem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int tc_tiles(int M, int N, int BN) { return ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN); }

int tc_items(int M, int N, int BN, int CM) {
  if (CM < 0) CM = -CM;  // -2: CTA pairs, counted like clusters of two
  const int tiles_m = (M + kBM - 1) / kBM;
  return ((tiles_m + CM - 1) / CM) * ((N + BN - 1) / BN);
}

cudaError_t launch_gemm_tc(const TcParams& p, int BN, bool x3, int num_sms, cudaStream_t s) {
  if (x3) {
    switch (BN) {
      case 64: return launch_bn<64, true>(p, num_sms, s);
      case 128: return launch_bn<128, true>(p, num_sms, s);
      case 256: return launch_bn<256, true>(p, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (BN) {
    case 64: return launch_bn<64, false>(p, num_sms, s);
    case 128: return launch_bn<128, false>(p, num_sms, s);
    case 192: return launch_bn<192, false>(p, num_sms, s);
    case 256: return launch_bn<256, false>(p, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------ tensor maps
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn get_encode() {
  static const EncodeFn fn = [] {  // initialised once, safe from several host threads
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeFn>(ptr);
    return static_cast<EncodeFn>(nullptr);
  }();
  return fn;
}
}  // namespace

bool encode_bf16_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int role) {
  EncodeFn enc = get_encode();
  if (enc == nullptr) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 2) % 16 != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * 2)};
  // role 0: 64 x 64 box, 128-byte swizzle (either operand, one product pass)
  // role 1: 32 (K) x 64 (rows) box, 64-byte swizzle (L operand of split products)
  // role 2: 64 (N) x 32 (K) box, 128-byte swizzle (R operand of split products)
  cuuint32_t box[2] = {role == 1 ? 32u : 64u, role == 2 ? 32u : 64u};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, role == 1 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_f32_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld) {
  EncodeFn enc = get_encode();
  if (enc == nullptr) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 4) % 16 != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * 4)};
  cuuint32_t box[2] = {32u, 64u};  // 32 f32 = 128 bytes of K, 64 rows
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace nsgb
