// CTA-pair variant of the persistent bf16 / split-bf16 GEMM (same fused
// epilogue as the one-CTA kernel: D = s L R + beta C + gamma I, f32 + bf16
// hi/lo outputs, per-tile partial sums of D^2).
//
// The two CTAs of a cluster of two form one tcgen05 MMA unit (cta_group::2):
// a work item is a 256 x 256 output tile; CTA r (r = 0, 1) stages the L rows
// m0 + 128r ... m0 + 128r + 127 and the R columns n0 + 128r ... n0 + 128r + 127
// in its own shared memory, and one thread of CTA 0 issues M = 256, N = 256
// MMAs that read both halves of both operands and accumulate rows
// m0 + 128r ... into the TMEM of CTA r.  Per SM this halves the R bytes a
// K-slice needs (16 + 16 KiB instead of 16 + 32 KiB for 128 x 256 outputs),
// so six stages fit next to the epilogue buffers instead of four, and the
// shared-memory ring covers 1.5x longer load latency at the same tensor rate.
//
// Synchronisation (all barriers live at the same offsets in both CTAs):
//   full[s]   CTA 0 only: one arrive.expect_tx of both CTAs' stage bytes; the
//             loads of both CTAs complete their bytes on it
//   empty[s]  both CTAs: the MMA commit multicasts one arrival to each
//   tfull[a]  both CTAs: accumulator a holds a finished tile (multicast commit)
//   tempty[a] CTA 0 only: one arrival per epilogue warp of either CTA (8)
// Every wait is bounded; a CTA that gives up raises its abort flag, records
// NS_ERR_TIMEOUT and unwinds, and its peer's waits then run out in turn.
// Both CTAs meet at a cluster barrier before the pair's TMEM is released and
// again before exit, so no arrival or load targets a CTA that has left.
//
// Wave balance: with T tiles on C clusters, a last wave of T mod C tiles
// leaves most clusters idle while it runs.  When 2 (T mod C) <= C those tiles
// run as two half-width items each (256 x 128, MMA N = 128, 64 R columns per
// CTA), which halves the last wave.  The partial sums of D^2 keep two slots of
// four per tile (one per half; a whole tile writes 0 to the second).
//
// Shared-memory layouts per CTA are those of the one-CTA kernel with 128 R
// columns: one pass -- L 128 x 64 (128-byte swizzle), R 64 x 128 as two 8 KiB
// chunks of 64 columns (32 KiB per stage, 6 stages); split products with NP
// parts per operand (NP = 2: hi, lo -- the bf16x3 terms; NP = 3: hi, lo, lo2
// -- the bf16x6 terms hi.hi, hi.lo, lo.hi, hi.lo2, lo.lo, lo2.hi) -- per
// 32-deep K slice, part p of L (128 x 32, 64-byte swizzle) and of R (32 x 128
// as two 4 KiB chunks) at p x 8 KiB: 32 KiB per stage and 6 stages for NP = 2,
// 48 KiB and 4 stages for NP = 3.
#include <mutex>
#include <cstdio>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace nsgb {

namespace {

constexpr int kRows = 128;     // output rows per CTA (256 per pair)
constexpr int kCols = 256;     // output columns per pair tile
constexpr int kHalf = kCols / 2;  // R columns staged by each CTA
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 2 * kCols;  // two accumulators of 128 lanes x 256 columns
constexpr int kBarBytes = 256;
constexpr int kEpiStride = 36;
constexpr int kEpiBytes = 4 * 32 * kEpiStride * 4;
constexpr int kPartBytes = 8192;  // one split part of a 32-deep K slice (L or R)

// Split term t as (L part, R part), in issue order: hi.hi, hi.lo, lo.hi,
// hi.lo2, lo.lo, lo2.hi; bf16x3 uses the first three.
__host__ __device__ constexpr int term_l(int t) { return (t == 2 || t == 4) ? 1 : (t == 5 ? 2 : 0); }
__host__ __device__ constexpr int term_r(int t) { return (t == 1 || t == 4) ? 1 : (t == 3 ? 2 : 0); }

// NP = 4: one TF32 pass; per CTA a stage holds L 128 rows x 32 K and 128 of
// the tile's R columns x 32 K, both as f32 words K-major (the transposed TF32
// form of R), 128-byte swizzle: 16 + 16 KiB.
// NP = 5: the two split terms hi.hi + lo.hi (L split, R's hi part only), for
// products whose R operand may lose its low part; per 32-deep K slice L hi
// and lo and R hi: 16 + 8 KiB.
template <int NP>
struct PairCfg {
  static constexpr int kLParts = NP == 5 ? 2 : ((NP == 1 || NP == 4) ? 1 : NP);  // split parts staged
  static constexpr int kRParts = NP == 5 ? 1 : kLParts;
  static constexpr int kBK = NP == 1 ? 64 : 32;          // K per stage
  static constexpr int kABytes = (NP == 1 || NP == 4) ? 16384 : kLParts * kPartBytes;
  static constexpr int kBBytes = (NP == 1 || NP == 4) ? 16384 : kRParts * kPartBytes;  // 128 of the tile's R columns
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = (196 * 1024) / kStageBytes > 6 ? 6 : (196 * 1024) / kStageBytes;
  static constexpr int kTerms = (NP == 1 || NP == 4) ? 1 : (NP == 2 ? 3 : (NP == 5 ? 2 : 6));
  static constexpr int kSmem = kStages * kStageBytes + kBarBytes + kEpiBytes + 1024;
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
  static_assert((3 * kStages + 5) * 8 + 8 <= kBarBytes, "barrier area");
};

// Work item w: problem, tile row (128-row units, this CTA's half of the pair
// tile), tile column, and which half of the tile's columns (-1: all 256).
__device__ __forceinline__ void pair_item(const TcParams& p, int w, int rank, int& pi, int& mt, int& nt, int& half) {
  const int split_from = p.total_tiles - p.pair_tail;
  int tile = w;
  half = -1;
  if (w >= split_from) {
    tile = split_from + ((w - split_from) >> 1);
    half = (w - split_from) & 1;
  }
  tc::decode_item(p, tile, rank, 2, pi, mt, nt);
}

__device__ __forceinline__ void spin_ns(uint64_t ns) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0; it < 0x10000000u; ++it)
    if (globaltimer_ns() - t0 > ns) break;
}

template <int NP>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc2(const __grid_constant__ TcParams p) {
  using Cfg = PairCfg<NP>;
  constexpr int kStages = Cfg::kStages, kABytes = Cfg::kABytes, kBBytes = Cfg::kBBytes, kBK = Cfg::kBK;
  // host-side guarantees, checked once more before any barrier: list mode and
  // multi-pass one-split products are not supported by the pair kernel
  if (p.gprob != nullptr || ((NP == 1 || NP == 4) && p.npass != 1)) {
    if (threadIdx.x == 0) atomicExch(p.err, DEV_TIMEOUT);
    return;
  }
  const int rank = static_cast<int>(cluster_ctarank());
  const int first = blockIdx.x / 2;
  const int stride = gridDim.x / 2;
  const int items = p.total_tiles + p.pair_tail;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* tfull = bars + 2 * kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* ebuf = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + kBarBytes);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 8);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_barrier_init();
    fence_proxy_async_smem();
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  // the peer's loads and arrivals target CTA 0's barriers: both must exist first
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint64_t tlim = p.timeout_ns;
  // CTA 0's full and tempty barriers in the cluster shared window
  const uint32_t full0 = mapa_u32(smem_u32(full), 0);
  const uint32_t tempty0 = mapa_u32(smem_u32(tempty), 0);

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producers (both CTAs)
    for (int i = 0; i < p.nprob; ++i) {
      for (int q = 0; q < Cfg::kLParts; ++q) tma_prefetch_desc(&p.prob[i].L[q]);
      for (int q = 0; q < Cfg::kRParts; ++q) tma_prefetch_desc(&p.prob[i].R[q]);
    }
    int armed[kStages];
    for (int s = 0; s < kStages; ++s) armed[s] = -1;
    int stage = 0;
    uint32_t phase = 0;
    int it = 0;
    bool ok = true;
    for (int w = first; w < items && ok; w += stride) {
      int pi, mt, nt, half;
      pair_item(p, w, rank, pi, mt, nt, half);
      const TcProblem& P = p.prob[pi];
      const int m0 = mt * kRows;                       // this CTA's L rows
      const int cw = half < 0 ? kHalf : kHalf / 2;     // R columns this CTA stages
      const int nb = nt * kCols + (half > 0 ? kHalf : 0) + rank * cw;
      const uint32_t tx = 2u * static_cast<uint32_t>(kABytes + (half < 0 ? kBBytes : kBBytes / 2));  // both CTAs
      const int nkb = (P.K + kBK - 1) / kBK;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(&empty[stage], phase ^ 1u, tlim, abort_flag)) {
          ok = false;
          break;
        }
        if (it != p.debug_stall_iter) {
          if (rank == 0) {
            mbar_arrive_expect_tx(&full[stage], tx);
            armed[stage] = static_cast<int>(phase);
          }
          const uint32_t bar = full0 + static_cast<uint32_t>(stage * 8);
          uint8_t* a = sA + stage * kABytes;
          uint8_t* b = sB + stage * kBBytes;
          if (NP == 4) {
            const int x = kb * kBK;
            tma_load_2d_pair(a, &P.L[0], bar, x, m0);
            tma_load_2d_pair(a + 8192, &P.L[0], bar, x, m0 + 64);
            tma_load_2d_pair(b, &P.R[0], bar, x, nb);
            if (half < 0) tma_load_2d_pair(b + 8192, &P.R[0], bar, x, nb + 64);
          } else if (NP > 1) {
            const int x = kb * kBK;
#pragma unroll
            for (int part = 0; part < Cfg::kLParts; ++part) {
              tma_load_2d_pair(a + part * kPartBytes, &P.L[part], bar, x, m0);
              tma_load_2d_pair(a + part * kPartBytes + 4096, &P.L[part], bar, x, m0 + 64);
            }
#pragma unroll
            for (int part = 0; part < Cfg::kRParts; ++part) {
              tma_load_2d_pair(b + part * kPartBytes, &P.R[part], bar, nb, x);
              if (half < 0) tma_load_2d_pair(b + part * kPartBytes + 4096, &P.R[part], bar, nb + 64, x);
            }
          } else {
            const int x = kb * kBK;
            tma_load_2d_pair(a, &P.L[0], bar, x, m0);
            tma_load_2d_pair(a + 8192, &P.L[0], bar, x, m0 + 64);
            tma_load_2d_pair(b, &P.R[0], bar, nb, x);
            if (half < 0) tma_load_2d_pair(b + 8192, &P.R[0], bar, nb + 64, x);
          }
        }
        ++it;
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, DEV_TIMEOUT);
      // let the loads in flight land before the CTA can leave: CTA 0 waits
      // (bounded) for the stages it armed, which also count the peer's bytes;
      // the peer's loads signal CTA 0's barriers, so it waits out a grace period
      volatile int never = 0;
      if (rank == 0) {
        for (int s = 0; s < kStages; ++s)
          if (armed[s] >= 0) mbar_wait(&full[s], static_cast<uint32_t>(armed[s]), 100000000ull, &never);
      } else {
        spin_ns(2000000ull);
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------ MMA issuer (CTA 0)
    constexpr uint32_t idesc_full =
        NP == 4 ? make_idesc_tf32(2 * kRows, kCols) : make_idesc_bf16(2 * kRows, kCols, 0, 1);
    constexpr uint32_t idesc_half =
        NP == 4 ? make_idesc_tf32(2 * kRows, kCols / 2) : make_idesc_bf16(2 * kRows, kCols / 2, 0, 1);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    bool issued = false;
    for (int w = first; w < items && ok; w += stride) {
      int pi, mt, nt, half;
      pair_item(p, w, 0, pi, mt, nt, half);
      const TcProblem& P = p.prob[pi];
      const int nkb = (P.K + kBK - 1) / kBK;
      const uint32_t idesc = half < 0 ? idesc_full : idesc_half;
      if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, tlim, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kCols);
      uint32_t accumulate = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(&full[stage], phase, tlim, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_u32(sA + stage * kABytes);
        const uint32_t b_base = smem_u32(sB + stage * kBBytes);
        if (NP == 4) {
#pragma unroll
          for (int k = 0; k < kBK / 8; ++k) {  // K = 8 per TF32 MMA (32 bytes)
            const uint64_t ad = make_sdesc(a_base + 32u * k, 16u, 1024u);
            const uint64_t bd = make_sdesc(b_base + 32u * k, 16u, 1024u);
            tc_mma_tf32_pair(d_tmem, ad, bd, idesc, accumulate);
            accumulate = 1;
          }
        } else if (NP > 1) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int tt = 0; tt < Cfg::kTerms; ++tt) {
              const int t = NP == 5 ? 2 * tt : tt;  // NP = 5: the terms hi.hi and lo.hi
              const uint64_t ad =
                  make_sdesc(a_base + static_cast<uint32_t>(term_l(t) * kPartBytes) + 32u * k, 16u, 512u, kSwz64);
              const uint64_t bd =
                  make_sdesc(b_base + static_cast<uint32_t>(term_r(t) * kPartBytes) + 2048u * k, 4096u, 1024u);
              tc_mma_bf16_pair(d_tmem, ad, bd, idesc, accumulate);
              accumulate = 1;
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const uint64_t ad = make_sdesc(a_base + 32u * k, 16u, 1024u);
            const uint64_t bd = make_sdesc(b_base + 2048u * k, 8192u, 1024u);
            tc_mma_bf16_pair(d_tmem, ad, bd, idesc, accumulate);
            accumulate = 1;
          }
        }
        issued = true;
        tc_commit_pair_mc(&empty[stage], 0x3);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      tc_commit_pair_mc(&tfull[acc], 0x3);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, DEV_TIMEOUT);
      if (issued) {
        // all MMAs issued must finish (they write both CTAs' TMEM) before release
        volatile int never = 0;
        tc_commit_pair(drain);
        mbar_wait(drain, 0, 100000000ull, &never);
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int w = first; w < items; w += stride) {
      int pi, mt, nt, half;
      pair_item(p, w, rank, pi, mt, nt, half);
      const TcProblem& P = p.prob[pi];
      const int m0 = mt * kRows, n0 = nt * kCols + (half > 0 ? kHalf : 0);

      bool ok = mbar_wait(&tfull[acc], acc_phase, tlim, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        *abort_flag = 1;
        if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
        break;
      }
      tc_fence_after();
      // whole and half-width tiles as separate constant-width instances
      const uint32_t tq = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(acc * kCols);
      float* wb = ebuf + q * 32 * kEpiStride;
      const float frob = half < 0 ? tc::epilogue_tile<kCols, kEpiStride, NP == 3>(P, m0, n0, q, lane, wb, tq)
                                  : tc::epilogue_tile<kHalf, kEpiStride, NP == 3>(P, m0, n0, q, lane, wb, tq);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty0 + static_cast<uint32_t>(acc * 8));
      if (P.frob_partials != nullptr && mt < P.tiles_m) {
        double f = static_cast<double>(frob);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0) {
          double* slot = P.frob_partials + (mt * P.tiles_n + nt) * 8 + q;
          slot[half > 0 ? 4 : 0] = f;
          if (half < 0) slot[4] = 0.0;
        }
      }
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // CTA 0's MMAs (which write both TMEMs) are complete or drained, and both
  // epilogues are done reading: the pair's TMEM can go
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kTmemCols);
  }
  cluster_sync_all();
}

template <int NP>
cudaError_t launch_pair(const TcParams& p, int num_sms, cudaStream_t s) {
  constexpr int kSmem = PairCfg<NP>::kSmem;
  static std::once_flag once;  // attribute and occupancy once, safe from several host threads
  static int max_clusters = 0;
  static cudaError_t init = cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  std::call_once(once, [&] {
    init = cudaFuncSetAttribute(k_gemm_tc2<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (init != cudaSuccess) return;
    cudaLaunchConfig_t c = cfg;
    c.gridDim = dim3(2 * (num_sms / 2));
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_gemm_tc2<NP>, &c);
    if (e != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = num_sms / 2;
    }
    max_clusters = n;
  });
  if (init != cudaSuccess) return init;
  if (p.total_tiles <= 0) return cudaSuccess;
  TcParams q = p;
  // a last wave of `tail` tiles on `max_clusters` clusters runs as 2 tail
  // half-width items where they still fit in one wave
  const int tail = p.total_tiles % max_clusters == 0 && p.total_tiles >= max_clusters
                       ? 0
                       : (p.total_tiles > max_clusters ? p.total_tiles % max_clusters : p.total_tiles);
  q.pair_tail = 2 * tail <= max_clusters ? tail : 0;
  const int items = q.total_tiles + q.pair_tail;
  const int clusters = items < max_clusters ? items : max_clusters;
  cfg.gridDim = dim3(2 * clusters);
  return cudaLaunchKernelEx(&cfg, k_gemm_tc2<NP>, q);
}

}  // namespace

cudaError_t launch_gemm_tc_pair(const TcParams& p, int parts, int num_sms, cudaStream_t s) {
  if (p.gprob != nullptr || ((parts == 1 || parts == 4) && p.npass != 1)) return cudaErrorInvalidValue;
  switch (parts) {
    case 1: return launch_pair<1>(p, num_sms, s);
    case 2: return launch_pair<2>(p, num_sms, s);
    case 3: return launch_pair<3>(p, num_sms, s);
    case 4: return launch_pair<4>(p, num_sms, s);
    case 5: return launch_pair<5>(p, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nsgb
