// FP64-accurate products on the bf16 tensor cores from exact integer slices
// (an Ozaki-style error-free splitting: Ozaki, Ogita, Rump, Oishi, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012):
//
//   L = diag(mu) sum_t 2^{-8t} A_t,  R = (sum_u 2^{-8u} B_u) diag(nu),
//   L R ~= diag(mu) [ sum_{t+u <= s+1} 2^{-8(t+u)} A_t B_u ] diag(nu),
//
// with powers of two mu_i >= max_k |L_ik|, nu_j >= max_k |R_kj| and integer
// slices |A_t|, |B_u| <= 255 stored as bf16 (exact: at most 8 significant
// bits).  One slice product over a K chunk of 256 sums at most 256 * 255^2 =
// 16,646,400 < 2^24 in magnitude, so the tensor core's f32 accumulation of
// integers is exact; the epilogue moves each chunk's result into int32
// registers (exact) and flushes the running integer sum of one level
// d = t + u into the FP64 output as D += s mu_i nu_j 2^{-8d} S, every 128
// rounds (128 * 16,646,400 < 2^31) or when the level changes.
//
// Kernel layout: CTA pairs (tcgen05 cta_group::2), 256 x 128 output tiles
// (CTA r: rows m0 + 128 r.., and R columns n0 + 64 r.. staged; its TMEM holds
// its 128 rows x 128 columns), 576 threads: warp 0 TMA producer, warp 1 TMEM
// allocation and (CTA 0) the MMA issuer, warps 2..17 epilogue (TMEM lane
// quarter warp % 4, column quarter (warp - 2) / 4: one row of 32 columns per
// thread, whose int32 sums live in registers; eighteen warps leave 96
// registers a thread, the register file being split over the SM's four
// sub-partitions).  A tile runs npairs * ceil(K / 256) rounds; each round is four
// 64-deep stages (L slice 128 x 64, R slice 64 x 64, 24 KiB per CTA) into one
// of four TMEM accumulators (all 512 columns), so the MMAs run up to three
// rounds ahead of the epilogue.  Synchronisation and bounded waits as in the pair kernel (gemm_tc2.cu).
#include "internal.h"
#include "ptx.cuh"

namespace nsgb {

namespace {

constexpr int kEpiWarps = 16;
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr int kRows = 128;
constexpr int kCols = 128;
constexpr int kHalfCols = 64;   // R columns staged by each CTA of the pair
constexpr int kColsPer = 32;    // output columns per epilogue thread
constexpr int kBK = 64;
constexpr int kChunk = 256;
constexpr int kABytes = kRows * kBK * 2;      // 16 KiB
constexpr int kBBytes = kHalfCols * kBK * 2;  // 8 KiB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kStages = 8;
constexpr int kAcc = 4;  // TMEM accumulators: the MMAs run up to three rounds ahead of the epilogue
constexpr uint32_t kTmemCols = kAcc * kCols;  // all 512 columns
constexpr int kBarBytes = 256;
constexpr int kSmem = kStages * kStageBytes + kBarBytes + 1024;
constexpr int kFlushRounds = 128;
static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
static_assert((2 * kStages + 2 * kAcc + 1) * 8 + 8 <= kBarBytes, "barrier area");

// Named barrier 2 over the epilogue warps with an AND over their votes: every
// epilogue thread learns whether all of them may go on (the waits before it
// are bounded, so every thread reaches it and the warps stop together).
__device__ __forceinline__ bool epi_all(bool ok) {
  uint32_t all;
  asm volatile(
      "{\n\t.reg .pred q, r;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred r, 2, %2, q;\n\t"
      "selp.u32 %0, 1, 0, r;\n\t}"
      : "=r"(all)
      : "r"(ok ? 1u : 0u), "r"(kEpiWarps * 32)
      : "memory");
  return all != 0;
}

__device__ __forceinline__ void spin_ns(uint64_t ns) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0; it < 0x10000000u; ++it)
    if (globaltimer_ns() - t0 > ns) break;
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_oz(const __grid_constant__ OzParams p) {
  const int rank = static_cast<int>(cluster_ctarank());
  const int first = blockIdx.x / 2;
  const int stride = gridDim.x / 2;
  const int nchunks = (p.K + kChunk - 1) / kChunk;
  const int rounds = p.npairs * nchunks;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* tfull = bars + 2 * kStages;
  uint64_t* tempty = tfull + kAcc;
  uint64_t* drain = tempty + kAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < kAcc; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 2);  // one arrival per CTA once its epilogue warps have read the accumulator
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
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint64_t tlim = p.timeout_ns;
  const uint32_t full0 = mapa_u32(smem_u32(full), 0);
  const uint32_t tempty0 = mapa_u32(smem_u32(tempty), 0);

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producers (both CTAs)
    for (int q = 0; q < p.slices; ++q) {
      tma_prefetch_desc(&p.L[q]);
      tma_prefetch_desc(&p.R[q]);
    }
    int armed[kStages];
    for (int s = 0; s < kStages; ++s) armed[s] = -1;
    int stage = 0;
    uint32_t phase = 0;
    int it = 0;
    bool ok = true;
    for (int w = first; w < p.total_tiles && ok; w += stride) {
      const int m0 = ((w / p.tiles_n) * 2 + rank) * kRows;
      const int nb = (w % p.tiles_n) * kCols + rank * kHalfCols;
      for (int r = 0; r < rounds && ok; ++r) {
        const int pr = r / nchunks, c = r % nchunks;
        const CUtensorMap* ml = &p.L[p.pair_t[pr] - 1];
        const CUtensorMap* mr = &p.R[p.pair_u[pr] - 1];
        for (int kb = 0; kb < kChunk / kBK; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, tlim, abort_flag)) {
            ok = false;
            break;
          }
          if (it != p.debug_stall_iter) {
            if (rank == 0) {
              mbar_arrive_expect_tx(&full[stage], 2 * kStageBytes);
              armed[stage] = static_cast<int>(phase);
            }
            const uint32_t bar = full0 + static_cast<uint32_t>(stage * 8);
            uint8_t* a = sA + stage * kABytes;
            uint8_t* b = sB + stage * kBBytes;
            const int x = c * kChunk + kb * kBK;  // past K the boxes read zeros
            tma_load_2d_pair(a, ml, bar, x, m0);
            tma_load_2d_pair(a + 8192, ml, bar, x, m0 + 64);
            tma_load_2d_pair(b, mr, bar, nb, x);
          }
          ++it;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, DEV_TIMEOUT);
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
    constexpr uint32_t idesc = make_idesc_bf16(2 * kRows, kCols, 0, 1);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    bool issued = false;
    for (int w = first; w < p.total_tiles && ok; w += stride) {
      for (int r = 0; r < rounds && ok; ++r) {
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, tlim, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kCols);
        uint32_t accumulate = 0;
        for (int kb = 0; kb < kChunk / kBK; ++kb) {
          if (!mbar_wait(&full[stage], phase, tlim, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(sA + stage * kABytes);
          const uint32_t b_base = smem_u32(sB + stage * kBBytes);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const uint64_t ad = make_sdesc(a_base + 32u * k, 16u, 1024u);
            const uint64_t bd = make_sdesc(b_base + 2048u * k, 8192u, 1024u);
            tc_mma_bf16_pair(d_tmem, ad, bd, idesc, accumulate);
            accumulate = 1;
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
        if (++acc == kAcc) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, DEV_TIMEOUT);
      if (issued) {
        volatile int never = 0;
        tc_commit_pair(drain);
        mbar_wait(drain, 0, 100000000ull, &never);
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int q = warp & 3;              // TMEM lane quarter
    const int h = (warp - 2) >> 2;       // column quarter of the tile
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int w = first; w < p.total_tiles && ok; w += stride) {
      const int row = ((w / p.tiles_n) * 2 + rank) * kRows + q * 32 + lane;
      const int col0 = (w % p.tiles_n) * kCols + h * kColsPer;
      const double mu = row < p.M ? p.mu[row] : 0.0;
      int s32[kColsPer];
#pragma unroll
      for (int j = 0; j < kColsPer; ++j) s32[j] = 0;
      int since = 0;
      for (int r = 0; r < rounds; ++r) {
        const bool got = mbar_wait(&tfull[acc], acc_phase, tlim, abort_flag);
        if (!epi_all(got)) {  // all epilogue warps stop at the same round
          *abort_flag = 1;
          if (!got) atomicExch(p.err, DEV_TIMEOUT);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tq = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                            static_cast<uint32_t>(acc * kCols + h * kColsPer);
#pragma unroll
        for (int part = 0; part < kColsPer / 16; ++part) {
          uint32_t v[16];
          tmem_ld_32x32b_x16(tq + 16u * part, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) s32[16 * part + j] += __float2int_rn(__uint_as_float(v[j]));
        }
        // all sixteen epilogue warps are done with this accumulator: one
        // arrival per CTA (a cluster-scope release per warp and round stalled
        // the warps on memory barriers).  No thread can leave between the
        // vote above and this barrier.
        tc_fence_before();
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
        if (threadIdx.x == 64) {
          if (rank == 0)
            mbar_arrive(&tempty[acc]);
          else
            mbar_arrive_cluster(tempty0 + static_cast<uint32_t>(acc * 8));
        }
        if (++acc == kAcc) {
          acc = 0;
          acc_phase ^= 1u;
        }
        ++since;
        const int pr = r / nchunks;
        const int d = p.pair_t[pr] + p.pair_u[pr];
        const bool last = r + 1 == rounds;
        const int dn = last ? 0 : p.pair_t[(r + 1) / nchunks] + p.pair_u[(r + 1) / nchunks];
        if (last || dn != d || since == kFlushRounds) {
          if (row < p.M) {
            const double sc = p.s * mu * ldexp(1.0, -8 * d);
            double* drow = p.D + static_cast<int64_t>(row) * p.ldd;
#pragma unroll
            for (int j = 0; j < kColsPer; ++j) {
              const int col = col0 + j;
              if (col < p.N) drow[col] += sc * p.nu[col] * static_cast<double>(s32[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < kColsPer; ++j) s32[j] = 0;
          since = 0;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kTmemCols);
  }
  cluster_sync_all();
}

// ---------------------------------------------------------------- slicing
// Power-of-two scale of each row (one warp per row): 2^e with max |x| = m 2^e,
// m in [0.5, 1); 1 for an all-zero row.
__global__ void k_oz_row_scale(const double* __restrict__ X, int64_t ld, int rows, int cols, double* __restrict__ mu) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  double m = 0.0;
  for (int c = lane; c < cols; c += 32) m = fmax(m, fabs(X[static_cast<int64_t>(row) * ld + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int e = 0;
    frexp(m, &e);
    mu[row] = m > 0.0 ? ldexp(1.0, e) : 1.0;
  }
}

// The same per column (one thread per column, rows walked in order).
__global__ void k_oz_col_scale(const double* __restrict__ X, int64_t ld, int rows, int cols, double* __restrict__ nu) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= cols) return;
  double m = 0.0;
  for (int r = 0; r < rows; ++r) m = fmax(m, fabs(X[static_cast<int64_t>(r) * ld + col]));
  int e = 0;
  frexp(m, &e);
  nu[col] = m > 0.0 ? ldexp(1.0, e) : 1.0;
}

// Integer slices of X / scale (scale per row if by_row, else per column):
// x <- 256 x, S_t = trunc(x), x <- x - S_t for t = 1..s, every step exact;
// slice t at out + (t - 1) * slice_stride, row-major with leading dimension ldo.
__global__ void k_oz_slice(const double* __restrict__ X, int64_t ld, int rows, int cols,
                           const double* __restrict__ scale, int by_row, int s, bf16* __restrict__ out, int64_t ldo,
                           int64_t slice_stride) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    double x = X[r * ld + c] / scale[by_row ? r : c];
    bf16* o = out + r * ldo + c;
    for (int t = 0; t < s; ++t) {
      x *= 256.0;
      const double a = trunc(x);
      x -= a;
      o[t * slice_stride] = __float2bfloat16_rn(static_cast<float>(a));
    }
  }
}

// D = beta C + gamma I (C may be null), the starting value the product adds into.
__global__ void k_oz_init(double* __restrict__ D, int64_t ldd, const double* __restrict__ C, int64_t ldc, double beta,
                          double gamma, int rows, int cols) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    double v = (C != nullptr && beta != 0.0) ? beta * C[r * ldc + c] : 0.0;
    if (r == c) v += gamma;
    D[r * ldd + c] = v;
  }
}

int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : static_cast<int>(g);
}

}  // namespace

cudaError_t launch_oz_prepare(const double* X, int64_t ld, int rows, int cols, bool by_row, int s, double* scale,
                              bf16* out, int64_t ldo, int64_t slice_stride, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (by_row)
    k_oz_row_scale<<<(rows + 7) / 8, 256, 0, st>>>(X, ld, rows, cols, scale);
  else
    k_oz_col_scale<<<(cols + 255) / 256, 256, 0, st>>>(X, ld, rows, cols, scale);
  k_oz_slice<<<grid_for(static_cast<int64_t>(rows) * cols), 256, 0, st>>>(X, ld, rows, cols, scale, by_row ? 1 : 0,
                                                                           s, out, ldo, slice_stride);
  return cudaGetLastError();
}

cudaError_t launch_oz_init(double* D, int64_t ldd, const double* C, int64_t ldc, double beta, double gamma, int rows,
                           int cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_oz_init<<<grid_for(static_cast<int64_t>(rows) * cols), 256, 0, st>>>(D, ldd, C, ldc, beta, gamma, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_gemm_oz(const OzParams& p, int num_sms, cudaStream_t s) {
  static int max_clusters = -1;
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
  if (max_clusters < 0) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2 * (num_sms / 2));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k_gemm_oz, &cfg);
    if (e != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = num_sms / 2;
    }
    max_clusters = n;
  }
  if (p.total_tiles <= 0) return cudaSuccess;
  const int clusters = p.total_tiles < max_clusters ? p.total_tiles : max_clusters;
  cfg.gridDim = dim3(2 * clusters);
  return cudaLaunchKernelEx(&cfg, k_gemm_oz, p);
}

}  // namespace nsgb
