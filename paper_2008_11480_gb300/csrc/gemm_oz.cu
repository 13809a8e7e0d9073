// FP64-accurate products on the bf16 tensor cores from exact integer slices
// (the error-free splitting of Ozaki, Ogita, Rump and Oishi, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), with
// signed-digit slices:
//
//   L = diag(2 mu) sum_t 256^{-t} A_t,  R = (sum_u 256^{-u} B_u) diag(2 nu),
//   L R ~= diag(2 mu) [ sum_{d=2}^{s+1} 256^{-d} S_d ] diag(2 nu),
//   S_d = sum_{t+u=d} A_t B_u,
//
// with powers of two mu_i > max_k |L_ik|, nu_j > max_k |R_kj| and digits
// |A_t|, |B_u| <= 128 (round to nearest of 256 x, x in [-1/2, 1/2]), exact in
// bf16.  A level d holds d - 1 slice pairs, so d - 1 products of K_c digits
// sum to at most (d - 1) K_c 2^14 in magnitude: the tensor core's f32
// accumulation is exact while that is <= 2^24, i.e. for K_c <= 1024 / (d - 1).
//
// Kernel (k_gemm_oz): one work item is one level d of one 256 x 256 output
// tile.  CTA pairs (tcgen05 cta_group::2) as in the bf16 pair kernel: CTA r
// stages L rows m0 + 128 r.. and R columns n0 + 128 r.., one thread of CTA 0
// issues M = 256, N = 256 MMAs.  A stage is one slice pair (t, d - t) over 64
// of K -- L_t 128 x 64 and R_{d-t} 64 x 128 per CTA, 32 KiB, the layouts of
// the one-pass bf16 product -- so every slice product reuses its operands as
// a plain bf16 product does.  The stages of one K_c chunk (all pairs of the
// level) accumulate into one of two TMEM accumulators (256 columns each);
// sixteen epilogue warps per CTA move each finished chunk into int32
// registers (exact; 64 columns a thread) while the MMAs fill the other
// accumulator, and write the level's integer sums S_d of the tile to an int32
// plane at the end of the item (|S_d| <= (d - 1) K 2^14 < 2^31 for K <= 16384).
//
// Combine (k_oz_combine, memory bound): D = s (2 mu_i)(2 nu_j) sum_d 256^{-d}
// S_d + beta C + gamma I.  Levels 2..5 and 6..s+1 each combine exactly in
// int64 (shifts of at most 24 bits of values below 2^31), so the sum has two
// roundings to binary64 and one more in the final scaled add; the FP64 work
// (slow on this part) is a few operations per output element, once.
#include <mutex>
#include "internal.h"
#include "ptx.cuh"

namespace nsgb {

namespace {

constexpr int kEpiWarps = 16;
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr int kRows = 128;     // output rows per CTA (256 per pair tile)
constexpr int kCols = 256;     // output columns per pair tile
constexpr int kHalf = 128;     // R columns staged by each CTA
constexpr int kColsPer = 64;   // output columns per epilogue thread
constexpr int kBK = 64;
constexpr int kABytes = kRows * kBK * 2;  // 16 KiB
constexpr int kBBytes = kHalf * kBK * 2;  // 16 KiB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kStages = 6;
constexpr uint32_t kTmemCols = 2 * kCols;  // two accumulators, all 512 columns
constexpr int kBarBytes = 256;
constexpr int kSmem = kStages * kStageBytes + kBarBytes + 1024;
static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
static_assert((2 * kStages + 5) * 8 + 8 <= kBarBytes, "barrier area");

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

// Work item w: level index (into p.lev_d), pair-tile row (256-row units) and
// tile column (256-column units).  Within a level the tiles run in bands of
// kBand tile rows, column by column inside a band, so that the items in
// flight at once (one per CTA pair) share both their L row panels and their
// R column panels in L2 (row-major order would share only the L panels).
constexpr int kBand = 8;
__device__ __forceinline__ void oz_item(const OzParams& p, int w, int& lev, int& mt2, int& nt) {
  const int per = p.tiles_m2 * p.tiles_n;
  lev = w / per;
  const int t = w - lev * per;
  const int band = t / (kBand * p.tiles_n);
  const int rows = min(kBand, p.tiles_m2 - band * kBand);
  const int idx = t - band * kBand * p.tiles_n;
  mt2 = band * kBand + idx % rows;
  nt = idx / rows;
}

// Slice pairs of level d: t = t_lo .. t_hi, u = d - t (1 <= t, u <= s).
__device__ __forceinline__ void level_pairs(int d, int s, int& t_lo, int& t_hi) {
  t_lo = d - s > 1 ? d - s : 1;
  t_hi = d - 1 < s ? d - 1 : s;
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_oz(const __grid_constant__ OzParams p) {
  const int rank = static_cast<int>(cluster_ctarank());
  const int first = blockIdx.x / 2;
  const int stride = gridDim.x / 2;
  const int nkb = (p.K + kBK - 1) / kBK;
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

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
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
  // the peer's loads and arrivals target CTA 0's barriers: both must exist first
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
    for (int w = first; w < p.total_items && ok; w += stride) {
      int lev, mt2, nt;
      oz_item(p, w, lev, mt2, nt);
      const int d = p.lev_d[lev];
      int t_lo, t_hi;
      level_pairs(d, p.slices, t_lo, t_hi);
      const int m0 = (mt2 * 2 + rank) * kRows;
      const int nb = nt * kCols + rank * kHalf;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int x = kb * kBK;  // past K the boxes read zeros
        for (int t = t_lo; t <= t_hi; ++t) {
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
            const CUtensorMap* ml = &p.L[t - 1];
            const CUtensorMap* mr = &p.R[d - t - 1];
            tma_load_2d_pair(a, ml, bar, x, m0);
            tma_load_2d_pair(a + 8192, ml, bar, x, m0 + 64);
            tma_load_2d_pair(b, mr, bar, nb, x);
            tma_load_2d_pair(b + 8192, mr, bar, nb + 64, x);
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
      // let the loads in flight land before the CTA can leave (the peer's
      // loads complete on CTA 0's barriers, so the peer waits out a grace period)
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
    for (int w = first; w < p.total_items && ok; w += stride) {
      int lev, mt2, nt;
      oz_item(p, w, lev, mt2, nt);
      const int d = p.lev_d[lev];
      const int kcb = p.lev_kcb[lev];  // 64-deep K blocks per exact chunk
      int t_lo, t_hi;
      level_pairs(d, p.slices, t_lo, t_hi);
      for (int c0 = 0; c0 < nkb && ok; c0 += kcb) {
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, tlim, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kCols);
        uint32_t accumulate = 0;
        const int c1 = c0 + kcb < nkb ? c0 + kcb : nkb;
        for (int kb = c0; kb < c1 && ok; ++kb) {
          for (int t = t_lo; t <= t_hi; ++t) {
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
        }
        if (!ok) break;
        tc_commit_pair_mc(&tfull[acc], 0x3);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1u;
        }
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
    const int q = warp & 3;         // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;  // column quarter of the tile
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int w = first; w < p.total_items && ok; w += stride) {
      int lev, mt2, nt;
      oz_item(p, w, lev, mt2, nt);
      const int kcb = p.lev_kcb[lev];
      const int row = (mt2 * 2 + rank) * kRows + q * 32 + lane;
      const int col0 = nt * kCols + h * kColsPer;
      int run[kColsPer];
#pragma unroll
      for (int j = 0; j < kColsPer; ++j) run[j] = 0;
      for (int c0 = 0; c0 < nkb; c0 += kcb) {
        const bool got = mbar_wait(&tfull[acc], acc_phase, tlim, abort_flag);
        if (!epi_all(got)) {  // all epilogue warps stop at the same chunk
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
          for (int j = 0; j < 16; ++j) run[16 * part + j] += __float2int_rn(__uint_as_float(v[j]));
        }
        // all sixteen epilogue warps are done with this accumulator: one
        // arrival per CTA.  No thread can leave between the vote and here.
        tc_fence_before();
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
        if (threadIdx.x == 64) {
          if (rank == 0)
            mbar_arrive(&tempty[acc]);
          else
            mbar_arrive_cluster(tempty0 + static_cast<uint32_t>(acc * 8));
        }
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
      if (!ok) break;
      if (row < p.M) {
        int32_t* dst = p.planes + static_cast<int64_t>(p.lev_d[lev] - 2) * p.plane_stride +
                       static_cast<int64_t>(row) * p.ldp + col0;
        if (col0 + kColsPer <= p.N) {
#pragma unroll
          for (int j = 0; j < kColsPer; j += 4)
            *reinterpret_cast<int4*>(dst + j) = make_int4(run[j], run[j + 1], run[j + 2], run[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < kColsPer; ++j)
            if (col0 + j < p.N) dst[j] = run[j];
        }
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

// ---------------------------------------------------------------- slicing
// Scales: the power of two 2^e with max |x| = f 2^e, f in [1/2, 1), found
// from the bit patterns (for doubles of one sign, larger magnitude = larger
// bits).  A line whose largest magnitude is 0 or below 2^-1000 gets scale 1
// and slices of zeros.
__device__ __forceinline__ double scale_from_maxbits(unsigned long long mb) {
  const int E = static_cast<int>(mb >> 52);  // biased exponent of the largest magnitude
  if (E < 23) return 1.0;                    // zero, subnormal or below 2^-1000
  return __longlong_as_double(static_cast<long long>(E + 1) << 52);
}

// One warp per row.
__global__ void k_oz_row_scale(const double* __restrict__ X, int64_t ld, int rows, int cols, double* __restrict__ mu) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  unsigned long long m = 0;
  const unsigned long long* x = reinterpret_cast<const unsigned long long*>(X + static_cast<int64_t>(row) * ld);
  for (int c = lane; c < cols; c += 32) m = max(m, x[c] & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) mu[row] = scale_from_maxbits(m);
}

// Column maxima of |X| as bit patterns: 256 consecutive columns per block
// (each warp reads 256 contiguous bytes of a row), kOzColRows rows per block,
// one atomicMax per column and block into mb (zeroed before).
constexpr int kOzColRows = 256;
__global__ void k_oz_col_maxbits(const double* __restrict__ X, int64_t ld, int rows, int cols,
                                 unsigned long long* __restrict__ mb) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= cols) return;
  const int r0 = blockIdx.y * kOzColRows;
  const int r1 = r0 + kOzColRows < rows ? r0 + kOzColRows : rows;
  const unsigned long long* x = reinterpret_cast<const unsigned long long*>(X) + col;
  unsigned long long m0 = 0, m1 = 0, m2 = 0, m3 = 0;
  int r = r0;
  for (; r + 4 <= r1; r += 4) {
    m0 = max(m0, x[static_cast<int64_t>(r) * ld] & 0x7FFFFFFFFFFFFFFFull);
    m1 = max(m1, x[static_cast<int64_t>(r + 1) * ld] & 0x7FFFFFFFFFFFFFFFull);
    m2 = max(m2, x[static_cast<int64_t>(r + 2) * ld] & 0x7FFFFFFFFFFFFFFFull);
    m3 = max(m3, x[static_cast<int64_t>(r + 3) * ld] & 0x7FFFFFFFFFFFFFFFull);
  }
  for (; r < r1; ++r) m0 = max(m0, x[static_cast<int64_t>(r) * ld] & 0x7FFFFFFFFFFFFFFFull);
  const unsigned long long m = max(max(m0, m1), max(m2, m3));
  if (m != 0) atomicMax(mb + col, m);
}

__global__ void k_oz_scale_from_bits(const unsigned long long* __restrict__ mb, int cols, double* __restrict__ nu) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col < cols) nu[col] = scale_from_maxbits(mb[col]);
}

// Signed digits of y = v / (2 scale) in (-1/2, 1/2): a_t = RN(256 x_{t-1}),
// x_t = 256 x_{t-1} - a_t (round to nearest, ties to even), computed in
// integers.  With T = 4 y 256^s as a fixed-point integer (two fraction bits
// and a sticky bit below them, which keep every rounding decision of digits
// at positions >= 2^2), a_t = RN(R / 2^p), p = 8 (s - t) + 2, R <- R - a_t 2^p.
// The digits of -v are those of v negated.  |a_t| <= 128.
__device__ __forceinline__ void signed_digits(double v, int scale_exp, int s, int (&a)[kOzMaxSlices]) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  int ev;
  if (E == 0) {
    ev = -1022;  // subnormal: v = M 2^{-1074}
  } else {
    M |= 1ull << 52;
    ev = E - 1023;
  }
  const int k = ev - 51 - scale_exp + 8 * s;  // 4 T = M 2^k, k <= 8 s - 52 <= 4
  long long R;
  if (M == 0) {
    R = 0;
  } else if (k >= 0) {
    R = static_cast<long long>(M << k);
  } else if (-k >= 60) {
    R = 1;  // sticky only
  } else {
    const int sh = -k;
    R = static_cast<long long>((M >> sh) | ((M & ((1ull << sh) - 1ull)) != 0ull ? 1ull : 0ull));
  }
  const bool neg = (b >> 63) != 0;
#pragma unroll
  for (int t = 0; t < kOzMaxSlices; ++t) {
    if (t >= s) {
      a[t] = 0;
      continue;
    }
    const int p = 8 * (s - 1 - t) + 2;
    long long q = R >> p;  // floor
    const long long r = R - (q << p);
    const long long half = 1ll << (p - 1);
    if (r > half || (r == half && (q & 1))) ++q;
    R -= q << p;
    a[t] = neg ? -static_cast<int>(q) : static_cast<int>(q);
  }
}

// s digit slices of X / (2 scale), scale per row (by_row) or per column; slice
// t at out + t * slice_stride, row-major with leading dimension ldo (even).
// Blocks walk rows; each thread cuts two neighbouring columns and stores
// their digits as one bf16 pair per slice.
__global__ void k_oz_slice(const double* __restrict__ X, int64_t ld, int rows, int cols,
                           const double* __restrict__ scale, int by_row, int s, bf16* __restrict__ out, int64_t ldo,
                           int64_t slice_stride) {
  auto exp_of = [](double sc) {
    return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(sc)) >> 52) & 0x7FF) - 1023;
  };
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const double* xr = X + static_cast<int64_t>(r) * ld;
    bf16* orow = out + static_cast<int64_t>(r) * ldo;
    const int er = by_row ? exp_of(scale[r]) : 0;
    for (int c = 2 * threadIdx.x; c < cols; c += 2 * blockDim.x) {
      int a0[kOzMaxSlices], a1[kOzMaxSlices];
      signed_digits(xr[c], by_row ? er : exp_of(scale[c]), s, a0);
      if (c + 1 < cols) {
        signed_digits(xr[c + 1], by_row ? er : exp_of(scale[c + 1]), s, a1);
#pragma unroll
        for (int t = 0; t < kOzMaxSlices; ++t)
          if (t < s)
            *reinterpret_cast<__nv_bfloat162*>(orow + t * slice_stride + c) =
                __floats2bfloat162_rn(static_cast<float>(a0[t]), static_cast<float>(a1[t]));
      } else {
#pragma unroll
        for (int t = 0; t < kOzMaxSlices; ++t)
          if (t < s) orow[t * slice_stride + c] = __float2bfloat16_rn(static_cast<float>(a0[t]));
      }
    }
  }
}

// ---------------------------------------------------------------- combine
// D_ij = s (2 mu_i)(2 nu_j) sum_{d=2}^{slices+1} 256^{-d} S_d,ij + beta C_ij + gamma [i = j],
// S_d from the int32 planes (plane of level d at planes + (d - 2) plane_stride).
// Levels 2..min(5, s+1) combine exactly into an int64 a, levels 6..s+1 into b:
//   sum = a 256^{-dA} + b 256^{-(s+1)},  dA = min(5, s + 1).
// One block per row band; per-block partial sums of D^2 when frob is set.
template <int S>
__global__ void k_oz_combine(const int32_t* __restrict__ planes, int64_t ldp, int64_t plane_stride, int rows,
                             int cols, const double* __restrict__ mu, const double* __restrict__ nu, double s,
                             const double* C, int64_t ldc, double beta, double gamma, double* D, int64_t ldd,
                             double* __restrict__ frob) {
  constexpr int dA = S + 1 < 5 ? S + 1 : 5;
  const double wa = s * 4.0 * exp2(-8.0 * dA);
  const double wb = s * 4.0 * exp2(-8.0 * (S + 1));
  const bool has_c = beta != 0.0 && C != nullptr;
  double f = 0.0;
  auto one = [&](int r, int c, const long long a, const long long b, double m) {
    const double mn = m * nu[c];  // product of two powers of two: exact
    double base = has_c ? beta * C[static_cast<int64_t>(r) * ldc + c] : 0.0;
    if (r == c) base += gamma;
    double v = fma(wa * mn, static_cast<double>(a), base);
    if (S + 1 >= 6) v = fma(wb * mn, static_cast<double>(b), v);
    D[static_cast<int64_t>(r) * ldd + c] = v;
    f = fma(v, v, f);
  };
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const double m = mu[r];
    const int32_t* pr = planes + static_cast<int64_t>(r) * ldp;
    for (int c = 2 * threadIdx.x; c < cols; c += 2 * blockDim.x) {
      // rows of the planes start 16-byte aligned (ldp a multiple of 4) and c is even
      long long a0 = 0, a1 = 0, b0 = 0, b1 = 0;
#pragma unroll
      for (int d = 2; d <= dA; ++d) {
        const int2 q = *reinterpret_cast<const int2*>(pr + (d - 2) * plane_stride + c);
        a0 += static_cast<long long>(q.x) << (8 * (dA - d));
        a1 += static_cast<long long>(q.y) << (8 * (dA - d));
      }
#pragma unroll
      for (int d = 6; d <= S + 1; ++d) {
        const int2 q = *reinterpret_cast<const int2*>(pr + (d - 2) * plane_stride + c);
        b0 += static_cast<long long>(q.x) << (8 * (S + 1 - d));
        b1 += static_cast<long long>(q.y) << (8 * (S + 1 - d));
      }
      one(r, c, a0, b0, m);
      if (c + 1 < cols) one(r, c + 1, a1, b1, m);
    }
  }
  if (frob != nullptr) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
      frob[blockIdx.x] = t;
    }
  }
}

cudaError_t launch_combine(int S, int nb, cudaStream_t st, const int32_t* planes, int64_t ldp, int64_t pstride,
                           int rows, int cols, const double* mu, const double* nu, double s, const double* C,
                           int64_t ldc, double beta, double gamma, double* D, int64_t ldd, double* frob) {
#define NSGB_OZ_COMBINE(K)                                                                                         \
  case K:                                                                                                          \
    k_oz_combine<K><<<nb, 256, 0, st>>>(planes, ldp, pstride, rows, cols, mu, nu, s, C, ldc, beta, gamma, D, ldd, \
                                        frob);                                                                     \
    break;
  switch (S) {
    NSGB_OZ_COMBINE(2)
    NSGB_OZ_COMBINE(3)
    NSGB_OZ_COMBINE(4)
    NSGB_OZ_COMBINE(5)
    NSGB_OZ_COMBINE(6)
    NSGB_OZ_COMBINE(7)
    default:
      return cudaErrorInvalidValue;
  }
#undef NSGB_OZ_COMBINE
  return cudaGetLastError();
}

// blocks of the slicing kernel: one row at a time, at most 16 per SM's worth
int slice_rows_grid(int rows) { return rows < 1 ? 1 : (rows < 152 * 16 ? rows : 152 * 16); }

cudaError_t launch_levels(const OzParams& p, int num_sms, cudaStream_t s) {
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
    init = cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (init != cudaSuccess) return;
    cudaLaunchConfig_t c = cfg;
    c.gridDim = dim3(2 * (num_sms / 2));
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_gemm_oz, &c);
    if (e != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = num_sms / 2;
    }
    max_clusters = n;
  });
  if (init != cudaSuccess) return init;
  if (p.total_items <= 0) return cudaSuccess;
  const int clusters = p.total_items < max_clusters ? p.total_items : max_clusters;
  cfg.gridDim = dim3(2 * clusters);
  return cudaLaunchKernelEx(&cfg, k_gemm_oz, p);
}

}  // namespace

int oz_combine_blocks(int rows) { return rows < 608 ? (rows < 1 ? 1 : rows) : 608; }

size_t oz_workspace_bytes(int64_t M, int64_t N, int64_t K, int slices) {
  const int64_t kb = K < kOzMaxK ? K : kOzMaxK;
  const int64_t ldk = (kb + 7) / 8 * 8, ldn = (N + 7) / 8 * 8, ldp = (N + 3) / 4 * 4;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) / 256 * 256; };
  add(sizeof(bf16) * static_cast<size_t>(M) * ldk * slices);
  add(sizeof(bf16) * static_cast<size_t>(kb) * ldn * slices);
  add(sizeof(double) * static_cast<size_t>(M));
  add(sizeof(double) * static_cast<size_t>(N));
  add(sizeof(int32_t) * static_cast<size_t>(M) * ldp * slices);
  add(sizeof(double) * static_cast<size_t>(oz_combine_blocks(static_cast<int>(M))));
  add(sizeof(unsigned long long) * static_cast<size_t>(N));
  return b;
}

// D = s L R + beta C + gamma I to the accuracy of `slices` digit slices per
// operand (binary64 with 7), L: M x K, R: K x N, all FP64 row-major on the
// device.  K is taken in blocks of at most kOzMaxK (each block adds into D);
// L and R are sliced before D is written, so D may alias L, R or C when
// K <= kOzMaxK.  frob_out (device, may be null) receives sum(D^2).
cudaError_t launch_oz_product(const OzArgs& g, int num_sms, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (g.slices < 2 || g.slices > kOzMaxSlices) return cudaErrorInvalidValue;
  const int64_t M = g.M, N = g.N;
  const int64_t kb0 = g.K < kOzMaxK ? g.K : kOzMaxK;
  const int64_t ldk = (kb0 + 7) / 8 * 8, ldn = (N + 7) / 8 * 8, ldp = (N + 3) / 4 * 4;
  char* w = static_cast<char*>(g.work);
  auto carve = [&](size_t bytes) {
    char* p = w;
    w += (bytes + 255) / 256 * 256;
    return p;
  };
  bf16* Ls = reinterpret_cast<bf16*>(carve(sizeof(bf16) * static_cast<size_t>(M) * ldk * g.slices));
  bf16* Rs = reinterpret_cast<bf16*>(carve(sizeof(bf16) * static_cast<size_t>(kb0) * ldn * g.slices));
  double* mu = reinterpret_cast<double*>(carve(sizeof(double) * static_cast<size_t>(M)));
  double* nu = reinterpret_cast<double*>(carve(sizeof(double) * static_cast<size_t>(N)));
  int32_t* planes = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * static_cast<size_t>(M) * ldp * g.slices));
  double* fparts = reinterpret_cast<double*>(carve(sizeof(double) * static_cast<size_t>(oz_combine_blocks(g.M))));
  unsigned long long* nub =
      reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long) * static_cast<size_t>(N)));
  const int64_t lstride = M * ldk, rstride = kb0 * ldn, pstride = M * ldp;
  cudaError_t e = cudaSuccess;
  for (int64_t k0 = 0; k0 < g.K && e == cudaSuccess; k0 += kOzMaxK) {
    const int kb = static_cast<int>(g.K - k0 < kOzMaxK ? g.K - k0 : kOzMaxK);
    const bool first = k0 == 0, last = k0 + kb >= g.K;
    // scales and slices of L[:, k0 : k0 + kb] and R[k0 : k0 + kb, :]
    k_oz_row_scale<<<(g.M + 7) / 8, 256, 0, st>>>(g.L + k0, g.ldl, g.M, kb, mu);
    e = cudaMemsetAsync(nub, 0, sizeof(unsigned long long) * static_cast<size_t>(N), st);
    if (e != cudaSuccess) break;
    k_oz_col_maxbits<<<dim3((g.N + 255) / 256, (kb + kOzColRows - 1) / kOzColRows), 256, 0, st>>>(
        g.R + k0 * g.ldr, g.ldr, kb, g.N, nub);
    k_oz_scale_from_bits<<<(g.N + 255) / 256, 256, 0, st>>>(nub, g.N, nu);
    k_oz_slice<<<slice_rows_grid(g.M), 256, 0, st>>>(g.L + k0, g.ldl, g.M, kb, mu, 1, g.slices, Ls, ldk, lstride);
    k_oz_slice<<<slice_rows_grid(kb), 256, 0, st>>>(g.R + k0 * g.ldr, g.ldr, kb, g.N, nu, 0, g.slices, Rs, ldn,
                                                    rstride);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    OzParams p;
    memset(&p, 0, sizeof(p));
    for (int t = 0; t < g.slices; ++t)
      if (!encode_bf16_map(&p.L[t], Ls + t * lstride, M, kb, ldk, 0) ||
          !encode_bf16_map(&p.R[t], Rs + t * rstride, kb, N, ldn, 0))
        return cudaErrorInvalidValue;
    p.M = g.M;
    p.N = g.N;
    p.K = kb;
    p.slices = g.slices;
    p.tiles_m2 = (g.M + 255) / 256;
    p.tiles_n = (g.N + 255) / 256;
    // levels with the most pairs first (largest items first balance the waves)
    p.nlev = 0;
    for (int d = g.slices + 1; d >= 2; --d) {
      int pairs = 0;
      for (int t = 1; t <= g.slices; ++t)
        if (d - t >= 1 && d - t <= g.slices) ++pairs;
      // exact f32 sums: pairs * K_c * 2^14 <= 2^24, K_c a multiple of 64
      int kc = (1024 / pairs) / 64 * 64;
      if (kc < 64) return cudaErrorInvalidValue;
      p.lev_d[p.nlev] = d;
      p.lev_kcb[p.nlev] = kc / 64;
      p.nlev++;
    }
    p.total_items = p.nlev * p.tiles_m2 * p.tiles_n;
    p.planes = planes;
    p.ldp = ldp;
    p.plane_stride = pstride;
    p.debug_stall_iter = g.debug_stall_iter;
    p.timeout_ns = g.timeout_ns;
    p.err = g.err;
    e = launch_levels(p, num_sms, st);
    if (e != cudaSuccess) break;
    const int nb = oz_combine_blocks(g.M);
    e = launch_combine(g.slices, nb, st, planes, ldp, pstride, g.M, g.N, mu, nu, g.s, first ? g.C : g.D,
                       first ? g.ldc : g.ldd, first ? g.beta : 1.0, first ? g.gamma : 0.0, g.D, g.ldd,
                       last && g.frob_out ? fparts : nullptr);
    if (e == cudaSuccess && last && g.frob_out) e = launch_reduce_sum(fparts, nb, 1, g.frob_out, st);
  }
  return e;
}

}  // namespace nsgb
