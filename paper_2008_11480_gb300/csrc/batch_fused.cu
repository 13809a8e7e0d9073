// Fused small-system solve: one CTA runs the whole solve of one system of
// n <= 256 -- norms and splits of A, G0, every Newton-Schulz step of the
// factorized chain on the tensor cores (tcgen05, 128 x 128 tiles, TMEM
// accumulators, TMA-fed shared-memory stages), the split-f32 Richardson
// sweeps and the per-system precision controller -- and then takes the next
// system.  A batch of thousands of such systems is one persistent launch and
// one host synchronisation instead of a few launches per product level and a
// host decision per pass.
//
// The arithmetic is the list-driven path's, instruction for instruction: the
// same problem descriptors (tensor maps of the slot's split buffers), the same
// MMA sequence and shared epilogue per output tile, the same row-kernel bodies
// (batch_rows.cuh) over the same 8-row blocks, and the controller of the host
// pass (decide(), pass() in batch.cu) written out per system.  A system's
// result is therefore the same here, alone, in any mix and on the list path.
//
// Roles during a product (256 threads): warp 0 lane 0 the TMA producer, warp
// 1 the TMEM allocator and lane 0 the MMA issuer, warps 2..5 the epilogue
// (TMEM lane quarter = warp % 4); warps 6, 7 wait.  Between phases every
// thread fences its global writes for the async proxy (the next product's TMA
// reads them) and the CTA synchronises.  Pipeline positions (stage, phase,
// accumulator) persist across products.  Every wait is bounded: a CTA whose
// wait runs out records NS_ERR_TIMEOUT, marks the system and stops taking
// systems.
#include <mutex>
#include <cmath>

#include "../../include/nsgb.h"
#include "batch_rows.cuh"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace nsgb {
namespace {

constexpr int kThreads = 256;
constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kABytes = kBM * kBK * 2;  // 16 KiB
constexpr int kBBytes = kBN * kBK * 2;  // 16 KiB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kStages = 4;
constexpr uint32_t kTmemCols = 2 * kBN;
constexpr int kBarBytes = 256;
constexpr int kEpiStride = 36;
constexpr int kEpiBytes = 4 * 32 * kEpiStride * 4;
constexpr int kSmem = kStages * kStageBytes + kBarBytes + kEpiBytes + 1024;
static_assert(kSmem <= 200 * 1024, "dynamic shared memory (the row bodies add static arrays)");

// Generic-proxy writes (global and shared) made visible to later async-proxy
// accesses: the next product's TMA reads global operands and overwrites the
// stage area the row phases use as scratch.
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async;" ::: "memory"); }

struct Pipe {
  uint8_t* sA;
  uint8_t* sB;
  uint64_t *full, *empty, *tfull, *tempty, *drain;
  float* ebuf;
  volatile int* abort_flag;
  uint32_t tmem;
  uint64_t tlim;
  int* err;
};

// Per-thread pipeline positions (each role advances its own copy in step).
struct Pos {
  int stage = 0, acc = 0;
  uint32_t phase = 0, acc_phase = 0;
};

// All output tiles of one n x n product D = s L R + beta C + gamma I (problem
// P of the slot's table), by this CTA.  Entered by all threads; returns after
// the CTA barrier, false when a bounded wait ran out.
__device__ bool cta_product(const TcProblem& P, bool x3, const Pipe& pp, Pos& ps) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = P.tiles_m * P.tiles_n;
  const int kstep = x3 ? kBK / 2 : kBK;
  const int nkb = (P.K + kstep - 1) / kstep;
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    tma_prefetch_desc(&P.L[0]);
    tma_prefetch_desc(&P.R[0]);
    tma_prefetch_desc(&P.L[1]);
    tma_prefetch_desc(&P.R[1]);
    int armed[kStages];
    for (int s = 0; s < kStages; ++s) armed[s] = -1;
    bool ok = true;
    for (int w = 0; w < tiles && ok; ++w) {
      const int m0 = (w / P.tiles_n) * kBM, n0 = (w % P.tiles_n) * kBN;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(&pp.empty[ps.stage], ps.phase ^ 1u, pp.tlim, pp.abort_flag)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&pp.full[ps.stage], kStageBytes);
        armed[ps.stage] = static_cast<int>(ps.phase);
        uint8_t* a = pp.sA + ps.stage * kABytes;
        uint8_t* b = pp.sB + ps.stage * kBBytes;
        if (x3) {
          const int x = kb * (kBK / 2);
          tma_load_2d(a, &P.L[0], &pp.full[ps.stage], x, m0);
          tma_load_2d(a + 4096, &P.L[0], &pp.full[ps.stage], x, m0 + 64);
          tma_load_2d(a + 8192, &P.L[1], &pp.full[ps.stage], x, m0);
          tma_load_2d(a + 12288, &P.L[1], &pp.full[ps.stage], x, m0 + 64);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int part = j >> 1, c = j & 1;
            tma_load_2d(b + part * (kBN * 64) + c * 4096, &P.R[part], &pp.full[ps.stage], n0 + 64 * c, x);
          }
        } else {
          tma_load_2d(a, &P.L[0], &pp.full[ps.stage], kb * kBK, m0);
          tma_load_2d(a + 8192, &P.L[0], &pp.full[ps.stage], kb * kBK, m0 + 64);
          tma_load_2d(b, &P.R[0], &pp.full[ps.stage], n0, kb * kBK);
          tma_load_2d(b + 8192, &P.R[0], &pp.full[ps.stage], n0 + 64, kb * kBK);
        }
        if (++ps.stage == kStages) {
          ps.stage = 0;
          ps.phase ^= 1u;
        }
      }
    }
    if (!ok) {
      *pp.abort_flag = 1;
      atomicExch(pp.err, DEV_TIMEOUT);
      volatile int never = 0;
      for (int s = 0; s < kStages; ++s)
        if (armed[s] >= 0) mbar_wait(&pp.full[s], static_cast<uint32_t>(armed[s]), 100000000ull, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idesc = make_idesc_bf16(kBM, kBN, 0, 1);
    bool ok = true, issued = false;
    for (int w = 0; w < tiles && ok; ++w) {
      if (!mbar_wait(&pp.tempty[ps.acc], ps.acc_phase ^ 1u, pp.tlim, pp.abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = pp.tmem + static_cast<uint32_t>(ps.acc * kBN);
      uint32_t accumulate = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(&pp.full[ps.stage], ps.phase, pp.tlim, pp.abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_u32(pp.sA + ps.stage * kABytes);
        const uint32_t b_base = smem_u32(pp.sB + ps.stage * kBBytes);
        if (x3) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint64_t ah = make_sdesc(a_base + 32u * k, 16u, 512u, kSwz64);
            const uint64_t al = make_sdesc(a_base + 8192u + 32u * k, 16u, 512u, kSwz64);
            const uint64_t bh = make_sdesc(b_base + 2048u * k, 4096u, 1024u);
            const uint64_t bl = make_sdesc(b_base + static_cast<uint32_t>(kBN * 64) + 2048u * k, 4096u, 1024u);
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
        tc_commit(&pp.empty[ps.stage]);
        if (++ps.stage == kStages) {
          ps.stage = 0;
          ps.phase ^= 1u;
        }
      }
      if (!ok) break;
      tc_commit(&pp.tfull[ps.acc]);
      if (++ps.acc == 2) {
        ps.acc = 0;
        ps.acc_phase ^= 1u;
      }
    }
    if (!ok) {
      *pp.abort_flag = 1;
      atomicExch(pp.err, DEV_TIMEOUT);
      if (issued) {
        volatile int never = 0;
        tc_commit(pp.drain);
        mbar_wait(pp.drain, 0, 100000000ull, &never);
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    for (int w = 0; w < tiles; ++w) {
      const int mt = w / P.tiles_n, nt = w % P.tiles_n;
      bool ok = mbar_wait(&pp.tfull[ps.acc], ps.acc_phase, pp.tlim, pp.abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        *pp.abort_flag = 1;
        if (lane == 0) atomicExch(pp.err, DEV_TIMEOUT);
        break;
      }
      tc_fence_after();
      const float frob = tc::epilogue_tile<kBN, kEpiStride>(
          P, mt * kBM, nt * kBN, q, lane, pp.ebuf + q * 32 * kEpiStride,
          pp.tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(ps.acc * kBN));
      tc_fence_before();
      mbar_arrive(&pp.tempty[ps.acc]);
      if (P.frob_partials != nullptr && mt < P.tiles_m) {
        double f = static_cast<double>(frob);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0) P.frob_partials[(mt * P.tiles_n + nt) * 4 + q] = f;
      }
      if (++ps.acc == 2) {
        ps.acc = 0;
        ps.acc_phase ^= 1u;
      }
    }
  }
  fence_async_global();
  __syncthreads();
  return *pp.abort_flag == 0;
}

// ---------------------------------------------------------------- whole-system row phases
// The row kernels' arithmetic for all rows of the system at once: the same
// per-row computation (a warp per row pair and half of the k range for the
// split-f32 residual and the update, a warp per row for the FP64 residual and
// the preparation), the same fixed-order sums of each 8-row block, but every
// warp takes several rows in turn with one barrier per phase instead of one
// per 8-row block.  Scratch lives in the stage area, idle between products.
constexpr int kMaxPairs = kFusedMaxN / 2;

// Split-f32 residual of right-hand sides [c0, c0 + NRW) (NRW = 1 or kBRhs).
template <int NRW>
__device__ void wide_resid_x2(const BInst& I, int c0, uint8_t* scratch) {
  float* rhi = reinterpret_cast<float*>(scratch);             // [pair][half][c][r]
  float* rlo = rhi + kMaxPairs * 2 * NRW * 2;
  double* sq = reinterpret_cast<double*>(rlo + kMaxPairs * 2 * NRW * 2);  // [row][c]
  const int n = I.n, nrhs = I.nrhs;
  const int64_t ld = I.ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntask = ((n + 1) / 2) * 2;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t = warp; t < ntask; t += 8) {
    const int pair = t >> 1, half = t & 1;
    const int row0 = 2 * pair;
    const bool r0 = row0 < n, r1 = row0 + 1 < n;
    const int64_t o0 = static_cast<int64_t>(r0 ? row0 : 0) * ld;
    const int64_t o1 = static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
    float hi[2][NRW], lo[2][NRW];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < NRW; ++c) hi[r][c] = lo[r][c] = 0.f;
#pragma unroll 1
    for (int k = 4 * lane + 128 * half; k < n4; k += 256) {
      const float4 x0 = r0 ? *reinterpret_cast<const float4*>(I.A1 + o0 + k) : z4;
      const float4 y0 = r0 ? *reinterpret_cast<const float4*>(I.A2 + o0 + k) : z4;
      const float4 x1 = r1 ? *reinterpret_cast<const float4*>(I.A1 + o1 + k) : z4;
      const float4 y1 = r1 ? *reinterpret_cast<const float4*>(I.A2 + o1 + k) : z4;
      const float a1v[2][4] = {{x0.x, x0.y, x0.z, x0.w}, {x1.x, x1.y, x1.z, x1.w}};
      const float a2v[2][4] = {{y0.x, y0.y, y0.z, y0.w}, {y1.x, y1.y, y1.z, y1.w}};
#pragma unroll
      for (int c = 0; c < NRW; ++c) {
        if (c0 + c >= nrhs) continue;
        const float4 u = *reinterpret_cast<const float4*>(I.T1 + (c0 + c) * ld + k);
        const float4 w = *reinterpret_cast<const float4*>(I.T2 + (c0 + c) * ld + k);
        const float t1v[4] = {u.x, u.y, u.z, u.w};
        const float t2v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float pv = a1v[r][j] * t1v[j];
            const float e = fmaf(a1v[r][j], t1v[j], -pv);
            brow::two_sum_acc(hi[r][c], lo[r][c], pv);
            lo[r][c] += fmaf(a1v[r][j], t2v[j], fmaf(a2v[r][j], t1v[j], e));
          }
      }
    }
    if (half == 0) {
      for (int k = n4 + lane; k < n; k += 32) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const bool okr = r == 0 ? r0 : r1;
          const int64_t o = r == 0 ? o0 : o1;
          const float x = okr ? I.A1[o + k] : 0.f, y = okr ? I.A2[o + k] : 0.f;
#pragma unroll
          for (int c = 0; c < NRW; ++c) {
            if (c0 + c >= nrhs) continue;
            const float t1 = I.T1[(c0 + c) * ld + k], t2 = I.T2[(c0 + c) * ld + k];
            const float pv = x * t1;
            const float e = fmaf(x, t1, -pv);
            brow::two_sum_acc(hi[r][c], lo[r][c], pv);
            lo[r][c] += fmaf(x, t2, fmaf(y, t1, e));
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < NRW; ++c) {
        brow::warp_sum_x2(hi[r][c], lo[r][c]);
        if (lane == 0) {
          rhi[((pair * 2 + half) * NRW + c) * 2 + r] = hi[r][c];
          rlo[((pair * 2 + half) * NRW + c) * 2 + r] = lo[r][c];
        }
      }
  }
  __syncthreads();
  const int nrow8 = (n + 7) / 8 * 8;
  for (int e = threadIdx.x; e < nrow8 * NRW; e += kThreads) {
    const int row = e / NRW, c = e % NRW;
    const int pr = row >> 1, r = row & 1;
    double v2 = 0.0;
    if (row < n && c0 + c < nrhs) {
      const double sdot = (static_cast<double>(rhi[((pr * 2 + 0) * NRW + c) * 2 + r]) +
                           static_cast<double>(rlo[((pr * 2 + 0) * NRW + c) * 2 + r])) +
                          (static_cast<double>(rhi[((pr * 2 + 1) * NRW + c) * 2 + r]) +
                           static_cast<double>(rlo[((pr * 2 + 1) * NRW + c) * 2 + r]));
      const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
      const double v = I.B[o] - sdot;
      I.R[o] = v;
      I.R32T[static_cast<int64_t>(c0 + c) * ld + row] = static_cast<float>(v);
      v2 = v * v;
    }
    sq[row * NRW + c] = v2;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (nrow8 / 8) * NRW; e += kThreads) {
    const int b = e / NRW, c = e % NRW;
    if (c0 + c >= nrhs) continue;
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sq[(8 * b + w) * NRW + c];
    I.part[static_cast<int64_t>(b) * nrhs + c0 + c] = t;
  }
  __syncthreads();
}

// The single right-hand side forms for n <= 256, where the k loop of a row
// task is one float4 step (k = 4 lane + 128 half < n & ~3) and a tail of at
// most three elements: each warp runs kU tasks at once, all loads first, the
// same operations per row as above.
constexpr int kU = 2;

__device__ void wide_resid_x2_1(const BInst& I, uint8_t* scratch) {
  constexpr int NRW = 1;
  float* rhi = reinterpret_cast<float*>(scratch);
  float* rlo = rhi + kMaxPairs * 2 * NRW * 2;
  double* sq = reinterpret_cast<double*>(rlo + kMaxPairs * 2 * NRW * 2);
  const int n = I.n;
  const int64_t ld = I.ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntask = ((n + 1) / 2) * 2;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int tb = warp; tb < ntask; tb += 8 * kU) {
    float4 x0[kU], y0[kU], x1[kU], y1[kU], u[kU], w[kU];
    bool main[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int t = tb + 8 * q;
      const int pair = t >> 1, half = t & 1;
      const int row0 = 2 * pair;
      const int k = 4 * lane + 128 * half;
      main[q] = t < ntask && k < n4;
      const bool r0 = row0 < n, r1 = row0 + 1 < n;
      const int64_t o0 = static_cast<int64_t>(r0 ? row0 : 0) * ld;
      const int64_t o1 = static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
      x0[q] = main[q] && r0 ? *reinterpret_cast<const float4*>(I.A1 + o0 + k) : z4;
      y0[q] = main[q] && r0 ? *reinterpret_cast<const float4*>(I.A2 + o0 + k) : z4;
      x1[q] = main[q] && r1 ? *reinterpret_cast<const float4*>(I.A1 + o1 + k) : z4;
      y1[q] = main[q] && r1 ? *reinterpret_cast<const float4*>(I.A2 + o1 + k) : z4;
      u[q] = main[q] ? *reinterpret_cast<const float4*>(I.T1 + k) : z4;
      w[q] = main[q] ? *reinterpret_cast<const float4*>(I.T2 + k) : z4;
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int t = tb + 8 * q;
      if (t >= ntask) break;  // warp-uniform
      const int pair = t >> 1, half = t & 1;
      const int row0 = 2 * pair;
      const bool r0 = row0 < n, r1 = row0 + 1 < n;
      const int64_t o0 = static_cast<int64_t>(r0 ? row0 : 0) * ld;
      const int64_t o1 = static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
      float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
      if (main[q]) {
        const float a1v[2][4] = {{x0[q].x, x0[q].y, x0[q].z, x0[q].w}, {x1[q].x, x1[q].y, x1[q].z, x1[q].w}};
        const float a2v[2][4] = {{y0[q].x, y0[q].y, y0[q].z, y0[q].w}, {y1[q].x, y1[q].y, y1[q].z, y1[q].w}};
        const float t1v[4] = {u[q].x, u[q].y, u[q].z, u[q].w};
        const float t2v[4] = {w[q].x, w[q].y, w[q].z, w[q].w};
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float pv = a1v[r][j] * t1v[j];
            const float e = fmaf(a1v[r][j], t1v[j], -pv);
            brow::two_sum_acc(hi[r], lo[r], pv);
            lo[r] += fmaf(a1v[r][j], t2v[j], fmaf(a2v[r][j], t1v[j], e));
          }
      }
      if (half == 0) {
        for (int k = n4 + lane; k < n; k += 32) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const bool okr = r == 0 ? r0 : r1;
            const int64_t o = r == 0 ? o0 : o1;
            const float x = okr ? I.A1[o + k] : 0.f, y = okr ? I.A2[o + k] : 0.f;
            const float t1 = I.T1[k], t2 = I.T2[k];
            const float pv = x * t1;
            const float e = fmaf(x, t1, -pv);
            brow::two_sum_acc(hi[r], lo[r], pv);
            lo[r] += fmaf(x, t2, fmaf(y, t1, e));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        brow::warp_sum_x2(hi[r], lo[r]);
        if (lane == 0) {
          rhi[(pair * 2 + half) * 2 + r] = hi[r];
          rlo[(pair * 2 + half) * 2 + r] = lo[r];
        }
      }
    }
  }
  __syncthreads();
  const int nrow8 = (n + 7) / 8 * 8;
  for (int row = threadIdx.x; row < nrow8; row += kThreads) {
    const int pr = row >> 1, r = row & 1;
    double v2 = 0.0;
    if (row < n) {
      const double sdot = (static_cast<double>(rhi[(pr * 2 + 0) * 2 + r]) + static_cast<double>(rlo[(pr * 2 + 0) * 2 + r])) +
                          (static_cast<double>(rhi[(pr * 2 + 1) * 2 + r]) + static_cast<double>(rlo[(pr * 2 + 1) * 2 + r]));
      const double v = I.B[row] - sdot;
      I.R[row] = v;
      I.R32T[row] = static_cast<float>(v);
      v2 = v * v;
    }
    sq[row] = v2;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nrow8 / 8; b += kThreads) {
    double t = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) t += sq[8 * b + w8];
    I.part[b] = t;
  }
  __syncthreads();
}

__device__ void wide_update_1(const BInst& I, int cur, uint8_t* scratch) {
  float* red = reinterpret_cast<float*>(scratch);
  const int n = I.n;
  const int64_t ld = I.ld;
  const float* G = I.G32[cur];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntask = ((n + 1) / 2) * 2;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int tb = warp; tb < ntask; tb += 8 * kU) {
    float4 x0[kU], x1[kU], tt[kU];
    bool main[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int t = tb + 8 * q;
      const int pair = t >> 1, half = t & 1;
      const int row0 = 2 * pair;
      const int k = 4 * lane + 128 * half;
      main[q] = t < ntask && k < n4;
      const bool r0 = row0 < n, r1 = row0 + 1 < n;
      x0[q] = main[q] && r0 ? *reinterpret_cast<const float4*>(G + static_cast<int64_t>(row0) * ld + k) : z4;
      x1[q] = main[q] && r1 ? *reinterpret_cast<const float4*>(G + static_cast<int64_t>(row0 + 1) * ld + k) : z4;
      tt[q] = main[q] ? *reinterpret_cast<const float4*>(I.R32T + k) : z4;
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int t = tb + 8 * q;
      if (t >= ntask) break;  // warp-uniform
      const int pair = t >> 1, half = t & 1;
      const int row0 = 2 * pair;
      const bool r0 = row0 < n, r1 = row0 + 1 < n;
      const float* g0 = G + static_cast<int64_t>(r0 ? row0 : 0) * ld;
      const float* g1 = G + static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
      float acc0 = 0.f, acc1 = 0.f;
      if (main[q]) {
        acc0 = fmaf(x0[q].x, tt[q].x, fmaf(x0[q].y, tt[q].y, fmaf(x0[q].z, tt[q].z, fmaf(x0[q].w, tt[q].w, acc0))));
        acc1 = fmaf(x1[q].x, tt[q].x, fmaf(x1[q].y, tt[q].y, fmaf(x1[q].z, tt[q].z, fmaf(x1[q].w, tt[q].w, acc1))));
      }
      if (half == 0) {
        for (int k = n4 + lane; k < n; k += 32) {
          const float a = r0 ? g0[k] : 0.f;
          const float b = r1 ? g1[k] : 0.f;
          const float tv = I.R32T[k];
          acc0 = fmaf(a, tv, acc0);
          acc1 = fmaf(b, tv, acc1);
        }
      }
      const float s0 = brow::warp_sum_f32(acc0);
      const float s1 = brow::warp_sum_f32(acc1);
      if (lane == 0) {
        red[(pair * 2 + half) * 2 + 0] = s0;
        red[(pair * 2 + half) * 2 + 1] = s1;
      }
    }
  }
  __syncthreads();
  for (int row = threadIdx.x; row < n; row += kThreads) {
    const int pr = row >> 1, r = row & 1;
    const double v = I.Th[row] + (static_cast<double>(red[(pr * 2 + 0) * 2 + r]) +
                                  static_cast<double>(red[(pr * 2 + 1) * 2 + r]));
    I.Th[row] = v;
    const float f1 = static_cast<float>(v);
    I.T1[row] = f1;
    I.T2[row] = static_cast<float>(v - static_cast<double>(f1));
  }
  __syncthreads();
}

// FP64 residual, one right-hand side: a warp per row as above, kU rows of a
// warp at once (each row's k loop and reduction unchanged).
__device__ void wide_resid64_1(const BInst& I, uint8_t* scratch) {
  double* sq = reinterpret_cast<double*>(scratch);
  const int n = I.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrow8 = (n + 7) / 8 * 8;
  for (int rb = warp; rb < nrow8; rb += 8 * kU) {
    double acc[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) acc[q] = 0.0;
    for (int k = lane; k < n; k += 32) {
      const double tk = I.Th[k];
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int row = rb + 8 * q;
        if (row < n) acc[q] = fma(I.A[static_cast<int64_t>(row) * n + k], tk, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int row = rb + 8 * q;
      const double dot = brow::warp_sum_f64(acc[q]);
      if (lane == 0 && row < nrow8) {
        double v2 = 0.0;
        if (row < n) {
          const double v = I.B[row] - dot;
          I.R[row] = v;
          I.R32T[row] = static_cast<float>(v);
          v2 = v * v;
        }
        sq[row] = v2;
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nrow8 / 8; b += kThreads) {
    double t = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) t += sq[8 * b + w8];
    I.part[b] = t;
  }
  __syncthreads();
}

// FP64 residual of right-hand sides [c0, c0 + NRW): a warp per row.
template <int NRW>
__device__ void wide_resid64(const BInst& I, int c0, uint8_t* scratch) {
  double* sq = reinterpret_cast<double*>(scratch);  // [row][c]
  const int n = I.n, nrhs = I.nrhs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrow8 = (n + 7) / 8 * 8;
  for (int row = warp; row < nrow8; row += 8) {
    double acc[NRW];
#pragma unroll
    for (int c = 0; c < NRW; ++c) acc[c] = 0.0;
    if (row < n) {
      const double* a = I.A + static_cast<int64_t>(row) * n;
      for (int k = lane; k < n; k += 32) {
        const double av = a[k];
        const double* t = I.Th + static_cast<int64_t>(k) * nrhs + c0;
#pragma unroll
        for (int c = 0; c < NRW; ++c)
          if (c0 + c < nrhs) acc[c] = fma(av, t[c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NRW; ++c) acc[c] = brow::warp_sum_f64(acc[c]);
    if (lane < NRW) {
      const int c = lane;
      double v2 = 0.0;
      if (row < n && c0 + c < nrhs) {
        double dot = 0.0;
#pragma unroll
        for (int j = 0; j < NRW; ++j)
          if (j == c) dot = acc[j];
        const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
        const double v = I.B[o] - dot;
        I.R[o] = v;
        I.R32T[static_cast<int64_t>(c0 + c) * I.ld + row] = static_cast<float>(v);
        v2 = v * v;
      }
      sq[row * NRW + c] = v2;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (nrow8 / 8) * NRW; e += kThreads) {
    const int b = e / NRW, c = e % NRW;
    if (c0 + c >= nrhs) continue;
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sq[(8 * b + w) * NRW + c];
    I.part[static_cast<int64_t>(b) * nrhs + c0 + c] = t;
  }
  __syncthreads();
}

// theta += G R for right-hand sides [c0, c0 + NRW) (G = the f32 master G[cur]).
template <int NRW>
__device__ void wide_update(const BInst& I, int c0, int cur, uint8_t* scratch) {
  float* red = reinterpret_cast<float*>(scratch);  // [pair][half][c][r]
  const int n = I.n, nrhs = I.nrhs;
  const int64_t ld = I.ld;
  const float* G = I.G32[cur];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntask = ((n + 1) / 2) * 2;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t = warp; t < ntask; t += 8) {
    const int pair = t >> 1, half = t & 1;
    const int row0 = 2 * pair;
    const bool r0 = row0 < n, r1 = row0 + 1 < n;
    const float* g0 = G + static_cast<int64_t>(r0 ? row0 : 0) * ld;
    const float* g1 = G + static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
    float acc[2][NRW];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < NRW; ++c) acc[r][c] = 0.f;
#pragma unroll 1
    for (int k = 4 * lane + 128 * half; k < n4; k += 256) {
      const float4 x0 = r0 ? *reinterpret_cast<const float4*>(g0 + k) : z4;
      const float4 x1 = r1 ? *reinterpret_cast<const float4*>(g1 + k) : z4;
#pragma unroll
      for (int c = 0; c < NRW; ++c) {
        if (c0 + c >= nrhs) continue;
        const float4 tt = *reinterpret_cast<const float4*>(I.R32T + (c0 + c) * ld + k);
        acc[0][c] = fmaf(x0.x, tt.x, fmaf(x0.y, tt.y, fmaf(x0.z, tt.z, fmaf(x0.w, tt.w, acc[0][c]))));
        acc[1][c] = fmaf(x1.x, tt.x, fmaf(x1.y, tt.y, fmaf(x1.z, tt.z, fmaf(x1.w, tt.w, acc[1][c]))));
      }
    }
    if (half == 0) {
      for (int k = n4 + lane; k < n; k += 32) {
        const float x0 = r0 ? g0[k] : 0.f;
        const float x1 = r1 ? g1[k] : 0.f;
#pragma unroll
        for (int c = 0; c < NRW; ++c) {
          if (c0 + c >= nrhs) continue;
          const float tt = I.R32T[(c0 + c) * ld + k];
          acc[0][c] = fmaf(x0, tt, acc[0][c]);
          acc[1][c] = fmaf(x1, tt, acc[1][c]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < NRW; ++c) {
        const float sred = brow::warp_sum_f32(acc[r][c]);
        if (lane == 0) red[((pair * 2 + half) * NRW + c) * 2 + r] = sred;
      }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * NRW; e += kThreads) {
    const int row = e / NRW, c = e % NRW;
    if (c0 + c >= nrhs) continue;
    const int pr = row >> 1, r = row & 1;
    const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
    const double v = I.Th[o] + (static_cast<double>(red[((pr * 2 + 0) * NRW + c) * 2 + r]) +
                                static_cast<double>(red[((pr * 2 + 1) * NRW + c) * 2 + r]));
    I.Th[o] = v;
    const float f1 = static_cast<float>(v);
    I.T1[static_cast<int64_t>(c0 + c) * ld + row] = f1;
    I.T2[static_cast<int64_t>(c0 + c) * ld + row] = static_cast<float>(v - static_cast<double>(f1));
  }
  __syncthreads();
}

// Norm partials, bf16 split and f32 limbs of A: a warp per row, block sums of
// 8 rows in order (as the row kernel).
__device__ void wide_prep(const BInst& I, uint8_t* scratch) {
  double* ss = reinterpret_cast<double*>(scratch);
  double* ra = ss + kFusedMaxN;
  const int n = I.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrow8 = (n + 7) / 8 * 8;
  for (int row = warp; row < nrow8; row += 8) {
    double s = 0.0, a = 0.0;
    if (row < n) {
      const double* p = I.A + static_cast<int64_t>(row) * n;
      const int64_t o = static_cast<int64_t>(row) * I.ld;
      for (int k = lane; k < n; k += 32) {
        const double v = p[k];
        s += v * v;
        a += fabs(v);
        float f1, f2;
        split_f64_f32(v, f1, f2);
        I.A1[o + k] = f1;
        I.A2[o + k] = f2;
        const bf16 h = __float2bfloat16_rn(f1);
        I.Ahi[o + k] = h;
        I.Alo[o + k] = __float2bfloat16_rn(f1 - __bfloat162float(h));
      }
    }
    s = brow::warp_sum_f64(s);
    a = brow::warp_sum_f64(a);
    if (lane == 0) {
      ss[row] = s;
      ra[row] = a;
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nrow8 / 8; b += kThreads) {
    double ts = 0.0, tm = 0.0;
    for (int w = 0; w < 8; ++w) {
      ts += ss[8 * b + w];
      tm = fmax(tm, ra[8 * b + w]);
    }
    I.part[2 * b] = ts;
    I.part[2 * b + 1] = tm;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- controller
// The host controller's record of one system (batch.cu, InstState) and its
// decision after a pass's norms are read (batch.cu, decide()), per system.
struct DState {
  int prec, cur, done, ns_active, finished, converged, recompute, sweeps_left;
  int stall, k_meas, resid64, status, sweeps, rollbacks, has_res, coupled, need_res, passes, prods1, prods3;
  double prev_frob, prev_ratio, frob_now, best_rr, last_rr_sweep, prev_sweep_ratio, proj_need, rel_res;
};

__device__ double step_cost_d(int n, int levels, int prec) {
  const double nd = n;
  const int prods = levels == 0 ? 3 : 2 * levels;
  return prods * 2.0 * nd * nd * nd * (prec == NS_BF16X3 ? 3.0 : 1.0) / 1.0e15 + 3e-6 * prods;
}
__device__ double sweep_cost_d(int n, int nrhs) {
  const double nd = n;
  return fmax(12.0 * nd * nd / 5.0e12, 22.0 * nd * nd * nrhs / 3.0e13) + 3e-5;
}

__device__ void decide_d(const FusedParams& p, const BInst& I, DState& s) {
  const double tol = p.tol;
  const double* sc = I.scal;
  const int nr = I.nrhs;
  double rr = INFINITY;
  s.recompute = 0;
  if (!s.has_res && s.ns_active && p.couple_frob > 0.0 && sqrt(sc[2]) <= p.couple_frob) {
    s.need_res = 1;  // the first G_k with ||I - A G_k||_F <= couple_frob
    return;
  }
  if (s.has_res) {
    rr = 0.0;
    for (int c = 0; c < nr; ++c) {
      const double bb = sc[kScalR + nr + c], r = sc[kScalR + c];
      const double q = bb > 0 ? sqrt(r / bb) : sqrt(r);
      rr = fmax(rr, isnan(q) ? INFINITY : q);
    }
    s.rel_res = rr;
    if (!isfinite(rr)) {
      s.finished = 1;
      s.status = NS_ERR_NONFINITE;
      return;
    }
    if (tol > 0 && rr <= tol) {
      s.finished = 1;
      s.converged = 1;
      s.status = NS_OK;
      return;
    }
  }
  if (!s.ns_active) {
    // Richardson alone: stop when it no longer contracts
    const double prev = s.last_rr_sweep;
    s.last_rr_sweep = rr;
    const double ratio = (isfinite(prev) && prev > 0.0) ? pow(rr / prev, 1.0 / s.k_meas) : INFINITY;
    if (isfinite(prev)) s.stall = ratio > 0.95 ? s.stall + 1 : 0;
    s.best_rr = fmin(s.best_rr, rr);
    bool stop = s.stall >= 4 || rr > 10.0 * s.best_rr;
    s.proj_need = 0.0;
    if (isfinite(ratio)) {
      const double rho = fmin(ratio, s.prev_sweep_ratio);
      s.prev_sweep_ratio = ratio;
      if (tol > 0 && rho < 1.0) {
        s.proj_need = log(tol / rr) / log(rho);
        if (s.proj_need > static_cast<double>(s.sweeps_left)) stop = true;
      }
    }
    if (stop && !s.resid64 && tol > 0 && s.sweeps_left > 0) {
      // the split-f32 residual may be what stalls: FP64 residual from here on
      s.resid64 = 1;
      s.stall = 0;
      s.best_rr = INFINITY;
      s.prev_sweep_ratio = INFINITY;
      s.proj_need = 0.0;
      stop = false;
    }
    if (stop) {
      s.finished = 1;
      s.status = NS_NOT_CONVERGED;
    }
    return;
  }
  const double frob = sqrt(sc[2]);
  if (!isfinite(frob)) {
    s.finished = 1;
    s.status = NS_ERR_NONFINITE;
    return;
  }
  const bool autop = p.precision == NS_AUTO;
  const double ratio = frob / s.prev_frob;
  if (autop && s.prec == NS_BF16 && s.done >= 2 && frob < s.prev_frob && ratio > s.prev_ratio + 0.02) {
    s.prec = NS_BF16X3;
    s.prev_ratio = INFINITY;
    s.recompute = 1;
    return;
  }
  if (autop && s.prec == NS_BF16 && s.done > 0 && frob >= s.prev_frob) {
    s.cur ^= 1;
    s.done--;
    s.prec = NS_BF16X3;
    s.prev_frob = INFINITY;
    s.rollbacks++;
    s.recompute = 1;
    return;
  }
  const double sqrt_n = sqrt(static_cast<double>(I.n));
  if (frob > 2.0 * sqrt_n + 1.0 && frob > 2.0 * s.prev_frob) {
    s.finished = 1;
    s.status = NS_ERR_DIVERGED;
    return;
  }
  if (p.ns_stop && (!autop || s.prec != NS_BF16)) {
    bool stop = frob <= p.ns_stop_frob;
    if (!stop && s.has_res && frob < 1.0 && tol > 0 && rr > tol) {
      const double need = ceil(log(tol / rr) / log(frob));
      const double tsw = sweep_cost_d(I.n, I.nrhs);
      if (need <= s.sweeps_left && need * tsw <= step_cost_d(I.n, p.levels, s.prec) + 2.0 * tsw) stop = true;
    }
    if (!stop && s.prev_frob < 1.0 && frob >= 0.5 * s.prev_frob) {
      stop = true;
      if (frob > s.prev_frob) s.cur ^= 1;
    }
    if (stop) s.ns_active = 0;
  }
  s.frob_now = frob;
}

// ---------------------------------------------------------------- the solve
__global__ void __launch_bounds__(kThreads, 1) k_bsolve(const __grid_constant__ FusedParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ DState S;
  __shared__ int sh_i, sh_k, sh_act;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_word;
  Pipe pp;
  pp.sA = smem;
  pp.sB = smem + kStages * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(pp.sB + kStages * kBBytes);
  pp.full = bars;
  pp.empty = bars + kStages;
  pp.tfull = bars + 2 * kStages;
  pp.tempty = pp.tfull + 2;
  pp.drain = pp.tempty + 2;
  pp.ebuf = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + kBarBytes);
  pp.abort_flag = &abort_word;
  pp.tlim = p.timeout_ns;
  pp.err = p.err;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&pp.full[s], 1);
      mbar_init(&pp.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&pp.tfull[a], 1);
      mbar_init(&pp.tempty[a], 128);
    }
    mbar_init(pp.drain, 1);
    abort_word = 0;
    fence_barrier_init();
    fence_proxy_async_smem();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pp.tmem = tmem_slot;
  Pos pos;

  for (;;) {
    if (tid == 0) {
      int k = abort_word ? p.count : atomicAdd(p.next, 1);
      sh_i = k < p.count ? p.list[k] : -1;
    }
    __syncthreads();
    const int i = sh_i;
    if (i < 0) break;
    const BInst& I = p.inst[i];
    const int n = I.n, nrhs = I.nrhs;
    const long long t_begin = clock64();
    auto prob = [&](int type) -> const TcProblem& {
      return p.prob[((static_cast<size_t>(i) * p.ntypes + type) * 2 + S.cur) * 2 + (S.prec == NS_BF16X3 ? 1 : 0)];
    };
    uint8_t* scratch = pp.sA;  // the stage area, idle between products
    auto residual = [&](bool rsq) {
      for (int c0 = 0; c0 < nrhs; c0 += kBRhs) {
        if (S.resid64) {
          if (nrhs == 1)
            wide_resid64_1(I, scratch);
          else
            wide_resid64<kBRhs>(I, c0, scratch);
        } else {
          if (nrhs == 1)
            wide_resid_x2_1(I, scratch);
          else
            wide_resid_x2<kBRhs>(I, c0, scratch);
        }
      }
      if (rsq) {
        brow::brsq_body(I);
        __syncthreads();
      }
    };
    auto update = [&](int cur) {
      for (int c0 = 0; c0 < nrhs; c0 += kBRhs) {
        if (nrhs == 1)
          wide_update_1(I, cur, scratch);
        else
          wide_update<kBRhs>(I, c0, cur, scratch);
      }
    };
    bool ok = true;
    auto product = [&](int type) {
      if (!ok) return;
      const bool x3 = S.prec == NS_BF16X3;
      ok = cta_product(prob(type), x3, pp, pos);
      if (tid == 0) {
        if (x3)
          S.prods3++;
        else
          S.prods1++;
      }
    };

    // ---- preparation: norms, splits and limbs of A; G0; theta = 0 and its limbs
    wide_prep(I, scratch);
    brow::bnorms_body(I);
    __syncthreads();
    for (int r0 = 0; r0 < n; r0 += 8) brow::bg0_body(I, BItem{i, r0, 0, 0}, p.g0_mode, 1);
    fence_async_global();
    if (tid == 0) {
      DState s;
      memset(&s, 0, sizeof(s));
      s.prec = p.precision == NS_AUTO ? NS_BF16 : p.precision;
      s.sweeps_left = p.max_sweeps;
      s.ns_active = p.iters > 0;
      s.status = NS_OK;
      s.prev_frob = s.prev_ratio = s.frob_now = s.best_rr = s.last_rr_sweep = s.prev_sweep_ratio = INFINITY;
      s.rel_res = INFINITY;
      s.k_meas = 1;
      S = s;
    }
    __syncthreads();

    // ---- controller passes (batch.cu, pass()) for this system alone
    while (ok) {
      if (tid == 0) {
        // Richardson-only systems far from tol take extra sweeps first
        S.k_meas = 1;
        int k = 0;
        if (!S.ns_active && S.proj_need >= 3.0) {
          k = static_cast<int>((S.proj_need - 1.0) / 2.0);
          k = min(min(k, p.max_pre), S.sweeps_left - 1);
          if (k < 1) k = 0;
        }
        sh_k = k;
      }
      __syncthreads();
      for (int j = 0; j < sh_k; ++j) {
        residual(false);
        update(S.cur);
        if (tid == 0) {
          S.sweeps++;
          S.sweeps_left--;
          S.k_meas++;
        }
        __syncthreads();
      }
      if (tid == 0) S.has_res = !S.ns_active || p.couple_frob <= 0.0 || S.coupled;
      __syncthreads();
      if (S.ns_active) {
        product(0);
        brow::bfrob_body(I);
        __syncthreads();
      }
      if (S.has_res) residual(true);
      if (tid == 0 && ok) decide_d(p, I, S);
      __syncthreads();
      // follow-ups: the coupling starts with this G_k (its residual), or the
      // precision switched / the step rolled back (F again)
      for (int guard = 0; guard < 8 && ok; ++guard) {
        if (tid == 0) {
          int act = 0;
          if (!S.finished) {
            if (S.need_res) {
              S.need_res = 0;
              S.has_res = S.coupled = 1;
              act = 1;
            } else if (S.recompute) {
              act = 2;
            }
          }
          sh_act = act;
        }
        __syncthreads();
        if (sh_act == 0) break;
        if (sh_act == 2) {
          product(0);
          brow::bfrob_body(I);
          __syncthreads();
        } else {
          residual(true);
        }
        if (tid == 0 && ok) decide_d(p, I, S);
        __syncthreads();
      }
      if (tid == 0) {
        int step = 0, upd = 0;
        if (!S.finished) {
          if (S.ns_active) {
            step = 1;
            upd = S.has_res;
          } else if (!S.has_res) {
            // Newton-Schulz stopped on a pass without a residual: the next pass forms it
          } else if (S.sweeps_left > 0) {
            upd = 1;
            S.sweeps_left--;
          } else {
            S.finished = 1;
            S.status = NS_NOT_CONVERGED;
          }
        }
        sh_act = step | (upd << 1);
      }
      __syncthreads();
      const int act = sh_act;
      if (act & 1) {
        // the chain reads G_k and writes the other G buffer
        if (p.levels == 0) {
          product(1);
          product(2);
        } else {
          for (int j = 0; j < p.levels; ++j) {
            product(1 + 2 * j);
            if (j + 1 < p.levels) product(2 + 2 * j);
          }
        }
      }
      if (act & 2) update(S.cur);  // theta += G_k r
      if (tid == 0) {
        if (act & 2) S.sweeps++;
        if (act & 1) {
          S.prev_ratio = (S.done > 0 && isfinite(S.prev_frob)) ? S.frob_now / S.prev_frob : INFINITY;
          S.prev_frob = S.frob_now;
          S.cur ^= 1;
          S.done++;
          if (S.done >= p.iters) S.ns_active = 0;
        }
        S.passes++;
        if (!S.finished && S.passes > 2 * p.iters + p.max_sweeps + 8) {
          S.finished = 1;
          S.status = NS_NOT_CONVERGED;
        }
        if (!ok) {
          S.finished = 1;
          S.status = NS_ERR_TIMEOUT;
        }
      }
      fence_async_global();
      __syncthreads();
      if (S.finished) break;
    }
    if (tid == 0) {
      if (!ok) S.status = NS_ERR_TIMEOUT;
      FusedOut o;
      o.status = S.status;
      o.done = S.done;
      o.sweeps = S.sweeps;
      o.rollbacks = S.rollbacks;
      o.converged = S.converged;
      o.passes = S.passes;
      o.prods1 = S.prods1;
      o.prods3 = S.prods3;
      o.rel_res = S.rel_res;
      o.cycles = clock64() - t_begin;
      uint32_t smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      o.sm = static_cast<int>(smid);
      o.pad = 0;
      p.out[i] = o;
    }
    __syncthreads();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(pp.tmem, kTmemCols);
  }
}

}  // namespace

cudaError_t launch_fused_solve(const FusedParams& p, int num_sms, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] { attr = cudaFuncSetAttribute(k_bsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem); });
  if (attr != cudaSuccess) return attr;
  if (p.count <= 0) return cudaSuccess;
  const int ctas = p.count < num_sms ? p.count : num_sms;
  k_bsolve<<<ctas, kThreads, kSmem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace nsgb
