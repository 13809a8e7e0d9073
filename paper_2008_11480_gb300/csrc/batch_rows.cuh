// Bodies of the batched row kernels (one block of 256 threads, one work item)
// shared by the list-driven launches (batch_vec.cu) and the fused small-system
// solve (batch_fused.cu), so that a system's arithmetic -- row blocks, k split,
// reduction order -- is the same on both paths.  Every body is entered by all
// 256 threads of the block together (they synchronise inside).
#pragma once
#include "batch.h"
#include "split.cuh"

namespace nsgb {
namespace brow {

constexpr int kRows = 8;  // rows per block, as in the single-system kernels

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p) {
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err;
}

__device__ __forceinline__ void warp_sum_x2(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = hi + oh;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (oh - bb);
    const float l = lo + ol + err;
    hi = s + l;
    lo = l - (hi - s);
  }
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- preparation of A
// 8 rows per block, one warp per row: norms partials (FP64), bf16 hi/lo and f32 limbs.
__device__ __forceinline__ void bprep_body(const BInst& I, const BItem it) {
  __shared__ double ss[8], ra[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = it.row0 + warp;
  const int n = I.n;
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
  s = warp_sum_f64(s);
  a = warp_sum_f64(a);
  if (lane == 0) {
    ss[warp] = s;
    ra[warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tm = 0.0;
    for (int w = 0; w < 8; ++w) {
      ts += ss[w];
      tm = fmax(tm, ra[w]);
    }
    const int b = it.row0 / kRows;
    I.part[2 * b] = ts;
    I.part[2 * b + 1] = tm;
  }
}

// Per instance (one block each): ||A||_F^2 and ||A||_inf from the row-block
// partials, in fixed order; also ||b_c||^2 per right-hand side.
__device__ __forceinline__ void bnorms_body(const BInst& I) {
  __shared__ double red[256], redm[256];
  const int nrb = (I.n + kRows - 1) / kRows;
  double s = 0.0, m = 0.0;
  for (int b = threadIdx.x; b < nrb; b += 256) {
    s += I.part[2 * b];
    m = fmax(m, I.part[2 * b + 1]);
  }
  red[threadIdx.x] = s;
  redm[threadIdx.x] = m;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[threadIdx.x] += red[threadIdx.x + h];
      redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    I.scal[0] = red[0];
    I.scal[1] = redm[0];
  }
  // ||b_c||^2: warp c handles rhs c, c + 8, ...
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < I.nrhs; c += 8) {
    double t = 0.0;
    for (int r = lane; r < I.n; r += 32) {
      const double v = I.B[static_cast<int64_t>(r) * I.nrhs + c];
      t += v * v;
    }
    t = warp_sum_f64(t);
    if (lane == 0) I.scal[kScalR + I.nrhs + c] = t;
  }
}

// G0 = alpha I with alpha = 1/||A||_F (mode 0) or 1/(||A||_inf/2 + eps) (mode 1),
// written into G[0] (f32 master and bf16 split) for rows [row0, row0 + 8); and
// the f32 limbs of theta for those rows.
__device__ __forceinline__ void bg0_body(const BInst& I, const BItem it, int mode, int zero_theta) {
  const double sA = I.scal[0], ninf = I.scal[1];
  const float alpha = static_cast<float>(mode == 0 ? 1.0 / sqrt(sA) : 1.0 / (0.5 * ninf + 1e-8 * ninf));
  const bf16 ah = __float2bfloat16_rn(alpha);
  const bf16 al = __float2bfloat16_rn(alpha - __bfloat162float(ah));
  const bf16 z = __float2bfloat16_rn(0.f);
  const int n = I.n;
  for (int e = threadIdx.x; e < kRows * n; e += 256) {
    const int r = it.row0 + e / n, c = e % n;
    if (r >= n) continue;
    const int64_t o = static_cast<int64_t>(r) * I.ld + c;
    const bool d = r == c;
    if (mode == 2) {
      // Jacobi splitting S = diag(A) (Section 2): G0 = S^{-1}, as the single-system kernel forms it
      const float f = d ? static_cast<float>(1.0 / I.A[static_cast<int64_t>(r) * n + r]) : 0.f;
      const bf16 h = __float2bfloat16_rn(f);
      I.G32[0][o] = f;
      I.Ghi[0][o] = d ? h : z;
      I.Glo[0][o] = d ? __float2bfloat16_rn(f - __bfloat162float(h)) : z;
      continue;
    }
    I.G32[0][o] = d ? alpha : 0.f;
    I.Ghi[0][o] = d ? ah : z;
    I.Glo[0][o] = d ? al : z;
  }
  for (int e = threadIdx.x; e < kRows * I.nrhs; e += 256) {
    const int r = it.row0 + e / I.nrhs, c = e % I.nrhs;
    if (r >= n) continue;
    double v = I.Th[static_cast<int64_t>(r) * I.nrhs + c];
    if (zero_theta) {
      v = 0.0;
      I.Th[static_cast<int64_t>(r) * I.nrhs + c] = 0.0;
    }
    const float f1 = static_cast<float>(v);
    I.T1[static_cast<int64_t>(c) * I.ld + r] = f1;
    I.T2[static_cast<int64_t>(c) * I.ld + r] = static_cast<float>(v - static_cast<double>(f1));
  }
}

// ---------------------------------------------------------------- residual
// Same arithmetic as the single-system split-f32 residual: warp = (row pair,
// half of the k range), kBRhs right-hand sides [c0, c0 + kBRhs) masked to nrhs.
__device__ __forceinline__ void bresid_body(const BInst& I, const BItem it) {
  constexpr int NR = kBRhs;
  __shared__ float red_hi[4][2][NR][2], red_lo[4][2][NR][2];
  __shared__ double sq[kRows][NR];
  const int n = I.n, nrhs = I.nrhs, c0 = it.c0;
  const int64_t ld = I.ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp & 3, half = warp >> 2;
  const int row0 = it.row0 + pair * 2;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const int64_t o0 = static_cast<int64_t>(r0 ? row0 : 0) * ld;
  const int64_t o1 = static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
  bool cv[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) cv[c] = c0 + c < nrhs;
  float hi[2][NR], lo[2][NR];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) hi[r][c] = lo[r][c] = 0.f;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
  for (int k = 4 * lane + 128 * half; k < n4; k += 256) {
    const float4 x0 = r0 ? *reinterpret_cast<const float4*>(I.A1 + o0 + k) : z4;
    const float4 y0 = r0 ? *reinterpret_cast<const float4*>(I.A2 + o0 + k) : z4;
    const float4 x1 = r1 ? *reinterpret_cast<const float4*>(I.A1 + o1 + k) : z4;
    const float4 y1 = r1 ? *reinterpret_cast<const float4*>(I.A2 + o1 + k) : z4;
    const float a1v[2][4] = {{x0.x, x0.y, x0.z, x0.w}, {x1.x, x1.y, x1.z, x1.w}};
    const float a2v[2][4] = {{y0.x, y0.y, y0.z, y0.w}, {y1.x, y1.y, y1.z, y1.w}};
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      if (!cv[c]) continue;
      const float4 u = *reinterpret_cast<const float4*>(I.T1 + (c0 + c) * ld + k);
      const float4 w = *reinterpret_cast<const float4*>(I.T2 + (c0 + c) * ld + k);
      const float t1v[4] = {u.x, u.y, u.z, u.w};
      const float t2v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = a1v[r][j] * t1v[j];
          const float e = fmaf(a1v[r][j], t1v[j], -p);
          two_sum_acc(hi[r][c], lo[r][c], p);
          lo[r][c] += fmaf(a1v[r][j], t2v[j], fmaf(a2v[r][j], t1v[j], e));
        }
    }
  }
  if (half == 0) {
    for (int k = n4 + lane; k < n; k += 32) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const bool ok = r == 0 ? r0 : r1;
        const int64_t o = r == 0 ? o0 : o1;
        const float x = ok ? I.A1[o + k] : 0.f, y = ok ? I.A2[o + k] : 0.f;
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          if (!cv[c]) continue;
          const float t1 = I.T1[(c0 + c) * ld + k], t2 = I.T2[(c0 + c) * ld + k];
          const float p = x * t1;
          const float e = fmaf(x, t1, -p);
          two_sum_acc(hi[r][c], lo[r][c], p);
          lo[r][c] += fmaf(x, t2, fmaf(y, t1, e));
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      warp_sum_x2(hi[r][c], lo[r][c]);
      if (lane == 0) {
        red_hi[pair][half][c][r] = hi[r][c];
        red_lo[pair][half][c][r] = lo[r][c];
      }
    }
  __syncthreads();
  if (threadIdx.x < kRows * NR) {
    const int rr = threadIdx.x / NR, c = threadIdx.x % NR;
    const int pr = rr >> 1, r = rr & 1;
    const int row = it.row0 + rr;
    double v2 = 0.0;
    if (row < n && c0 + c < nrhs) {
      const double sdot = (static_cast<double>(red_hi[pr][0][c][r]) + static_cast<double>(red_lo[pr][0][c][r])) +
                          (static_cast<double>(red_hi[pr][1][c][r]) + static_cast<double>(red_lo[pr][1][c][r]));
      const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
      const double v = I.B[o] - sdot;
      I.R[o] = v;
      I.R32T[static_cast<int64_t>(c0 + c) * ld + row] = static_cast<float>(v);
      v2 = v * v;
    }
    sq[rr][c] = v2;
  }
  __syncthreads();
  if (threadIdx.x < NR && c0 + static_cast<int>(threadIdx.x) < nrhs) {
    double t = 0.0;
    for (int w = 0; w < kRows; ++w) t += sq[w][threadIdx.x];
    I.part[static_cast<int64_t>(it.row0 / kRows) * nrhs + c0 + threadIdx.x] = t;
  }
}

// FP64 residual for systems whose split-f32 residual stalled above tol:
// R = B - A Theta from the caller's FP64 A and the FP64 theta, one warp per row
// (lanes stride k, fixed-order shuffle reduction), 8 rows x kBRhs RHS per
// block; also R32T (the update's operand) and the block's sums of R^2.
__device__ __forceinline__ void bresid64_body(const BInst& I, const BItem it) {
  constexpr int NR = kBRhs;
  __shared__ double sq[kRows][NR];
  const int n = I.n, nrhs = I.nrhs, c0 = it.c0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = it.row0 + warp;
  double acc[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = 0.0;
  if (row < n) {
    const double* a = I.A + static_cast<int64_t>(row) * n;
    for (int k = lane; k < n; k += 32) {
      const double av = a[k];
      const double* t = I.Th + static_cast<int64_t>(k) * nrhs + c0;
#pragma unroll
      for (int c = 0; c < NR; ++c)
        if (c0 + c < nrhs) acc[c] = fma(av, t[c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = warp_sum_f64(acc[c]);
  if (lane < NR) {
    const int c = lane;
    double v2 = 0.0;
    if (row < n && c0 + c < nrhs) {
      double dot = 0.0;
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (j == c) dot = acc[j];
      const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
      const double v = I.B[o] - dot;
      I.R[o] = v;
      I.R32T[static_cast<int64_t>(c0 + c) * I.ld + row] = static_cast<float>(v);
      v2 = v * v;
    }
    sq[warp][c] = v2;
  }
  __syncthreads();
  if (threadIdx.x < NR && c0 + static_cast<int>(threadIdx.x) < nrhs) {
    double t = 0.0;
    for (int w = 0; w < kRows; ++w) t += sq[w][threadIdx.x];
    I.part[static_cast<int64_t>(it.row0 / kRows) * nrhs + c0 + threadIdx.x] = t;
  }
}

// Per instance: ||r_c||^2 from the residual's row-block partials (fixed order).
__device__ __forceinline__ void brsq_body(const BInst& I) {
  const int nrb = (I.n + kRows - 1) / kRows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < I.nrhs; c += 8) {
    double t = 0.0;
    for (int b = lane; b < nrb; b += 32) t += I.part[static_cast<int64_t>(b) * I.nrhs + c];
    t = warp_sum_f64(t);
    if (lane == 0) I.scal[kScalR + c] = t;
  }
}

// Theta += G R (G = the instance's f32 master G[cur]); new theta's limbs too.
__device__ __forceinline__ void bupdate_body(const BInst& I, const BItem it) {
  constexpr int NR = kBRhs;
  __shared__ float red[4][2][NR][2];
  const int n = I.n, nrhs = I.nrhs, c0 = it.c0;
  const int64_t ld = I.ld;
  const float* G = I.G32[it.cur];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp & 3, half = warp >> 2;
  const int row0 = it.row0 + pair * 2;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const float* g0 = G + static_cast<int64_t>(r0 ? row0 : 0) * ld;
  const float* g1 = G + static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
  bool cv[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) cv[c] = c0 + c < nrhs;
  float acc[2][NR];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[r][c] = 0.f;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
  for (int k = 4 * lane + 128 * half; k < n4; k += 256) {
    const float4 x0 = r0 ? *reinterpret_cast<const float4*>(g0 + k) : z4;
    const float4 x1 = r1 ? *reinterpret_cast<const float4*>(g1 + k) : z4;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      if (!cv[c]) continue;
      const float4 t = *reinterpret_cast<const float4*>(I.R32T + (c0 + c) * ld + k);
      acc[0][c] = fmaf(x0.x, t.x, fmaf(x0.y, t.y, fmaf(x0.z, t.z, fmaf(x0.w, t.w, acc[0][c]))));
      acc[1][c] = fmaf(x1.x, t.x, fmaf(x1.y, t.y, fmaf(x1.z, t.z, fmaf(x1.w, t.w, acc[1][c]))));
    }
  }
  if (half == 0) {
    for (int k = n4 + lane; k < n; k += 32) {
      const float x0 = r0 ? g0[k] : 0.f;
      const float x1 = r1 ? g1[k] : 0.f;
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        if (!cv[c]) continue;
        const float t = I.R32T[(c0 + c) * ld + k];
        acc[0][c] = fmaf(x0, t, acc[0][c]);
        acc[1][c] = fmaf(x1, t, acc[1][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const float sred = warp_sum_f32(acc[r][c]);
      if (lane == 0) red[pair][half][c][r] = sred;
    }
  __syncthreads();
  if (threadIdx.x < kRows * NR) {
    const int rr = threadIdx.x / NR, c = threadIdx.x % NR;
    const int pr = rr >> 1, r = rr & 1;
    const int row = it.row0 + rr;
    if (row < n && c0 + c < nrhs) {
      const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
      const double v = I.Th[o] + (static_cast<double>(red[pr][0][c][r]) + static_cast<double>(red[pr][1][c][r]));
      I.Th[o] = v;
      const float f1 = static_cast<float>(v);
      I.T1[static_cast<int64_t>(c0 + c) * ld + row] = f1;
      I.T2[static_cast<int64_t>(c0 + c) * ld + row] = static_cast<float>(v - static_cast<double>(f1));
    }
  }
}

// Per instance: ||F||_F^2 from the product kernel's per-tile partials.
__device__ __forceinline__ void bfrob_body(const BInst& I) {
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < I.nfrob; b += 256) s += I.fpart[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) I.scal[2] = red[0];
}

}  // namespace brow
}  // namespace nsgb
