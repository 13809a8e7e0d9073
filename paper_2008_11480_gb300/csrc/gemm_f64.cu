// Plain FP64 GEMM on the CUDA cores with the Newton-Schulz epilogue
//   D = s * (L R) + beta * C + gamma * I
// used by the all-FP64 path (the baseline the mixed-precision path is
// measured against).  64 x 64 output tile per 256-thread block, each thread a
// 4 x 4 sub-tile strided by 16 so that shared-memory reads are broadcast /
// conflict-free; K staged in slabs of 16.  One partial sum of D^2 per tile.
#include "internal.h"

namespace nsgb {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) k_gemm_f64(F64Gemm g) {
  __shared__ double sL[TK][TM + 1];
  __shared__ double sR[TK][TN + 1];
  __shared__ double red[8];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < g.K; k0 += TK) {
    // L tile: 64 rows x 16 k (4 per thread), stored transposed sL[k][m]
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      const int m = idx / TK, k = idx % TK;
      const int gm = m0 + m, gk = k0 + k;
      sL[k][m] = (gm < g.M && gk < g.K) ? g.L[static_cast<int64_t>(gm) * g.ldl + gk] : 0.0;
    }
    // R tile: 16 k x 64 cols
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      const int k = idx / TN, n = idx % TN;
      const int gk = k0 + k, gn = n0 + n;
      sR[k][n] = (gk < g.K && gn < g.N) ? g.R[static_cast<int64_t>(gk) * g.ldr + gn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sL[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sR[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  double frob = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = m0 + ty + 16 * i;
    if (row >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + tx + 16 * j;
      if (col >= g.N) continue;
      double v = g.s * acc[i][j];
      if (g.C != nullptr && g.beta != 0.0) v += g.beta * g.C[static_cast<int64_t>(row) * g.ldc + col];
      if (row == col) v += g.gamma;
      g.D[static_cast<int64_t>(row) * g.ldd + col] = v;
      frob += v * v;
    }
  }
  if (g.frob_partials != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) frob += __shfl_xor_sync(0xffffffffu, frob, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = frob;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      g.frob_partials[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Small products (fewer 64 x 64 tiles than half the SMs): 16 x 16 output tiles,
// one output per thread, so that e.g. n = 64 spreads over 16 SMs instead of one.
constexpr int TS = 16;

__global__ void __launch_bounds__(256) k_gemm_f64_small(F64Gemm g) {
  __shared__ double sL[TS][TS + 1];
  __shared__ double sR[TS][TS + 1];
  __shared__ double red[8];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * TS + ty, col = blockIdx.x * TS + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < g.K; k0 += TS) {
    const int lk = k0 + tx, rk = k0 + ty;
    sL[ty][tx] = (row < g.M && lk < g.K) ? g.L[static_cast<int64_t>(row) * g.ldl + lk] : 0.0;
    sR[ty][tx] = (rk < g.K && col < g.N) ? g.R[static_cast<int64_t>(rk) * g.ldr + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TS; ++k) acc = fma(sL[ty][k], sR[k][tx], acc);
    __syncthreads();
  }
  double frob = 0.0;
  if (row < g.M && col < g.N) {
    double v = g.s * acc;
    if (g.C != nullptr && g.beta != 0.0) v += g.beta * g.C[static_cast<int64_t>(row) * g.ldc + col];
    if (row == col) v += g.gamma;
    g.D[static_cast<int64_t>(row) * g.ldd + col] = v;
    frob = v * v;
  }
  if (g.frob_partials != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) frob += __shfl_xor_sync(0xffffffffu, frob, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = frob;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      g.frob_partials[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

bool use_small(int M, int N) { return ((M + TM - 1) / TM) * ((N + TN - 1) / TN) < 76; }

}  // namespace

int f64_tiles(int M, int N) {
  if (use_small(M, N)) return ((M + TS - 1) / TS) * ((N + TS - 1) / TS);
  return ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
}

cudaError_t launch_gemm_f64(const F64Gemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (use_small(g.M, g.N)) {
    dim3 grid((g.N + TS - 1) / TS, (g.M + TS - 1) / TS);
    k_gemm_f64_small<<<grid, 256, 0, s>>>(g);
  } else {
    dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM);
    k_gemm_f64<<<grid, 256, 0, s>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace nsgb
