// Memory-bound kernels around the GEMM chain: the Richardson residual
// R = B - A Theta (FP64), the update Theta += G R, matrix/column norms,
// fixed-order (deterministic) reductions, the bf16 hi/lo splits and G0.
#include "internal.h"
#include "ptx.cuh"
#include "split.cuh"

namespace nsgb {
namespace {

constexpr int kRowsPerWarp = 2;
constexpr int kWarps = 8;
constexpr int kRowsPerBlock = kRowsPerWarp * kWarps;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- residual
// Each warp owns two consecutive rows; lanes stride the row with 16-byte
// loads (two doubles) when rows are 16-byte aligned.  NR right-hand sides
// [c0, c0+NR) are handled per launch.
template <int NR, bool VEC>
__global__ void __launch_bounds__(256) k_resid(const double* __restrict__ A, int64_t lda,
                                               const double* __restrict__ Th, const double* __restrict__ B,
                                               double* __restrict__ R, int n, int nrhs, int c0,
                                               double* __restrict__ partials) {
  __shared__ double sq[kWarps][NR];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * kRowsPerBlock + warp * kRowsPerWarp;
  double acc[kRowsPerWarp][NR];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[r][c] = 0.0;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const double* a0p = A + static_cast<int64_t>(r0 ? row0 : 0) * lda;
  const double* a1p = A + static_cast<int64_t>(r1 ? row0 + 1 : 0) * lda;
  int kend = 0;
  if (VEC) {
    const int n2 = n & ~1;
#pragma unroll 4
    for (int k = 2 * lane; k < n2; k += 64) {
      const double2 x0 = r0 ? *reinterpret_cast<const double2*>(a0p + k) : make_double2(0.0, 0.0);
      const double2 x1 = r1 ? *reinterpret_cast<const double2*>(a1p + k) : make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const double t0 = __ldg(Th + static_cast<int64_t>(k) * nrhs + c0 + c);
        const double t1 = __ldg(Th + static_cast<int64_t>(k + 1) * nrhs + c0 + c);
        acc[0][c] = fma(x0.x, t0, acc[0][c]);
        acc[0][c] = fma(x0.y, t1, acc[0][c]);
        acc[1][c] = fma(x1.x, t0, acc[1][c]);
        acc[1][c] = fma(x1.y, t1, acc[1][c]);
      }
    }
    kend = n2;
  }
  for (int k = kend + lane; k < n; k += 32) {
    const double x0 = r0 ? a0p[k] : 0.0;
    const double x1 = r1 ? a1p[k] : 0.0;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double t = __ldg(Th + static_cast<int64_t>(k) * nrhs + c0 + c);
      acc[0][c] = fma(x0, t, acc[0][c]);
      acc[1][c] = fma(x1, t, acc[1][c]);
    }
  }
  double mysq[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) mysq[c] = 0.0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double s = warp_sum(acc[r][c]);
      const int row = row0 + r;
      if (lane == 0 && row < n) {
        const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
        const double v = B[o] - s;
        R[o] = v;
        mysq[c] += v * v;
      }
    }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NR; ++c) sq[warp][c] = mysq[c];
  __syncthreads();
  if (threadIdx.x < NR) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += sq[w][threadIdx.x];
    partials[static_cast<int64_t>(blockIdx.x) * nrhs + c0 + threadIdx.x] = t;
  }
}

template <int NR>
void resid_chunk(const double* A, int64_t lda, const double* Th, const double* B, double* R, int n, int nrhs,
                 int c0, double* partials, int nb, bool vec, cudaStream_t s) {
  if (vec)
    k_resid<NR, true><<<nb, 256, 0, s>>>(A, lda, Th, B, R, n, nrhs, c0, partials);
  else
    k_resid<NR, false><<<nb, 256, 0, s>>>(A, lda, Th, B, R, n, nrhs, c0, partials);
}

// ---------------------------------------------------------------- update
// Theta[i][c] += sum_k G[i][k] R[k][c].  With an f32 G the products and each
// lane's running sum are f32 (G itself is only an f32 approximation of the
// inverse, so this adds an error well below G's own); lane sums are combined
// in f64 and added to the f64 Theta.
template <int NR, bool VEC>
__global__ void __launch_bounds__(256) k_update_f32(const float* __restrict__ G, int64_t ldg,
                                                    const double* __restrict__ Rm, double* __restrict__ Th, int n,
                                                    int nrhs, int c0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * kRowsPerBlock + warp * kRowsPerWarp;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const float* g0 = G + static_cast<int64_t>(r0 ? row0 : 0) * ldg;
  const float* g1 = G + static_cast<int64_t>(r1 ? row0 + 1 : 0) * ldg;
  float acc[kRowsPerWarp][NR];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[r][c] = 0.f;
  int kend = 0;
  if (VEC) {
    const int n4 = n & ~3;
#pragma unroll 2
    for (int k = 4 * lane; k < n4; k += 128) {
      const float4 x0 = r0 ? *reinterpret_cast<const float4*>(g0 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 x1 = r1 ? *reinterpret_cast<const float4*>(g1 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const float t0 = static_cast<float>(__ldg(Rm + static_cast<int64_t>(k) * nrhs + c0 + c));
        const float t1 = static_cast<float>(__ldg(Rm + static_cast<int64_t>(k + 1) * nrhs + c0 + c));
        const float t2 = static_cast<float>(__ldg(Rm + static_cast<int64_t>(k + 2) * nrhs + c0 + c));
        const float t3 = static_cast<float>(__ldg(Rm + static_cast<int64_t>(k + 3) * nrhs + c0 + c));
        acc[0][c] = fmaf(x0.x, t0, fmaf(x0.y, t1, fmaf(x0.z, t2, fmaf(x0.w, t3, acc[0][c]))));
        acc[1][c] = fmaf(x1.x, t0, fmaf(x1.y, t1, fmaf(x1.z, t2, fmaf(x1.w, t3, acc[1][c]))));
      }
    }
    kend = n4;
  }
  for (int k = kend + lane; k < n; k += 32) {
    const float x0 = r0 ? g0[k] : 0.f;
    const float x1 = r1 ? g1[k] : 0.f;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const float t = static_cast<float>(__ldg(Rm + static_cast<int64_t>(k) * nrhs + c0 + c));
      acc[0][c] = fmaf(x0, t, acc[0][c]);
      acc[1][c] = fmaf(x1, t, acc[1][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double s = warp_sum(static_cast<double>(acc[r][c]));
      const int row = row0 + r;
      if (lane == 0 && row < n) Th[static_cast<int64_t>(row) * nrhs + c0 + c] += s;
    }
}

template <int NR, bool VEC>
__global__ void __launch_bounds__(256) k_update_f64(const double* __restrict__ G, int64_t ldg,
                                                    const double* __restrict__ Rm, double* __restrict__ Th, int n,
                                                    int nrhs, int c0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * kRowsPerBlock + warp * kRowsPerWarp;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const double* g0 = G + static_cast<int64_t>(r0 ? row0 : 0) * ldg;
  const double* g1 = G + static_cast<int64_t>(r1 ? row0 + 1 : 0) * ldg;
  double acc[kRowsPerWarp][NR];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[r][c] = 0.0;
  int kend = 0;
  if (VEC) {
    const int n2 = n & ~1;
#pragma unroll 4
    for (int k = 2 * lane; k < n2; k += 64) {
      const double2 x0 = r0 ? *reinterpret_cast<const double2*>(g0 + k) : make_double2(0.0, 0.0);
      const double2 x1 = r1 ? *reinterpret_cast<const double2*>(g1 + k) : make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const double t0 = __ldg(Rm + static_cast<int64_t>(k) * nrhs + c0 + c);
        const double t1 = __ldg(Rm + static_cast<int64_t>(k + 1) * nrhs + c0 + c);
        acc[0][c] = fma(x0.x, t0, fma(x0.y, t1, acc[0][c]));
        acc[1][c] = fma(x1.x, t0, fma(x1.y, t1, acc[1][c]));
      }
    }
    kend = n2;
  }
  for (int k = kend + lane; k < n; k += 32) {
    const double x0 = r0 ? g0[k] : 0.0;
    const double x1 = r1 ? g1[k] : 0.0;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double t = __ldg(Rm + static_cast<int64_t>(k) * nrhs + c0 + c);
      acc[0][c] = fma(x0, t, acc[0][c]);
      acc[1][c] = fma(x1, t, acc[1][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double s = warp_sum(acc[r][c]);
      const int row = row0 + r;
      if (lane == 0 && row < n) Th[static_cast<int64_t>(row) * nrhs + c0 + c] += s;
    }
}

// ---------------------------------------------------------------- norms
// One block per column: fixed-order strided sums then a fixed-order tree.
__global__ void k_colsumsq(const double* __restrict__ X, int64_t ldx, int rows, int cols,
                           double* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < rows; r += 256) {
    const double v = X[static_cast<int64_t>(r) * ldx + c];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// One warp per row: sum of squares and sum of |a|; block partials (8 rows).
__global__ void __launch_bounds__(256) k_matnorms(const double* __restrict__ A, int64_t lda, int n,
                                                  double* __restrict__ ss_part, double* __restrict__ rm_part) {
  __shared__ double ss[kWarps], ra[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kWarps + warp;
  double s = 0.0, a = 0.0;
  if (row < n) {
    const double* p = A + static_cast<int64_t>(row) * lda;
    for (int k = lane; k < n; k += 32) {
      const double v = p[k];
      s += v * v;
      a += fabs(v);
    }
  }
  s = warp_sum(s);
  a = warp_sum(a);
  if (lane == 0) {
    ss[warp] = s;
    ra[warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tm = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      ts += ss[w];
      tm = fmax(tm, ra[w]);
    }
    ss_part[blockIdx.x] = ts;
    rm_part[blockIdx.x] = tm;
  }
}

__global__ void k_reduce_sum(const double* __restrict__ part, int nblocks, int ncols, double* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) s += part[static_cast<int64_t>(b) * ncols + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

__global__ void k_reduce_max(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) s = fmax(s, part[b]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// ---------------------------------------------------------------- splits
// hi = RN_bf16(RN_f32(x)), lo = RN_bf16(RN_f32(x) - hi) (difference exact in f32).
// bf16 split of binary32 values: hi = bf16(v), lo = bf16(v - hi) and, when
// lo2 is given, lo2 = bf16(v - hi - lo); every difference is exact in binary32.
__device__ __forceinline__ void split_store(float v, bf16* hi, bf16* lo, bf16* lo2, int64_t o) {
  const bf16 h = __float2bfloat16_rn(v);
  const float r = v - __bfloat162float(h);
  const bf16 l = __float2bfloat16_rn(r);
  hi[o] = h;
  lo[o] = l;
  if (lo2 != nullptr) lo2[o] = __float2bfloat16_rn(r - __bfloat162float(l));
}

__global__ void k_split_f64(const double* __restrict__ X, int64_t ldx, int rows, int cols, bf16* __restrict__ hi,
                            bf16* __restrict__ lo, bf16* __restrict__ lo2, float* __restrict__ x32, int64_t ld) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    const float v = static_cast<float>(X[r * ldx + c]);
    split_store(v, hi, lo, lo2, r * ld + c);
    if (x32 != nullptr) x32[r * ld + c] = v;
  }
}

__global__ void k_split_f32(const float* __restrict__ X, int64_t ldx, int rows, int cols, bf16* __restrict__ hi,
                            bf16* __restrict__ lo, bf16* __restrict__ lo2, int64_t ld) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    split_store(X[r * ldx + c], hi, lo, lo2, r * ld + c);
  }
}

__device__ __forceinline__ double g0_alpha(const double* scal, int mode) {
  if (mode == 0) return 1.0 / sqrt(scal[0]);
  const double ninf = scal[1];
  return 1.0 / (0.5 * ninf + 1e-8 * ninf);
}

__global__ void k_init_g0_mp(const double* __restrict__ scal, int mode, int n, int64_t ld, float* __restrict__ G32,
                             bf16* __restrict__ hi, bf16* __restrict__ lo) {
  const float a = static_cast<float>(g0_alpha(scal, mode));
  const bf16 ah = __float2bfloat16_rn(a);
  const bf16 al = __float2bfloat16_rn(a - __bfloat162float(ah));
  const bf16 z = __float2bfloat16_rn(0.f);
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n, c = e % n;
    const bool d = r == c;
    G32[r * ld + c] = d ? a : 0.f;
    hi[r * ld + c] = d ? ah : z;
    lo[r * ld + c] = d ? al : z;
  }
}

__global__ void k_init_g0_f64(const double* __restrict__ scal, int mode, int n, int64_t ld, double* __restrict__ G) {
  const double a = g0_alpha(scal, mode);
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n, c = e % n;
    G[r * ld + c] = (r == c) ? a : 0.0;
  }
}

// Jacobi preconditioner S^{-1} = diag(A)^{-1} (Section 2, S = diag(A)) as G0:
// the f32 master and bf16 split (mixed path) or FP64.
__global__ void k_init_g0_jacobi(const double* __restrict__ A, int64_t lda, int n, int64_t ld,
                                 float* __restrict__ G32, bf16* __restrict__ hi, bf16* __restrict__ lo,
                                 double* __restrict__ G64) {
  const int64_t total = static_cast<int64_t>(n) * n;
  const bf16 z = __float2bfloat16_rn(0.f);
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n, c = e % n;
    const double d = r == c ? 1.0 / A[r * lda + r] : 0.0;
    if (G64 != nullptr) {
      G64[r * ld + c] = d;
    } else {
      const float f = static_cast<float>(d);
      const bf16 h = __float2bfloat16_rn(f);
      G32[r * ld + c] = f;
      hi[r * ld + c] = r == c ? h : z;
      lo[r * ld + c] = r == c ? __float2bfloat16_rn(f - __bfloat162float(h)) : z;
    }
  }
}

__global__ void k_f32_to_f64(const float* __restrict__ X, int64_t ldx, int rows, int cols, double* __restrict__ Y,
                             int64_t ldy) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    Y[r * ldy + c] = static_cast<double>(X[r * ldx + c]);
  }
}

// Rademacher probe matrix Z (rows x probes, row-major, ld = probes): entry
// (i, j) is -1 when the top bit of SplitMix64 output number k = j rows + i
// after state `seed` is set, else +1.  SplitMix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", 2014): output k is
// mix(seed + (k + 1) * 0x9E3779B97F4A7C15) with the finalizer below.
__global__ void k_rademacher(double* __restrict__ Z, int rows, int probes, unsigned long long seed) {
  const int64_t total = static_cast<int64_t>(rows) * probes;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    unsigned long long z = seed + static_cast<unsigned long long>(k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int64_t i = k % rows, j = k / rows;
    Z[i * probes + j] = (z >> 63) ? -1.0 : 1.0;
  }
}

__global__ void k_copy_f64(const double* __restrict__ X, int64_t ldx, int rows, int cols, double* __restrict__ Y,
                           int64_t ldy) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    Y[r * ldy + c] = X[r * ldx + c];
  }
}

int ew_grid(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : static_cast<int>(g);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }


// TF32 forms of an f32 matrix: Y = RN_tf32(X) (row-major, ldt) and
// YT = RN_tf32(X)^T (ldt), through a 32 x 33 shared tile so that both the
// reads and the transposed writes cover whole rows of 32 words.
__global__ void __launch_bounds__(256) k_tf32_pack(const float* __restrict__ X, int64_t ld, int rows, int cols,
                                                   float* __restrict__ Y, float* __restrict__ YT, int64_t ldt) {
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32 threads
  for (int r = ty; r < 32; r += 8) {
    const int row = by + r, col = bx + tx;
    float v = 0.f;
    if (row < rows && col < cols) {
      v = rna_tf32(X[static_cast<int64_t>(row) * ld + col]);
      if (Y != nullptr) Y[static_cast<int64_t>(row) * ldt + col] = v;
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  if (YT == nullptr) return;
  for (int r = ty; r < 32; r += 8) {
    const int orow = bx + r, ocol = by + tx;  // YT row = X column
    if (orow < cols && ocol < rows) YT[static_cast<int64_t>(orow) * ldt + ocol] = tile[tx][r];
  }
}

}  // namespace

int resid_blocks(int n) { return (n + kRowsPerBlock - 1) / kRowsPerBlock; }

cudaError_t launch_resid(const double* A, int64_t lda, const double* Th, const double* B, double* R, int n, int nrhs,
                         double* partials, int* nblocks_out, cudaStream_t s) {
  const int nb = resid_blocks(n);
  if (nblocks_out) *nblocks_out = nb;
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const bool vec = (lda % 2 == 0) && aligned16(A);
  int c0 = 0;
  while (c0 < nrhs) {
    const int left = nrhs - c0;
    if (left >= 8) {
      resid_chunk<8>(A, lda, Th, B, R, n, nrhs, c0, partials, nb, vec, s);
      c0 += 8;
    } else if (left >= 4) {
      resid_chunk<4>(A, lda, Th, B, R, n, nrhs, c0, partials, nb, vec, s);
      c0 += 4;
    } else if (left >= 2) {
      resid_chunk<2>(A, lda, Th, B, R, n, nrhs, c0, partials, nb, vec, s);
      c0 += 2;
    } else {
      resid_chunk<1>(A, lda, Th, B, R, n, nrhs, c0, partials, nb, vec, s);
      c0 += 1;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_update_f32(const float* G, int64_t ldg, const double* R, double* Th, int n, int nrhs,
                              cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int nb = resid_blocks(n);
  const bool vec = (ldg % 4 == 0) && aligned16(G);
  int c0 = 0;
  while (c0 < nrhs) {
    const int left = nrhs - c0;
    const int nr = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
#define NSGB_UPD(NRV)                                                                  \
  if (nr == NRV) {                                                                     \
    if (vec)                                                                           \
      k_update_f32<NRV, true><<<nb, 256, 0, s>>>(G, ldg, R, Th, n, nrhs, c0);          \
    else                                                                               \
      k_update_f32<NRV, false><<<nb, 256, 0, s>>>(G, ldg, R, Th, n, nrhs, c0);         \
  }
    NSGB_UPD(8) NSGB_UPD(4) NSGB_UPD(2) NSGB_UPD(1)
#undef NSGB_UPD
    c0 += nr;
  }
  return cudaGetLastError();
}

cudaError_t launch_update_f64(const double* G, int64_t ldg, const double* R, double* Th, int n, int nrhs,
                              cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int nb = resid_blocks(n);
  const bool vec = (ldg % 2 == 0) && aligned16(G);
  int c0 = 0;
  while (c0 < nrhs) {
    const int left = nrhs - c0;
    const int nr = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
#define NSGB_UPD(NRV)                                                                  \
  if (nr == NRV) {                                                                     \
    if (vec)                                                                           \
      k_update_f64<NRV, true><<<nb, 256, 0, s>>>(G, ldg, R, Th, n, nrhs, c0);          \
    else                                                                               \
      k_update_f64<NRV, false><<<nb, 256, 0, s>>>(G, ldg, R, Th, n, nrhs, c0);         \
  }
    NSGB_UPD(8) NSGB_UPD(4) NSGB_UPD(2) NSGB_UPD(1)
#undef NSGB_UPD
    c0 += nr;
  }
  return cudaGetLastError();
}

cudaError_t launch_colsumsq(const double* X, int64_t ldx, int rows, int cols, double* out, int* nblocks_out,
                            cudaStream_t s) {
  if (nblocks_out) *nblocks_out = 1;
  if (cols <= 0) return cudaSuccess;
  k_colsumsq<<<cols, 256, 0, s>>>(X, ldx, rows, cols, out);
  return cudaGetLastError();
}

cudaError_t launch_matnorms(const double* A, int64_t lda, int n, double* ss_part, double* rm_part, int* nblocks_out,
                            cudaStream_t s) {
  const int nb = (n + kWarps - 1) / kWarps;
  if (nblocks_out) *nblocks_out = nb;
  if (n <= 0) return cudaSuccess;
  k_matnorms<<<nb, 256, 0, s>>>(A, lda, n, ss_part, rm_part);
  return cudaGetLastError();
}

cudaError_t launch_reduce_sum(const double* part, int nblocks, int ncols, double* out, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  k_reduce_sum<<<ncols, 256, 0, s>>>(part, nblocks, ncols, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_max(const double* part, int nblocks, double* out, cudaStream_t s) {
  k_reduce_max<<<1, 256, 0, s>>>(part, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_split_f64(const double* X, int64_t ldx, int rows, int cols, bf16* hi, bf16* lo, float* x32,
                             int64_t ld, cudaStream_t s, bf16* lo2) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  if (total <= 0) return cudaSuccess;
  k_split_f64<<<ew_grid(total), 256, 0, s>>>(X, ldx, rows, cols, hi, lo, lo2, x32, ld);
  return cudaGetLastError();
}

cudaError_t launch_split_f32(const float* X, int64_t ldx, int rows, int cols, bf16* hi, bf16* lo, int64_t ld,
                             cudaStream_t s, bf16* lo2) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  if (total <= 0) return cudaSuccess;
  k_split_f32<<<ew_grid(total), 256, 0, s>>>(X, ldx, rows, cols, hi, lo, lo2, ld);
  return cudaGetLastError();
}

cudaError_t launch_init_g0_mp(const double* scal, int mode, int n, int64_t ld, float* G32, bf16* hi, bf16* lo,
                              cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_init_g0_mp<<<ew_grid(total), 256, 0, s>>>(scal, mode, n, ld, G32, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_init_g0_f64(const double* scal, int mode, int n, int64_t ld, double* G, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_init_g0_f64<<<ew_grid(total), 256, 0, s>>>(scal, mode, n, ld, G);
  return cudaGetLastError();
}

cudaError_t launch_init_g0_jacobi(const double* A, int64_t lda, int n, int64_t ld, float* G32, bf16* hi, bf16* lo,
                                  double* G64, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_init_g0_jacobi<<<ew_grid(total), 256, 0, s>>>(A, lda, n, ld, G32, hi, lo, G64);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* X, int64_t ldx, int rows, int cols, double* Y, int64_t ldy,
                              cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  if (total <= 0) return cudaSuccess;
  k_f32_to_f64<<<ew_grid(total), 256, 0, s>>>(X, ldx, rows, cols, Y, ldy);
  return cudaGetLastError();
}

cudaError_t launch_rademacher(double* Z, int rows, int probes, unsigned long long seed, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(rows) * probes;
  if (total <= 0) return cudaSuccess;
  k_rademacher<<<ew_grid(total), 256, 0, s>>>(Z, rows, probes, seed);
  return cudaGetLastError();
}

cudaError_t launch_copy_f64(const double* X, int64_t ldx, int rows, int cols, double* Y, int64_t ldy,
                            cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(rows) * cols;
  if (total <= 0) return cudaSuccess;
  k_copy_f64<<<ew_grid(total), 256, 0, s>>>(X, ldx, rows, cols, Y, ldy);
  return cudaGetLastError();
}


// ==================================================================== split-f32 Richardson kernels
// GB300 executes FP64 at ~1/60 of its f32 rate, so an FP64 residual GEMV is
// compute-bound.  The mixed-precision solve instead keeps A as two f32 limbs
// a1 = RN32(a), a2 = RN32(a - a1) (|a - a1 - a2| <= 2^-48 |a|) and theta as
// t1, t2 likewise, and forms each product a*theta as the exact f32 product
// a1*t1 = p + e (TwoProd through fma) plus the f32 corrections e + a1 t2 +
// a2 t1.  p is accumulated with TwoSum into an f32 pair (hi, lo), so each
// lane's partial sum carries ~48 significant bits; lane sums are combined in
// FP64.  The result matches an FP64 GEMV to within a few units of 2^-48
// relative to sum |a||theta| -- the same order as FP64's own accumulation error
// at these sizes.
namespace {

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p) {
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err;
}

// Fused preparation pass over A (FP64): partial sums of a^2 and of |a| per
// row block, the bf16 hi/lo operands of the tensor-core products, and the two
// f32 limbs used by the residual.
__global__ void __launch_bounds__(256) k_prep_a(const double* __restrict__ A, int64_t lda, int n,
                                                bf16* __restrict__ hi, bf16* __restrict__ lo, float* __restrict__ a1,
                                                float* __restrict__ a2, int64_t ld, double* __restrict__ ss_part,
                                                double* __restrict__ rm_part) {
  __shared__ double ss[8], ra[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  double s = 0.0, a = 0.0;
  if (row < n) {
    const double* p = A + static_cast<int64_t>(row) * lda;
    const int64_t o = static_cast<int64_t>(row) * ld;
    int kbeg = 0;
    // 16-byte vector path: four double pairs per lane in flight (needs even
    // lda and ld and a 16-byte aligned A)
    if ((lda & 1) == 0 && (ld & 1) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
      const int n2 = n & ~1;
      for (int k0 = 2 * lane; k0 < n2; k0 += 256) {
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 64 * u;
          v[u] = k < n2 ? __ldcs(reinterpret_cast<const double2*>(p + k)) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 64 * u;
          if (k >= n2) continue;
          const double e[2] = {v[u].x, v[u].y};
          float f1[2], f2[2];
          bf16 h[2], l[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            s += e[t] * e[t];
            a += fabs(e[t]);
            split_f64_f32(e[t], f1[t], f2[t]);
            h[t] = __float2bfloat16_rn(f1[t]);
            l[t] = __float2bfloat16_rn(f1[t] - __bfloat162float(h[t]));
          }
          *reinterpret_cast<float2*>(a1 + o + k) = make_float2(f1[0], f1[1]);
          *reinterpret_cast<float2*>(a2 + o + k) = make_float2(f2[0], f2[1]);
          __nv_bfloat162 hh, ll;
          hh.x = h[0];
          hh.y = h[1];
          ll.x = l[0];
          ll.y = l[1];
          *reinterpret_cast<__nv_bfloat162*>(hi + o + k) = hh;
          *reinterpret_cast<__nv_bfloat162*>(lo + o + k) = ll;
        }
      }
      kbeg = n2;
    }
    for (int k = kbeg + lane; k < n; k += 32) {
      const double v = p[k];
      s += v * v;
      a += fabs(v);
      float f1, f2;
      split_f64_f32(v, f1, f2);
      a1[o + k] = f1;
      a2[o + k] = f2;
      const bf16 h = __float2bfloat16_rn(f1);
      hi[o + k] = h;
      lo[o + k] = __float2bfloat16_rn(f1 - __bfloat162float(h));
    }
  }
  s = warp_sum(s);
  a = warp_sum(a);
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
    ss_part[blockIdx.x] = ts;
    rm_part[blockIdx.x] = tm;
  }
}

// theta (n x nrhs, FP64, row-major) -> limbs T1[c][k], T2[c][k] (ldt per rhs).
__global__ void k_split_theta(const double* __restrict__ Th, int n, int nrhs, float* __restrict__ T1,
                              float* __restrict__ T2, int64_t ldt) {
  const int64_t total = static_cast<int64_t>(n) * nrhs;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t k = e / nrhs, c = e % nrhs;
    const double v = Th[e];
    const float f1 = static_cast<float>(v);
    T1[c * ldt + k] = f1;
    T2[c * ldt + k] = static_cast<float>(v - static_cast<double>(f1));
  }
}

// A32 += B32 on n x n (leading dimension ld) and the bf16 hi/lo split of the
// sum (the elementwise sum of two powers inside the nested order-45 chain).
__global__ void k_add_split(float* __restrict__ a32, const float* __restrict__ b32, bf16* __restrict__ hi,
                            bf16* __restrict__ lo, int n, int64_t ld) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = (e / n) * ld + e % n;
    const float v = a32[o] + b32[o];
    a32[o] = v;
    const bf16 h = __float2bfloat16_rn(v);
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

__global__ void k_add_f64(double* __restrict__ a, const double* __restrict__ b, int n, int64_t ld) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = (e / n) * ld + e % n;
    a[o] += b[o];
  }
}

// D = a + cb b + cd I over n x n (leading dimension ld; b may be null): the
// matrix sums of the recursive omega_k schedule (Section 6.2: omega_k - SG_k,
// and I + Gamma), f32 master with its bf16 hi / lo split, and in FP64.
__global__ void k_lin_split(float* __restrict__ d32, bf16* __restrict__ hi, bf16* __restrict__ lo,
                            const float* __restrict__ a32, const float* __restrict__ b32, float cb, float cd, int n,
                            int64_t ld) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const int64_t o = i * ld + j;
    float v = a32[o];
    if (b32 != nullptr) v = fmaf(cb, b32[o], v);
    if (i == j) v += cd;
    d32[o] = v;
    const bf16 h = __float2bfloat16_rn(v);
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

__global__ void k_lin_f64(double* __restrict__ d, const double* __restrict__ a, const double* __restrict__ b,
                          double cb, double cd, int n, int64_t ld) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const int64_t o = i * ld + j;
    double v = a[o];
    if (b != nullptr) v = fma(cb, b[o], v);
    if (i == j) v += cd;
    d[o] = v;
  }
}

// Theta += U (n x nrhs, row-major FP64); with T1 non-null also the f32 limbs
// of the new theta (T1/T2[c][k], leading dimension ldt).
__global__ void k_axpy_theta(double* __restrict__ Th, const double* __restrict__ U, int n, int nrhs,
                             float* __restrict__ T1, float* __restrict__ T2, int64_t ldt) {
  const int64_t total = static_cast<int64_t>(n) * nrhs;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = Th[e] + U[e];
    Th[e] = v;
    if (T1 != nullptr) {
      const int64_t k = e / nrhs, c = e % nrhs;
      float f1, f2;
      split_f64_f32(v, f1, f2);
      T1[c * ldt + k] = f1;
      T2[c * ldt + k] = f2;
    }
  }
}

// Lane reduction of a paired-f32 value (hi, lo) across the warp with TwoSum at
// every step, so the ~48-bit partial sums stay ~48-bit (FP64 instructions are
// rate-limited on this GPU; this uses the f32 pipes and shuffles only).
__device__ __forceinline__ void warp_sum_x2(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = hi + oh;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (oh - bb);
    const float l = lo + ol + err;
    hi = s + l;  // renormalise (FastTwoSum; |s| >= |l|)
    lo = l - (hi - s);
  }
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Residual and update kernels: a block of 256 threads covers 8 rows; warp w
// takes the row pair (w & 3) and the half (w >> 2) of the k range (128-column
// steps interleaved), so 4096 warps are in flight at n = 4096.  The two halves
// meet in shared memory.
constexpr int kXRows = 8;

// R = B - A Theta from the f32 limbs; also R32T[c][row] = RN32(R) (the
// operand of the update) and per-block partial sums of R^2.  ld % 4 == 0.
template <int NR>
__global__ void __launch_bounds__(256, 3) k_resid_x2(const float* __restrict__ A1, const float* __restrict__ A2,
                                                     int64_t ld, const float* __restrict__ T1,
                                                     const float* __restrict__ T2, int64_t ldt,
                                                     const double* __restrict__ B, double* __restrict__ R,
                                                     float* __restrict__ R32T, int n, int nrhs, int c0,
                                                     double* __restrict__ partials) {
  __shared__ float red_hi[4][2][NR][2], red_lo[4][2][NR][2];
  __shared__ double sq[kXRows][NR];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp & 3, half = warp >> 2;
  const int row0 = blockIdx.x * kXRows + pair * 2;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const int64_t o0 = static_cast<int64_t>(r0 ? row0 : 0) * ld;
  const int64_t o1 = static_cast<int64_t>(r1 ? row0 + 1 : 0) * ld;
  float hi[2][NR], lo[2][NR];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) hi[r][c] = lo[r][c] = 0.f;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int kfirst = 4 * lane + 128 * half;
  float4 nx0 = z4, ny0 = z4, nx1 = z4, ny1 = z4;
  if (kfirst < n4) {
    if (r0) {
      nx0 = __ldcs(reinterpret_cast<const float4*>(A1 + o0 + kfirst));
      ny0 = __ldcs(reinterpret_cast<const float4*>(A2 + o0 + kfirst));
    }
    if (r1) {
      nx1 = __ldcs(reinterpret_cast<const float4*>(A1 + o1 + kfirst));
      ny1 = __ldcs(reinterpret_cast<const float4*>(A2 + o1 + kfirst));
    }
  }
#pragma unroll 1
  for (int k = kfirst; k < n4; k += 256) {
    const float4 x0 = nx0, y0 = ny0, x1 = nx1, y1 = ny1;
    const int kn = k + 256;
    if (kn < n4) {
      if (r0) {
        nx0 = __ldcs(reinterpret_cast<const float4*>(A1 + o0 + kn));
        ny0 = __ldcs(reinterpret_cast<const float4*>(A2 + o0 + kn));
      }
      if (r1) {
        nx1 = __ldcs(reinterpret_cast<const float4*>(A1 + o1 + kn));
        ny1 = __ldcs(reinterpret_cast<const float4*>(A2 + o1 + kn));
      }
    }
    const float a1v[2][4] = {{x0.x, x0.y, x0.z, x0.w}, {x1.x, x1.y, x1.z, x1.w}};
    const float a2v[2][4] = {{y0.x, y0.y, y0.z, y0.w}, {y1.x, y1.y, y1.z, y1.w}};
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const float4 u = *reinterpret_cast<const float4*>(T1 + (c0 + c) * ldt + k);
      const float4 w = *reinterpret_cast<const float4*>(T2 + (c0 + c) * ldt + k);
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
        const float x = ok ? A1[o + k] : 0.f, y = ok ? A2[o + k] : 0.f;
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          const float t1 = T1[(c0 + c) * ldt + k], t2 = T2[(c0 + c) * ldt + k];
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
  // one thread per (row, rhs) of the block combines the two halves in FP64
  if (threadIdx.x < kXRows * NR) {
    const int rr = threadIdx.x / NR, c = threadIdx.x % NR;
    const int pr = rr >> 1, r = rr & 1;
    const int row = blockIdx.x * kXRows + rr;
    double v2 = 0.0;
    if (row < n) {
      const double sdot = (static_cast<double>(red_hi[pr][0][c][r]) + static_cast<double>(red_lo[pr][0][c][r])) +
                          (static_cast<double>(red_hi[pr][1][c][r]) + static_cast<double>(red_lo[pr][1][c][r]));
      const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
      const double v = B[o] - sdot;
      R[o] = v;
      R32T[static_cast<int64_t>(c0 + c) * ldt + row] = static_cast<float>(v);
      v2 = v * v;
    }
    sq[rr][c] = v2;
  }
  __syncthreads();
  if (threadIdx.x < NR) {
    double t = 0.0;
    for (int w = 0; w < kXRows; ++w) t += sq[w][threadIdx.x];
    partials[static_cast<int64_t>(blockIdx.x) * nrhs + c0 + threadIdx.x] = t;
  }
}

// Theta += G R with G f32 (ld % 4 == 0) and R given as f32 R32T[c][k]; the new
// theta is also written as its f32 limbs for the next residual.  Products and
// sums are f32 (G is itself an f32 approximation of the inverse, so this adds
// an error well below G's own); the new theta is formed in FP64.
template <int NR>
__global__ void __launch_bounds__(256, 4) k_update_x2(const float* __restrict__ G, int64_t ldg,
                                                      const float* __restrict__ R32T, int64_t ldt,
                                                      double* __restrict__ Th, float* __restrict__ T1,
                                                      float* __restrict__ T2, int n, int nrhs, int c0) {
  __shared__ float red[4][2][NR][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp & 3, half = warp >> 2;
  const int row0 = blockIdx.x * kXRows + pair * 2;
  const bool r0 = row0 < n, r1 = row0 + 1 < n;
  const float* g0 = G + static_cast<int64_t>(r0 ? row0 : 0) * ldg;
  const float* g1 = G + static_cast<int64_t>(r1 ? row0 + 1 : 0) * ldg;
  float acc[2][NR];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[r][c] = 0.f;
  const int n4 = n & ~3;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int kfirst = 4 * lane + 128 * half;
  float4 nx0 = z4, nx1 = z4;
  if (kfirst < n4) {
    if (r0) nx0 = __ldcs(reinterpret_cast<const float4*>(g0 + kfirst));
    if (r1) nx1 = __ldcs(reinterpret_cast<const float4*>(g1 + kfirst));
  }
#pragma unroll 1
  for (int k = kfirst; k < n4; k += 256) {
    const float4 x0 = nx0, x1 = nx1;
    const int kn = k + 256;
    if (kn < n4) {
      if (r0) nx0 = __ldcs(reinterpret_cast<const float4*>(g0 + kn));
      if (r1) nx1 = __ldcs(reinterpret_cast<const float4*>(g1 + kn));
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const float4 t = *reinterpret_cast<const float4*>(R32T + (c0 + c) * ldt + k);
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
        const float t = R32T[(c0 + c) * ldt + k];
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
  if (threadIdx.x < kXRows * NR) {
    const int rr = threadIdx.x / NR, c = threadIdx.x % NR;
    const int pr = rr >> 1, r = rr & 1;
    const int row = blockIdx.x * kXRows + rr;
    if (row < n) {
      const int64_t o = static_cast<int64_t>(row) * nrhs + c0 + c;
      const double v = Th[o] + (static_cast<double>(red[pr][0][c][r]) + static_cast<double>(red[pr][1][c][r]));
      Th[o] = v;
      const float f1 = static_cast<float>(v);
      T1[static_cast<int64_t>(c0 + c) * ldt + row] = f1;
      T2[static_cast<int64_t>(c0 + c) * ldt + row] = static_cast<float>(v - static_cast<double>(f1));
    }
  }
}

}  // namespace

cudaError_t launch_prep_a(const double* A, int64_t lda, int n, bf16* hi, bf16* lo, float* a1, float* a2, int64_t ld,
                          double* ss_part, double* rm_part, int* nblocks_out, cudaStream_t s) {
  const int nb = (n + 7) / 8;
  if (nblocks_out) *nblocks_out = nb;
  if (n <= 0) return cudaSuccess;
  k_prep_a<<<nb, 256, 0, s>>>(A, lda, n, hi, lo, a1, a2, ld, ss_part, rm_part);
  return cudaGetLastError();
}

cudaError_t launch_split_theta(const double* Th, int n, int nrhs, float* T1, float* T2, int64_t ldt, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * nrhs;
  if (total <= 0) return cudaSuccess;
  k_split_theta<<<ew_grid(total), 256, 0, s>>>(Th, n, nrhs, T1, T2, ldt);
  return cudaGetLastError();
}

cudaError_t launch_add_split(float* a32, const float* b32, bf16* hi, bf16* lo, int n, int64_t ld, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_add_split<<<ew_grid(total), 256, 0, s>>>(a32, b32, hi, lo, n, ld);
  return cudaGetLastError();
}

cudaError_t launch_lin_split(float* d32, bf16* hi, bf16* lo, const float* a32, const float* b32, float cb, float cd,
                             int n, int64_t ld, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_lin_split<<<ew_grid(total), 256, 0, s>>>(d32, hi, lo, a32, b32, cb, cd, n, ld);
  return cudaGetLastError();
}

cudaError_t launch_lin_f64(double* d, const double* a, const double* b, double cb, double cd, int n, int64_t ld,
                           cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_lin_f64<<<ew_grid(total), 256, 0, s>>>(d, a, b, cb, cd, n, ld);
  return cudaGetLastError();
}

cudaError_t launch_add_f64(double* a, const double* b, int n, int64_t ld, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * n;
  if (total <= 0) return cudaSuccess;
  k_add_f64<<<ew_grid(total), 256, 0, s>>>(a, b, n, ld);
  return cudaGetLastError();
}

cudaError_t launch_axpy_theta(double* Th, const double* U, int n, int nrhs, float* T1, float* T2, int64_t ldt,
                              cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(n) * nrhs;
  if (total <= 0) return cudaSuccess;
  k_axpy_theta<<<ew_grid(total), 256, 0, s>>>(Th, U, n, nrhs, T1, T2, ldt);
  return cudaGetLastError();
}

int resid_x2_blocks(int n) { return (n + kXRows - 1) / kXRows; }

cudaError_t launch_resid_x2(const float* A1, const float* A2, int64_t ld, const float* T1, const float* T2,
                            int64_t ldt, const double* B, double* R, float* R32T, int n, int nrhs,
                            double* partials, int* nblocks_out, cudaStream_t s) {
  const int nb = resid_x2_blocks(n);
  if (nblocks_out) *nblocks_out = nb;
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (ld % 4 || ldt % 4 || !aligned16(A1) || !aligned16(A2) || !aligned16(T1) || !aligned16(T2))
    return cudaErrorInvalidValue;
  int c0 = 0;
  while (c0 < nrhs) {
    const int left = nrhs - c0;
    const int nr = left >= 4 ? 4 : left >= 2 ? 2 : 1;
    if (nr == 4)
      k_resid_x2<4><<<nb, 256, 0, s>>>(A1, A2, ld, T1, T2, ldt, B, R, R32T, n, nrhs, c0, partials);
    else if (nr == 2)
      k_resid_x2<2><<<nb, 256, 0, s>>>(A1, A2, ld, T1, T2, ldt, B, R, R32T, n, nrhs, c0, partials);
    else
      k_resid_x2<1><<<nb, 256, 0, s>>>(A1, A2, ld, T1, T2, ldt, B, R, R32T, n, nrhs, c0, partials);
    c0 += nr;
  }
  return cudaGetLastError();
}

cudaError_t launch_update_x2(const float* G, int64_t ldg, const float* R32T, int64_t ldt, double* Th, float* T1,
                             float* T2, int n, int nrhs, cudaStream_t s) {
  const int nb = resid_x2_blocks(n);
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (ldg % 4 || ldt % 4 || !aligned16(G) || !aligned16(R32T)) return cudaErrorInvalidValue;
  int c0 = 0;
  while (c0 < nrhs) {
    const int left = nrhs - c0;
    const int nr = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    if (nr == 8)
      k_update_x2<8><<<nb, 256, 0, s>>>(G, ldg, R32T, ldt, Th, T1, T2, n, nrhs, c0);
    else if (nr == 4)
      k_update_x2<4><<<nb, 256, 0, s>>>(G, ldg, R32T, ldt, Th, T1, T2, n, nrhs, c0);
    else if (nr == 2)
      k_update_x2<2><<<nb, 256, 0, s>>>(G, ldg, R32T, ldt, Th, T1, T2, n, nrhs, c0);
    else
      k_update_x2<1><<<nb, 256, 0, s>>>(G, ldg, R32T, ldt, Th, T1, T2, n, nrhs, c0);
    c0 += nr;
  }
  return cudaGetLastError();
}


cudaError_t launch_tf32_pack(const float* X, int64_t ld, int rows, int cols, float* Y, float* YT, int64_t ldt,
                             cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_tf32_pack<<<grid, 256, 0, s>>>(X, ld, rows, cols, Y, YT, ldt);
  return cudaGetLastError();
}

}  // namespace nsgb
