// Internal interfaces between the solver runtime and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace nsgb {

using bf16 = __nv_bfloat16;

// Device error word values written by kernels whose bounded waits ran out.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1 };

constexpr int kTcMaxProblems = 4;

// One GEMM of a grouped tcgen05 launch:
//   D = s * (sum over passes of L_a R_b) + beta * C + gamma * I
// L is M x K and R is K x N, both row-major bf16 reached through 2-D tensor
// maps (box 64 x 64, 128-byte swizzle).  Index 0 of L/R is the hi part of the
// split, index 1 the lo part.  Outputs (each optional): the f32 master D32,
// the bf16 split Dhi/Dlo, and per-(tile, epilogue warp) partial sums of D^2.
struct TcProblem {
  CUtensorMap L[3];  // split parts hi, lo, lo2 (lo2: split-bf16 x6 products only)
  CUtensorMap R[3];
  int M, N, K;
  int tiles_m;     // ceil(M / 128)
  int tiles_n;     // ceil(N / BN)
  int tile_begin;  // first global work item of this problem (a work item is
                   // one tile, or for CTA pairs two vertically adjacent tiles)
  int tile_count;  // work items of this problem
  
  float s, beta, gamma;
  int ldc, ldd32, ldd16;
  const float* C;
  float* D32;
  bf16* Dhi;
  bf16* Dlo;
  bf16* Dlo2;  // third split part of D (x6 products), may be null
  float* Dt;   // TF32 forms of D (RN to 10 stored bits, ties away): row-major
  float* DtT;  // and transposed (the K-major R operand of a TF32 product); may be null
  int ldt;
  double* frob_partials;  // 4 values per tile (tiles_m * tiles_n * 4); the CTA-pair
                          // kernel writes 8 (two half-width slots of 4)
};

// A work item of a list-driven launch: problem index and tile coordinates.
struct TcItem {
  int prob, mt, nt, pad;
};

struct TcParams {
  TcProblem prob[kTcMaxProblems];
  int nprob;
  int total_tiles;  // work items over all problems
  // List-driven mode (batched / served solves): when gprob is non-null, the
  // problems live in device memory (64-byte aligned, tensor maps included) and
  // work item w is items[w]; prob[] and nprob are unused (one-CTA kernel only).
  const TcProblem* gprob;
  const TcItem* items;
  int npass;  // 1: hi*hi (bf16); 3: hi*hi + hi*lo + lo*hi (bf16x3); 6: those and
              // hi*lo2 + lo*lo + lo2*hi (bf16x6), one pass per term
  int debug_stall_iter;  // -1 for none; else the producer withholds that load
  int pair_tail;  // CTA-pair kernel: the last pair_tail tiles each run as two
                  // half-width (256 x 128) items (set by its launcher)
  unsigned long long timeout_ns;
  int* err;
};

// TF32 forms of an f32 matrix (rows x cols, ld): Y = RN_tf32(X) row-major and
// YT = RN_tf32(X)^T (cols x rows, leading dimension ldt); either may be null.
cudaError_t launch_tf32_pack(const float* X, int64_t ld, int rows, int cols, float* Y, float* YT, int64_t ldt,
                             cudaStream_t s);
// Encode a 2-D f32 tensor map (rows x cols, leading dimension ld elements):
// 32-column (128-byte) x 64-row box, 128-byte swizzle (TF32 operands, K-major).
bool encode_f32_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld);

// Launch a grouped tcgen05 GEMM, one CTA per 128 x BN tile: BN in {64, 128,
// 192, 256} output columns per tile.  x3 selects the split-product kernel (L/R
// maps of roles 1/2 below; BN 64, 128 or 256; p.npass ignored); otherwise
// p.npass passes over role-0 maps.
cudaError_t launch_gemm_tc(const TcParams& p, int BN, bool x3, int num_sms, cudaStream_t s);
// CTA-pair variant (cta_group::2): 256 x 256 output tiles, clusters of two
// (parts 4: one TF32 pass, L[0] the row-major TF32 form of L and R[0] the
// transposed TF32 form of R, both encode_f32_map maps)
// CTAs along M, tile bookkeeping of BN = 256, CM = 2 (tc_items(M, N, 256, 2)
// tiles, 8 partial sums per tc_tiles(M, N, 256) tile).  Single-problem-table
// mode only (p.gprob == nullptr).  parts: 1 one bf16 pass (p.npass == 1);
// 2 the bf16x3 terms of L[0..1], R[0..1] (role 1 / 2 maps); 3 the bf16x6 terms
// of L[0..2], R[0..2], D written with its third part (Dlo2).  Tiles of a last,
// partial wave run as two half-width items each when that shortens the wave.
cudaError_t launch_gemm_tc_pair(const TcParams& p, int parts, int num_sms, cudaStream_t s);
int tc_tiles(int M, int N, int BN);

// ---- FP64-accurate products from signed-digit bf16 slices (gemm_oz.cu)
constexpr int kOzMaxSlices = 7;      // 7 digits of 8 bits cover binary64
constexpr int64_t kOzMaxK = 16384;   // K per level-kernel launch: |S_d| < 2^31
// The level kernel's launch: every level d of every 256 x 256 pair tile of
// D = L R (M x N, K <= kOzMaxK) as one work item; writes the level sums S_d
// (int32) to planes + (d - 2) plane_stride (leading dimension ldp).
struct OzParams {
  CUtensorMap L[kOzMaxSlices];  // slices of L: M x K bf16 (role 0 maps, 64 x 64 boxes)
  CUtensorMap R[kOzMaxSlices];  // slices of R: K x N bf16
  int M, N, K;
  int slices;
  int tiles_m2;     // ceil(M / 256)
  int tiles_n;      // ceil(N / 256)
  int nlev;         // levels in this launch, in work-item order
  int lev_d[kOzMaxSlices];    // level d = t + u
  int lev_kcb[kOzMaxSlices];  // 64-deep K blocks per exactly summed chunk of that level
  int total_items;  // nlev * tiles_m2 * tiles_n
  int32_t* planes;
  int64_t ldp, plane_stride;
  int debug_stall_iter;
  unsigned long long timeout_ns;
  int* err;
};
// One slice product D = s L R + beta C + gamma I (FP64 row-major, device),
// with its workspace (oz_workspace_bytes) at `work`.
struct OzArgs {
  const double* L;
  int64_t ldl;
  const double* R;
  int64_t ldr;
  int M, N, K, slices;
  double s;
  const double* C;
  int64_t ldc;
  double beta, gamma;
  double* D;
  int64_t ldd;
  double* frob_out;  // device double receiving sum(D^2), or null
  void* work;
  int debug_stall_iter;
  unsigned long long timeout_ns;
  int* err;
};
size_t oz_workspace_bytes(int64_t M, int64_t N, int64_t K, int slices);
cudaError_t launch_oz_product(const OzArgs& g, int num_sms, cudaStream_t st);
int tc_items(int M, int N, int BN, int CM);

// Encode a 2-D bf16 tensor map (rows x cols, leading dimension ld elements).
// role 0: 64x64 box, 128 B swizzle; role 1: 32(K)x64 box, 64 B swizzle (L of
// split products); role 2: 64x32(K) box, 128 B swizzle (R of split products).
bool encode_bf16_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int role = 0);

// ---- FP64 CUDA-core GEMM with the same epilogue (plain FP64 path)
struct F64Gemm {
  int M, N, K;
  const double* L; int ldl;
  const double* R; int ldr;
  double s, beta, gamma;
  const double* C; int ldc;
  double* D; int ldd;
  double* frob_partials;  // one per 64x64 tile (row-major tile order), may be null
};
cudaError_t launch_gemm_f64(const F64Gemm& g, cudaStream_t s);
int f64_tiles(int M, int N);

// ---- HBM-bound FP64 kernels
// R = B - A Theta; per-block partial sums of R^2 per column (nblocks x nrhs).
cudaError_t launch_resid(const double* A, int64_t lda, const double* Theta, const double* B, double* R,
                         int n, int nrhs, double* partials, int* nblocks_out, cudaStream_t s);
int resid_blocks(int n);
// Theta += G R with G float (ldg) or double.
cudaError_t launch_update_f32(const float* G, int64_t ldg, const double* R, double* Theta, int n, int nrhs,
                              cudaStream_t s);
cudaError_t launch_update_f64(const double* G, int64_t ldg, const double* R, double* Theta, int n, int nrhs,
                              cudaStream_t s);
// Column sums of squares of a rows x cols row-major matrix -> partials (nblocks x cols).
cudaError_t launch_colsumsq(const double* X, int64_t ldx, int rows, int cols, double* partials,
                            int* nblocks_out, cudaStream_t s);
// Sum of squares and max row |.|-sum of an n x n FP64 matrix -> partials.
cudaError_t launch_matnorms(const double* A, int64_t lda, int n, double* ss_partials, double* rowmax_partials,
                            int* nblocks_out, cudaStream_t s);
// out[c] = sum_b partials[b * ncols + c] (fixed order) for c < ncols.
cudaError_t launch_reduce_sum(const double* partials, int nblocks, int ncols, double* out, cudaStream_t s);
cudaError_t launch_reduce_max(const double* partials, int nblocks, double* out, cudaStream_t s);
// Split an FP64 or FP32 rows x cols matrix into bf16 hi/lo (ld elements) and,
// optionally, its f32 rounding.
// (lo2, when given: the third part bf16(v - hi - lo) of bf16x6 operands)
cudaError_t launch_split_f64(const double* X, int64_t ldx, int rows, int cols, bf16* hi, bf16* lo, float* x32,
                             int64_t ld, cudaStream_t s, bf16* lo2 = nullptr);
cudaError_t launch_split_f32(const float* X, int64_t ldx, int rows, int cols, bf16* hi, bf16* lo, int64_t ld,
                             cudaStream_t s, bf16* lo2 = nullptr);
// G = alpha I where alpha is read on the device: mode 0 -> 1/sqrt(scal[0])
// (Frobenius), mode 1 -> 1/(scal[1]/2 + 1e-8 scal[1]) (infinity norm).
cudaError_t launch_init_g0_mp(const double* scal, int mode, int n, int64_t ld, float* G32, bf16* hi, bf16* lo,
                              cudaStream_t s);
cudaError_t launch_init_g0_f64(const double* scal, int mode, int n, int64_t ld, double* G, cudaStream_t s);
cudaError_t launch_init_g0_jacobi(const double* A, int64_t lda, int n, int64_t ld, float* G32, bf16* hi, bf16* lo,
                                  double* G64, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float* X, int64_t ldx, int rows, int cols, double* Y, int64_t ldy,
                              cudaStream_t s);
cudaError_t launch_copy_f64(const double* X, int64_t ldx, int rows, int cols, double* Y, int64_t ldy,
                            cudaStream_t s);
// Rademacher probes (rows x probes, ld = probes) from SplitMix64 outputs j rows + i.
cudaError_t launch_rademacher(double* Z, int rows, int probes, unsigned long long seed, cudaStream_t s);

// ---- split-f32 Richardson path (mixed precision)
// One pass over A: sum a^2 / max row |a| partials, bf16 hi/lo, f32 limbs a1/a2.
cudaError_t launch_prep_a(const double* A, int64_t lda, int n, bf16* hi, bf16* lo, float* a1, float* a2, int64_t ld,
                          double* ss_part, double* rm_part, int* nblocks_out, cudaStream_t s);
// theta (n x nrhs) -> f32 limbs T1/T2 stored per right-hand side (leading dimension ldt).
cudaError_t launch_split_theta(const double* Th, int n, int nrhs, float* T1, float* T2, int64_t ldt, cudaStream_t s);
cudaError_t launch_axpy_theta(double* Th, const double* U, int n, int nrhs, float* T1, float* T2, int64_t ldt,
                              cudaStream_t s);
cudaError_t launch_add_split(float* a32, const float* b32, bf16* hi, bf16* lo, int n, int64_t ld, cudaStream_t s);
cudaError_t launch_add_f64(double* a, const double* b, int n, int64_t ld, cudaStream_t s);
// D = a + cb b + cd I (b may be null); the split form also writes D's bf16 hi / lo
cudaError_t launch_lin_split(float* d32, bf16* hi, bf16* lo, const float* a32, const float* b32, float cb, float cd,
                             int n, int64_t ld, cudaStream_t s);
cudaError_t launch_lin_f64(double* d, const double* a, const double* b, double cb, double cd, int n, int64_t ld,
                           cudaStream_t s);
// R = B - A theta from the limbs; R (FP64, n x nrhs), R32T (f32, per rhs), partial R^2
// (resid_x2_blocks(n) blocks x nrhs partials).
int resid_x2_blocks(int n);
cudaError_t launch_resid_x2(const float* A1, const float* A2, int64_t ld, const float* T1, const float* T2,
                            int64_t ldt, const double* B, double* R, float* R32T, int n, int nrhs,
                            double* partials, int* nblocks_out, cudaStream_t s);
// Theta += G R32 (G f32), writing the new theta's limbs.
cudaError_t launch_update_x2(const float* G, int64_t ldg, const float* R32T, int64_t ldt, double* Th, float* T1,
                             float* T2, int n, int nrhs, cudaStream_t s);

}  // namespace nsgb
