// Batched solves: per-instance descriptors shared by the batched kernels and
// the batch runtime.
#pragma once
#include "internal.h"

namespace nsgb {

// Scalar block of one instance: [0] ||A||_F^2, [1] ||A||_inf, [2] ||F||_F^2,
// [3] unused, [kScalR + c] ||r_c||^2, [kScalR + nrhs + c] ||b_c||^2.
constexpr int kScalR = 4;

struct BInst {
  int n, nrhs, ld, nfrob;  // nfrob: partial sums of ||F||^2 written by the product kernel
  const double* A;         // caller's A (n x n, leading dimension n)
  const double* B;         // caller's B (n x nrhs)
  double* Th;              // theta (n x nrhs), the caller's output buffer
  double* R;               // residual (n x nrhs)
  bf16* Ahi;               // ld x ld
  bf16* Alo;
  float* A1;               // n x ld
  float* A2;
  float* G32[2];           // f32 masters of the two G buffers (ld x ld)
  bf16* Ghi[2];
  bf16* Glo[2];
  float* T1;               // theta limbs, nrhs x ld
  float* T2;
  float* R32T;             // f32 residual, nrhs x ld
  double* part;            // row-block partials
  double* fpart;           // product-kernel partials of ||F||^2
  double* scal;            // scalar block
};

// Right-hand sides per block of the batched residual and update kernels.
constexpr int kBRhs = 8;

// Work item of a batched row kernel: 8 rows [row0, row0 + 8) and kBRhs
// right-hand sides [c0, c0 + kBRhs) of one instance; cur selects the G buffer.
struct BItem {
  int inst, row0, c0, cur;
};

cudaError_t launch_bprep(const BInst* insts, const BItem* items, int nitems, cudaStream_t s);
cudaError_t launch_bnorms(const BInst* insts, const int* list, int ninst, cudaStream_t s);
cudaError_t launch_bg0(const BInst* insts, const BItem* items, int nitems, int mode, int zero_theta,
                       cudaStream_t s);
cudaError_t launch_bresid(const BInst* insts, const BItem* items, int nitems, cudaStream_t s);
cudaError_t launch_bresid64(const BInst* insts, const BItem* items, int nitems, cudaStream_t s);
cudaError_t launch_brsq(const BInst* insts, const int* list, int ninst, cudaStream_t s);
cudaError_t launch_bupdate(const BInst* insts, const BItem* items, int nitems, cudaStream_t s);
cudaError_t launch_bfrob(const BInst* insts, const int* list, int ninst, cudaStream_t s);

// ---- fused small-system solve (batch_fused.cu): one CTA runs the whole solve
// of one system of n <= kFusedMaxN (preparation, G0, every Newton-Schulz step
// on the tensor cores, Richardson sweeps, the precision controller) and then
// takes the next system of `list` (an atomic counter, largest systems first).
constexpr int kFusedMaxN = 256;

// Outcome of one system (the fields of the host controller's record).
struct FusedOut {
  int status, done, sweeps, rollbacks, converged, passes;
  int prods1, prods3;  // products run in bf16 (one pass) and in bf16x3
  double rel_res;
  long long cycles;    // SM clock cycles the CTA spent on this system
  int sm, pad;         // the SM that solved it
};

struct FusedParams {
  const TcProblem* prob;  // problem table (ntypes x 2 G buffers x 2 precisions per slot)
  const BInst* inst;
  const int* list;        // slots to solve, in the order they are taken
  int count;
  int* next;              // work counter (zero on entry)
  FusedOut* out;          // per slot
  int ntypes, levels;
  int precision;          // NS_AUTO, NS_BF16 or NS_BF16X3
  int g0_mode, ns_stop, max_sweeps, max_pre, iters;
  double ns_stop_frob, couple_frob, tol;
  unsigned long long timeout_ns;
  int* err;
};
cudaError_t launch_fused_solve(const FusedParams& p, int num_sms, cudaStream_t s);

}  // namespace nsgb
