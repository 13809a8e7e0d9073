// Batched memory-bound kernels for many independent systems of uneven size:
// fused preparation of A, G0, the split-f32 Richardson residual and update,
// and the per-instance reductions.  One launch covers every instance: block b
// processes work item items[b] = (instance, first row, first rhs).  Each
// instance's arithmetic (row blocks, k split, reduction order) is the same as
// when it is alone in the batch, so results do not depend on the mix.
#include "batch_rows.cuh"

namespace nsgb {
namespace {

using namespace brow;

__global__ void __launch_bounds__(256) k_bprep(const BInst* __restrict__ insts, const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  bprep_body(insts[it.inst], it);
}
__global__ void __launch_bounds__(256) k_bnorms(const BInst* __restrict__ insts, const int* __restrict__ list) {
  bnorms_body(insts[list[blockIdx.x]]);
}
__global__ void __launch_bounds__(256) k_bg0(const BInst* __restrict__ insts, const BItem* __restrict__ items,
                                             int mode, int zero_theta) {
  const BItem it = items[blockIdx.x];
  bg0_body(insts[it.inst], it, mode, zero_theta);
}
__global__ void __launch_bounds__(256, 2) k_bresid(const BInst* __restrict__ insts, const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  bresid_body(insts[it.inst], it);
}
__global__ void __launch_bounds__(256) k_bresid64(const BInst* __restrict__ insts, const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  bresid64_body(insts[it.inst], it);
}
__global__ void __launch_bounds__(256) k_brsq(const BInst* __restrict__ insts, const int* __restrict__ list) {
  brsq_body(insts[list[blockIdx.x]]);
}
__global__ void __launch_bounds__(256, 3) k_bupdate(const BInst* __restrict__ insts,
                                                    const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  bupdate_body(insts[it.inst], it);
}
__global__ void __launch_bounds__(256) k_bfrob(const BInst* __restrict__ insts, const int* __restrict__ list) {
  bfrob_body(insts[list[blockIdx.x]]);
}

}  // namespace

cudaError_t launch_bprep(const BInst* insts, const BItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_bprep<<<nitems, 256, 0, s>>>(insts, items);
  return cudaGetLastError();
}
cudaError_t launch_bnorms(const BInst* insts, const int* list, int ninst, cudaStream_t s) {
  if (ninst <= 0) return cudaSuccess;
  k_bnorms<<<ninst, 256, 0, s>>>(insts, list);
  return cudaGetLastError();
}
cudaError_t launch_bg0(const BInst* insts, const BItem* items, int nitems, int mode, int zero_theta,
                       cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_bg0<<<nitems, 256, 0, s>>>(insts, items, mode, zero_theta);
  return cudaGetLastError();
}
cudaError_t launch_bresid(const BInst* insts, const BItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_bresid<<<nitems, 256, 0, s>>>(insts, items);
  return cudaGetLastError();
}
cudaError_t launch_bresid64(const BInst* insts, const BItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_bresid64<<<nitems, 256, 0, s>>>(insts, items);
  return cudaGetLastError();
}
cudaError_t launch_brsq(const BInst* insts, const int* list, int ninst, cudaStream_t s) {
  if (ninst <= 0) return cudaSuccess;
  k_brsq<<<ninst, 256, 0, s>>>(insts, list);
  return cudaGetLastError();
}
cudaError_t launch_bupdate(const BInst* insts, const BItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_bupdate<<<nitems, 256, 0, s>>>(insts, items);
  return cudaGetLastError();
}
cudaError_t launch_bfrob(const BInst* insts, const int* list, int ninst, cudaStream_t s) {
  if (ninst <= 0) return cudaSuccess;
  k_bfrob<<<ninst, 256, 0, s>>>(insts, list);
  return cudaGetLastError();
}

}  // namespace nsgb
