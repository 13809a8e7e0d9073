// Allocation-free variant of the FP64 Richardson residual entry point.
//
// ns_k_resid needs a small scratch buffer for its per-block partial sums of
// ||R_c||^2 and takes it from the stream-ordered allocator on every call.
// Some callers cannot allocate device memory at call time: a serving loop
// whose device memory is fully reserved up front by its admission budget, a
// latency-critical loop that must not touch the allocator (cudaMalloc and
// cudaFree can synchronise the device), or a process whose policy forbids
// allocation after initialisation.  For them this file keeps the scratch in a
// fixed device array that exists for as long as the library is loaded.
#include <mutex>

#include "../../include/nsgb.h"
#include "internal.h"

namespace {

// Capacity of the fixed scratch: one double per (block of 16 rows, rhs).
constexpr int64_t kNoAllocMaxN = 32768;
constexpr int kNoAllocMaxRhs = 16;
constexpr int64_t kNoAllocSlots = ((kNoAllocMaxN + 15) / 16) * kNoAllocMaxRhs;  // 32768 doubles = 256 KiB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_resid_partials[kNoAllocSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Device address of the array on the current device.  Host code may not pass
// &g_resid_partials to a kernel (on the host that name is only a stand-in);
// the address is looked up once per device, with that device current.
ns_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_partials_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_resid_partials) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return NS_ERR_CUDA;
    }
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return NS_OK;
}

}  // namespace

extern "C" ns_status ns_k_resid_noalloc(const double* A, int64_t lda, const double* Theta, const double* B,
                                        double* R, int64_t n, int nrhs, double* rsq_out, void* stream) {
  if (!A || !Theta || !B || !R || n <= 0 || nrhs <= 0 || lda < n) return NS_ERR_ARG;
  if (n > kNoAllocMaxN || nrhs > kNoAllocMaxRhs) return NS_ERR_ARG;  // beyond the fixed scratch
  double* part = nullptr;
  const ns_status s0 = scratch_for_current_device(&part);
  if (s0 != NS_OK) return s0;
  // Every partial read by the reduction is written by this call's residual
  // kernel first, so nothing in the array needs clearing.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int nb = 0;
  cudaError_t e = nsgb::launch_resid(A, lda, Theta, B, R, static_cast<int>(n), nrhs, part, &nb, st);
  if (e == cudaSuccess && rsq_out) e = nsgb::launch_reduce_sum(part, nb, nrhs, rsq_out, st);
  return e == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}
