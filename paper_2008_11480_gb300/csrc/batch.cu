// Many independent SPD systems of uneven size advanced together: the batched
// solve (a fixed set of systems) and the continuous-batching server (systems
// arrive and leave).  Every system runs the method of ns_richardson_solve --
// factorized product chain of order 2^m or 3, bf16 / split-bf16 products with
// its own precision controller, split-f32 Richardson -- but one controller
// pass advances all of them with a handful of launches: one list-driven
// tcgen05 launch per product level (per tile width and precision group) and
// one launch per batched row kernel.
//
// Systems live in slots.  A slot's workspace is carved from one device arena
// (first fit, zeroed on admission); its tcgen05 problem descriptors (every
// product type x current G buffer x precision) and its row-kernel descriptor
// sit at the slot's index in device tables, so admitting or retiring a system
// touches only its own slot.
//
// Invariance: a system's tile width depends only on its own size and all of
// its reductions run in a fixed order inside its own blocks, so its result is
// bitwise the same whether it is solved alone or together with any others.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <array>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/nsgb.h"
#include "arena.h"
#include "batch.h"

using namespace nsgb;

namespace {

size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }

struct BMat {
  float* m32 = nullptr;
  bf16* hi = nullptr;
  bf16* lo = nullptr;
  CUtensorMap map_hi, map_lo, l3_hi, l3_lo, r3_hi, r3_lo;
};

struct InstState {
  int prec = NS_BF16;
  int cur = 0;
  int done = 0;
  bool ns_active = true;
  bool finished = false;
  bool converged = false;
  bool recompute = false;
  int sweeps_left = 0;
  double prev_frob = INFINITY, prev_ratio = INFINITY, frob_now = INFINITY;
  double best_rr = INFINITY;        // smallest residual of the Richardson-only phase
  double last_rr_sweep = INFINITY;  // residual of the previous Richardson-only pass
  int stall = 0;                    // consecutive Richardson-only passes with < 5 % progress
  double prev_sweep_ratio = INFINITY;  // previous contraction ratio of the Richardson-only phase
  double proj_need = 0.0;  // sweeps still needed after the last measured residual (projection)
  int k_meas = 1;          // sweeps applied between the previous measured residual and this one
  bool resid64 = false;    // residual escalated to FP64 (the split-f32 one stalled above tol)
  int status = NS_OK;
  int sweeps = 0;
  int rollbacks = 0;
  double rel_res = INFINITY;
  bool has_res = false;   // this pass formed the residual (the Richardson branch ran)
  bool coupled = false;   // delayed coupling has started (opt.couple_frob > 0)
  bool need_res = false;  // coupling starts with this pass's G_k: form its residual
  int iters = 0;      // cap on Newton-Schulz steps
  double tol = 0.0;   // relative residual target
};

// Matrices of one system, in the order the problem table uses.
enum { MA = 0, MG0, MG1, MX0, MX1, MF, MP0, MP1, kNumMats };

// Layout of one slot's workspace (offsets from the slot's arena region).
struct SlotLayout {
  size_t mat[kNumMats][3];  // f32 master (or SIZE_MAX), hi, lo
  size_t a1, a2, t1, t2, r32t, r, part, fpart, acopy, bcopy, tcopy;
  size_t bytes;
};

// ---- tile width of a system's list-driven products, by a measured choice
// Systems of n <= 256 keep 128-column tiles: the fused small-system kernel
// runs them on 128 x 128 tiles, and the pass-by-pass path must form ||F||^2
// from the same tiles for the two paths to agree bit for bit.  Above that the
// width (128 or 256 columns; the K order of every output, hence the product,
// does not depend on it) is measured once per process and size bucket: a
// grouped launch of copies of one product of the bucket's largest size on
// each candidate, the faster kept.  It depends on n alone, so a system gets
// the same width alone and in any mix.
std::mutex g_tune_mu;
int g_tune[6] = {0, 0, 0, 0, 0, 0};  // buckets n <= 512, 1024, 2048, 4096, 8192, 16384
int g_tune_n[6] = {512, 1024, 2048, 4096, 8192, 16384};

int tune_bucket(int n) {
  for (int b = 0; b < 6; ++b)
    if (n <= g_tune_n[b]) return b;
  return 5;
}

double time_width(int n, int bn, const CUtensorMap& mL, const CUtensorMap& mR, float* D32, bf16* Dhi, bf16* Dlo,
                  int* err, int sms, cudaStream_t st) {
  TcParams p;
  memset(&p, 0, sizeof(p));
  const int tiles = tc_tiles(n, n, bn);
  const int copies = std::max(1, std::min(kTcMaxProblems, (2 * sms + tiles - 1) / tiles));
  int tile = 0;
  for (int i = 0; i < copies; ++i) {
    TcProblem& P = p.prob[i];
    P.L[0] = P.L[1] = mL;
    P.R[0] = P.R[1] = mR;
    P.M = P.N = P.K = n;
    P.tiles_m = (n + 127) / 128;
    P.tiles_n = (n + bn - 1) / bn;
    P.tile_begin = tile;
    P.tile_count = tiles;
    tile += tiles;
    P.s = -1.f;
    P.gamma = 1.f;
    P.ldc = P.ldd32 = P.ldd16 = static_cast<int>(rup(n, 64));
    P.D32 = D32;  // every copy writes the same values
    P.Dhi = Dhi;
    P.Dlo = Dlo;
  }
  p.nprob = copies;
  p.total_tiles = tile;
  p.npass = 1;
  p.debug_stall_iter = -1;
  p.timeout_ns = 2000000000ull;
  p.err = err;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    const cudaError_t e = launch_gemm_tc(p, bn, false, sms, st);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      best = 1e30;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, static_cast<double>(ms) / copies);  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  return best;
}

int tune_width(int b, int sms) {
  const int n = g_tune_n[b];
  const size_t ld = rup(n, 64), cnt = ld * ld;
  char* w = nullptr;
  const size_t bytes = cnt * (2 * 2 + 4 + 2 * 2) + 256;
  if (cudaMalloc(&w, bytes) != cudaSuccess) {
    cudaGetLastError();
    return n <= 512 ? 128 : 256;  // no room to measure: the width measured on the development box
  }
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaMemsetAsync(w, 0, bytes, st);
  bf16* L = reinterpret_cast<bf16*>(w);
  bf16* R = L + cnt;
  float* D32 = reinterpret_cast<float*>(R + cnt);
  bf16* Dhi = reinterpret_cast<bf16*>(D32 + cnt);
  bf16* Dlo = Dhi + cnt;
  int* err = reinterpret_cast<int*>(Dlo + cnt);
  CUtensorMap mL, mR;
  int pick = n <= 512 ? 128 : 256;
  if (encode_bf16_map(&mL, L, ld, ld, ld, 0) && encode_bf16_map(&mR, R, ld, ld, ld, 0)) {
    const double t128 = time_width(n, 128, mL, mR, D32, Dhi, Dlo, err, sms, st);
    const double t256 = time_width(n, 256, mL, mR, D32, Dhi, Dlo, err, sms, st);
    if (t128 < 1e30 && t256 < 1e30) pick = t128 <= t256 ? 128 : 256;
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  cudaFree(w);
  cudaGetLastError();
  return pick;
}

int tile_width(int n, int sms) {
  if (n <= kFusedMaxN) return 128;
  const int b = tune_bucket(n);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune[b] == 0) g_tune[b] = tune_width(b, sms);
  return g_tune[b];
}

SlotLayout slot_layout(int n, int nrhs, bool copies) {
  SlotLayout L;
  size_t total = 0;
  auto take = [&](size_t bytes) {
    const size_t off = rup(total, 256);
    total = off + bytes;
    return off;
  };
  const size_t ld = rup(n, 64);
  const size_t sq = ld * ld;
  for (int m = 0; m < kNumMats; ++m) {
    const bool with32 = m == MG0 || m == MG1 || m == MX0 || m == MX1 || m == MF;
    L.mat[m][0] = with32 ? take(sq * 4) : SIZE_MAX;
    L.mat[m][1] = take(sq * 2);
    L.mat[m][2] = take(sq * 2);
  }
  const size_t nrb = (n + 7) / 8;
  // partial sums of ||F||^2 for the narrowest tile width a system can get (128)
  const size_t tiles = static_cast<size_t>((n + 127) / 128) * ((n + 127) / 128);
  L.a1 = take(n * ld * 4);
  L.a2 = take(n * ld * 4);
  L.t1 = take(nrhs * ld * 4);
  L.t2 = take(nrhs * ld * 4);
  L.r32t = take(nrhs * ld * 4);
  L.r = take(static_cast<size_t>(n) * nrhs * 8);
  L.part = take(std::max(2 * nrb, nrb * nrhs) * 8);
  L.fpart = take(tiles * 4 * 8);
  L.acopy = copies ? take(static_cast<size_t>(n) * n * 8) : SIZE_MAX;
  L.bcopy = copies ? take(static_cast<size_t>(n) * nrhs * 8) : SIZE_MAX;
  L.tcopy = copies ? take(static_cast<size_t>(n) * nrhs * 8) : SIZE_MAX;
  L.bytes = rup(total, 256);
  return L;
}

}  // namespace

struct ns_batch {
  // slice hand-over workers: per worker a stream and its single-system contexts (by n)
  std::vector<std::map<int, ns_ctx*>> retry;
  std::vector<cudaStream_t> retry_streams;
  int cap = 0;  // slots
  int order = 4, levels = 2, ntypes = 0;
  int max_nrhs = 1, scal_stride = 0;
  ns_options opt;
  cudaStream_t stream = nullptr;   // row kernels (residual, update, preparation) and copies
  cudaStream_t pstream = nullptr;  // tensor-core products (owned); joins `stream` once per pass
  cudaEvent_t ev_r = nullptr, ev_p = nullptr;
  int device = 0, num_sms = 148;
  std::string err;
  void* dmem = nullptr;
  char* abase = nullptr;
  size_t asize = 0;
  nsgb::Arena arena;
  TcProblem* dprob = nullptr;
  BInst* dinst = nullptr;
  double* dscal = nullptr;
  int* derr = nullptr;
  char* dstage = nullptr;
  char* hstage = nullptr;
  size_t stage_cap = 0, stage_used = 0;
  double* hscal = nullptr;
  std::vector<char> used;
  std::vector<size_t> reg_off;
  std::vector<SlotLayout> lay;
  std::vector<int> n, nrhs, ld, bn, tiles_m, tiles_n;
  std::vector<std::array<BMat, kNumMats>> mats;
  std::vector<BInst> hinst;
  std::vector<InstState> st;
  ns_batch_stats* stats = nullptr;
  double wait_ms = 0.0;  // host time blocked in the per-pass stream synchronisation
  FusedOut* dfout = nullptr;  // fused launch: per-slot outcome
  int* dnext = nullptr;       // fused launch: work counter
  int fixed_count = 0;  // systems of a fixed batch (slots 0 .. fixed_count - 1)
  int max_pre = 0;      // extra Richardson-only sweeps per pass (fixed batches: fewer syncs;
                        // the server keeps ticks short for latency)
};

namespace {

ns_status bfail(ns_batch* b, ns_status s, const std::string& m) {
  b->err = m;
  return s;
}

#define B_CK(call)                                                                                          \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess) return bfail(b, NS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define B_TRY(expr)        \
  do {                     \
    ns_status s_ = (expr); \
    if (s_ < 0) return s_; \
  } while (0)

// Copy host bytes into the device staging area (stream ordered); the host side
// is a pinned mirror at the same offsets and the bump pointer is reset only
// after a stream synchronisation, so no region is rewritten before its copy.
void* stage(ns_batch* b, const void* src, size_t bytes, cudaStream_t st) {
  const size_t off = rup(b->stage_used, 256);
  if (off + bytes > b->stage_cap - 256) return nullptr;
  memcpy(b->hstage + off, src, bytes);
  if (cudaMemcpyAsync(b->dstage + off, b->hstage + off, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return nullptr;
  b->stage_used = off + bytes;
  return b->dstage + off;
}

size_t prob_index(const ns_batch* b, int i, int type, int cur, int x3) {
  return ((static_cast<size_t>(i) * b->ntypes + type) * 2 + cur) * 2 + x3;
}

// Product types of one step: order 2^m -> 0: F = I - A G; 1 + 2j: X_{j+1} =
// X_j + X_j P_j; 2 + 2j: P_{j+1} = P_j P_j (j < m - 1).  Order 3 -> 0: F
// (with f32 master), 1: W = F + F F, 2: G' = G + G W.
TcProblem make_problem(const ns_batch* b, int i, int type, int cur, int x3) {
  const auto& M = b->mats[i];
  const BMat& Gc = M[cur ? MG1 : MG0];
  const BMat& Gn = M[cur ? MG0 : MG1];
  const BMat *L = nullptr, *R = nullptr, *D = nullptr;
  const float* C = nullptr;
  float s = 1.f, beta = 0.f, gamma = 0.f;
  bool want32 = false, frob = false;
  if (type == 0) {
    L = &M[MA];
    R = &Gc;
    D = &M[MF];
    s = -1.f;
    gamma = 1.f;
    want32 = b->levels == 0;
    frob = true;
  } else if (b->levels == 0) {
    if (type == 1) {
      L = &M[MF];
      R = &M[MF];
      C = M[MF].m32;
      beta = 1.f;
      D = &M[MP0];
    } else {
      L = &Gc;
      R = &M[MP0];
      C = Gc.m32;
      beta = 1.f;
      D = &Gn;
      want32 = true;
    }
  } else {
    const int j = (type - 1) / 2;
    const BMat& Xj = j == 0 ? Gc : M[(j - 1) & 1 ? MX1 : MX0];
    const BMat& Pj = j == 0 ? M[MF] : M[(j - 1) & 1 ? MP1 : MP0];
    if ((type - 1) % 2 == 0) {
      L = &Xj;
      R = &Pj;
      C = Xj.m32;
      beta = 1.f;
      D = j == b->levels - 1 ? &Gn : &M[j & 1 ? MX1 : MX0];
      want32 = true;
    } else {
      L = &Pj;
      R = &Pj;
      D = &M[j & 1 ? MP1 : MP0];
    }
  }
  TcProblem P;
  memset(&P, 0, sizeof(P));
  P.L[0] = x3 ? L->l3_hi : L->map_hi;
  P.L[1] = x3 ? L->l3_lo : L->map_lo;
  P.R[0] = x3 ? R->r3_hi : R->map_hi;
  P.R[1] = x3 ? R->r3_lo : R->map_lo;
  const int n = b->n[i];
  P.M = P.N = P.K = n;
  P.tiles_m = b->tiles_m[i];
  P.tiles_n = b->tiles_n[i];
  P.s = s;
  P.beta = beta;
  P.gamma = gamma;
  P.C = C;
  P.ldc = P.ldd32 = P.ldd16 = b->ld[i];
  P.D32 = want32 ? D->m32 : nullptr;
  P.Dhi = D->hi;
  P.Dlo = D->lo;
  P.frob_partials = frob ? b->hinst[i].fpart : nullptr;
  return P;
}

double step_cost_i(const ns_batch* b, int i, int prec) {
  const double n = b->n[i];
  const int prods = b->levels == 0 ? 3 : 2 * b->levels;
  return prods * 2.0 * n * n * n * (prec == NS_BF16X3 ? 3.0 : 1.0) / 1.0e15 + 3e-6 * prods;
}
double sweep_cost_i(const ns_batch* b, int i) {
  const double n = b->n[i];
  return std::max(12.0 * n * n / 5.0e12, 22.0 * n * n * b->nrhs[i] / 3.0e13) + 3e-5;
}

// Allocate and build a slot for (n, nrhs); -1 when no slot or memory is free.
// With `copies` the slot also holds A, B and theta (a server request); else
// the caller's buffers are attached by attach_fixed().
int add_slot(ns_batch* b, int n, int nrhs, bool copies) {
  int i = -1;
  for (int k = 0; k < b->cap; ++k)
    if (!b->used[k]) {
      i = k;
      break;
    }
  if (i < 0) return -1;
  const SlotLayout L = slot_layout(n, nrhs, copies);
  const size_t off = b->arena.alloc(L.bytes);
  if (off == SIZE_MAX) return -1;
  char* base = b->abase + off;
  if (cudaMemsetAsync(base, 0, L.bytes, b->stream) != cudaSuccess) {
    cudaGetLastError();
    b->arena.release(off, L.bytes);
    return -1;
  }
  b->used[i] = 1;
  b->reg_off[i] = off;
  b->lay[i] = L;
  b->n[i] = n;
  b->nrhs[i] = nrhs;
  b->ld[i] = static_cast<int>(rup(n, 64));
  b->bn[i] = tile_width(n, b->num_sms);
  b->tiles_m[i] = (n + 127) / 128;
  b->tiles_n[i] = (n + b->bn[i] - 1) / b->bn[i];
  const int64_t ldi = b->ld[i];
  for (int m = 0; m < kNumMats; ++m) {
    BMat& M = b->mats[i][m];
    M.m32 = L.mat[m][0] == SIZE_MAX ? nullptr : reinterpret_cast<float*>(base + L.mat[m][0]);
    M.hi = reinterpret_cast<bf16*>(base + L.mat[m][1]);
    M.lo = reinterpret_cast<bf16*>(base + L.mat[m][2]);
    encode_bf16_map(&M.map_hi, M.hi, ldi, ldi, ldi, 0);
    encode_bf16_map(&M.map_lo, M.lo, ldi, ldi, ldi, 0);
    encode_bf16_map(&M.l3_hi, M.hi, ldi, ldi, ldi, 1);
    encode_bf16_map(&M.l3_lo, M.lo, ldi, ldi, ldi, 1);
    encode_bf16_map(&M.r3_hi, M.hi, ldi, ldi, ldi, 2);
    encode_bf16_map(&M.r3_lo, M.lo, ldi, ldi, ldi, 2);
  }
  BInst& I = b->hinst[i];
  memset(&I, 0, sizeof(I));
  I.n = n;
  I.nrhs = nrhs;
  I.ld = b->ld[i];
  I.nfrob = b->tiles_m[i] * b->tiles_n[i] * 4;
  I.Ahi = b->mats[i][MA].hi;
  I.Alo = b->mats[i][MA].lo;
  I.A1 = reinterpret_cast<float*>(base + L.a1);
  I.A2 = reinterpret_cast<float*>(base + L.a2);
  I.T1 = reinterpret_cast<float*>(base + L.t1);
  I.T2 = reinterpret_cast<float*>(base + L.t2);
  I.R32T = reinterpret_cast<float*>(base + L.r32t);
  I.R = reinterpret_cast<double*>(base + L.r);
  I.part = reinterpret_cast<double*>(base + L.part);
  I.fpart = reinterpret_cast<double*>(base + L.fpart);
  I.scal = b->dscal + static_cast<size_t>(i) * b->scal_stride;
  if (copies) {
    I.A = reinterpret_cast<const double*>(base + L.acopy);
    I.B = reinterpret_cast<const double*>(base + L.bcopy);
    I.Th = reinterpret_cast<double*>(base + L.tcopy);
  }
  for (int c = 0; c < 2; ++c) {
    const BMat& G = b->mats[i][c ? MG1 : MG0];
    I.G32[c] = G.m32;
    I.Ghi[c] = G.hi;
    I.Glo[c] = G.lo;
  }
  b->st[i] = InstState();
  return i;
}

void free_slot(ns_batch* b, int i) {
  if (i < 0 || i >= b->cap || !b->used[i]) return;
  b->arena.release(b->reg_off[i], b->lay[i].bytes);
  b->used[i] = 0;
}

// Upload a slot's row-kernel descriptor and all its product descriptors.
ns_status publish_slot(ns_batch* b, int i, bool problems) {
  if (problems) {
    std::vector<TcProblem> probs(static_cast<size_t>(b->ntypes) * 4);
    for (int t = 0; t < b->ntypes; ++t)
      for (int c = 0; c < 2; ++c)
        for (int x = 0; x < 2; ++x) probs[(static_cast<size_t>(t) * 2 + c) * 2 + x] = make_problem(b, i, t, c, x);
    const void* dp = stage(b, probs.data(), probs.size() * sizeof(TcProblem), b->stream);
    if (!dp) return bfail(b, NS_ERR_OOM, "staging area exhausted");
    B_CK(cudaMemcpyAsync(b->dprob + prob_index(b, i, 0, 0, 0), dp, probs.size() * sizeof(TcProblem),
                         cudaMemcpyDeviceToDevice, b->stream));
  }
  const void* di = stage(b, &b->hinst[i], sizeof(BInst), b->stream);
  if (!di) return bfail(b, NS_ERR_OOM, "staging area exhausted");
  B_CK(cudaMemcpyAsync(b->dinst + i, di, sizeof(BInst), cudaMemcpyDeviceToDevice, b->stream));
  return NS_OK;
}

// Algorithmic HBM bytes of one product of system i (type t): its operands once
// (hi only for a bf16 pass, hi and lo for bf16x3), the C term, and the outputs
// (f32 master where kept, bf16 hi and lo) -- the flags of make_problem.
double product_bytes(const ns_batch* b, int i, int t, int x3) {
  const double e = static_cast<double>(b->n[i]) * b->n[i];
  bool c = false, d32 = false;
  if (t == 0) {
    d32 = b->levels == 0;
  } else if (b->levels == 0) {
    c = true;
    d32 = t == 2;
  } else {
    c = d32 = (t - 1) % 2 == 0;
  }
  return e * (2.0 * (x3 ? 4.0 : 2.0) + (c ? 4.0 : 0.0) + (d32 ? 4.0 : 0.0) + 4.0);
}

ns_status launch_products(ns_batch* b, const std::vector<int>& ids, const std::vector<int>& types) {
  for (int bnv : {128, 256}) {
    for (int x3 = 0; x3 < 2; ++x3) {
      std::vector<TcItem> items;
      double flops = 0.0, bytes = 0.0;
      for (int i : ids) {
        if (b->bn[i] != bnv || (b->st[i].prec == NS_BF16X3) != (x3 == 1)) continue;
        for (int t : types) {
          const int pi = static_cast<int>(prob_index(b, i, t, b->st[i].cur, x3));
          for (int mt = 0; mt < b->tiles_m[i]; ++mt)
            for (int nt = 0; nt < b->tiles_n[i]; ++nt) items.push_back(TcItem{pi, mt, nt, 0});
          flops += 2.0 * b->n[i] * static_cast<double>(b->n[i]) * b->n[i] * (x3 ? 3 : 1);
          bytes += product_bytes(b, i, t, x3);
        }
      }
      if (items.empty()) continue;
      const TcItem* ditems =
          static_cast<const TcItem*>(stage(b, items.data(), items.size() * sizeof(TcItem), b->pstream));
      if (!ditems) return bfail(b, NS_ERR_OOM, "staging area exhausted");
      TcParams p;
      memset(&p, 0, sizeof(p));
      p.gprob = b->dprob;
      p.items = ditems;
      p.total_tiles = static_cast<int>(items.size());
      p.npass = 1;
      p.debug_stall_iter = -1;
      p.timeout_ns = static_cast<unsigned long long>(b->opt.timeout_s * 1e9);
      p.err = b->derr;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (b->opt.profile) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, b->pstream);
      }
      B_CK(launch_gemm_tc(p, bnv, x3 == 1, b->num_sms, b->pstream));
      if (b->stats) {
        b->stats->gemm_launches++;
        b->stats->kernel_launches++;
        b->stats->gemm_flops += flops;
        b->stats->gemm_bytes += bytes;
      }
      if (b->opt.profile) {
        cudaEventRecord(e1, b->pstream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (b->stats) b->stats->gemm_ms += ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
      }
    }
  }
  return NS_OK;
}

std::vector<BItem> row_items(const ns_batch* b, const std::vector<int>& ids, bool with_rhs);
template <typename F>
ns_status run_rows(ns_batch* b, const std::vector<BItem>& items, F launch);

// Residuals of the systems in `ids`: split-f32 for most, FP64 for those escalated.
ns_status launch_residuals(ns_batch* b, const std::vector<int>& ids) {
  std::vector<int> x2, f64;
  for (int i : ids) (b->st[i].resid64 ? f64 : x2).push_back(i);
  B_TRY(run_rows(b, row_items(b, x2, true),
                 [&](const BItem* d, int k) { return launch_bresid(b->dinst, d, k, b->stream); }));
  B_TRY(run_rows(b, row_items(b, f64, true),
                 [&](const BItem* d, int k) { return launch_bresid64(b->dinst, d, k, b->stream); }));
  return NS_OK;
}

std::vector<BItem> row_items(const ns_batch* b, const std::vector<int>& ids, bool with_rhs) {
  std::vector<BItem> it;
  for (int i : ids) {
    const int cmax = with_rhs ? b->nrhs[i] : 1;
    for (int r = 0; r < b->n[i]; r += 8)
      for (int c = 0; c < cmax; c += kBRhs) it.push_back(BItem{i, r, c, b->st[i].cur});
  }
  return it;
}

// Make `to` wait for everything enqueued on `from` so far.
ns_status join(ns_batch* b, cudaStream_t from, cudaStream_t to) {
  cudaEvent_t ev = from == b->stream ? b->ev_r : b->ev_p;
  B_CK(cudaEventRecord(ev, from));
  B_CK(cudaStreamWaitEvent(to, ev, 0));
  return NS_OK;
}

// Read every slot's scalars and the device error word: the product stream
// joins the row stream, which is then synchronised.
ns_status sync_read(ns_batch* b) {
  B_TRY(join(b, b->pstream, b->stream));
  int hi_slot = 0;
  for (int k = 0; k < b->cap; ++k)
    if (b->used[k]) hi_slot = k + 1;
  if (hi_slot > 0)
    B_CK(cudaMemcpyAsync(b->hscal, b->dscal, static_cast<size_t>(hi_slot) * b->scal_stride * sizeof(double),
                         cudaMemcpyDeviceToHost, b->stream));
  char* herr_slot = b->hstage + b->stage_cap - 64;
  B_CK(cudaMemcpyAsync(herr_slot, b->derr, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  const auto w0 = std::chrono::steady_clock::now();
  B_CK(cudaStreamSynchronize(b->stream));
  b->wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  b->stage_used = 0;
  int herr = 0;
  memcpy(&herr, herr_slot, sizeof(int));
  if (herr != DEV_OK) {
    cudaMemsetAsync(b->derr, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    return bfail(b, NS_ERR_TIMEOUT, "a bounded device-side wait ran out (tcgen05 GEMM)");
  }
  return NS_OK;
}

template <typename F>
ns_status run_rows(ns_batch* b, const std::vector<BItem>& items, F launch) {
  if (items.empty()) return NS_OK;
  const BItem* d = static_cast<const BItem*>(stage(b, items.data(), items.size() * sizeof(BItem), b->stream));
  if (!d) return bfail(b, NS_ERR_OOM, "staging area exhausted");
  B_CK(launch(d, static_cast<int>(items.size())));
  if (b->stats) b->stats->kernel_launches++;
  return NS_OK;
}

ns_status run_list(ns_batch* b, const std::vector<int>& ids,
                   cudaError_t (*launch)(const BInst*, const int*, int, cudaStream_t), cudaStream_t st) {
  if (ids.empty()) return NS_OK;
  const int* d = static_cast<const int*>(stage(b, ids.data(), ids.size() * sizeof(int), st));
  if (!d) return bfail(b, NS_ERR_OOM, "staging area exhausted");
  B_CK(launch(b->dinst, d, static_cast<int>(ids.size()), st));
  if (b->stats) b->stats->kernel_launches++;
  return NS_OK;
}

// One controller decision for system i after its residual (and ||F||, while
// its Newton-Schulz loop runs) were read.  Same rules as the single-system run.
void decide(ns_batch* b, int i) {
  InstState& s = b->st[i];
  const double tol = s.tol;
  const double* sc = b->hscal + static_cast<size_t>(i) * b->scal_stride;
  const int nr = b->nrhs[i];
  double rr = INFINITY;
  s.recompute = false;
  if (!s.has_res && s.ns_active && b->opt.couple_frob > 0.0 && std::sqrt(sc[2]) <= b->opt.couple_frob) {
    s.need_res = true;  // the first G_k with ||I - A G_k||_F <= couple_frob
    return;
  }
  if (s.has_res) {
    rr = 0.0;
    for (int c = 0; c < nr; ++c) {
      const double bb = sc[kScalR + nr + c], r = sc[kScalR + c];
      const double q = bb > 0 ? std::sqrt(r / bb) : std::sqrt(r);
      rr = std::max(rr, std::isnan(q) ? INFINITY : q);
    }
    s.rel_res = rr;
    if (!std::isfinite(rr)) {
      s.finished = true;
      s.status = NS_ERR_NONFINITE;
      return;
    }
    if (tol > 0 && rr <= tol) {
      s.finished = true;
      s.converged = true;
      s.status = NS_OK;
      return;
    }
  }
  if (!s.ns_active) {
    // Richardson alone: stop when it no longer contracts (rho(I - A G) ~ 1 at
    // this precision) instead of spending the whole sweep budget
    const double prev = s.last_rr_sweep;
    s.last_rr_sweep = rr;
    // contraction per sweep over the k_meas sweeps since the previous measurement
    const double ratio = (std::isfinite(prev) && prev > 0.0) ? std::pow(rr / prev, 1.0 / s.k_meas) : INFINITY;
    if (std::isfinite(prev)) s.stall = ratio > 0.95 ? s.stall + 1 : 0;
    s.best_rr = std::min(s.best_rr, rr);
    bool stop = s.stall >= 4 || rr > 10.0 * s.best_rr;
    // ... or when even the better of the last two contraction ratios cannot
    // reach tol within the sweeps left (an optimistic projection)
    s.proj_need = 0.0;
    if (std::isfinite(ratio)) {
      const double rho = std::min(ratio, s.prev_sweep_ratio);
      s.prev_sweep_ratio = ratio;
      if (tol > 0 && rho < 1.0) {
        s.proj_need = std::log(tol / rr) / std::log(rho);
        if (s.proj_need > static_cast<double>(s.sweeps_left)) stop = true;
      }
    }
    if (stop && !s.resid64 && tol > 0 && s.sweeps_left > 0) {
      // the split-f32 residual may be what stalls: form it in FP64 from here on
      s.resid64 = true;
      s.stall = 0;
      s.best_rr = INFINITY;
      s.prev_sweep_ratio = INFINITY;
      s.proj_need = 0.0;
      stop = false;
    }
    if (stop) {
      s.finished = true;
      s.status = NS_NOT_CONVERGED;
    }
    return;
  }
  const double frob = std::sqrt(sc[2]);
  if (!std::isfinite(frob)) {
    s.finished = true;
    s.status = NS_ERR_NONFINITE;
    return;
  }
  const bool autop = b->opt.precision == NS_AUTO;
  const double ratio = frob / s.prev_frob;
  if (autop && s.prec == NS_BF16 && s.done >= 2 && frob < s.prev_frob && ratio > s.prev_ratio + 0.02) {
    s.prec = NS_BF16X3;
    s.prev_ratio = INFINITY;
    s.recompute = true;
    return;
  }
  if (autop && s.prec == NS_BF16 && s.done > 0 && frob >= s.prev_frob) {
    s.cur ^= 1;
    s.done--;
    s.prec = NS_BF16X3;
    s.prev_frob = INFINITY;
    s.rollbacks++;
    s.recompute = true;
    return;
  }
  const double sqrt_n = std::sqrt(static_cast<double>(b->n[i]));
  if (frob > 2.0 * sqrt_n + 1.0 && frob > 2.0 * s.prev_frob) {
    s.finished = true;
    s.status = NS_ERR_DIVERGED;
    return;
  }
  if (b->opt.ns_stop && (!autop || s.prec != NS_BF16)) {
    bool stop = frob <= b->opt.ns_stop_frob;
    if (!stop && s.has_res && frob < 1.0 && tol > 0 && rr > tol) {
      const double need = std::ceil(std::log(tol / rr) / std::log(frob));
      if (need <= s.sweeps_left && need * sweep_cost_i(b, i) <= step_cost_i(b, i, s.prec) + 2.0 * sweep_cost_i(b, i))
        stop = true;
    }
    if (!stop && s.prev_frob < 1.0 && frob >= 0.5 * s.prev_frob) {
      stop = true;
      if (frob > s.prev_frob) s.cur ^= 1;
    }
    if (stop) s.ns_active = false;
  }
  s.frob_now = frob;
}

// Preparation of newly admitted systems: norms, splits and limbs of A, G0,
// theta = 0 and its limbs.  iters[k] / tol[k] belong to ids[k].
ns_status prep_slots(ns_batch* b, const std::vector<int>& ids, const std::vector<int>& iters,
                     const std::vector<double>& tol) {
  if (ids.empty()) return NS_OK;
  for (size_t k = 0; k < ids.size(); ++k) {
    const int i = ids[k];
    InstState s;
    s.prec = b->opt.precision == NS_AUTO ? NS_BF16 : b->opt.precision;
    s.sweeps_left = b->opt.max_sweeps;
    s.ns_active = iters[k] > 0;
    s.iters = iters[k];
    s.tol = tol[k];
    b->st[i] = s;
  }
  B_TRY(run_rows(b, row_items(b, ids, false),
                 [&](const BItem* d, int k) { return launch_bprep(b->dinst, d, k, b->stream); }));
  B_TRY(run_list(b, ids, launch_bnorms, b->stream));
  B_TRY(run_rows(b, row_items(b, ids, false), [&](const BItem* d, int k) {
    return launch_bg0(b->dinst, d, k, b->opt.g0_mode, 1, b->stream);
  }));
  // the products read the splits of A and G0 (and the tables just published)
  return join(b, b->stream, b->pstream);
}

// One controller pass over the active systems.  Two streams: the product
// stream forms F = I - A G (and ||F||) for the systems whose Newton-Schulz
// loop runs while the row stream forms the residuals (Richardson branch); one
// join and device sync; host decisions; then the product chain and the
// Richardson update, again on the two streams.  With opt.couple_frob > 0 a
// system's Richardson branch starts with its first G_k whose ||I - A G_k||_F
// is at most that (its residual is then formed after the sync).
ns_status pass(ns_batch* b, const std::vector<int>& act) {
  const double couple = b->opt.couple_frob;
  std::vector<int> nsact, rich;
  // Richardson-only systems far from tol take extra sweeps before this pass's
  // measured residual: at most half of the (optimistic) projected remainder, so
  // no system is swept past the sweep where it would have met tol
  std::vector<int> pre(b->cap, 0);
  int max_pre = 0;
  for (int i : act) {
    InstState& s = b->st[i];
    s.k_meas = 1;
    if (s.ns_active || s.proj_need < 3.0) continue;
    int k = static_cast<int>((s.proj_need - 1.0) / 2.0);
    k = std::min(std::min(k, b->max_pre), s.sweeps_left - 1);
    if (k < 1) continue;
    pre[i] = k;
    max_pre = std::max(max_pre, k);
  }
  for (int j = 0; j < max_pre; ++j) {
    std::vector<int> sw;
    for (int i : act)
      if (pre[i] > j) sw.push_back(i);
    B_TRY(launch_residuals(b, sw));
    B_TRY(run_rows(b, row_items(b, sw, true),
                   [&](const BItem* d, int k) { return launch_bupdate(b->dinst, d, k, b->stream); }));
    for (int i : sw) {
      InstState& s = b->st[i];
      s.sweeps++;
      s.sweeps_left--;
      s.k_meas++;
    }
  }
  for (int i : act) {
    InstState& s = b->st[i];
    if (s.ns_active) nsact.push_back(i);
    s.has_res = !s.ns_active || couple <= 0.0 || s.coupled;
    if (s.has_res) rich.push_back(i);
  }
  if (!nsact.empty()) {
    B_TRY(launch_products(b, nsact, {0}));
    B_TRY(run_list(b, nsact, launch_bfrob, b->pstream));
  }
  B_TRY(launch_residuals(b, rich));
  B_TRY(run_list(b, rich, launch_brsq, b->stream));
  B_TRY(sync_read(b));
  for (int i : act) decide(b, i);
  // follow-ups, then decide again: systems whose coupling starts with this
  // pass's G_k need their residual; systems that switched precision or rolled
  // back need F formed again
  for (int guard = 0; guard < 8; ++guard) {
    std::vector<int> late, redo;
    for (int i : act) {
      InstState& s = b->st[i];
      if (s.finished) continue;
      if (s.need_res) {
        s.need_res = false;
        s.has_res = s.coupled = true;
        late.push_back(i);
      } else if (s.recompute) {
        redo.push_back(i);
      }
    }
    if (late.empty() && redo.empty()) break;
    if (!redo.empty()) {
      B_TRY(launch_products(b, redo, {0}));
      B_TRY(run_list(b, redo, launch_bfrob, b->pstream));
    }
    if (!late.empty()) {
      B_TRY(launch_residuals(b, late));
      B_TRY(run_list(b, late, launch_brsq, b->stream));
    }
    B_TRY(sync_read(b));
    for (int i : late) decide(b, i);
    for (int i : redo) decide(b, i);
  }
  std::vector<int> step, upd;
  for (int i : act) {
    InstState& s = b->st[i];
    if (s.finished) continue;
    if (s.ns_active) {
      step.push_back(i);
      if (s.has_res) upd.push_back(i);
    } else if (!s.has_res) {
      // Newton-Schulz stopped on a pass without a residual: the next pass forms it
    } else if (s.sweeps_left > 0) {
      upd.push_back(i);
      s.sweeps_left--;
    } else {
      s.finished = true;
      s.status = NS_NOT_CONVERGED;
    }
  }
  // the chain reads G_k and writes the other G buffer; the update applies G_k
  if (!step.empty()) {
    if (b->levels == 0) {
      B_TRY(launch_products(b, step, {1}));
      B_TRY(launch_products(b, step, {2}));
    } else {
      for (int j = 0; j < b->levels; ++j) {
        if (j + 1 < b->levels)
          B_TRY(launch_products(b, step, {1 + 2 * j, 2 + 2 * j}));
        else
          B_TRY(launch_products(b, step, {1 + 2 * j}));
      }
    }
  }
  if (!upd.empty())
    B_TRY(run_rows(b, row_items(b, upd, true),
                   [&](const BItem* d, int k) { return launch_bupdate(b->dinst, d, k, b->stream); }));
  for (int i : upd) b->st[i].sweeps++;
  for (int i : step) {
    InstState& s = b->st[i];
    s.prev_ratio = (s.done > 0 && std::isfinite(s.prev_frob)) ? s.frob_now / s.prev_frob : INFINITY;
    s.prev_frob = s.frob_now;
    s.cur ^= 1;
    s.done++;
    if (s.done >= s.iters) s.ns_active = false;
  }
  return NS_OK;
}

// A fixed batch whose systems all fit one CTA: one persistent launch solves
// every system whole (batch_fused.cu), largest first; one synchronisation.
ns_status fused_solve(ns_batch* b, int count, int iters, double tol, ns_batch_stats* stats) {
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->n[x] > b->n[y]; });
  const int* dl = static_cast<const int*>(stage(b, order.data(), order.size() * sizeof(int), b->stream));
  if (!dl) return bfail(b, NS_ERR_OOM, "staging area exhausted");
  B_CK(cudaMemsetAsync(b->dnext, 0, sizeof(int), b->stream));
  FusedParams p;
  memset(&p, 0, sizeof(p));
  p.prob = b->dprob;
  p.inst = b->dinst;
  p.list = dl;
  p.count = count;
  p.next = b->dnext;
  p.out = b->dfout;
  p.ntypes = b->ntypes;
  p.levels = b->levels;
  p.precision = b->opt.precision;
  p.g0_mode = b->opt.g0_mode;
  p.ns_stop = b->opt.ns_stop;
  p.max_sweeps = b->opt.max_sweeps;
  p.max_pre = b->max_pre;
  p.iters = iters;
  p.ns_stop_frob = b->opt.ns_stop_frob;
  p.couple_frob = b->opt.couple_frob;
  p.tol = tol;
  p.timeout_ns = static_cast<unsigned long long>(b->opt.timeout_s * 1e9);
  p.err = b->derr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (b->opt.profile) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
  }
  B_CK(launch_fused_solve(p, b->num_sms, b->stream));
  if (b->opt.profile) cudaEventRecord(e1, b->stream);
  const size_t off = rup(b->stage_used, 256);
  const size_t bytes = sizeof(FusedOut) * static_cast<size_t>(count);
  if (off + bytes + 64 > b->stage_cap) return bfail(b, NS_ERR_OOM, "staging area exhausted");
  FusedOut* hout = reinterpret_cast<FusedOut*>(b->hstage + off);
  int* herr = reinterpret_cast<int*>(b->hstage + off + bytes);
  B_CK(cudaMemcpyAsync(hout, b->dfout, bytes, cudaMemcpyDeviceToHost, b->stream));
  B_CK(cudaMemcpyAsync(herr, b->derr, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  B_CK(cudaStreamSynchronize(b->stream));
  b->stage_used = 0;
  float ms = 0.f;
  if (b->opt.profile) {
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (*herr != DEV_OK) {
    cudaMemsetAsync(b->derr, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    return bfail(b, NS_ERR_TIMEOUT, "a bounded device-side wait ran out (fused small-system solve)");
  }
  int passes = 0;
  double useful = 0.0, executed = 0.0;
  for (int i = 0; i < count; ++i) {
    const FusedOut& o = hout[i];
    InstState& st = b->st[i];
    st = InstState();
    st.finished = true;
    st.status = o.status;
    st.converged = o.converged != 0;
    st.done = o.done;
    st.sweeps = o.sweeps;
    st.rollbacks = o.rollbacks;
    st.rel_res = o.rel_res;
    passes = std::max(passes, o.passes);
    const double f = 2.0 * b->n[i] * static_cast<double>(b->n[i]) * b->n[i];
    useful += f * (o.prods1 + o.prods3);
    executed += f * (o.prods1 + 3.0 * o.prods3);
  }
  if (const char* path = std::getenv("NSGB_FUSED_TRACE")) {
    // per-system record of the fused launch, for profiling: n, outcome, steps,
    // sweeps, passes, SM cycles and SM
    if (FILE* f = std::fopen(path, "w")) {
      std::fprintf(f, "slot,n,status,ns_iters,sweeps,passes,cycles,sm\n");
      for (int i = 0; i < count; ++i)
        std::fprintf(f, "%d,%d,%d,%d,%d,%d,%lld,%d\n", i, b->n[i], hout[i].status, hout[i].done, hout[i].sweeps,
                     hout[i].passes, hout[i].cycles, hout[i].sm);
      std::fclose(f);
    }
  }
  if (stats) {
    stats->passes = passes;
    stats->kernel_launches = 1;
    stats->gemm_flops = executed;
    stats->useful_flops = useful;
    stats->fused = 1;
    stats->fused_ms = ms;
  }
  return NS_OK;
}

// Options the batched path supports, checked for both the batch and the server.
ns_status check_opts(ns_options* o, const ns_options* opt, int order) {
  if (opt)
    *o = *opt;
  else
    ns_default_options(o);
  if (o->form != 0 || o->pow_mode != 0 || o->g0_mode < 0 || o->g0_mode > 2 || o->g0_order != 0) return NS_ERR_UNSUPPORTED;
  if (o->precision != NS_AUTO && o->precision != NS_BF16 && o->precision != NS_BF16X3) return NS_ERR_UNSUPPORTED;
  if (order != 3 && (order < 2 || order > 64 || (order & (order - 1)) != 0)) return NS_ERR_ARG;
  if (o->timeout_s <= 0) o->timeout_s = 2.0;
  return NS_OK;
}

// Tables, staging and arena in one device allocation.
ns_status alloc_batch(ns_batch* b, int cap, int max_nrhs, size_t arena_bytes) {
  b->cap = cap;
  b->max_nrhs = max_nrhs;
  b->scal_stride = kScalR + 2 * max_nrhs;
  b->stage_cap = std::max<size_t>(16u << 20, static_cast<size_t>(cap) * 48 * 1024);
  size_t total = 0;
  auto take = [&](size_t bytes) {
    const size_t off = rup(total, 256);
    total = off + bytes;
    return off;
  };
  const size_t o_prob = take(sizeof(TcProblem) * static_cast<size_t>(cap) * b->ntypes * 4 + 64);
  const size_t o_inst = take(sizeof(BInst) * static_cast<size_t>(cap));
  const size_t o_scal = take(sizeof(double) * static_cast<size_t>(cap) * b->scal_stride);
  const size_t o_err = take(64);
  const size_t o_fout = take(sizeof(FusedOut) * static_cast<size_t>(cap) + 64);
  const size_t o_stage = take(b->stage_cap);
  const size_t o_arena = take(arena_bytes);
  if (cudaMalloc(&b->dmem, total) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_OOM;
  }
  char* base = static_cast<char*>(b->dmem);
  if (cudaMemset(base, 0, o_arena) != cudaSuccess || cudaMallocHost(&b->hscal, sizeof(double) * cap * b->scal_stride) !=
                                                         cudaSuccess ||
      cudaMallocHost(&b->hstage, b->stage_cap) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_OOM;
  }
  b->dprob = reinterpret_cast<TcProblem*>(rup(reinterpret_cast<uintptr_t>(base + o_prob), 64));
  b->dinst = reinterpret_cast<BInst*>(base + o_inst);
  b->dscal = reinterpret_cast<double*>(base + o_scal);
  b->derr = reinterpret_cast<int*>(base + o_err);
  b->dnext = b->derr + 4;
  b->dfout = reinterpret_cast<FusedOut*>(base + o_fout);
  b->dstage = base + o_stage;
  b->abase = base + o_arena;
  b->asize = arena_bytes;
  b->arena.init(arena_bytes);
  b->used.assign(cap, 0);
  b->reg_off.assign(cap, 0);
  b->lay.assign(cap, SlotLayout());
  b->n.assign(cap, 0);
  b->nrhs.assign(cap, 0);
  b->ld.assign(cap, 0);
  b->bn.assign(cap, 0);
  b->tiles_m.assign(cap, 0);
  b->tiles_n.assign(cap, 0);
  b->mats.assign(cap, std::array<BMat, kNumMats>());
  b->hinst.assign(cap, BInst());
  b->st.assign(cap, InstState());
  return NS_OK;
}

ns_status init_batch(ns_batch* b, int order, const ns_options* opt) {
  ns_status s = check_opts(&b->opt, opt, order);
  if (s != NS_OK) return s;
  b->order = order;
  b->levels = 0;
  if (order != 3)
    while ((1 << b->levels) < order) ++b->levels;
  b->ntypes = order == 3 ? 3 : 2 * b->levels;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (cudaStreamCreateWithFlags(&b->pstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_r, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_p, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

void release_batch(ns_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& m : b->retry)
    for (auto& kv : m) ns_destroy(kv.second);
  for (cudaStream_t st : b->retry_streams) cudaStreamDestroy(st);
  if (b->pstream) {
    cudaStreamSynchronize(b->pstream);
    cudaStreamDestroy(b->pstream);
  }
  if (b->ev_r) cudaEventDestroy(b->ev_r);
  if (b->ev_p) cudaEventDestroy(b->ev_p);
  if (b->dmem) cudaFree(b->dmem);
  if (b->hscal) cudaFreeHost(b->hscal);
  if (b->hstage) cudaFreeHost(b->hstage);
  delete b;
}

}  // namespace

// ============================================================== server state
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  ns_request r;
  Clock::time_point t_submit, t_admit;
  bool done = false;
  ns_result res;
};

}  // namespace

struct ns_server {
  ns_batch* b = nullptr;
  cudaStream_t own_stream = nullptr;
  std::mutex mu;       // queue, request records, slot tickets, statistics
  std::mutex tick_mu;  // one tick at a time
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<uint64_t> slot_ticket;  // 0: slot free or not yet owned
  std::vector<int> retiring;          // slots whose theta copy is in flight
  uint64_t next_ticket = 1;
  std::thread worker;
  bool running = false, stopping = false;
  ns_server_stats stats;
  ns_batch_stats bst;  // launch and flop counters of the passes (tick thread only)
  std::string err;
};

// ====================================================================== ABI
extern "C" {

ns_status ns_batch_create(int count, const int64_t* n, const int* nrhs, int order, const ns_options* opt,
                          ns_batch** out) {
  if (!out || count <= 0 || !n || !nrhs) return NS_ERR_ARG;
  int max_nrhs = 1;
  for (int i = 0; i < count; ++i) {
    if (n[i] <= 0 || n[i] > 16384 || nrhs[i] <= 0 || nrhs[i] > 1024) return NS_ERR_ARG;
    max_nrhs = std::max(max_nrhs, nrhs[i]);
  }
  ns_batch* b = new ns_batch();
  ns_status s = init_batch(b, order, opt);
  if (s != NS_OK) {
    delete b;
    return s;
  }
  size_t arena = 0;
  for (int i = 0; i < count; ++i) arena += slot_layout(static_cast<int>(n[i]), nrhs[i], false).bytes;
  s = alloc_batch(b, count, max_nrhs, arena);
  if (s != NS_OK) {
    release_batch(b);
    return s;
  }
  for (int i = 0; i < count; ++i) {
    if (add_slot(b, static_cast<int>(n[i]), nrhs[i], false) != i || publish_slot(b, i, true) != NS_OK) {
      release_batch(b);
      return NS_ERR_OOM;
    }
    if (b->stage_used > b->stage_cap / 2) {
      cudaStreamSynchronize(b->stream);
      b->stage_used = 0;
    }
  }
  b->fixed_count = count;
  b->max_pre = 7;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    release_batch(b);
    return NS_ERR_CUDA;
  }
  b->stage_used = 0;
  *out = b;
  return NS_OK;
}

ns_status ns_batch_destroy(ns_batch* b) {
  release_batch(b);
  return NS_OK;
}

ns_status ns_batch_set_stream(ns_batch* b, void* stream) {
  if (!b) return NS_ERR_ARG;
  b->stream = static_cast<cudaStream_t>(stream);
  return NS_OK;
}

const char* ns_batch_last_error(const ns_batch* b) { return b ? b->err.c_str() : "null batch"; }

namespace {
// Option fp64_slices on a batch: every system the batched solve did not
// converge (the binary32 masters cannot carry it) is solved again alone by the
// single-system AUTO path with s-digit slice products (its hand-over to the
// FP64 path from the binary32 floor), from theta = 0.  Each such solve is
// latency-bound on a few SMs, so kRetryWorkers host threads run them at once,
// each on its own stream with its own contexts; system k goes to worker
// k mod kRetryWorkers, and a system's arithmetic does not depend on which
// systems run beside it.  Its outcome replaces the batched one; ns_iters and
// sweeps add up both attempts.
constexpr int kRetryWorkers = 16;

ns_status slice_handover(ns_batch* b, const double* const* A, const double* const* B, double* const* Theta, int iters,
                         double tol, ns_batch_stats* stats) {
  const auto t0 = Clock::now();
  std::vector<int> todo;
  for (int i = 0; i < b->fixed_count; ++i) {
    const InstState& s = b->st[i];
    if (!s.converged && (s.status == NS_NOT_CONVERGED || s.status == NS_ERR_DIVERGED)) todo.push_back(i);
  }
  const int nw = std::min<int>(kRetryWorkers, static_cast<int>(todo.size()));
  if ((int)b->retry.size() < nw) b->retry.resize(nw);
  while ((int)b->retry_streams.size() < nw) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, NS_ERR_CUDA, "slice hand-over: stream");
    }
    b->retry_streams.push_back(st);
  }
  std::vector<ns_status> werr(nw, NS_OK);
  std::vector<std::string> wmsg(nw);
  std::vector<ns_status> out(todo.size(), NS_NOT_CONVERGED);
  std::vector<int> out_ns(todo.size(), 0), out_sw(todo.size(), 0);
  std::vector<double> out_rr(todo.size(), INFINITY);
  auto work = [&](int w) {
    if (cudaSetDevice(b->device) != cudaSuccess) {
      werr[w] = NS_ERR_CUDA;
      return;
    }
    for (size_t k = w; k < todo.size(); k += nw) {
      const int i = todo[k];
      const int n = b->n[i];
      auto it = b->retry[w].find(n);
      if (it == b->retry[w].end()) {
        ns_options o = b->opt;
        o.precision = NS_AUTO;
        o.batch_fused = 0;
        o.profile = 0;
        ns_ctx* c = nullptr;
        const ns_status r = ns_create(n, b->order, nullptr, 0, &o, &c);
        if (r != NS_OK) {
          werr[w] = r;
          wmsg[w] = "slice hand-over: context";
          return;
        }
        ns_set_stream(c, b->retry_streams[w]);
        it = b->retry[w].emplace(n, c).first;
      }
      ns_stats st;
      const ns_status r = ns_richardson_solve(it->second, A[i], B[i], b->nrhs[i], nullptr, iters, tol, Theta[i], &st);
      if (r < 0 && r != NS_ERR_DIVERGED && r != NS_ERR_NONFINITE) {
        werr[w] = r;
        wmsg[w] = ns_last_error(it->second);
        return;
      }
      out[k] = r;
      out_ns[k] = st.ns_iters;
      out_sw[k] = st.sweeps;
      if (r == NS_OK) {
        std::vector<double> rr(b->nrhs[i]);
        if (ns_residual(it->second, A[i], Theta[i], B[i], b->nrhs[i], rr.data()) == NS_OK)
          out_rr[k] = *std::max_element(rr.begin(), rr.end());
      }
      if (cudaStreamSynchronize(b->retry_streams[w]) != cudaSuccess) {
        werr[w] = NS_ERR_CUDA;
        wmsg[w] = "slice hand-over: stream";
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < nw; ++w) pool.emplace_back(work, w);
  if (nw > 0) work(0);
  for (auto& t : pool) t.join();
  B_CK(cudaSetDevice(b->device));
  for (int w = 0; w < nw; ++w)
    if (werr[w] != NS_OK) return bfail(b, werr[w], wmsg[w]);
  int conv = 0;
  for (size_t k = 0; k < todo.size(); ++k) {
    InstState& s = b->st[todo[k]];
    s.done += out_ns[k];
    s.sweeps += out_sw[k];
    s.status = out[k];
    s.converged = out[k] == NS_OK;
    if (s.converged) {
      conv++;
      s.rel_res = out_rr[k];
    }
  }
  if (stats) {
    stats->slice_retried = static_cast<int>(todo.size());
    stats->slice_retried_converged = conv;
    stats->slice_retry_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  return NS_OK;
}
}  // namespace

ns_status ns_batch_solve(ns_batch* b, const double* const* A, const double* const* B, double* const* Theta,
                         int iters, double tol, ns_batch_stats* stats) {
  if (!b || !A || !B || !Theta || iters < 0 || b->fixed_count <= 0) return NS_ERR_ARG;
  const auto t0 = Clock::now();
  b->err.clear();
  b->stats = stats;
  if (stats) memset(stats, 0, sizeof(*stats));
  B_CK(cudaSetDevice(b->device));
  const int count = b->fixed_count;
  b->stage_used = 0;
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) {
    if (!A[i] || !B[i] || !Theta[i]) return bfail(b, NS_ERR_ARG, "null instance pointer");
    all[i] = i;
    b->hinst[i].A = A[i];
    b->hinst[i].B = B[i];
    b->hinst[i].Th = Theta[i];
  }
  B_CK(cudaMemcpyAsync(b->dinst, b->hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, b->stream));
  bool fuse = b->opt.batch_fused != 0;
  for (int i = 0; i < count && fuse; ++i) fuse = b->n[i] <= kFusedMaxN;
  int passes = 0;
  if (fuse) {
    B_TRY(fused_solve(b, count, iters, tol, stats));
    passes = stats ? stats->passes : 0;
  } else {
    B_TRY(prep_slots(b, all, std::vector<int>(count, iters), std::vector<double>(count, tol)));
  }
  for (; !fuse;) {
    std::vector<int> act;
    for (int i = 0; i < count; ++i)
      if (!b->st[i].finished) act.push_back(i);
    if (act.empty()) break;
    ++passes;
    B_TRY(pass(b, act));
    if (passes > 2 * iters + b->opt.max_sweeps + 8) break;
  }
  B_TRY(join(b, b->pstream, b->stream));
  B_CK(cudaStreamSynchronize(b->stream));
  b->stage_used = 0;
  for (int i = 0; i < count; ++i)
    if (!b->st[i].finished) {
      b->st[i].finished = true;
      b->st[i].status = NS_NOT_CONVERGED;
    }
  if (b->opt.fp64_slices > 0 && tol > 0) B_TRY(slice_handover(b, A, B, Theta, iters, tol, stats));
  int nconv = 0, nfail = 0;
  for (int i = 0; i < count; ++i) {
    if (b->st[i].converged)
      nconv++;
    else
      nfail++;
  }
  if (stats) {
    stats->passes = passes;
    stats->converged = nconv;
    stats->not_converged = nfail;
    stats->wall_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    double useful = 0.0;
    for (int i = 0; i < count; ++i) useful += 2.0 * b->n[i] * static_cast<double>(b->n[i]) * b->n[i];
    stats->useful_flops_per_product = useful;
  }
  b->stats = nullptr;
  return nfail == 0 ? NS_OK : NS_NOT_CONVERGED;
}

ns_status ns_batch_result(const ns_batch* b, int i, int* status, int* ns_iters, int* sweeps, double* rel_res) {
  if (!b || i < 0 || i >= b->fixed_count) return NS_ERR_ARG;
  const InstState& s = b->st[i];
  if (status) *status = s.status;
  if (ns_iters) *ns_iters = s.done;
  if (sweeps) *sweeps = s.sweeps;
  if (rel_res) *rel_res = s.rel_res;
  return NS_OK;
}

// ------------------------------------------------------------------ server
ns_status ns_server_create(size_t mem_budget_bytes, int max_requests, int max_nrhs, int order,
                           const ns_options* opt, ns_server** out) {
  if (!out || mem_budget_bytes < (1u << 20) || max_requests <= 0 || max_requests > 65536 || max_nrhs <= 0 ||
      max_nrhs > 1024)
    return NS_ERR_ARG;
  ns_server* sv = new ns_server();
  sv->b = new ns_batch();
  ns_status s = init_batch(sv->b, order, opt);
  if (s == NS_OK && cudaStreamCreateWithFlags(&sv->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s = NS_ERR_CUDA;
  }
  sv->b->stream = sv->own_stream;
  if (s == NS_OK) s = alloc_batch(sv->b, max_requests, max_nrhs, mem_budget_bytes);
  if (s != NS_OK) {
    release_batch(sv->b);
    if (sv->own_stream) cudaStreamDestroy(sv->own_stream);
    delete sv;
    return s;
  }
  sv->slot_ticket.assign(max_requests, 0);
  memset(&sv->stats, 0, sizeof(sv->stats));
  memset(&sv->bst, 0, sizeof(sv->bst));
  sv->b->stats = &sv->bst;
  *out = sv;
  return NS_OK;
}

ns_status ns_server_set_stream(ns_server* sv, void* stream) {
  if (!sv) return NS_ERR_ARG;
  std::lock_guard<std::mutex> tk(sv->tick_mu);
  cudaStreamSynchronize(sv->b->stream);
  cudaStreamSynchronize(sv->b->pstream);
  sv->b->stream = stream ? static_cast<cudaStream_t>(stream) : sv->own_stream;
  return NS_OK;
}

const char* ns_server_last_error(const ns_server* sv) {
  if (!sv) return "null server";
  return sv->err.empty() ? sv->b->err.c_str() : sv->err.c_str();
}

ns_status ns_server_submit(ns_server* sv, const ns_request* rq, uint64_t* ticket) {
  if (!sv || !rq || !ticket || rq->n <= 0 || rq->n > 16384 || rq->nrhs <= 0 || rq->nrhs > sv->b->max_nrhs ||
      rq->iters < 0 || !(rq->tol >= 0.0) || !rq->A || !rq->B || !rq->Theta)
    return NS_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  const uint64_t t = sv->next_ticket++;
  Req& r = sv->reqs[t];
  r.r = *rq;
  r.t_submit = Clock::now();
  memset(&r.res, 0, sizeof(r.res));
  r.res.status = NS_NOT_CONVERGED;
  sv->queue.push_back(t);
  sv->stats.submitted++;
  *ticket = t;
  sv->cv.notify_all();
  return NS_OK;
}

ns_status ns_server_poll(ns_server* sv, uint64_t ticket, ns_result* out) {
  if (!sv || !out) return NS_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return NS_ERR_ARG;
  *out = it->second.res;
  out->done = it->second.done ? 1 : 0;
  return NS_OK;
}

ns_status ns_server_release(ns_server* sv, uint64_t ticket) {
  if (!sv) return NS_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end() || !it->second.done) return NS_ERR_ARG;
  sv->reqs.erase(it);
  return NS_OK;
}

ns_status ns_server_tick(ns_server* sv, int* active_out) {
  if (!sv) return NS_ERR_ARG;
  std::lock_guard<std::mutex> tk(sv->tick_mu);
  const auto t_tick = Clock::now();
  ns_batch* b = sv->b;
  if (cudaSetDevice(b->device) != cudaSuccess) return NS_ERR_CUDA;
  // ---- admission, first come first served, while a slot and memory are free
  std::vector<int> fresh;
  std::vector<std::pair<int, ns_request>> copies;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    while (!sv->queue.empty() && b->stage_used < b->stage_cap / 2) {
      const uint64_t t = sv->queue.front();
      Req& r = sv->reqs[t];
      if (slot_layout(static_cast<int>(r.r.n), r.r.nrhs, true).bytes > b->asize) {  // never fits
        sv->queue.pop_front();
        r.done = true;
        r.res.status = NS_ERR_OOM;
        sv->stats.rejected++;
        continue;
      }
      const int slot = add_slot(b, static_cast<int>(r.r.n), r.r.nrhs, true);
      if (slot < 0) break;
      sv->queue.pop_front();
      r.t_admit = Clock::now();
      sv->slot_ticket[slot] = t;
      copies.emplace_back(slot, r.r);
      fresh.push_back(slot);
      sv->stats.admitted++;
    }
  }
  for (size_t k = 0; k < copies.size(); ++k) {
    const int slot = copies[k].first;
    const ns_request& q = copies[k].second;
    const BInst& I = b->hinst[slot];
    B_CK(cudaMemcpyAsync(const_cast<double*>(I.A), q.A, static_cast<size_t>(q.n) * q.n * sizeof(double),
                         cudaMemcpyDefault, b->stream));
    B_CK(cudaMemcpyAsync(const_cast<double*>(I.B), q.B, static_cast<size_t>(q.n) * q.nrhs * sizeof(double),
                         cudaMemcpyDefault, b->stream));
    B_TRY(publish_slot(b, slot, true));
  }
  {
    std::vector<int> it;
    std::vector<double> tl;
    for (const auto& c : copies) {
      it.push_back(c.second.iters);
      tl.push_back(c.second.tol);
    }
    B_TRY(prep_slots(b, fresh, it, tl));
  }
  // ---- one controller pass over every request on the device
  std::vector<int> act;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int k = 0; k < b->cap; ++k)
      if (sv->slot_ticket[k] != 0 && !b->st[k].finished) act.push_back(k);
  }
  if (!act.empty()) {
    B_TRY(pass(b, act));
  } else if (!sv->retiring.empty() || !fresh.empty()) {
    B_TRY(sync_read(b));
  }
  // ---- retirement: copies started by the previous tick have landed (the
  // pass above synchronised the stream after them); start the copies of the
  // requests that finished in this pass
  std::vector<int> finishing;
  for (int k : act)
    if (b->st[k].finished) finishing.push_back(k);
  for (int k : finishing) {
    Req* r = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      r = &sv->reqs[sv->slot_ticket[k]];
    }
    const size_t nb = static_cast<size_t>(b->n[k]) * b->nrhs[k] * sizeof(double);
    B_CK(cudaMemcpyAsync(r->r.Theta, b->hinst[k].Th, nb, cudaMemcpyDefault, b->stream));
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    const auto now = Clock::now();
    for (int k : sv->retiring) {
      Req& r = sv->reqs[sv->slot_ticket[k]];
      const InstState& st = b->st[k];
      r.res.status = st.status;
      r.res.ns_iters = st.done;
      r.res.sweeps = st.sweeps;
      r.res.rel_res = st.rel_res;
      r.res.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
      r.res.queue_ms = std::chrono::duration<double, std::milli>(r.t_admit - r.t_submit).count();
      r.done = true;
      if (st.converged) sv->stats.converged++;
      sv->stats.completed++;
      sv->slot_ticket[k] = 0;
      free_slot(b, k);
    }
    sv->retiring = finishing;
    int on_device = 0;
    for (int k = 0; k < b->cap; ++k)
      if (sv->slot_ticket[k] != 0) on_device++;
    sv->stats.active = on_device;
    sv->stats.queued = static_cast<int>(sv->queue.size());
    sv->stats.ticks++;
    if (!act.empty()) sv->stats.passes++;
    sv->stats.gemm_launches = sv->bst.gemm_launches;
    sv->stats.kernel_launches = sv->bst.kernel_launches;
    sv->stats.gemm_flops = sv->bst.gemm_flops;
    sv->stats.wait_ms = b->wait_ms;
    sv->stats.tick_ms += std::chrono::duration<double, std::milli>(Clock::now() - t_tick).count();
    if (active_out) *active_out = on_device;
  }
  return NS_OK;
}

ns_status ns_server_start(ns_server* sv) {
  if (!sv) return NS_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->running) return NS_OK;
  sv->running = true;
  sv->stopping = false;
  sv->worker = std::thread([sv]() {
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(sv->mu);
        bool busy = !sv->retiring.empty();
        for (uint64_t t : sv->slot_ticket) busy = busy || t != 0;
        if (!busy && sv->queue.empty()) {
          if (sv->stopping) break;
          sv->cv.wait_for(lk, std::chrono::milliseconds(5));
          continue;
        }
      }
      const ns_status s = ns_server_tick(sv, nullptr);
      if (s < 0) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->err = sv->b->err.empty() ? std::string("server tick failed: ") + ns_status_string(s) : sv->b->err;
        sv->stats.last_error = s;
        break;
      }
    }
  });
  return NS_OK;
}

ns_status ns_server_stop(ns_server* sv) {
  if (!sv) return NS_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->running) return NS_OK;
    sv->stopping = true;
    sv->cv.notify_all();
  }
  sv->worker.join();
  sv->running = false;
  return sv->stats.last_error < 0 ? static_cast<ns_status>(sv->stats.last_error) : NS_OK;
}

ns_status ns_server_get_stats(ns_server* sv, ns_server_stats* out) {
  if (!sv || !out) return NS_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  return NS_OK;
}

ns_status ns_server_destroy(ns_server* sv) {
  if (!sv) return NS_OK;
  ns_server_stop(sv);
  release_batch(sv->b);
  if (sv->own_stream) cudaStreamDestroy(sv->own_stream);
  delete sv;
  return NS_OK;
}

}  // extern "C"
