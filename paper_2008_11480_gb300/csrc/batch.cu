// Batched solves of many independent SPD systems of uneven size (the batched
// mode of Newton-Schulz coupled to Richardson).  Every instance runs the same
// method as ns_richardson_solve -- factorized product chain of order 2^m or 3,
// bf16 / split-bf16 products with the per-instance precision controller,
// split-f32 Richardson -- but each pass advances all instances with a handful
// of launches: one list-driven tcgen05 launch per product level (per tile
// width and precision group) and one launch per batched row kernel.
//
// Batch invariance: an instance's tile width depends only on its own size and
// all its reductions run in a fixed order inside its own blocks, so its result
// is the same whether it is solved alone or in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nsgb.h"
#include "batch.h"

using namespace nsgb;

namespace {

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

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
  double prev_frob = INFINITY, prev_ratio = INFINITY, last_rr = INFINITY, frob_now = INFINITY;
  int status = NS_OK;
  int sweeps = 0;
  int rollbacks = 0;
  double rel_res = INFINITY;
};

// Matrices of one instance, in the order the problem table uses.
enum { MA = 0, MG0, MG1, MX0, MX1, MF, MP0, MP1, kNumMats };

}  // namespace

struct ns_batch {
  int count = 0;
  int order = 4;
  int levels = 2;  // order 2^levels, or 0 for order 3
  int ntypes = 0;
  ns_options opt;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 148;
  std::string err;
  void* dmem = nullptr;
  size_t dbytes = 0;
  std::vector<int> n, nrhs, ld, bn, tiles_m, tiles_n;
  std::vector<std::vector<BMat>> mats;  // [inst][kNumMats]
  std::vector<BInst> hinst;
  BInst* dinst = nullptr;
  TcProblem* dprob = nullptr;
  double* dscal = nullptr;
  double* hscal = nullptr;
  std::vector<size_t> scal_off;
  size_t scal_total = 0;
  char* hstage = nullptr;
  char* dstage = nullptr;
  size_t stage_cap = 0, stage_used = 0;
  int* derr = nullptr;
  std::vector<InstState> st;
  std::vector<const double*> A, B;
  std::vector<double*> Th;
  ns_batch_stats* stats = nullptr;
};

namespace {

ns_status bfail(ns_batch* b, ns_status s, const std::string& m) {
  b->err = m;
  return s;
}

#define B_CK(call)                                                                              \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return bfail(b, NS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define B_TRY(expr)           \
  do {                        \
    ns_status s_ = (expr);    \
    if (s_ < 0) return s_;    \
  } while (0)

// Copy `bytes` from host memory into the device staging area (stream ordered);
// returns the device address.  The host side is a pinned mirror of the same
// offsets, so a region is never rewritten before its copy has run: the bump
// pointer is reset only after a stream synchronisation.
void* stage(ns_batch* b, const void* src, size_t bytes) {
  const size_t off = rup(b->stage_used, 256);
  if (off + bytes > b->stage_cap) return nullptr;
  memcpy(b->hstage + off, src, bytes);
  if (cudaMemcpyAsync(b->dstage + off, b->hstage + off, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return nullptr;
  b->stage_used = off + bytes;
  return b->dstage + off;
}

// Product types of one step: order 2^m -> 0: F = I - A G; 1 + 2j: X_{j+1} =
// X_j + X_j P_j; 2 + 2j: P_{j+1} = P_j P_j (j < m - 1).  Order 3 -> 0: F
// (with f32 master), 1: W = F + F F, 2: G' = G + G W.
TcProblem make_problem(const ns_batch* b, int i, int type, int cur, int x3) {
  const std::vector<BMat>& M = b->mats[i];
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

size_t prob_index(const ns_batch* b, int i, int type, int cur, int x3) {
  return ((static_cast<size_t>(i) * b->ntypes + type) * 2 + cur) * 2 + x3;
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

// Launch the products of `types` for the instances in `ids` (each with its own
// current G and precision), one list-driven launch per (tile width, precision).
ns_status launch_products(ns_batch* b, const std::vector<int>& ids, const std::vector<int>& types) {
  for (int bnv : {128, 256}) {
    for (int x3 = 0; x3 < 2; ++x3) {
      std::vector<TcItem> items;
      double flops = 0.0;
      for (int i : ids) {
        if (b->bn[i] != bnv || (b->st[i].prec == NS_BF16X3) != (x3 == 1)) continue;
        for (int t : types) {
          const int pi = static_cast<int>(prob_index(b, i, t, b->st[i].cur, x3));
          for (int mt = 0; mt < b->tiles_m[i]; ++mt)
            for (int nt = 0; nt < b->tiles_n[i]; ++nt) items.push_back(TcItem{pi, mt, nt, 0});
          flops += 2.0 * b->n[i] * static_cast<double>(b->n[i]) * b->n[i] * (x3 ? 3 : 1);
        }
      }
      if (items.empty()) continue;
      const TcItem* ditems = static_cast<const TcItem*>(stage(b, items.data(), items.size() * sizeof(TcItem)));
      if (!ditems) return bfail(b, NS_ERR_OOM, "batch staging area exhausted");
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
        cudaEventRecord(e0, b->stream);
      }
      B_CK(launch_gemm_tc(p, bnv, 1, x3 == 1, b->num_sms, b->stream));
      if (b->stats) {
        b->stats->gemm_launches++;
        b->stats->kernel_launches++;
        b->stats->gemm_flops += flops;
      }
      if (b->opt.profile) {
        cudaEventRecord(e1, b->stream);
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

std::vector<BItem> row_items(const ns_batch* b, const std::vector<int>& ids, bool with_rhs) {
  std::vector<BItem> it;
  for (int i : ids) {
    const int cmax = with_rhs ? b->nrhs[i] : 1;
    for (int r = 0; r < b->n[i]; r += 8)
      for (int c = 0; c < cmax; c += 4) it.push_back(BItem{i, r, c, b->st[i].cur});
  }
  return it;
}

ns_status sync_read(ns_batch* b) {
  B_CK(cudaMemcpyAsync(b->hscal, b->dscal, b->scal_total * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  int herr = 0;
  B_CK(cudaMemcpyAsync(&herr, b->derr, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  B_CK(cudaStreamSynchronize(b->stream));
  b->stage_used = 0;
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
  const BItem* d = static_cast<const BItem*>(stage(b, items.data(), items.size() * sizeof(BItem)));
  if (!d) return bfail(b, NS_ERR_OOM, "batch staging area exhausted");
  B_CK(launch(d, static_cast<int>(items.size())));
  if (b->stats) b->stats->kernel_launches++;
  return NS_OK;
}

ns_status run_list(ns_batch* b, const std::vector<int>& ids,
                   cudaError_t (*launch)(const BInst*, const int*, int, cudaStream_t)) {
  if (ids.empty()) return NS_OK;
  const int* d = static_cast<const int*>(stage(b, ids.data(), ids.size() * sizeof(int)));
  if (!d) return bfail(b, NS_ERR_OOM, "batch staging area exhausted");
  B_CK(launch(b->dinst, d, static_cast<int>(ids.size()), b->stream));
  if (b->stats) b->stats->kernel_launches++;
  return NS_OK;
}

// One controller decision for instance i after its residual (and ||F||, when
// its Newton-Schulz loop is active) were read.  Mirrors the single-system run.
void decide(ns_batch* b, int i, double tol) {
  InstState& s = b->st[i];
  const double* sc = b->hscal + b->scal_off[i];
  const int nr = b->nrhs[i];
  double rr = 0.0;
  for (int c = 0; c < nr; ++c) {
    const double bb = sc[kScalR + nr + c], r = sc[kScalR + c];
    const double q = bb > 0 ? std::sqrt(r / bb) : std::sqrt(r);
    rr = std::max(rr, std::isnan(q) ? INFINITY : q);
  }
  s.rel_res = rr;
  s.last_rr = rr;
  s.recompute = false;
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
  if (!s.ns_active) return;
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
    if (!stop && frob < 1.0 && tol > 0 && rr > tol) {
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
  s.frob_now = frob;  // bookkeeping of the step that follows
}

}  // namespace

extern "C" {

ns_status ns_batch_create(int count, const int64_t* n, const int* nrhs, int order, const ns_options* opt,
                          ns_batch** out) {
  if (!out || count <= 0 || !n || !nrhs) return NS_ERR_ARG;
  ns_options o;
  if (opt)
    o = *opt;
  else
    ns_default_options(&o);
  if (o.form != 0 || o.pow_mode != 0) return NS_ERR_UNSUPPORTED;
  if (o.precision != NS_AUTO && o.precision != NS_BF16 && o.precision != NS_BF16X3) return NS_ERR_UNSUPPORTED;
  if (order != 3 && (order < 2 || (order & (order - 1)) != 0)) return NS_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (n[i] <= 0 || n[i] > 16384 || nrhs[i] <= 0 || nrhs[i] > 1024) return NS_ERR_ARG;
  if (o.timeout_s <= 0) o.timeout_s = 2.0;
  ns_batch* b = new ns_batch();
  b->count = count;
  b->order = order;
  b->levels = 0;
  if (order != 3)
    while ((1 << b->levels) < order) ++b->levels;
  b->ntypes = order == 3 ? 3 : 2 * b->levels;
  b->opt = o;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return NS_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  b->n.assign(n, n + count);
  b->nrhs.assign(nrhs, nrhs + count);
  b->ld.resize(count);
  b->bn.resize(count);
  b->tiles_m.resize(count);
  b->tiles_n.resize(count);
  // ---- sizes and offsets of every per-instance region inside one allocation
  struct Reg {
    size_t off, bytes;
  };
  size_t total = 0;
  auto take = [&](size_t bytes) {
    const size_t off = rup(total, 256);
    total = off + bytes;
    return off;
  };
  std::vector<std::vector<size_t>> off(count);
  b->scal_off.resize(count);
  size_t scal_total = 0;
  for (int i = 0; i < count; ++i) {
    const int ni = static_cast<int>(n[i]);
    const int64_t ldi = rup(ni, 64);
    b->ld[i] = static_cast<int>(ldi);
    b->bn[i] = ni <= 512 ? 128 : 256;
    b->tiles_m[i] = (ni + 127) / 128;
    b->tiles_n[i] = (ni + b->bn[i] - 1) / b->bn[i];
    const size_t sq = static_cast<size_t>(ldi) * ldi;
    std::vector<size_t>& o2 = off[i];
    for (int m = 0; m < kNumMats; ++m) {
      const bool with32 = m == MG0 || m == MG1 || m == MX0 || m == MX1 || m == MF;
      o2.push_back(with32 ? take(sq * 4) : SIZE_MAX);
      o2.push_back(take(sq * 2));
      o2.push_back(take(sq * 2));
    }
    const int nrb = (ni + 7) / 8;
    o2.push_back(take(static_cast<size_t>(ni) * ldi * 4));                        // A1
    o2.push_back(take(static_cast<size_t>(ni) * ldi * 4));                        // A2
    o2.push_back(take(static_cast<size_t>(nrhs[i]) * ldi * 4));                   // T1
    o2.push_back(take(static_cast<size_t>(nrhs[i]) * ldi * 4));                   // T2
    o2.push_back(take(static_cast<size_t>(nrhs[i]) * ldi * 4));                   // R32T
    o2.push_back(take(static_cast<size_t>(ni) * nrhs[i] * 8));                    // R
    o2.push_back(take(static_cast<size_t>(std::max(2 * nrb, nrb * nrhs[i])) * 8));  // part
    o2.push_back(take(static_cast<size_t>(b->tiles_m[i]) * b->tiles_n[i] * 4 * 8));  // fpart
    b->scal_off[i] = scal_total;
    scal_total += kScalR + 2 * static_cast<size_t>(nrhs[i]);
  }
  b->scal_total = scal_total;
  const size_t probs_off = take(sizeof(TcProblem) * static_cast<size_t>(count) * b->ntypes * 4 + 64);
  const size_t inst_off = take(sizeof(BInst) * static_cast<size_t>(count));
  const size_t scal_off = take(scal_total * 8);
  const size_t err_off = take(64);
  b->stage_cap = std::max<size_t>(16u << 20, static_cast<size_t>(count) * 64 * 1024);
  const size_t stage_off = take(b->stage_cap);
  b->dbytes = total;
  if (cudaMalloc(&b->dmem, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return NS_ERR_OOM;
  }
  char* base = static_cast<char*>(b->dmem);
  if (cudaMemset(base, 0, total) != cudaSuccess || cudaMallocHost(&b->hscal, scal_total * 8) != cudaSuccess ||
      cudaMallocHost(&b->hstage, b->stage_cap) != cudaSuccess) {
    cudaGetLastError();
    ns_batch_destroy(b);
    return NS_ERR_OOM;
  }
  b->dprob = reinterpret_cast<TcProblem*>(rup(reinterpret_cast<uintptr_t>(base + probs_off), 64));
  b->dinst = reinterpret_cast<BInst*>(base + inst_off);
  b->dscal = reinterpret_cast<double*>(base + scal_off);
  b->derr = reinterpret_cast<int*>(base + err_off);
  b->dstage = base + stage_off;
  // ---- matrices, tensor maps, instance descriptors
  b->mats.assign(count, std::vector<BMat>(kNumMats));
  b->hinst.resize(count);
  for (int i = 0; i < count; ++i) {
    const int64_t ldi = b->ld[i];
    const std::vector<size_t>& o2 = off[i];
    for (int m = 0; m < kNumMats; ++m) {
      BMat& M = b->mats[i][m];
      M.m32 = o2[3 * m] == SIZE_MAX ? nullptr : reinterpret_cast<float*>(base + o2[3 * m]);
      M.hi = reinterpret_cast<bf16*>(base + o2[3 * m + 1]);
      M.lo = reinterpret_cast<bf16*>(base + o2[3 * m + 2]);
      if (!encode_bf16_map(&M.map_hi, M.hi, ldi, ldi, ldi, 0) || !encode_bf16_map(&M.map_lo, M.lo, ldi, ldi, ldi, 0) ||
          !encode_bf16_map(&M.l3_hi, M.hi, ldi, ldi, ldi, 1) || !encode_bf16_map(&M.l3_lo, M.lo, ldi, ldi, ldi, 1) ||
          !encode_bf16_map(&M.r3_hi, M.hi, ldi, ldi, ldi, 2) || !encode_bf16_map(&M.r3_lo, M.lo, ldi, ldi, ldi, 2)) {
        ns_batch_destroy(b);
        return NS_ERR_CUDA;
      }
    }
    const size_t k0 = 3 * kNumMats;
    BInst& I = b->hinst[i];
    memset(&I, 0, sizeof(I));
    I.n = b->n[i];
    I.nrhs = b->nrhs[i];
    I.ld = b->ld[i];
    I.nfrob = b->tiles_m[i] * b->tiles_n[i] * 4;
    I.Ahi = b->mats[i][MA].hi;
    I.Alo = b->mats[i][MA].lo;
    I.A1 = reinterpret_cast<float*>(base + o2[k0]);
    I.A2 = reinterpret_cast<float*>(base + o2[k0 + 1]);
    I.T1 = reinterpret_cast<float*>(base + o2[k0 + 2]);
    I.T2 = reinterpret_cast<float*>(base + o2[k0 + 3]);
    I.R32T = reinterpret_cast<float*>(base + o2[k0 + 4]);
    I.R = reinterpret_cast<double*>(base + o2[k0 + 5]);
    I.part = reinterpret_cast<double*>(base + o2[k0 + 6]);
    I.fpart = reinterpret_cast<double*>(base + o2[k0 + 7]);
    I.scal = b->dscal + b->scal_off[i];
    for (int c = 0; c < 2; ++c) {
      const BMat& G = b->mats[i][c ? MG1 : MG0];
      I.G32[c] = G.m32;
      I.Ghi[c] = G.hi;
      I.Glo[c] = G.lo;
    }
  }
  std::vector<TcProblem> probs(static_cast<size_t>(count) * b->ntypes * 4);
  for (int i = 0; i < count; ++i)
    for (int t = 0; t < b->ntypes; ++t)
      for (int c = 0; c < 2; ++c)
        for (int x = 0; x < 2; ++x) probs[prob_index(b, i, t, c, x)] = make_problem(b, i, t, c, x);
  if (cudaMemcpy(b->dprob, probs.data(), probs.size() * sizeof(TcProblem), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    ns_batch_destroy(b);
    return NS_ERR_CUDA;
  }
  b->st.assign(count, InstState());
  *out = b;
  return NS_OK;
}

ns_status ns_batch_destroy(ns_batch* b) {
  if (!b) return NS_OK;
  cudaStreamSynchronize(b->stream);
  if (b->dmem) cudaFree(b->dmem);
  if (b->hscal) cudaFreeHost(b->hscal);
  if (b->hstage) cudaFreeHost(b->hstage);
  delete b;
  return NS_OK;
}

ns_status ns_batch_set_stream(ns_batch* b, void* stream) {
  if (!b) return NS_ERR_ARG;
  b->stream = static_cast<cudaStream_t>(stream);
  return NS_OK;
}

const char* ns_batch_last_error(const ns_batch* b) { return b ? b->err.c_str() : "null batch"; }

ns_status ns_batch_solve(ns_batch* b, const double* const* A, const double* const* B, double* const* Theta,
                         int iters, double tol, ns_batch_stats* stats) {
  if (!b || !A || !B || !Theta || iters < 0) return NS_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  b->err.clear();
  b->stats = stats;
  if (stats) memset(stats, 0, sizeof(*stats));
  B_CK(cudaSetDevice(b->device));
  const int count = b->count;
  for (int i = 0; i < count; ++i) {
    if (!A[i] || !B[i] || !Theta[i]) return bfail(b, NS_ERR_ARG, "null instance pointer");
    b->hinst[i].A = A[i];
    b->hinst[i].B = B[i];
    b->hinst[i].Th = Theta[i];
  }
  B_CK(cudaMemcpyAsync(b->dinst, b->hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, b->stream));
  b->stage_used = 0;
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) {
    all[i] = i;
    InstState s;
    s.prec = b->opt.precision == NS_AUTO ? NS_BF16 : b->opt.precision;
    s.sweeps_left = b->opt.max_sweeps;
    s.ns_active = iters > 0;
    b->st[i] = s;
  }
  // ---- preparation: norms, operand splits, G0, theta = 0 and its limbs
  B_TRY(run_rows(b, row_items(b, all, false),
                 [&](const BItem* d, int k) { return launch_bprep(b->dinst, d, k, b->stream); }));
  B_TRY(run_list(b, all, launch_bnorms));
  B_TRY(run_rows(b, row_items(b, all, false), [&](const BItem* d, int k) {
    return launch_bg0(b->dinst, d, k, b->opt.g0_mode, 1, b->stream);
  }));
  int passes = 0;
  for (;;) {
    std::vector<int> act, nsact;
    for (int i = 0; i < count; ++i) {
      if (b->st[i].finished) continue;
      act.push_back(i);
      if (b->st[i].ns_active) nsact.push_back(i);
    }
    if (act.empty()) break;
    ++passes;
    B_TRY(run_rows(b, row_items(b, act, true),
                   [&](const BItem* d, int k) { return launch_bresid(b->dinst, d, k, b->stream); }));
    B_TRY(run_list(b, act, launch_brsq));
    if (!nsact.empty()) {
      B_TRY(launch_products(b, nsact, {0}));
      B_TRY(run_list(b, nsact, launch_bfrob));
    }
    B_TRY(sync_read(b));
    for (int i : act) decide(b, i, tol);
    // instances whose F must be formed again (precision switch / rollback)
    for (int guard = 0; guard < 4; ++guard) {
      std::vector<int> redo;
      for (int i : act)
        if (b->st[i].recompute && !b->st[i].finished) redo.push_back(i);
      if (redo.empty()) break;
      B_TRY(launch_products(b, redo, {0}));
      B_TRY(run_list(b, redo, launch_bfrob));
      B_TRY(sync_read(b));
      for (int i : redo) decide(b, i, tol);
    }
    // actions: next NS step (+ coupled sweep) or plain sweeps
    std::vector<int> step, upd;
    std::vector<int> gused(count, 0);
    for (int i : act) {
      InstState& s = b->st[i];
      if (s.finished) continue;
      if (s.ns_active) {
        step.push_back(i);
        upd.push_back(i);
        gused[i] = s.cur;
      } else if (s.sweeps_left > 0) {
        upd.push_back(i);
        gused[i] = s.cur;
        s.sweeps_left--;
      } else {
        s.finished = true;
        s.status = NS_NOT_CONVERGED;
      }
    }
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
    if (!upd.empty()) {
      std::vector<BItem> it = row_items(b, upd, true);
      for (BItem& x : it) x.cur = gused[x.inst];
      B_TRY(run_rows(b, it, [&](const BItem* d, int k) { return launch_bupdate(b->dinst, d, k, b->stream); }));
    }
    for (int i : upd) b->st[i].sweeps++;
    for (int i : step) {
      InstState& s = b->st[i];
      const double frob = s.frob_now;
      s.prev_ratio = (s.done > 0 && std::isfinite(s.prev_frob)) ? frob / s.prev_frob : INFINITY;
      s.prev_frob = frob;
      s.cur ^= 1;
      s.done++;
      if (s.done >= iters) s.ns_active = false;
    }
    if (passes > iters + b->opt.max_sweeps + 8) break;
  }
  B_CK(cudaStreamSynchronize(b->stream));
  int nconv = 0, nfail = 0;
  for (int i = 0; i < count; ++i) {
    if (b->st[i].converged)
      nconv++;
    else
      nfail++;
    if (!b->st[i].finished) b->st[i].status = NS_NOT_CONVERGED;
  }
  if (stats) {
    stats->passes = passes;
    stats->converged = nconv;
    stats->not_converged = nfail;
    stats->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    double useful = 0.0;
    for (int i = 0; i < count; ++i) useful += 2.0 * b->n[i] * static_cast<double>(b->n[i]) * b->n[i];
    stats->useful_flops_per_product = useful;
  }
  b->stats = nullptr;
  return nfail == 0 ? NS_OK : NS_NOT_CONVERGED;
}

ns_status ns_batch_result(const ns_batch* b, int i, int* status, int* ns_iters, int* sweeps, double* rel_res) {
  if (!b || i < 0 || i >= b->count) return NS_ERR_ARG;
  const InstState& s = b->st[i];
  if (status) *status = s.status;
  if (ns_iters) *ns_iters = s.done;
  if (sweeps) *sweeps = s.sweeps;
  if (rel_res) *rel_res = s.rel_res;
  return NS_OK;
}

}  // extern "C"
