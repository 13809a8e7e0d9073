/*
 * nsgb -- factorized high-order Newton-Schulz inversion of SPD matrices coupled
 * to Richardson iteration, on GB300 (sm_103a).
 *
 * The method is A. Stotsky, "Convergence Rate Improvement of Richardson and
 * Newton-Schulz Iterations" (arXiv 2008.11480):
 *   problem        A theta_* = b with A symmetric positive definite (Section 1, eq. ae1)
 *   G0             S^{-1} = alpha I (Section 2; default alpha = 1/||A||_F, option
 *                  alpha = 1/(||A||_inf/2 + eps))
 *   NS step        G_{k+1} = {sum_{j<n} F_k^j} G_k, error F_k = F_0^{n^k} (Section 3,
 *                  eqs. ns, fk1), evaluated in the factorized product form of Section 4
 *                  and Appendix Tables t1-t2: order 2^m as
 *                  G (I + F)(I + F^2)...(I + F^{2^{m-1}}), F = I - A G (2m products);
 *                  order 3 as G + G (F + F F) (3 products); or unfactorized (Horner).
 *   Richardson     theta_{k+1} = theta_k + G_k (b - A theta_k) (Section 6, eq. ttk1 with
 *                  the current inverse estimate as the gain).
 *
 * Conventions for every call below.
 *   - Matrices are row-major FP64, n x n (A, G) or n x nrhs (B, theta), contiguous.
 *   - Pointers may be device pointers (cudaMalloc / torch) or host pointers (pinned or
 *     pageable); host buffers are staged through the context's device workspace, so a
 *     host-pointer call includes the host<->device copies.
 *   - The caller owns every buffer it passes; the library never frees caller memory.
 *     The context owns its workspace (bf16 splits, f32 masters, residuals, scalars).
 *   - Calls run on the context's stream (ns_set_stream, default: the legacy default
 *     stream) and return after the stream has been synchronised, because the
 *     convergence controller reads norms on the host once per iteration.
 *   - Errors are return codes; no exception crosses the ABI.  ns_last_error() gives
 *     a one-line message for the last failing call on a context.
 *   - One context may not be used from two threads at once.
 */
#ifndef NSGB_H
#define NSGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns_ctx ns_ctx;

typedef enum ns_status {
  NS_OK = 0,
  NS_NOT_CONVERGED = 1,   /* soft: results are written, tolerance not met */
  NS_ERR_ARG = -1,        /* bad size, order, pointer or option */
  NS_ERR_CUDA = -2,       /* a CUDA runtime call failed (see ns_last_error) */
  NS_ERR_OOM = -3,        /* device workspace could not be allocated */
  NS_ERR_DIVERGED = -4,   /* ||F_k||_F grew past sqrt(n) + 1: no contraction */
  NS_ERR_TIMEOUT = -5,    /* a bounded device-side wait ran out; context stays usable */
  NS_ERR_NONFINITE = -6,  /* a norm became NaN or Inf */
  NS_ERR_UNSUPPORTED = -7 /* option combination not built */
} ns_status;

typedef enum ns_precision {
  NS_FP64 = 0,   /* every product in FP64 on the CUDA cores (plain path) */
  NS_TF32 = 1,   /* one pass of TF32 operands (binary32 rounded to nearest, ties away, to
                    10 stored significand bits), f32 accumulation (tcgen05 kind::tf32, CTA
                    pairs); between bf16 (8 bits) and bf16x3 (16) at 2x the bf16 cost */
  NS_BF16 = 2,   /* products hi*hi of bf16 operands, f32 accumulation (tcgen05) */
  NS_BF16X3 = 3, /* split bf16: hi*hi + hi*lo + lo*hi into one f32 accumulator */
  NS_BF16X6 = 4, /* three-part split hi, lo = bf16(x - hi), lo2 = bf16(x - hi - lo):
                    hi*hi + hi*lo + lo*hi + hi*lo2 + lo*lo + lo2*hi into one f32
                    accumulator (tcgen05 CTA pairs); not with composite rates or form 3 */
  NS_AUTO = 5,   /* bf16 while ||F_k||_F keeps falling, then bf16x3 (one-step rollback);
                    bf16x6 where bf16x3 stalls at a floor Richardson cannot finish from */
  NS_BF16X2 = 6  /* product form only (ns_k_gemm_bf16; the X_j P_j updates of bf16x3 steps
                    with option xp_bf16x2), not a solve precision: L split, R's hi part,
                    Lhi*Rhi + Llo*Rhi into one f32 accumulator (tcgen05 CTA pairs) */
} ns_precision;

typedef struct ns_options {
  int precision;       /* ns_precision; default NS_AUTO */
  int form;            /* 0 factorized (orders 3 and 2^m), 1 unfactorized Horner (any order),
                          2 the Appendix tool-kit (Tables t1-t3) for orders 2..19 (p + w + 1
                          products, +1 for the eq. ztab2 rows), 3 nested order 45 in ten
                          products (Section 4, eqs. ex1-ex3; order must be 45) */
  int pow_mode;        /* 0: F^{2^{j+1}} = F^{2^j} F^{2^j}; 1: F^{2^{j+1}} = I - A X_{j+1} (eq. ua1) */
  int g0_mode;         /* 0: alpha = 1/||A||_F; 1: alpha = 1/(||A||_inf/2 + 1e-8 ||A||_inf);
                          2: Jacobi, G0 = diag(A)^{-1} (Section 2, strictly diagonally dominant A;
                          single-system and batched / served paths) */
  int ns_stop;         /* 0: take exactly `iters` NS steps; 1: stop NS at the precision floor */
  double ns_stop_frob; /* with ns_stop = 1, also stop once ||F_k||_F <= this; default 0.02 */
  int max_sweeps;      /* Richardson-only sweeps allowed after NS stops; default 200 */
  int use_updated_G;   /* 1: theta_{k+1} = theta_k + G_{k+1} r_k (ordering of eq. ttk1) */
  int profile;         /* 1: time each GEMM launch with CUDA events (ns_stats.gemm_ms) */
  int gemm_bn;         /* 0: automatic; else 64, 128, 192 or 256 output columns per tile */
  double timeout_s;    /* bound on every device-side wait; default 2 s */
  int aux_ahead;       /* composite only: 1 starts the auxiliary loops one step ahead,
                          T_i = NS_{m_i}(G0), so rates = {n} gives the double Newton-Schulz
                          method of Section 5.1 (eqs. gamk11-fks1); 0: T_i start at G0 */
  int gemm_cluster;    /* product-kernel grouping: 0 automatic (CTA pairs wherever 256-column
                          tiles are chosen and ceil(n / 128) is even, else one CTA per tile);
                          1 one CTA per tile; -2 CTA pairs sharing each MMA (tcgen05
                          cta_group::2, 256 x 256 tiles) where they apply, else automatic.
                          Other values: NS_ERR_ARG */
  double couple_frob;  /* 0 (default): the Richardson branch (residual, test, update) runs on
                          every NS step, as in Section 6.  > 0: it starts with the first
                          G_k whose ||I - A G_k||_F <= couple_frob and stays on.  Earlier G_k
                          need not contract (rho(I - A G_k) may be ~1) and, with
                          F_k = F_0^{n^k}, the residual factor they contribute is negligible
                          next to the last step's.  1.0 skips exactly the sweeps without a
                          contraction bound (costs one extra device sync where it starts). */
  int accel_richardson; /* 1: accelerated Richardson of Section 6 (eq. ttk1 with q = n): while
                          Newton-Schulz runs, theta_k = theta_{k-1} + omega_k r with
                          omega_k = L_k + Gamma_k^n {sum_{j<n} F_k^j} G_k from the double
                          Newton-Schulz state (eqs. gamk11-fks1), so the error follows
                          (S^{-1}D)^{gamma_k} of eq. riem6; theta starts at L_0 b unless
                          Theta0 is given.  Needs rates = {order} and aux_ahead = 1 (the
                          double NS method); ns_create returns NS_ERR_ARG otherwise.  omega_k r
                          is applied as u = X_k r, u += L_k (r - A u) without forming omega_k.
                          2: the same iterates by the recursive schedule of Section 6.2 (eqs.
                          redttk1, redttk2, gkrecu1): omega_k is formed as a matrix (one product),
                          Q = sum_{j<n} Gamma^j from Gamma = Gamma_k^n (factorized for orders 2^m,
                          else Horner), then G_{k+1} = Q (omega_k - SG_k) + SG_k and L_{k+1} =
                          Q L_k in one grouped launch, Gamma_{k+1}^n = I - L_{k+1} A; theta +=
                          omega_k r is one pass over omega_k (cheaper for many right-hand sides).
                          Other values: NS_ERR_ARG. */
  int g0_order;         /* 0 or 1: G0 = S^{-1} (g0_mode); h = 2..19: the initial series of Section 3
                          (eq. g01), G0 = {sum_{j<h} (S^{-1}D)^j} S^{-1}, by one tool-kit step of
                          order h from S^{-1} (bf16x3 products on the mixed path) */
  int final_check;      /* after ns_invert / ns_richardson_solve: 0 (default) none; -1 ||I - A G||_F of
                          the final G by one FP64 product; s = 1..4096 Hutchinson's estimate with s
                          Rademacher probes and seed 0 (see ns_inverse_residual); -2 the FP64
                          product for n <= 4096 and 8 probes above; into
                          ns_stats.final_frob.  On the mixed path G is the f32 master, widened. */
  int fp64_slices;      /* 0 (default): FP64 products on the CUDA cores.  s = 2..7: FP64-accurate
                          products on the bf16 tensor cores from s signed digits of 8 bits per
                          operand (see ns_k_gemm_oz; 7 covers binary64) -- for precision NS_FP64,
                          and with NS_AUTO (no composite rates) for a solve the binary32 masters
                          cannot finish: where bf16x3 leaves the contraction region, or stalls
                          above ||F||_F = 1 and the Richardson sweeps from its best G then give
                          up, the FP64 path continues Newton-Schulz from the last contracting G
                          with these products (theta from theta0); after NS_NOT_CONVERGED or
                          divergence otherwise it starts over on the FP64 path from G0.
                          ns_batch_solve: every system the batch did not converge is solved
                          again alone by that AUTO path (ns_batch_stats.slice_retried) */
  int fp64_slices_early; /* slices of the products while ||F_k||_F >= 1 (their error is corrected
                          by the later steps); the full fp64_slices take over below one or at
                          the reduced count's floor.  Default 4; 0: always fp64_slices */
  int pow_bf16;         /* 0: the powers F^{2^{j+1}} = F^{2^j} F^{2^j} of a factorized step run
                          in the step's precision.  1: in bf16x3 steps they run as one bf16
                          pass, in their own launch (their error reaches G_{k+1} only through
                          X P, quadratic in F_k); pow_mode 0 only.  2 (default of
                          ns_default_options): 1 where n >= 4096, else 0 */
  int tf32_rung;        /* NS_AUTO: 1 puts TF32 products between bf16 and bf16x3 (bf16 until its
                          contraction worsens, then TF32 until TF32's does, then bf16x3); 0
                          (default) goes from bf16 straight to bf16x3 */
  int fp64_slices_pow;  /* slice products (fp64_slices): digits of the powers F^{2^{j+1}} =
                          F^{2^j} F^{2^j} of a factorized step, 2..7; 0 (default): the step's.
                          Their error reaches F_{k+1} through A X ~ I, not amplified by kappa */
  int batch_fused;      /* batched solves (ns_batch_solve): 1 (default of ns_default_options) runs
                          a batch whose systems all have n <= 256 as one persistent launch, one
                          CTA per system solving it whole (same arithmetic and controller as the
                          pass-by-pass path, so the same results); 0 always runs pass by pass
                          (one launch per product level and one host decision per pass) */
  int xp_bf16x2;        /* bf16x3 steps of the factorized chain: the updates X_j P_j with j >= 1
                          as NS_BF16X2 products (P_j's low part dropped: its error reaches
                          F_{k+1} only through A X_j ~ I, as ~2^-9 |F_k|^(2^j)).  0 (default of
                          ns_default_options): three terms; 1: on; 2: on where n >= 4096 */
} ns_options;

#define NS_MAX_HIST 256

typedef struct ns_stats {
  int status;                        /* ns_status of the call */
  int ns_iters;                      /* accepted Newton-Schulz steps */
  int sweeps;                        /* Richardson updates applied */
  int rollbacks;                     /* rejected bf16 steps redone in bf16x3 */
  int n_frob;                        /* entries in frob_F / prec_hist */
  int n_res;                         /* entries in rel_res_hist */
  double rel_res;                    /* last max_c ||b_c - A theta_c|| / ||b_c|| */
  double frob_F[NS_MAX_HIST];        /* ||F_k||_F, F_k = I - A G_k, per computed F */
  int prec_hist[NS_MAX_HIST];        /* precision used for that F and step */
  double rel_res_hist[NS_MAX_HIST];  /* relative residual before each update */
  long long gemm_launches;           /* GEMM kernel launches */
  long long kernel_launches;         /* all kernel launches of the call */
  double gemm_flops;                 /* executed products: sum of 2 M N K per bf16 pass / fp64 */
  double gemm_ms;                    /* summed GEMM durations (profile = 1) */
  double tc_gemm_ms;                 /* ... of tcgen05 launches only */
  long long tc_gemm_launches;
  double tc_gemm_flops;
  double wall_ms;                    /* host wall time of the call */
  double final_frob;                 /* ||I - A G||_F of the final G in FP64 (option final_check);
                                        -1 when not computed */
  double tc_gemm_alg_flops;          /* algorithmic work of the tcgen05 launches: 2 M N K per
                                        product, whatever its passes (bf16x3 counts once) */
  double slice_pair_flops;           /* slice products: 2 M N K per digit pair run (s digits:
                                        s (s + 1) / 2 pairs per product) */
} ns_stats;

/* Fill *opt with the defaults documented in ns_options. */
void ns_default_options(ns_options* opt);

/* Create a context for n x n systems (paper: A theta = b, Section 1, eq. ae1).
 *   order   Newton-Schulz order n of eq. ns: 2, 3, 4, 8, 16 (factorized) or any
 *           order >= 2 with form = 1.
 *   rates   composite mixed-rate orders m_i of eqs. gkgen1-ga1 (Section 5): n_rates
 *           auxiliary expansions T_i with x_i = m_i^k; n_rates = 0 for plain NS.
 *   opt     NULL for defaults.
 * Errors: NS_ERR_ARG (n <= 0 or n > 2^20, order < 2, order not factorizable with form = 0,
 * n_rates < 0 or a rate < 1, an option outside its documented range),
 * NS_ERR_UNSUPPORTED (NS_BF16X6 with composite rates or form 3), NS_ERR_CUDA (no
 * device), NS_ERR_OOM.  On success *out
 * owns the workspace (about 14 n^2 bytes for NS_FP64 plus 32 n^2 for mixed precision,
 * allocated on first use). */
ns_status ns_create(int64_t n, int order, const int* rates, int n_rates, const ns_options* opt, ns_ctx** out);

/* Release the context and its workspace.  NULL is accepted. */
ns_status ns_destroy(ns_ctx* ctx);

/* Run subsequent calls on `cuda_stream` (a cudaStream_t; NULL = legacy default). */
ns_status ns_set_stream(ns_ctx* ctx, void* cuda_stream);

/* Newton-Schulz inversion (Section 3, eqs. ns, fk1; factorized per Section 4).
 *   A      n x n SPD (read only).
 *   G0     n x n initial estimate, or NULL for alpha I (Section 2).
 *   iters  number of NS steps (a cap when opt.ns_stop = 1).
 *   G_out  n x n result (FP64; from the f32 master on the mixed-precision paths),
 *          or NULL to keep it resident in the context only.
 *   st     optional statistics.
 * Returns NS_OK, or an error above. */
ns_status ns_invert(ns_ctx* ctx, const double* A, const double* G0, int iters, double* G_out, ns_stats* st);

/* Newton-Schulz coupled to Richardson iteration for A Theta = B (nrhs columns).
 * Each pass forms R = B - A Theta in FP64 and its relative residual
 * max_c ||R_c|| / ||B_c||; the call stops once that is <= tol (tol <= 0: never).
 * While fewer than `iters` NS steps were taken (and the precision floor is not
 * reached when opt.ns_stop = 1) it applies Theta += G_k R and advances
 * G_{k+1} = NS(G_k); afterwards up to opt.max_sweeps updates Theta += G R.
 *   Theta0     n x nrhs start, or NULL for zero.
 *   Theta_out  n x nrhs result (may alias Theta0).
 * Returns NS_OK when tol was met, NS_NOT_CONVERGED when it was not (results
 * written), or an error. */
ns_status ns_richardson_solve(ns_ctx* ctx, const double* A, const double* B, int nrhs, const double* Theta0,
                              int iters, double tol, double* Theta_out, ns_stats* st);

/* Relative residuals rel_res_out[c] = ||B_c - A Theta_c||_2 / ||B_c||_2 in FP64
 * (the parameter-estimation error of eq. ttk1 measured through A). */
ns_status ns_residual(ns_ctx* ctx, const double* A, const double* Theta, const double* B, int nrhs,
                      double* rel_res_out);

/* Final check of an inverse estimate (precision control): ||I - A G||_F in FP64 for n x n A and
 * G (row-major FP64, lda = ldg = n, device or host; the context's n).
 *   probes = 0: I - A G formed by one FP64 product (2 n^3 flop) with its sum of squares.
 *   probes = s > 0: Hutchinson's estimate sqrt((1/s) sum_j ||z_j - A (G z_j)||^2) over s
 *   Rademacher probes (two FP64 products n x n x s): unbiased for ||I - A G||_F^2, exact when
 *   I - A G is diagonal.  Probe entry (i, j) is -1 when the top bit of SplitMix64 output
 *   k = j n + i from state `seed` is set, else +1; SplitMix64 (Steele, Lea, Flood 2014):
 *   output k = mix(seed + (k + 1) * 0x9E3779B97F4A7C15), mix(z): z ^= z >> 30,
 *   z *= 0xBF58476D1CE4E5B9, z ^= z >> 27, z *= 0x94D049BB133111EB, z ^= z >> 31.
 * *frob_out (host) receives the value.  Workspace (n^2 or 3 n s doubles) is taken per call
 * from the stream-ordered allocator; the context's stream is synchronised.
 * Errors: NS_ERR_ARG (null pointer, probes < 0 or > 4096), NS_ERR_OOM, NS_ERR_CUDA. */
ns_status ns_inverse_residual(ns_ctx* ctx, const double* A, const double* G, int probes,
                              unsigned long long seed, double* frob_out);

/* Message for the last failing call on ctx ("" if none).  NULL: the last failure of a
 * single-kernel entry point (ns_k_gemm_oz) on the calling host thread. */
const char* ns_last_error(const ns_ctx* ctx);
const char* ns_status_string(ns_status s);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent SPD systems A_i theta_i = B_i of uneven size
 * advanced together, each by the method of ns_richardson_solve (factorized order
 * 2^m or 3, precision controller per instance, split-f32 Richardson).  Each pass
 * issues one list-driven tensor-core launch per product level (per tile width
 * and precision) for all instances, and one launch per batched row kernel.
 * An instance's arithmetic does not depend on the other instances (tile width
 * from its own size, fixed-order reductions inside its own blocks), so its
 * result is bitwise the same alone or in any mix.
 * ------------------------------------------------------------------------- */
typedef struct ns_batch ns_batch;

typedef struct ns_batch_stats {
  int passes;                       /* controller passes (one device sync each) */
  int converged;                    /* instances that met tol */
  int not_converged;                /* instances that did not (diverged, floor, budget) */
  long long gemm_launches;
  long long kernel_launches;
  double gemm_flops;                /* executed: 2 n^3 per product pass (bf16x3 = 3 passes) */
  double gemm_ms;                   /* summed product-launch durations (opt.profile = 1) */
  double useful_flops_per_product;  /* sum over instances of 2 n_i^3 */
  double wall_ms;
  double gemm_bytes;                /* algorithmic HBM bytes of the products: operands once
                                       (hi, or hi and lo), C term, outputs */
  int fused;                        /* 1: the batch ran as one fused launch (opt.batch_fused) */
  int fused_pad;
  double fused_ms;                  /* duration of that launch (opt.profile = 1), else 0 */
  double useful_flops;              /* fused launch: sum over systems of their products x 2 n^3 */
  int slice_retried;                /* option fp64_slices: systems solved again alone (slice path) */
  int slice_retried_converged;      /* ... of which converged */
  double slice_retry_ms;            /* host wall time of those solves */
} ns_batch_stats;

/* Create a batch of `count` systems; n[i] in [1, 16384], nrhs[i] in [1, 1024].
 * order: 3 or a power of two.  opt: precision NS_AUTO, NS_BF16 or NS_BF16X3,
 * form 0, pow_mode 0, g0_mode 0..2, g0_order 0 (others return NS_ERR_UNSUPPORTED).  Allocates all workspace
 * (one device allocation) and the per-instance product descriptors. */
ns_status ns_batch_create(int count, const int64_t* n, const int* nrhs, int order, const ns_options* opt,
                          ns_batch** out);
ns_status ns_batch_destroy(ns_batch* b);
ns_status ns_batch_set_stream(ns_batch* b, void* cuda_stream);
const char* ns_batch_last_error(const ns_batch* b);

/* Solve all systems from Theta = 0.  A[i] (n_i x n_i), B[i] (n_i x nrhs_i) and
 * Theta[i] (n_i x nrhs_i, output) are DEVICE pointers, row-major FP64; the
 * arrays of pointers are host arrays.  iters caps the NS steps per instance;
 * tol the relative residual.  Returns NS_OK when every instance met tol,
 * NS_NOT_CONVERGED otherwise (per-instance status via ns_batch_result), or an
 * error for the whole call. */
ns_status ns_batch_solve(ns_batch* b, const double* const* A, const double* const* B, double* const* Theta,
                         int iters, double tol, ns_batch_stats* stats);

/* Per-instance outcome of the last ns_batch_solve. */
ns_status ns_batch_result(const ns_batch* b, int i, int* status, int* ns_iters, int* sweeps, double* rel_res);

/* ---------------------------------------------------------------------------
 * Continuous-batching server.  Requests (independent SPD systems, each solved
 * by the method of ns_batch_solve) join and leave between scheduling ticks.
 * A tick (1) admits queued requests first come, first served while a request
 * slot is free and its workspace fits the memory budget (first-fit arena,
 * zeroed on admission), copying A and B into the slot; (2) runs ONE
 * controller pass over every request on the device: its residual, and while
 * its Newton-Schulz loop runs, F = I - A G, then its Richardson update and
 * next product chain, with the launches of the batched solve; (3) retires each
 * finished request on its own (theta copied to the caller's buffer; the
 * request is reported done once that copy has landed).  A request's
 * arithmetic is that of the same system solved alone (own tile width, own
 * fixed-order reductions), so its theta is bitwise independent of the mix.
 * The paper has no serving loop; this is the batched path run continuously.
 * ------------------------------------------------------------------------- */
typedef struct ns_server ns_server;

typedef struct ns_request {
  int64_t n;            /* system size, 1..16384 */
  int nrhs;             /* 1..max_nrhs of the server */
  int iters;            /* cap on Newton-Schulz steps */
  double tol;           /* relative residual target (max over right-hand sides) */
  const double* A;      /* n x n row-major FP64, host (pinned or pageable) or device */
  const double* B;      /* n x nrhs row-major FP64 */
  double* Theta;        /* n x nrhs output; written when the request is done */
} ns_request;           /* A, B and Theta stay owned by the caller and valid until done */

typedef struct ns_result {
  int status;           /* NS_OK converged, NS_NOT_CONVERGED, NS_ERR_DIVERGED / NONFINITE, NS_ERR_OOM (never fits) */
  int done;             /* 1 once Theta holds the result */
  int ns_iters;
  int sweeps;
  double rel_res;       /* last measured max_c ||B_c - A theta_c|| / ||B_c|| */
  double queue_ms;      /* submit -> admission */
  double latency_ms;    /* submit -> done */
} ns_result;

typedef struct ns_server_stats {
  long long submitted, admitted, completed, converged, rejected;
  long long ticks, passes;
  int active;           /* requests holding a slot after the last tick */
  int queued;           /* requests waiting for admission */
  int last_error;       /* error of the background thread (0 if none) */
  long long gemm_launches;   /* tensor-core product launches so far */
  long long kernel_launches; /* all kernel launches so far */
  double gemm_flops;         /* product flops so far (2 n^3 per product; bf16x3 = 3 passes) */
  double tick_ms;            /* host time spent inside ticks */
  double wait_ms;            /* ... of which blocked waiting for the device */
} ns_server_stats;

/* mem_budget_bytes: device arena for request workspaces (slot footprint of a
 * request about 68 ld^2 + 36 ld nrhs bytes, ld = n rounded up to 64); tables
 * and staging are allocated beside it.  max_requests: slots.
 * order and opt as for ns_batch_create.  The server owns a non-blocking stream. */
ns_status ns_server_create(size_t mem_budget_bytes, int max_requests, int max_nrhs, int order,
                           const ns_options* opt, ns_server** out);
/* Stops the background thread (after the queue drains) and frees everything. */
ns_status ns_server_destroy(ns_server* srv);
ns_status ns_server_set_stream(ns_server* srv, void* cuda_stream /* NULL: the server's own */);
const char* ns_server_last_error(const ns_server* srv);
/* Thread-safe.  Device buffers must hold their data when submit is called. */
ns_status ns_server_submit(ns_server* srv, const ns_request* req, uint64_t* ticket);
/* Non-blocking, thread-safe.  NS_ERR_ARG for an unknown ticket. */
ns_status ns_server_poll(ns_server* srv, uint64_t ticket, ns_result* out);
/* Forget a finished request's record (NS_ERR_ARG if not done). */
ns_status ns_server_release(ns_server* srv, uint64_t ticket);
/* One scheduling tick on the calling thread (synchronises the stream once
 * per pass).  *active = requests holding a slot afterwards. */
ns_status ns_server_tick(ns_server* srv, int* active);
/* Run ticks on a background thread until ns_server_stop (which waits for
 * every submitted request to finish).  Do not call ns_server_tick meanwhile. */
ns_status ns_server_start(ns_server* srv);
ns_status ns_server_stop(ns_server* srv);
ns_status ns_server_get_stats(ns_server* srv, ns_server_stats* out);

/* ---------------------------------------------------------------------------
 * Single-kernel entry points.  Device pointers only; `stream` is a cudaStream_t
 * (NULL = legacy default).  Each returns after launching, without synchronising,
 * except where a result is returned through a host pointer.  Scratch memory they
 * need is allocated stream-ordered (cudaMallocAsync) and freed after use.
 * ------------------------------------------------------------------------- */

/* Split X (rows x cols, leading dimension ldx; x_dtype 0 = FP64, 1 = FP32) into
 * bf16 hi = RN(RN32(x)) and lo = RN(RN32(x) - hi) with leading dimension ld
 * (a multiple of 8).  This is the operand format of the tensor-core products. */
ns_status ns_k_split(const void* X, int x_dtype, int64_t rows, int64_t cols, int64_t ldx, void* hi, void* lo,
                     int64_t ld, void* stream);

/* Tensor-core product with the Newton-Schulz epilogue (Section 4 factor products).
 * Synchronises `stream` before returning, to read the kernel's error word:
 *   D = s * P + beta * C + gamma * I,  P = Lhi Rhi            (precision NS_BF16)
 *                                     P = Lhi Rhi + Lhi Rlo + Llo Rhi (NS_BF16X3)
 * L is M x K (ldl), R is K x N (ldr), bf16 splits from ns_k_split; C (f32, ldc) may
 * be NULL.  Outputs (each may be NULL): D32 f32 (ldd32), Dhi/Dlo bf16 split of D
 * (ldd16), frob_out a device double receiving sum(D^2).  Leading dimensions of bf16
 * arrays must be multiples of 8 and of f32 arrays multiples of 4; base pointers
 * 16-byte aligned.  bn = 0 picks the tile width (64, 128, 192 or 256 columns);
 * cluster_m: 1 runs one CTA per tile; -2 runs CTA pairs that share each MMA (tcgen05
 * cta_group::2, 256 x 256 tiles: bn must be 0 or 256 and ceil(M / 128) even); 0 picks
 * CTA pairs where they apply (bn = 256, ceil(M / 128) even), else one CTA per tile.
 * Other values, and violations of the rules above, return NS_ERR_ARG. */
ns_status ns_k_gemm_bf16(int precision, int64_t M, int64_t N, int64_t K, const void* Lhi, const void* Llo,
                         int64_t ldl, const void* Rhi, const void* Rlo, int64_t ldr, float s, const float* C,
                         int64_t ldc, float beta, float gamma, float* D32, int64_t ldd32, void* Dhi, void* Dlo,
                         int64_t ldd16, double* frob_out, int bn, int cluster_m, void* stream);

/* Three-part bf16 split for bf16x6 products: x32 = binary32 rounding of X (FP64, x_dtype 0)
 * or X itself (f32, x_dtype 1), hi = bf16(x32), lo = bf16(x32 - hi), lo2 = bf16(x32 - hi -
 * lo), each rounded to nearest even; every difference is exact in binary32, so x32 = hi +
 * lo + lo2.  Layouts and errors as ns_k_split (lo2 must not be NULL). */
ns_status ns_k_split3(const void* X, int x_dtype, int64_t rows, int64_t cols, int64_t ldx, void* hi, void* lo,
                      void* lo2, int64_t ld, void* stream);

/* Split-bf16 x6 product on tcgen05 CTA pairs (256 x 256 tiles), same epilogue as
 * ns_k_gemm_bf16:
 *   D = s * P + beta * C + gamma * I,
 *   P = Lhi Rhi + Lhi Rlo + Llo Rhi + Lhi Rlo2 + Llo Rlo + Llo2 Rhi   (f32 accumulation)
 * L[3] and R[3] are host arrays of the device parts {hi, lo, lo2} from ns_k_split3 (M x K,
 * ldl; K x N, ldr; multiples of 8 elements, 16-byte aligned).  D is NULL or a host array
 * {Dhi, Dlo, Dlo2} of optional outputs (ldd16): the three-part split of D (a part may be
 * NULL only when the later ones are).  Any M (an odd number of 128-row tiles is allowed).
 * Synchronises `stream`.  Errors: NS_ERR_ARG, NS_ERR_OOM, NS_ERR_CUDA, NS_ERR_TIMEOUT. */
ns_status ns_k_gemm_bf16x6(int64_t M, int64_t N, int64_t K, const void* const* L, int64_t ldl, const void* const* R,
                           int64_t ldr, float s, const float* C, int64_t ldc, float beta, float gamma, float* D32,
                           int64_t ldd32, void* const* D, int64_t ldd16, double* frob_out, void* stream);

/* TF32 tensor-core product (tcgen05 kind::tf32 on CTA pairs) with the Newton-Schulz
 * epilogue: D = s * RN_tf32(L) RN_tf32(R) + beta C + gamma I, L (M x K, ldl) and R
 * (K x N, ldr) f32 on the device, rounded to TF32 (nearest, ties away from zero) into
 * scratch taken from the stream-ordered allocator (L row-major, R transposed: both
 * operands K-major), f32 accumulation.  Outputs (each may be NULL): D32 (ldd32), the
 * TF32 forms of D row-major (Dt) and transposed (DtT, column j at DtT + j ldt; ldt >=
 * max(M, N)), frob_out a device double receiving sum(D^2).  Pointers 16-byte aligned,
 * f32 leading dimensions multiples of 4; `stream` is synchronised.  Errors:
 * NS_ERR_ARG, NS_ERR_OOM, NS_ERR_CUDA, NS_ERR_TIMEOUT. */
ns_status ns_k_gemm_tf32(int64_t M, int64_t N, int64_t K, const float* L, int64_t ldl, const float* R, int64_t ldr,
                         float s, const float* C, int64_t ldc, float beta, float gamma, float* D32, int64_t ldd32,
                         float* Dt, float* DtT, int64_t ldt, double* frob_out, void* stream);

/* FP64-accurate product on the bf16 tensor cores by an Ozaki-style error-free splitting
 * (Ozaki, Ogita, Rump, Oishi, Numer. Algorithms 59, 2012), with signed digits:
 *   D = s L R + beta C + gamma I   (L M x K, R K x N, C and D M x N: FP64, row-major)
 * Each row i of L is scaled by the power of two mu_i > max_k |L_ik| and L_ik / (2 mu_i),
 * in (-1/2, 1/2), is cut into `slices` digits a_t = RN(256 x), x <- 256 x - a_t (|a_t| <= 128,
 * exact in bf16); each column of R likewise (lines whose largest magnitude is below 2^-1000
 * are taken as zero).  The digit products of level d = t + u <= slices + 1 run on tcgen05
 * CTA pairs, summed exactly in f32 over chunks of 1024 / (d - 1) of K and in int32 over
 * K; D = s (2 mu)(2 nu) sum_d 256^-d S_d + beta C + gamma I is then formed once per element
 * (levels 2..5 and 6..s+1 exactly in int64, then binary64).  slices = 7 carries 56 bits per
 * line (binary64: 53).  K is taken in blocks of at most 16384.  Workspace (slices x (2 M +
 * 2 N) x min(K, 16384) + 4 M N slices bytes and a few vectors) is taken from the
 * stream-ordered allocator; `stream` is synchronised.  frob_out (device double, may be NULL)
 * receives sum(D^2).  D may alias C, and L or R when K <= 16384.
 * Errors: NS_ERR_ARG (sizes, leading dimensions, null pointers, slices outside 2..7, D
 * aliasing L or R with K > 16384), NS_ERR_OOM, NS_ERR_CUDA, NS_ERR_TIMEOUT. */
ns_status ns_k_gemm_oz(int64_t M, int64_t N, int64_t K, const double* L, int64_t ldl, const double* R, int64_t ldr,
                       double s, const double* C, int64_t ldc, double beta, double gamma, double* D, int64_t ldd,
                       int slices, double* frob_out, void* stream);

/* FP64 product with the same epilogue: D = s L R + beta C + gamma I (C may be NULL). */
ns_status ns_k_gemm_f64(int64_t M, int64_t N, int64_t K, const double* L, int64_t ldl, const double* R,
                        int64_t ldr, double s, const double* C, int64_t ldc, double beta, double gamma, double* D,
                        int64_t ldd, double* frob_out, void* stream);

/* Richardson residual R = B - A Theta (n x nrhs, FP64); rsq_out (device, nrhs
 * doubles, may be NULL) receives ||R_c||^2. */
ns_status ns_k_resid(const double* A, int64_t lda, const double* Theta, const double* B, double* R, int64_t n,
                     int nrhs, double* rsq_out, void* stream);

/* Richardson update Theta += G R; G is f32 (g_dtype 1) or FP64 (g_dtype 0) with
 * leading dimension ldg. */
ns_status ns_k_update(const void* G, int g_dtype, int64_t ldg, const double* R, double* Theta, int64_t n, int nrhs,
                      void* stream);

/* One fused pass over A (FP64, n x n, leading dimension lda) that prepares every
 * mixed-precision operand: the bf16 hi/lo split of each element (as ns_k_split,
 * leading dimension ld, a multiple of 8), its two f32 limbs a1 = RN32(a),
 * a2 = RN32(a - a1) (leading dimension ld), and, when non-NULL, the device doubles
 * ss_out[0] = sum a_ij^2 (for G0 = I/||A||_F, Section 2) and
 * rowabs_out[0] = max_i sum_j |a_ij| (= ||A||_inf, Section 2). */
ns_status ns_k_prep_a(const double* A, int64_t lda, int64_t n, void* hi, void* lo, float* a1, float* a2,
                      int64_t ld, double* ss_out, double* rowabs_out, void* stream);

/* Richardson residual R = B - A Theta (FP64 result) evaluated from A's f32 limbs
 * (a1, a2 from ns_k_prep_a; ld a multiple of 4, 16-byte aligned) and Theta's limbs,
 * with exact f32 products and paired-f32 accumulation: each row sum carries about
 * 48 significant bits, the accuracy of an FP64 GEMV at these sizes.  rsq_out
 * (device, nrhs doubles, may be NULL) receives ||R_c||^2.  This is the residual the
 * mixed-precision solve uses (FP64 arithmetic is rate-limited on GB300). */
ns_status ns_k_resid_x2(const float* a1, const float* a2, int64_t ld, const double* Theta, const double* B,
                        double* R, int64_t n, int nrhs, double* rsq_out, void* stream);

/* Same computation as ns_k_resid, but it allocates nothing: for callers that cannot
 * allocate device memory at call time (a serving loop whose device memory is all
 * reserved up front by its admission budget, a latency-critical loop that must not
 * enter the allocator, which can synchronise the device, or a process that forbids
 * allocation after start-up).  The paper has no counterpart; this is an interface
 * convenience.
 *   - Its scratch (partial sums of ||R_c||^2) is one fixed 256 KiB device array that
 *     every GPU which loads the library keeps until the process exits.
 *   - Limits: n <= 32768 and nrhs <= 16; larger sizes return NS_ERR_ARG.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call before
 *     any stream capture.
 *   - All calls share the array, which keeps the last call's contents (nothing in it
 *     needs to start at zero).  Calls whose work overlaps on the GPU (different
 *     streams, or different host threads on one device) race on it: serialise them.
 * Returns NS_OK, NS_ERR_ARG, or NS_ERR_CUDA. */
ns_status ns_k_resid_noalloc(const double* A, int64_t lda, const double* Theta, const double* B, double* R,
                             int64_t n, int nrhs, double* rsq_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NSGB_H */
