"""Benchmark: SPD solves/s at relative residual <= 1e-10, mixed precision
against the plain FP64 method, on one GB300.

Default workload (the metric's largest single-GPU configuration): the
least-squares Gram system n = 16384, A = X^T X with cond(A) = 1e6 (X = U
diag(sigma) V^T, sigma log-uniform in [1e-3, 1]), b = X^T y, order-8
factorized Newton-Schulz coupled to FP64 Richardson.  Products run in bf16,
then bf16x3, and where binary32 masters stop contracting, FP64-accurate
4-digit slice products on the bf16 tensor cores continue from the last
contracting G.  The dense n = 4096 system (kappa = 1e4, 4 RHS) is measured
beside it (variants.dense_n4096; --workload dense makes it the line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete solve from the system alone (norms, splits, G0, every
NS step and Richardson sweep until the residual test passes), inputs resident
in HBM.  512 MiB is written between timed steps, outside the timed events.
Under torchrun each rank solves its own system (independent replicas; the
problem does not shard without an exchange per product).  Rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SPD solves/s at rel. residual ≤1e-10 vs plain FP64 NS on GB300; p50/p99 latency"
UNIT = "solves/s"


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def workload_config(a):
    return {
        "workload": f"dense SPD n={a.n} kappa={a.kappa:g} nrhs={a.nrhs}: A = Q diag(lambda) Q^T, Q Haar, "
                    f"lambda log-uniform in [1, kappa]; B ~ N(0,1)",
        "n": a.n, "kappa": a.kappa, "nrhs": a.nrhs, "order": a.order, "form": "factorized",
        "precision": "auto: bf16 products while ||F||_F falls, then bf16x3; f32 accumulate; FP64 residual "
                     "and Richardson",
        "tol": 1e-10, "l2": "flushed between timed steps (512 MiB write)", "seed": 1,
        "couple_frob": a.couple,
        **({"gemm_cluster": a.gemm_cluster} if getattr(a, "gemm_cluster", 0) else {}),
        "pow_bf16": getattr(a, "pow_bf16", 2),
    }


def recorded_traffic(profile_name):
    """Per-launch DRAM bytes (read + write) of the product kernel recorded by one
    ncu capture, summarised in profiles/<profile_name>; None once any of the
    kernel sources listed there hashes differently from the capture's build."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile_name)).read()
        want = re.search(r"kernel_sources_sha256: ([0-9a-f]{64})", txt).group(1)
        nbytes = float(re.search(r"traffic_bytes_per_launch: ([0-9.eE+]+)", txt).group(1))
        files = re.search(r"kernel_sources: (.+)", txt).group(1).split()
        h = hashlib.sha256()
        for f in files:
            h.update(open(os.path.join(ROOT, f), "rb").read())
    except Exception:
        return None
    return nbytes if h.hexdigest() == want else None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks
# Batched and served systems are independent: under torchrun each rank takes a
# share of them (no data-path collective); only timings and counts are
# reduced, and rank 0 prints.
def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_balanced(costs, world):
    """Largest-first greedy split of units with the given costs over `world`
    ranks (deterministic, ties broken by index); one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(q) for q in parts]


def reduce_over_ranks(values, op, device="cpu"):
    """Element-wise max or sum of a list of floats over all ranks (identity
    without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.tolist()


def gather_lists(values):
    """Concatenation of every rank's list (all ranks receive it)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(values))
    return [v for part in out for v in part]


# ------------------------------------------------------------------ oracle (CPU) leg
def oracle_sample(a, ns_iters: int, sweeps: int, reps: int = 1):
    """Time the FP64 oracle as it stands on the host cores: one Newton-Schulz
    step of the configured order plus one Richardson sweep on the same system,
    and extrapolate to a whole solve with the given step / sweep counts."""
    import oracle as O
    from workloads import make_spd
    p = make_spd(a.n, a.kappa, nrhs=a.nrhs, seed=1)
    G = O.alpha_frobenius(p.A) * np.eye(a.n)
    theta = np.zeros_like(p.B)
    t_ns, t_sw = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        G1, _ = O.ns_step(p.A, G, a.order)
        t1 = time.perf_counter()
        O.richardson_step(p.A, p.B, theta, G1)
        t2 = time.perf_counter()
        t_ns.append(t1 - t0)
        t_sw.append(t2 - t1)
    tns, tsw = min(t_ns), min(t_sw)
    solve_s = ns_iters * tns + max(sweeps, ns_iters) * tsw
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one order-{a.order} NS step ({tns:.2f} s) + one Richardson sweep ({tsw:.3f} s) of the "
                      f"numpy FP64 oracle at n={a.n}, extrapolated to {ns_iters} NS steps + "
                      f"{max(sweeps, ns_iters)} sweeps (the FP64 GPU path's counts for this system)"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ns_iters, sweeps = a.ref_ns_iters, a.ref_sweeps
    for _ in range(a.warmup if a.warmup < 1 else 1):
        oracle_sample(a, ns_iters, sweeps)
    vals = []
    t0 = time.perf_counter()
    for _ in range(a.steps):
        vals.append(oracle_sample(a, ns_iters, sweeps))
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(a),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ the Gram system (default workload)
# Least-squares Gram system of the metric's largest single-GPU configuration:
# n = 16384, A = X^T X with cond(A) = 1e6, b = X^T y, order 8 factorized.
GRAM_SIGMA_LO, GRAM_SEED, GRAM_ORDER, GRAM_SLICES, GRAM_SLICES_POW, GRAM_XP = 1e-3, 5, 8, 4, 2, 2


def gram_xp(a):
    """Option xp_bf16x2 of the Gram line: the flag's value when given, else 2
    (two-term updates in bf16x3 steps: 5.8 % less time per solve on this
    system, measured interleaved, from higher clocks under the power cap)."""
    v = getattr(a, "xp_bf16x2", None)
    return GRAM_XP if v is None else v


def gram_config(a):
    n = a.gram_n
    return {
        "workload": f"least-squares Gram system n={n}: A = X^T X, b = X^T y for a {2 * n} x {n} design "
                    f"X = U diag(sigma) V^T, sigma log-uniform in [1e-3, 1] (cond(A) = 1e6), y ~ N(0,1); 1 RHS",
        "n": n, "kappa": 1e6, "nrhs": 1, "order": GRAM_ORDER, "form": "factorized (I+F)(I+F^2)(I+F^4)",
        "precision": "auto: bf16 products while ||F||_F falls, then bf16x3 (f32 accumulate; the updates "
                     "X_j P_j, j >= 1, as two terms hi(X)hi(P) + lo(X)hi(P)); at the binary32 "
                     "floor Richardson sweeps from the best G (FP64 residual); if they give up, the FP64 path with "
                     "4-digit slice products (bf16 tensor cores, exact integer accumulation; powers in 2 digits) "
                     "continues from that G",
        "tol": 1e-10, "l2": "inputs larger than L2 (A: 2 GiB FP64); 512 MiB written between timed steps",
        "seed": GRAM_SEED, "couple_frob": a.couple, "fp64_slices": GRAM_SLICES, "fp64_slices_early": 0,
        "fp64_slices_pow": GRAM_SLICES_POW, "xp_bf16x2": gram_xp(a)}


def plain_fp64_model(n, seed=GRAM_SEED, order=GRAM_ORDER, stop=0.02, tol=1e-10):
    """Work of the plain FP64 method on the Gram system, from its exact-arithmetic
    iterates: with G_0 = I / ||A||_F, F_k = (I - A/||A||_F)^{order^k}, so
    ||F_k||_F^2 = sum_i (1 - lambda_i / ||A||_F)^{2 order^k} over the generator's
    spectrum lambda = sigma^2.  Newton-Schulz runs until ||F_k||_F <= stop (the
    library's ns_stop_frob), 2 m products a step for order 2^m (the residual
    product included), then Richardson sweeps at the rate ||F_k||_F.
    Returns (steps, products, sweeps)."""
    from workloads import gram_spectrum
    sigma, _, _ = gram_spectrum(n, GRAM_SIGMA_LO, seed)
    lam = sigma ** 2
    le = np.log1p(-lam / np.sqrt(np.sum(lam * lam)))  # log(1 - alpha lambda) < 0
    k, frob = 0, float(np.sqrt(n))
    while frob > stop and k < 64:
        k += 1
        frob = float(np.sqrt(np.sum(np.exp(2.0 * order ** k * le))))
    m = int(round(np.log2(order)))
    sweeps = max(1, int(np.ceil(np.log(tol) / np.log(max(frob, 1e-300)))))
    return k, 2 * m * k, sweeps


def oracle_sample_gram(a, L, R, x):
    """Time the FP64 oracle as it stands on the host cores on a bounded piece of
    the Gram workload: one oracle product of a rows x n panel by an n x n
    matrix (the solve's products are n x n x n) and one matrix-vector product
    (a Richardson sweep is two), extrapolated with plain_fp64_model's counts."""
    import oracle as O
    rows, n = L.shape
    t0 = time.perf_counter()
    O.mm(L, R)
    t1 = time.perf_counter()
    R @ x
    t2 = time.perf_counter()
    t_prod = (t1 - t0) * n / rows
    t_sweep = 2.0 * (t2 - t1)
    k, prods, sweeps = plain_fp64_model(n)
    solve_s = prods * t_prod + sweeps * t_sweep
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one numpy FP64 oracle product of a {rows} x {n} panel by an {n} x {n} matrix "
                      f"({t1 - t0:.2f} s, scaled to n rows) and one matrix-vector product, extrapolated to the "
                      f"plain method's {prods} products ({k} order-{GRAM_ORDER} steps) + {sweeps} sweeps on this system"}


def gram_oracle_operands(n, rows):
    rng = np.random.default_rng(11)
    return rng.standard_normal((rows, n)), rng.standard_normal((n, n)), rng.standard_normal((n, 1))


def run_reference_gram(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    L, R, x = gram_oracle_operands(a.gram_n, a.ref_rows)
    for _ in range(min(a.warmup, 1)):
        oracle_sample_gram(a, L, R, x)
    vals = []
    t0 = time.perf_counter()
    for _ in range(a.steps):
        vals.append(oracle_sample_gram(a, L, R, x))
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": gram_config(a),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s": wall}
    print(json.dumps(line), flush=True)


def run_gram(a):
    """The default line: the n = 16384 Gram system (cond 1e6), one solve per step
    from the system alone to a verified relative residual <= 1e-10."""
    import torch
    import torch.distributed as dist

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_gram_device

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n = a.gram_n
    A, B, V, sg, z = make_gram_device(n, GRAM_SIGMA_LO, seed=GRAM_SEED + rank, device=dev, return_factors=True,
                                      qr_on_host=a.gram_qr_host)
    tstar = V @ (z / sg[:, None])
    del V
    out = torch.empty_like(B)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    opts = dict(order=GRAM_ORDER, stream=stream, couple_frob=a.couple, fp64_slices=GRAM_SLICES, fp64_slices_early=0,
                fp64_slices_pow=GRAM_SLICES_POW, xp_bf16x2=gram_xp(a))
    ctx = nsgb.Context(n, profile=1, **opts)
    for _ in range(max(3, a.warmup)):
        r = ctx.solve(A, B, iters=80, tol=1e-10, out=out)
    assert r.status == nsgb.NS_OK, f"solve did not converge: {r.stats.res_history()}"

    sampler = ClockSampler(local)
    step_ms, ns_it, sw = [], [], []
    acc = dict(tc_ms=0.0, tc_flops=0.0, tc_alg=0.0, tc_l=0, gemm_ms=0.0, gemm_l=0, launches=0, pair_flops=0.0)
    barrier()
    sampler.start()
    for _ in range(a.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ctx.solve(A, B, iters=80, tol=1e-10, out=out)
        e1.record(stream)
        e1.synchronize()
        assert r.status == nsgb.NS_OK
        step_ms.append(e0.elapsed_time(e1))
        st = r.stats
        acc["tc_ms"] += st.tc_gemm_ms
        acc["tc_flops"] += st.tc_gemm_flops
        acc["tc_alg"] += st.tc_gemm_alg_flops
        acc["tc_l"] += st.tc_gemm_launches
        acc["gemm_ms"] += st.gemm_ms
        acc["gemm_l"] += st.gemm_launches
        acc["launches"] += st.kernel_launches
        acc["pair_flops"] += st.slice_pair_flops
        ns_it.append(st.ns_iters)
        sw.append(st.sweeps)
    barrier()
    clocks = sampler.stop()
    rel = max(ctx.residual(A, out, B))
    th_err = float(torch.linalg.norm(out - tstar) / torch.linalg.norm(tstar))
    total_s = reduce_over_ranks([sum(step_ms) / 1e3], "max", dev)[0]
    value = world * a.steps / total_s

    # end to end through the same C-ABI call with host (pinned) buffers: the
    # host->device copy of A and b and the device->host copy of theta are
    # inside the timed region
    Ah = A.cpu().pin_memory()
    Bh = B.cpu().pin_memory()
    Th = torch.empty_like(Bh).pin_memory()
    ctx_h = nsgb.Context(n, **opts)
    ctx_h.solve(Ah, Bh, iters=80, tol=1e-10, out=Th)
    e2e_steps = max(1, min(a.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rh = ctx_h.solve(Ah, Bh, iters=80, tol=1e-10, out=Th)
        assert rh.status == nsgb.NS_OK
    torch.cuda.synchronize(dev)
    e2e_s = reduce_over_ranks([time.perf_counter() - t0], "max", dev)[0]
    ctx_h.close()
    del Ah
    e2e = {"value": world * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(n * n * 8 + Bh.numel() * 8), "d2h_bytes_per_step": int(Th.numel() * 8)}

    # the plain FP64 method on the GPU (CUDA-core FP64 products, FP64
    # Richardson), priced: one timed n^3 product x its product count
    fp64 = None
    if not a.no_fp64:
        D = torch.empty_like(A)
        nsgb.ns_k_gemm_f64(256, 256, 256, A, n, A, n, 1.0, None, 0, 0.0, 0.0, D, n, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nsgb.ns_k_gemm_f64(n, n, n, A, n, A, n, -1.0, None, 0, 0.0, 1.0, D, n, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t_prod = e0.elapsed_time(e1) / 1e3
        del D
        k, prods, sweeps = plain_fp64_model(n)
        est = prods * t_prod
        fp64 = {"value": 1.0 / est, "unit": UNIT, "ms_per_step": est * 1e3, "fp64_product_s": t_prod,
                "ns_iters": k, "products": prods, "sweeps": sweeps,
                "how": "one event-timed CUDA-core FP64 product (k_gemm_f64) x the plain method's products on this "
                       "system (its exact-arithmetic iterates; sweeps are negligible)",
                "speedup_of_mixed": value / max(world, 1) * est}

    # roofline of the dominant kernel by event-timed share: the tcgen05 bf16 /
    # bf16x3 products (k_gemm_tc2) or the slice products (k_gemm_oz with its
    # slicing and combine kernels).  achieved counts algorithmic work, 2 n^3
    # per product of the method whatever its passes or digit pairs
    pk, pk_kind = peaks()
    sus = pk["bf16_tflops_sustained"]
    f3 = 2.0 * float(n) ** 3
    oz_ms = acc["gemm_ms"] - acc["tc_ms"]
    oz_l = acc["gemm_l"] - acc["tc_l"]
    pairs = acc["pair_flops"] / (oz_l * f3) if oz_l else 0.0  # mean digit pairs per slice product
    kern = {
        "k_gemm_tc2": {"ms_per_step": acc["tc_ms"] / a.steps, "launches_per_step": acc["tc_l"] / a.steps,
                       "achieved_tflops": acc["tc_alg"] / (acc["tc_ms"] / 1e3) / 1e12 if acc["tc_ms"] else None,
                       "executed_tflops": acc["tc_flops"] / (acc["tc_ms"] / 1e3) / 1e12 if acc["tc_ms"] else None},
        "k_gemm_oz": {"ms_per_step": oz_ms / a.steps, "products_per_step": oz_l / a.steps, "digit_pairs_mean": pairs,
                      "achieved_tflops": oz_l * f3 / (oz_ms / 1e3) / 1e12 if oz_ms > 0 else None,
                      "executed_tflops": acc["pair_flops"] / (oz_ms / 1e3) / 1e12 if oz_ms > 0 else None,
                      "note": "time of the whole slice product: scales, digit slicing, level kernel, combine"}}
    dom = "k_gemm_oz" if oz_ms > acc["tc_ms"] else "k_gemm_tc2"
    kd = kern[dom]
    ach, exe = kd["achieved_tflops"], kd["executed_tflops"]
    roof = {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": sus, "unit": "TFLOP/s",
            "frac": ach / sus if ach else None,
            "peak_kind": f"bf16 dense sustained ({pk_kind}); kernel timed inside back-to-back solves; achieved and "
                         "frac count algorithmic flops (2 n^3 per product)",
            "executed": exe, "frac_executed": exe / sus if exe else None,
            "executed_note": "bf16 tensor work run: bf16x3 = 3 passes, an s-digit slice product = s (s + 1) / 2 digit "
                             "pairs",
            "traffic": recorded_traffic("traffic_k_gemm_oz_gram16384.md" if dom == "k_gemm_oz"
                                        else "traffic_k_gemm_tc2_gram16384.md"),
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "avg_launch_ms": (oz_ms / max(oz_l, 1)) if dom == "k_gemm_oz" else acc["tc_ms"] / max(acc["tc_l"], 1),
            "flops_per_launch": f3 if dom == "k_gemm_oz" else acc["tc_alg"] / max(acc["tc_l"], 1),
            "kernels": kern}
    variants = {}
    if world == 1 and not a.no_variants:
        try:
            variants["dense_n4096"] = dense_variant(a, dev, stream, flush)
        except Exception as ex:  # reported, never fatal to the headline line
            variants["dense_n4096"] = {"error": str(ex)[:300]}
    if rank == 0:
        cpu = None
        if not a.no_cpu:
            L, R, x = gram_oracle_operands(n, a.ref_rows)
            cpu = oracle_sample_gram(a, L, R, x)
            del L, R, x
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 / bf16x3 / bf16 digit slices (FP64-accurate); FP64 Richardson",
            "data": "synthetic", "config": gram_config(a),
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                           "min": srt[0], "max": srt[-1]},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(acc["launches"]), "roofline": roof,
            "cpu_baseline": cpu, "fp64_path": fp64, "verified_rel_res": rel, "theta_rel_err_vs_closed_form": th_err,
            "ns_iters": int(statistics.median(ns_it)), "sweeps": int(statistics.median(sw)),
            "prec_history": r.stats.prec_history(), "frob_history": [round(f, 4) for f in r.stats.frob_history()],
            **({"variants": variants} if variants else {}),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def dense_variant(a, dev, stream, flush):
    """The dense n = 4096 system (kappa = 1e4, 4 RHS, order 8), measured beside
    the headline on the same box: solves/s, the product kernels' algorithmic
    roofline fraction, and the plain FP64 method timed on the GPU."""
    import torch

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_spd
    n, kappa, nrhs = 4096, 1e4, 4
    p = make_spd(n, kappa, nrhs=nrhs, seed=1)
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    out = torch.empty_like(B)
    ctx = nsgb.Context(n, order=8, stream=stream, profile=1, couple_frob=a.couple, xp_bf16x2=a.xp_bf16x2 or 0)
    for _ in range(3):
        ctx.solve(A, B, iters=a.iters, tol=1e-10, out=out)
    ms, tc_ms, tc_alg, tc_fl, tc_l, it, sw = [], 0.0, 0.0, 0.0, 0, [], []
    for _ in range(max(1, min(a.steps, 20))):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ctx.solve(A, B, iters=a.iters, tol=1e-10, out=out)
        e1.record(stream)
        e1.synchronize()
        assert r.status == nsgb.NS_OK
        ms.append(e0.elapsed_time(e1))
        tc_ms += r.stats.tc_gemm_ms
        tc_alg += r.stats.tc_gemm_alg_flops
        tc_fl += r.stats.tc_gemm_flops
        tc_l += r.stats.tc_gemm_launches
        it.append(r.stats.ns_iters)
        sw.append(r.stats.sweeps)
    rel = max(ctx.residual(A, out, B))
    ctx.close()
    pk, pk_kind = peaks()
    sus = pk["bf16_tflops_sustained"]
    ach = tc_alg / (tc_ms / 1e3) / 1e12
    exe = tc_fl / (tc_ms / 1e3) / 1e12
    res = {"workload": "dense SPD n=4096 kappa=1e4 nrhs=4 (A = Q diag(lambda) Q^T, Q Haar, lambda log-uniform), "
                       "order 8 factorized, auto bf16/bf16x3, FP64 Richardson",
           "value": 1e3 / statistics.mean(ms), "unit": UNIT, "ms_per_step": statistics.mean(ms), "steps": len(ms),
           "verified_rel_res": rel, "ns_iters": int(statistics.median(it)), "sweeps": int(statistics.median(sw)),
           "roofline": {"bound": "tensor", "kernel": "k_gemm_tc2", "achieved": ach, "peak": sus, "unit": "TFLOP/s",
                        "frac": ach / sus, "executed": exe, "frac_executed": exe / sus,
                        "peak_kind": f"bf16 dense sustained ({pk_kind}); achieved counts 2 n^3 per product",
                        "traffic": recorded_traffic("traffic_k_gemm_tc2_dense_n4096.md"),
                        "traffic_unit": "bytes per launch (ncu dram read + write)",
                        "avg_launch_ms": tc_ms / max(tc_l, 1)}}
    if not a.no_fp64:
        with nsgb.Context(n, order=8, stream=stream, precision=nsgb.NS_FP64, couple_frob=a.couple, xp_bf16x2=a.xp_bf16x2 or 0) as c64:
            out64 = torch.empty_like(B)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r64 = c64.solve(A, B, iters=a.iters, tol=1e-10, out=out64)
            e1.record(stream)
            e1.synchronize()
            ms64 = e0.elapsed_time(e1)
        res["fp64_path"] = {"value": 1e3 / ms64, "ms_per_step": ms64, "status": int(r64.status),
                            "ns_iters": r64.stats.ns_iters, "sweeps": r64.stats.sweeps, "rel_res": r64.stats.rel_res,
                            "speedup_of_mixed": res["value"] / (1e3 / ms64)}
    return res


# ------------------------------------------------------------------ GPU leg
def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_spd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    p = make_spd(a.n, a.kappa, nrhs=a.nrhs, seed=1 + rank)
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    out = torch.empty_like(B)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    ctx = nsgb.Context(a.n, order=a.order, stream=stream, profile=1, couple_frob=a.couple,
                       gemm_cluster=a.gemm_cluster, pow_bf16=a.pow_bf16, xp_bf16x2=a.xp_bf16x2 or 0)
    for _ in range(max(3, a.warmup)):
        r = ctx.solve(A, B, iters=a.iters, tol=1e-10, out=out)
    assert r.status == nsgb.NS_OK, f"solve did not converge: {r.stats.res_history()}"

    sampler = ClockSampler(local)
    step_ms, tc_ms, tc_flops, tc_alg, tc_launch, launches, ns_it, sw = [], 0.0, 0.0, 0.0, 0, 0, [], []
    barrier()
    sampler.start()
    for _ in range(a.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ctx.solve(A, B, iters=a.iters, tol=1e-10, out=out)
        e1.record(stream)
        e1.synchronize()
        assert r.status == nsgb.NS_OK
        step_ms.append(e0.elapsed_time(e1))
        st = r.stats
        tc_ms += st.tc_gemm_ms
        tc_flops += st.tc_gemm_flops
        tc_alg += st.tc_gemm_alg_flops
        tc_launch += st.tc_gemm_launches
        launches += st.kernel_launches
        ns_it.append(st.ns_iters)
        sw.append(st.sweeps)
    barrier()
    clocks = sampler.stop()
    rel = max(ctx.residual(A, out, B))
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * a.steps / total_s

    # the powers of bf16x3 steps in the step's own precision (pow_bf16 = 0),
    # measured beside the headline configuration on the same box; the
    # library's default runs them as one bf16 pass from n = 4096
    variants = {}
    if world == 1 and a.pow_bf16 == 2 and not a.no_variants:
        try:
            out_v = torch.empty_like(B)
            cv = nsgb.Context(a.n, order=a.order, stream=stream, couple_frob=a.couple, gemm_cluster=a.gemm_cluster,
                              pow_bf16=0)
            for _ in range(3):
                cv.solve(A, B, iters=a.iters, tol=1e-10, out=out_v)
            vms, vit, vsw = [], [], []
            for _ in range(max(1, min(a.steps, 20))):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = cv.solve(A, B, iters=a.iters, tol=1e-10, out=out_v)
                e1.record(stream)
                e1.synchronize()
                assert r.status == nsgb.NS_OK
                vms.append(e0.elapsed_time(e1))
                vit.append(r.stats.ns_iters)
                vsw.append(r.stats.sweeps)
            variants["pow_bf16_off"] = {"value": 1e3 / statistics.mean(vms), "unit": UNIT,
                                    "ms_per_step": statistics.mean(vms), "steps": len(vms),
                                    "verified_rel_res": max(cv.residual(A, out_v, B)),
                                    "ns_iters": int(statistics.median(vit)), "sweeps": int(statistics.median(vsw))}
            cv.close()
        except Exception as ex:  # reported, never fatal to the headline line
            variants["pow_bf16_off"] = {"error": str(ex)[:200]}

    # end to end through the same C-ABI call with host (pinned) buffers: the
    # host->device copy of A and B and the device->host copy of theta are
    # inside the timed region
    Ah = torch.from_numpy(p.A).pin_memory()
    Bh = torch.from_numpy(p.B).pin_memory()
    Th = torch.empty_like(Bh).pin_memory()
    ctx_h = nsgb.Context(a.n, order=a.order, stream=stream, couple_frob=a.couple, gemm_cluster=a.gemm_cluster,
                         pow_bf16=a.pow_bf16, xp_bf16x2=a.xp_bf16x2 or 0)
    ctx_h.solve(Ah, Bh, iters=a.iters, tol=1e-10, out=Th)
    e2e_steps = max(1, min(a.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r = ctx_h.solve(Ah, Bh, iters=a.iters, tol=1e-10, out=Th)
        assert r.status == nsgb.NS_OK
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    ctx_h.close()
    e2e = {"value": world * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(Ah.numel() * 8 + Bh.numel() * 8), "d2h_bytes_per_step": int(Th.numel() * 8)}

    # plain FP64 Newton-Schulz + FP64 Richardson on the GPU (same algorithm, same stopping rule)
    fp64 = None
    if not a.no_fp64:
        ctx64 = nsgb.Context(a.n, order=a.order, stream=stream, precision=nsgb.NS_FP64, couple_frob=a.couple)
        small = make_spd(256, a.kappa, nrhs=a.nrhs, seed=2)
        with nsgb.Context(256, order=a.order, precision=nsgb.NS_FP64) as cw:
            cw.solve(torch.from_numpy(small.A).to(dev), torch.from_numpy(small.B).to(dev), iters=a.iters, tol=1e-10)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        out64 = torch.empty_like(B)
        e0.record(stream)
        r64 = ctx64.solve(A, B, iters=a.iters, tol=1e-10, out=out64)
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64, "status": int(r64.status),
                "ns_iters": r64.stats.ns_iters, "sweeps": r64.stats.sweeps, "rel_res": r64.stats.rel_res,
                "speedup_of_mixed": value / max(world, 1) / (1e3 / ms64)}
        ctx64.close()

    pk, pk_kind = peaks()
    # achieved: algorithmic work, 2 n^3 per product of the method (a bf16x3
    # product counts once), over the event-timed duration of the launches;
    # executed: every bf16 pass the tensor pipe ran (bf16x3 = 3 passes)
    achieved = tc_alg / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    executed = tc_flops / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    # the capture's workload: the default single system (n = 4096, order 8, 4 RHS)
    default_cfg = (a.n, a.kappa, a.nrhs, a.order, a.couple, a.gemm_cluster, a.pow_bf16) == (4096, 1e4, 4, 8, 1.0, 0, 2)
    traffic = recorded_traffic("traffic_k_gemm_tc2_dense_n4096.md") if default_cfg else None
    sus = pk["bf16_tflops_sustained"]
    roof = {"bound": "tensor",
            "kernel": "k_gemm_tc2 / k_gemm_tc (tcgen05 bf16 / bf16x3 products with fused NS epilogue; "
                      "CTA pairs wherever 256-column tiles apply, as at n = 4096)",
            "achieved": achieved, "peak": sus, "unit": "TFLOP/s",
            "frac": achieved / sus if achieved else None,
            "peak_kind": f"bf16 dense sustained ({pk_kind}); kernel timed inside back-to-back solves; "
                         "achieved and frac count algorithmic flops (2 n^3 per product)",
            "frac_of_burst": achieved / pk["bf16_tflops"] if achieved else None,
            "executed": executed,
            "frac_executed": executed / sus if executed else None,
            "executed_note": "every bf16 pass the tensor pipe ran (a bf16x3 product = 3 passes)",
            "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write, both instantiations)",
            "launches_timed": tc_launch,
            "flops_per_launch": tc_alg / max(tc_launch, 1),
            "executed_flops_per_launch": tc_flops / max(tc_launch, 1),
            "avg_launch_ms": tc_ms / max(tc_launch, 1)}
    if rank == 0:
        ns_med = int(statistics.median(ns_it))
        cpu = None
        if not a.no_cpu:
            ref_it = fp64["ns_iters"] if fp64 else ns_med
            ref_sw = fp64["sweeps"] if fp64 else int(statistics.median(sw))
            cpu = oracle_sample(a, ref_it, ref_sw)
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": workload_config(a),
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                           "min": srt[0], "max": srt[-1]},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu,
            "fp64_path": fp64, "verified_rel_res": rel, "ns_iters": ns_med, "sweeps": int(statistics.median(sw)),
            "gemm_ms_per_step": tc_ms / a.steps,
            **({"variants": variants} if variants else {}),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_kernel_gemm(a):
    """Single-product microbenchmark of the tcgen05 GEMM (D = I - L R on
    n x n bf16 splits), the launch configuration the solve uses; intended as
    the target of ncu captures.  Prints one JSON line with the per-launch time
    (CUDA events around `steps` back-to-back calls, each of which also reads
    back the kernel's error word)."""
    import torch

    import paper_2008_11480_gb300 as nsgb
    dev = torch.device("cuda:0")
    n = a.n
    g = torch.Generator(device=dev).manual_seed(7)
    L = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g) * 0.02
    mk = lambda dt=torch.bfloat16: torch.zeros((n, n), dtype=dt, device=dev)  # noqa: E731
    Lh, Ll = mk(), mk()
    nsgb.ns_k_split(L, Lh, Ll, n, n, n, n)
    D32, Dh, Dl = mk(torch.float32), mk(), mk()
    prec = {"bf16": nsgb.NS_BF16, "bf16x3": nsgb.NS_BF16X3, "bf16x6": nsgb.NS_BF16X6,
            "fp64slices": nsgb.NS_FP64}[a.precision]
    D64 = torch.empty((n, n), dtype=torch.float64, device=dev) if prec == nsgb.NS_FP64 else None
    if prec == nsgb.NS_BF16X6:
        L3, D2 = mk(), mk()
        nsgb.ns_k_split3(L, Lh, Ll, L3, n, n, n, n)

    def call():
        if prec == nsgb.NS_FP64:
            nsgb.ns_k_gemm_oz(n, n, n, L, n, L, n, -1.0, None, 0, 0.0, 1.0, D64, n, a.slices)
            return
        if prec == nsgb.NS_BF16X6:
            nsgb.ns_k_gemm_bf16x6(n, n, n, (Lh, Ll, L3), n, (Lh, Ll, L3), n, -1.0, None, 0, 0.0, 1.0, D32, n,
                                  (Dh, Dl, D2), n)
            return
        nsgb.ns_k_gemm_bf16(prec, n, n, n, Lh, Ll, n, Lh, Ll, n, -1.0, None, 0, 0.0, 1.0, D32, n, Dh, Dl, n,
                            None, a.bn, a.cm)
    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        call()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    passes = {nsgb.NS_BF16: 1, nsgb.NS_BF16X3: 3, nsgb.NS_BF16X6: 6,
              nsgb.NS_FP64: a.slices * (a.slices + 1) // 2}[prec]
    print(json.dumps({"kernel": "k_gemm_tc", "n": n, "precision": a.precision, "bn": a.bn, "cm": a.cm,
                      "ms_per_call": ms, "tflops_incl_call_overhead": passes * 2 * n ** 3 / (ms * 1e-3) / 1e12}))


def run_batched(a):
    """Batched harmonic-regressor Gram systems: `a.count` instances, m ~ U{8..128}
    (n = 2m), T = 4n samples, A = sum phi phi^T + 1e-6 I, b = A theta*.  One
    step = one ns_batch_solve of every instance from theta = 0; value = instances
    that reached the tolerance per second (the others are counted, not hidden)."""
    import torch

    import torch.distributed as dist

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_harmonic_batch
    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    probs_all = make_harmonic_batch(a.count, seed=3)
    mine = shard_balanced([float(p.n) ** 3 for p in probs_all], world)[rank]
    probs = [probs_all[i] for i in mine]
    As = [torch.from_numpy(p.A).to(dev) for p in probs]
    Bs = [torch.from_numpy(p.B).to(dev) for p in probs]
    outs = [torch.empty_like(b) for b in Bs]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    bt = nsgb.Batch([p.n for p in probs], [1] * len(probs), order=a.order, stream=stream, profile=1,
                    couple_frob=a.couple, batch_fused=a.batch_fused)
    for _ in range(max(3, a.warmup)):
        _, status, st = bt.solve(As, Bs, iters=a.iters, tol=1e-10, outs=outs)
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms, conv, gflops, gms, gbytes, fused_ms, useful = [], [], 0.0, 0.0, 0.0, 0.0, 0.0
    for _ in range(a.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, status, st = bt.solve(As, Bs, iters=a.iters, tol=1e-10, outs=outs)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        conv.append(st.converged)
        gflops += st.gemm_flops
        gms += st.gemm_ms
        gbytes += st.gemm_bytes
        fused_ms += st.fused_ms
        useful += st.useful_flops
    clocks = sampler.stop()
    import oracle as O
    worst = 0.0
    kap_conv, kap_fail = [], []
    for p, t, i in zip(probs, outs, range(len(probs))):
        kap = float(np.linalg.cond(p.A))  # reported beside each outcome (outside the timed region)
        if bt.result(i)["status"] == nsgb.NS_OK:
            worst = max(worst, float(np.max(O.rel_residual(p.A, t.cpu().numpy(), p.B))))
            kap_conv.append(kap)
        else:
            kap_fail.append(kap)
    # variant: option fp64_slices = 7, the systems the batch leaves unconverged
    # solved again alone by the single-system slice hand-over (after the timed
    # region; one batch, wall-timed)
    variants = {}
    if not a.no_variants:
        bs = nsgb.Batch([p.n for p in probs], [1] * len(probs), order=a.order, stream=stream,
                        couple_frob=a.couple, batch_fused=a.batch_fused, fp64_slices=7)
        outs_s = [torch.empty_like(b) for b in Bs]
        bs.solve(As, Bs, iters=a.iters, tol=1e-10, outs=outs_s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, sts = bs.solve(As, Bs, iters=a.iters, tol=1e-10, outs=outs_s)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        worst_s = 0.0
        for p, t, i in zip(probs, outs_s, range(len(probs))):
            if bs.result(i)["status"] == nsgb.NS_OK:
                worst_s = max(worst_s, float(np.max(O.rel_residual(p.A, t.cpu().numpy(), p.B))))
        variants["slice_handover"] = {
            "converged": sts.converged, "not_converged": sts.not_converged, "ms_per_batch": wall * 1e3,
            "retried": sts.slice_retried, "retried_converged": sts.slice_retried_converged,
            "retry_ms": sts.slice_retry_ms, "worst_verified_rel_res_of_converged": worst_s,
            "how": "option fp64_slices = 7: each system the batch did not converge solved again alone by the "
                   "single-system AUTO path with 7-digit slice products (16 host worker threads, one stream "
                   "each); wall time of one batch, this rank"}
        bs.close()
    if world > 1:
        dist.barrier()
    pk, pk_kind = peaks()
    ach = gflops / (gms / 1e3) / 1e12 if gms > 0 else None
    hbm_gbs = gbytes / (gms / 1e3) / 1e9 if gms > 0 else None
    # whole job: converged systems of all ranks over the slowest rank's time
    t_max = reduce_over_ranks([sum(ms)], "max", dev)[0]
    conv_all = reduce_over_ranks([float(sum(conv))], "sum", dev)[0]
    worst = reduce_over_ranks([worst], "max", dev)[0]
    value = conv_all / (t_max / 1e3)
    if rank != 0:
        bt.close()
        return
    if st.fused:
        # the fused launch solves every system whole: tensor-core products,
        # row kernels and the controller in one kernel; its time is the bound
        f_ach = useful / (fused_ms / 1e3) / 1e12 if fused_ms > 0 else None
        f_exe = gflops / (fused_ms / 1e3) / 1e12 if fused_ms > 0 else None
        roof = {"bound": "tensor", "kernel": "k_bsolve (fused small-system solve, one CTA per system)",
                "achieved": f_ach, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "frac": f_ach / pk["bf16_tflops_sustained"] if f_ach else None,
                "executed": f_exe, "traffic": None,
                "note": "achieved: the systems' products x 2 n^3 over the whole fused launch (products, "
                        "Richardson sweeps, preparation and control of every system); executed counts bf16x3 "
                        f"as 3 passes; {pk_kind} sustained bf16 peak"}
    else:
        roof = {"bound": "hbm", "achieved": hbm_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": hbm_gbs / pk["hbm_gbs"] if hbm_gbs else None, "traffic": None,
                "note": "list-driven product launches: algorithmic bytes (operands once, C term, f32 and "
                        "bf16 outputs) / their event time; tiles of K <= 256 have ~30 flop/B, below the "
                        f"bf16 ridge, so HBM bounds them ({pk_kind} copy peak)",
                "tensor_tflops": ach, "tensor_frac_of_sustained": ach / pk["bf16_tflops_sustained"] if ach
                else None}
    print(json.dumps({
        "metric": METRIC + " (batched harmonic-regressor systems)", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"{a.count} harmonic-regressor Gram systems, m ~ U{{8..128}}, n = 2m, T = 4n, "
                               f"ridge 1e-6, b = A theta*, 1 RHS", "order": a.order, "tol": 1e-10, "couple_frob": a.couple,
                   "l2": "flushed between timed steps (512 MiB write)"},
        "instances": a.count, "converged_per_step": conv_all / a.steps,
        "not_converged_per_step": a.count - conv_all / a.steps,
        "worst_verified_rel_res_of_converged": worst, "passes": st.passes,
        "kappa": {"converged_max": max(kap_conv) if kap_conv else None,
                  "not_converged_min": min(kap_fail) if kap_fail else None,
                  "not_converged_median": float(np.median(kap_fail)) if kap_fail else None,
                  "not_converged_count": len(kap_fail), "how": "numpy cond(A) of this rank's systems"},
        "gemm_launches_per_step": st.gemm_launches, "kernel_launches_per_step": st.kernel_launches,
        "gpu_launches": int(st.kernel_launches) * a.steps, "fused": int(st.fused),
        "host_syncs_per_step": 1 if st.fused else int(st.passes), "roofline": roof,
        "useful_flops_per_product_level": st.useful_flops_per_product, "clocks": clocks,
        "variants": variants}), flush=True)
    bt.close()


def run_serving(a):
    """Continuous-batching serving: Poisson arrivals at `a.rate` req/s for
    `a.duration` s; each request an SPD system Q diag(lambda) Q^T with n
    log-uniform in [32, 2048], kappa log-uniform in [1e2, 1e6], 1..64 RHS,
    solved to a 1e-10 relative residual by order-4 Newton-Schulz (bf16 /
    bf16x3 products) coupled to Richardson.  The A matrices come from a pool
    of `a.pool` systems drawn from that distribution (request i uses pool entry
    i mod pool); every request has its own B.  The server runs on its own
    thread; requests are submitted at their arrival times from this thread.
    value = converged requests / (last completion - first arrival)."""
    import torch

    import torch.distributed as dist

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_serving_trace, make_spd_device
    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    defs = make_serving_trace(1e6, 2.0 * a.pool / 1e6 + 1e-3, seed=11)[:a.pool]
    pool = [make_spd_device(r.n, r.kappa, nrhs=1, seed=r.seed, device=dev, qr_on_host=a.pool_qr_host)[0]
            for r in defs]
    trace_all = make_serving_trace(a.rate, a.duration, seed=a.seed)
    # each rank serves every world-th arrival of the one trace on its own GPU
    trace = [r for i, r in enumerate(trace_all) if i % world == rank]
    gen = torch.Generator(device=dev)
    gen.manual_seed(a.seed + rank)
    reqs = []
    for i, r in zip(range(rank, len(trace_all), world), trace):
        A = pool[i % len(pool)]
        B = torch.randn(A.shape[0], r.nrhs, generator=gen, device=dev, dtype=torch.float64)
        reqs.append((r.arrival_s, A, B, torch.empty_like(B)))
    warm = [(pool[j], torch.randn(pool[j].shape[0], 8, generator=gen, device=dev, dtype=torch.float64))
            for j in range(min(len(pool), max(3, a.warmup) * 8))]
    torch.cuda.synchronize()
    srv = nsgb.Server(int(a.budget_gb * (1 << 30)), a.max_requests, 64, order=a.order, couple_frob=a.couple)
    srv.start()
    wt = [srv.submit(A, B, torch.empty_like(B), iters=a.iters, tol=1e-10) for A, B in warm]
    while not all(srv.poll(t)["done"] for t in wt):
        time.sleep(0.01)
    st0 = srv.stats()
    sampler = ClockSampler(local)
    sampler.start()
    tickets, t_sub = [], []
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for arr, A, B, T in reqs:
        while True:
            dt = t0 + arr - time.perf_counter()
            if dt <= 0:
                break
            if dt > 2e-4:
                time.sleep(dt - 1e-4)
        t_sub.append(time.perf_counter() - t0)
        tickets.append(srv.submit(A, B, T, iters=a.iters, tol=1e-10))
    deadline = time.perf_counter() + 4 * a.duration + 60
    res = [None] * len(tickets)
    left = list(range(len(tickets)))
    while left and time.perf_counter() < deadline:
        nxt = []
        for k in left:
            r = srv.poll(tickets[k])
            if r["done"]:
                res[k] = r
            else:
                nxt.append(k)
        left = nxt
        if left:
            time.sleep(0.005)
    clocks = sampler.stop()
    st1 = srv.stats()
    done = [(k, r) for k, r in enumerate(res) if r is not None]
    conv = [(k, r) for k, r in done if r["status"] == nsgb.NS_OK]
    t_end = max(t_sub[k] + r["latency_ms"] / 1e3 for k, r in done) if done else float("nan")
    lat = np.array([r["latency_ms"] for _, r in conv]) if conv else np.array([float("nan")])
    qms = np.array([r["queue_ms"] for _, r in conv]) if conv else np.array([float("nan")])
    # spot-check converged results in FP64 on the device
    worst = 0.0
    for k, r in conv[:: max(1, len(conv) // 64)]:
        _, A, B, T = reqs[k]
        rr = torch.linalg.vector_norm(B - A @ T, dim=0) / torch.linalg.vector_norm(B, dim=0)
        worst = max(worst, float(rr.max()))
    flops = st1["gemm_flops"] - st0["gemm_flops"]
    # whole job over ranks: counts summed, the slowest rank's span, latencies pooled
    if world > 1:
        dist.barrier()
    t_end = reduce_over_ranks([t_end], "max", dev)[0]
    n_req, n_done, n_conv, n_left, flops, worst = (
        reduce_over_ranks([float(len(reqs)), float(len(done)), float(len(conv)), float(len(left)), flops], "sum",
                          dev) + reduce_over_ranks([worst], "max", dev))
    lat = np.array(gather_lists(lat.tolist()))
    qms = np.array(gather_lists(qms.tolist()))
    if rank != 0:
        if left:
            os._exit(0)
        srv.stop()
        srv.close()
        return
    pk, pk_kind = peaks()
    ach = flops / t_end / 1e12 if n_done else None
    print(json.dumps({
        "metric": METRIC + " (serving)", "value": n_conv / t_end if n_done else 0.0, "unit": UNIT,
        "n_gpus": world, "steps": 1, "warmup": a.warmup, "ms_per_step": t_end * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"serving trace: Poisson arrivals {a.rate:g} req/s for {a.duration:g} s; n log-uniform "
                               f"[32, 2048], kappa log-uniform [1e2, 1e6], nrhs U{{1..64}}; A from a pool of "
                               f"{a.pool} systems, own B per request", "order": a.order, "tol": 1e-10, "couple_frob": a.couple,
                   "budget_gb": a.budget_gb, "max_requests": a.max_requests, "buffers": "device (HBM)",
                   "l2": "inputs of the whole trace exceed L2"},
        "requests": int(n_req), "completed": int(n_done), "converged": int(n_conv),
        "not_converged": int(n_done - n_conv), "unfinished": int(n_left),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_ms": {"p50": float(np.percentile(qms, 50)), "p99": float(np.percentile(qms, 99))},
        "offered_rate": n_req / a.duration, "passes": st1["passes"] - st0["passes"],
        "worst_sampled_rel_res": worst,
        "server_host_ms": st1["tick_ms"] - st0["tick_ms"], "server_wait_ms": st1["wait_ms"] - st0["wait_ms"],
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "roofline": {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                     "frac": ach / pk["bf16_tflops_sustained"] if ach else None, "traffic": None,
                     "note": "executed product flops over the whole serving wall time (a lower bound on the "
                             f"product kernels' rate); peak {pk_kind} sustained bf16"},
        "clocks": clocks}), flush=True)
    if left:  # requests still running: do not wait for them on the way out
        os._exit(0)
    srv.stop()
    srv.close()


def run_orders(a):
    """Order / form comparison on the n = 4096, kappa = 1e4, 4-RHS system (the
    paper's cost analysis: mmm per step against the order reached): factorized
    orders 2, 3, 4, 8, 16, tool-kit orders 5, 7, 12, nested order 45, composite
    rates {2} and {2, 3}, double NS, accelerated Richardson.  Each entry: solves/s
    (device time, median of a.steps solves), NS steps, sweeps, products per solve.
    value = the best entry's solves/s."""
    import torch

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_spd
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = make_spd(a.n, a.kappa, nrhs=a.nrhs, seed=1)
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    out = torch.empty_like(B)
    variants = [("factorized order 2", 2, (), {}), ("order 3", 3, (), {}), ("factorized order 4", 4, (), {}),
                ("factorized order 8", 8, (), {}), ("factorized order 16", 16, (), {}),
                ("tool-kit order 5", 5, (), {"form": 2}), ("tool-kit order 7", 7, (), {"form": 2}),
                ("tool-kit order 12", 12, (), {"form": 2}), ("nested order 45", 45, (), {"form": 3}),
                ("composite order 2, rates {2}", 2, (2,), {}), ("composite order 2, rates {2,3}", 2, (2, 3), {}),
                ("double NS order 4", 4, (4,), {"aux_ahead": 1}),
                ("accelerated Richardson, double NS order 4", 4, (4,), {"aux_ahead": 1, "accel_richardson": 1})]
    table = []
    for name, order, rates, kw in variants:
        ctx = nsgb.Context(a.n, order=order, rates=rates, stream=stream, couple_frob=a.couple, **kw)
        for _ in range(2):
            r = ctx.solve(A, B, iters=a.iters, tol=1e-10, out=out)
        ms = []
        for _ in range(max(3, a.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = ctx.solve(A, B, iters=a.iters, tol=1e-10, out=out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ctx.close()
        med = statistics.median(ms)
        table.append({"variant": name, "status": r.status, "solves_per_s": 1e3 / med, "ms": med,
                      "ns_iters": r.stats.ns_iters, "sweeps": r.stats.sweeps,
                      "products": int(r.stats.gemm_launches), "rel_res": r.stats.rel_res})
    best = max((t for t in table if t["status"] == 0), key=lambda t: t["solves_per_s"])
    print(json.dumps({
        "metric": METRIC + " (order and form comparison)", "value": best["solves_per_s"], "unit": UNIT,
        "n_gpus": 1, "steps": max(3, a.steps), "warmup": 2, "ms_per_step": best["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": dict(workload_config(a), order="per variant"), "best": best["variant"], "variants": table}),
        flush=True)


def run_small(a):
    """Configuration 1: n = 64, lambda log-uniform in [1, 100], one RHS, order 4,
    G0 = I/||A||_F, 8 coupled iterations in FP64 (the plain path; the oracle's
    parity case) and the mixed path to 1e-10: latency of one solve, and
    throughput of many independent copies solved together as one batch."""
    import torch

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_spd
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = make_spd(64, 100.0, nrhs=1, seed=0)
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    lat = {}
    for name, kw, iters, tol in [("fp64, 8 coupled iterations", {"precision": nsgb.NS_FP64, "ns_stop": 0,
                                                                 "max_sweeps": 0}, 8, 0.0),
                                 ("mixed, to 1e-10", {}, 60, 1e-10)]:
        with nsgb.Context(64, order=4, stream=stream, **kw) as ctx:
            for _ in range(5):
                r = ctx.solve(A, B, iters=iters, tol=tol)
            ms = []
            for _ in range(max(10, a.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = ctx.solve(A, B, iters=iters, tol=tol)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        lat[name] = {"us_per_solve": 1e3 * statistics.median(ms), "status": r.status,
                     "rel_res": r.stats.rel_res, "ns_iters": r.stats.ns_iters, "sweeps": r.stats.sweeps}
    copies = a.count
    probs = [make_spd(64, 100.0, nrhs=1, seed=1000 + i) for i in range(copies)]
    As = [torch.from_numpy(q.A).to(dev) for q in probs]
    Bs = [torch.from_numpy(q.B).to(dev) for q in probs]
    outs = [torch.empty_like(b) for b in Bs]
    with nsgb.Batch([64] * copies, [1] * copies, order=4, stream=stream, couple_frob=a.couple) as bt:
        for _ in range(3):
            _, status, st = bt.solve(As, Bs, iters=60, tol=1e-10, outs=outs)
        ms = []
        for _ in range(max(3, a.steps // 4)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, status, st = bt.solve(As, Bs, iters=60, tol=1e-10, outs=outs)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    import oracle as O
    worst = max(float(np.max(O.rel_residual(q.A, t.cpu().numpy(), q.B))) for q, t in zip(probs[:64], outs[:64]))
    med = statistics.median(ms)
    print(json.dumps({
        "metric": METRIC + " (n = 64 systems)", "value": st.converged / (med / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": len(ms), "warmup": 3, "ms_per_step": med, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"{copies} copies of the n = 64 system (lambda log-uniform [1, 100], 1 RHS, order 4, "
                               "G0 = I/||A||_F) solved as one batch to 1e-10; single-solve latencies alongside",
                   "couple_frob": a.couple},
        "converged": st.converged, "passes": st.passes, "worst_verified_rel_res_first64": worst,
        "single_solve_latency": lat}), flush=True)


def run_ill(a):
    """Configuration 5 size: one ill-conditioned SPD system n = 16384, kappa =
    1e6 (A = V diag(sigma^2) V^T with sigma log-uniform in [1e-3, 1], the Gram
    matrix X^T X of X = U diag(sigma) V^T; built as Q diag(lambda) Q^T with
    lambda log-uniform in [1e-6, 1] scaled), one RHS, order 8, tol 1e-10.  The
    mixed path cannot carry G at this kappa and n (binary32 masters); AUTO with
    fp64_slices = 7 hands the solve to the FP64 path with FP64-accurate
    slice products on the tensor cores.  The plain FP64 path (products on the
    CUDA cores) is estimated from one timed FP64 product times the products of
    the seven-slices-throughout run, whose iterates are the plain path's (a
    full run takes minutes)."""
    import torch

    import paper_2008_11480_gb300 as nsgb
    from workloads import make_spd_device
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n, kappa = a.n if "--n" in sys.argv else 16384, a.kappa if "--kappa" in sys.argv else 1e6
    A, B = make_spd_device(n, kappa, nrhs=1, seed=a.seed, device=dev)
    out = torch.empty_like(B)
    runs = {}
    for name, kw in [("auto + fp64 slice products", {"fp64_slices": 7}),
                     ("fp64 path, slice products", {"precision": nsgb.NS_FP64, "fp64_slices": 7}),
                     ("fp64 path, seven slices throughout",
                      {"precision": nsgb.NS_FP64, "fp64_slices": 7, "fp64_slices_early": 0})]:
        with nsgb.Context(n, order=8, stream=stream, couple_frob=a.couple, **kw) as ctx:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = ctx.solve(A, B, iters=80, tol=1e-10, out=out)
            e1.record(stream)
            e1.synchronize()
            rr = max(ctx.residual(A, out, B))
        runs[name] = {"s": e0.elapsed_time(e1) / 1e3, "status": int(r.status), "rel_res": rr,
                      "ns_iters": r.stats.ns_iters, "sweeps": r.stats.sweeps,
                      "products": int(r.stats.gemm_launches), "prec_history": r.stats.prec_history()}
    with nsgb.Context(n, order=8, stream=stream) as ctx:
        r = ctx.solve(A, B, iters=80, tol=1e-10, out=out)
        runs["mixed alone"] = {"status": int(r.status), "rel_res": max(ctx.residual(A, out, B))}
    L = A
    D = torch.empty_like(A)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nsgb.ns_k_gemm_f64(n, n, n, L, n, L, n, 1.0, None, 0, 0.0, 0.0, D, n, stream=stream)
    e1.record(stream)
    e1.synchronize()
    f64_product_s = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    nsgb.ns_k_gemm_oz(n, n, n, L, n, L, n, D=D, ldd=n, slices=7, stream=stream)
    e1.record(stream)
    e1.synchronize()
    oz_product_s = e0.elapsed_time(e1) / 1e3
    # the seven-slice run takes the CUDA-core FP64 path's steps (the same
    # iterates to binary64 rounding): its product count prices the plain path
    est_plain = f64_product_s * runs["fp64 path, seven slices throughout"]["products"]
    print(json.dumps({
        "metric": METRIC + " (ill-conditioned n = 16384 system)", "value": 1.0 / runs["auto + fp64 slice products"]["s"],
        "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (bf16 integer slices, exact accumulation)", "data": "synthetic",
        "config": {"workload": f"dense SPD n={n} kappa={kappa:g} (Gram matrix of X = U diag(sigma) V^T, sigma "
                               "log-uniform [1e-3, 1]), 1 RHS, order 8, tol 1e-10", "seed": a.seed},
        "runs": runs, "fp64_product_s": f64_product_s, "slice_product_s": oz_product_s,
        "plain_fp64_path_estimate": {"s": est_plain, "solves_per_s": 1.0 / est_plain,
                                     "how": "one timed CUDA-core FP64 product x the products of the "
                                            "seven-slice run (the plain path's iterates)"}}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--kappa", type=float, default=1e4)
    ap.add_argument("--nrhs", type=int, default=4)
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--iters", type=int, default=60)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-ns-iters", type=int, default=8)
    ap.add_argument("--ref-sweeps", type=int, default=9)
    ap.add_argument("--kernel", default="", choices=["", "gemm"],
                    help="microbenchmark one kernel instead of the solve")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16", "bf16x3", "bf16x6", "fp64slices"])
    ap.add_argument("--bn", type=int, default=256)
    ap.add_argument("--cm", type=int, default=0)
    ap.add_argument("--slices", type=int, default=7, help="--kernel gemm --precision fp64slices: digits per operand")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the pow_bf16 variant measured beside the default single-system line")
    ap.add_argument("--xp-bf16x2", type=int, default=None, choices=(0, 1, 2),
                    help="option xp_bf16x2: X_j P_j (j >= 1) of bf16x3 steps as two-term products "
                         "(default: 2 on the Gram line, 0 elsewhere)")
    ap.add_argument("--pow-bf16", type=int, default=2, choices=(0, 1, 2),
                    help="powers F^(2^j) of bf16x3 steps in one bf16 pass (library option pow_bf16: "
                         "0 off, 1 on, 2 on from n = 4096)")
    ap.add_argument("--gemm-cluster", type=int, default=0, choices=(0, 1, -2),
                    help="single workload: product-kernel grouping (0 automatic, 1 one CTA per tile, -2 CTA pairs)")
    ap.add_argument("--workload", default="gram",
                    choices=["gram", "single", "dense", "batched", "serving", "orders", "small", "ill"],
                    help="gram (default): the n = 16384 least-squares Gram system, cond 1e6; single / dense: the "
                         "n = 4096 dense system; batched: many harmonic systems; serving: continuous batching of a "
                         "Poisson request trace")
    ap.add_argument("--gram-n", type=int, default=16384, help="gram workload: system size")
    ap.add_argument("--gram-qr-host", action="store_true",
                    help="gram workload: draw the orthogonal factor with a host QR (e.g. under a profiler)")
    ap.add_argument("--ref-rows", type=int, default=512,
                    help="gram workload: rows of the panel the oracle sample multiplies")
    ap.add_argument("--count", type=int, default=2048)
    ap.add_argument("--batch-fused", type=int, default=1, choices=(0, 1),
                    help="batched workload: 1 one fused launch (systems of n <= 256), 0 pass by pass")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--pool", type=int, default=256)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--max-requests", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--couple", type=float, default=1.0,
                    help="couple_frob: Richardson starts once ||F_{k-1}||_F <= this (0: from the first step)")
    ap.add_argument("--pool-qr-host", action="store_true",
                    help="draw the serving pool's orthogonal factors with a host QR (e.g. under a profiler)")
    a = ap.parse_args()
    if a.workload == "orders" and a.impl == "ours":
        if "--steps" not in sys.argv:
            a.steps = 5
        run_orders(a)
        return
    if a.workload == "small" and a.impl == "ours":
        if "--steps" not in sys.argv:
            a.steps = 20
        run_small(a)
        return
    if a.workload == "ill" and a.impl == "ours":
        run_ill(a)
        return
    if a.workload == "serving" and a.impl == "ours":
        if a.order == 8 and "--order" not in sys.argv:
            a.order = 4
        if a.iters == 60 and "--iters" not in sys.argv:
            a.iters = 80
        run_serving(a)
        return
    if a.workload == "batched" and a.impl == "ours":
        if a.order == 8 and "--order" not in sys.argv:
            a.order = 4
        run_batched(a)
        return
    if a.kernel == "gemm":
        run_kernel_gemm(a)
        return
    if a.warmup < 3 and a.impl == "ours":
        a.warmup = 3
    if a.workload == "gram":
        if a.impl == "reference":
            run_reference_gram(a)
        else:
            run_gram(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
