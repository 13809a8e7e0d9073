"""Failure detection without a GPU fault.

Every wait inside the tensor-core product kernel (TMA stage barriers, TMEM
accumulator barriers) is bounded.  The host can make one wait run out on
purpose: NSGB_INJECT_WITHHOLD_LOAD=k makes the producer skip its k-th stage
load, so the barrier of that stage is never armed -- a flag that nothing sets.
The kernel must then report NS_ERR_TIMEOUT through its error word within the
wait bound (NSGB_WAIT_LIMIT_MS), release its tensor memory, and leave the
context usable: the next product and the next solve are correct."""
import os
import time

import numpy as np
import pytest
import torch

import oracle as O
import paper_2008_11480_gb300 as nsgb
from workloads import make_spd

pytestmark = pytest.mark.gpu
dev = torch.device("cuda:0")


def operands(M, N, K, seed):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((M, K)) * 0.05
    R = rng.standard_normal((K, N)) * 0.05
    out = []
    for X in (L, R):
        x = torch.from_numpy(X).to(dev)
        hi = torch.zeros(X.shape, dtype=torch.bfloat16, device=dev)
        lo = torch.zeros_like(hi)
        nsgb.ns_k_split(x, hi, lo, X.shape[0], X.shape[1], X.shape[1], X.shape[1])
        out += [hi, lo]
    return L, R, out


def gemm(prec, M, N, K, parts, D32, bn=128, cm=1):
    Lh, Ll, Rh, Rl = parts
    nsgb.ns_k_gemm_bf16(prec, M, N, K, Lh, Ll, K, Rh, Rl, N, -1.0, None, 0, 0.0, 1.0, D32, N, None, None, 0,
                        None, bn, cm)


@pytest.fixture
def inject(monkeypatch):
    def on(k, limit_ms=50):
        monkeypatch.setenv("NSGB_INJECT_WITHHOLD_LOAD", str(k))
        monkeypatch.setenv("NSGB_WAIT_LIMIT_MS", str(limit_ms))

    def off():
        monkeypatch.delenv("NSGB_INJECT_WITHHOLD_LOAD", raising=False)
        monkeypatch.delenv("NSGB_WAIT_LIMIT_MS", raising=False)

    yield on, off
    off()


@pytest.mark.parametrize("bn,cm", [(128, 1), (256, -2)])
@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
@pytest.mark.parametrize("k", [0, 5])
def test_withheld_stage_load_times_out_and_context_recovers(inject, prec, k, bn, cm):
    """cm = -2: both CTAs of each MMA pair withhold the load, so the stage
    barrier of the pair's first CTA is never armed; both CTAs must give up,
    release the pair's tensor memory together and exit."""
    on, off = inject
    M, N, K = 256, 256, 512
    L, R, parts = operands(M, N, K, seed=60 + k)
    D32 = torch.zeros((M, N), dtype=torch.float32, device=dev)
    on(k)
    t0 = time.perf_counter()
    with pytest.raises(nsgb.NSError) as ei:
        gemm(prec, M, N, K, parts, D32, bn, cm)
    elapsed = time.perf_counter() - t0
    assert ei.value.status == nsgb.NS_ERR_TIMEOUT
    assert elapsed < 5.0
    off()
    # the same product right after is complete and correct
    gemm(prec, M, N, K, parts, D32, bn, cm)
    torch.cuda.synchronize()
    name = "bf16" if prec == nsgb.NS_BF16 else "bf16x3"
    ref = np.eye(M, N) - O.split_product(L, R, name)
    tol = K * 2.0 ** -23 * O.split_abs_product(L, R, name) + 2.0 ** -22 * (np.abs(ref) + 1.0)
    assert np.all(np.abs(D32.cpu().numpy() - ref) <= tol)


def test_solve_after_injected_timeout(inject):
    on, off = inject
    M = N = K = 256
    _, _, parts = operands(M, N, K, seed=70)
    D32 = torch.zeros((M, N), dtype=torch.float32, device=dev)
    on(3)
    with pytest.raises(nsgb.NSError):
        gemm(nsgb.NS_BF16, M, N, K, parts, D32)
    off()
    p = make_spd(200, 1e3, nrhs=2, seed=71)
    with nsgb.Context(200, order=4) as ctx:
        r = ctx.solve(torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev), iters=60, tol=1e-10)
    assert r.status == nsgb.NS_OK
    assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1e-10


def test_x6_pair_withheld_load_times_out(inject):
    on, off = inject
    M, N, K = 256, 256, 256
    rng = np.random.default_rng(80)
    parts = []
    for shape in ((M, K), (K, N)):
        X = torch.from_numpy(rng.standard_normal(shape) * 0.05).to(dev)
        p3 = [torch.zeros(shape, dtype=torch.bfloat16, device=dev) for _ in range(3)]
        nsgb.ns_k_split3(X, *p3, shape[0], shape[1], shape[1], shape[1])
        parts.append(p3)
    D32 = torch.zeros((M, N), dtype=torch.float32, device=dev)
    on(2)
    with pytest.raises(nsgb.NSError) as ei:
        nsgb.ns_k_gemm_bf16x6(M, N, K, parts[0], K, parts[1], N, -1.0, None, 0, 0.0, 1.0, D32, N)
    assert ei.value.status == nsgb.NS_ERR_TIMEOUT
    off()
    nsgb.ns_k_gemm_bf16x6(M, N, K, parts[0], K, parts[1], N, -1.0, None, 0, 0.0, 1.0, D32, N)
    torch.cuda.synchronize()
    assert torch.isfinite(D32).all()


def test_slice_product_withheld_load_times_out(inject):
    on, off = inject
    n = 256
    rng = np.random.default_rng(81)
    L = torch.from_numpy(rng.standard_normal((n, n))).to(dev)
    R = torch.from_numpy(rng.standard_normal((n, n))).to(dev)
    D = torch.zeros((n, n), dtype=torch.float64, device=dev)
    on(3)
    with pytest.raises(nsgb.NSError) as ei:
        nsgb.ns_k_gemm_oz(n, n, n, L, n, R, n, D=D, ldd=n)
    assert ei.value.status == nsgb.NS_ERR_TIMEOUT
    off()
    nsgb.ns_k_gemm_oz(n, n, n, L, n, R, n, D=D, ldd=n)
    torch.cuda.synchronize()
    ref = L.cpu().numpy() @ R.cpu().numpy()
    assert np.allclose(D.cpu().numpy(), ref, rtol=1e-13, atol=1e-12)
