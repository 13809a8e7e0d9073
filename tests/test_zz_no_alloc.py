"""The allocation-free residual entry point (ns_k_resid_noalloc) against the
regular one (ns_k_resid), through the C ABI.

Some callers cannot allocate device memory while they run -- a serving loop
whose memory is all reserved by its admission budget, a latency-critical loop
that must stay out of the allocator -- so the library offers this variant with
a fixed scratch array.  This file is named to be collected last, so that a run
that stops at the first failure has already run every other test; it also
passes on its own in a fresh process."""
import numpy as np
import pytest
import torch

import paper_2008_11480_gb300 as nsgb

pytestmark = pytest.mark.gpu
dev = torch.device("cuda:0")


def _case(n, nrhs, seed):
    rng = np.random.default_rng(seed)
    A, Th, B = (rng.standard_normal(s) for s in ((n, n), (n, nrhs), (n, nrhs)))
    return A, Th, B


@pytest.mark.parametrize("n,nrhs", [(1000, 4), (257, 9), (4096, 16)])
def test_noalloc_matches_regular_on_two_calls(n, nrhs):
    for call, seed in enumerate((31, 32)):        # two calls in a row, different data
        A, Th, B = _case(n, nrhs, seed + n)
        Ad, Thd, Bd = (torch.from_numpy(x).to(dev) for x in (A, Th, B))
        R_ref = torch.zeros((n, nrhs), dtype=torch.float64, device=dev)
        rsq_ref = torch.zeros(nrhs, dtype=torch.float64, device=dev)
        nsgb.ns_k_resid(Ad, n, Thd, Bd, R_ref, n, nrhs, rsq_ref)
        R = torch.full((n, nrhs), 7.0, dtype=torch.float64, device=dev)
        rsq = torch.full((nrhs,), 7.0, dtype=torch.float64, device=dev)
        assert nsgb.ns_k_resid_noalloc(Ad, n, Thd, Bd, R, n, nrhs, rsq) == nsgb.NS_OK
        torch.cuda.synchronize()
        # same tolerance as the regular residual's parity test (FP64 accumulation)
        tol = n * 2.0 ** -52 * (np.abs(A) @ np.abs(Th) + np.abs(B))
        assert np.all(np.abs(R.cpu().numpy() - R_ref.cpu().numpy()) <= tol), f"call {call}"
        assert np.allclose(rsq.cpu().numpy(), rsq_ref.cpu().numpy(), rtol=1e-12), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    A = torch.zeros((2, 2), dtype=torch.float64, device=dev)
    th = torch.zeros((2, 17), dtype=torch.float64, device=dev)
    R = torch.zeros_like(th)
    assert nsgb.ns_k_resid_noalloc(A, 2, th, th, R, 2, 17) == nsgb.NS_ERR_ARG
    big = 32769
    assert nsgb.ns_k_resid_noalloc(A, big, th, th, R, big, 1) == nsgb.NS_ERR_ARG
