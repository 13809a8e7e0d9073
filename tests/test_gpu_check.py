"""The final inverse check ||I - A G||_F (precision control): the FP64 product
form and Hutchinson's estimate through the C ABI against the oracle on the
same G and the same SplitMix64 probes, the exact cases, and the final_check
option of the solver calls."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2008_11480_gb300 as nsgb
from workloads import make_spd, make_spd_device

pytestmark = pytest.mark.gpu
dev = torch.device("cuda:0")


def tens(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


@pytest.mark.parametrize("n", [1, 64, 130, 300])
def test_exact_check_matches_oracle(n):
    p = make_spd(n, 1e3, seed=40 + n)
    with nsgb.Context(n, order=4) as ctx:
        G, _ = ctx.invert(tens(p.A), iters=6)
        got = ctx.inverse_residual(tens(p.A), G)
    want = O.inverse_residual(p.A, G.cpu().numpy())
    assert got == pytest.approx(want, rel=1e-10, abs=1e-13)


@pytest.mark.parametrize("n,s,seed", [(64, 1, 0), (257, 7, 12345), (300, 32, 2 ** 63 + 5)])
def test_hutchinson_matches_oracle_probe_for_probe(n, s, seed):
    p = make_spd(n, 1e2, seed=50)
    G = O.alpha_frobenius(p.A) * np.eye(n) + 1e-3 * np.random.default_rng(1).standard_normal((n, n))
    with nsgb.Context(n, order=2) as ctx:
        got = ctx.inverse_residual(tens(p.A), tens(G), probes=s, seed=seed)
    want = O.inverse_residual_hutchinson(p.A, G, s, seed)
    assert got == pytest.approx(want, rel=1e-12)


def test_hutchinson_exact_cases_on_device():
    n = 200
    rng = np.random.default_rng(3)
    A = np.diag(rng.uniform(1, 10, n))
    with nsgb.Context(n, order=2) as ctx:
        # G = 0: every probe has ||z||^2 = n
        assert ctx.inverse_residual(tens(A), tens(np.zeros((n, n))), probes=5, seed=9) == math.sqrt(n)
        # one nonzero per row of I - A G: exact for every probe
        w = rng.uniform(0.1, 3.0, n)
        N_ = np.roll(np.diag(w), 1, axis=1)
        G = np.linalg.solve(A, np.eye(n) - N_)
        got = ctx.inverse_residual(tens(A), tens(G), probes=3, seed=4)
    assert got == pytest.approx(math.sqrt(float(np.sum(w * w))), rel=1e-12)


def test_host_buffers_and_argument_errors():
    n = 96
    p = make_spd(n, 1e2, seed=51)
    G = O.alpha_frobenius(p.A) * np.eye(n)
    with nsgb.Context(n, order=2) as ctx:
        a = ctx.inverse_residual(tens(p.A), tens(G))
        b = ctx.inverse_residual(torch.from_numpy(p.A).pin_memory(), torch.from_numpy(G).pin_memory())
        assert a == b
        for bad in (-1, 4097):
            with pytest.raises(nsgb.NSError) as ei:
                ctx.inverse_residual(tens(p.A), tens(G), probes=bad)
            assert ei.value.status == nsgb.NS_ERR_ARG
        # the context stays usable
        assert ctx.inverse_residual(tens(p.A), tens(G), probes=2) > 0


@pytest.mark.parametrize("precision", [nsgb.NS_AUTO, nsgb.NS_FP64])
@pytest.mark.parametrize("check", [-1, -2, 16])
def test_final_check_option(precision, check):
    n = 200
    p = make_spd(n, 1e3, nrhs=2, seed=52)
    with nsgb.Context(n, order=4, precision=precision, final_check=check) as ctx:
        G, st = ctx.invert(tens(p.A), iters=5)
        Gn = G.cpu().numpy()
        # -2 takes the exact form at this size
        want = O.inverse_residual(p.A, Gn) if check < 0 else O.inverse_residual_hutchinson(p.A, Gn, check, 0)
        assert st.final_frob == pytest.approx(want, rel=1e-10, abs=1e-13)
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
        assert r.status == nsgb.NS_OK and r.stats.final_frob >= 0
        # the final G of a converged solve is a contraction: ||I - A G||_F < 1 bounds rho
        if check < 0:
            assert r.stats.final_frob < 1.0
    with nsgb.Context(n, order=4, precision=precision) as ctx:
        _, st = ctx.invert(tens(p.A), iters=2)
        assert st.final_frob == -1.0


@pytest.mark.parametrize("precision", [nsgb.NS_AUTO, nsgb.NS_FP64])
def test_final_check_auto_uses_probes_above_4096(precision):
    """final_check = -2 above n = 4096: Hutchinson's estimate with 8 probes and
    seed 0, the same number the oracle's estimator gives for the same G."""
    n = 4100
    A, _ = make_spd_device(n, 1e2, nrhs=1, seed=53, device=torch.device("cuda:0"))
    with nsgb.Context(n, order=4, precision=precision, final_check=-2) as ctx:
        G, st = ctx.invert(A, iters=3)
        want = O.inverse_residual_hutchinson(A.cpu().numpy(), G.cpu().numpy(), 8, 0)
        assert st.final_frob == pytest.approx(want, rel=1e-9, abs=1e-12)
