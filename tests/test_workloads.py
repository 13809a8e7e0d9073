"""The seeded input generators: the spectrum and conditioning they promise,
and the device-built variant drawing the same system as the host one."""
import numpy as np
import torch

from workloads import make_serving_trace, make_spd, make_spd_device


def test_make_spd_condition_and_symmetry():
    p = make_spd(40, 1e3, nrhs=3, seed=4)
    assert np.array_equal(p.A, p.A.T)
    ev = np.linalg.eigvalsh(p.A)
    assert ev.min() > 0
    assert abs(ev.max() / ev.min() - 1e3) / 1e3 < 1e-9


def test_make_spd_device_matches_host_draws():
    for n, kappa, nrhs, seed in [(33, 1e2, 2, 1), (96, 1e5, 5, 9)]:
        p = make_spd(n, kappa, nrhs=nrhs, seed=seed)
        A, B = make_spd_device(n, kappa, nrhs=nrhs, seed=seed, device="cpu")
        assert torch.equal(B, torch.from_numpy(p.B))
        assert torch.equal(A, A.T)
        assert np.max(np.abs(A.numpy() - p.A)) <= 1e-12 * kappa


def test_serving_trace_distribution():
    tr = make_serving_trace(2000.0, 2.0, seed=3)
    gaps = np.diff([0.0] + [r.arrival_s for r in tr])
    assert 3600 < len(tr) < 4400
    assert abs(gaps.mean() - 1 / 2000.0) < 0.1 / 2000.0
    ns = np.array([r.n for r in tr])
    assert ns.min() >= 32 and ns.max() <= 2048
    # log-uniform: the median of log n sits mid-way
    assert abs(np.median(np.log(ns)) - 0.5 * (np.log(32) + np.log(2048))) < 0.15
    assert all(1 <= r.nrhs <= 64 for r in tr) and all(1e2 <= r.kappa <= 1e6 for r in tr)


def test_make_gram_device_is_the_gram_system():
    """A = V diag(sigma^2) V^T with cond(A) = sigma_lo^-2 exactly, b = V (sigma z),
    and theta* = V (z / sigma) solves it; checked against an explicit design
    X = U diag(sigma) V^T built from the returned factors (A = X^T X, b = X^T y
    with y = U z for U with orthonormal columns)."""
    from workloads import make_gram_device
    n = 48
    A, b, V, s, z = make_gram_device(n, sigma_lo=1e-2, seed=7, device="cpu", return_factors=True)
    A, b, V, s, z = (t.numpy() for t in (A, b, V, s, z))
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert abs(ev.max() / ev.min() - 1e4) / 1e4 < 1e-8
    U = np.linalg.qr(np.random.default_rng(1).standard_normal((2 * n, n)))[0]
    X = (U * s[None, :]) @ V.T
    y = U @ z
    assert np.allclose(X.T @ X, A, rtol=0, atol=1e-14)
    assert np.allclose(X.T @ y, b, rtol=0, atol=1e-13)
    theta = V @ (z / s[:, None])
    assert np.linalg.norm(A @ theta - b) <= 1e-11 * np.linalg.norm(b) * 1e4
