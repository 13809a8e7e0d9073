"""Seeded synthetic SPD systems shaped like the problems the paper targets.

This module only draws inputs; it holds none of the solver arithmetic. Both the
FP64 oracle tests and the CUDA-path tests/bench take their inputs from here, so
the two sides always see the same bytes for the same seed.

The paper (Section 1, eq. ae1) solves A theta_* = b with A symmetric positive
definite; it names harmonic-regressor information matrices and Gram matrices
X^T X as the motivating cases but publishes no data.  The generators below
stand in for those:

* ``make_spd``        -- A = Q diag(lambda) Q^T, Q Haar-orthogonal, lambda
                         log-uniform in [1, kappa] with both ends pinned, so
                         cond(A) = kappa exactly; B ~ N(0, 1)^{n x nrhs}.
* ``make_harmonic``   -- A = sum_t phi_t phi_t^T + 1e-6 I with
                         phi_t = [cos(w_i t), sin(w_i t)]_{i=1..m}, t = 1..4n,
                         theta_* ~ N(0, 1), b = A theta_*.
* ``make_harmonic_batch`` -- many such instances with m ~ U{8..128}.
* ``make_serving_trace``  -- Poisson arrival times with per-request (n, kappa,
                         nrhs) drawn as described in each docstring.
* ``make_spd_device``     -- make_spd's system built with torch on a device.
* ``make_gram_device``    -- the Gram system A = X^T X, b = X^T y of a design
                         X = U diag(sigma) V^T, sigma log-uniform, on a device.

Draw order inside one generator is fixed (Q, then lambda, then B) so that a
seed always yields the same system.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SPDProblem",
    "haar_orthogonal",
    "make_spd",
    "make_harmonic",
    "make_harmonic_batch",
    "make_serving_trace",
    "make_spd_device",
    "make_gram_device",
    "gram_spectrum",
    "ServingRequest",
]


@dataclass
class SPDProblem:
    """One SPD system A theta = B with its known spectral factors.

    ``A`` is n x n float64, row-major, exactly symmetric.  ``B`` is n x nrhs
    float64.  ``Q``/``lam`` give A = Q diag(lam) Q^T (up to rounding), so
    closed forms such as A^{-1} and (I - alpha A)^e are available to tests.
    ``theta_star`` is set when the generator knows the exact solution.
    """

    A: np.ndarray
    B: np.ndarray
    Q: np.ndarray | None = None
    lam: np.ndarray | None = None
    theta_star: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def nrhs(self) -> int:
        return self.B.shape[1]


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix: QR of a Gaussian matrix with
    the sign of diag(R) folded into Q (Mezzadri, "How to generate random
    matrices from the classical compact groups", 2007)."""
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    Q = Q * np.sign(np.diag(R))[None, :]
    return Q


def _log_uniform_spectrum(n: int, kappa: float, rng: np.random.Generator) -> np.ndarray:
    lam = np.exp(rng.uniform(0.0, np.log(kappa), size=n))
    if n >= 2:
        # pin both ends so that cond(A) is exactly kappa
        lam[0] = 1.0
        lam[1] = float(kappa)
    return lam


def make_spd(n: int, kappa: float, nrhs: int = 1, seed: int = 0) -> SPDProblem:
    """A = Q diag(lam) Q^T with Q Haar, lam log-uniform in [1, kappa] (ends
    pinned), B ~ N(0,1)^{n x nrhs}.  Symmetrised exactly: A = (A + A^T)/2."""
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(n, rng)
    lam = _log_uniform_spectrum(n, kappa, rng)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    B = rng.standard_normal((n, nrhs))
    return SPDProblem(A=np.ascontiguousarray(A), B=np.ascontiguousarray(B), Q=Q, lam=lam,
                      meta={"kind": "spd", "n": n, "kappa": float(kappa), "nrhs": nrhs, "seed": seed})


def make_harmonic(m: int, seed: int = 0, T: int | None = None, ridge: float = 1e-6,
                  rng: np.random.Generator | None = None) -> SPDProblem:
    """Harmonic-regressor information matrix with m frequencies (n = 2m).

    phi_t = [cos(w_1 t), sin(w_1 t), ..., cos(w_m t), sin(w_m t)], t = 1..T,
    T = 4n by default, w_i ~ U(0, pi); A = sum_t phi_t phi_t^T + ridge*I;
    theta_* ~ N(0,1)^n and b = A theta_* (so the exact answer is known)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    n = 2 * m
    if T is None:
        T = 4 * n
    w = rng.uniform(0.0, np.pi, size=m)
    t = np.arange(1, T + 1, dtype=np.float64)
    Phi = np.empty((T, n))
    Phi[:, 0::2] = np.cos(np.outer(t, w))
    Phi[:, 1::2] = np.sin(np.outer(t, w))
    A = Phi.T @ Phi + ridge * np.eye(n)
    A = 0.5 * (A + A.T)
    theta = rng.standard_normal((n, 1))
    b = A @ theta
    return SPDProblem(A=np.ascontiguousarray(A), B=np.ascontiguousarray(b), theta_star=theta,
                      meta={"kind": "harmonic", "n": n, "m": m, "T": T, "omega": w})


def make_harmonic_batch(count: int, seed: int = 0, m_lo: int = 8, m_hi: int = 128) -> list[SPDProblem]:
    """``count`` harmonic-regressor systems with m ~ U{m_lo..m_hi} (n = 2m)."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    return [make_harmonic(int(m), rng=rng) for m in ms]


@dataclass
class ServingRequest:
    arrival_s: float
    n: int
    kappa: float
    nrhs: int
    seed: int


def make_serving_trace(rate_per_s: float, duration_s: float, seed: int = 0,
                       n_lo: int = 32, n_hi: int = 2048, k_lo: float = 1e2, k_hi: float = 1e6,
                       nrhs_lo: int = 1, nrhs_hi: int = 64) -> list[ServingRequest]:
    """Poisson arrivals (exponential gaps at ``rate_per_s``) over ``duration_s``;
    per request n log-uniform in [n_lo, n_hi], kappa log-uniform in [k_lo, k_hi],
    nrhs uniform in {nrhs_lo..nrhs_hi}.  Each request carries its own seed for
    ``make_spd``."""
    rng = np.random.default_rng(seed)
    out: list[ServingRequest] = []
    t = 0.0
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        kappa = float(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi))))
        nrhs = int(rng.integers(nrhs_lo, nrhs_hi + 1))
        out.append(ServingRequest(t, n, kappa, nrhs, seed * 1_000_003 + i))
        i += 1
    return out


def make_spd_device(n: int, kappa: float, nrhs: int = 1, seed: int = 0, device="cuda", qr_on_host: bool = False,
                    return_factors: bool = False):
    """The system ``make_spd(n, kappa, nrhs, seed)`` describes, built on a torch
    device: the same Gaussian draws, spectrum and B from the same seed, with
    the QR and Q diag(lam) Q^T done in FP64 by torch on ``device`` (so large
    pools of systems can be drawn quickly; A agrees with make_spd's to
    rounding).  ``qr_on_host`` does the QR with torch on the CPU instead.
    Returns (A, B) as device tensors, or (A, B, Q, lam) with
    ``return_factors`` (the closed-form solution is Q diag(1/lam) Q^T B)."""
    import torch

    rng = np.random.default_rng(seed)
    Z = torch.from_numpy(rng.standard_normal((n, n)))
    lam = torch.from_numpy(_log_uniform_spectrum(n, kappa, rng)).to(device)
    B = torch.from_numpy(rng.standard_normal((n, nrhs))).to(device)
    if qr_on_host:
        Q, R = torch.linalg.qr(Z)
        Q, R = Q.to(device), R.to(device)
    else:
        Q, R = torch.linalg.qr(Z.to(device))
    Q = Q * torch.sign(torch.diagonal(R))[None, :]
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    if return_factors:
        return A.contiguous(), B.contiguous(), Q, lam
    return A.contiguous(), B.contiguous()


def gram_spectrum(n: int, sigma_lo: float = 1e-3, seed: int = 0) -> tuple[np.ndarray, np.ndarray, np.random.Generator]:
    """The host draws of ``make_gram_device`` in its order: sigma (n, log-uniform
    in [sigma_lo, 1], ends pinned), z = U^T y (n x 1, standard normal); returns
    (sigma, z, rng) with rng positioned for the Gaussian matrix of V."""
    rng = np.random.default_rng(seed)
    sigma = np.exp(rng.uniform(np.log(sigma_lo), 0.0, size=n))
    if n >= 2:
        sigma[0] = sigma_lo
        sigma[1] = 1.0
    z = rng.standard_normal((n, 1))
    return sigma, z, rng


def make_gram_device(n: int, sigma_lo: float = 1e-3, seed: int = 0, device="cuda", return_factors: bool = False,
                     qr_on_host: bool = False):
    """The least-squares Gram system of an m x n design X = U diag(sigma) V^T
    (m >= n, U with orthonormal columns and V Haar), sigma log-uniform in
    [sigma_lo, 1] with both ends pinned, built on a torch device in FP64:

        A = X^T X = V diag(sigma^2) V^T      (cond(A) = sigma_lo^-2 exactly)
        b = X^T y = V diag(sigma) (U^T y),   y ~ N(0, 1)^m.

    For U with orthonormal columns drawn independently of y, z = U^T y is
    N(0, 1)^n, so b = V (sigma * z) is drawn directly (X itself is never
    formed; its m only fixes that z is standard normal).  The exact solution
    is theta* = V (z / sigma).  Draw order: sigma, z, the Gaussian matrix of V
    (``gram_spectrum`` gives the first two without the matrix).
    Returns (A, b) as device tensors (b: n x 1), or (A, b, V, sigma, z) with
    ``return_factors``.  ``qr_on_host`` does the QR with torch on the CPU."""
    import torch

    sigma, z, rng = gram_spectrum(n, sigma_lo, seed)
    Zg = torch.from_numpy(rng.standard_normal((n, n)))
    if qr_on_host:
        V, R = torch.linalg.qr(Zg)
        V, R = V.to(device), R.to(device)
    else:
        V, R = torch.linalg.qr(Zg.to(device))
    V = V * torch.sign(torch.diagonal(R))[None, :]
    s = torch.from_numpy(sigma).to(device)
    A = (V * (s * s)[None, :]) @ V.T
    A = 0.5 * (A + A.T)
    zt = torch.from_numpy(z).to(device)
    b = V @ (s[:, None] * zt)
    if return_factors:
        return A.contiguous(), b.contiguous(), V, s, zt
    return A.contiguous(), b.contiguous()
