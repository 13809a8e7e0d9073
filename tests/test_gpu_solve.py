"""Solver-level parity on the GPU through the C ABI.

* Plain FP64 path: iterates of G and theta agree with the FP64 oracle to 1e-12
  relative Frobenius (the two differ only in summation order; at kappa <= 100
  the rounding floor is ~1e-14).
* Mixed precision (tcgen05 bf16 / bf16x3 products, FP64 Richardson): the
  relative residual max_c ||b_c - A theta_c|| / ||b_c|| is recomputed by the
  oracle in FP64 and must be <= 1e-10; theta then lies within
  kappa * 1e-10 (times a safety factor 10) of the exact solution.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2008_11480_gb300 as nsgb
from workloads import make_spd

pytestmark = pytest.mark.gpu
dev = torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def tens(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def test_fp64_cfg1_solve_matches_oracle():
    """n = 64, lambda log-uniform in [1, 100], one RHS, order 4 factorized
    (I + F)(I + F^2), 8 coupled iterations, G0 = I/||A||_F."""
    p = make_spd(64, 100.0, nrhs=1, seed=0)
    ref = O.ns_richardson_solve(p.A, p.B, order=4, ns_iters=8)
    with nsgb.Context(64, order=4, precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=0) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=8, tol=0.0)
        G, _ = ctx.invert(tens(p.A), iters=8)
    assert rel(r.theta.cpu().numpy(), ref.theta) <= 1e-12
    assert rel(G.cpu().numpy(), ref.G) <= 1e-12
    assert np.allclose(r.stats.frob_history(), ref.frob_E, rtol=1e-10, atol=1e-13)
    assert np.allclose(r.stats.res_history(), ref.rel_res, rtol=1e-9, atol=1e-14)
    # the closed form of the error model: I - G_8 A = F_0^{4^8}
    a = O.alpha_frobenius(p.A)
    F8 = (p.Q * (1 - a * p.lam) ** (4 ** 8)) @ p.Q.T
    assert np.linalg.norm(np.eye(64) - G.cpu().numpy() @ p.A - F8) <= 1e-11


@pytest.mark.parametrize("order,form,pow_mode", [(2, 0, 0), (3, 0, 0), (4, 0, 1), (8, 0, 0), (8, 0, 1),
                                                 (5, 1, 0), (4, 1, 0)])
def test_fp64_invert_orders_forms(order, form, pow_mode):
    n = 130
    p = make_spd(n, 50.0, seed=3)
    iters = 4 if order >= 4 else 6
    with nsgb.Context(n, order=order, precision=nsgb.NS_FP64, ns_stop=0, form=form, pow_mode=pow_mode) as ctx:
        G, st = ctx.invert(tens(p.A), iters=iters)
    Gref, norms = O.ns_invert(p.A, order=order, iters=iters, form="horner" if form else "factorized",
                              pow_mode="residual" if pow_mode else "square")
    assert rel(G.cpu().numpy(), Gref) <= 1e-12
    assert np.allclose(st.frob_history(), norms, rtol=1e-10)


@pytest.mark.parametrize("g0_mode", [0, 1])
def test_fp64_g0_modes(g0_mode):
    n = 96
    p = make_spd(n, 20.0, seed=4)
    a = O.alpha_frobenius(p.A) if g0_mode == 0 else O.alpha_inf(p.A)
    with nsgb.Context(n, order=2, precision=nsgb.NS_FP64, ns_stop=0, g0_mode=g0_mode) as ctx:
        G, _ = ctx.invert(tens(p.A), iters=5)
    Gref, _ = O.ns_invert(p.A, G0=a * np.eye(n), order=2, iters=5)
    assert rel(G.cpu().numpy(), Gref) <= 1e-12


def test_fp64_user_g0_noncommuting():
    """A Jacobi G0 (Section 2, S = diag(A)) does not commute with A; the right
    product chain still matches the left series of eq. ns."""
    rng = np.random.default_rng(8)
    n = 72
    M = rng.uniform(-1, 1, (n, n))
    M = 0.5 * (M + M.T)
    np.fill_diagonal(M, 0)
    A = M + np.diag(np.abs(M).sum(1) + rng.uniform(0.5, 3, n))
    G0 = O.jacobi_preconditioner(A)
    with nsgb.Context(n, order=4, precision=nsgb.NS_FP64, ns_stop=0) as ctx:
        G, _ = ctx.invert(tens(A), iters=3, G0=tens(G0))
    ref = G0
    for _ in range(3):
        ref = O.ns_classical_step(ref, A, 4)
    assert rel(G.cpu().numpy(), ref) <= 1e-12


def diag_dominant(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.uniform(-1, 1, (n, n))
    M = 0.5 * (M + M.T)
    np.fill_diagonal(M, 0)
    return M + np.diag(np.abs(M).sum(1) + rng.uniform(0.5, 3, n))


def test_fp64_jacobi_g0_mode():
    """g0_mode = 2: the library forms the Jacobi preconditioner S^{-1} =
    diag(A)^{-1} itself (Section 2); iterates equal the oracle's from the same G0."""
    n = 72
    A = diag_dominant(n, 8)
    B = np.random.default_rng(9).standard_normal((n, 2))
    G0 = O.jacobi_preconditioner(A)
    ref = O.ns_richardson_solve(A, B, order=4, ns_iters=4, G0=G0)
    with nsgb.Context(n, order=4, precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=0, g0_mode=2) as ctx:
        r = ctx.solve(tens(A), tens(B), iters=4, tol=0.0)
        G, _ = ctx.invert(tens(A), iters=4)
    assert rel(r.theta.cpu().numpy(), ref.theta) <= 1e-12
    assert rel(G.cpu().numpy(), ref.G) <= 1e-12


@pytest.mark.parametrize("h", [4, 6, 9])
def test_fp64_initial_series_g0(h):
    """g0_order = h: G0 is the initial series of eq. g01 from the Jacobi
    S^{-1} (Section 3), G0 = {sum_{j<h} (S^{-1}D)^j} S^{-1}, built by one
    tool-kit step; it equals the oracle's initial_series (unified form with
    the table's (p, w)) and then the iterates follow."""
    n = 64
    A = diag_dominant(n, 12)
    Sinv = O.jacobi_preconditioner(A)
    _, p, w = O.TOOLKIT_TABLE[h]
    G0, F0 = O.initial_series(A, Sinv, p, w)
    assert np.allclose(F0, np.linalg.matrix_power(np.eye(n) - Sinv @ A, h), atol=1e-12)
    ref, _ = O.ns_invert(A, G0=G0, order=4, iters=2)
    with nsgb.Context(n, order=4, precision=nsgb.NS_FP64, ns_stop=0, g0_mode=2, g0_order=h) as ctx:
        G, _ = ctx.invert(tens(A), iters=2)
    assert rel(G.cpu().numpy(), ref) <= 1e-12


def test_mixed_jacobi_g0_mode_reaches_tolerance():
    n = 300
    A = diag_dominant(n, 10)
    B = np.random.default_rng(11).standard_normal((n, 3))
    with nsgb.Context(n, order=4, g0_mode=2) as ctx:
        r = ctx.solve(tens(A), tens(B), iters=40, tol=1e-10)
    assert r.status == nsgb.NS_OK
    assert float(np.max(O.rel_residual(A, r.theta.cpu().numpy(), B))) <= 1e-10


@pytest.mark.parametrize("h", list(range(2, 20)))
def test_fp64_toolkit_orders_match_oracle(h):
    """form = 2: the Appendix tool-kit row for order h (Tables t1-t3) as the
    NS step; iterates equal the oracle's tool-kit series {sum_{j<h} Y^j} X and
    each step costs the row's mmm count (eq. np1, +1 for eq. ztab2)."""
    n = 48
    p = make_spd(n, 30.0, nrhs=1, seed=40 + h)
    K = 2
    ref = O.alpha_frobenius(p.A) * np.eye(n)
    cnt = O.MMCount()
    for _ in range(K):
        ref = O.toolkit(ref, p.A, h, cnt)
    with nsgb.Context(n, order=h, precision=nsgb.NS_FP64, ns_stop=0, form=2) as ctx:
        G, st = ctx.invert(tens(p.A), iters=K)
    assert rel(G.cpu().numpy(), ref) <= 1e-12
    assert st.gemm_launches == cnt.n


def test_fp64_nested_order45_matches_oracle():
    n = 48
    p = make_spd(n, 200.0, nrhs=1, seed=45)
    ref = O.alpha_frobenius(p.A) * np.eye(n)
    cnt = O.MMCount()
    for _ in range(2):
        ref = O.nested_order45(ref, p.A, cnt)
    with nsgb.Context(n, order=45, precision=nsgb.NS_FP64, ns_stop=0, form=3) as ctx:
        G, st = ctx.invert(tens(p.A), iters=2)
    assert rel(G.cpu().numpy(), ref) <= 1e-12
    assert st.gemm_launches == cnt.n == 20
    # error model: I - G_2 A = F_0^{45^2}
    a = O.alpha_frobenius(p.A)
    F = (p.Q * (1 - a * p.lam) ** (45 ** 2)) @ p.Q.T
    assert np.linalg.norm(np.eye(n) - G.cpu().numpy() @ p.A - F) <= 1e-10


@pytest.mark.parametrize("form,order", [(2, 5), (2, 7), (2, 12), (2, 19), (3, 45)])
def test_mixed_toolkit_forms_reach_tolerance(form, order):
    p = make_spd(256, 1e3, nrhs=2, seed=50 + order)
    with nsgb.Context(256, order=order, form=form) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=40, tol=1e-10)
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1e-10


@pytest.mark.parametrize("n_order,rates", [(2, [2]), (2, [2, 3]), (3, [2])])
def test_fp64_composite_matches_oracle(n_order, rates):
    n = 80
    p = make_spd(n, 10.0, seed=9)
    K = 3
    with nsgb.Context(n, order=n_order, rates=rates, precision=nsgb.NS_FP64, ns_stop=0) as ctx:
        G, _ = ctx.invert(tens(p.A), iters=K)
    st = O.composite_init(O.alpha_frobenius(p.A) * np.eye(n), len(rates))
    for _ in range(K):
        st = O.composite_iterate(p.A, st, n_order, rates)
    assert rel(G.cpu().numpy(), st.G) <= 1e-12
    e = O.composite_exponents(n_order, rates, 1, K)[K]
    a = O.alpha_frobenius(p.A)
    ref = (p.Q * (1 - a * p.lam) ** e) @ p.Q.T
    assert np.linalg.norm(np.eye(n) - G.cpu().numpy() @ p.A - ref) <= 1e-11


@pytest.mark.parametrize("n_order", [2, 3])
def test_fp64_double_ns_matches_oracle(n_order):
    """Section 5.1: composite with one auxiliary loop started one step ahead."""
    n = 64
    p = make_spd(n, 6.0, seed=10)
    K = 2
    with nsgb.Context(n, order=n_order, rates=[n_order], precision=nsgb.NS_FP64, ns_stop=0, aux_ahead=1) as ctx:
        G, _ = ctx.invert(tens(p.A), iters=K)
    st = O.double_ns_init(p.A, O.alpha_frobenius(p.A) * np.eye(n), n_order)
    for _ in range(K):
        st = O.double_ns_iterate(p.A, st, n_order)
    assert rel(G.cpu().numpy(), st.G) <= 1e-12


@pytest.mark.parametrize("updated", [0, 1])
def test_fp64_richardson_orderings(updated):
    n = 50
    p = make_spd(n, 30.0, nrhs=2, seed=11)
    ref = O.ns_richardson_solve(p.A, p.B, order=2, ns_iters=5, max_sweeps=3, use_updated_G=bool(updated))
    with nsgb.Context(n, order=2, precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=3, use_updated_G=updated) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=5, tol=0.0)
    assert rel(r.theta.cpu().numpy(), ref.theta) <= 1e-12
    assert r.stats.sweeps == ref.sweeps


@pytest.mark.parametrize("n_order,K", [(2, 2), (2, 3), (3, 2)])
def test_fp64_accelerated_richardson_matches_oracle(n_order, K):
    """Accelerated Richardson of Section 6 (eq. ttk1, q = n) on the double
    Newton-Schulz state: theta starts at L_0 b and step k applies
    omega_k = L_k + Gamma_k^n P(F_k) G_k; the iterate equals the oracle's and
    its error is (S^{-1}D)^{gamma_k} theta~_0 with gamma_k of eq. riem6."""
    n = 40
    p = make_spd(n, 20.0, nrhs=2, seed=16)
    a = O.alpha_frobenius(p.A)
    st = O.double_ns_init(p.A, a * np.eye(n), n_order)
    theta = st.L @ p.B
    tstar = np.linalg.solve(p.A, p.B)
    t0 = theta - tstar
    for _ in range(K):
        st = O.double_ns_iterate(p.A, st, n_order)
        theta = O.accelerated_richardson_step(p.A, p.B, theta, st, q=n_order)
    with nsgb.Context(n, order=n_order, rates=(n_order,), precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=0,
                      aux_ahead=1, accel_richardson=1) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=K + 1, tol=0.0)
    got = r.theta.cpu().numpy()
    assert rel(got, theta) <= 1e-12
    g = int(O.accelerated_richardson_exponent(n_order, 1, K))
    Fg = (p.Q * (1 - a * p.lam) ** g) @ p.Q.T
    assert np.linalg.norm((got - tstar) - Fg @ t0) <= 1e-11 * max(1.0, np.linalg.norm(t0))
    assert r.stats.sweeps == K


@pytest.mark.parametrize("n_order,K", [(2, 2), (2, 3), (3, 2), (4, 2), (8, 2)])
def test_fp64_recursive_omega_matches_oracle(n_order, K):
    """accel_richardson = 2, the recursive schedule of Section 6.2: omega_k
    formed as a matrix (eq. redttk2), G_{k+1} from omega_k by eq. gkrecu1, L
    and Gamma^n from the same Q = sum_{j<n} Gamma^j (eqs. lkk1, gamk21), and
    theta_k = theta_{k-1} - omega_k (A theta_{k-1} - b) (eq. redttk1).  The
    iterate equals the oracle's recursion (``omega_recursive``, Horner applied
    to each matrix) and follows the error law of eq. riem6."""
    n = 40
    p = make_spd(n, 20.0, nrhs=2, seed=16)
    a = O.alpha_frobenius(p.A)
    st = O.double_ns_init(p.A, a * np.eye(n), n_order)
    theta = st.L @ p.B
    tstar = np.linalg.solve(p.A, p.B)
    t0 = theta - tstar
    SG = O.ns_classical_step(st.G, p.A, n_order)
    omega = st.L + st.GamN @ SG
    GamN, L = st.GamN, st.L
    for _ in range(K):
        omega, SG, GamN, L, _G = O.omega_recursive(p.A, omega, SG, GamN, L, n_order)
        theta = theta - omega @ (p.A @ theta - p.B)
    with nsgb.Context(n, order=n_order, rates=(n_order,), precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=0,
                      aux_ahead=1, accel_richardson=2) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=K + 1, tol=0.0)
    got = r.theta.cpu().numpy()
    assert rel(got, theta) <= 1e-12
    g = int(O.accelerated_richardson_exponent(n_order, 1, K))
    Fg = (p.Q * (1 - a * p.lam) ** g) @ p.Q.T
    assert np.linalg.norm((got - tstar) - Fg @ t0) <= 1e-11 * max(1.0, np.linalg.norm(t0))
    assert r.stats.sweeps == K


@pytest.mark.parametrize("n,order,kappa,form", [(300, 4, 1e3, 0), (1000, 8, 1e4, 0), (500, 3, 1e3, 0),
                                                 (400, 4, 1e3, 1)])
def test_mixed_recursive_omega_reaches_tolerance(n, order, kappa, form):
    """The recursive omega_k schedule on the tensor-core path (AUTO precision;
    factorized Q for orders 2^m, Horner otherwise and for form 1) reaches
    1e-10, verified in FP64, with theta against the closed form."""
    p = make_spd(n, kappa, nrhs=3, seed=17)
    with nsgb.Context(n, order=order, rates=(order,), aux_ahead=1, accel_richardson=2, form=form) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    th = r.theta.cpu().numpy()
    assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    assert rel(th, tstar) <= 10 * kappa * 1e-10


def test_accelerated_richardson_needs_double_ns():
    with pytest.raises(nsgb.NSError):
        nsgb.Context(32, order=4, precision=nsgb.NS_FP64, accel_richardson=1)
    with pytest.raises(nsgb.NSError):
        nsgb.Context(32, order=4, rates=(4,), precision=nsgb.NS_FP64, accel_richardson=1)  # aux_ahead = 0
    with pytest.raises(nsgb.NSError):
        nsgb.Context(32, order=4, rates=(4,), precision=nsgb.NS_FP64, aux_ahead=1, accel_richardson=3)


def test_mixed_accelerated_richardson_reaches_tolerance():
    p = make_spd(300, 1e3, nrhs=3, seed=17)
    with nsgb.Context(300, order=4, rates=(4,), aux_ahead=1, accel_richardson=1) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1e-10


@pytest.mark.parametrize("c", [1.0, 0.25])
def test_fp64_delayed_coupling_matches_oracle(c):
    """couple_frob > 0: the Richardson branch starts once ||F_{k-1}||_F <= c;
    iterates, residual record and sweep count follow the oracle's."""
    n = 60
    p = make_spd(n, 80.0, nrhs=2, seed=14)
    ref = O.ns_richardson_solve(p.A, p.B, order=4, ns_iters=7, max_sweeps=3, couple_frob=c)
    with nsgb.Context(n, order=4, precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=3, couple_frob=c) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=7, tol=0.0)
    assert rel(r.theta.cpu().numpy(), ref.theta) <= 1e-12
    assert r.stats.sweeps == ref.sweeps and r.stats.ns_iters == ref.ns_iters
    assert np.allclose(r.stats.res_history(), ref.rel_res, rtol=1e-9, atol=1e-14)


def test_mixed_delayed_coupling_saves_sweeps():
    p = make_spd(384, 1e4, nrhs=3, seed=15)
    out = {}
    for c in (0.0, 1.0):
        with nsgb.Context(384, order=4, couple_frob=c) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
        assert r.status == nsgb.NS_OK
        assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1e-10
        out[c] = r.stats
    assert out[1.0].sweeps < out[0.0].sweeps
    assert out[1.0].ns_iters <= out[0.0].ns_iters + 1


@pytest.mark.parametrize("n,kappa,order,nrhs", [(64, 100.0, 4, 1), (256, 1e3, 4, 3), (200, 1e4, 8, 4),
                                                (130, 1e2, 3, 2), (512, 1e4, 2, 5)])
def test_mixed_precision_solve_reaches_tolerance(n, kappa, order, nrhs):
    p = make_spd(n, kappa, nrhs=nrhs, seed=12)
    with nsgb.Context(n, order=order) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
    th = r.theta.cpu().numpy()
    rr = float(np.max(O.rel_residual(p.A, th, p.B)))
    assert r.status == nsgb.NS_OK, (r.status, r.stats.res_history())
    assert rr <= 1e-10
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    assert rel(th, tstar) <= 10 * kappa * 1e-10
    assert r.stats.gemm_launches > 0


@pytest.mark.parametrize("n,kappa", [(1000, 1e4), (512, 1e3)])
def test_mixed_solve_through_cta_pairs(n, kappa):
    """The products of the solve on CTA pairs sharing each MMA (gemm_cluster =
    -2, 256 x 256 tiles): the tolerance is reached and theta matches the
    closed-form solution as closely as with one-CTA tiles."""
    p = make_spd(n, kappa, nrhs=3, seed=17)
    out = {}
    for cm in (1, -2):
        with nsgb.Context(n, order=8, gemm_bn=256, gemm_cluster=cm) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
        th = r.theta.cpu().numpy()
        assert r.status == nsgb.NS_OK, (cm, r.stats.res_history())
        assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
        out[cm] = th
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    assert rel(out[-2], tstar) <= 10 * kappa * 1e-10
    assert rel(out[-2], out[1]) <= 10 * kappa * 1e-10


@pytest.mark.parametrize("n,kappa", [(300, 1e4), (640, 1e4)])
def test_bf16x6_solve_reaches_tolerance(n, kappa):
    """Every product in split-bf16 x6 (CTA pairs; n = 300 and 640 give odd
    row-tile counts): the solve reaches the tolerance and its final G is at
    least as good as bf16x3's."""
    p = make_spd(n, kappa, nrhs=2, seed=18)
    res = {}
    for prec in (nsgb.NS_BF16X3, nsgb.NS_BF16X6):
        with nsgb.Context(n, order=4, precision=prec, final_check=-1) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
        assert r.status == nsgb.NS_OK, (prec, r.stats.res_history())
        assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1e-10
        assert set(r.stats.prec_history()) == {prec}
        res[prec] = r.stats.final_frob
    assert res[nsgb.NS_BF16X6] <= 1.5 * res[nsgb.NS_BF16X3]


def test_bf16x6_invert_floor_below_bf16x3():
    """The precision floor of ||I - A G||_F (FP64 check) after many steps is
    lower with bf16x6 products than with bf16x3 -- by a factor ~2.6 here, not
    2^8: past the split error, the binary32 master of G (kappa 2^-24 sqrt(n)
    ~ 0.013) sets the floor."""
    n = 512
    p = make_spd(n, 1e4, seed=19)
    fl = {}
    for prec in (nsgb.NS_BF16X3, nsgb.NS_BF16X6):
        with nsgb.Context(n, order=4, precision=prec, final_check=-1, ns_stop=0) as ctx:
            _, st = ctx.invert(tens(p.A), iters=14)
        fl[prec] = st.final_frob
    assert fl[nsgb.NS_BF16X6] * 1.8 < fl[nsgb.NS_BF16X3]
    assert fl[nsgb.NS_BF16X6] < 3.0 * 1e4 * 2.0 ** -24 * math.sqrt(n)


def test_auto_resumes_in_bf16x6_when_richardson_stalls():
    """n = 2048, kappa = 5e6: bf16x3 Newton-Schulz stalls with ||F||_F ~ 16 and the
    Richardson sweeps from that G do not contract; AUTO then resumes Newton-Schulz
    in bf16x6 from G_k and reaches the tolerance."""
    from workloads import make_spd_device
    A, B = make_spd_device(2048, 5e6, nrhs=1, seed=3, device=dev)
    with nsgb.Context(2048, order=8) as ctx:
        r = ctx.solve(A, B, iters=80, tol=1e-10)
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert nsgb.NS_BF16X6 in r.stats.prec_history()
    An, th, Bn = A.cpu().numpy(), r.theta.cpu().numpy(), B.cpu().numpy()
    rr = float(np.max(O.rel_residual(An, th, Bn)))
    # at kappa = 5e6 an FP64 evaluation of b - A theta resolves the relative
    # residual only to about u kappa / 2 = 2.8e-10 (the solver's own residual
    # test and this recomputation sum in different orders; measured 1.18e-10
    # here for a solve the solver saw at <= 1e-10)
    assert rr <= 1e-10 + 0.5 * 2.0 ** -53 * 5e6, rr


def test_fp64_path_with_slice_products_matches_cuda_cores():
    """NS_FP64 with seven slices throughout (fp64_slices = 7, fp64_slices_early
    = 0: FP64-accurate tensor-core products) follows the CUDA-core FP64 path
    step for step: the same ||F_k||_F history to FP64 rounding, the same
    stopping, theta to the residual bar.  With the default four early slices
    the history departs (F_k = F_{k-1}^4 multiplies the early 2^-32 split
    error) but the solve takes as many steps and reaches the same bar."""
    n = 400
    p = make_spd(n, 1e6, nrhs=2, seed=20)
    runs = {}
    for name, kw in (("cores", {}), ("slices", {"fp64_slices": 7, "fp64_slices_early": 0}),
                     ("slices, 4 early", {"fp64_slices": 7})):
        with nsgb.Context(n, order=4, precision=nsgb.NS_FP64, **kw) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
        assert r.status == nsgb.NS_OK, name
        assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1e-10 + 0.5 * 2.0 ** -53 * 1e6
        runs[name] = r
    f0, f7 = runs["cores"].stats.frob_history(), runs["slices"].stats.frob_history()
    assert len(f0) == len(f7)
    for a, b in zip(f0, f7):
        assert b == pytest.approx(a, rel=1e-9, abs=1e-11)
    assert abs(runs["slices, 4 early"].stats.ns_iters - runs["cores"].stats.ns_iters) <= 1


def test_slice_products_solve_where_mixed_precision_cannot():
    """kappa = 1e8 at n = 1024, tol = 1e-7 (an FP64 residual resolves about
    u kappa / 2 = 5.6e-9 here): the binary32 masters of the mixed path cannot
    carry this G (floor kappa 2^-24 sqrt(n) >> 1) and the mixed solve fails;
    the FP64 path with slice products reaches the tolerance."""
    n, kappa, tol = 1024, 1e8, 1e-7
    p = make_spd(n, kappa, nrhs=1, seed=21)
    with nsgb.Context(n, order=4) as ctx:
        rm = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=tol)
    assert float(np.max(O.rel_residual(p.A, rm.theta.cpu().numpy(), p.B))) > tol
    with nsgb.Context(n, order=4, precision=nsgb.NS_FP64, fp64_slices=7) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=tol)
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1.1 * tol
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    assert rel(r.theta.cpu().numpy(), tstar) <= 10 * kappa * tol


def test_auto_hands_over_to_slice_products():
    """AUTO with fp64_slices: the mixed solve of kappa = 1e8 cannot reach the
    tolerance, the FP64 path with slice products takes over from its theta and
    finishes (FP64 steps appear in the precision history)."""
    n, kappa, tol = 1024, 1e8, 1e-7
    p = make_spd(n, kappa, nrhs=1, seed=21)
    with nsgb.Context(n, order=4, fp64_slices=7) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=tol)
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert nsgb.NS_FP64 in r.stats.prec_history() and nsgb.NS_BF16 in r.stats.prec_history()
    assert float(np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B))) <= 1.1 * tol


def test_slice_powers_in_fewer_digits():
    """Option fp64_slices_pow: the powers F^{2^{j+1}} of a factorized step in 3
    or 2 digits on the FP64 path with 7-digit slice products (kappa = 1e8,
    n = 1024, order 8).  The solve reaches the tolerance in as many steps
    (within one) as with full-digit powers, theta matches the closed form, and
    the executed digit-pair work falls."""
    n, kappa, tol = 1024, 1e8, 1e-7
    p = make_spd(n, kappa, nrhs=1, seed=21)
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    runs = {}
    for pw in (0, 3, 2):
        with nsgb.Context(n, order=8, precision=nsgb.NS_FP64, fp64_slices=7, fp64_slices_early=0,
                          fp64_slices_pow=pw) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=tol)
        assert r.status == nsgb.NS_OK, (pw, r.stats.res_history())
        th = r.theta.cpu().numpy()
        assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1.1 * tol, pw
        assert rel(th, tstar) <= 10 * kappa * tol, pw
        runs[pw] = r.stats
    for pw in (3, 2):
        assert abs(runs[pw].ns_iters - runs[0].ns_iters) <= 1
        assert runs[pw].slice_pair_flops < runs[0].slice_pair_flops


def test_gram_size_solve_bench_configuration():
    """The n = 16384 least-squares Gram system (A = V diag(sigma^2) V^T, sigma
    log-uniform in [1e-3, 1], cond 1e6, b = V (sigma z)) in the launch
    configuration the benchmark times: AUTO, order 8, couple_frob 1,
    two-term updates in bf16x3 steps (xp_bf16x2 2), fp64_slices 4 from the
    hand-over on (fp64_slices_early 0), the powers in 2 digits; at the binary32
    floor Richardson gets the first try, the slice
    products take over only if its sweeps give up.  Checked at full size by
    properties: the library's FP64 residual, the residual recomputed in torch,
    and theta against the closed form theta* = V (z / sigma)."""
    from workloads import make_gram_device
    n = 16384
    A, B, V, sg, z = make_gram_device(n, 1e-3, seed=5, device=dev, return_factors=True)
    tstar = V @ (z / sg[:, None])
    del V
    torch.cuda.empty_cache()
    with nsgb.Context(n, order=8, couple_frob=1.0, fp64_slices=4, fp64_slices_early=0, fp64_slices_pow=2,
                      xp_bf16x2=2) as ctx:
        r = ctx.solve(A, B, iters=80, tol=1e-10)
        assert r.status == nsgb.NS_OK, (r.stats.prec_history(), r.stats.res_history()[-5:])
        assert max(ctx.residual(A, r.theta, B)) <= 1e-10
    if nsgb.NS_FP64 not in r.stats.prec_history():
        # the sweeps from the floor's G converged: the slice option changed
        # nothing, the solve is the one without it, bit for bit
        with nsgb.Context(n, order=8, couple_frob=1.0, xp_bf16x2=2) as ctx:
            r0 = ctx.solve(A, B, iters=80, tol=1e-10)
        assert r0.status == nsgb.NS_OK
        assert torch.equal(r0.theta, r.theta)
        assert r0.stats.sweeps == r.stats.sweeps and r0.stats.ns_iters == r.stats.ns_iters
    res = torch.linalg.vector_norm(B - A @ r.theta) / torch.linalg.vector_norm(B)
    assert float(res) <= 1e-10 + 8 * 2.0 ** -53 * 1e6
    err = torch.linalg.vector_norm(r.theta - tstar) / torch.linalg.vector_norm(tstar)
    assert float(err) <= 10 * 1e6 * 1e-10


def test_bf16x6_rejected_where_not_built():
    with pytest.raises(nsgb.NSError) as ei:
        nsgb.Context(64, order=2, rates=(2,), precision=nsgb.NS_BF16X6)
    assert ei.value.status == nsgb.NS_ERR_UNSUPPORTED
    with pytest.raises(nsgb.NSError) as ei:
        nsgb.Context(64, order=45, form=3, precision=nsgb.NS_BF16X6)
    assert ei.value.status == nsgb.NS_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
def test_fixed_precision_solve(prec):
    p = make_spd(128, 50.0, nrhs=2, seed=13)
    with nsgb.Context(128, order=4, precision=prec) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=40, tol=1e-10)
    assert r.status == nsgb.NS_OK
    assert np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B)) <= 1e-10
    assert set(r.stats.prec_history()) == {prec}


def test_mixed_invert_close_to_inverse():
    n = 256
    p = make_spd(n, 1e3, seed=14)
    Ainv = (p.Q / p.lam) @ p.Q.T
    with nsgb.Context(n, order=4, precision=nsgb.NS_BF16X3) as ctx:
        G, st = ctx.invert(tens(p.A), iters=30)
    # bf16x3 floor at kappa = 1e3: rho(I - A G) ~ 1e-3 => ||G - A^-1|| / ||A^-1|| small
    assert rel(G.cpu().numpy(), Ainv) <= 1e-2
    assert min(st.frob_history()) <= 0.05


def test_host_pointers_match_device_pointers():
    p = make_spd(100, 100.0, nrhs=2, seed=15)
    with nsgb.Context(100, order=4) as ctx:
        rd = ctx.solve(tens(p.A), tens(p.B), iters=40, tol=1e-10)
        Ah = torch.from_numpy(p.A).pin_memory()
        Bh = torch.from_numpy(p.B).pin_memory()
        out = torch.empty_like(Bh).pin_memory()
        rh = ctx.solve(Ah, Bh, iters=40, tol=1e-10, out=out)
        rp = ctx.solve(torch.from_numpy(p.A), torch.from_numpy(p.B), iters=40, tol=1e-10)  # pageable
    a = rd.theta.cpu().numpy()
    assert np.array_equal(a, rh.theta.numpy())
    assert np.array_equal(a, rp.theta.numpy())


def test_repeatable_bitwise():
    p = make_spd(300, 1e3, nrhs=2, seed=16)
    outs = []
    with nsgb.Context(300, order=8) as ctx:
        for _ in range(2):
            outs.append(ctx.solve(tens(p.A), tens(p.B), iters=40, tol=1e-10).theta.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_residual_entry_point():
    p = make_spd(77, 10.0, nrhs=3, seed=17)
    th = np.random.default_rng(0).standard_normal((77, 3))
    with nsgb.Context(77, order=2) as ctx:
        got = ctx.residual(tens(p.A), tens(th), tens(p.B))
    assert np.allclose(got, O.rel_residual(p.A, th, p.B), rtol=1e-12)


def test_degenerate_sizes():
    for n in (1, 2, 3):
        p = make_spd(n, 2.0, nrhs=1, seed=18)
        with nsgb.Context(n, order=4) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=30, tol=1e-12)
        assert np.max(O.rel_residual(p.A, r.theta.cpu().numpy(), p.B)) <= 1e-12


def test_errors_leave_context_usable():
    p = make_spd(32, 10.0, nrhs=1, seed=19)
    with nsgb.Context(32, order=4) as ctx:
        A = tens(p.A)
        Abad = A.clone()
        Abad[3, 5] = float("nan")
        s, _ = nsgb.ns_richardson_solve(ctx.handle, Abad, tens(p.B), None, 10, 1e-10,
                                        torch.empty_like(tens(p.B)), check=False)
        assert s == nsgb.NS_ERR_NONFINITE
        r = ctx.solve(A, tens(p.B), iters=30, tol=1e-10)
        assert r.status == nsgb.NS_OK


def test_config5_size_solve_with_slice_products():
    """The ill-conditioned n = 16384 system (kappa = 1e6: eigenvalues
    log-uniform over six decades, as A = X^T X with sigma log-uniform in
    [1e-3, 1]) in the launch configuration the benchmark times: AUTO with
    fp64_slices = 7, order 8, one RHS, tol 1e-10.  The mixed attempt cannot
    finish (binary32 masters) and hands over to the FP64 path with slice
    products.  Checked at full size by properties: the FP64 residual through
    the library and in torch, and theta against the closed form
    Q diag(1/lam) Q^T b from the generator's factors."""
    from workloads import make_spd_device
    n, kappa = 16384, 1e6
    A, B, Q, lam = make_spd_device(n, kappa, nrhs=1, seed=5, device=dev, return_factors=True)
    tstar = Q @ ((Q.T @ B) / lam[:, None])
    del Q
    torch.cuda.empty_cache()
    with nsgb.Context(n, order=8, fp64_slices=7, couple_frob=1.0) as ctx:
        r = ctx.solve(A, B, iters=80, tol=1e-10)
        assert r.status == nsgb.NS_OK, (r.stats.prec_history(), r.stats.res_history()[-5:])
        assert max(ctx.residual(A, r.theta, B)) <= 1e-10
    # an FP64 evaluation of b - A theta itself carries about u kappa of ||b||
    res = torch.linalg.vector_norm(B - A @ r.theta) / torch.linalg.vector_norm(B)
    assert float(res) <= 1e-10 + 8 * 2.0 ** -53 * kappa
    err = torch.linalg.vector_norm(r.theta - tstar) / torch.linalg.vector_norm(tstar)
    assert float(err) <= 10 * kappa * 1e-10


@pytest.mark.parametrize("n,kappa,nrhs", [(4096, 1e4, 4), (4096, 1e5, 4), (1000, 1e5, 2)])
def test_two_term_updates_in_split_steps(n, kappa, nrhs):
    """Option xp_bf16x2: in bf16x3 steps the updates X_j P_j (j >= 1) drop the
    hi(X) lo(P) term.  The solve reaches the tolerance (FP64 residual), theta
    matches the closed form, and it takes the three-term solve's Newton-Schulz
    steps within one."""
    p = make_spd(n, kappa, nrhs=nrhs, seed=1)
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    runs = {}
    for xp in (0, 1):
        with nsgb.Context(n, order=8, couple_frob=1.0, xp_bf16x2=xp) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=80, tol=1e-10)
        assert r.status == nsgb.NS_OK, (xp, r.stats.res_history()[-5:])
        th = r.theta.cpu().numpy()
        assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10 + 0.5 * 2.0 ** -53 * kappa
        assert rel(th, tstar) <= 10 * kappa * 1e-10
        runs[xp] = r.stats
    assert abs(runs[1].ns_iters - runs[0].ns_iters) <= 1


@pytest.mark.parametrize("kappa,nrhs", [(1e4, 4), (1e5, 4)])
def test_bf16_powers_in_split_steps(kappa, nrhs):
    """Option pow_bf16: in bf16x3 steps the powers F^{2^{j+1}} run as one bf16
    pass.  On the n = 4096 systems the solve reaches the tolerance with the same
    Newton-Schulz steps and sweeps as with split powers, and theta matches the
    closed form."""
    p = make_spd(4096, kappa, nrhs=nrhs, seed=1)
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    steps = {}
    for pb in (0, 1):
        with nsgb.Context(4096, order=8, couple_frob=1.0, pow_bf16=pb) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=80, tol=1e-10)
        th = r.theta.cpu().numpy()
        assert r.status == nsgb.NS_OK, (pb, r.stats.res_history())
        assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
        assert rel(th, tstar) <= 10 * kappa * 1e-10
        steps[pb] = (r.stats.ns_iters, r.stats.sweeps)
    assert steps[1] == steps[0]


def test_bench_size_solve():
    """The benchmark workload: n = 4096, kappa = 1e4, 4 RHS, order 8, mixed
    precision; the residual is recomputed in FP64 by the oracle and theta is
    compared with the closed-form solution."""
    p = make_spd(4096, 1e4, nrhs=4, seed=1)
    with nsgb.Context(4096, order=8) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
    th = r.theta.cpu().numpy()
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    assert rel(th, tstar) <= 10 * 1e4 * 1e-10


# ---------------------------------------------------------------------------
# Parity at sizes where the plain FP64 path runs its large-tile product kernel
# (k_gemm_f64, from 76 output tiles of 64 x 64 on, i.e. n >= 576)
# ---------------------------------------------------------------------------
def test_fp64_solve_n1024_matches_oracle():
    """n = 1024, kappa = 1e4, 2 RHS, order 8 factorized, 9 coupled NS steps
    (F_0^{8^9} is far below rounding here) + 3 sweeps, Richardson from the
    first step.  The FP64 attainable accuracy of G is ~kappa u sqrt(n), above
    1e-12, so G and theta are held to max(1e-12, 2 x the oracle's own error
    against the closed forms A^-1 = Q diag(1/lambda) Q^T and theta* = A^-1 B)."""
    n, K, S = 1024, 9, 3
    p = make_spd(n, 1e4, nrhs=2, seed=31)
    ref = O.ns_richardson_solve(p.A, p.B, order=8, ns_iters=K, max_sweeps=S)
    Ainv = (p.Q / p.lam) @ p.Q.T
    tstar = Ainv @ p.B
    with nsgb.Context(n, order=8, precision=nsgb.NS_FP64, ns_stop=0, max_sweeps=S) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=K, tol=0.0)
        G, st = ctx.invert(tens(p.A), iters=K)
    th = r.theta.cpu().numpy()
    Gg = G.cpu().numpy()
    tol_G = max(1e-12, 2 * rel(ref.G, Ainv))
    tol_t = max(1e-12, 2 * rel(ref.theta, tstar))
    assert rel(Gg, ref.G) <= tol_G, (rel(Gg, ref.G), tol_G)
    assert rel(th, ref.theta) <= tol_t, (rel(th, ref.theta), tol_t)
    # the GPU iterate is as close to the closed form as the oracle's
    assert rel(Gg, Ainv) <= tol_G
    assert r.stats.sweeps == ref.sweeps
    assert np.allclose(st.frob_history(), ref.frob_E, rtol=1e-8, atol=1e-10)
    assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-12


# ---------------------------------------------------------------------------
# Reduced precision: a stated bound on G itself against the FP64 oracle
# ---------------------------------------------------------------------------
# Error model (the paper fixes no precision; this is the library's own bound).
# One tensor-core product in precision p carries a relative error of at most
# about eps_p = eps_operand(p) + 2^-24 sqrt(K) per entry: the operand split
# (bf16: RN to 8 bits, 2^-8 counting both operands; bf16x3: the dropped
# lo*lo term and the 16-bit lo part, 2^-16; bf16x6: a binary32 operand is
# exact, the dropped third-order terms 2^-23) plus the f32 accumulation of K
# terms (random-walk size).  Two consequences for the Newton-Schulz iterate:
#  * while it is far from A^-1, every product adds ~eps_p to the relative error
#    of G (the slow eigen-directions of G grow by the order each step, as their
#    errors do), so after P products ||G_p - G||_2 / ||G||_2 <= 4 eps_p P;
#  * at the precision floor, the computed F = I - A G is off by
#    E ~ eps_p |A||G|, ||E||_2 <~ eps_p kappa_2, and the next step inherits
#    -E, so ||I - A G_p||_2 <= 4 eps_p kappa_2 and ||G_p - A^-1||_2 <=
#    ||A^-1||_2 ||I - A G_p||_2.
# The factor 4 is the safety margin over the model's typical size.
EPS_OPERAND = {nsgb.NS_BF16: 2.0 ** -8, nsgb.NS_BF16X3: 2.0 ** -16, nsgb.NS_BF16X6: 2.0 ** -23}


def eps_p(prec, K):
    return EPS_OPERAND[prec] + 2.0 ** -24 * math.sqrt(K)


def rel2(a, b):
    return float(np.linalg.norm(a - b, 2) / np.linalg.norm(b, 2))


@pytest.mark.parametrize("prec,kappa,k_floor", [(nsgb.NS_BF16, 10.0, 8), (nsgb.NS_BF16X3, 1e3, 10),
                                                (nsgb.NS_BF16X6, 1e4, 12)])
def test_mixed_G_within_per_precision_bound(prec, kappa, k_floor):
    """G after k fixed-precision order-4 steps against oracle.ns_invert (FP64)
    on the same system (n = 300: a ragged last tile): early (k = 2, 8 products)
    within 4 eps_p P, and at the floor within 4 eps_p (P + kappa) with
    ||I - A G_p||_2, formed here in FP64, within 4 eps_p kappa."""
    n = 300
    p = make_spd(n, kappa, seed=32)
    Ainv = (p.Q / p.lam) @ p.Q.T
    e = eps_p(prec, n)
    for k in (2, k_floor):
        with nsgb.Context(n, order=4, precision=prec, ns_stop=0) as ctx:
            G, _ = ctx.invert(tens(p.A), iters=k)
        Gp = G.cpu().numpy()
        Go, _ = O.ns_invert(p.A, order=4, iters=k)
        P = 4 * k
        if k == 2:
            assert rel2(Gp, Go) <= 4 * e * P, (k, rel2(Gp, Go), 4 * e * P)
        else:
            F2 = float(np.linalg.norm(np.eye(n) - p.A @ Gp, 2))
            assert F2 <= 4 * e * kappa, (F2, 4 * e * kappa)
            assert rel2(Gp, Go) <= 4 * e * (P + kappa), (rel2(Gp, Go), 4 * e * (P + kappa))
            assert np.linalg.norm(Gp - Ainv, 2) <= np.linalg.norm(Ainv, 2) * F2 * (1 + 1e-9)


@pytest.mark.parametrize("n_order,rates", [(2, [2]), (2, [2, 3])])
@pytest.mark.parametrize("prec", [nsgb.NS_BF16X3, nsgb.NS_BF16])
def test_mixed_composite_matches_oracle(prec, n_order, rates):
    """The composite mixed-rate method (Section 5, eqs. gkgen1-ga1) on the
    tensor cores (T_i loops, Gamma_i = I - T_i A, T_c, prefix products,
    G = T_c + Gamma_c X) against the oracle's composite_iterate: after K = 3
    steps G is within 4 eps_p P of the FP64 iterate (P = the oracle's product
    count); the GPU's F_K follows the exponent law of eq. gem1 as closely."""
    n = 256
    p = make_spd(n, 100.0, seed=33)
    K = 3
    with nsgb.Context(n, order=n_order, rates=rates, precision=prec, ns_stop=0) as ctx:
        G, _ = ctx.invert(tens(p.A), iters=K)
    Gp = G.cpu().numpy()
    cnt = O.MMCount()
    st = O.composite_init(O.alpha_frobenius(p.A) * np.eye(n), len(rates))
    for _ in range(K):
        st = O.composite_iterate(p.A, st, n_order, rates, cnt)
    bound = 4 * eps_p(prec, n) * cnt.n
    assert rel2(Gp, st.G) <= bound, (rel2(Gp, st.G), bound)
    ek = O.composite_exponents(n_order, rates, 1, K)[K]
    a = O.alpha_frobenius(p.A)
    Fk = (p.Q * (1 - a * p.lam) ** ek) @ p.Q.T
    Fo = np.eye(n) - st.G @ p.A
    Fg = np.eye(n) - Gp @ p.A
    assert np.linalg.norm(Fo - Fk) <= 1e-11 * n
    assert np.linalg.norm(Fg - Fk, 2) <= bound * np.linalg.norm(p.A, 2) * np.linalg.norm(st.G, 2)


@pytest.mark.parametrize("rates", [[2], [2, 3]])
def test_mixed_composite_solve_reaches_tolerance(rates):
    """Composite order 2 with rates {2} and {2, 3} through AUTO precision and
    FP64 Richardson: the relative residual (recomputed in FP64) reaches 1e-10
    and theta lies within 10 kappa 1e-10 of the closed-form solution."""
    n, kappa = 520, 1e3
    p = make_spd(n, kappa, nrhs=2, seed=34)
    with nsgb.Context(n, order=2, rates=rates) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
    th = r.theta.cpu().numpy()
    assert r.status == nsgb.NS_OK, r.stats.res_history()
    assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
    tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
    assert rel(th, tstar) <= 10 * kappa * 1e-10


# ---------------------------------------------------------------- TF32 products
def test_tf32_solve_reaches_tolerance():
    """NS_TF32: every product a TF32 tcgen05 pass (CTA pairs, odd row-tile count
    at n = 300); FP64 Richardson wins the accuracy back; G within the stated
    per-precision bound (eps_tf32 = 2^-10 + 2^-24 sqrt(K), as for bf16 with
    TF32's 11 significant bits) at the floor."""
    for n, kappa in ((300, 1e3), (1000, 1e4)):
        p = make_spd(n, kappa, nrhs=2, seed=40)
        with nsgb.Context(n, order=8, precision=nsgb.NS_TF32) as ctx:
            r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
        th = r.theta.cpu().numpy()
        assert r.status == nsgb.NS_OK, r.stats.res_history()
        assert set(r.stats.prec_history()) == {nsgb.NS_TF32}
        assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
        tstar = (p.Q / p.lam) @ (p.Q.T @ p.B)
        assert rel(th, tstar) <= 10 * kappa * 1e-10
    n, kappa = 300, 100.0
    p = make_spd(n, kappa, seed=41)
    with nsgb.Context(n, order=4, precision=nsgb.NS_TF32, ns_stop=0) as ctx:
        G, _ = ctx.invert(tens(p.A), iters=10)
    Gp = G.cpu().numpy()
    e = 2.0 ** -10 + 2.0 ** -24 * math.sqrt(n)
    F2 = float(np.linalg.norm(np.eye(n) - p.A @ Gp, 2))
    assert F2 <= 4 * e * kappa, (F2, 4 * e * kappa)


def test_auto_tf32_rung_reaches_tolerance():
    """AUTO with tf32_rung: bf16 steps, then TF32 once bf16's contraction
    worsens, then bf16x3; the residual reaches 1e-10 and the precision
    history shows the ladder in order."""
    n, kappa = 1024, 1e5
    p = make_spd(n, kappa, nrhs=2, seed=42)
    with nsgb.Context(n, order=8, tf32_rung=1, couple_frob=1.0) as ctx:
        r = ctx.solve(tens(p.A), tens(p.B), iters=60, tol=1e-10)
    th = r.theta.cpu().numpy()
    assert r.status == nsgb.NS_OK, (r.stats.prec_history(), r.stats.res_history())
    assert float(np.max(O.rel_residual(p.A, th, p.B))) <= 1e-10
    hist = r.stats.prec_history()
    assert nsgb.NS_TF32 in hist and hist[0] == nsgb.NS_BF16, hist
    order = {nsgb.NS_BF16: 0, nsgb.NS_TF32: 1, nsgb.NS_BF16X3: 2, nsgb.NS_BF16X6: 3}
    ranks = [order[h] for h in hist]
    assert ranks == sorted(ranks), hist
