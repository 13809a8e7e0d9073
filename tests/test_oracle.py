"""Pins for the FP64 oracle: every check compares the oracle with something
other than itself -- eigen-decomposition closed forms, the paper's printed
counts, brute-force series on tiny matrices, scipy's Cholesky solve, torch's
bfloat16 conversion -- so that a dropped term, a wrong sign, a wrong index or a
transposed operand fails at least one of them (see also test_oracle_mutations)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from workloads import make_spd

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def spd(n=20, kappa=30.0, nrhs=2, seed=0):
    return make_spd(n, kappa, nrhs=nrhs, seed=seed)


def sdd_spd(n=12, seed=3):
    """Strictly diagonally dominant SPD matrix with a non-constant diagonal, so
    the Jacobi preconditioner does not commute with A (Section 2)."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(-1, 1, (n, n))
    M = 0.5 * (M + M.T)
    np.fill_diagonal(M, 0.0)
    d = np.abs(M).sum(1) + rng.uniform(0.5, 3.0, n)
    return M + np.diag(d)


def eig_power(prob, alpha, e):
    """(I - alpha A)^e from the generator's spectral factors (closed form)."""
    Q, lam = prob.Q, prob.lam
    return (Q * (1.0 - alpha * lam) ** e) @ Q.T


def eig_series(prob, alpha, h):
    """{sum_{j<h} (I - alpha A)^j} alpha I in closed form."""
    Q, lam = prob.Q, prob.lam
    x = 1.0 - alpha * lam
    s = np.array([alpha * sum(xi ** j for j in range(h)) for xi in x])
    return (Q * s) @ Q.T


def fro(X):
    return float(np.sqrt(np.sum(X * X)))


# ---------------------------------------------------------------- Section 2

def test_alpha_frobenius_gives_contraction():
    p = spd(16, 50.0)
    a = O.alpha_frobenius(p.A)
    assert a == pytest.approx(1.0 / np.linalg.norm(p.A, "fro"), rel=1e-15)
    x = 1.0 - a * p.lam
    assert np.all(x >= 0) and np.all(x < 1)


def test_alpha_inf_matches_definition_and_contracts():
    p = spd(16, 50.0)
    a = O.alpha_inf(p.A)
    ninf = np.linalg.norm(p.A, np.inf)
    assert 1.0 / a == pytest.approx(ninf / 2 * (1 + 2e-8), rel=1e-14)
    # 2S - A = ||A||_inf I + 2 eps I - A is PD => rho(I - a A) < 1 (eq. spro)
    ev = np.linalg.eigvalsh(np.eye(16) - a * p.A)
    assert np.max(np.abs(ev)) < 1


def test_jacobi_splitting_contracts_for_sdd():
    A = sdd_spd()
    Sinv = O.jacobi_preconditioner(A)
    assert np.allclose(np.diag(Sinv) * np.diag(A), 1.0)
    rho = np.max(np.abs(np.linalg.eigvals(O.splitting_residual(A, Sinv))))
    assert rho < 1


# ---------------------------------------------------------------- Section 3

@pytest.mark.parametrize("order", [2, 3, 4, 8])
@pytest.mark.parametrize("form", ["factorized", "horner"])
def test_exponent_law_plain_ns(order, form):
    """eq. fk1: I - G_k A = F_0^{n^k}, and the right residual I - A G_k too."""
    p = spd(20, 30.0)
    a = O.alpha_frobenius(p.A)
    G = a * np.eye(20)
    for k in range(1, 4):
        G, _ = O.ns_step(p.A, G, order, form)
        ref = eig_power(p, a, order ** k)
        assert fro(O.residual_left(G, p.A) - ref) <= 1e-12
        assert fro(O.residual_right(p.A, G) - ref) <= 1e-12


@pytest.mark.parametrize("order", [2, 3, 5])
def test_classical_step_exponent_law(order):
    """eq. ns with eq. fk1 on the left form (Horner evaluation)."""
    p = spd(14, 20.0, seed=4)
    a = O.alpha_frobenius(p.A)
    G = a * np.eye(14)
    for k in range(1, 4):
        G = O.ns_classical_step(G, p.A, order)
        assert fro(O.residual_left(G, p.A) - eig_power(p, a, order ** k)) <= 1e-12


@pytest.mark.parametrize("p_,w", [(0, 3), (1, 1), (1, 2), (2, 2), (3, 2), (2, 3)])
def test_initial_series_g01_g03(p_, w):
    """eqs. g01-g03 with S^{-1} = alpha I: G0 = sum_{j<h} (S^{-1}D)^j S^{-1},
    F0 = (S^{-1}D)^h."""
    p = spd(12, 10.0, seed=5)
    a = O.alpha_frobenius(p.A)
    G0, F0 = O.initial_series(p.A, a * np.eye(12), p_, w)
    h = w * (p_ + 1)
    assert fro(G0 - eig_series(p, a, h)) <= 1e-13
    assert fro(F0 - eig_power(p, a, h)) <= 1e-13


def test_special_case_n_w_m_equal_one():
    """Remark after eq. ga1: for n = w = m = 1 the composite method is
    G_k = (S^{-1}D) G_{k-1} + S^{-1}."""
    p = spd(10, 8.0, seed=6)
    a = O.alpha_frobenius(p.A)
    Sinv = a * np.eye(10)
    SD = O.splitting_residual(p.A, Sinv)
    st = O.composite_init(Sinv, 1)
    G = Sinv.copy()
    for _ in range(4):
        st = O.composite_iterate(p.A, st, 1, [1])
        G = SD @ G + Sinv
        assert fro(st.G - G) <= 1e-14 * max(1, fro(G))


# ---------------------------------------------------------------- Section 4

def brute_series(X, A, h):
    """sum_{j<h} Y^j X by explicit powers (brute force)."""
    Y = np.eye(A.shape[0]) - X @ A
    out = np.zeros_like(X)
    P = np.eye(A.shape[0])
    for _ in range(h):
        out += P @ X
        P = P @ Y
    return out


@pytest.mark.parametrize("h", list(range(2, 20)))
def test_toolkit_rows_equal_series(h):
    """Tables t1-t3: every factorized row equals the unfactorized series
    (eq. z1a), both for a commuting X = alpha I (closed form) and a
    non-commuting Jacobi X (brute force)."""
    p = spd(10, 6.0, seed=7)
    a = O.alpha_frobenius(p.A)
    Z = O.toolkit(a * np.eye(10), p.A, h)
    assert fro(Z - eig_series(p, a, h)) <= 1e-13 * max(1, fro(Z))
    A = sdd_spd(9)
    X = O.jacobi_preconditioner(A)
    Z = O.toolkit(X, A, h)
    ref = brute_series(X, A, h)
    assert fro(Z - ref) <= 1e-12 * max(1, fro(ref))


def test_toolkit_table_matches_paper_rows():
    rows = GOLD["toolkit_rows"]["rows"]
    assert {int(k): tuple(v) for k, v in rows.items()} == O.TOOLKIT_TABLE
    for h, (kind, p_, w) in O.TOOLKIT_TABLE.items():
        assert h == w * (p_ + 1) + (1 if kind == "z1" else 0)   # eqs. hape, hape1


@pytest.mark.parametrize("p_,w", [(1, 1), (2, 1), (0, 2), (0, 4), (1, 2), (3, 2), (2, 3), (4, 2), (8, 5),
                                  (5, 3), (2, 6), (8, 2), (1, 9)])
def test_unified_factorization_order_and_mmm(p_, w):
    """eqs. h1, np1: order w(p+1) in p + w + 1 mmm (p + 1 if w = 1, w if p = 0)."""
    pr = spd(8, 4.0, seed=8)
    a = O.alpha_frobenius(pr.A)
    cnt = O.MMCount()
    Z = O.unified_factorization(a * np.eye(8), pr.A, p_, w, cnt)
    h = w * (p_ + 1)
    assert fro(Z - eig_series(pr, a, h)) <= 1e-13 * max(1, fro(Z))
    expect = p_ + 1 if w == 1 else (w if p_ == 0 else p_ + w + 1)
    assert cnt.n == expect


def test_order18_four_factorizations():
    """Appendix: the four (p, w) choices for order 18 give the same series."""
    pr = spd(8, 4.0, seed=9)
    a = O.alpha_frobenius(pr.A)
    ref = eig_series(pr, a, 18)
    for p_, w in GOLD["order18_alternatives"]["pw"]:
        assert w * (p_ + 1) == 18
        Z = O.unified_factorization(a * np.eye(8), pr.A, p_, w)
        assert fro(Z - ref) <= 1e-13 * fro(ref)


def test_binary_chain_mmm_counts_match_paper():
    """Appendix: orders 4 and 8 in 4 and 6 mmm; order 2 in 2; order 3 in 3."""
    pr = spd(8, 4.0)
    G = O.alpha_frobenius(pr.A) * np.eye(8)
    for order, mmm in GOLD["binary_orders_mmm"]["values"].items():
        cnt = O.MMCount()
        O.ns_step(pr.A, G, int(order), "factorized", "square", cnt)
        assert cnt.n == mmm
        cnt = O.MMCount()
        O.ns_step(pr.A, G, int(order), "factorized", "residual", cnt)
        assert cnt.n == mmm
    for order, mmm in ((2, 2), (3, 3)):
        cnt = O.MMCount()
        O.ns_step(pr.A, G, order, "factorized", "square", cnt)
        assert cnt.n == mmm


def test_pow_modes_agree():
    """eq. ua1: Y^{p+1} = I - U A equals the square of Y (exact arithmetic)."""
    pr = spd(16, 20.0, seed=2)
    G = O.alpha_frobenius(pr.A) * np.eye(16)
    for order in (4, 8):
        G1, _ = O.ns_step(pr.A, G, order, "factorized", "square")
        G2, _ = O.ns_step(pr.A, G, order, "factorized", "residual")
        assert fro(G1 - G2) <= 1e-14 * fro(G1)


def test_nested_order45_ten_mmm():
    """Section 4 example, eqs. ex1-ex3."""
    g = GOLD["nested_order45"]
    pr = spd(8, 3.0, seed=10)
    a = O.alpha_frobenius(pr.A)
    cnt = O.MMCount()
    Z = O.nested_order45(a * np.eye(8), pr.A, cnt)
    assert cnt.n == g["mmm"]
    assert fro(Z - eig_series(pr, a, g["order"])) <= 1e-13 * fro(Z)
    A = sdd_spd(7, seed=11)
    X = O.jacobi_preconditioner(A)
    Z = O.nested_order45(X, A)
    ref = brute_series(X, A, 45)
    assert fro(Z - ref) <= 1e-11 * fro(ref)
    # eq. ex1 alone: p = 8, w = 5 costs p + w + 1 = 14 mmm
    cnt = O.MMCount()
    O.unified_factorization(a * np.eye(8), pr.A, g["ex1_p"], g["ex1_w"], cnt)
    assert cnt.n == g["ex1_mmm"]
    # efficiency index of eq. ei generalised to (order, mmm): 45^(1/10)
    assert round(g["order"] ** (1.0 / g["mmm"]), 4) == g["ei"]


def test_efficiency_index_order2():
    """eq. ei with p = 1, w = 1: EI = 2^(1/2) (Section 4)."""
    p_, w = 1, 1
    ei = (w * (p_ + 1)) ** (1.0 / (p_ + w))   # order 2 costs p + 1 = 2 mmm
    assert round(ei, 4) == GOLD["ei_order2"]["value"]


def test_identity_ex3():
    """eq. ex3: I + Y + Y^2 = 3I + (XA)(-3I + XA) with Y = I - XA."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((6, 6))
    A = rng.standard_normal((6, 6))
    I = np.eye(6)
    Y = I - X @ A
    assert fro(I + Y + Y @ Y - (3 * I + (X @ A) @ (-3 * I + X @ A))) <= 1e-12


def test_push_through_right_equals_left_noncommuting():
    """The right chain G (I + F)(I + F^2)... with F = I - A G equals the left
    series {sum_j (I - G A)^j} G for a G0 that does not commute with A."""
    A = sdd_spd(10, seed=12)
    G = O.jacobi_preconditioner(A)
    assert fro(G @ A - A @ G) > 1e-3
    for order in (2, 3, 4, 8):
        Gr, _ = O.ns_step(A, G, order, "factorized")
        Gl = O.ns_classical_step(G, A, order)
        assert fro(Gr - Gl) <= 1e-13 * fro(Gl)


def test_commutation_with_scalar_g0():
    pr = spd(24, 50.0, seed=13)
    G = O.alpha_frobenius(pr.A) * np.eye(24)
    for order in (2, 3, 4, 8):
        Gk = G
        for _ in range(3):
            Gk, _ = O.ns_step(pr.A, Gk, order)
            assert fro(Gk @ pr.A - pr.A @ Gk) <= 1e-13 * fro(pr.A) * fro(Gk)


def test_brute_force_tiny_order2():
    """N = 4, order 2, k steps: G_k = sum_{j < 2^k} F_0^j G_0 (eq. ser1 with
    h = 1, n = 2), by explicit powers."""
    pr = spd(4, 5.0, seed=14)
    A = pr.A
    G0 = O.alpha_frobenius(A) * np.eye(4)
    F0 = np.eye(4) - G0 @ A
    G = G0
    for k in range(1, 5):
        G, _ = O.ns_step(A, G, 2)
        ref = sum(np.linalg.matrix_power(F0, j) for j in range(2 ** k)) @ G0
        assert fro(G - ref) <= 1e-13 * fro(ref)


@pytest.mark.parametrize("order", [2, 3, 4, 8])
def test_converges_to_closed_form_inverse(order):
    pr = spd(16, 10.0, seed=15)
    Ainv = (pr.Q / pr.lam) @ pr.Q.T
    G, norms = O.ns_invert(pr.A, order=order, iters=40 if order == 2 else 20)
    assert fro(G - Ainv) / fro(Ainv) <= 1e-13
    assert norms[0] > norms[-1]


# ---------------------------------------------------------------- Section 5

@pytest.mark.parametrize("n,rates", [(2, [2]), (2, [2, 3]), (3, [2]), (2, [3, 2, 2])])
def test_composite_exponent_law(n, rates):
    """eqs. rel1, gem1 with eqs. ti/ga1 (x_i = m_i^k): F_k = (S^{-1}D)^{e_k},
    e_0 = 1, e_k = sum_i m_i^k + n e_{k-1}."""
    pr = spd(12, 6.0, seed=16)
    a = O.alpha_frobenius(pr.A)
    st = O.composite_init(a * np.eye(12), len(rates))
    e = O.composite_exponents(n, rates, 1, 3)
    for k in range(1, 4):
        st = O.composite_iterate(pr.A, st, n, rates)
        for Ti, m in zip(st.T, rates):
            assert fro(O.residual_left(Ti, pr.A) - eig_power(pr, a, m ** k)) <= 1e-12
        assert fro(O.residual_left(st.G, pr.A) - eig_power(pr, a, e[k])) <= 1e-12


def test_composite_exponent_values():
    """n = 2, rates (2, 3): e = 1, 7, 27, 89 (worked by hand from eq. gem1)."""
    assert O.composite_exponents(2, [2, 3], 1, 3) == [1, 7, 27, 89]


def test_composite_telescoping_noncommuting():
    """eq. rel1 T_c A = I - Gamma_c and eq. gem1 F_k = Gamma_c F_{k-1}^n hold
    for any T_i, including ones that do not commute with A."""
    A = sdd_spd(9, seed=17)
    rng = np.random.default_rng(1)
    T = [O.jacobi_preconditioner(A) + 0.01 * rng.standard_normal((9, 9)) for _ in range(3)]
    Tc, Gc = O.composite_combine(A, T)
    assert fro(Tc @ A - (np.eye(9) - Gc)) <= 1e-13 * fro(Tc @ A)
    Gprev = O.jacobi_preconditioner(A)
    Fprev = np.eye(9) - Gprev @ A
    G = O.composite_step(A, Gprev, T, 3)
    assert fro((np.eye(9) - G @ A) - Gc @ np.linalg.matrix_power(Fprev, 3)) <= 1e-13


@pytest.mark.parametrize("n", [2, 3])
def test_double_ns_exponent(n):
    """eq. ermoex1: F_k = (S^{-1}D)^{h (k n^{k+1} + n^k)} with G0 = S^{-1} (h = 1)
    and with the order-2 initial series (h = 2)."""
    pr = spd(12, 5.0, seed=18)
    a = O.alpha_frobenius(pr.A)
    for h, G0 in ((1, a * np.eye(12)), (2, O.initial_series(pr.A, a * np.eye(12), 1, 1)[0])):
        st = O.double_ns_init(pr.A, G0, n)
        for k in range(1, 3):
            st = O.double_ns_iterate(pr.A, st, n)
            e = O.double_ns_exponent(n, h, k)
            assert fro(st.F - eig_power(pr, a, e)) <= 1e-12
            assert fro(st.GamN - eig_power(pr, a, h * n ** (k + 1))) <= 1e-12


def test_double_ns_exponent_values():
    assert [O.double_ns_exponent(3, 1, k) for k in (1, 2, 3)] == [12, 63, 270]


# ---------------------------------------------------------------- Section 6

@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("updated", [False, True])
def test_richardson_error_model(order, updated):
    """theta_{k+1} - theta_* = (I - G_k A)(theta_k - theta_*) with
    I - G_k A = F_0^{n^k}, so after K coupled steps the error is
    F_0^{(n^K - 1)/(n - 1)} theta~_0 (G_k applied), or F_0^{n (n^K-1)/(n-1)}
    theta~_0 when G_{k+1} is applied (eq. ttk1 ordering)."""
    pr = spd(14, 8.0, nrhs=2, seed=19)
    a = O.alpha_frobenius(pr.A)
    tstar = np.linalg.solve(pr.A, pr.B)
    for K in (1, 2, 3):
        r = O.ns_richardson_solve(pr.A, pr.B, order=order, ns_iters=K, use_updated_G=updated)
        e = (order ** K - 1) // (order - 1)
        if updated:
            e *= order
        ref = eig_power(pr, a, e) @ (0 - tstar)
        assert fro((r.theta - tstar) - ref) <= 1e-11 * max(1, fro(tstar))


@pytest.mark.parametrize("order", [2, 4])
def test_delayed_coupling_error_model(order):
    """With the coupling delayed until the first G_k with ||I - A G_k||_F <= c,
    only the coupled steps k contribute their factor I - G_k A = F_0^{n^k}: the
    error after K steps is F_0^e theta~_0 with e the sum of n^k over the
    coupled k, and the steps before leave theta (and the residual record)
    alone."""
    pr = spd(16, 30.0, nrhs=2, seed=23)
    a = O.alpha_frobenius(pr.A)
    tstar = np.linalg.solve(pr.A, pr.B)
    K = 12 if order == 2 else 6
    for c in (1.0, 0.3):
        r = O.ns_richardson_solve(pr.A, pr.B, order=order, ns_iters=K, couple_frob=c)
        k0 = next(k for k in range(K) if r.frob_E[k] <= c)
        coupled = list(range(k0, K))
        assert 0 < len(coupled) < K
        e = sum(order ** k for k in coupled)
        ref = eig_power(pr, a, e) @ (0 - tstar)
        assert fro((r.theta - tstar) - ref) <= 1e-11 * max(1, fro(tstar))
        # one residual per coupled step plus the final one
        assert len(r.rel_res) == len(coupled) + 1 and r.sweeps == len(coupled)
    # c = 0 is the paper's coupling from the first step
    r0 = O.ns_richardson_solve(pr.A, pr.B, order=order, ns_iters=K, couple_frob=0.0)
    r1 = O.ns_richardson_solve(pr.A, pr.B, order=order, ns_iters=K)
    assert np.array_equal(r0.theta, r1.theta)


def test_rel_residual_closed_forms():
    """theta = (1 - t_c) A^{-1} b_c leaves r_c = t_c b_c, so the per-column
    relative residual is t_c exactly (to rounding); theta = 0 gives 1."""
    pr = spd(12, 10.0, nrhs=3, seed=23)
    t = np.array([1.0, 0.5, 1e-3])
    theta = np.linalg.solve(pr.A, pr.B) * (1.0 - t)[None, :]
    assert np.allclose(O.rel_residual(pr.A, theta, pr.B), t, rtol=1e-9, atol=1e-13)
    assert np.array_equal(O.rel_residual(pr.A, np.zeros_like(pr.B), pr.B), np.ones(3))


def test_richardson_converges_to_cholesky():
    pr = spd(32, 100.0, nrhs=3, seed=20)
    r = O.ns_richardson_solve(pr.A, pr.B, order=4, ns_iters=8, tol=1e-12, max_sweeps=50)
    ref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(pr.A), pr.B)
    assert r.converged
    assert fro(r.theta - ref) / fro(ref) <= 1e-10
    assert np.max(O.rel_residual(pr.A, r.theta, pr.B)) <= 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_accelerated_richardson_gamma(n):
    """eqs. riem1-riem6 (q = n): theta~_k = (S^{-1}D)^{gamma_k} theta~_0 with
    theta_0 = L_0 b."""
    pr = spd(10, 3.0, nrhs=1, seed=21)
    a = O.alpha_frobenius(pr.A)
    tstar = np.linalg.solve(pr.A, pr.B)
    st = O.double_ns_init(pr.A, a * np.eye(10), n)
    theta = st.L @ pr.B
    t0 = theta - tstar
    for k in range(1, 3):
        st = O.double_ns_iterate(pr.A, st, n)
        theta = O.accelerated_richardson_step(pr.A, pr.B, theta, st, q=n)
        g = O.accelerated_richardson_exponent(n, 1, k)
        assert g == int(g)
        ref = eig_power(pr, a, int(g)) @ t0
        assert fro((theta - tstar) - ref) <= 1e-12 * max(1.0, fro(t0))


def test_gamma_closed_form_equals_sum():
    """eq. riem6 equals the running sum of the per-step exponents of eq. riem4."""
    for n in (2, 3, 4):
        for k in (1, 2, 3):
            s = sum(i * n ** (i + 2) + 2 * n ** (i + 1) for i in range(1, k + 1))
            assert O.accelerated_richardson_exponent(n, 1, k) == s
    assert O.accelerated_richardson_exponent(2, 1, 1) == 16


def test_omega_recursive_equals_direct():
    """eq. gkrecu1 and the second part (L_k, Gamma_k^n) reproduce eq. redttk2."""
    pr = spd(10, 4.0, seed=22)
    a = O.alpha_frobenius(pr.A)
    n = 2
    st = O.double_ns_init(pr.A, a * np.eye(10), n)
    st = O.double_ns_iterate(pr.A, st, n)
    SG = O.ns_classical_step(st.G, pr.A, n)
    omega = st.L + st.GamN @ SG
    for _ in range(2):
        st_next = O.double_ns_iterate(pr.A, st, n)
        omega, SG, GamN, L, G = O.omega_recursive(pr.A, omega, SG, st.GamN, st.L, n)
        direct = st_next.L + st_next.GamN @ O.ns_classical_step(st_next.G, pr.A, n)
        assert fro(G - st_next.G) <= 1e-13 * fro(G)
        assert fro(omega - direct) <= 1e-13 * fro(direct)
        st = st_next


# ---------------------------------------------------------------- precision defs

def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, -1.0e-40, 1e-45])])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    got = O.round_bf16(x32)
    assert np.array_equal(got, ref)


def _tf32_nearest_brute(x32):
    """Nearest TF32 value of each binary32 x by explicit comparison of its two
    TF32 neighbours in magnitude (ties away from zero), in float64."""
    out = np.empty_like(x32, dtype=np.float64)
    for i, v in enumerate(x32):
        if np.isnan(v):
            out[i] = np.nan
            continue
        m = abs(float(v))
        u = np.array([m], dtype=np.float32).view(np.uint32)[0]
        lo_bits = np.uint32(u & np.uint32(0xFFFFE000))
        lo = float(np.array([lo_bits], dtype=np.uint32).view(np.float32)[0])
        if lo == m:
            r = m
        else:
            hi_bits = np.uint64(lo_bits) + np.uint64(0x2000)
            hi = float(np.array([hi_bits], dtype=np.uint64).astype(np.uint32).view(np.float32)[0]) \
                if hi_bits < 0x7F800000 else np.inf
            dl, dh = m - lo, hi - m
            if hi_bits >= 0x7F800000:
                # beyond the largest TF32 value: the half-way point to 2^128
                r = np.inf if m >= lo + 2.0 ** 116 else lo  # half the TF32 spacing 2^117 at 2^127
            else:
                r = hi if dh <= dl else lo
        out[i] = -r if v < 0 else r
    return out


def test_round_tf32_nearest_ties_away():
    """TF32 rounding (10 stored significand bits): worked cases -- ties go away
    from zero, not to even -- and agreement with a brute-force search of the
    two TF32 neighbours on random and edge values."""
    one = 1.0
    cases = {one + 2.0 ** -12: one, one + 2.0 ** -11: one + 2.0 ** -10,       # tie -> away
             one + 3 * 2.0 ** -11: one + 2.0 ** -9,                             # tie (odd) -> away
             one + 2.0 ** -11 + 2.0 ** -23: one + 2.0 ** -10,
             -(one + 2.0 ** -11): -(one + 2.0 ** -10), 0.0: 0.0, 2.0 ** -130: 2.0 ** -130,
             3.4028234663852886e38: np.inf}
    for x, want in cases.items():
        assert O.round_tf32(np.array([x]))[0] == want, (x, O.round_tf32(np.array([x]))[0], want)
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.uniform(-35, 35, 3000),
                        np.array([1e-45, -3e-39, 65504.0, 1.0 + 2.0 ** -11, -0.0])])
    x32 = x.astype(np.float32)
    got = O.round_tf32(x32)
    ref = _tf32_nearest_brute(x32)
    assert np.array_equal(got, ref)
    fin = np.isfinite(got) & (np.abs(x32) > 1e-37)
    assert np.all(np.abs(got[fin] - x32[fin]) <= 2.0 ** -11 * np.abs(x32[fin].astype(np.float64)))
    assert np.all((got[np.isfinite(got)].astype(np.float32).view(np.uint32) & 0x1FFF) == 0)


def test_tf32_split_product():
    """The tf32 product is the exact product of the rounded operands: equal to
    a float64 product of round_tf32 values, off the float64 product by at most
    ~2 2^-11 |L||R|, and exact for operands with 11 significant bits."""
    rng = np.random.default_rng(4)
    L, R = rng.standard_normal((12, 40)), rng.standard_normal((40, 7))
    P = O.split_product(L, R, "tf32")
    assert np.array_equal(P, O.round_tf32(L) @ O.round_tf32(R))
    ab = np.abs(L) @ np.abs(R)
    assert np.all(np.abs(P - L @ R) <= 2.1 * 2.0 ** -11 * ab)
    Li = rng.integers(-1024, 1024, (5, 9)).astype(float)
    Ri = rng.integers(-1024, 1024, (9, 3)).astype(float)
    assert np.array_equal(O.split_product(Li, Ri, "tf32"), Li @ Ri)
    assert np.array_equal(O.split_abs_product(Li, Ri, "tf32"), np.abs(Li) @ np.abs(Ri))


def test_split_bf16_error_bound():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(10000)
    x32 = O.round_f32(x)
    hi, lo = O.split_bf16(x)
    assert np.array_equal(O.round_bf16(hi), hi) and np.array_equal(O.round_bf16(lo), lo)
    # bf16 keeps 8 significant bits: |x32 - hi| <= 2^-8 |x32| (half an ulp),
    # and lo rounds that difference to 8 bits again
    assert np.all(np.abs(x32 - hi) <= 2.0 ** -8 * np.abs(x32))
    assert np.all(np.abs(x32 - hi - lo) <= 2.0 ** -16 * np.abs(x32))


def test_split_product_terms():
    """bf16x3 drops only lo*lo: its error against the binary32 product is
    bounded by the three neglected pieces."""
    rng = np.random.default_rng(2)
    L = rng.standard_normal((8, 16))
    R = rng.standard_normal((16, 5))
    Lh, Ll = O.split_bf16(L)
    Rh, Rl = O.split_bf16(R)
    assert np.array_equal(O.split_product(L, R, "bf16"), Lh @ Rh)
    d = O.split_product(L, R, "bf16x3") - (Lh @ Rh + Lh @ Rl + Ll @ Rh)
    assert np.max(np.abs(d)) <= 1e-14
    full = O.round_f32(L) @ O.round_f32(R)
    # dropped lo*lo (<= 2^-16) plus the two split remainders (<= 2^-16 each)
    bound = 3 * 2.0 ** -16 * (np.abs(L) @ np.abs(R)) + 1e-12
    assert np.all(np.abs(O.split_product(L, R, "bf16x3") - full) <= bound)


def test_split_product_two_terms():
    """bf16x2 keeps hi*hi and lo*hi: it is L's binary32 value (hi + lo to 16
    bits) times R's bfloat16 part.  For R exact in bfloat16 (Rlo = 0) it equals
    bf16x3 exactly; for L exact in bfloat16 it equals the one-pass bf16
    product; in general its error against the binary32 product is bounded by
    R's rounding (2^-8) plus L's split remainder (2^-16)."""
    rng = np.random.default_rng(21)
    L = rng.standard_normal((7, 24))
    R = rng.standard_normal((24, 6))
    Lh, Ll = O.split_bf16(L)
    Rh, _ = O.split_bf16(R)
    assert np.max(np.abs(O.split_product(L, R, "bf16x2") - (Lh + Ll) @ Rh)) <= 1e-13
    Rb = O.round_bf16(O.round_f32(R))
    assert np.max(np.abs(O.split_product(L, Rb, "bf16x2") - O.split_product(L, Rb, "bf16x3"))) <= 1e-13
    Lb = O.round_bf16(O.round_f32(L))
    assert np.array_equal(O.split_product(Lb, R, "bf16x2"), O.split_product(Lb, R, "bf16"))
    full = O.round_f32(L) @ O.round_f32(R)
    bound = (2.0 ** -8 + 2.0 ** -16) * (np.abs(L) @ np.abs(R)) + 1e-12
    assert np.all(np.abs(O.split_product(L, R, "bf16x2") - full) <= bound)
    ab = O.split_abs_product(L, R, "bf16x2")
    assert np.all(np.abs(O.split_product(L, R, "bf16x2")) <= ab)


def _step_with_rounded_factor(A, G, which):
    """One order-8 factorized step (three levels) with, for j >= 1, the factor
    `which` of X_j P_j rounded to bfloat16 (its low part dropped); returns
    F_{k+1} = I - A G_{k+1}."""
    n = A.shape[0]
    X, P = G, np.eye(n) - A @ G
    for j in range(3):
        if j >= 1 and which == "P":
            XP = X @ O.round_bf16(O.round_f32(P))
        elif j >= 1 and which == "X":
            XP = O.round_bf16(O.round_f32(X)) @ P
        else:
            XP = X @ P
        if j + 1 < 3:
            P = P @ P
        X = X + XP
    return np.eye(n) - A @ X


def test_dropped_power_bits_enter_unamplified():
    """The reading behind the reduced-precision powers and updates (bf16
    powers, two-term updates, fewer-digit slice powers): in a factorized step,
    an error in P_j = F_k^(2^j) reaches F_{k+1} = I - A G_{k+1} through
    A X_j ~ I, so rounding P_j to bfloat16 moves F_{k+1} by about
    2^-8 |F_k^(2^j)| whatever kappa, while rounding X_j by the same relative
    amount is amplified by ||A|| ||X_j|| ~ kappa."""
    dps = {}
    for kappa in (1e3, 1e5):
        p = spd(60, kappa, nrhs=1, seed=30)
        A = p.A
        G = O.alpha_frobenius(A) * np.eye(60)
        for _ in range(20):
            if np.linalg.norm(np.eye(60) - A @ G, 2) < 0.5:
                break
            G, _ = O.ns_step_binary(A, G, 3)
        F0 = np.eye(60) - A @ G
        Fe = _step_with_rounded_factor(A, G, "none")
        dp = np.linalg.norm(_step_with_rounded_factor(A, G, "P") - Fe)
        dx = np.linalg.norm(_step_with_rounded_factor(A, G, "X") - Fe)
        bound = 2.0 ** -8 * np.linalg.norm(A @ G, 2) * sum(np.linalg.norm(np.linalg.matrix_power(F0, 2 ** j))
                                                            for j in (1, 2))
        assert dp <= bound
        assert dx >= kappa / 100.0 * dp
        dps[kappa] = dp
    assert dps[1e5] <= 10.0 * dps[1e3]


def test_split3_exact_and_matches_torch():
    """hi + lo + lo2 reproduces binary32 exactly, each part is a bfloat16, and
    the parts equal torch's own bfloat16 rounding of the successive binary32
    remainders."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, 1.0, -1.0, 3.0e38, 1.0e-30]])
    x32 = O.round_f32(x)
    hi, lo, lo2 = O.split3_bf16(x)
    assert np.array_equal(hi + lo + lo2, x32)
    for part in (hi, lo, lo2):
        assert np.array_equal(O.round_bf16(part), part)
    t = torch.from_numpy(x32.astype(np.float32))
    th = t.to(torch.bfloat16).float()
    tl = (t - th).to(torch.bfloat16).float()
    t2 = (t - th - tl).to(torch.bfloat16).float()
    assert np.array_equal(th.double().numpy(), hi)
    assert np.array_equal(tl.double().numpy(), lo)
    assert np.array_equal(t2.double().numpy(), lo2)
    h2, l2 = O.split_bf16(x)
    assert np.array_equal(h2, hi) and np.array_equal(l2, lo)


def test_split_abs_product_bounds():
    """sum_k |L_ik||R_kj| over the split terms: for operands that bf16 holds
    exactly (lo = lo2 = 0) it is |L| |R| in every precision; in general it
    bounds the split product's magnitude and grows with the terms kept."""
    rng = np.random.default_rng(14)
    Lb = O.round_bf16(O.round_f32(rng.standard_normal((6, 20))))
    Rb = O.round_bf16(O.round_f32(rng.standard_normal((20, 4))))
    for prec in ("bf16", "bf16x3", "bf16x6"):
        assert np.array_equal(O.split_abs_product(Lb, Rb, prec), np.abs(Lb) @ np.abs(Rb))
    L = rng.standard_normal((6, 20))
    R = rng.standard_normal((20, 4))
    prev = None
    for prec in ("bf16", "bf16x3", "bf16x6"):
        ab = O.split_abs_product(L, R, prec)
        assert np.all(np.abs(O.split_product(L, R, prec)) <= ab)
        if prev is not None:
            assert np.all(ab >= prev)
        prev = ab


def test_split_product_x6_terms():
    """bf16x6 = the six terms of order <= 2; against the binary32 product its
    error is the three dropped terms only (each <= 2^-24 relative, as x32 =
    hi + lo + lo2 exactly), far below bf16x3's."""
    rng = np.random.default_rng(12)
    L = rng.standard_normal((9, 33))
    R = rng.standard_normal((33, 7))
    Lh, Ll, L2 = O.split3_bf16(L)
    Rh, Rl, R2 = O.split3_bf16(R)
    want = Lh @ Rh + Lh @ Rl + Ll @ Rh + Lh @ R2 + Ll @ Rl + L2 @ Rh
    assert np.max(np.abs(O.split_product(L, R, "bf16x6") - want)) <= 1e-13
    full = O.round_f32(L) @ O.round_f32(R)
    ab = np.abs(L) @ np.abs(R)
    err6 = np.abs(O.split_product(L, R, "bf16x6") - full)
    assert np.all(err6 <= 3 * 2.0 ** -24 * ab + 1e-13)
    err3 = np.abs(O.split_product(L, R, "bf16x3") - full)
    assert np.max(err3 / ab) > 100 * np.max(err6 / ab)


def test_gemm_epilogue_forms():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((5, 5))
    C = rng.standard_normal((5, 5))
    assert np.allclose(O.gemm_epilogue(P, -1.0, gamma=1.0), np.eye(5) - P)
    assert np.allclose(O.gemm_epilogue(P, 1.0, C, 1.0), C + P)


# ---------------------------------------------------------------- final inverse check
SM64 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.json")))


def test_splitmix64_published_outputs():
    for seed, outs in SM64["outputs"].items():
        for k, v in enumerate(outs):
            assert O.splitmix64(int(seed), k) == int(v, 0)


def test_rademacher_probes_follow_published_outputs():
    """Probe entries are -1 exactly where the published SplitMix64 output has
    its top bit set (a column of three probes per seed, and a row)."""
    for seed, outs in SM64["outputs"].items():
        want = np.array([-1.0 if int(v, 0) >> 63 else 1.0 for v in outs])
        assert np.array_equal(O.rademacher_probes(len(outs), 1, int(seed))[:, 0], want)
        assert np.array_equal(O.rademacher_probes(1, len(outs), int(seed))[0], want)


def test_rademacher_probes_balanced_and_uncorrelated():
    Z = O.rademacher_probes(64, 64, seed=99)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(float(np.mean(Z))) < 5 / math.sqrt(Z.size)           # P(-1) = 1/2
    C = Z.T @ Z / 64.0
    off = C[~np.eye(64, dtype=bool)]
    assert np.all(np.abs(off) < 5 / math.sqrt(64))                    # E z_j^T z_k = 0
    assert not np.array_equal(O.rademacher_probes(64, 4, 1), O.rademacher_probes(64, 4, 2))


def test_inverse_residual_closed_forms():
    p = spd(n=30, kappa=50.0, seed=21)
    c = 1.0 / p.lam.max()
    # G = c I: I - c A = Q diag(1 - c lambda) Q^T
    want = math.sqrt(float(np.sum((1.0 - c * p.lam) ** 2)))
    assert O.inverse_residual(p.A, c * np.eye(30)) == pytest.approx(want, rel=1e-12)
    Ainv = (p.Q / p.lam) @ p.Q.T
    assert O.inverse_residual(p.A, Ainv) < 1e-12


def test_hutchinson_exact_cases():
    rng = np.random.default_rng(5)
    n = 40
    # G = 0: every probe gives ||z||^2 = n
    assert O.inverse_residual_hutchinson(np.diag(rng.uniform(1, 2, n)), np.zeros((n, n)), 3, 7) == math.sqrt(n)
    # diagonal I - A G: z_i^2 = 1 makes every probe exact
    A = np.diag(rng.uniform(1, 10, n))
    G = np.diag(rng.uniform(0.05, 0.2, n))
    assert O.inverse_residual_hutchinson(A, G, 2, 11) == pytest.approx(O.inverse_residual(A, G), rel=1e-13)
    # likewise whenever each row of I - A G has one nonzero: G = A^{-1} (I - N), N a
    # scaled cyclic shift, so I - A G = N with ||N||_F^2 = sum of its entries squared
    w = rng.uniform(0.1, 3.0, n)
    N_ = np.roll(np.diag(w), 1, axis=1)
    G = np.linalg.solve(A, np.eye(n) - N_)
    assert O.inverse_residual_hutchinson(A, G, 3, 13) == pytest.approx(math.sqrt(float(np.sum(w * w))), rel=1e-12)


def test_hutchinson_unbiased_within_its_variance():
    """E z^T M z = tr M and Var = 2 sum_{i != j} M_ij^2 for Rademacher z and
    symmetric M = R^T R, R = I - A G: the s-probe mean of ||R z||^2 must lie
    within 5 standard errors of ||R||_F^2."""
    p = spd(n=24, kappa=20.0, seed=8)
    G = O.alpha_frobenius(p.A) * np.eye(24) + 0.01 * np.random.default_rng(2).standard_normal((24, 24))
    R = np.eye(24) - p.A @ G
    M = R.T @ R
    var = 2.0 * float(np.sum(M * M) - np.sum(np.diag(M) ** 2))
    s = 1500
    est2 = O.inverse_residual_hutchinson(p.A, G, s, 3) ** 2
    assert abs(est2 - float(np.trace(M))) <= 5.0 * math.sqrt(var / s)


# ---------------------------------------------------------------- FP64-accurate products (integer slices)
def test_ozaki_slices_exact_integers_and_reconstruction():
    from fractions import Fraction
    rng = np.random.default_rng(13)
    X = rng.standard_normal((17, 29)) * 10.0 ** rng.integers(-8, 8, (17, 1))
    X[3] = 0.0
    for axis in (0, 1):
        sc = O.ozaki_scales(X, axis)
        assert np.all(np.log2(sc) == np.round(np.log2(sc)))           # powers of two
        lim = np.max(np.abs(X), axis=axis)
        assert np.all((lim < sc) & ((lim >= sc / 2) | (lim == 0)))
        sl7 = O.ozaki_slices(X, sc, axis, 7)
        sl9 = O.ozaki_slices(X, sc, axis, 9)
        for a in sl9:
            assert np.array_equal(a, np.trunc(a)) and np.max(np.abs(a)) <= 255
            assert np.all(a * X >= 0)  # truncation: every slice has the element's sign (or is 0)
        for i, j in zip(rng.integers(0, 17, 120), rng.integers(0, 29, 120)):
            scale = Fraction(float(sc[i] if axis == 1 else sc[j]))
            x = Fraction(float(X[i, j]))
            r7 = scale * sum(Fraction(int(a[i, j])) / 256 ** (t + 1) for t, a in enumerate(sl7))
            assert abs(x - r7) < scale / 2 ** 56      # truncation after 7 slices
            if abs(x) >= scale / 2 ** 19:             # 53 bits within 72: 9 slices are exact
                r9 = scale * sum(Fraction(int(a[i, j])) / 256 ** (t + 1) for t, a in enumerate(sl9))
                assert r9 == x


def test_ozaki_pairs_count():
    assert O.ozaki_pairs(7) == sorted(O.ozaki_pairs(7), key=lambda p: p[0] + p[1])
    assert len(O.ozaki_pairs(7)) == 28 and len(O.ozaki_pairs(2)) == 3
    assert all(t + u <= 8 for t, u in O.ozaki_pairs(7))


def test_ozaki_product_against_exact_arithmetic():
    """Against the exact product (Python fractions on a small case) the error is
    far below an FP64 GEMM's bound K u |L||R|, and small integer matrices
    multiply exactly."""
    from fractions import Fraction
    rng = np.random.default_rng(14)
    L = rng.standard_normal((6, 40)) * 10.0 ** rng.integers(-3, 3, (6, 1))
    R = rng.standard_normal((40, 5))
    P = O.ozaki_product(L, R, 7)
    ab = np.abs(L) @ np.abs(R)
    for i in range(6):
        for j in range(5):
            exact = sum(Fraction(float(L[i, k])) * Fraction(float(R[k, j])) for k in range(40))
            assert abs(float(Fraction(float(P[i, j])) - exact)) <= 2.0 ** -50 * ab[i, j]
    Li = rng.integers(-1000, 1000, (9, 13)).astype(float)
    Ri = rng.integers(-1000, 1000, (13, 7)).astype(float)
    assert np.array_equal(O.ozaki_product(Li, Ri, 7), Li @ Ri)


def test_solve_reaches_harmonic_exact_answer():
    """Harmonic-regressor Gram systems are built as b = A theta* (theta* drawn
    by the generator), so the oracle's solve must land on theta* within
    cond(A) times its residual: an independent pin of the whole solve
    (Newton-Schulz, Richardson, stopping) on the batched workload's systems."""
    from workloads import make_harmonic
    rng = np.random.default_rng(21)
    checked = 0
    for m in (4, 6, 9, 12, 16):
        p = make_harmonic(m, rng=rng)
        kap = float(np.linalg.cond(p.A))
        if kap > 1e7:
            continue
        r = O.ns_richardson_solve(p.A, p.B, order=4, ns_iters=40, tol=1e-12, max_sweeps=400)
        assert r.converged, (m, kap, r.rel_res[-3:])
        err = np.linalg.norm(r.theta - p.theta_star) / np.linalg.norm(p.theta_star)
        assert err <= 10 * kap * (1e-12 + p.n * 2.0 ** -53), (m, kap, err)
        checked += 1
    assert checked >= 3


def test_solve_reaches_gram_closed_form():
    """The Gram system of the large ill-conditioned workload, at a small size:
    X = U diag(sigma) V^T (2n x n, U and V Haar), A = X^T X, b = X^T y.  Its
    exact answer is theta* = V diag(1/sigma) U^T y (the least-squares solution
    of X theta = y), known from the factors without any solve; the oracle's
    order-8 solve reaches it within cond(A) times its residual."""
    n = 48
    rng = np.random.default_rng(22)
    U, _ = np.linalg.qr(rng.standard_normal((2 * n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sigma = np.exp(rng.uniform(np.log(1e-2), 0.0, n))
    X = (U * sigma) @ V.T
    y = rng.standard_normal((2 * n, 1))
    A = X.T @ X
    A = 0.5 * (A + A.T)
    b = X.T @ y
    tstar = V @ ((U.T @ y) / sigma[:, None])
    kap = float((sigma.max() / sigma.min()) ** 2)
    r = O.ns_richardson_solve(A, b, order=8, ns_iters=30, tol=1e-12, max_sweeps=400)
    assert r.converged, r.rel_res[-3:]
    err = np.linalg.norm(r.theta - tstar) / np.linalg.norm(tstar)
    assert err <= 10 * kap * (1e-12 + n * 2.0 ** -53), (kap, err)



def test_ozaki_signed_digits_exact_and_bounded():
    """Signed-digit slices: integers of at most 128 in magnitude, and the
    rational reconstruction 2 scale sum_t S_t 256^{-t} is within
    scale 256^{-s} of x (exactly x once the digits cover its 53 bits)."""
    from fractions import Fraction
    rng = np.random.default_rng(15)
    X = rng.standard_normal((13, 21)) * 10.0 ** rng.integers(-6, 6, (13, 1))
    X[2] = 0.0
    X[4, 3] = np.max(np.abs(X[4])) * 1.0     # the line maximum itself
    for axis in (0, 1):
        sc = O.ozaki_scales(X, axis)
        sl7 = O.ozaki_slices_signed(X, sc, axis, 7)
        sl9 = O.ozaki_slices_signed(X, sc, axis, 9)
        for a in sl9:
            assert np.array_equal(a, np.rint(a)) and np.max(np.abs(a)) <= 128
        for i, j in zip(rng.integers(0, 13, 100), rng.integers(0, 21, 100)):
            scale = Fraction(float(sc[i] if axis == 1 else sc[j]))
            x = Fraction(float(X[i, j]))
            r7 = 2 * scale * sum(Fraction(int(a[i, j])) / 256 ** (t + 1) for t, a in enumerate(sl7))
            assert abs(x - r7) <= scale / 256 ** 7
            if abs(x) >= scale / 2 ** 18:
                r9 = 2 * scale * sum(Fraction(int(a[i, j])) / 256 ** (t + 1) for t, a in enumerate(sl9))
                assert r9 == x


def test_ozaki_signed_chunk_sums_exact_in_binary32():
    """Any 1024-term dot product of signed digits stays within 2^24, so its
    binary32 sum in any order is exact: checked against int64 on digits drawn
    to the extremes (sums of exactly 2^24 included)."""
    rng = np.random.default_rng(16)
    # magnitudes just below the unit scale: first digits RN(128 (1 - delta)) = 128
    X = rng.choice([-1.0, 1.0], (64, 1024)) * (1.0 - rng.uniform(0, 1e-3, (64, 1024)))
    Y = rng.choice([-1.0, 1.0], (1024, 48)) * (1.0 - rng.uniform(0, 1e-3, (1024, 48)))
    X[:8] = np.abs(X[:8])          # first digits all +128: those sums reach 2^24 itself
    Y[:, :8] = np.abs(Y[:, :8])
    A = O.ozaki_slices_signed(X, np.full(64, 1.0), 1, 2)
    B = O.ozaki_slices_signed(Y, np.full(48, 1.0), 0, 2)
    for a in A:
        for b in B:
            exact = a.astype(np.int64) @ b.astype(np.int64)
            assert np.max(np.abs(exact)) <= 2 ** 24
            if a is A[0] and b is B[0]:
                assert np.max(np.abs(exact)) == 2 ** 24
            f32 = np.zeros(exact.shape, dtype=np.float32)
            for k in range(1024):
                f32 += np.outer(a[:, k], b[k, :]).astype(np.float32)
            assert np.array_equal(f32.astype(np.int64), exact)


def test_ozaki_signed_product_matches_truncated_and_exact():
    """Both slicing rules give the product to binary64 accuracy: against the
    exact rational product on a small case, and against each other."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    L = rng.standard_normal((5, 9)) * 10.0 ** rng.integers(-3, 3, (5, 1))
    R = rng.standard_normal((9, 4)) * 10.0 ** rng.integers(-3, 3, (1, 4))
    got = O.ozaki_product_signed(L, R, 7)
    for i in range(5):
        for j in range(4):
            ex = sum(Fraction(float(L[i, k])) * Fraction(float(R[k, j])) for k in range(9))
            ab = sum(abs(float(L[i, k]) * float(R[k, j])) for k in range(9))
            assert abs(Fraction(float(got[i, j])) - ex) <= Fraction(2.0 ** -50 * ab)
    tr = O.ozaki_product(L, R, 7)
    assert np.all(np.abs(got - tr) <= 2.0 ** -49 * (np.abs(L) @ np.abs(R)))
