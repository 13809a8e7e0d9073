"""Plant plausible mistakes in the oracle (on the CPU, via monkeypatch) and
check that the pins in test_oracle.py catch each one.  A pin that still passed
with a mistake planted would not be pinning anything."""
import numpy as np
import pytest

import oracle as O
import oracle.ns_oracle as N
import tests.test_oracle as T


def _patch(mp, name, fn):
    """Replace an oracle function both in its module and in the package
    namespace the tests call through."""
    mp.setattr(N, name, fn)
    if hasattr(O, name):
        mp.setattr(O, name, fn)


def _fails(fn, *args, **kw):
    try:
        fn(*args, **kw)
    except AssertionError:
        return True
    return False


def test_sign_flip_in_right_residual(monkeypatch):
    _patch(monkeypatch, "residual_right", lambda A, G, cnt=None: N.mm(A, G, cnt) - np.eye(A.shape[0]))
    assert _fails(T.test_exponent_law_plain_ns, 4, "factorized")


def test_dropped_identity_term_in_chain(monkeypatch):
    orig = N.ns_step_binary

    def bad(A, G, levels, pow_mode="square", cnt=None):
        F = N.residual_right(A, G, cnt)
        X, P = G, F
        for j in range(levels):
            X = N.mm(X, P, cnt)            # "X +" dropped
            if j + 1 < levels:
                P = N.mm(P, P, cnt)
        return X, F
    _patch(monkeypatch, "ns_step_binary", bad)
    assert _fails(T.test_exponent_law_plain_ns, 2, "factorized")
    _patch(monkeypatch, "ns_step_binary", orig)


def test_transposed_operand_in_chain(monkeypatch):
    """X + P X instead of X + X P: invisible for G0 = alpha I (everything
    commutes), caught by the non-commuting push-through pin."""
    def bad(A, G, levels, pow_mode="square", cnt=None):
        F = N.residual_right(A, G, cnt)
        X, P = G, F
        for j in range(levels):
            X = X + N.mm(P, X, cnt)
            if j + 1 < levels:
                P = N.mm(P, P, cnt)
        return X, F
    _patch(monkeypatch, "ns_step_binary", bad)
    T.test_exponent_law_plain_ns(4, "factorized")          # commuting case passes
    assert _fails(T.test_push_through_right_equals_left_noncommuting)


def test_wrong_power_index(monkeypatch):
    """Squaring skipped (P stays F): order 4 becomes G(I+F)^2, exponent 3."""
    def bad(A, G, levels, pow_mode="square", cnt=None):
        F = N.residual_right(A, G, cnt)
        X = G
        for _ in range(levels):
            X = X + N.mm(X, F, cnt)
        return X, F
    _patch(monkeypatch, "ns_step_binary", bad)
    assert _fails(T.test_exponent_law_plain_ns, 4, "factorized")


def test_composite_wrong_prefix_order(monkeypatch):
    def bad(A, Tl, cnt=None):
        I = np.eye(A.shape[0])
        Gam = [I - N.mm(Ti, A, cnt) for Ti in Tl]
        Tc = Tl[0].copy()
        prefix = Gam[0]
        for i in range(1, len(Tl)):
            Tc = Tc + N.mm(Tl[i], prefix, cnt)      # transposed
            prefix = N.mm(Gam[i], prefix, cnt)
        return Tc, prefix
    _patch(monkeypatch, "composite_combine", bad)
    assert _fails(T.test_composite_telescoping_noncommuting)


def test_composite_missing_gamma(monkeypatch):
    def bad(A, G_prev, Tl, n, cnt=None):
        Tc, Gc = N.composite_combine(A, Tl, cnt)
        return Tc + N.ns_classical_step(G_prev, A, n, cnt)
    _patch(monkeypatch, "composite_step", bad)
    assert _fails(T.test_composite_exponent_law, 2, [2])


def test_double_ns_first_order_error(monkeypatch):
    """Using G_{k-1} in place of {sum_j F_{k-1}^j} G_{k-1} (the Remark 2
    algorithm's first-order error) changes the exponent of eq. ermoex1."""
    def bad(A, st, n, cnt=None):
        L = N.ns_classical_step(st.L, A, n, cnt)
        GamN = N.residual_left(L, A, cnt)
        G = L + N.mm(GamN, st.G, cnt)
        return N.DoubleNSState(G=G, L=L, GamN=GamN, F=N.residual_left(G, A), k=st.k + 1)
    _patch(monkeypatch, "double_ns_iterate", bad)
    assert _fails(T.test_double_ns_exponent, 2)


def test_richardson_sign(monkeypatch):
    _patch(monkeypatch, "richardson_step", lambda A, B, th, G: (th - G @ (B - A @ th), B - A @ th))
    orig = N.ns_richardson_solve

    def bad(A, B, **kw):
        r = orig(A, B, **kw)
        r.theta = -r.theta
        return r
    _patch(monkeypatch, "ns_richardson_solve", bad)
    assert _fails(T.test_richardson_error_model, 2, False)


def test_bf16_truncation_instead_of_rounding(monkeypatch):
    pytest.importorskip("torch")

    def trunc(x):
        f = np.asarray(x, dtype=np.float64).astype(np.float32)
        u = f.view(np.uint32) & np.uint32(0xFFFF0000)
        return u.view(np.float32).astype(np.float64)
    _patch(monkeypatch, "round_bf16", trunc)
    assert _fails(T.test_round_bf16_matches_torch)


def test_split_dropping_cross_term(monkeypatch):
    monkeypatch.setitem(N.SPLIT_PASSES, "bf16x3", (("hi", "hi"), ("hi", "lo")))
    assert _fails(T.test_split_product_terms)


def test_two_term_split_wrong_terms(monkeypatch):
    # the term kept by mistake is the one the reading drops (hi of L times lo
    # of R) instead of lo of L times hi of R
    monkeypatch.setitem(N.SPLIT_PASSES, "bf16x2", (("hi", "hi"), ("hi", "lo")))
    assert _fails(T.test_split_product_two_terms)
    monkeypatch.setitem(N.SPLIT_PASSES, "bf16x2", (("hi", "hi"),))
    assert _fails(T.test_split_product_two_terms)


def test_splitmix64_wrong_shift(monkeypatch):
    def bad(seed, k):
        z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & N._U64
        z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & N._U64   # 31 where the finalizer shifts by 30
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & N._U64
        return z ^ (z >> 31)
    _patch(monkeypatch, "splitmix64", bad)
    assert _fails(T.test_splitmix64_published_outputs)


def test_hutchinson_missing_probe_mean(monkeypatch):
    def bad(A, G, s, seed):
        Z = N.rademacher_probes(A.shape[0], s, seed)
        R = Z - A @ (G @ Z)
        return float(np.sqrt(np.sum(R * R)))   # sum over probes, not the mean
    _patch(monkeypatch, "inverse_residual_hutchinson", bad)
    assert _fails(T.test_hutchinson_exact_cases)


def test_hutchinson_transposed_product(monkeypatch):
    def bad(A, G, s, seed):
        Z = N.rademacher_probes(A.shape[0], s, seed)
        R = Z - G @ (A @ Z)   # I - G A instead of I - A G
        return float(np.sqrt(np.sum(R * R) / s))
    _patch(monkeypatch, "inverse_residual_hutchinson", bad)
    assert _fails(T.test_hutchinson_exact_cases)


def test_inverse_residual_sign(monkeypatch):
    _patch(monkeypatch, "inverse_residual", lambda A, G: float(np.linalg.norm(np.eye(A.shape[0]) + A @ G)))
    assert _fails(T.test_inverse_residual_closed_forms)


def test_x6_dropping_a_second_order_term(monkeypatch):
    monkeypatch.setitem(N.SPLIT_PASSES, "bf16x6",
                        (("hi", "hi"), ("hi", "lo"), ("lo", "hi"), ("hi", "lo2"), ("lo2", "hi")))
    assert _fails(T.test_split_product_x6_terms)


def test_split3_truncated_third_part(monkeypatch):
    orig = N.split3_bf16

    def bad(x):
        hi, lo, lo2 = orig(x)
        return hi, lo, np.trunc(lo2 * 2.0 ** 30) / 2.0 ** 30
    _patch(monkeypatch, "split3_bf16", bad)
    assert _fails(T.test_split3_exact_and_matches_torch)


def test_ozaki_rounding_instead_of_truncation(monkeypatch):
    def bad(X, scale, axis, s):
        x = X / (scale[:, None] if axis == 1 else scale[None, :])
        out = []
        for _ in range(s):
            x = x * 256.0
            a = np.round(x)
            x = x - a
            out.append(a)
        return out
    _patch(monkeypatch, "ozaki_slices", bad)
    assert _fails(T.test_ozaki_slices_exact_integers_and_reconstruction)


def test_ozaki_level_weight_off_by_one(monkeypatch):
    def bad(L, R, s=7):
        mu, nu = N.ozaki_scales(L, 1), N.ozaki_scales(R, 0)
        A = [a.astype(np.int64) for a in N.ozaki_slices(L, mu, 1, s)]
        B = [b.astype(np.int64) for b in N.ozaki_slices(R, nu, 0, s)]
        out = np.zeros((L.shape[0], R.shape[1]))
        for t, u in N.ozaki_pairs(s):
            out += np.ldexp((A[t - 1] @ B[u - 1]).astype(np.float64), -8 * (t + u - 1))
        return out * mu[:, None] * nu[None, :]
    _patch(monkeypatch, "ozaki_product", bad)
    assert _fails(T.test_ozaki_product_against_exact_arithmetic)


def test_alpha_inf_missing_half(monkeypatch):
    """alpha_s = ||A||_inf + eps instead of ||A||_inf / 2 + eps (Section 2)."""
    _patch(monkeypatch, "alpha_inf", lambda A, eps=None: 1.0 / (1.0 + 1e-8) / np.linalg.norm(A, np.inf))
    assert _fails(T.test_alpha_inf_matches_definition_and_contracts)


def test_jacobi_returns_diagonal_not_inverse(monkeypatch):
    _patch(monkeypatch, "jacobi_preconditioner", lambda A: np.diag(np.diag(A)))
    assert _fails(T.test_jacobi_splitting_contracts_for_sdd)


def test_initial_series_one_term_short(monkeypatch):
    """G0 = sum_{j < h-1} (S^{-1}D)^j S^{-1}: one term of eq. g01 dropped."""
    orig = N.initial_series

    def bad(A, S_inv, p, w, cnt=None):
        G0, F0 = orig(A, S_inv, p, w, cnt)
        SD = N.splitting_residual(A, S_inv)
        return G0 - np.linalg.matrix_power(SD, w * (p + 1) - 1) @ S_inv, F0
    _patch(monkeypatch, "initial_series", bad)
    assert _fails(T.test_initial_series_g01_g03, 1, 2)


def test_toolkit_p_and_w_swapped(monkeypatch):
    """Reading a table row's (p, w) the wrong way round: h = 5 (eq. ztab2 with
    p = 1, w = 2) becomes order w (p + 1) + 1 = 4 with the pair swapped."""
    def bad(X, A, h, cnt=None):
        kind, p, w = N.TOOLKIT_TABLE[h]
        if kind == "z":
            return N.unified_factorization(X, A, w, p, cnt)
        return N.schroder_traub(X, A, w, p, cnt)
    _patch(monkeypatch, "toolkit", bad)
    assert _fails(T.test_toolkit_rows_equal_series, 5)


def test_order3_dropped_linear_term(monkeypatch):
    """W = F F instead of F + F F: G (I + F^2) is not the order-3 step."""
    def bad(A, G, cnt=None):
        F = N.residual_right(A, G, cnt)
        return G + N.mm(G, N.mm(F, F, cnt), cnt), F
    _patch(monkeypatch, "ns_step_order3", bad)
    assert _fails(T.test_exponent_law_plain_ns, 3, "factorized")


def test_nested45_missing_square_in_outer_factor(monkeypatch):
    """Outer factor (I + Y18)(Y9) instead of (I + Y18)(Y9 + Y18) (eq. ex3)."""
    def bad(X, A, cnt=None):
        I = N._eye_like(A)
        XA = N.mm(X, A, cnt)
        W3 = N.mm(3.0 * I + N.mm(XA, -3.0 * I + XA, cnt), X, cnt)
        Y3 = I - N.mm(W3, A, cnt)
        W9 = N.mm(Y3, N.mm(Y3, W3, cnt) + W3, cnt) + W3
        Y9 = I - N.mm(W9, A, cnt)
        Y18 = N.mm(Y9, Y9, cnt)
        Q = N.mm(I + Y18, Y9, cnt)
        return W9 + N.mm(Q, W9, cnt)
    _patch(monkeypatch, "nested_order45", bad)
    assert _fails(T.test_nested_order45_ten_mmm)


def test_gemm_epilogue_identity_sign(monkeypatch):
    def bad(prod, s=1.0, C=None, beta=0.0, gamma=0.0):
        D = s * prod
        if C is not None and beta != 0.0:
            D = D + beta * C
        return D - gamma * np.eye(D.shape[0])
    _patch(monkeypatch, "gemm_epilogue", bad)
    assert _fails(T.test_gemm_epilogue_forms)


def test_ozaki_scale_not_a_power_of_two(monkeypatch):
    """Scaling by the line's exact maximum: slicing x / max is no longer exact."""
    _patch(monkeypatch, "ozaki_scales",
           lambda X, axis: np.where(np.max(np.abs(X), axis=axis) > 0, np.max(np.abs(X), axis=axis) * 1.5, 1.0))
    assert _fails(T.test_ozaki_slices_exact_integers_and_reconstruction)


def test_relative_residual_not_normalised(monkeypatch):
    _patch(monkeypatch, "rel_residual", lambda A, theta, B: np.sqrt(np.sum((B - A @ theta) ** 2, axis=0)))
    assert _fails(T.test_rel_residual_closed_forms)


def test_accelerated_richardson_plain_G(monkeypatch):
    """theta - G_k (A theta - b): the omega_k of eq. ttk1 replaced by G_k."""
    _patch(monkeypatch, "accelerated_richardson_step", lambda A, b, theta, st, q: theta - st.G @ (A @ theta - b))
    assert _fails(T.test_accelerated_richardson_gamma, 2)


def test_rademacher_low_bit(monkeypatch):
    """Sign from the lowest bit instead of the top bit of each output."""
    def bad(n, s, seed):
        Z = np.empty((n, s))
        for j in range(s):
            for i in range(n):
                Z[i, j] = -1.0 if N.splitmix64(seed, j * n + i) & 1 else 1.0
        return Z
    _patch(monkeypatch, "rademacher_probes", bad)
    assert _fails(T.test_rademacher_probes_follow_published_outputs)


def test_horner_right_one_product_short(monkeypatch):
    """X = G + X F repeated n - 2 times: order n - 1 instead of n."""
    def bad(A, G, n, cnt=None):
        F = N.residual_right(A, G, cnt)
        X = G.copy()
        for _ in range(n - 2):
            X = G + N.mm(X, F, cnt)
        return X, F
    _patch(monkeypatch, "ns_step_horner_right", bad)
    assert _fails(T.test_exponent_law_plain_ns, 4, "horner")


def test_left_residual_transposed_product(monkeypatch):
    """I - A G where the left form I - G A is meant: equal while G commutes
    with A, caught by the non-commuting push-through pin."""
    _patch(monkeypatch, "residual_left", lambda G, A, cnt=None: np.eye(A.shape[0]) - N.mm(A, G, cnt))
    T.test_exponent_law_plain_ns(2, "factorized")
    assert _fails(T.test_push_through_right_equals_left_noncommuting)


def test_abs_product_taken_after_the_sum(monkeypatch):
    """|sum of the split terms| instead of the sum of |terms|: no longer an
    error scale (it vanishes where the terms cancel)."""
    orig = N.split_product
    _patch(monkeypatch, "split_abs_product", lambda L, R, precision: np.abs(orig(L, R, precision)))
    assert _fails(T.test_split_abs_product_bounds)


def test_ozaki_last_level_dropped(monkeypatch):
    """Pairs of level t + u <= s only: the s pairs of the last level missing."""
    _patch(monkeypatch, "ozaki_pairs",
           lambda s: [(t, d - t) for d in range(2, s + 1) for t in range(1, d) if 1 <= d - t <= s])
    assert _fails(T.test_ozaki_pairs_count)
    assert _fails(T.test_ozaki_product_against_exact_arithmetic)


def test_composite_aux_loops_at_the_main_order(monkeypatch):
    """Every auxiliary loop advanced with the main order n instead of its own
    rate m_i (eq. ti with x_i = m_i^k)."""
    def bad(A, st, n, rates, cnt=None):
        T_new = [N.ns_classical_step(Ti, A, n, cnt) for Ti in st.T]
        return N.CompositeState(G=N.composite_step(A, st.G, T_new, n, cnt), T=T_new, k=st.k + 1)
    _patch(monkeypatch, "composite_iterate", bad)
    assert _fails(T.test_composite_exponent_law, 2, [3])


def test_composite_exponent_recursion_without_rates(monkeypatch):
    """e_k = n e_{k-1}: the auxiliary loops' contribution sum_i m_i^k dropped."""
    def bad(n, rates, h, K):
        e = [h]
        for _ in range(K):
            e.append(n * e[-1])
        return e
    _patch(monkeypatch, "composite_exponents", bad)
    assert _fails(T.test_composite_exponent_values)


def test_double_ns_exponent_power_off_by_one(monkeypatch):
    """h (k n^k + n^k) instead of h (k n^{k+1} + n^k) (eq. ermoex1)."""
    _patch(monkeypatch, "double_ns_exponent", lambda n, h, k: h * (k * n ** k + n ** k))
    assert _fails(T.test_double_ns_exponent_values)
    assert _fails(T.test_double_ns_exponent, 2)


def test_accelerated_exponent_missing_factor(monkeypatch):
    """gamma_k of eq. riem6 without its leading factor n."""
    def bad(n, h, k):
        num = k * n ** (k + 2) - (k - 1) * n ** (k + 1) - 2 * n ** k - n + 2
        return h * n * num / (n - 1) ** 2
    _patch(monkeypatch, "accelerated_richardson_exponent", bad)
    assert _fails(T.test_gamma_closed_form_equals_sum)


def test_signed_digits_truncated(monkeypatch):
    """trunc in place of round-to-nearest: digits reach 255 and the 1024-term
    sums leave binary32's exact range."""
    def bad(X, scale, axis, s):
        x = X / (2.0 * (scale[:, None] if axis == 1 else scale[None, :]))
        out = []
        for _ in range(s):
            x = x * 256.0
            a = np.trunc(x)
            x = x - a
            out.append(a)
        return out
    _patch(monkeypatch, "ozaki_slices_signed", bad)
    assert _fails(T.test_ozaki_signed_digits_exact_and_bounded)


def test_signed_product_missing_factor_two(monkeypatch):
    """The scales mu, nu of the truncated rule reused without the signed rule's 2."""
    orig = N.ozaki_product_signed
    _patch(monkeypatch, "ozaki_product_signed", lambda L, R, s=7: 0.25 * orig(L, R, s))
    assert _fails(T.test_ozaki_signed_product_matches_truncated_and_exact)


def test_tf32_ties_to_even(monkeypatch):
    """TF32 rounding with ties to even instead of away from zero."""
    def bad(x):
        f = np.asarray(x, dtype=np.float64).astype(np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        lsb = (u >> np.uint64(13)) & np.uint64(1)
        r = ((u + np.uint64(0xFFF) + lsb) >> np.uint64(13)) << np.uint64(13)
        return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    _patch(monkeypatch, "round_tf32", bad)
    assert _fails(T.test_round_tf32_nearest_ties_away)


def test_tf32_truncation(monkeypatch):
    """TF32 by truncation (the low 13 bits dropped, as an input conversion
    that ignores them would do)."""
    def bad(x):
        f = np.asarray(x, dtype=np.float64).astype(np.float32)
        u = f.view(np.uint32) & np.uint32(0xFFFFE000)
        return u.view(np.float32).astype(np.float64)
    _patch(monkeypatch, "round_tf32", bad)
    assert _fails(T.test_round_tf32_nearest_ties_away)
