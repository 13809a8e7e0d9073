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
