"""FP64 oracle for factorized high-order Newton-Schulz inversion, its composite
and double-loop variants, and Richardson iteration (A. Stotsky, "Convergence
Rate Improvement of Richardson and Newton-Schulz Iterations", arXiv 2008.11480).

TEST INFRASTRUCTURE ONLY.  This module is imported by the test-suite, by the
package's smoke check and by the benchmark's CPU-baseline leg.  The CUDA
library never imports, links or calls it, and it shares no code with it.

Everything here is plain numpy in float64: each matrix product is one
``numpy.matmul`` (the paper's cost unit, a "mmm"), with no blocking, fusion or
reordering beyond what the cited equation states, so the code can be checked
against the paper by eye.  Every function names the passage it follows.

Notation follows the paper: A is SPD, S^{-1} the preconditioner, G_k the
estimate of A^{-1}, F_k = I - G_k A the (left) inversion error, n the
Newton-Schulz order, Y = I - X A and Z = {sum_{j<h} Y^j} X the generic series
of Section 4.  The "right" residual I - A G_k used by the GPU chain is the
mirror image; the push-through identity (I - G A)^j G = G (I - A G)^j makes both
forms produce the same iterates in exact arithmetic (tested).

Reduced-precision definitions (bf16 rounding, the hi/lo split and split
products) at the end of the file define what the mixed-precision GEMMs compute;
the paper fixes no precision, so those are this library's own definitions.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# mmm counting (Section 4, eq. np1: the cost of an algorithm is its number of
# matrix-by-matrix multiplications)
# --------------------------------------------------------------------------


@dataclass
class MMCount:
    """Counts matrix-matrix multiplications ("mmm", Section 4)."""

    n: int = 0


def mm(X: np.ndarray, Y: np.ndarray, cnt: MMCount | None = None) -> np.ndarray:
    """One matrix-by-matrix multiplication, counted in ``cnt``."""
    if cnt is not None:
        cnt.n += 1
    return X @ Y


def _eye_like(A: np.ndarray) -> np.ndarray:
    return np.eye(A.shape[0], dtype=np.float64)


# --------------------------------------------------------------------------
# Section 2: splitting and preconditioning, A = S - D, rho(S^{-1} D) < 1
# --------------------------------------------------------------------------


def alpha_frobenius(A: np.ndarray) -> float:
    """Scale of the scalar preconditioner S^{-1} = alpha I with
    alpha = 1/||A||_F.  For SPD A, ||A||_2 <= ||A||_F, so the eigenvalues of
    S^{-1} D = I - alpha A lie in [0, 1) and rho(S^{-1} D) < 1 (Section 2,
    eqs. minus-spro; 2S - A = 2||A||_F I - A is positive definite)."""
    return 1.0 / float(np.sqrt(np.sum(A * A)))


def alpha_inf(A: np.ndarray, eps: float | None = None) -> float:
    """Section 2: S^{-1} = I/alpha_s with alpha_s = ||A||_inf/2 + eps, where
    ||.||_inf is the maximum row sum norm and eps > 0 small.  The paper leaves
    eps open; the default here is eps = 1e-8 ||A||_inf.  Returns 1/alpha_s."""
    ninf = float(np.max(np.sum(np.abs(A), axis=1)))
    if eps is None:
        eps = 1e-8 * ninf
    return 1.0 / (ninf / 2.0 + eps)


def jacobi_preconditioner(A: np.ndarray) -> np.ndarray:
    """Section 2: for strictly diagonally dominant SPD A, S = diag(A); returns
    S^{-1} as a dense diagonal matrix."""
    return np.diag(1.0 / np.diag(A))


def splitting_residual(A: np.ndarray, S_inv: np.ndarray) -> np.ndarray:
    """S^{-1} D = I - S^{-1} A (Section 2, eq. sp1)."""
    return _eye_like(A) - S_inv @ A


# --------------------------------------------------------------------------
# Residuals (eq. g03 / fk1 / xa1), left and right forms
# --------------------------------------------------------------------------


def residual_left(G: np.ndarray, A: np.ndarray, cnt: MMCount | None = None) -> np.ndarray:
    """F = I - G A (eqs. g03, fk1; Y = I - X A in eq. xa1)."""
    return _eye_like(A) - mm(G, A, cnt)


def residual_right(A: np.ndarray, G: np.ndarray, cnt: MMCount | None = None) -> np.ndarray:
    """F = I - A G, the right-multiplied residual of the product chain
    G (I + F)(I + F^2)... ."""
    return _eye_like(A) - mm(A, G, cnt)


# --------------------------------------------------------------------------
# Section 3: initial series and the classical high-order iteration
# --------------------------------------------------------------------------


def initial_series(A: np.ndarray, S_inv: np.ndarray, p: int, w: int,
                   cnt: MMCount | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Section 3, eqs. g01-g03: G0 = sum_{j<w} (S^{-1}D)^{(p+1)j}
    {sum_{d<=p} (S^{-1}D)^d} S^{-1} = sum_{j<h} (S^{-1}D)^j S^{-1}, h = w(p+1),
    and F0 = I - G0 A = (S^{-1}D)^h.  Evaluated with the unified factorization
    of Section 4 (eq. z2 "represents (g01)" with Y = S^{-1}D, X = S^{-1})."""
    G0 = unified_factorization(S_inv, A, p, w, cnt)
    F0 = residual_left(G0, A)
    return G0, F0


def ns_classical_step(G: np.ndarray, A: np.ndarray, n: int,
                      cnt: MMCount | None = None) -> np.ndarray:
    """Section 3, eq. ns: G_k = {sum_{j<n} F_{k-1}^j} G_{k-1},
    F_{k-1} = I - G_{k-1} A, evaluated by Horner's scheme (n mmm)."""
    return series_horner(G, A, n, cnt)


# --------------------------------------------------------------------------
# Section 4: power series Z = {sum_{j<h} Y^j} X, Y = I - X A, and its
# unified factorization
# --------------------------------------------------------------------------


def series_horner(X: np.ndarray, A: np.ndarray, h: int,
                  cnt: MMCount | None = None) -> np.ndarray:
    """Eqs. z1, xa1 by Horner's scheme: Y = I - X A (1 mmm), then
    Z_0 = X, Z_i = Y Z_{i-1} + X for i = 1..h-1 (h-1 mmm); h mmm in total."""
    if h < 1:
        raise ValueError("order h must be >= 1")
    Y = residual_left(X, A, cnt)
    Z = X.copy()
    for _ in range(h - 1):
        Z = mm(Y, Z, cnt) + X
    return Z


def unified_factorization(X: np.ndarray, A: np.ndarray, p: int, w: int,
                          cnt: MMCount | None = None, Y: np.ndarray | None = None) -> np.ndarray:
    """Section 4, eqs. xa2-z2 with the recursion zi1:

        Y = I - X A                           (1 mmm)
        U = {sum_{d=0}^{p} Y^d} X              (p mmm, Horner)
        Y^{p+1} = I - U A                      (1 mmm)
        Z = {sum_{j=0}^{w-1} Y^{(p+1)j}} U     (w-1 mmm: Z_i = Y^{p+1} Z_{i-1} + U)

    Order h = w(p+1) (eq. h1) in N_p = p + w + 1 mmm (eq. np1), or p + 1 mmm
    when w = 1.  The p = 0 case needs no Y and no U products (U = X), so it
    costs w mmm, as the paper notes after eq. zi1.  A precomputed Y may be
    passed in (it is then not counted again)."""
    if p < 0 or w < 1:
        raise ValueError("need p >= 0 and w >= 1")
    if p == 0:
        U = X
    else:
        if Y is None:
            Y = residual_left(X, A, cnt)
        U = X.copy()
        for _ in range(p):
            U = mm(Y, U, cnt) + X
    if w == 1:
        return U
    Yp1 = residual_left(U, A, cnt)
    Z = U.copy()
    for _ in range(w - 1):
        Z = mm(Yp1, Z, cnt) + U
    return Z


def schroder_traub(X: np.ndarray, A: np.ndarray, p: int, w: int,
                   cnt: MMCount | None = None) -> np.ndarray:
    """Appendix, eqs. ztab2, hape1: Z_1 = (I + Y {sum_j Y^{(p+1)j}}
    {sum_{d<=p} Y^d}) X = X + Y Z, raising the order of eq. ztab1 from h to
    h + 1 with one more mmm (Y of eq. xanew is shared with Z)."""
    Y = residual_left(X, A, cnt)
    Z = unified_factorization(X, A, p, w, cnt, Y=Y)
    return X + mm(Y, Z, cnt)


def nested_order45(X: np.ndarray, A: np.ndarray, cnt: MMCount | None = None) -> np.ndarray:
    """Section 4, eqs. ex1-ex3: order 45 in ten mmm.

        inner order 3:  W3 = [3I + (XA)(-3I + XA)] X = (I + Y + Y^2) X
        Y^3 = I - W3 A
        inner order 9:  W9 = [I + Y^3 + Y^6] W3     (Horner in Y^3)
        Y^9 = I - W9 A
        outer:          Z = {I + (I + (Y^9)^2)(Y^9 + (Y^9)^2)} W9
    """
    I = _eye_like(A)
    XA = mm(X, A, cnt)                                   # 1
    W3 = mm(3.0 * I + mm(XA, -3.0 * I + XA, cnt), X, cnt)  # 2, 3
    Y3 = I - mm(W3, A, cnt)                              # 4
    W9 = mm(Y3, mm(Y3, W3, cnt) + W3, cnt) + W3          # 5, 6
    Y9 = I - mm(W9, A, cnt)                              # 7
    Y18 = mm(Y9, Y9, cnt)                                # 8
    Q = mm(I + Y18, Y9 + Y18, cnt)                       # 9
    return W9 + mm(Q, W9, cnt)                           # 10


# Appendix, Tables t1-t3: the unified form each row uses, as (kind, p, w) with
# kind "z" for eq. ztab1 and "z1" for eq. ztab2.  For h = 10, 11 the tables give
# two forms; the first listed is used here.
TOOLKIT_TABLE: dict[int, tuple[str, int, int]] = {
    2: ("z", 1, 1), 3: ("z1", 1, 1), 4: ("z", 1, 2), 5: ("z1", 1, 2),
    6: ("z", 2, 2), 7: ("z1", 2, 2), 8: ("z", 3, 2), 9: ("z", 2, 3),
    10: ("z1", 2, 3), 11: ("z1", 4, 2), 12: ("z", 3, 3), 13: ("z1", 3, 3),
    14: ("z", 6, 2), 15: ("z", 2, 5), 16: ("z", 3, 4), 17: ("z1", 3, 4),
    18: ("z", 5, 3), 19: ("z1", 5, 3),
}


def toolkit(X: np.ndarray, A: np.ndarray, h: int, cnt: MMCount | None = None) -> np.ndarray:
    """Order-h series {sum_{j<h} Y^j} X by the Appendix tool-kit row for h."""
    kind, p, w = TOOLKIT_TABLE[h]
    if kind == "z":
        return unified_factorization(X, A, p, w, cnt)
    return schroder_traub(X, A, p, w, cnt)


# --------------------------------------------------------------------------
# The product chain used by the GPU path (right form):
#   G_{k+1} = G_k (I + F_k)(I + F_k^2)(I + F_k^4)...,  F_k = I - A G_k.
# Tables t1/t2 rows h = 2, 4, 8 ((I+Y)X, (I+Y^2)(I+Y)X, (I+Y^4)(I+Y^2)(I+Y)X)
# mirrored by push-through; row h = 3 is (I + Y(I + Y)) X.
# --------------------------------------------------------------------------


def ns_step_binary(A: np.ndarray, G: np.ndarray, levels: int, pow_mode: str = "square",
                   cnt: MMCount | None = None) -> tuple[np.ndarray, np.ndarray]:
    """One iteration of order 2^levels in product form (Tables t1/t2 rows
    h = 2, 4, 8; Appendix remark that orders 4 and 8 cost 4 and 6 mmm).

        F = I - A G                  (1 mmm)
        X_0 = G, P_0 = F
        X_{j+1} = X_j + X_j P_j      (1 mmm)
        P_{j+1} = P_j P_j            ("square", 1 mmm)   or
        P_{j+1} = I - A X_{j+1}      ("residual": eq. ua1, Y^{p+1} = I - U A)

    Returns (G_{k+1}, F_k)."""
    if levels < 1:
        raise ValueError("levels >= 1")
    F = residual_right(A, G, cnt)
    X, P = G, F
    for j in range(levels):
        X = X + mm(X, P, cnt)
        if j + 1 < levels:
            if pow_mode == "square":
                P = mm(P, P, cnt)
            elif pow_mode == "residual":
                P = residual_right(A, X, cnt)
            else:
                raise ValueError(pow_mode)
    return X, F


def ns_step_order3(A: np.ndarray, G: np.ndarray,
                   cnt: MMCount | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Order 3, Table t1 row h = 3: (I + Y(I + Y)) X, mirrored to the right
    form G (I + (I + F) F) = G + G (F + F F); 3 mmm.  Returns (G_{k+1}, F_k)."""
    F = residual_right(A, G, cnt)
    W = F + mm(F, F, cnt)
    return G + mm(G, W, cnt), F


def ns_step_horner_right(A: np.ndarray, G: np.ndarray, n: int,
                         cnt: MMCount | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Unfactorized right form G {sum_{j<n} F^j}, F = I - A G, by Horner:
    X = G, then X = G + X F repeated n-1 times (n mmm)."""
    F = residual_right(A, G, cnt)
    X = G.copy()
    for _ in range(n - 1):
        X = G + mm(X, F, cnt)
    return X, F


def ns_step(A: np.ndarray, G: np.ndarray, order: int, form: str = "factorized",
            pow_mode: str = "square", cnt: MMCount | None = None) -> tuple[np.ndarray, np.ndarray]:
    """One Newton-Schulz step of the given order in the right form.
    ``form`` = "factorized" (orders 2, 3, 4, 8, 16, ...) or "horner" (any order)."""
    if form == "horner":
        return ns_step_horner_right(A, G, order, cnt)
    if order == 3:
        return ns_step_order3(A, G, cnt)
    levels = int(round(np.log2(order)))
    if order < 2 or 2 ** levels != order:
        raise ValueError("factorized form supports order 3 and powers of two")
    return ns_step_binary(A, G, levels, pow_mode, cnt)


# --------------------------------------------------------------------------
# Section 5: composite expansion with mixed rates
# --------------------------------------------------------------------------


def composite_combine(A: np.ndarray, T: list[np.ndarray],
                      cnt: MMCount | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Eqs. tc, gc with eq. rterm1: Gamma_i = I - T_i A, T_c = T_1 + Gamma_1 T_2
    + ... + (prod_{p<w} Gamma_p) T_w, Gamma_c = Gamma_1 ... Gamma_w.
    Returns (T_c, Gamma_c)."""
    I = _eye_like(A)
    Gam = [I - mm(Ti, A, cnt) for Ti in T]
    Tc = T[0].copy()
    prefix = Gam[0]
    for i in range(1, len(T)):
        Tc = Tc + mm(prefix, T[i], cnt)
        prefix = mm(prefix, Gam[i], cnt)
    return Tc, prefix


def composite_step(A: np.ndarray, G_prev: np.ndarray, T: list[np.ndarray], n: int,
                   cnt: MMCount | None = None) -> np.ndarray:
    """Eq. gkgen1: G_k = T_c + Gamma_c {sum_{j<n} F_{k-1}^j} G_{k-1}, with
    F_{k-1} = I - G_{k-1} A; error model F_k = Gamma_c F_{k-1}^n (eq. gem1)."""
    Tc, Gc = composite_combine(A, T, cnt)
    X = ns_classical_step(G_prev, A, n, cnt)
    return Tc + mm(Gc, X, cnt)


@dataclass
class CompositeState:
    """State of the composite iteration: G_k and the auxiliary expansions T_i."""

    G: np.ndarray
    T: list[np.ndarray]
    k: int = 0


def composite_init(G0: np.ndarray, n_rates: int) -> CompositeState:
    """Each auxiliary expansion T_i starts from S^{-1} = G0 (h = 1)."""
    return CompositeState(G=G0.copy(), T=[G0.copy() for _ in range(n_rates)], k=0)


def composite_iterate(A: np.ndarray, st: CompositeState, n: int, rates: list[int],
                      cnt: MMCount | None = None) -> CompositeState:
    """One step k-1 -> k of the mixed-rate composite method (Section 5, eqs.
    gkgen1-ga1).  Each T_i is an independent Newton-Schulz loop of order m_i
    started at S^{-1}, so after k steps T_i = {sum_{j < m_i^k} (S^{-1}D)^j}
    S^{-1}, i.e. eq. ti with rate x_i = m_i^k, and Gamma_i = (S^{-1}D)^{m_i^k}
    (eq. ga1).  The paper leaves the loops that produce T_i open; this is the
    reading x_i = m^k it names as an example."""
    T_new = [ns_classical_step(Ti, A, m, cnt) for Ti, m in zip(st.T, rates)]
    G_new = composite_step(A, st.G, T_new, n, cnt)
    return CompositeState(G=G_new, T=T_new, k=st.k + 1)


def composite_exponents(n: int, rates: list[int], h: int, K: int) -> list[int]:
    """Exponent e_k with F_k = (S^{-1}D)^{e_k} for the composite method:
    e_0 = h, e_k = sum_i m_i^k + n e_{k-1} (eq. gem1 with eq. ga1, x_i = m_i^k)."""
    e = [h]
    for k in range(1, K + 1):
        e.append(sum(m ** k for m in rates) + n * e[-1])
    return e


# --------------------------------------------------------------------------
# Section 5.1: double Newton-Schulz with a high-order residual accelerator
# --------------------------------------------------------------------------


@dataclass
class DoubleNSState:
    G: np.ndarray            # G_k
    L: np.ndarray            # L_k
    GamN: np.ndarray         # Gamma_k^n = I - L_k A
    F: np.ndarray            # F_k = I - G_k A
    k: int = 0


def double_ns_init(A: np.ndarray, T0: np.ndarray, n: int,
                   cnt: MMCount | None = None) -> DoubleNSState:
    """Precomputed start of Section 5.1: T_0 = G_0, Gamma_0 = I - T_0 A,
    L_0 = {sum_{j<n} Gamma_0^j} T_0, and G_0, F_0 = I - G_0 A."""
    L0 = ns_classical_step(T0, A, n, cnt)
    GamN0 = residual_left(L0, A, cnt)
    F0 = residual_left(T0, A, cnt)
    return DoubleNSState(G=T0.copy(), L=L0, GamN=GamN0, F=F0, k=0)


def double_ns_iterate(A: np.ndarray, st: DoubleNSState, n: int,
                      cnt: MMCount | None = None) -> DoubleNSState:
    """Section 5.1, eqs. gamk11-fks1:
        Gamma_k   = I - L_{k-1} A
        L_k       = {sum_{j<n} Gamma_k^j} L_{k-1}
        Gamma_k^n = I - L_k A
        G_k       = L_k + Gamma_k^n {sum_{j<n} F_{k-1}^j} G_{k-1}
        F_k       = I - G_k A = Gamma_k^n F_{k-1}^n."""
    L = ns_classical_step(st.L, A, n, cnt)
    GamN = residual_left(L, A, cnt)
    X = ns_classical_step(st.G, A, n, cnt)
    G = L + mm(GamN, X, cnt)
    F = residual_left(G, A)
    return DoubleNSState(G=G, L=L, GamN=GamN, F=F, k=st.k + 1)


def double_ns_exponent(n: int, h: int, k: int) -> int:
    """Eq. ermoex1: F_k = (S^{-1}D)^{h (k n^{k+1} + n^k)}."""
    return h * (k * n ** (k + 1) + n ** k)


# --------------------------------------------------------------------------
# Section 6: Richardson iteration
# --------------------------------------------------------------------------


def richardson_step(A: np.ndarray, B: np.ndarray, theta: np.ndarray,
                    G: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """theta_{k+1} = theta_k + G (B - A theta_k): the Richardson iteration of
    Section 6 (eq. ttk1 is theta_k = theta_{k-1} - omega_k (A theta_{k-1} - b))
    with omega = G, the current inverse estimate.  Returns (theta_new, R)."""
    R = B - A @ theta
    return theta + G @ R, R


def accelerated_richardson_step(A: np.ndarray, b: np.ndarray, theta: np.ndarray,
                                st: DoubleNSState, q: int) -> np.ndarray:
    """Eq. ttk1: theta_k = theta_{k-1} - [L_k + Gamma_k^n {sum_{j<q} F_k^j} G_k]
    (A theta_{k-1} - b), with L_k, Gamma_k^n, F_k, G_k of step k (Section 5.1)."""
    SG = ns_classical_step(st.G, A, q) if q > 1 else st.G
    omega = st.L + st.GamN @ SG
    return theta - omega @ (A @ theta - b)


def accelerated_richardson_exponent(n: int, h: int, k: int) -> float:
    """Eq. riem6 (q = n): gamma_k with theta~_k = (S^{-1}D)^{gamma_k} theta~_0."""
    num = k * n ** (k + 2) - (k - 1) * n ** (k + 1) - 2 * n ** k - n + 2
    return h * n * n * num / (n - 1) ** 2


def omega_recursive(A: np.ndarray, omega_prev: np.ndarray, SG_prev: np.ndarray,
                    GamN_prev: np.ndarray, L_prev: np.ndarray, n: int,
                    cnt: MMCount | None = None):
    """Section 6.2, eqs. redttk1, redttk2, gkrecu1.  With Gamma_k = Gamma_{k-1}^n
    and P(.) = sum_{j<n} (.)^j:
        G_k     = P(Gamma_k) [omega_{k-1} - P(F_{k-1}) G_{k-1}] + P(F_{k-1}) G_{k-1}
        L_k     = P(Gamma_k) L_{k-1},   Gamma_k^n = I - L_k A
        omega_k = L_k + Gamma_k^n P(F_k) G_k.
    ``SG_prev`` is P(F_{k-1}) G_{k-1}.  Returns (omega_k, P(F_k) G_k, Gamma_k^n, L_k, G_k)."""
    I = _eye_like(A)
    Gam = GamN_prev
    # P(Gamma_k) applied to a matrix M by Horner: M, Gam M + M, ...
    def P_apply(M):
        out = M.copy()
        for _ in range(n - 1):
            out = mm(Gam, out, cnt) + M
        return out
    G = P_apply(omega_prev - SG_prev) + SG_prev
    L = P_apply(L_prev)
    GamN = I - mm(L, A, cnt)
    SG = ns_classical_step(G, A, n, cnt)
    omega = L + mm(GamN, SG, cnt)
    return omega, SG, GamN, L, G


# --------------------------------------------------------------------------
# Drivers
# --------------------------------------------------------------------------


@dataclass
class SolveResult:
    theta: np.ndarray
    G: np.ndarray
    ns_iters: int
    sweeps: int
    converged: bool
    frob_E: list = field(default_factory=list)      # ||F_k||_F per NS step
    rel_res: list = field(default_factory=list)     # max_c ||r_c|| / ||b_c|| per sweep
    mmm: int = 0


def rel_residual(A: np.ndarray, theta: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Per right-hand side ||b_c - A theta_c||_2 / ||b_c||_2."""
    R = B - A @ theta
    return np.sqrt(np.sum(R * R, axis=0)) / np.sqrt(np.sum(B * B, axis=0))


# --------------------------------------------------------------------------
# Final check of an inverse estimate: ||I - A G||_F, the quantity whose powers
# bound the Newton-Schulz error (Section 3: F_k = F_0^{n^k}) and whose norm
# bounds the Richardson contraction (Section 6).  The exact value is one FP64
# product; Hutchinson's estimator replaces it by products with s random sign
# vectors z_j: E ||(I - A G) z||^2 = ||I - A G||_F^2 when the entries of z are
# independent +-1 (E z z^T = I), exactly so for every z when I - A G is
# diagonal (z_i^2 = 1).
# --------------------------------------------------------------------------

_U64 = (1 << 64) - 1


def splitmix64(seed: int, k: int) -> int:
    """Output number k (0-based) of SplitMix64 from state `seed` (Steele, Lea,
    Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
    state advances by the odd constant 0x9E3779B97F4A7C15, and each state is
    finalised by two xor-shift-multiply rounds and a last xor-shift.  Exact
    integer arithmetic mod 2^64."""
    z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & _U64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _U64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _U64
    return z ^ (z >> 31)


def rademacher_probes(n: int, s: int, seed: int) -> np.ndarray:
    """n x s matrix of +-1: entry (i, j) is -1 when the top bit of SplitMix64
    output j n + i is set (the library's documented probe layout)."""
    Z = np.empty((n, s))
    for j in range(s):
        for i in range(n):
            Z[i, j] = -1.0 if splitmix64(seed, j * n + i) >> 63 else 1.0
    return Z


def inverse_residual(A: np.ndarray, G: np.ndarray) -> float:
    """||I - A G||_F, formed with one product."""
    return float(np.linalg.norm(_eye_like(A) - A @ G))


def inverse_residual_hutchinson(A: np.ndarray, G: np.ndarray, s: int, seed: int) -> float:
    """sqrt((1/s) sum_j ||z_j - A (G z_j)||^2) over the s probes above."""
    Z = rademacher_probes(A.shape[0], s, seed)
    R = Z - A @ (G @ Z)
    return float(np.sqrt(np.sum(R * R) / s))


def ns_invert(A: np.ndarray, G0: np.ndarray | None = None, order: int = 2, iters: int = 10,
              form: str = "factorized", pow_mode: str = "square") -> tuple[np.ndarray, list]:
    """Run ``iters`` Newton-Schulz steps of the given order (Section 3, eq. ns,
    in the factorized right form).  G0 defaults to I/||A||_F.  Returns
    (G_iters, [||F_k||_F for k < iters])."""
    G = G0 if G0 is not None else alpha_frobenius(A) * _eye_like(A)
    norms = []
    for _ in range(iters):
        G, F = ns_step(A, G, order, form, pow_mode)
        norms.append(float(np.sqrt(np.sum(F * F))))
    return G, norms


def ns_richardson_solve(A: np.ndarray, B: np.ndarray, order: int = 4, ns_iters: int = 8,
                        tol: float | None = None, max_sweeps: int = 0,
                        theta0: np.ndarray | None = None, G0: np.ndarray | None = None,
                        form: str = "factorized", pow_mode: str = "square",
                        use_updated_G: bool = False, couple_frob: float = 0.0) -> SolveResult:
    """Newton-Schulz inversion coupled to Richardson iteration.

    Each pass first forms r = B - A theta and its relative residual
    max_c ||r_c||/||b_c|| (recorded; the solve stops when it is <= ``tol``).
    Then, while fewer than ``ns_iters`` Newton-Schulz steps were taken,
        theta <- theta + G_k r,   G_{k+1} = NS step of G_k
    (``use_updated_G`` applies G_{k+1} instead, the ordering of eq. ttk1 where
    the newest operator is applied); afterwards up to ``max_sweeps`` plain
    sweeps theta <- theta + G r with the last G.  The returned theta is always
    the one whose residual was recorded last.

    ``couple_frob`` > 0 delays the coupling (a library option; the paper
    couples from the first step): passes take the NS step alone until the
    first G_k with ||I - A G_k||_F <= ``couple_frob``; from that pass on (and
    once Newton-Schulz has stopped) every pass forms the residual and updates
    theta as above."""
    G = G0 if G0 is not None else alpha_frobenius(A) * _eye_like(A)
    theta = np.zeros_like(B) if theta0 is None else theta0.copy()
    bn = np.sqrt(np.sum(B * B, axis=0))
    res = SolveResult(theta=theta, G=G, ns_iters=0, sweeps=0, converged=False)
    cnt = MMCount()
    sweeps_left = max_sweeps
    coupled = couple_frob <= 0.0
    while True:
        if not coupled and res.ns_iters < ns_iters:
            # the norm of the F the coming step forms (not a separate mmm)
            E = residual_right(A, G)
            coupled = float(np.sqrt(np.sum(E * E))) <= couple_frob
        if not coupled and res.ns_iters < ns_iters:
            G_new, F = ns_step(A, G, order, form, pow_mode, cnt)
            res.frob_E.append(float(np.sqrt(np.sum(F * F))))
            G = G_new
            res.ns_iters += 1
            continue
        R = B - A @ theta
        rr = float(np.max(np.sqrt(np.sum(R * R, axis=0)) / bn))
        res.rel_res.append(rr)
        if tol is not None and rr <= tol:
            res.converged = True
            break
        if res.ns_iters < ns_iters:
            G_new, F = ns_step(A, G, order, form, pow_mode, cnt)
            res.frob_E.append(float(np.sqrt(np.sum(F * F))))
            theta = theta + (G_new if use_updated_G else G) @ R
            G = G_new
            res.ns_iters += 1
        elif sweeps_left > 0:
            theta = theta + G @ R
            sweeps_left -= 1
        else:
            break
        res.sweeps += 1
    res.theta, res.G, res.mmm = theta, G, cnt.n
    return res


# --------------------------------------------------------------------------
# Reduced-precision definitions used by the mixed-precision GEMMs
# (library design; the paper fixes no precision)
# --------------------------------------------------------------------------


def round_f32(x: np.ndarray) -> np.ndarray:
    """Round to nearest IEEE binary32 (ties to even), returned as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round binary32 values to bfloat16 (8-bit significand), round to nearest,
    ties to even, written out on the bit pattern: keep the top 16 bits of the
    binary32 word after adding 0x7FFF plus the lowest kept bit.  NaN stays NaN.
    Input is first rounded to binary32; the result is returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    r = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def round_tf32(x: np.ndarray) -> np.ndarray:
    """Round binary32 values to TF32 (binary32 with 10 stored significand bits,
    the low 13 bits zero): round to nearest, ties away from zero, written out
    on the sign-magnitude bit pattern -- add half of the dropped range
    (0x1000) to the magnitude and clear the low 13 bits.  A magnitude that
    carries past the largest finite value becomes infinity.  NaN stays NaN.
    Input is first rounded to binary32; the result is returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    sign = u & np.uint64(0x80000000)
    mag = u & np.uint64(0x7FFFFFFF)
    r = ((mag + np.uint64(0x1000)) & np.uint64(0xFFFFE000)) | sign
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def split_bf16(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two-term bfloat16 split of binary32 values: x32 = RN32(x),
    hi = RNbf16(x32), lo = RNbf16(x32 - hi) (the difference is exact in
    binary32).  hi + lo carries about 16 significand bits of x32."""
    x32 = round_f32(x)
    hi = round_bf16(x32)
    lo = round_bf16(round_f32(x32 - hi))
    return hi, lo


def split3_bf16(x: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Three-term bfloat16 split of binary32 values: hi and lo as in
    ``split_bf16``, lo2 = RNbf16(x32 - hi - lo).  Each difference is exact in
    binary32 and the last remainder fits a bfloat16, so hi + lo + lo2 = x32."""
    x32 = round_f32(x)
    hi = round_bf16(x32)
    r1 = round_f32(x32 - hi)
    lo = round_bf16(r1)
    lo2 = round_bf16(round_f32(r1 - lo))
    return hi, lo, lo2


# Split terms of each precision, as (L part, R part).  bf16x6 keeps every term
# whose parts' orders add to at most 2 (hi = 0, lo = 1, lo2 = 2): relative size
# down to 2^-16, dropping lo*lo2, lo2*lo, lo2*lo2 (2^-24 and below).
SPLIT_PASSES = {"bf16": (("hi", "hi"),),
                "bf16x2": (("hi", "hi"), ("lo", "hi")),
                "bf16x3": (("hi", "hi"), ("hi", "lo"), ("lo", "hi")),
                "bf16x6": (("hi", "hi"), ("hi", "lo"), ("lo", "hi"), ("hi", "lo2"), ("lo", "lo"), ("lo2", "hi"))}


def _split_parts(L: np.ndarray, R: np.ndarray, f=lambda v: v) -> dict:
    Lh, Ll, L2 = split3_bf16(L)
    Rh, Rl, R2 = split3_bf16(R)
    return {"hi": (f(Lh), f(Rh)), "lo": (f(Ll), f(Rl)), "lo2": (f(L2), f(R2))}


def split_product(L: np.ndarray, R: np.ndarray, precision: str) -> np.ndarray:
    """Exact (float64) value of the split product the tensor cores form:
    tf32:   RNtf32(L) RNtf32(R)   (one pass; operands rounded by round_tf32)
    bf16:   Lhi Rhi
    bf16x2: Lhi Rhi + Llo Rhi             (R's low part dropped)
    bf16x3: Lhi Rhi + Lhi Rlo + Llo Rhi   (the lo*lo term is dropped)
    bf16x6: those and Lhi Rlo2 + Llo Rlo + Llo2 Rhi.
    L and R are first rounded to binary32 and split with ``split3_bf16``
    (whose hi and lo are those of ``split_bf16``)."""
    if precision == "tf32":
        return round_tf32(round_f32(L)) @ round_tf32(round_f32(R))
    parts = _split_parts(L, R)
    out = np.zeros((L.shape[0], R.shape[1]))
    for a, b in SPLIT_PASSES[precision]:
        out += parts[a][0] @ parts[b][1]
    return out


def split_abs_product(L: np.ndarray, R: np.ndarray, precision: str) -> np.ndarray:
    """sum_k |L_ik| |R_kj| over the same split terms (for error bounds)."""
    if precision == "tf32":
        return np.abs(round_tf32(round_f32(L))) @ np.abs(round_tf32(round_f32(R)))
    parts = _split_parts(L, R, np.abs)
    out = np.zeros((L.shape[0], R.shape[1]))
    for a, b in SPLIT_PASSES[precision]:
        out += parts[a][0] @ parts[b][1]
    return out


# --------------------------------------------------------------------------
# FP64-accurate products from exact integer slices (an Ozaki-style error-free
# splitting: T. Ozaki, T. Ogita, S. M. Rump, S. Oishi, "Error-free
# transformations of matrix multiplication by using fast routines of matrix
# multiplication and its applications", Numer. Algorithms 59, 2012).  Each row
# i of L is written as mu_i sum_t 2^{-8t} A_t[i, :] and each column j of R as
# nu_j sum_u 2^{-8u} B_u[:, j] with integer slices |A_t|, |B_u| <= 255 and
# powers of two mu_i >= max_k |L_ik|, nu_j >= max_k |R_kj|; every slice
# product A_t B_u is then an exact integer matrix.
# --------------------------------------------------------------------------


def ozaki_scales(X: np.ndarray, axis: int) -> np.ndarray:
    """Power-of-two scale per row (axis = 1: max over each row) or per column
    (axis = 0): 2^e with max |x| = m 2^e, m in [0.5, 1), so |x| / scale < 1;
    1 for an all-zero line."""
    mx = np.max(np.abs(X), axis=axis)
    _, e = np.frexp(mx)
    return np.where(mx > 0, np.ldexp(1.0, e), 1.0)


def ozaki_slices(X: np.ndarray, scale: np.ndarray, axis: int, s: int) -> list:
    """Integer slices S_1..S_s of X / scale (scale broadcast along rows for
    axis = 1, along columns for axis = 0): x <- 256 x, S_t = trunc(x),
    x <- x - S_t, each step exact in binary64, |S_t| <= 255."""
    x = X / (scale[:, None] if axis == 1 else scale[None, :])
    out = []
    for _ in range(s):
        x = x * 256.0
        a = np.trunc(x)
        x = x - a
        out.append(a)
    return out


def ozaki_pairs(s: int) -> list:
    """Slice pairs (t, u), 1 <= t, u <= s, kept by the product: t + u <= s + 1
    (the others weigh at most 2^{-8(s+2)} relative), ordered by d = t + u."""
    return [(t, d - t) for d in range(2, s + 2) for t in range(1, d) if 1 <= d - t <= s]


def ozaki_product(L: np.ndarray, R: np.ndarray, s: int = 7) -> np.ndarray:
    """sum over kept pairs of mu_i nu_j 2^{-8(t+u)} (A_t B_u)_ij, with every
    A_t B_u formed exactly in integer arithmetic (int64) and the per-level sums
    S_d = sum_{t+u=d} A_t B_u combined in binary64."""
    mu = ozaki_scales(L, 1)
    nu = ozaki_scales(R, 0)
    A = [a.astype(np.int64) for a in ozaki_slices(L, mu, 1, s)]
    B = [b.astype(np.int64) for b in ozaki_slices(R, nu, 0, s)]
    out = np.zeros((L.shape[0], R.shape[1]))
    for d in range(2, s + 2):
        S = np.zeros_like(out, dtype=np.int64)
        for t, u in ozaki_pairs(s):
            if t + u == d:
                S += A[t - 1] @ B[u - 1]
        out += np.ldexp(S.astype(np.float64), -8 * d)
    return out * mu[:, None] * nu[None, :]


def ozaki_slices_signed(X: np.ndarray, scale: np.ndarray, axis: int, s: int) -> list:
    """Signed-digit slices of X / (2 scale), a second slicing rule for the same
    splitting: x starts in (-1/2, 1/2); x <- 256 x, S_t = RN(x) (nearest, ties
    to even), x <- x - S_t.  Every step is exact in binary64 (x - RN(x) is),
    |x| <= 1/2 after each step, so |S_t| <= 128 and
    X = 2 scale (sum_t S_t 256^{-t} + r) with |r| <= 256^{-s} / 2.  With digits
    of at most 2^7 a pair's products sum exactly in binary32 over 1024 of K
    (1024 * 2^14 = 2^24), four times the truncated slices' 256."""
    x = X / (2.0 * (scale[:, None] if axis == 1 else scale[None, :]))
    out = []
    for _ in range(s):
        x = x * 256.0
        a = np.rint(x)
        x = x - a
        out.append(a)
    return out


def ozaki_product_signed(L: np.ndarray, R: np.ndarray, s: int = 7) -> np.ndarray:
    """ozaki_product with the signed-digit slices: sum over the kept pairs of
    (2 mu_i)(2 nu_j) 2^{-8(t+u)} (A_t B_u)_ij, each A_t B_u exact in int64."""
    mu = ozaki_scales(L, 1)
    nu = ozaki_scales(R, 0)
    A = [a.astype(np.int64) for a in ozaki_slices_signed(L, mu, 1, s)]
    B = [b.astype(np.int64) for b in ozaki_slices_signed(R, nu, 0, s)]
    out = np.zeros((L.shape[0], R.shape[1]))
    for d in range(2, s + 2):
        S = np.zeros_like(out, dtype=np.int64)
        for t, u in ozaki_pairs(s):
            if t + u == d:
                S += A[t - 1] @ B[u - 1]
        out += np.ldexp(S.astype(np.float64), -8 * d)
    return out * (2.0 * mu)[:, None] * (2.0 * nu)[None, :]


def gemm_epilogue(prod: np.ndarray, s: float = 1.0, C: np.ndarray | None = None,
                  beta: float = 0.0, gamma: float = 0.0) -> np.ndarray:
    """D = s * prod + beta * C + gamma * I: the affine forms every step of the
    chain takes (F = I - A G: s = -1, gamma = 1; X + X P: beta = 1)."""
    D = s * prod
    if C is not None and beta != 0.0:
        D = D + beta * C
    if gamma != 0.0:
        D = D + gamma * np.eye(D.shape[0], D.shape[1])
    return D
