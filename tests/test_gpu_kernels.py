"""Kernel-level parity on the GPU, through the C ABI, against the FP64 oracle on
the same seeded inputs.

Tolerances follow from the arithmetic:
* bf16 splits are integer-like (round-to-nearest-even of a fixed value):
  compared bit for bit.
* Tensor-core products: every bf16 x bf16 product is exact in f32, so the only
  error is the f32 accumulation of K terms plus the f32 epilogue.  Whatever the
  summation order, |err| <= K * 2^-23 * sum_k |terms| + 2^-22 (|D| + |beta C|
  + |gamma|) (2^-23 allows truncating adds).  A dropped pass (2^-9 relative)
  or a wrong operand (O(1)) fails it.  The typical error is also checked:
  median(|err| / sum|terms|) <= 2^-20.
* FP64 products: |err| <= K * 2^-52 * sum|L||R| + 2^-51 |D|.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2008_11480_gb300 as nsgb

pytestmark = pytest.mark.gpu
dev = torch.device("cuda:0")


def rnd(shape, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal(shape) * scale


def to_dev_padded(X, ld, dtype=torch.float64):
    rows, cols = X.shape
    t = torch.zeros((rows, ld), dtype=dtype, device=dev)
    t[:, :cols] = torch.from_numpy(X).to(dtype)
    return t


def gpu_split(X, ld):
    rows, cols = X.shape
    x = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    hi = torch.zeros((rows, ld), dtype=torch.bfloat16, device=dev)
    lo = torch.zeros((rows, ld), dtype=torch.bfloat16, device=dev)
    nsgb.ns_k_split(x, hi, lo, rows, cols, cols, ld)
    return hi, lo


def rup(x, m=8):
    return (x + m - 1) // m * m


@pytest.mark.parametrize("rows,cols", [(1, 1), (7, 13), (130, 70), (64, 64), (513, 257)])
def test_split_bit_exact(rows, cols):
    X = rnd((rows, cols), 1, 10.0) * np.exp(np.random.default_rng(2).uniform(-20, 20, (rows, cols)))
    ld = rup(cols)
    hi, lo = gpu_split(X, ld)
    rh, rl = O.split_bf16(X)
    gh = hi.float().cpu().numpy()[:, :cols].astype(np.float64)
    gl = lo.float().cpu().numpy()[:, :cols].astype(np.float64)
    assert np.array_equal(gh, rh)
    assert np.array_equal(gl, rl)
    assert not torch.any(hi[:, cols:].float() != 0)


def run_gemm(prec, M, N, K, seed, s=1.0, beta=0.0, gamma=0.0, with_c=False, bn=0, scale=1.0, cm=0):
    L = rnd((M, K), seed, scale)
    R = rnd((K, N), seed + 1, scale)
    C = rnd((M, N), seed + 2) if with_c else None
    ldl, ldr, ldd = rup(K), rup(N), rup(N)
    Lh, Ll = gpu_split(L, ldl)
    Rh, Rl = gpu_split(R, ldr)
    Cd = to_dev_padded(O.round_f32(C), ldd, torch.float32) if with_c else None
    D32 = torch.full((M, ldd), 7.0, dtype=torch.float32, device=dev)
    Dh = torch.zeros((M, ldd), dtype=torch.bfloat16, device=dev)
    Dl = torch.zeros((M, ldd), dtype=torch.bfloat16, device=dev)
    fro = torch.zeros(1, dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_bf16(prec, M, N, K, Lh, Ll, ldl, Rh, Rl, ldr, s, Cd, ldd if with_c else 0, beta, gamma,
                        D32, ldd, Dh, Dl, ldd, fro, bn, cm)
    torch.cuda.synchronize()
    pname = {nsgb.NS_BF16: "bf16", nsgb.NS_BF16X3: "bf16x3", nsgb.NS_BF16X2: "bf16x2"}[prec]
    prod = O.split_product(L, R, pname)
    absprod = O.split_abs_product(L, R, pname)
    ref = O.gemm_epilogue(prod, s, O.round_f32(C) if with_c else None, beta, gamma)
    out = D32.cpu().numpy()[:, :N].astype(np.float64)
    assert np.all(D32.cpu().numpy()[:, N:] == 7.0), "wrote past N"
    cabs = np.abs(beta * O.round_f32(C)) if with_c else 0.0
    tol = K * 2.0 ** -23 * absprod * abs(s) + 2.0 ** -22 * (np.abs(ref) + cabs + abs(gamma)) + 1e-30
    err = np.abs(out - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"
    assert np.median(err / (absprod * abs(s) + 1e-30)) <= 2.0 ** -20
    hi = Dh.float().cpu().numpy()[:, :N].astype(np.float64)
    lo = Dl.float().cpu().numpy()[:, :N].astype(np.float64)
    assert np.all(np.abs(hi + lo - ref) <= tol + 2.0 ** -16 * np.abs(ref))
    assert np.all(np.abs(hi - ref) <= tol + 2.0 ** -8 * np.abs(ref))
    f = float(fro.item())
    assert f == pytest.approx(float(np.sum(ref * ref)), rel=1e-4)
    return err, tol


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (130, 200, 70), (256, 512, 1024), (64, 64, 64), (1, 1, 1),
                                   (17, 33, 9), (300, 130, 257)])
def test_gemm_tc_plain(prec, M, N, K):
    run_gemm(prec, M, N, K, seed=M + N + K)


@pytest.mark.parametrize("M,N,K", [(256, 512, 1024), (130, 200, 70), (300, 130, 257), (640, 768, 333), (1, 1, 1)])
def test_gemm_two_term_pairs(M, N, K):
    """NS_BF16X2 (Lhi Rhi + Llo Rhi, CTA pairs, any row-tile count) against the
    oracle's bf16x2 terms, with the C and identity terms of the NS epilogue."""
    run_gemm(nsgb.NS_BF16X2, M, N, K, seed=3 * M + K, s=-1.0, beta=1.0, with_c=True, gamma=1.0)


@pytest.mark.parametrize("bn", [64, 128, 256])
@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
def test_gemm_tc_tile_widths(prec, bn):
    run_gemm(prec, 390, 520, 200, seed=11, bn=bn)


@pytest.mark.parametrize("bn", [192, 256])
@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
@pytest.mark.parametrize("M,N,K", [(512, 520, 200), (300, 400, 129), (1024, 1024, 1024)])
def test_gemm_tc_wide_tiles_one_cta(prec, bn, M, N, K):
    """Wide tiles on the one-CTA kernel (cluster_m = 1; bf16x3 with 192-column
    tiles runs as three one-pass products); M = 300 leaves a last tile row
    mostly past the matrix."""
    run_gemm(prec, M, N, K, seed=M + bn, bn=bn, cm=1, s=-1.0, gamma=1.0, scale=0.05)


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (250, 300, 129), (200, 130, 33), (512, 520, 200),
                                   (1024, 1024, 1024)])
def test_gemm_tc_pair(prec, M, N, K):
    """CTA pairs sharing each MMA (cta_group::2): 256 x 256 tiles split as two
    128-row halves in two TMEMs, R columns split between the two shared
    memories.  Ragged M, N and K tails; s = -1, gamma = 1 as in F = I - A G."""
    run_gemm(prec, M, N, K, seed=M + N + K + 7, bn=256, cm=-2, s=-1.0, gamma=1.0, scale=0.05)


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
@pytest.mark.parametrize("M,N,K", [(3072, 2048, 192), (3584, 2304, 128)])
def test_gemm_tc_pair_waves(prec, M, N, K):
    """Wave balance of the pair kernel on 152 SMs (76 pairs): 96 tiles leave a
    last wave of 20, run as 40 half-width items; 126 tiles leave 50, which
    would not fit one wave as halves and run whole.  (Fewer tiles than pairs,
    in the cases above, run entirely as halves.)"""
    run_gemm(prec, M, N, K, seed=M + N + K + 9, bn=256, cm=-2, s=-1.0, gamma=1.0, scale=0.05)


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
def test_gemm_tc_pair_accumulate_epilogue(prec):
    """X + X P form through CTA pairs: C = X, beta = 1."""
    run_gemm(prec, 500, 333, 333, seed=16, beta=1.0, with_c=True, bn=256, cm=-2)


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
def test_gemm_tc_residual_epilogue(prec):
    """F = I - A G form: s = -1, gamma = 1 on a square problem."""
    run_gemm(prec, 200, 200, 200, seed=5, s=-1.0, gamma=1.0, scale=0.07)


@pytest.mark.parametrize("prec", [nsgb.NS_BF16, nsgb.NS_BF16X3])
def test_gemm_tc_accumulate_epilogue(prec):
    """X + X P form: C = X, beta = 1."""
    run_gemm(prec, 333, 333, 333, seed=6, beta=1.0, with_c=True)


@pytest.mark.parametrize("prec,bn,cm", [(nsgb.NS_BF16X3, 256, 1), (nsgb.NS_BF16X3, 256, -2),
                                        (nsgb.NS_BF16, 256, 1), (nsgb.NS_BF16, 256, -2)])
def test_gemm_tc_full_size_sampled(prec, bn, cm):
    """4096^3 products (the bench's product size and launch configurations):
    sampled outputs recomputed one by one by the oracle."""
    n = 4096
    pname = "bf16x3" if prec == nsgb.NS_BF16X3 else "bf16"
    rng = np.random.default_rng(40)
    L = rng.standard_normal((n, n)) * 0.02
    R = rng.standard_normal((n, n)) * 0.02
    Lh, Ll = gpu_split(L, n)
    Rh, Rl = gpu_split(R, n)
    D32 = torch.zeros((n, n), dtype=torch.float32, device=dev)
    nsgb.ns_k_gemm_bf16(prec, n, n, n, Lh, Ll, n, Rh, Rl, n, -1.0, None, 0, 0.0, 1.0, D32, n,
                        None, None, 0, None, bn, cm)
    torch.cuda.synchronize()
    idx = rng.integers(0, n, (96, 2))
    idx[:8, 1] = idx[:8, 0]   # include diagonal entries (identity term)
    out = D32.cpu().numpy()
    for i, j in idx:
        p = O.split_product(L[i:i + 1], R[:, j:j + 1], pname)[0, 0]
        a = O.split_abs_product(L[i:i + 1], R[:, j:j + 1], pname)[0, 0]
        ref = -p + (1.0 if i == j else 0.0)
        tol = n * 2.0 ** -23 * a + 2.0 ** -22 * (abs(ref) + 1.0)
        assert abs(out[i, j] - ref) <= tol, (i, j, out[i, j], ref)


@pytest.mark.parametrize("M,N,K", [(64, 64, 64), (130, 70, 33), (1, 1, 1), (200, 300, 150),
                                   # 76 or more 64 x 64 output tiles: the large-tile kernel
                                   # k_gemm_f64 (the plain FP64 path's product from n = 576 on),
                                   # with ragged row, column and K tails
                                   (640, 576, 200), (1000, 1030, 333), (1024, 1024, 1024)])
def test_gemm_f64(M, N, K):
    L, R, C = rnd((M, K), 1), rnd((K, N), 2), rnd((M, N), 3)
    Ld, Rd, Cd = (torch.from_numpy(x).to(dev) for x in (L, R, C))
    D = torch.zeros((M, N), dtype=torch.float64, device=dev)
    fro = torch.zeros(1, dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_f64(M, N, K, Ld, K, Rd, N, -0.5, Cd, N, 2.0, 1.0, D, N, fro)
    torch.cuda.synchronize()
    ref = O.gemm_epilogue(L @ R, -0.5, C, 2.0, 1.0)
    tol = K * 2.0 ** -52 * 0.5 * (np.abs(L) @ np.abs(R)) + 2.0 ** -51 * (np.abs(ref) + 2 * np.abs(C) + 1)
    assert np.all(np.abs(D.cpu().numpy() - ref) <= tol)
    assert float(fro.item()) == pytest.approx(float(np.sum(ref * ref)), rel=1e-12)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (64, 1), (130, 3), (257, 9), (1000, 4), (33, 16)])
def test_resid_and_update(n, nrhs):
    A, Th, B = rnd((n, n), 4), rnd((n, nrhs), 5), rnd((n, nrhs), 6)
    Ad, Thd, Bd = (torch.from_numpy(x).to(dev) for x in (A, Th, B))
    R = torch.zeros((n, nrhs), dtype=torch.float64, device=dev)
    rsq = torch.zeros(nrhs, dtype=torch.float64, device=dev)
    nsgb.ns_k_resid(Ad, n, Thd, Bd, R, n, nrhs, rsq)
    torch.cuda.synchronize()
    ref = B - A @ Th
    tol = n * 2.0 ** -52 * (np.abs(A) @ np.abs(Th) + np.abs(B))
    assert np.all(np.abs(R.cpu().numpy() - ref) <= tol)
    assert np.allclose(rsq.cpu().numpy(), np.sum(ref * ref, axis=0), rtol=1e-12)
    # update with an FP64 gain: Theta += G R
    G = rnd((n, n), 7)
    Gd = torch.from_numpy(G).to(dev)
    th1 = Thd.clone()
    nsgb.ns_k_update(Gd, n, R, th1, n, nrhs)
    torch.cuda.synchronize()
    Rn = R.cpu().numpy()
    ref1 = Th + G @ Rn
    tol1 = n * 2.0 ** -52 * (np.abs(G) @ np.abs(Rn)) + 2.0 ** -52 * np.abs(ref1)
    assert np.all(np.abs(th1.cpu().numpy() - ref1) <= tol1)
    # update with an f32 gain: products and lane sums in f32 (ceil(n/32) terms per lane)
    G32 = O.round_f32(G)
    G32d = torch.from_numpy(G32).to(dev).float()
    th2 = Thd.clone()
    nsgb.ns_k_update(G32d, n, R, th2, n, nrhs)
    torch.cuda.synchronize()
    ref2 = Th + G32 @ Rn
    terms = -(-n // 32) + 2
    tol2 = terms * 2.0 ** -23 * (np.abs(G32) @ np.abs(Rn)) + 2.0 ** -52 * np.abs(ref2)
    assert np.all(np.abs(th2.cpu().numpy() - ref2) <= tol2)


@pytest.mark.parametrize("n", [1, 7, 130, 1000])
def test_prep_a_bit_exact(n):
    """Fused pass over A: bf16 hi/lo and f32 limbs equal the oracle's
    definitions bit for bit; the norms match to rounding."""
    A = rnd((n, n), 21) * np.exp(np.random.default_rng(22).uniform(-5, 5, (n, n)))
    ld = rup(n, 8)
    Ad = torch.from_numpy(A).to(dev)
    hi = torch.zeros((n, ld), dtype=torch.bfloat16, device=dev)
    lo = torch.zeros_like(hi)
    a1 = torch.zeros((n, ld), dtype=torch.float32, device=dev)
    a2 = torch.zeros_like(a1)
    ss = torch.zeros(1, dtype=torch.float64, device=dev)
    rm = torch.zeros(1, dtype=torch.float64, device=dev)
    nsgb.ns_k_prep_a(Ad, n, n, hi, lo, a1, a2, ld, ss, rm)
    torch.cuda.synchronize()
    rh, rl = O.split_bf16(A)
    assert np.array_equal(hi.float().cpu().numpy()[:, :n].astype(np.float64), rh)
    assert np.array_equal(lo.float().cpu().numpy()[:, :n].astype(np.float64), rl)
    r1 = O.round_f32(A)
    r2 = O.round_f32(A - r1)
    assert np.array_equal(a1.cpu().numpy()[:, :n].astype(np.float64), r1)
    assert np.array_equal(a2.cpu().numpy()[:, :n].astype(np.float64), r2)
    assert float(ss.item()) == pytest.approx(float(np.sum(A * A)), rel=1e-13)
    assert float(rm.item()) == pytest.approx(float(np.max(np.sum(np.abs(A), axis=1))), rel=1e-13)


def test_prep_a_split_edge_cases():
    """The two-limb split on values chosen to hit its corner cases: ties at
    the 24-bit rounding point (both parities), significands of all ones
    (rounding carries into the exponent), both ends of the integer fast path
    (|v| near 2^-74 and 2^127) and beyond, doubles that are exactly floats,
    zeros and negative values; limbs equal RN32(v) and RN32(v - RN32(v))."""
    rng = np.random.default_rng(31)
    vals = []
    for e in (-80, -75, -74, -73, -30, -1, 0, 1, 30, 100, 126, 127):
        for sig in (0x0000000000000, 0xFFFFFFFFFFFFF, 0x0000010000000, 0x0000030000000, 0x0000010000001,
                    0x000002FFFFFFF, 0x8000010000000):
            bits = ((e + 1023) << 52) | sig
            vals.append(np.array([bits], dtype=np.uint64).view(np.float64)[0])
    vals += [0.0, -0.0, 1.0, -1.0, 3.0e38, -3.0e38, 1e-300, -1e-300, 5e-324, 2.0 ** -126, 1.5 * 2.0 ** -149]
    vals = np.array(vals)
    with np.errstate(over="ignore"):
        vals = vals[np.isfinite(O.round_f32(vals))]  # leave out values whose f32 rounding overflows
    vals = np.concatenate([vals, -vals, rng.standard_normal(8) * 2.0 ** rng.integers(-70, 120, 8)])
    n = 64
    A = np.resize(vals, (n, n)).copy()
    hi = torch.zeros((n, n), dtype=torch.bfloat16, device=dev)
    lo = torch.zeros_like(hi)
    a1 = torch.zeros((n, n), dtype=torch.float32, device=dev)
    a2 = torch.zeros_like(a1)
    nsgb.ns_k_prep_a(torch.from_numpy(A).to(dev), n, n, hi, lo, a1, a2, n)
    torch.cuda.synchronize()
    r1 = O.round_f32(A)
    r2 = O.round_f32(A - r1)
    g1 = a1.cpu().numpy().astype(np.float64)
    g2 = a2.cpu().numpy().astype(np.float64)
    assert np.array_equal(g1, r1)
    assert np.array_equal(g2, r2)
    rh, rl = O.split_bf16(A)
    assert np.array_equal(hi.float().cpu().numpy().astype(np.float64), rh)
    assert np.array_equal(lo.float().cpu().numpy().astype(np.float64), rl)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (64, 1), (130, 3), (257, 9), (1000, 4), (4096, 4)])
def test_resid_x2(n, nrhs):
    """R = B - A Theta from f32 limbs (double-f32 accumulation).  Bound: split
    and product corrections <= 2^-45 sum|a||theta| per row, the f32 'lo'
    accumulator over m = ceil(n/32) terms per lane <= 2 m^2 2^-48 sum|a||theta|,
    FP64 combination <= 2^-50 (|B| + sum|a||theta|)."""
    rng = np.random.default_rng(n + nrhs)
    A = rng.standard_normal((n, n))
    Th = rng.standard_normal((n, nrhs))
    B = A @ Th + 1e-6 * rng.standard_normal((n, nrhs))   # near-cancelling residual
    ld = rup(n, 8)
    Ad = torch.from_numpy(A).to(dev)
    hi = torch.zeros((n, ld), dtype=torch.bfloat16, device=dev)
    lo = torch.zeros_like(hi)
    a1 = torch.zeros((n, ld), dtype=torch.float32, device=dev)
    a2 = torch.zeros_like(a1)
    nsgb.ns_k_prep_a(Ad, n, n, hi, lo, a1, a2, ld)
    R = torch.zeros((n, nrhs), dtype=torch.float64, device=dev)
    rsq = torch.zeros(nrhs, dtype=torch.float64, device=dev)
    nsgb.ns_k_resid_x2(a1, a2, ld, torch.from_numpy(Th).to(dev), torch.from_numpy(B).to(dev), R, n, nrhs, rsq)
    torch.cuda.synchronize()
    ref = B - A @ Th
    absp = np.abs(A) @ np.abs(Th)
    m = -(-n // 32)
    tol = (2.0 ** -45 + 2 * m * m * 2.0 ** -48 + 2.0 ** -50) * absp + 2.0 ** -50 * np.abs(B)
    err = np.abs(R.cpu().numpy() - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"
    assert np.median(err / absp) <= 2.0 ** -44
    assert np.allclose(rsq.cpu().numpy(), np.sum(ref * ref, axis=0), rtol=1e-6)


# ---------------------------------------------------------------- split-bf16 x6
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rows,cols", [(1, 1), (130, 70), (513, 257)])
def test_split3_bit_exact(dtype, rows, cols):
    X = rnd((rows, cols), 90 + rows, scale=3.0)
    ld = rup(cols)
    Xd = torch.from_numpy(X).to(dev).to(dtype)
    parts = [torch.zeros((rows, ld), dtype=torch.bfloat16, device=dev) for _ in range(3)]
    nsgb.ns_k_split3(Xd, *parts, rows, cols, cols, ld)
    torch.cuda.synchronize()
    want = O.split3_bf16(Xd.double().cpu().numpy())
    for got, w in zip(parts, want):
        assert np.array_equal(got[:, :cols].double().cpu().numpy(), w)


def gpu_split3(X, ld):
    Xd = to_dev_padded(X, ld)
    parts = [torch.zeros((X.shape[0], ld), dtype=torch.bfloat16, device=dev) for _ in range(3)]
    nsgb.ns_k_split3(Xd, *parts, X.shape[0], X.shape[1], ld, ld)
    return parts


def run_gemm_x6(M, N, K, seed, s=1.0, beta=0.0, gamma=0.0, with_c=False, scale=1.0, frob=True):
    L = rnd((M, K), seed, scale)
    R = rnd((K, N), seed + 1, scale)
    C = rnd((M, N), seed + 2) if with_c else None
    ldl, ldr, ldd = rup(K), rup(N), rup(N)
    Lp, Rp = gpu_split3(L, ldl), gpu_split3(R, ldr)
    Cd = to_dev_padded(O.round_f32(C), ldd, torch.float32) if with_c else None
    D32 = torch.full((M, ldd), 7.0, dtype=torch.float32, device=dev)
    Dp = [torch.zeros((M, ldd), dtype=torch.bfloat16, device=dev) for _ in range(3)]
    fro = torch.zeros(1, dtype=torch.float64, device=dev) if frob else None
    nsgb.ns_k_gemm_bf16x6(M, N, K, Lp, ldl, Rp, ldr, s, Cd, ldd if with_c else 0, beta, gamma, D32, ldd, Dp, ldd,
                          fro)
    torch.cuda.synchronize()
    prod = O.split_product(L, R, "bf16x6")
    absprod = O.split_abs_product(L, R, "bf16x6")
    ref = O.gemm_epilogue(prod, s, O.round_f32(C) if with_c else None, beta, gamma)
    out = D32.cpu().numpy()[:, :N].astype(np.float64)
    assert np.all(D32.cpu().numpy()[:, N:] == 7.0), "wrote past N"
    cabs = np.abs(beta * O.round_f32(C)) if with_c else 0.0
    tol = K * 2.0 ** -23 * absprod * abs(s) + 2.0 ** -22 * (np.abs(ref) + cabs + abs(gamma)) + 1e-30
    err = np.abs(out - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"
    # the three outputs are the exact split of the f32 result
    parts = [d.double().cpu().numpy()[:, :N] for d in Dp]
    assert np.array_equal(parts[0] + parts[1] + parts[2], out)
    want = O.split3_bf16(out)
    for got, w in zip(parts, want):
        assert np.array_equal(got, w)
    if frob:
        assert float(fro.item()) == pytest.approx(float(np.sum(out * out)), rel=1e-6)
    return err, tol


@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (250, 300, 129), (200, 130, 33), (384, 520, 200),
                                   (1, 1, 1), (640, 512, 1024)])
def test_gemm_x6_pairs(M, N, K):
    """Split-bf16 x6 on CTA pairs: six terms per 32-deep K slice; ragged tails
    and odd row-tile counts (M = 384, 640: the last pair's second CTA lies past
    M); the F = I - A G epilogue."""
    run_gemm_x6(M, N, K, seed=M + 3 * N + K, s=-1.0, gamma=1.0, scale=0.05)


def test_gemm_x6_accumulate_epilogue():
    run_gemm_x6(500, 333, 333, seed=17, beta=1.0, with_c=True)


def test_gemm_x6_reproduces_binary32_operand():
    """L I with R = I adds nothing but zeros, so the product is exact in any
    accumulator: bf16x6 must give L's binary32 values bit for bit (hi + lo +
    lo2 = x32), while bf16x3 gives hi + lo and loses the third part."""
    M = K = N = 256
    L = rnd((M, K), 5, 1.0)
    R = np.eye(K, N)
    L32 = O.round_f32(L)
    Lp, Rp = gpu_split3(L, K), gpu_split3(R, N)
    D6 = torch.zeros((M, N), dtype=torch.float32, device=dev)
    nsgb.ns_k_gemm_bf16x6(M, N, K, Lp, K, Rp, N, 1.0, None, 0, 0.0, 0.0, D6, N)
    D3 = torch.zeros((M, N), dtype=torch.float32, device=dev)
    nsgb.ns_k_gemm_bf16(nsgb.NS_BF16X3, M, N, K, Lp[0], Lp[1], K, Rp[0], Rp[1], N, 1.0, None, 0, 0.0, 0.0, D3, N)
    torch.cuda.synchronize()
    assert np.array_equal(D6.cpu().numpy().astype(np.float64), L32)
    hi, lo, lo2 = O.split3_bf16(L)
    assert np.array_equal(D3.cpu().numpy().astype(np.float64), hi + lo)
    assert np.count_nonzero(lo2) > M * K // 2


def test_gemm_x6_full_size_sampled():
    """4096^3 bf16x6 (the launch the solve uses past the bf16x3 floor): sampled
    outputs recomputed one by one by the oracle."""
    n = 4096
    rng = np.random.default_rng(41)
    L = rng.standard_normal((n, n)) * 0.02
    R = rng.standard_normal((n, n)) * 0.02
    Lp, Rp = gpu_split3(L, n), gpu_split3(R, n)
    D32 = torch.zeros((n, n), dtype=torch.float32, device=dev)
    nsgb.ns_k_gemm_bf16x6(n, n, n, Lp, n, Rp, n, -1.0, None, 0, 0.0, 1.0, D32, n)
    torch.cuda.synchronize()
    idx = rng.integers(0, n, (64, 2))
    idx[:8, 1] = idx[:8, 0]
    out = D32.cpu().numpy()
    for i, j in idx:
        p = O.split_product(L[i:i + 1], R[:, j:j + 1], "bf16x6")[0, 0]
        a = O.split_abs_product(L[i:i + 1], R[:, j:j + 1], "bf16x6")[0, 0]
        ref = -p + (1.0 if i == j else 0.0)
        tol = n * 2.0 ** -23 * a + 2.0 ** -22 * (abs(ref) + 1.0)
        assert abs(out[i, j] - ref) <= tol, (i, j, out[i, j], ref)


# ---------------------------------------------------------------- FP64-accurate products from signed-digit slices
def run_gemm_oz(M, N, K, seed, s=1.0, beta=0.0, gamma=0.0, with_c=False, slices=7, spread=True):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((M, K))
    R = rng.standard_normal((K, N))
    if spread:  # rows and columns of very different magnitudes: the scales must follow them
        L *= 10.0 ** rng.integers(-6, 6, (M, 1))
        R *= 10.0 ** rng.integers(-6, 6, (1, N))
    C = rng.standard_normal((M, N)) if with_c else None
    Ld, Rd = torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)
    Cd = torch.from_numpy(C).to(dev) if with_c else None
    D = torch.full((M, N), 7.0, dtype=torch.float64, device=dev)
    fro = torch.zeros(1, dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_oz(M, N, K, Ld, K, Rd, N, s, Cd, N if with_c else 0, beta, gamma, D, N, slices, fro)
    torch.cuda.synchronize()
    prod = O.ozaki_product_signed(L, R, slices)
    ref = O.gemm_epilogue(prod, s, C, beta, gamma)
    out = D.cpu().numpy()
    ab = np.abs(L) @ np.abs(R)
    # same digits and exact integer level sums; only the binary64 combination
    # of the levels (the kernel: two int64 groups, three roundings; the
    # oracle: one rounding per level) differs
    tol = 16 * 2.0 ** -53 * (abs(s) * ab + np.abs(ref)) + 1e-300
    err = np.abs(out - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"
    assert float(fro.item()) == pytest.approx(float(np.sum(out * out)), rel=1e-12)
    return L, R, out


@pytest.mark.parametrize("M,N,K", [(256, 128, 256), (300, 200, 130), (513, 257, 1000), (128, 64, 4096), (1, 1, 1),
                                   (640, 384, 33)])
def test_gemm_oz_matches_oracle(M, N, K):
    run_gemm_oz(M, N, K, seed=M + 7 * N + K)


def test_gemm_oz_epilogues_and_slices():
    run_gemm_oz(300, 300, 300, seed=3, s=-1.0, gamma=1.0, spread=False)
    run_gemm_oz(257, 129, 200, seed=4, beta=1.0, with_c=True)
    run_gemm_oz(200, 160, 300, seed=5, slices=3)


@pytest.mark.parametrize("slices", [2, 3, 4, 5, 6])
def test_gemm_oz_slice_counts(slices):
    """Every digit count: levels d = 2 .. s + 1, each with its own exactly
    summed chunk length (1024 / (d - 1) of K) and int64 grouping (levels
    2..5 and 6..s+1), against the oracle's signed-digit product; K spans
    several chunks of every level and a ragged last one."""
    run_gemm_oz(520, 300, 1100, seed=50 + slices, slices=slices, s=-1.0, gamma=1.0)


def test_gemm_oz_K_in_blocks():
    """K beyond one level-kernel launch (16384): the blocks are sliced with
    their own scales and added into D; against the exact product."""
    M, N, K = 130, 70, 20000
    rng = np.random.default_rng(60)
    L, R, C = rng.standard_normal((M, K)), rng.standard_normal((K, N)), rng.standard_normal((M, N))
    D = torch.zeros((M, N), dtype=torch.float64, device=dev)
    fro = torch.zeros(1, dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_oz(M, N, K, torch.from_numpy(L).to(dev), K, torch.from_numpy(R).to(dev), N, 0.5,
                      torch.from_numpy(C).to(dev), N, 2.0, 1.0, D, N, 7, fro)
    torch.cuda.synchronize()
    out = D.cpu().numpy()
    exact = (0.5 * (L.astype(np.longdouble) @ R.astype(np.longdouble)) + 2.0 * C + np.eye(M, N)).astype(np.float64)
    ab = np.abs(L) @ np.abs(R)
    assert np.all(np.abs(out - exact) <= 16 * 2.0 ** -53 * (ab + np.abs(exact)))
    assert float(fro.item()) == pytest.approx(float(np.sum(out * out)), rel=1e-12)


def test_gemm_oz_fp64_accuracy():
    """Against the product in (quad on the GPU machine's host, else extended)
    precision the slice product is as accurate as binary64 allows: far inside
    an FP64 GEMM's K u |L||R| bound, and exact for small integer matrices."""
    L, R, out = run_gemm_oz(200, 150, 2048, seed=6)
    exact = (L.astype(np.longdouble) @ R.astype(np.longdouble)).astype(np.float64)
    ab = np.abs(L) @ np.abs(R)
    assert np.all(np.abs(out - exact) <= 8 * 2.0 ** -53 * ab + 4 * 2.0 ** -53 * np.abs(exact))
    rng = np.random.default_rng(7)
    Li = rng.integers(-1000, 1000, (130, 300)).astype(float)
    Ri = rng.integers(-1000, 1000, (300, 70)).astype(float)
    D = torch.zeros((130, 70), dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_oz(130, 70, 300, torch.from_numpy(Li).to(dev), 300, torch.from_numpy(Ri).to(dev), 70, D=D, ldd=70)
    torch.cuda.synchronize()
    assert np.array_equal(D.cpu().numpy(), Li @ Ri)


def test_gemm_oz_full_size_sampled():
    """n = 4096 (seven slices, 28 slice pairs, 16 chunks): sampled entries
    against the exact dot product."""
    n = 4096
    rng = np.random.default_rng(42)
    L = rng.standard_normal((n, n))
    R = rng.standard_normal((n, n))
    D = torch.zeros((n, n), dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_oz(n, n, n, torch.from_numpy(L).to(dev), n, torch.from_numpy(R).to(dev), n, -1.0, None, 0, 0.0,
                      1.0, D, n, 7)
    torch.cuda.synchronize()
    out = D.cpu().numpy()
    idx = rng.integers(0, n, (64, 2))
    idx[:8, 1] = idx[:8, 0]
    for i, j in idx:
        ex = float(-(L[i].astype(np.longdouble) @ R[:, j].astype(np.longdouble)) + (1.0 if i == j else 0.0))
        ab = float(np.abs(L[i]) @ np.abs(R[:, j]))
        assert abs(out[i, j] - ex) <= 16 * 2.0 ** -53 * (ab + abs(ex)), (i, j)


# ---------------------------------------------------------------- TF32 products (tcgen05 kind::tf32)
def run_gemm_tf32(M, N, K, seed, s=1.0, beta=0.0, gamma=0.0, with_c=False):
    """D = s RN_tf32(L) RN_tf32(R) + beta C + gamma I against the oracle's
    split_product("tf32"): the product of the rounded operands is exact in
    float64 and the kernel adds K of them in f32, so the bound is the bf16
    one (K 2^-23 sum|terms| + 2^-22 (|D| + |beta C| + |gamma|)).  The TF32
    forms the epilogue writes for the next product are RN_tf32 of the kernel's
    own D32, bit for bit, row-major and transposed."""
    rng = np.random.default_rng(seed)
    L = O.round_f32(rng.standard_normal((M, K)))
    R = O.round_f32(rng.standard_normal((K, N)))
    C = O.round_f32(rng.standard_normal((M, N))) if with_c else None
    ldl, ldr, ldd = rup(K, 4), rup(N, 4), rup(N, 4)
    ldt = rup(max(M, N), 4)
    Ld = to_dev_padded(L, ldl, torch.float32)
    Rd = to_dev_padded(R, ldr, torch.float32)
    Cd = to_dev_padded(C, ldd, torch.float32) if with_c else None
    D32 = torch.full((M, ldd), 7.0, dtype=torch.float32, device=dev)
    Dt = torch.zeros((M, ldt), dtype=torch.float32, device=dev)
    DtT = torch.zeros((N, ldt), dtype=torch.float32, device=dev)
    fro = torch.zeros(1, dtype=torch.float64, device=dev)
    nsgb.ns_k_gemm_tf32(M, N, K, Ld, ldl, Rd, ldr, s, Cd, ldd if with_c else 0, beta, gamma, D32, ldd, Dt, DtT, ldt,
                        fro)
    torch.cuda.synchronize()
    prod = O.split_product(L, R, "tf32")
    absprod = O.split_abs_product(L, R, "tf32")
    ref = O.gemm_epilogue(prod, s, C, beta, gamma)
    out = D32.cpu().numpy()[:, :N].astype(np.float64)
    assert np.all(D32.cpu().numpy()[:, N:] == 7.0), "wrote past N"
    cabs = np.abs(beta * C) if with_c else 0.0
    tol = K * 2.0 ** -23 * absprod * abs(s) + 2.0 ** -22 * (np.abs(ref) + cabs + abs(gamma)) + 1e-30
    err = np.abs(out - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"
    # a bf16 product of the same operands would be off by ~2^-8: TF32 keeps 2^-11
    assert np.median(err / (absprod * abs(s) + 1e-30)) <= 2.0 ** -20
    want_t = O.round_tf32(out)
    assert np.array_equal(Dt.cpu().numpy()[:, :N].astype(np.float64), want_t)
    assert np.array_equal(DtT.cpu().numpy()[:, :M].astype(np.float64), want_t.T)
    assert float(fro.item()) == pytest.approx(float(np.sum(out * out)), rel=1e-5)


@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 130, 257), (512, 520, 200), (1024, 1024, 1024),
                                   (129, 1000, 31)])
def test_gemm_tf32(M, N, K):
    """TF32 CTA-pair products: whole and ragged tiles, an odd number of 128-row
    tiles (the last pair's second CTA covers rows past M), K not a multiple of
    the 32-deep stage."""
    run_gemm_tf32(M, N, K, seed=M + 3 * N + K)


def test_gemm_tf32_epilogues():
    run_gemm_tf32(333, 333, 333, seed=8, s=-1.0, gamma=1.0)
    run_gemm_tf32(257, 300, 129, seed=9, beta=1.0, with_c=True)


def test_gemm_tf32_differs_from_bf16():
    """The TF32 path really reads 10 stored bits: on operands that bf16 rounds
    but TF32 keeps exactly (11 significant bits) the TF32 product is exact."""
    rng = np.random.default_rng(10)
    M = N = 256
    K = 16  # products are multiples of 2^-20 below 1, so K = 16 of them sum exactly within 24 bits
    L = rng.integers(-1023, 1024, (M, K)).astype(np.float64) / 1024.0
    R = rng.integers(-1023, 1024, (K, N)).astype(np.float64) / 1024.0
    Ld, Rd = to_dev_padded(L, K, torch.float32), to_dev_padded(R, N, torch.float32)
    D32 = torch.zeros((M, N), dtype=torch.float32, device=dev)
    nsgb.ns_k_gemm_tf32(M, N, K, Ld, K, Rd, N, 1.0, None, 0, 0.0, 0.0, D32, N)
    torch.cuda.synchronize()
    exact = L @ R
    assert np.array_equal(D32.cpu().numpy().astype(np.float64), exact)
    assert not np.array_equal(O.round_bf16(L), L)  # bf16 would have rounded the operands
