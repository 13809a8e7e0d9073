"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/nsgb.h declares, its structs have the layout the
binding assumes, and argument validation answers before any CUDA call."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_2008_11480_gb300 as nsgb
from paper_2008_11480_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return nsgb.lib()


def test_exports_every_declared_symbol(L):
    names = nsgb.declared_functions()
    assert "ns_create" in names and "ns_richardson_solve" in names and "ns_k_gemm_bf16" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/nsgb.h but not exported"


def test_struct_layout_matches_header(L):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "nsgb.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ns_options), offsetof(ns_options, ns_stop_frob),
         offsetof(ns_options, timeout_s), offsetof(ns_options, aux_ahead), sizeof(ns_stats));
  printf("%zu %zu %zu %zu\n", offsetof(ns_stats, frob_F), offsetof(ns_stats, rel_res_hist),
         offsetof(ns_stats, gemm_launches), offsetof(ns_stats, wall_ms));
  printf("%zu %zu %zu %zu\n", sizeof(ns_batch_stats), offsetof(ns_batch_stats, gemm_launches),
         offsetof(ns_batch_stats, wall_ms), offsetof(ns_batch_stats, gemm_bytes));
  printf("%zu %zu %zu %zu\n", sizeof(ns_request), offsetof(ns_request, tol), offsetof(ns_request, A),
         offsetof(ns_request, Theta));
  printf("%zu %zu %zu\n", sizeof(ns_result), offsetof(ns_result, rel_res), offsetof(ns_result, latency_ms));
  printf("%zu %zu %zu %zu\n", sizeof(ns_server_stats), offsetof(ns_server_stats, active),
         offsetof(ns_server_stats, last_error), offsetof(ns_server_stats, wait_ms));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    O, S = nsgb.ns_options, nsgb.ns_stats
    BS, Q, R, SS = nsgb.ns_batch_stats, nsgb.ns_request, nsgb.ns_result, nsgb.ns_server_stats
    want = [ctypes.sizeof(O), O.ns_stop_frob.offset, O.timeout_s.offset, O.aux_ahead.offset, ctypes.sizeof(S),
            S.frob_F.offset, S.rel_res_hist.offset, S.gemm_launches.offset, S.wall_ms.offset,
            ctypes.sizeof(BS), BS.gemm_launches.offset, BS.wall_ms.offset, BS.gemm_bytes.offset,
            ctypes.sizeof(Q), Q.tol.offset, Q.A.offset, Q.Theta.offset,
            ctypes.sizeof(R), R.rel_res.offset, R.latency_ms.offset,
            ctypes.sizeof(SS), SS.active.offset, SS.last_error.offset, SS.wait_ms.offset]
    assert got == want


def test_default_options(L):
    o = nsgb.default_options()
    assert o.precision == nsgb.NS_AUTO and o.form == 0 and o.pow_mode == 0 and o.g0_mode == 0
    assert o.ns_stop == 1 and o.ns_stop_frob == pytest.approx(0.02) and o.max_sweeps == 200
    assert o.timeout_s == pytest.approx(2.0) and o.aux_ahead == 0 and o.use_updated_G == 0


def test_status_strings(L):
    for name in ("NS_OK", "NS_NOT_CONVERGED", "NS_ERR_ARG", "NS_ERR_CUDA", "NS_ERR_OOM", "NS_ERR_DIVERGED",
                 "NS_ERR_TIMEOUT", "NS_ERR_NONFINITE", "NS_ERR_UNSUPPORTED"):
        assert nsgb.ns_status_string(getattr(nsgb, name)) == name


@pytest.mark.parametrize("n,order,rates", [(0, 4, ()), (-3, 2, ()), ((1 << 20) + 1, 4, ()), (16, 1, ()), (16, 5, ()),
                                           (16, 6, ()), (16, 4, (0,)), (16, 4, (5,))])
def test_create_rejects_bad_arguments(L, n, order, rates):
    opt = nsgb.default_options()
    arr = (ctypes.c_int * max(1, len(rates)))(*rates) if rates else None
    h = ctypes.c_void_p()
    s = L.ns_create(n, order, arr, len(rates), ctypes.byref(opt), ctypes.byref(h))
    assert s == nsgb.NS_ERR_ARG


@pytest.mark.parametrize("form,order", [(2, 1), (2, 20), (3, 44), (3, 9), (4, 4)])
def test_create_rejects_bad_form_orders(L, form, order):
    opt = nsgb.default_options(form=form)
    h = ctypes.c_void_p()
    assert L.ns_create(64, order, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG


def test_create_rejects_bad_g0_mode_and_accel(L):
    h = ctypes.c_void_p()
    opt = nsgb.default_options(g0_mode=3)
    assert L.ns_create(64, 4, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    opt = nsgb.default_options(accel_richardson=1, aux_ahead=1)
    arr = (ctypes.c_int * 1)(2)
    assert L.ns_create(64, 4, arr, 1, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    # the recursive schedule (2) has the same requirements; 3 is no schedule
    opt = nsgb.default_options(accel_richardson=2, aux_ahead=1)
    assert L.ns_create(64, 4, arr, 1, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    arr4 = (ctypes.c_int * 1)(4)
    for bad in (3, -1):
        opt = nsgb.default_options(accel_richardson=bad, aux_ahead=1)
        assert L.ns_create(64, 4, arr4, 1, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG


def test_create_rejects_bad_precision(L):
    opt = nsgb.default_options(precision=7)
    h = ctypes.c_void_p()
    assert L.ns_create(16, 4, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG


def test_create_validates_precision_options(L):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * 1)(2)
    for kw in ({"precision": 6}, {"precision": -1}, {"tf32_rung": 2}, {"fp64_slices": 1}, {"fp64_slices": 8}, {"fp64_slices": 9}, {"fp64_slices_early": 1},
               {"fp64_slices_early": 8}, {"fp64_slices_early": 9}, {"final_check": -3}, {"final_check": 4097}, {"pow_bf16": 3}, {"pow_bf16": -1},
               {"gemm_cluster": 2}, {"gemm_cluster": 4}, {"fp64_slices_pow": 1}, {"fp64_slices_pow": 8},
               {"fp64_slices_pow": -1}, {"xp_bf16x2": 3}, {"xp_bf16x2": -1}):
        opt = nsgb.default_options(**kw)
        assert L.ns_create(64, 4, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG, kw
    # bf16x6 needs the third split part, which composite loops and form 3 do not carry
    opt = nsgb.default_options(precision=nsgb.NS_BF16X6)
    assert L.ns_create(64, 4, arr, 1, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_UNSUPPORTED
    opt = nsgb.default_options(precision=nsgb.NS_BF16X6, form=3)
    assert L.ns_create(64, 45, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_UNSUPPORTED
    # TF32 products likewise (fixed, or as AUTO's rung)
    for kw in ({"precision": nsgb.NS_TF32}, {"tf32_rung": 1}):
        opt = nsgb.default_options(**kw)
        assert L.ns_create(64, 4, arr, 1, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_UNSUPPORTED, kw
        opt = nsgb.default_options(form=3, **kw)
        assert L.ns_create(64, 45, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_UNSUPPORTED, kw
    d = nsgb.default_options()
    assert d.fp64_slices == 0 and d.fp64_slices_early == 4 and d.final_check == 0 and d.pow_bf16 == 2
    assert d.tf32_rung == 0 and d.batch_fused == 1 and d.fp64_slices_pow == 0 and d.xp_bf16x2 == 0


def test_new_kernel_entry_points_validate_before_launch(L):
    vp = ctypes.c_void_p
    three = (vp * 3)(16, 16, 16)
    none3 = (vp * 3)(16, None, 16)
    # x6 products: null parts, K = 0, unaligned leading dimensions
    assert L.ns_k_gemm_bf16x6(64, 64, 64, none3, 64, three, 64, 1.0, None, 0, 0.0, 0.0, None, 0, None, 0, None,
                              None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16x6(64, 64, 0, three, 64, three, 64, 1.0, None, 0, 0.0, 0.0, None, 0, None, 0, None,
                              None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16x6(64, 64, 64, three, 60, three, 64, 1.0, None, 0, 0.0, 0.0, None, 0, None, 0, None,
                              None) == nsgb.NS_ERR_ARG
    assert L.ns_k_split3(16, 0, 4, 4, 4, 16, 16, None, 4, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_split3(16, 2, 4, 4, 4, 16, 16, 16, 4, None) == nsgb.NS_ERR_ARG
    # slice products: slice count outside 2..7, null output, short leading dimension,
    # an output aliasing an operand when K is taken in several blocks
    for sl in (1, 8, 9):
        assert L.ns_k_gemm_oz(8, 8, 8, 16, 8, 16, 8, 1.0, None, 0, 0.0, 0.0, 16, 8, sl, None, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_oz(8, 8, 8, 16, 8, 16, 8, 1.0, None, 0, 0.0, 0.0, None, 8, 7, None, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_oz(8, 8, 8, 16, 4, 16, 8, 1.0, None, 0, 0.0, 0.0, 16, 8, 7, None, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_oz(8, 8, 20000, 16, 20000, 32, 8, 1.0, None, 0, 0.0, 0.0, 16, 8, 7, None,
                          None) == nsgb.NS_ERR_ARG


def test_horner_form_accepts_any_order(L):
    opt = nsgb.default_options(form=1)
    h = ctypes.c_void_p()
    s = L.ns_create(16, 5, None, 0, ctypes.byref(opt), ctypes.byref(h))
    # without a GPU the context cannot bind a device; with one it is created
    assert s in (nsgb.NS_OK, nsgb.NS_ERR_CUDA)
    if s == nsgb.NS_OK:
        L.ns_destroy(h)


def test_kernel_entry_points_validate_before_launch(L):
    # wrong precision, non-positive sizes and unaligned leading dimensions are
    # rejected on the host
    assert L.ns_k_gemm_bf16(7, 64, 64, 64, 16, 16, 64, 16, 16, 64, 1.0, None, 0, 0.0, 0.0, None, 0, None, None, 0,
                            None, 0, 0, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 0, 64, 64, 16, 16, 64, 16, 16, 64, 1.0, None, 0, 0.0, 0.0, None, 0,
                            None, None, 0, None, 0, 0, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 64, 64, 64, 16, 16, 60, 16, 16, 64, 1.0, None, 0, 0.0, 0.0, None, 0,
                            None, None, 0, None, 0, 0, None) == nsgb.NS_ERR_ARG
    # groupings other than 0 (automatic), 1 (one CTA per tile) and -2 (CTA pairs) are
    # rejected: there are no multi-CTA clusters sharing loads
    for cm in (2, 3, 4):
        assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 256, 256, 64, 16, 16, 64, 16, 16, 256, 1.0, None, 0, 0.0, 0.0, None,
                                0, None, None, 0, None, 256, cm, None) == nsgb.NS_ERR_ARG
    # CTA pairs (cluster_m = -2) need 256-column tiles and an even number of 128-row tiles
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 256, 256, 64, 16, 16, 64, 16, 16, 256, 1.0, None, 0, 0.0, 0.0, None,
                            0, None, None, 0, None, 128, -2, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16X3, 300, 256, 64, 16, 16, 64, 16, 16, 256, 1.0, None, 0, 0.0, 0.0, None,
                            0, None, None, 0, None, 0, -2, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 256, 256, 64, 16, 16, 64, 16, 16, 256, 1.0, None, 0, 0.0, 0.0, None,
                            0, None, None, 0, None, 256, -4, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_resid(None, 4, None, None, None, 4, 1, None, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_update(16, 2, 4, 16, 16, 4, 1, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_split(16, 3, 4, 4, 4, 16, 16, 8, None) == nsgb.NS_ERR_ARG


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(nsgb, "_LIB", None)
    monkeypatch.setattr(nsgb, "lib_path", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        nsgb.lib()


def test_batch_and_server_validate_before_cuda(L):
    h = ctypes.c_void_p()
    opt = nsgb.default_options()
    n = (ctypes.c_int64 * 2)(16, 0)
    r = (ctypes.c_int * 2)(1, 1)
    assert L.ns_batch_create(2, n, r, 4, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    assert L.ns_batch_create(0, n, r, 4, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    # budget below 1 MiB, no slots, nrhs out of range
    assert L.ns_server_create(1 << 10, 8, 4, 4, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    assert L.ns_server_create(1 << 30, 0, 4, 4, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    assert L.ns_server_create(1 << 30, 8, 0, 4, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    # the batched path supports the factorized form, orders 3 and 2^m, bf16 precisions
    bad = nsgb.default_options(form=1)
    assert L.ns_server_create(1 << 30, 8, 4, 4, ctypes.byref(bad), ctypes.byref(h)) == nsgb.NS_ERR_UNSUPPORTED
    bad = nsgb.default_options(precision=nsgb.NS_FP64)
    assert L.ns_server_create(1 << 30, 8, 4, 4, ctypes.byref(bad), ctypes.byref(h)) == nsgb.NS_ERR_UNSUPPORTED
    assert L.ns_server_create(1 << 30, 8, 4, 6, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG
    # null handles
    t = ctypes.c_uint64()
    q = nsgb.ns_request(16, 1, 8, 1e-10, 1, 1, 1)
    assert L.ns_server_submit(None, ctypes.byref(q), ctypes.byref(t)) == nsgb.NS_ERR_ARG
    assert L.ns_server_tick(None, None) == nsgb.NS_ERR_ARG
    assert L.ns_server_destroy(None) == nsgb.NS_OK


def test_arena_first_fit_and_merge():
    """The server's workspace allocator: first fit, 256-byte granules, and
    freed neighbours merge back into one range."""
    gxx = shutil.which("g++") or shutil.which("c++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    src = r"""
#include <cstdio>
#include "arena.h"
int main() {
  nsgb::Arena a;
  a.init(4096);
  size_t x = a.alloc(100), y = a.alloc(256), z = a.alloc(1000), w = a.alloc(4096);
  std::printf("%zu %zu %zu %zu %zu\n", x, y, z, w == SIZE_MAX, a.free_bytes());
  a.release(y, 256);                      // hole of 256 between x and z
  size_t u = a.alloc(300);                // does not fit the hole: goes after z
  size_t v = a.alloc(200);                // first fit: the hole
  std::printf("%zu %zu %zu\n", u, v, a.free_.size());
  a.release(x, 100); a.release(v, 200); a.release(z, 1000); a.release(u, 300);
  std::printf("%zu %zu %zu\n", a.free_.size(), a.free_.begin()->first, a.free_.begin()->second);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "arena.cc")
        exe = os.path.join(d, "arena")
        open(c, "w").write(src)
        subprocess.run([gxx, "-std=c++17", "-I", os.path.join(ROOT, "paper_2008_11480_gb300", "csrc"), c, "-o", exe],
                       check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    assert [int(v) for v in lines[0].split()] == [0, 256, 512, 1, 4096 - 1536]
    assert [int(v) for v in lines[1].split()] == [1536, 256, 1]
    assert [int(v) for v in lines[2].split()] == [1, 0, 4096]
