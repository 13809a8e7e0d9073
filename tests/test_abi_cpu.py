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
    want = [ctypes.sizeof(O), O.ns_stop_frob.offset, O.timeout_s.offset, O.aux_ahead.offset, ctypes.sizeof(S),
            S.frob_F.offset, S.rel_res_hist.offset, S.gemm_launches.offset, S.wall_ms.offset]
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


@pytest.mark.parametrize("n,order,rates", [(0, 4, ()), (-3, 2, ()), (16, 1, ()), (16, 5, ()), (16, 6, ()),
                                           (16, 4, (0,)), (16, 4, (5,))])
def test_create_rejects_bad_arguments(L, n, order, rates):
    opt = nsgb.default_options()
    arr = (ctypes.c_int * max(1, len(rates)))(*rates) if rates else None
    h = ctypes.c_void_p()
    s = L.ns_create(n, order, arr, len(rates), ctypes.byref(opt), ctypes.byref(h))
    assert s == nsgb.NS_ERR_ARG


def test_create_rejects_bad_precision(L):
    opt = nsgb.default_options(precision=7)
    h = ctypes.c_void_p()
    assert L.ns_create(16, 4, None, 0, ctypes.byref(opt), ctypes.byref(h)) == nsgb.NS_ERR_ARG


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
    # cluster sizes other than 1, 2, 4, and clusters with narrow tiles, are rejected
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 64, 64, 64, 16, 16, 64, 16, 16, 64, 1.0, None, 0, 0.0, 0.0, None, 0,
                            None, None, 0, None, 256, 3, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_gemm_bf16(nsgb.NS_BF16, 64, 64, 64, 16, 16, 64, 16, 16, 64, 1.0, None, 0, 0.0, 0.0, None, 0,
                            None, None, 0, None, 128, 2, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_resid(None, 4, None, None, None, 4, 1, None, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_update(16, 2, 4, 16, 16, 4, 1, None) == nsgb.NS_ERR_ARG
    assert L.ns_k_split(16, 3, 4, 4, 4, 16, 16, 8, None) == nsgb.NS_ERR_ARG


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(nsgb, "_LIB", None)
    monkeypatch.setattr(nsgb, "lib_path", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        nsgb.lib()
