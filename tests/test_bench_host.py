"""Host-side logic of the benchmark that needs no GPU: the per-launch DRAM
traffic recorded with an ncu capture is reported only while the kernel
sources hash to the values recorded with it."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record(tmp_path, files, nbytes, digest):
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "t.md").write_text(
        "# capture\n\ntraffic_bytes_per_launch: %d\nkernel_sources: %s\nkernel_sources_sha256: %s\n"
        % (nbytes, " ".join(files), digest))


def test_recorded_traffic_follows_the_sources(tmp_path, monkeypatch):
    (tmp_path / "k1.cu").write_text("kernel one\n")
    (tmp_path / "k2.cuh").write_text("kernel two\n")
    h = hashlib.sha256()
    for f in ("k1.cu", "k2.cuh"):
        h.update((tmp_path / f).read_bytes())
    _record(tmp_path, ["k1.cu", "k2.cuh"], 123456789, h.hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("t.md") == 123456789.0
    (tmp_path / "k2.cuh").write_text("kernel two, changed\n")
    assert bench.recorded_traffic("t.md") is None            # kernel changed since the capture
    assert bench.recorded_traffic("missing.md") is None      # no capture


def test_repository_record_is_well_formed():
    txt = open(os.path.join(ROOT, "profiles", "traffic_k_gemm_tc2_dense_n4096.md")).read()
    assert "traffic_bytes_per_launch:" in txt and "kernel_sources_sha256:" in txt
    for f in txt.split("kernel_sources:")[1].splitlines()[0].split():
        assert os.path.exists(os.path.join(ROOT, f)), f


def _reference_line(args):
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"] + args,
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_gram_line():
    """The default (Gram) workload's reference arm, on a small Gram system:
    the contract's keys, the workload's config, and an oracle sample whose
    extrapolation uses the plain method's product count on that system."""
    d = _reference_line(["--gram-n", "512", "--ref-rows", "64", "--steps", "2", "--warmup", "1"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["config"]["n"] == 512 and d["config"]["kappa"] == 1e6 and "Gram" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and "products" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_plain_fp64_model_counts():
    """The plain method's work on the Gram system from its exact iterates: the
    step count makes ||F_K||_F <= 0.02 and ||F_{K-1}||_F > 0.02 on the
    generator's spectrum, 2 m products per order-2^m step."""
    import numpy as np

    from workloads import gram_spectrum
    n = 2048
    k, prods, sweeps = bench.plain_fp64_model(n, order=8)
    lam = gram_spectrum(n, 1e-3, bench.GRAM_SEED)[0] ** 2
    a = 1.0 / np.sqrt(np.sum(lam * lam))
    frob = lambda j: np.sqrt(np.sum((1 - a * lam) ** (2 * 8 ** j)))  # noqa: E731
    assert frob(k) <= 0.02 < frob(k - 1)
    assert prods == 6 * k and sweeps >= 1


def test_reference_arm_line_follows_the_contract():
    """`bench.py --impl reference --workload dense` (the oracle on the host
    cores) prints one JSON line with the contract's keys; checked on a small
    system so that it runs in seconds without a GPU."""
    d = _reference_line(["--workload", "dense", "--n", "256", "--steps", "2", "--warmup", "1"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["higher_is_better"] is True
    assert d["config"]["workload"] and d["config"]["n"] == 256
    assert {"value", "unit", "cores", "kind", "sample"} <= set(d["cpu_baseline"]) and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs and prints the reference line."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64",
                          "--steps", "1", "--warmup", "0", "--gpus", "2"], capture_output=True, text=True,
                         timeout=120, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
