"""Host logic of bench.py (no GPU): the roofline a kernel class is reported against, the measured
peaks, the oracle's core count, which workloads get a whole oracle pass, and the reference arm
launched as two ranks."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp64_class_is_alu_bound(bench):
    from paper_2405_09494_gb300 import configs

    prof = {"sigma_pvg": (211.5, 257.1, 5), "p0_gram": (132.4, 125.9, 5), "gram_reduce": (1.0, 0.0, 20)}
    r = bench._roofline(prof, configs.get("c2"), 108, 5, 0.104)
    assert r["bound"] == "alu" and r["kernel"] == "sigma_pvg" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert r["frac"] == pytest.approx((257.1 / 211.5) / bench.FP64_PEAK_TFLOPS)


def test_tensor_class_is_tensor_bound_with_the_sustained_peak_in_long_steps(bench):
    from paper_2405_09494_gb300 import configs

    cfg = configs.get("c3")
    prof = {"sigma_pvg_tc": (427.6, 40240.2, 50), "w_solve": (5.0, 1.0, 50)}
    long_step = bench._roofline(prof, cfg, 512, 1, 1.77)
    short_step = bench._roofline(prof, cfg, 512, 1, 0.5)
    assert long_step["bound"] == short_step["bound"] == "tensor"
    _, bf16, bf16_sus, _ = bench.measured_peaks()
    assert long_step["peak"] == pytest.approx(bf16_sus * 1.1 / 2.25 / 3)
    assert short_step["peak"] == pytest.approx(bf16 * 1.1 / 2.25 / 3)
    assert long_step["frac"] >= short_step["frac"]
    # the minimum bytes of a chain launch: V once, complex64
    assert long_step["algorithmic_bytes_per_launch"] == pytest.approx(8.0 * 512 * 300 * 52 * 52)


def test_measured_peaks_are_read_from_the_file_or_fall_back(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, 1900.0, 1700.0, "of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0}))
    assert bench.measured_peaks() == (6000.0, 1800.0, 1600.0, "of measured")


def test_whole_oracle_pass_only_where_it_fits(bench):
    from paper_2405_09494_gb300 import configs

    assert bench.full_pass_fits(configs.get("c1")) and bench.full_pass_fits(configs.get("c2"))
    assert not any(bench.full_pass_fits(configs.get(n)) for n in ("c3", "c4", "c5"))


def test_oracle_core_count_follows_the_blas_thread_variables(bench, monkeypatch):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.delenv(var, raising=False)
    assert bench.blas_threads() == (os.cpu_count() or 1)
    monkeypatch.setenv("OMP_NUM_THREADS", "1")
    assert bench.blas_threads() == 1
    monkeypatch.setenv("OMP_NUM_THREADS", "6")
    monkeypatch.setenv("OPENBLAS_NUM_THREADS", "4")
    assert bench.blas_threads() == 4


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0(tmp_path):
    """`bench.py --impl reference` launched as two ranks (the driver's multi-GPU launch): rank 0
    times the oracle on workload c1 and prints the one JSON line; rank 1 exits 0 without work."""
    import socket
    import subprocess
    import sys

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--config", "c1", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["config"]["name"] == "c1"
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["cores"] == 2
