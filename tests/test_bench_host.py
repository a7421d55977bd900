"""Host logic of bench.py (no GPU): which roofline bound a kernel class is reported against."""
import importlib.util
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
    r = bench._roofline(prof, "c2", configs.get("c2"), 108, 5, 0.104)
    assert r["bound"] == "alu" and r["kernel"] == "sigma_pvg" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert r["frac"] == pytest.approx((257.1 / 211.5) / bench.FP64_PEAK_TFLOPS)
    assert r["traffic"] == bench.DRAM_TRAFFIC_BYTES[("c2", "sigma_pvg")]


def test_tensor_class_below_balance_point_is_hbm_bound(bench):
    from paper_2405_09494_gb300 import configs

    cfg = configs.get("c2")
    # 51.4 GFLOP per launch over 2 x 108 x 50 x 100 x 18^2 x 8 bytes: about 18 flop per byte
    prof = {"sigma_pvg_tc": (1.18, 51.42, 1), "p0_gram_tc": (0.9, 25.2, 1)}
    r = bench._roofline(prof, "c2", cfg, 108, 1, 0.0097)
    nbytes = 2.0 * 108 * cfg.ntau * cfg.naux * cfg.nao ** 2 * 8
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(nbytes / 1.18e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.HBM_PEAK_GBS)
    assert r["flop_per_byte"] < bench.TF32_X3_PEAK_TFLOPS * 1e3 / bench.HBM_PEAK_GBS


def test_tensor_class_above_balance_point_uses_the_sustained_peak_in_long_steps(bench):
    from paper_2405_09494_gb300 import configs

    cfg = configs.get("c3")
    prof = {"sigma_pvg_tc": (427.6, 40240.2, 50)}
    long_step = bench._roofline(prof, "c3", cfg, 512, 1, 1.77)
    short_step = bench._roofline(prof, "c3", cfg, 512, 1, 0.5)
    assert long_step["bound"] == short_step["bound"] == "tensor"
    assert long_step["peak"] == pytest.approx(bench.TF32_X3_SUSTAINED_TFLOPS)
    assert short_step["peak"] == pytest.approx(bench.TF32_X3_PEAK_TFLOPS)
    assert long_step["frac"] > short_step["frac"]


def test_oracle_core_count_follows_the_blas_thread_variables(bench, monkeypatch):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.delenv(var, raising=False)
    assert bench.blas_threads() == (os.cpu_count() or 1)
    monkeypatch.setenv("OMP_NUM_THREADS", "1")
    assert bench.blas_threads() == 1
    monkeypatch.setenv("OMP_NUM_THREADS", "6")
    monkeypatch.setenv("OPENBLAS_NUM_THREADS", "4")
    assert bench.blas_threads() == 4
