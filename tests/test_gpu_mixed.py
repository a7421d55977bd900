"""Chosen form (mixed precision) against the oracle, error stated per quantity.

The V-G-V and V-G-P-V chains run with complex64 operands and FP32
accumulation; the W solve, Dyson, mu search and transforms stay FP64.  The
gate is 1e-5 relative max-norm on P0, P, Sigma~ and the energy (the bound the
chosen form is held to); the measured errors are printed.  Both builds of the
chains are checked: the tensor-core one (tcgen05, TF32 head/tail products,
the default) and the FP32 FMA one (selected with SGW_TC=0).
"""
import os

import numpy as np
import pytest

from oracle import gw
from tests.gpu_helpers import oracle_grid, rel_err, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", params=["tensor_core", "fp32_fma"])
def mixed_t1(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_09494_gb300 import api, configs, sgw

    cfg = configs.get("t1")
    if request.param == "fp32_fma":
        os.environ["SGW_TC"] = "0"
    try:
        sess = api.Session(cfg, precision=sgw.SGW_MIXED_FP32)
    finally:
        os.environ.pop("SGW_TC", None)
    s = sess.sys
    V = s.V_full()
    og = oracle_grid(cfg)
    mu0 = gw.mu_noninteracting(s.H0, s.S, cfg.beta, cfg.n_elec)
    G0 = gw.g0_tau(s.H0, s.S, mu0, cfg.beta, og["tau"])
    P0 = gw.polarization(G0, V, cfg.nk)
    P, _, _ = gw.screened_interaction(P0, og["TB"], og["TBbar"])
    Sig = gw.self_energy(G0, P, V, cfg.nk)
    Shf, _, _ = gw.hartree_fock(gw.density_matrix(G0), V, cfg.nk)
    G1, mu1 = gw.dyson(s.H0, s.S, Shf, Sig, mu0, og, cfg.n_elec, search_mu=True)
    E = gw.energy(s.H0, s.S, G1, Shf, Sig, cfg.beta)
    lG0, lmu0 = sess.g0()
    lP0 = sess.polarization(lG0)
    lP = sess.screened(lP0)
    lSig = sess.self_energy(lG0, lP)
    lShf = sess.hartree_fock(lG0)
    lG1, lmu1 = sess.dyson(lSig, lShf, lmu0, True)
    lE = sess.energy(lG1, lShf, lSig)
    kernels = set(sgw.sgw_profile_read(sess.ctx))
    out = dict(
        P0=rel_err(to_np(sess.unfold(1, lP0)), P0),
        P=rel_err(to_np(sess.unfold(1, lP)), P),
        Sigma=rel_err(to_np(sess.unfold(0, lSig)), Sig),
        HF=rel_err(to_np(sess.unfold(0, lShf))[:, 0], Shf),  # one matrix per k: drop the series axis
        G=rel_err(to_np(sess.unfold(0, lG1)), G1),
        mu=abs(lmu1 - mu1),
        E=abs(lE[0] - E[0].real) / max(1.0, abs(E[0])),
    )
    print(request.param, "chosen-form errors vs the FP64 oracle:", {k: f"{v:.2e}" for k, v in out.items()})
    sess.close()
    out["kernels"] = kernels
    out["impl"] = request.param
    return out


@pytest.mark.parametrize("q", ["P0", "P", "Sigma", "HF", "G", "E"])
def test_mixed_form_error_per_quantity(mixed_t1, q):
    assert mixed_t1[q] < TOL, (q, mixed_t1[q])


def test_mixed_form_is_not_the_plain_form(mixed_t1):
    # the FP32 chains leave a visible rounding signature: not bitwise the FP64 result
    assert mixed_t1["P0"] > 1e-12


def test_mixed_form_runs_the_selected_chains(mixed_t1):
    tc = {"p0_vg_tc", "p0_gvg_tc", "p0_gram_tc", "sigma_vg_tc", "sigma_pvg_tc", "sigma_gram_tc"}
    if mixed_t1["impl"] == "tensor_core":
        assert tc <= mixed_t1["kernels"], mixed_t1["kernels"]
    else:
        assert not (tc & mixed_t1["kernels"]) and "p0_gram_f32" in mixed_t1["kernels"]


def _chain_errors(cfg):
    from paper_2405_09494_gb300 import api, sgw

    sess = api.Session(cfg, precision=sgw.SGW_MIXED_FP32)
    s = sess.sys
    V = s.V_full()
    og = oracle_grid(cfg)
    mu0 = gw.mu_noninteracting(s.H0, s.S, cfg.beta, cfg.n_elec)
    G0 = gw.g0_tau(s.H0, s.S, mu0, cfg.beta, og["tau"])
    P0 = gw.polarization(G0, V, cfg.nk)
    P, _, _ = gw.screened_interaction(P0, og["TB"], og["TBbar"])
    Sig = gw.self_energy(G0, P, V, cfg.nk)
    lG0, _ = sess.g0()
    lP0 = sess.polarization(lG0)
    lP = sess.screened(lP0)
    lSig = sess.self_energy(lG0, lP)
    out = dict(P0=rel_err(to_np(sess.unfold(1, lP0)), P0), P=rel_err(to_np(sess.unfold(1, lP)), P),
               Sigma=rel_err(to_np(sess.unfold(0, lSig)), Sig))
    kernels = set(sgw.sgw_profile_read(sess.ctx))
    sess.close()
    return out, kernels


@pytest.mark.parametrize("case", ["one_block_160", "diamond_2", "nao_72"])
def test_mixed_chains_on_large_and_nonsymmorphic_blocks(case):
    """Auxiliary blocks above one 128-row tile (several M and N tiles per block), the
    non-symmorphic diamond group (odd block starts, fractional translations), and more than 64
    orbitals (two output-column tiles in the orbital multiplies and in the Sigma Gram, blocks
    that straddle them)."""
    import dataclasses

    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_09494_gb300 import configs

    base = configs.get("t1")
    if case == "one_block_160":
        cfg = dataclasses.replace(base, name="none-160", structure="none", nk=(1, 1, 2), ao_shells=(0,) * 8,
                                  aux_shells=(0,) * 160)
    elif case == "nao_72":
        cfg = dataclasses.replace(base, name="none-72", structure="none", nk=(1, 1, 2), ao_shells=(0,) * 72,
                                  aux_shells=(0,) * 40)
    else:
        cfg = dataclasses.replace(base, name="diamond-2", index=3, structure="diamond")
    errs, kernels = _chain_errors(cfg)
    print(case, {k: f"{v:.2e}" for k, v in errs.items()})
    assert "p0_gram_tc" in kernels and "sigma_pvg_tc" in kernels
    for q, e in errs.items():
        assert e < TOL, (case, q, e)
