"""Tau chunking and the degenerate one-point mesh (GPU).

* Workload c2 with a small workspace (SGW_WORKSPACE_GB=0.4): the contractions run in many tau
  chunks with a ragged last one (FP64 path: 16 chunks of 3 and one of 2; tensor-core path: 12 of
  4 and one of 2).  P0 and Sigma~ must equal the single-chunk results of the default workspace:
  1e-12 in the plain form, 1e-6 in the chosen form (the split-K grouping of its FP32 partial
  tiles follows the chunking).
* The chosen form with its tau chunk forced (SGW_TC_NC = 1, 3, 7: one tau value per Gram tile row
  group, a ragged chunking, a prime one) against its autotuned default: 1e-6 (the tau chunk sets
  the Gram tiles and the split-K grouping, so only the FP32 summation order changes).
* A Gamma-only mesh (n_k = 1, no symmetry and rocksalt O_h): the whole chain against the oracle.
"""
import dataclasses
import os

import numpy as np
import pytest

from oracle import gw
from tests.gpu_helpers import oracle_grid, rel_err, to_np, with_grid

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _chain(sess):
    G, _ = sess.g0()
    P0 = sess.polarization(G)
    P = sess.screened(P0)
    Sig = sess.self_energy(G, P)
    return to_np(P0), to_np(Sig)


@pytest.mark.parametrize("form,tol", [("plain", 1e-12), ("mixed", 1e-6)])
def test_many_tau_chunks_equal_one_chunk(form, tol):
    _need_gpu()
    from paper_2405_09494_gb300 import api, configs, sgw, synth

    cfg = configs.get("c2")
    system = synth.System(cfg)
    prec = sgw.SGW_FP64 if form == "plain" else sgw.SGW_MIXED_FP32
    one = api.Session(cfg, precision=prec, system=system)
    ref = _chain(one)
    one.close()
    os.environ["SGW_WORKSPACE_GB"] = "0.4"
    try:
        many = api.Session(cfg, precision=prec, system=system)
        out = _chain(many)
        many.close()
    finally:
        os.environ.pop("SGW_WORKSPACE_GB", None)
    for a, b in zip(out, ref):
        assert rel_err(a, b) < tol, (form, rel_err(a, b))


@pytest.fixture(scope="module")
def c2_default_chain():
    _need_gpu()
    from paper_2405_09494_gb300 import api, configs, sgw, synth

    cfg = configs.get("c2")
    system = synth.System(cfg)
    sess = api.Session(cfg, precision=sgw.SGW_MIXED_FP32, system=system)
    ref = _chain(sess)
    sess.close()
    return cfg, system, ref


@pytest.mark.parametrize("nc", ["1", "3", "7"])
def test_forced_tau_chunks_of_the_chosen_form(c2_default_chain, nc):
    from paper_2405_09494_gb300 import api, sgw

    cfg, system, ref = c2_default_chain
    os.environ["SGW_TC_NC"] = nc
    try:
        sess = api.Session(cfg, precision=sgw.SGW_MIXED_FP32, system=system)
        out = _chain(sess)
        sess.close()
    finally:
        os.environ.pop("SGW_TC_NC", None)
    for a, b in zip(out, ref):
        assert rel_err(a, b) < 1e-6, (nc, rel_err(a, b))


@pytest.mark.parametrize("structure", ["none", "rocksalt"])
def test_gamma_only_mesh_matches_oracle(structure):
    _need_gpu()
    from paper_2405_09494_gb300 import api, configs

    if structure == "none":
        base = configs.get("c1")
        cfg = dataclasses.replace(base, name="gamma-none", nk=(1, 1, 1))
    else:
        base = configs.get("c2")
        cfg = dataclasses.replace(base, name="gamma-rocksalt", nk=(1, 1, 1), ao_shells=(0, 1), aux_shells=(0, 0, 1, 2))
        cfg = with_grid(cfg, 10.0, 16, "")
    sess = api.Session(cfg)
    try:
        s = sess.sys
        V = s.V_full()
        og = oracle_grid(cfg)
        mu0 = gw.mu_noninteracting(s.H0, s.S, cfg.beta, cfg.n_elec, cfg.spin)
        G0 = gw.g0_tau(s.H0, s.S, mu0, cfg.beta, og["tau"])
        P0 = gw.polarization(G0, V, cfg.nk, cfg.spin, cfg.loop_sign)
        P, _, _ = gw.screened_interaction(P0, og["TB"], og["TBbar"])
        Sig = gw.self_energy(G0, P, V, cfg.nk)
        Shf, _, _ = gw.hartree_fock(gw.density_matrix(G0), V, cfg.nk, cfg.spin)
        lG, lmu = sess.g0()
        lP0 = sess.polarization(lG)
        lP = sess.screened(lP0)
        lSig = sess.self_energy(lG, lP)
        lShf = sess.hartree_fock(lG)
        assert abs(lmu - mu0) < 1e-10
        assert rel_err(to_np(sess.unfold(0, lG)), G0) < 1e-10
        assert rel_err(to_np(sess.unfold(1, lP0)), P0) < 1e-10
        assert rel_err(to_np(sess.unfold(1, lP)), P) < 1e-10
        assert rel_err(to_np(sess.unfold(0, lSig)), Sig) < 1e-10
        assert rel_err(to_np(sess.unfold(0, lShf))[:, 0], Shf) < 1e-10
        assert np.isfinite(to_np(lSig)).all()
    finally:
        sess.close()
