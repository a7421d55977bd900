"""Full-size parity on workload c2 (rocksalt O_h, 3x3x3, nao 18, naux 100, 50 tau), bench launch setup.

The library runs exactly as bench.py runs it (default workspace, whole-wedge launches).  The
oracle cannot afford the whole zone at this size inside a test, so it computes sampled outputs
one by one: P0 at two q (all k, all tau), Sigma~ at every wedge point and one star member fed
the GPU's P, the W solve at every q fed the GPU's P0, and G0 everywhere (closed form).  Plain
form: 1e-10; chosen form 1e-5.  The chosen form runs once with the split-K unit its autotuner
picks and once with each candidate forced (SGW_TC_KCHUNK), since a fresh box may pick any of them.
"""
import os

import numpy as np
import pytest

from oracle import gw
from tests.gpu_helpers import oracle_grid, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_09494_gb300 import api, configs

    cfg = configs.get("c2")
    plain = api.Session(cfg)
    og = oracle_grid(cfg)
    s = plain.sys
    cache = {}

    def V(a, b):
        if (a, b) not in cache:
            cache[(a, b)] = s.V(a, b)
        return cache[(a, b)]

    mu0 = gw.mu_noninteracting(s.H0, s.S, cfg.beta, cfg.n_elec)
    G0 = gw.g0_tau(s.H0, s.S, mu0, cfg.beta, og["tau"])
    out = dict(cfg=cfg, plain=plain, og=og, V=V, mu0=mu0, G0=G0)
    yield out
    plain.close()


def _chain(sess):
    G, mu = sess.g0()
    P0 = sess.polarization(G)
    P = sess.screened(P0)
    Sig = sess.self_energy(G, P)
    return G, mu, P0, P, Sig


@pytest.mark.parametrize("form,unit,tol", [("plain", None, 1e-10), ("mixed", None, 1e-5), ("mixed", "64", 1e-5),
                                           ("mixed", "128", 1e-5), ("mixed", "256", 1e-5)])
def test_c2_full_size_sampled(c2, form, unit, tol):
    from paper_2405_09494_gb300 import api, sgw

    cfg, og, V = c2["cfg"], c2["og"], c2["V"]
    if form == "plain":
        sess, own = c2["plain"], False
        G, mu, P0, P, Sig = _chain(sess)
    else:
        # the split-K unit is fixed when the context builds its plans, on its first calls
        if unit is not None:
            os.environ["SGW_TC_KCHUNK"] = unit
        try:
            sess, own = api.Session(cfg, precision=sgw.SGW_MIXED_FP32, system=c2["plain"].sys), True
            G, mu, P0, P, Sig = _chain(sess)
        finally:
            os.environ.pop("SGW_TC_KCHUNK", None)
        assert {"p0_gram_tc", "sigma_gram_tc"} <= set(sgw.sgw_profile_read(sess.ctx))
    sgw.sgw_sync(sess.ctx)
    try:
        assert abs(mu - c2["mu0"]) < 1e-10
        assert rel_err(to_np(sess.unfold(0, G)), c2["G0"]) < 1e-10
        P0u = to_np(sess.unfold(1, P0))
        # P0 at one q in the wedge and one q outside it (star member), every k and tau
        for q in (sess.wedge[1], 5):
            ref = gw.polarization(c2["G0"], V, cfg.nk, qs=[int(q)])[int(q)]
            assert rel_err(P0u[q], ref) < tol, (form, unit, q)
        # the W solve at every q, fed the GPU's P0 (FP64 in both forms)
        Pref, _, _ = gw.screened_interaction(P0u, og["TB"], og["TBbar"])
        Pu = to_np(sess.unfold(1, P))
        assert rel_err(Pu, Pref) < 1e-10
        # Sigma at every wedge point and one star member, fed the GPU's P
        Sigu = to_np(sess.unfold(0, Sig))
        for k in list(sess.wedge) + [7]:
            ref = gw.self_energy(c2["G0"], Pu, V, cfg.nk, ks=[int(k)])[int(k)]
            assert rel_err(Sigu[k], ref) < tol, (form, unit, k)
        # invariants at full size: Hermiticity per tau of P0 and Sigma~ (both forms mirror the
        # upper triangles of Hermitian blocks, so only the unfolding's rounding remains)
        assert np.abs(P0u - P0u.conj().transpose(0, 1, 3, 2)).max() < 1e-12 * np.abs(P0u).max()
        assert np.abs(Sigu - Sigu.conj().transpose(0, 1, 3, 2)).max() < 1e-12 * np.abs(Sigu).max()
    finally:
        if own:
            sess.close()
