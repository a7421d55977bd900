"""Full-size parity on workload c2 (rocksalt O_h, 3x3x3, nao 18, naux 100, 50 tau), bench launch setup.

The library runs exactly as bench.py runs it (default workspace, whole-wedge launches).  The
oracle cannot afford the whole zone at this size inside a test, so it computes sampled outputs
one by one: P0 at one q (all k, all tau), Sigma~ at one wedge k fed the GPU's P, the W solve at
every q fed the GPU's P0, and G0 everywhere (closed form).  Plain form: 1e-10; chosen form 1e-5.
"""
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
    from paper_2405_09494_gb300 import api, configs, sgw

    cfg = configs.get("c2")
    plain = api.Session(cfg)
    mixed = api.Session(cfg, precision=sgw.SGW_MIXED_FP32, system=plain.sys)
    og = oracle_grid(cfg)
    s = plain.sys
    cache = {}

    def V(a, b):
        if (a, b) not in cache:
            cache[(a, b)] = s.V(a, b)
        return cache[(a, b)]

    mu0 = gw.mu_noninteracting(s.H0, s.S, cfg.beta, cfg.n_elec)
    G0 = gw.g0_tau(s.H0, s.S, mu0, cfg.beta, og["tau"])
    out = dict(cfg=cfg, plain=plain, mixed=mixed, og=og, V=V, mu0=mu0, G0=G0)
    yield out
    plain.close()
    mixed.close()


def _chain(sess):
    G, mu = sess.g0()
    P0 = sess.polarization(G)
    P = sess.screened(P0)
    Sig = sess.self_energy(G, P)
    return G, mu, P0, P, Sig


@pytest.mark.parametrize("form,tol", [("plain", 1e-10), ("mixed", 1e-5)])
def test_c2_full_size_sampled(c2, form, tol):
    cfg, og, V = c2["cfg"], c2["og"], c2["V"]
    sess = c2[form]
    G, mu, P0, P, Sig = _chain(sess)
    assert abs(mu - c2["mu0"]) < 1e-10
    assert rel_err(to_np(sess.unfold(0, G)), c2["G0"]) < 1e-10
    P0u = to_np(sess.unfold(1, P0))
    # P0 at one q in the wedge and one q outside it (star member), every k and tau
    for q in (sess.wedge[1], 5):
        ref = gw.polarization(c2["G0"], V, cfg.nk, qs=[int(q)])[int(q)]
        assert rel_err(P0u[q], ref) < tol, (form, q)
    # the W solve at every q, fed the GPU's P0 (FP64 in both forms)
    Pref, _, _ = gw.screened_interaction(P0u, og["TB"], og["TBbar"])
    Pu = to_np(sess.unfold(1, P))
    assert rel_err(Pu, Pref) < 1e-10
    # Sigma at one wedge point and one star member, fed the GPU's P
    Sigu = to_np(sess.unfold(0, Sig))
    for k in (sess.wedge[2], 7):
        ref = gw.self_energy(c2["G0"], Pu, V, cfg.nk, ks=[int(k)])[int(k)]
        assert rel_err(Sigu[k], ref) < tol, (form, k)
    # invariants at full size: Hermiticity per tau (to the form's own bound: the chosen form
    # accumulates the two orientations of each block in separate FP32 sums)
    herm = 1e-9 if form == "plain" else tol
    assert np.abs(P0u - P0u.conj().transpose(0, 1, 3, 2)).max() < herm * np.abs(P0u).max()
