"""Failure detection and checkpoint/resume on the GPU, with every fault made on the host.

* A chemical potential out of reach (n_elec above the s nao electrons the basis holds) ends the
  mu search without meeting its tolerance: sgw_dyson and sgw_iterate return SGW_ERR_NOCONV.
* NaN injected into P0(tau) makes every pivot of the W solve fail its magnitude test: the next
  synchronising call returns SGW_ERR_SINGULAR, and the context is usable afterwards.
* An allocation failure injected through SGW_FAIL_ALLOC_ABOVE_MB returns SGW_ERR_OOM; the same
  call succeeds once the injection is lifted.
* Resuming the loop from a saved state reproduces an uninterrupted run bit for bit (plain form).
* A bounded wait of the tensor-core pipeline kernel that runs out: with the wait limit set to 0
  the first wait that is not already satisfied gives up (no copy is broken: the copies land, the
  kernel just stops waiting for them); the call then reports SGW_ERR_TIMEOUT at the next
  synchronisation, and the same context computes normally once the limit is restored.
"""
import dataclasses
import os

import numpy as np
import pytest

from tests.gpu_helpers import to_np

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def c1():
    _need_gpu()
    from paper_2405_09494_gb300 import api, configs

    sess = api.Session(configs.get("c1"))
    yield sess
    sess.close()


def test_unreachable_particle_number_is_no_convergence():
    torch = _need_gpu()
    from paper_2405_09494_gb300 import api, configs, sgw

    base = configs.get("c1")

    class Overfilled(type(base)):
        @property
        def n_elec(self) -> float:  # four electrons more than the basis can hold
            return float(self.spin * self.nao + 4)

    cfg = Overfilled(**{f.name: getattr(base, f.name) for f in dataclasses.fields(base)})
    sess = api.Session(cfg)
    try:
        G, _ = sess.g0()  # mu0 pinned at its bracket's end; G0 is still a valid start
        Sig = sess.g_series()
        Shf = sess.zeros(sess.layout.g_elems)
        with pytest.raises(sgw.SGWError) as e:
            sess.dyson(Sig, Shf, 0.0, True)
        assert e.value.status == 5, e.value  # SGW_ERR_NOCONV
        stream = torch.cuda.Stream()
        with pytest.raises(sgw.SGWError) as e:
            sgw.sgw_iterate(sess.ctx, 2, 0.5, 0.0, G, Sig, Shf, 0.0, stream)
        assert e.value.status == 5, e.value
        # the context still works: a fixed-mu Dyson call succeeds
        Gf, _ = sess.dyson(Sig, Shf, 0.1, False)
        sgw.sgw_sync(sess.ctx)
        assert torch.isfinite(torch.view_as_real(Gf)).all()
    finally:
        sess.close()


def test_nan_in_p0_is_reported_singular_and_context_recovers(c1):
    torch = _need_gpu()
    from paper_2405_09494_gb300 import sgw

    G, _ = c1.g0()
    P0 = c1.polarization(G)
    sgw.sgw_sync(c1.ctx)
    bad = P0.clone()
    bad[0, 0] = complex(float("nan"), 0.0)
    c1.screened(bad)
    with pytest.raises(sgw.SGWError) as e:
        sgw.sgw_sync(c1.ctx)
    assert e.value.status == 4, e.value  # SGW_ERR_SINGULAR
    P = c1.screened(P0)
    sgw.sgw_sync(c1.ctx)
    assert torch.isfinite(torch.view_as_real(P)).all()


def test_injected_allocation_failure_is_out_of_memory():
    _need_gpu()
    from paper_2405_09494_gb300 import api, configs, sgw

    sess = api.Session(configs.get("c1"))
    try:
        G, _ = sess.g0()
        os.environ["SGW_FAIL_ALLOC_ABOVE_MB"] = "0"
        try:
            with pytest.raises(sgw.SGWError) as e:
                sess.polarization(G)
            assert e.value.status == 3, e.value  # SGW_ERR_OOM
        finally:
            os.environ.pop("SGW_FAIL_ALLOC_ABOVE_MB", None)
        P0 = sess.polarization(G)
        sgw.sgw_sync(sess.ctx)
        assert float(P0.abs().max()) > 0
    finally:
        sess.close()


def test_resume_from_saved_state_is_bitwise(tmp_path):
    torch = _need_gpu()
    from paper_2405_09494_gb300 import api, configs, sgw

    cfg = configs.get("c1")

    def fresh():
        s = api.Session(cfg)
        G, mu = s.g0()
        return s, G, s.g_series(), s.zeros(s.layout.g_elems), mu

    # uninterrupted: two passes
    s1, G, Sig, Shf, mu = fresh()
    stream = torch.cuda.Stream()
    mu_a, _ = sgw.sgw_iterate(s1.ctx, 1, 0.5, 0.0, G, Sig, Shf, mu, stream)
    mu_a, _ = sgw.sgw_iterate(s1.ctx, 1, 0.5, 0.0, G, Sig, Shf, mu_a, stream)
    torch.cuda.synchronize()
    ref = (to_np(G), to_np(Sig), to_np(Shf), mu_a)
    # interrupted: one pass, save, a new context, load, one more pass
    s2, G, Sig, Shf, mu = fresh()
    mu_b, _ = sgw.sgw_iterate(s2.ctx, 1, 0.5, 0.0, G, Sig, Shf, mu, stream)
    torch.cuda.synchronize()
    path = str(tmp_path / "state.npz")
    s2.save_state(path, G, Sig, Shf, mu_b, iteration=1)
    s2.close()
    s3 = api.Session(cfg, system=s1.sys)
    G, Sig, Shf, mu_c, head = s3.load_state(path)
    assert head["iteration"] == 1
    mu_c, _ = sgw.sgw_iterate(s3.ctx, 1, 0.5, 0.0, G, Sig, Shf, mu_c, stream)
    torch.cuda.synchronize()
    out = (to_np(G), to_np(Sig), to_np(Shf), mu_c)
    for a, b in zip(ref[:3], out[:3]):
        assert np.array_equal(a, b)
    assert ref[3] == out[3]
    # a state of another workload is refused
    other = api.Session(dataclasses.replace(cfg, name="c1-other"), system=s1.sys)
    with pytest.raises(ValueError):
        other.load_state(path)
    for s in (s1, s3, other):
        s.close()


def test_pipeline_wait_over_its_limit_is_timeout_and_context_recovers():
    torch = _need_gpu()
    from paper_2405_09494_gb300 import api, configs, sgw

    cfg = configs.get("t1")
    sess = api.Session(cfg, precision=sgw.SGW_MIXED_FP32)
    try:
        G, mu = sess.g0()
        ref = sess.polarization(G)  # default limit: a normal call
        sgw.sgw_sync(sess.ctx)
        sgw.sgw_set_wait_limit(sess.ctx, 0)
        sess.polarization(G)
        with pytest.raises(sgw.SGWError) as e:
            sgw.sgw_sync(sess.ctx)
        assert e.value.status == 6, e.value  # SGW_ERR_TIMEOUT
        sgw.sgw_sync(sess.ctx)  # the status word was cleared by the report
        sgw.sgw_set_wait_limit(sess.ctx, 2_000_000_000)
        again = sess.polarization(G)
        sgw.sgw_sync(sess.ctx)
        torch.cuda.synchronize()
        assert torch.equal(again, ref)
    finally:
        sess.close()
