"""The tau reflection of P0 (Algorithm 3 loops tau to n_tau/2; here without its time reversal).

From Eq. (P0) with antiperiodicity and the Hermitian pairing of V, P0^q(tau) = P0^{-q}(beta - tau)^T;
on the Chebyshev nodes beta - tau_j = tau_{n-1-j}.  The library contracts the first ceil(n_tau / 2)
tau values and fills the rest from that relation in block coordinates.  Checked here against the
same library with the reflection off (SGW_P0_REFLECT=0: every tau contracted): plain form 1e-12,
chosen form 1e-6 (its own rounding), on a cell without symmetry, the rocksalt and the
non-symmorphic diamond cells, and workload c2; and that the reflection kernel ran.  (The oracle
parity tests elsewhere compare the reflected tau values with the oracle's full contraction.)
"""
import dataclasses
import os

import pytest

from tests.gpu_helpers import rel_err, to_np

pytestmark = pytest.mark.gpu


def _cfg(name):
    from paper_2405_09494_gb300 import configs

    if name == "diamond-t1":
        return dataclasses.replace(configs.get("t1"), name="diamond-t1", index=3, structure="diamond")
    return configs.get(name)


@pytest.mark.parametrize("form", ["plain", "mixed"])
@pytest.mark.parametrize("name", ["c1", "t1", "diamond-t1", "c2"])
def test_reflected_p0_equals_the_full_contraction(name, form):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_09494_gb300 import api, sgw, synth

    cfg = _cfg(name)
    system = synth.System(cfg)
    prec = sgw.SGW_FP64 if form == "plain" else sgw.SGW_MIXED_FP32
    a = api.Session(cfg, precision=prec, system=system)
    G, _ = a.g0()
    P0a = to_np(a.polarization(G))
    ran = set(sgw.sgw_profile_read(a.ctx))
    a.close()
    os.environ["SGW_P0_REFLECT"] = "0"
    try:
        b = api.Session(cfg, precision=prec, system=system)
    finally:
        os.environ.pop("SGW_P0_REFLECT", None)
    Gb, _ = b.g0()
    P0b = to_np(b.polarization(Gb))
    ran_b = set(sgw.sgw_profile_read(b.ctx))
    b.close()
    assert "p0_reflect" in ran and "p0_reflect" not in ran_b, (ran, ran_b)
    err = rel_err(P0a, P0b)
    print(name, form, f"reflected vs full contraction {err:.1e}")
    assert err < (1e-12 if form == "plain" else 1e-6), err
