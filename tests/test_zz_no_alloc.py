"""The allocation-free entry point against the allocating one (GPU).

sgw_screened_interaction_noalloc serves callers that may not allocate device memory when
they call in (inside another component's CUDA-graph capture, or under a device-memory budget
fixed at start-up).  It must give the result of sgw_screened_interaction, call after call,
while its scratch lives in the library's fixed array.  This file is collected last so that a
failure here cannot hide the other GPU tests; it also passes on its own in a fresh process.
"""
import pytest

from tests.gpu_helpers import rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def session():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_09494_gb300 import api, configs

    sess = api.Session(configs.get("t1"))
    yield sess
    sess.close()


def test_noalloc_requires_the_launch_tables_first(session):
    from paper_2405_09494_gb300 import configs, sgw
    from paper_2405_09494_gb300 import api

    fresh = api.Session(configs.get("t1"), system=session.sys)
    G, _ = fresh.g0()
    P0 = fresh.polarization(G)
    with pytest.raises(sgw.SGWError) as e:
        sgw.sgw_screened_interaction_noalloc(fresh.ctx, P0, fresh.p_series())
    assert e.value.status == 8
    fresh.close()


def test_noalloc_matches_allocating_entry_point_twice(session):
    import torch

    from paper_2405_09494_gb300 import sgw

    G, _ = session.g0()
    P0 = session.polarization(G)
    ref = to_np(session.screened(P0))  # the allocating entry point (builds the launch tables)
    for _ in range(2):
        P = session.p_series()
        sgw.sgw_screened_interaction_noalloc(session.ctx, P0, P)
        torch.cuda.synchronize()
        assert rel_err(to_np(P), ref) < 1e-10
