"""The allocation-free entry point against the allocating one (GPU).

sgw_screened_interaction_noalloc serves callers that may not allocate device memory when
they call in (inside another component's CUDA-graph capture, or under a device-memory budget
fixed at start-up).  It must give the result of sgw_screened_interaction, call after call,
while its scratch lives in the library's fixed array; a direct call must leave the device's free
memory unchanged, and the call must be capturable in a CUDA graph whose replays give that result.
Problems its fixed scratch cannot hold (2 nw_b p_elems above 4 Mi complex numbers, auxiliary
blocks above 90) are refused with an argument error and the output left unwritten.  This file is
collected last so that a failure here cannot hide the other GPU tests; it also passes on its own
in a fresh process.
"""
import dataclasses

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


def test_noalloc_leaves_device_memory_unchanged(session):
    import torch

    from paper_2405_09494_gb300 import sgw

    G, _ = session.g0()
    P0 = session.polarization(G)
    ref = to_np(session.screened(P0))
    P = session.p_series()
    sgw.sgw_screened_interaction_noalloc(session.ctx, P0, P)  # warm-up: every kernel of the path loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch0 = torch.cuda.memory_allocated()
    for _ in range(3):
        sgw.sgw_screened_interaction_noalloc(session.ctx, P0, P)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == torch0
    assert rel_err(to_np(P), ref) < 1e-10
    # its launches are counted, and timed with profiling on, like those of the allocating call
    sgw.sgw_profile_read(session.ctx, reset=True)
    sgw.sgw_profile_enable(session.ctx, True)
    try:
        sgw.sgw_screened_interaction_noalloc(session.ctx, P0, P)
        torch.cuda.synchronize()
        prof = sgw.sgw_profile_read(session.ctx, reset=True)
    finally:
        sgw.sgw_profile_enable(session.ctx, False)
    assert prof["ft"][2] == 2 and prof["w_solve"][2] == 1, prof
    assert prof["ft"][0] > 0 and prof["w_solve"][0] > 0 and prof["w_solve"][1] > 0, prof


def test_noalloc_is_captured_in_a_cuda_graph_and_replayed(session):
    import torch

    from paper_2405_09494_gb300 import sgw

    G, _ = session.g0()
    P0 = session.polarization(G)
    ref = to_np(session.screened(P0))
    ref_half = to_np(session.screened(0.5 * P0))
    P = session.p_series()
    sgw.sgw_screened_interaction_noalloc(session.ctx, P0, P)  # first call on this device before capture
    torch.cuda.synchronize()
    P.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sgw.sgw_screened_interaction_noalloc(session.ctx, P0, P, torch.cuda.current_stream())
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert rel_err(to_np(P), ref) < 1e-10
    # a replay reads the input buffer as it is then
    P0.mul_(0.5)
    graph.replay()
    torch.cuda.synchronize()
    assert rel_err(to_np(P), ref_half) < 1e-10
    del graph


def _uncovered(case):
    """A cell without symmetry (one auxiliary block per point) past one of the scratch limits."""
    from paper_2405_09494_gb300 import configs

    base = configs.get("t1")
    if case == "aux_block_100":  # 2 x 17 x 2 x 100^2 = 0.68 Mi complex numbers, block of 100
        return dataclasses.replace(base, name="none-8-100", structure="none", nk=(1, 1, 2), ao_shells=(0,) * 8,
                                   aux_shells=(0,) * 100, extra={"vscale": 0.3})
    c2 = configs.get("c2")  # 2 x 51 x 8 x 80^2 = 5.0 Mi complex numbers, blocks of 80
    return dataclasses.replace(base, name="none-8-80", structure="none", nk=(2, 2, 2), ao_shells=(0,) * 8,
                               aux_shells=(0,) * 80, ntau=c2.ntau, beta=c2.beta, mats_f=c2.mats_f,
                               mats_b=c2.mats_b, extra={"vscale": 0.3})


@pytest.mark.parametrize("case", ["aux_block_100", "scratch_above_64MiB"])
def test_noalloc_refuses_what_its_scratch_cannot_hold(session, case):
    import torch

    from paper_2405_09494_gb300 import api, sgw

    cfg = _uncovered(case)
    sess = api.Session(cfg)
    try:
        L = sess.layout
        over = 2 * len(cfg.mats_b) * int(L.p_elems) > (4 << 20)
        assert (L.max_aux_block > 90, over) == ((True, False) if case == "aux_block_100" else (False, True))
        G, _ = sess.g0()
        P0 = sess.polarization(G)
        sess.screened(P0)  # the launch tables
        P = sess.p_series()
        P.fill_(complex(7.0, -3.0))
        torch.cuda.synchronize()
        with pytest.raises(sgw.SGWError) as e:
            sgw.sgw_screened_interaction_noalloc(sess.ctx, P0, P)
        assert e.value.status == 1  # SGW_ERR_ARG
        torch.cuda.synchronize()
        assert bool((P == complex(7.0, -3.0)).all())
    finally:
        sess.close()
