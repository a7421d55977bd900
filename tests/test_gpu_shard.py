"""The sharded path: partial P0 and Sigma~ over ranges of the pair list (Sec. 5.2, Algorithms 3-4).

Workload c2 (rocksalt O_h, 3x3x3 mesh, nao 18, naux 100, 50 tau).  The pair list of each
orientation is partitioned with ``shard.partition`` on the block-form flops per pair (the plan a
multi-GPU run uses).  On one GPU, the library computes the partial sum of every range
(sgw_polarization_pairs, sgw_self_energy_pairs); the partials must add up to one whole call
(plain form 1e-12; the chosen form to its own whole call within the FP32 sum-order change, and to
the plain form within 1e-5), an empty range must give zeros, and a bad range an argument error.
The partials are then all-reduced by two ``gloo`` ranks on the CPU (one process per rank, as the
ranks of a multi-GPU run would sum them) and the reduced result checked against the whole call.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2405_09494_gb300 import shard

pytestmark = pytest.mark.gpu


def _ranges(sess, cfg, nranks):
    from paper_2405_09494_gb300 import api, sgw

    lat, pos, rot, tra, aos, axs = api.structure_arrays(cfg)
    nw, rep, ao, ax = sgw.sgw_host_symmetry(cfg.nk, cfg.nao, cfg.naux, lat, pos, rot, tra, aos, axs)
    wedge = [int(k) for k in sess.wedge]
    out = []
    for o in (0, 1):
        # the planner's pair order is the library's
        assert shard.pair_list(cfg.nk, wedge, o) == list(zip(*[map(int, x) for x in sess.pairs[o]]))
        out.append(shard.partition(shard.pair_weights(cfg.nk, rep, wedge, ao, ax, cfg.nao, cfg.naux, o), nranks))
    return out


@pytest.fixture(scope="module")
def c2s():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_09494_gb300 import api, configs, sgw

    cfg = configs.get("c2")
    plain = api.Session(cfg)
    mixed = api.Session(cfg, precision=sgw.SGW_MIXED_FP32, system=plain.sys)
    G, _ = plain.g0()
    P = plain.screened(plain.polarization(G))
    yield dict(cfg=cfg, plain=plain, mixed=mixed, G=G, P=P, torch=torch, sgw=sgw)
    plain.close()
    mixed.close()


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("nranks", [2, 3])
def test_partial_sums_over_the_pair_ranges_add_up(c2s, nranks):
    cfg, G, P, sgw = c2s["cfg"], c2s["G"], c2s["P"], c2s["sgw"]
    whole = {}
    for form in ("plain", "mixed"):
        sess = c2s[form]
        r0, r1 = _ranges(sess, cfg, nranks)
        assert all(b > a for a, b in r0 + r1)
        P0 = sess.polarization(G)
        Sg = sess.self_energy(G, P)
        P0s = sum(sess.polarization(G, pairs=r) for r in r0)
        Sgs = sum(sess.self_energy(G, P, pairs=r) for r in r1)
        tol = 1e-12 if form == "plain" else 1e-6
        assert _rel(P0s, P0) < tol, (form, _rel(P0s, P0))
        assert _rel(Sgs, Sg) < tol, (form, _rel(Sgs, Sg))
        # one range alone is only part of the sum
        assert _rel(sess.polarization(G, pairs=r0[0]), P0) > 1e-3
        whole[form] = (P0s, Sgs)
    assert _rel(whole["mixed"][0], whole["plain"][0]) < 1e-5
    assert _rel(whole["mixed"][1], whole["plain"][1]) < 1e-5


def test_empty_and_invalid_ranges(c2s):
    sess, G, P, sgw = c2s["plain"], c2s["G"], c2s["P"], c2s["sgw"]
    npairs = int(sess.layout.npairs)
    assert float(sess.polarization(G, pairs=(5, 5)).abs().max()) == 0.0
    assert float(sess.self_energy(G, P, pairs=(npairs, npairs)).abs().max()) == 0.0
    for bad in ((-1, 3), (4, 2), (0, npairs + 1)):
        with pytest.raises(sgw.SGWError) as e:
            sess.polarization(G, pairs=bad)
        assert e.value.status == 1  # SGW_ERR_ARG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, in_path, out_path):
    # a CPU rank: loads the partial sums the library computed for its ranges and all-reduces them
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    z = np.load(in_path)
    out = []
    for name in ("P0", "Sig"):
        t = torch.from_numpy(np.ascontiguousarray(z[f"{name}{rank}"].view(np.float64)))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        out.append(t.numpy().view(np.complex128))
    if rank == 0:
        np.savez(out_path, P0=out[0], Sig=out[1])
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_ranks_reduce_the_library_partials(c2s):
    import multiprocessing as mp

    cfg, sess, G, P = c2s["cfg"], c2s["plain"], c2s["G"], c2s["P"]
    world = 2
    r0, r1 = _ranges(sess, cfg, world)
    parts = {}
    for r in range(world):
        parts[f"P0{r}"] = sess.polarization(G, pairs=r0[r]).cpu().numpy()
        parts[f"Sig{r}"] = sess.self_energy(G, P, pairs=r1[r]).cpu().numpy()
    P0 = sess.polarization(G).cpu().numpy()
    Sg = sess.self_energy(G, P).cpu().numpy()
    with tempfile.TemporaryDirectory() as d:
        in_path, out_path = os.path.join(d, "parts.npz"), os.path.join(d, "reduced.npz")
        np.savez(in_path, **parts)
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, in_path, out_path)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0, 0], codes
        got = np.load(out_path)
    assert np.abs(got["P0"] - P0).max() <= 1e-12 * np.abs(P0).max()
    assert np.abs(got["Sig"] - Sg).max() <= 1e-12 * np.abs(Sg).max()
