"""Partition of the pair units across ranks, and the sum that recombines them (no GPU).

* ``partition`` covers the pair list with contiguous ranges, each pair exactly once, and no
  rank carries more than its share of the weight plus one pair.
* ``pair_list`` reproduces the pair order of both orientations, checked against the momentum
  relations of Eqs. (P0) and (sigma).
* ``pair_weights`` on the rocksalt O_h mesh (blocks from the library's host-only star
  analysis) sums to the flop count of the block form, which is far below the dense count.
* Two ``gloo`` ranks on the CPU each compute the oracle's P0 and Sigma~ over their own pairs;
  the all-reduced partials equal the single-process result.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

from oracle import gw
from paper_2405_09494_gb300 import shard


def test_partition_covers_and_balances():
    rng = np.random.default_rng(3)
    for n, nranks in [(1, 1), (5, 8), (64, 2), (729, 3), (1000, 7)]:
        w = rng.gamma(0.7, size=n) + 1e-3
        ranges = shard.partition(w, nranks)
        assert len(ranges) == nranks
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c and a <= b
        loads = [w[a:b].sum() for a, b in ranges]
        assert abs(sum(loads) - w.sum()) < 1e-9 * w.sum()
        assert max(loads) <= w.sum() / nranks + w.max() + 1e-9
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_pair_list_momentum_relations():
    nk = (3, 2, 2)
    Nk = 12
    wedge = [0, 3, 7]
    p0 = shard.pair_list(nk, wedge, 0)
    p1 = shard.pair_list(nk, wedge, 1)
    assert len(p0) == len(p1) == len(wedge) * Nk
    for w, kw in enumerate(wedge):
        for k in range(Nk):
            k1, k2 = p0[w * Nk + k]
            assert k1 == k and gw.ksub(nk, k2, k1) == kw  # (k, k + q_w)
            assert p1[w * Nk + k] == (kw, k)  # (k_w, k2)


def test_pair_weights_rocksalt_block_form():
    from paper_2405_09494_gb300 import build, configs, sgw, synth

    if not os.path.exists(sgw.LIB_PATH):
        try:
            build.build()
        except RuntimeError as e:
            pytest.skip(str(e))
    cfg = configs.get("c2")
    ops = synth.space_group(cfg.structure)
    rot = np.stack([R for R, _ in ops])
    tra = np.stack([v for _, v in ops])
    nw, rep, ao, ax = sgw.sgw_host_symmetry(cfg.nk, cfg.nao, cfg.naux, synth.FCC,
                                            synth.atom_positions(cfg.structure), rot, tra,
                                            list(cfg.ao_shells), list(cfg.aux_shells))
    Nk = len(rep)
    wedge = [int(np.flatnonzero(rep == w)[0]) for w in range(nw)]
    for o in (0, 1):
        wts = shard.pair_weights(cfg.nk, rep, wedge, ao, ax, cfg.nao, cfg.naux, o)
        assert wts.shape == (nw * Nk,) and np.all(wts > 0)
        dense = 8.0 * nw * Nk * (2 * cfg.naux * cfg.nao ** 3 + cfg.nao ** 2 * cfg.naux ** 2)
        assert wts.sum() < 0.5 * dense
        # every block-diagonal term is bounded by its dense counterpart
        assert wts.max() <= dense / (nw * Nk)
        ranges = shard.partition(wts, 4)
        loads = np.array([wts[a:b].sum() for a, b in ranges])
        assert loads.max() <= wts.sum() / 4 + wts.max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ranges, out_path, seed):
    import torch
    import torch.distributed as dist

    from tests.conftest import random_system

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nk, nao, naux, nt = (2, 2, 1), 4, 6, 5
    H, S, V = random_system(nk, nao, naux, seed)
    tau = np.linspace(0.0, 4.0, nt)
    G = gw.g0_tau(H, S, 0.0, 4.0, tau)
    Nk = 4
    wedge = list(range(Nk))  # no symmetry: the wedge is the whole mesh
    (a0, b0), (a1, b1) = ranges[0][rank], ranges[1][rank]
    own0 = set(shard.pair_list(nk, wedge, 0)[a0:b0])
    own1 = set(shard.pair_list(nk, wedge, 1)[a1:b1])
    P0 = gw.polarization(G, V, nk, pairs=own0)
    Sig = gw.self_energy(G, gw.polarization(G, V, nk), V, nk, pairs=own1)  # any P serves here
    out = []
    for X in (P0, Sig):
        t = torch.from_numpy(np.ascontiguousarray(X.view(np.float64)))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        out.append(t.numpy().view(np.complex128))
    if rank == 0:
        np.savez(out_path, P0=out[0], Sig=out[1])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_full_result():
    pytest.importorskip("torch")
    import multiprocessing as mp

    from tests.conftest import random_system

    nk, nao, naux, nt = (2, 2, 1), 4, 6, 5
    Nk, world, seed = 4, 2, 11
    rep = list(range(Nk))
    ao, ax = [[nao]] * Nk, [[naux]] * Nk
    ranges = [shard.partition(shard.pair_weights(nk, rep, rep, ao, ax, nao, naux, o), world) for o in (0, 1)]
    for r in ranges:
        assert r[0][1] - r[0][0] > 0 and r[1][1] - r[1][0] > 0  # both ranks own pairs
    with tempfile.TemporaryDirectory() as d:
        out_path = os.path.join(d, "reduced.npz")
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, ranges, out_path, seed)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=240)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0, 0], codes
        got = np.load(out_path)
        H, S, V = random_system(nk, nao, naux, seed)
        G = gw.g0_tau(H, S, 0.0, 4.0, np.linspace(0.0, 4.0, nt))
        P0 = gw.polarization(G, V, nk)
        Sig = gw.self_energy(G, P0, V, nk)
        assert np.abs(got["P0"] - P0).max() <= 1e-13 * np.abs(P0).max()
        assert np.abs(got["Sig"] - Sig).max() <= 1e-13 * np.abs(Sig).max()
        # each rank alone holds only part of the sum
        own0 = set(shard.pair_list(nk, rep, 0)[slice(*ranges[0][0])])
        part = gw.polarization(G, V, nk, pairs=own0)
        assert np.abs(part - P0).max() > 1e-3 * np.abs(P0).max()
