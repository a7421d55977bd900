"""Helpers shared by the GPU parity tests: the oracle's view of a workload."""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import grid, gw


def rel_err(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def oracle_grid(cfg):
    TF = grid.forward_map(cfg.mats_f, cfg.beta, cfg.ntau, "F")
    TB = grid.forward_map(cfg.mats_b, cfg.beta, cfg.ntau, "B")
    return dict(TF=TF, TFbar=grid.backward_map(TF), TB=TB, TBbar=grid.backward_map(TB),
                nu_f=grid.matsubara_nu(cfg.mats_f, cfg.beta, "F"), tau=grid.tau_nodes(cfg.beta, cfg.ntau))


def with_grid(cfg, beta, ntau, name_suffix="-fine"):
    """Same system (same seed), another grid: greedy Matsubara sets from the oracle's offline search."""
    from oracle import choose_matsubara as cm

    return dataclasses.replace(cfg, name=cfg.name + name_suffix, beta=beta, ntau=ntau,
                               mats_f=cm.greedy_indices(ntau, beta, "F"), mats_b=cm.greedy_indices(ntau, beta, "B"))


def to_np(t):
    return t.detach().cpu().numpy()
