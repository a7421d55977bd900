"""Partition of the pair units of the contractions across ranks (multi-GPU plan).

The contractions of Eq. (P0) and Eq. (sigma) are sums over independent (k1, k2) pairs
(Sec. 5, Algorithms 3 and 4): each rank can own a contiguous range of the library's pair
list, compute the partial P0 (or Sigma~) of its pairs, and one sum over the ranks (an
all-reduce of the packed blocks) gives the full result; the W solve, Dyson and the mu search
then run on every rank.  This module plans the ranges from the block structure alone (host
data, no device), balancing the algorithmic flops of the block form per pair.

Pair order (the library's, see ``sgw_get_pairs``): orientation 0 lists (k, k + q_w) as
p = w N_k + k; orientation 1 lists (k_w, k2) as p = w N_k + k2.
"""
from __future__ import annotations

import numpy as np


def _kvec(nk, k):
    n1, n2, n3 = nk
    return (k // (n2 * n3), (k // n3) % n2, k % n3)


def _kidx(nk, v):
    n1, n2, n3 = nk
    return ((v[0] % n1) * n2 + (v[1] % n2)) * n3 + (v[2] % n3)


def pair_list(nk, wedge_k, orientation):
    """(k1, k2) of every pair in the library's order."""
    Nk = nk[0] * nk[1] * nk[2]
    out = []
    for w, kw in enumerate(wedge_k):
        a = _kvec(nk, kw)
        for k in range(Nk):
            b = _kvec(nk, k)
            if orientation == 0:
                out.append((k, _kidx(nk, (b[0] + a[0], b[1] + a[1], b[2] + a[2]))))
            else:
                out.append((kw, k))
    return out


def pair_weights(nk, rep, wedge_k, ao_blocks, aux_blocks, nao, naux, orientation):
    """Algorithmic flops per pair of the block form (8 per complex multiply-add, per tau).

    orientation 0 (P0):    naux nao (sum_I n_I^2 + sum_J n_J^2) + nao^2 sum_B n_B^2
    orientation 1 (Sigma): naux nao sum_J n_J^2 + nao^2 sum_B n_B^2 + naux nao sum_I n_I^2
    with I the blocks at k1, J at k2 and B at q (= k2 - k1, or k1 - k2 for orientation 1).
    """
    ao2 = [sum(b * b for b in bl) for bl in ao_blocks]
    ax2 = [sum(b * b for b in bl) for bl in aux_blocks]
    w = []
    for k1, k2 in pair_list(nk, wedge_k, orientation):
        a, b = _kvec(nk, k1), _kvec(nk, k2)
        if orientation == 0:
            q = _kidx(nk, (b[0] - a[0], b[1] - a[1], b[2] - a[2]))
        else:
            q = _kidx(nk, (a[0] - b[0], a[1] - b[1], a[2] - b[2]))
        w.append(8.0 * (naux * nao * (ao2[rep[k1]] + ao2[rep[k2]]) + nao * nao * ax2[rep[q]]))
    return np.asarray(w)


def partition(weights, nranks):
    """Contiguous ranges [begin, end) of the pair list, one per rank, splitting the cumulative
    weight at multiples of total / nranks (every pair in exactly one range)."""
    weights = np.asarray(weights, dtype=float)
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    cum = np.concatenate([[0.0], np.cumsum(weights)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, nranks):
        cuts.append(int(np.searchsorted(cum, total * r / nranks, side="left")))
    cuts.append(len(weights))
    cuts = np.maximum.accumulate(np.asarray(cuts))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(nranks)]
