"""Shared pytest configuration: the ``gpu`` marker and small input builders."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def random_system(nk, nao, naux, seed, vscale=1.0, real=False):
    """Tiny random system (H0, S, V full array) for oracle pins, Hermitian-paired V."""
    rng = np.random.default_rng(seed)
    Nk = nk[0] * nk[1] * nk[2]

    def cg(*shape):
        z = rng.normal(size=shape)
        if not real:
            z = z + 1j * rng.normal(size=shape)
        return z.astype(np.complex128)

    H = cg(Nk, nao, nao)
    H = 0.5 * (H + H.conj().transpose(0, 2, 1))
    H /= np.max([np.linalg.norm(h, 2) for h in H])
    B = cg(Nk, nao, nao)
    A = B @ B.conj().transpose(0, 2, 1)
    S = np.eye(nao)[None] + 0.1 * A / np.max([np.linalg.norm(a, 2) for a in A])
    V = cg(Nk, Nk, naux, nao, nao) * (vscale / np.sqrt(naux))
    for k1 in range(Nk):
        for k2 in range(Nk):
            if k1 < k2:
                V[k2, k1] = V[k1, k2].conj().transpose(0, 2, 1)
            elif k1 == k2:
                V[k1, k1] = 0.5 * (V[k1, k1] + V[k1, k1].conj().transpose(0, 2, 1))
    return H, S, V


_GRID_CACHE = {}


def grid_ops(beta, n):
    """Oracle transform operators on a greedy Matsubara set (cached per (beta, n))."""
    key = (float(beta), int(n))
    if key not in _GRID_CACHE:
        from oracle import choose_matsubara as cm
        from oracle import grid

        fi = cm.greedy_indices(n, beta, "F")
        bi = cm.greedy_indices(n, beta, "B")
        TF = grid.forward_map(fi, beta, n, "F")
        TB = grid.forward_map(bi, beta, n, "B")
        _GRID_CACHE[key] = dict(
            mats_f=fi, mats_b=bi, TF=TF, TB=TB, TFbar=grid.backward_map(TF), TBbar=grid.backward_map(TB),
            nu_f=grid.matsubara_nu(fi, beta, "F"), nu_b=grid.matsubara_nu(bi, beta, "B"),
            tau=grid.tau_nodes(beta, n))
    return _GRID_CACHE[key]


@pytest.fixture(scope="session")
def fine_grid():
    """beta = 3 with 40 Chebyshev nodes: the interpolant of the test functions is exact to ~1e-13."""
    return 3.0, 40, grid_ops(3.0, 40)
