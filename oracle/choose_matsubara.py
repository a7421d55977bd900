"""Pick the finite Matsubara index sets used by the configurations.

TEST INFRASTRUCTURE (an offline script of the oracle): it calls only
``oracle.grid`` and prints integer index lists that are then written, as plain
input data, into the configuration table of the package.  Both the oracle and
the library build their own transform matrices from those integers.

Reading of the paper (Sec. 5.1 uses an IR grid, replaced here by a Chebyshev
representation): the frequency set must make the map from the n
Chebyshev-node values to the sampled Matsubara values well conditioned.  The
set is chosen greedily by volume.  A frequency pair (nu, -nu) contributes the
real rows Re I(nu) and Im I(nu) of the integral matrix (the complex rows of
nu and -nu are conjugate, so the complex matrix has the same singular values
as the stacked real one, times sqrt 2).  Each step adds the candidate pair
whose rows, projected off the span already chosen, have the largest Gram
determinant.  Fermionic sets have n/2 pairs (n_w = n); bosonic sets always hold
Omega_0 and n/2 pairs (n_w = n + 1 for even n, solved by least squares).

Usage:  python -m oracle.choose_matsubara 20:100 50:100 ...
"""
from __future__ import annotations

import sys

import numpy as np

from .grid import chebyshev_fourier_integrals, forward_map, matsubara_nu


def _candidates(n: int) -> np.ndarray:
    dense = np.arange(0, 3 * n + 1)
    tail = np.unique(np.round(np.geomspace(3 * n + 1, 2 * n * n + 10, 8 * n)).astype(np.int64))
    return np.unique(np.concatenate([dense, tail]))


def greedy_indices(n: int, beta: float, statistics: str) -> list[int]:
    cand = _candidates(n)
    nu = matsubara_nu(cand, beta, statistics)
    I = chebyshev_fourier_integrals(nu, beta, n, statistics)  # (ncand, n) complex
    basis = np.zeros((0, n))
    chosen: list[int] = []
    rows_needed = n
    rows = 0
    if statistics == "B":
        r0 = I[0].real
        basis = (r0 / np.linalg.norm(r0))[None, :]
        chosen.append(0)
        rows = 1
        rows_needed = n + 1
    used = np.zeros(cand.size, dtype=bool)
    used[0] = statistics == "B"
    while rows < rows_needed:
        best = (-1.0, -1, None)
        for c in range(cand.size):
            if used[c]:
                continue
            R = np.stack([I[c].real, I[c].imag])
            R = R - (R @ basis.T) @ basis
            g = R @ R.T
            det = g[0, 0] * g[1, 1] - g[0, 1] * g[1, 0]
            score = det if rows + 2 <= n else max(g[0, 0], g[1, 1])
            if score > best[0]:
                best = (score, c, R)
        _, c, R = best
        used[c] = True
        chosen.append(int(cand[c]))
        for r in R:
            r = r - (r @ basis.T) @ basis
            nr = np.linalg.norm(r)
            if nr > 1e-300 and basis.shape[0] < n:
                basis = np.vstack([basis, r / nr])
        rows += 2
    pos = sorted(set(chosen))
    if statistics == "F":
        return sorted([-p - 1 for p in pos] + pos)
    return sorted([-p for p in pos if p > 0] + pos)


def main(argv: list[str]) -> None:
    for spec in argv:
        n_s, b_s = spec.split(":")
        n, beta = int(n_s), float(b_s)
        out = {}
        for st in ("F", "B"):
            idx = greedy_indices(n, beta, st)
            T = forward_map(idx, beta, n, st)
            out[st] = (idx, float(np.linalg.cond(T)))
        print(f"n={n} beta={beta}")
        for st in ("F", "B"):
            idx, c = out[st]
            print(f"  {st} n_w={len(idx)} cond={c:.3e} indices={idx}")
        sys.stdout.flush()


if __name__ == "__main__":
    main(sys.argv[1:])
