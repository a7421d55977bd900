"""Imaginary-time grid and Matsubara transforms of the oracle.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct CPU
reference of the symmetry-adapted finite-temperature GW step.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library never does.

What is computed (paper Sec. 4.1):

* the fermionic transform G(i w_n) = int_0^beta G(tau) exp(i w_n tau) dtau with
  w_n = (2n+1) pi / beta (Sec. 4.1, the Matsubara-transform equation that
  follows Eq. (scalar_S));
* the bosonic pair of Eq. (P02P): Omega_n = 2 n pi / beta, and the inverse
  P(tau) = (1/beta) sum_n P(i Omega_n) exp(-i Omega_n tau).

The paper evaluates these on an IR grid; here a Chebyshev representation is
used instead (reading of the paper: tau functions are represented
by their values at the n Chebyshev roots mapped to [0, beta]; a transform is
the exact Fourier integral of the interpolating polynomial; the inverse is the
least-squares inverse (pseudo-inverse) of the forward map on the chosen,
finite set of Matsubara indices).  The integrals
I_l(nu) = int_0^beta exp(i nu tau) T_l(2 tau / beta - 1) dtau are evaluated by
composite Gauss-Legendre quadrature, refined until two successive panel
counts agree to the rounding floor (adaptive in the panel count), or, at
frequencies far above the polynomial degree, by the exact finite
integration-by-parts sum.

Pins (tests/test_oracle_grid.py): exactness on polynomials of degree < n,
the constant function at Omega_0, the exponential against its analytic
transform, the round trip tau -> i nu -> tau.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tau_nodes",
    "cheb_values_to_coeffs",
    "matsubara_nu",
    "chebyshev_fourier_integrals",
    "forward_map",
    "backward_map",
    "value_at_beta_minus",
]


def tau_nodes(beta: float, n: int) -> np.ndarray:
    """Chebyshev roots x_j = -cos(pi (j + 1/2) / n), mapped to tau = beta (1 + x) / 2.

    Ascending, strictly inside (0, beta), and mirror symmetric:
    tau_{n-1-j} = beta - tau_j.
    """
    j = np.arange(n, dtype=np.float64)
    x = -np.cos(np.pi * (j + 0.5) / n)
    return 0.5 * beta * (1.0 + x)


def _cheb_T(lmax: int, x: np.ndarray) -> np.ndarray:
    """T_l(x) for l = 0..lmax-1 by the three-term recurrence; shape (lmax, len(x))."""
    x = np.asarray(x, dtype=np.float64)
    T = np.empty((lmax, x.size), dtype=np.float64)
    T[0] = 1.0
    if lmax > 1:
        T[1] = x
    for l in range(2, lmax):
        T[l] = 2.0 * x * T[l - 1] - T[l - 2]
    return T


def cheb_values_to_coeffs(n: int) -> np.ndarray:
    """Matrix C (n x n) with c_l = sum_j C[l, j] f(tau_j).

    Discrete Chebyshev orthogonality at the roots gives
    c_l = ((2 - delta_l0) / n) sum_j f(x_j) T_l(x_j); the interpolant is
    p(x) = sum_l c_l T_l(x).
    """
    j = np.arange(n, dtype=np.float64)
    x = -np.cos(np.pi * (j + 0.5) / n)
    T = _cheb_T(n, x)
    w = np.full(n, 2.0 / n)
    w[0] = 1.0 / n
    return w[:, None] * T


def matsubara_nu(indices, beta: float, statistics: str) -> np.ndarray:
    """nu = (2n+1) pi / beta (fermions) or 2 n pi / beta (bosons)."""
    idx = np.asarray(indices, dtype=np.float64)
    if statistics == "F":
        return (2.0 * idx + 1.0) * np.pi / beta
    if statistics == "B":
        return 2.0 * idx * np.pi / beta
    raise ValueError("statistics must be 'F' or 'B'")


def _gauss_legendre_panels(n_panels: int, order: int = 32):
    """Nodes and weights of composite Gauss-Legendre on [-1, 1]."""
    t, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(-1.0, 1.0, n_panels + 1)
    half = 0.5 * (edges[1:] - edges[:-1])
    mid = 0.5 * (edges[1:] + edges[:-1])
    x = (mid[:, None] + half[:, None] * t[None, :]).ravel()
    wx = (half[:, None] * w[None, :]).ravel()
    return x, wx


def _ibp_integrals(a: float, n: int, statistics: str, beta: float) -> np.ndarray:
    """Exact integration by parts for one Matsubara frequency, a = nu beta / 2.

    For a polynomial p of degree < n,
        int_{-1}^{1} e^{i a x} p(x) dx = sum_k (-1)^k [p^(k)(x) e^{i a x}]_{-1}^{1} / (i a)^(k+1),
    a finite sum.  With T_l^(k)(1) = prod_{j<k} (l^2 - j^2) / (2 j + 1),
    T_l^(k)(-1) = (-1)^(l+k) T_l^(k)(1) and e^{2 i a} = e^{i nu beta} = -1
    (fermions) or +1 (bosons), no oscillating phase is evaluated at all.  For
    |a| >= (n-1)^2 every term is smaller than the one before, so the sum is
    evaluated without cancellation.
    """
    zeta = -1.0 if statistics == "F" else 1.0
    out = np.zeros(n, dtype=np.complex128)
    ia = 1j * a
    for l in range(n):
        deriv = 1.0  # T_l^(k)(1)
        acc = 0.0 + 0.0j
        power = ia  # (i a)^(k+1)
        for k in range(l + 1):
            term = ((-1.0) ** k) * deriv * (zeta - (-1.0) ** (l + k)) / power
            acc += term
            deriv *= (l * l - k * k) / (2.0 * k + 1.0)
            power *= ia
        out[l] = 0.5 * beta * acc
    return out


def chebyshev_fourier_integrals(nu: np.ndarray, beta: float, n: int, statistics: str, tol: float = 1e-14) -> np.ndarray:
    """I[m, l] = int_0^beta exp(i nu_m tau) T_l(2 tau / beta - 1) dtau, l < n.

    With tau = beta (1 + x) / 2 the integral is
    (beta / 2) int_{-1}^{1} exp(i nu_m beta (1 + x) / 2) T_l(x) dx.
    High frequencies (|a| >= (n-1)^2, a = nu beta / 2) use the exact finite
    integration-by-parts sum.  Lower ones are integrated on a composite
    32-point Gauss-Legendre rule: the first rule already resolves the integrand
    (one panel per half oscillation of exp(i a x) T_l(x)); the panel count is
    then doubled until the result changes by less than tol * beta, the rounding
    floor of a sum over ~1e5 nodes.
    """
    nu = np.atleast_1d(np.asarray(nu, dtype=np.float64))
    out = np.empty((nu.size, n), dtype=np.complex128)
    for m, v in enumerate(nu):
        a = 0.5 * v * beta
        if abs(a) >= max(1.0, (n - 1.0) ** 2):
            out[m] = _ibp_integrals(a, n, statistics, beta)
            continue
        panels = max(2, int(np.ceil((abs(a) + n) / np.pi)) + 2)
        prev = None
        while True:
            x, wx = _gauss_legendre_panels(panels)
            # the node sum in blocks of 2^15 nodes keeps the n x nodes table small at high
            # frequencies (the same quadrature; only the order of the partial sums differs)
            acc = np.zeros(n, dtype=np.complex128)
            for c0 in range(0, x.size, 1 << 15):
                xs = x[c0:c0 + (1 << 15)]
                acc += _cheb_T(n, xs) @ (np.exp(1j * a * (1.0 + xs)) * wx[c0:c0 + (1 << 15)])
            cur = 0.5 * beta * acc
            if prev is not None and np.max(np.abs(cur - prev)) <= tol * beta:
                break
            prev = cur
            panels *= 2
            if panels > 1 << 22:
                raise RuntimeError("quadrature did not converge")
        out[m] = cur
    return out


def forward_map(indices, beta: float, n: int, statistics: str) -> np.ndarray:
    """T (n_w x n): F(i nu_m) = sum_j T[m, j] f(tau_j) for the interpolant of f."""
    nu = matsubara_nu(indices, beta, statistics)
    I = chebyshev_fourier_integrals(nu, beta, n, statistics)
    return I @ cheb_values_to_coeffs(n)


def backward_map(T: np.ndarray) -> np.ndarray:
    """T_bar = pinv(T): least-squares values at the tau nodes from Matsubara data."""
    return np.linalg.pinv(T, rcond=1e-14)


def value_at_beta_minus(n: int) -> np.ndarray:
    """Row vector r with f(beta^-) = r . f(tau_nodes) for the interpolant.

    At x = 1 every T_l equals 1, so f(beta^-) = sum_l c_l.
    """
    return cheb_values_to_coeffs(n).sum(axis=0)
