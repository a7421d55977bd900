"""Pins of the oracle's tau grid and Matsubara transforms (Sec. 4.1 and Eq. (P02P)).

Every expected value here comes from mathematics that does not go through the
oracle's quadrature: exact integrals of polynomials (high-precision mpmath
quadrature), the closed form of the transform of an exponential, the constant
at Omega_0, and the identity of the least-squares round trip.
"""
import numpy as np
import pytest

from oracle import grid


def test_nodes_ascending_and_mirror_symmetric():
    beta, n = 7.0, 17
    t = grid.tau_nodes(beta, n)
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < beta
    np.testing.assert_allclose(t[::-1], beta - t, rtol=0, atol=1e-13)


def test_coefficients_reproduce_chebyshev_polynomials():
    n = 9
    x = -np.cos(np.pi * (np.arange(n) + 0.5) / n)
    C = grid.cheb_values_to_coeffs(n)
    for l in range(n):
        c = C @ np.cos(l * np.arccos(x))
        e = np.zeros(n)
        e[l] = 1.0
        np.testing.assert_allclose(c, e, atol=1e-13)


@pytest.mark.parametrize("stat", ["F", "B"])
def test_polynomials_transform_exactly(stat):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    beta, n = 2.5, 10
    idx = [-7, -3, -1, 0, 1, 2, 5, 40] if stat == "F" else [-6, -2, 0, 1, 3, 9, 50]
    T = grid.forward_map(idx, beta, n, stat)
    nu = grid.matsubara_nu(idx, beta, stat)
    tau = grid.tau_nodes(beta, n)
    for p in (0, 1, 4, n - 1):
        f = (tau / beta) ** p
        got = T @ f
        for m, v in enumerate(nu):
            ref = mp.quad(lambda t: (t / beta) ** p * mp.exp(1j * v * t), [0, beta])
            assert abs(got[m] - complex(ref)) < 1e-12 * beta, (p, m)


def test_constant_at_omega_zero_is_beta():
    beta, n = 37.0, 16
    T = grid.forward_map([0, 3], beta, n, "B")
    np.testing.assert_allclose(T @ np.ones(n), [beta, 0.0], atol=1e-12 * beta)


@pytest.mark.parametrize("stat", ["F", "B"])
def test_exponential_against_closed_form(stat):
    # int_0^beta e^{(i nu - a) tau} dtau = (1 + e^{-a beta})/(a - i nu) (fermions), (1 - e^{-a beta})/(a - i nu) (bosons)
    beta, n, a = 4.0, 40, 1.3
    idx = list(range(-6, 6)) + [25, -40]
    T = grid.forward_map(idx, beta, n, stat)
    nu = grid.matsubara_nu(idx, beta, stat)
    f = np.exp(-a * grid.tau_nodes(beta, n))
    zeta = 1.0 if stat == "F" else -1.0
    ref = (1.0 + zeta * np.exp(-a * beta)) / (a - 1j * nu)
    np.testing.assert_allclose(T @ f, ref, rtol=0, atol=1e-12)


def test_integration_by_parts_branch_matches_quadrature():
    from oracle.grid import _cheb_T, _gauss_legendre_panels, _ibp_integrals

    n, beta = 12, 7.0
    for stat, i in (("F", 200), ("B", 150), ("F", -201)):
        nu = grid.matsubara_nu([i], beta, stat)[0]
        a = 0.5 * nu * beta
        x, w = _gauss_legendre_panels(4000)
        quad = 0.5 * beta * (_cheb_T(n, x) @ (np.exp(1j * a * (1 + x)) * w))
        np.testing.assert_allclose(_ibp_integrals(a, n, stat, beta), quad, rtol=0, atol=1e-14)


def test_round_trip_is_identity(fine_grid):
    beta, n, ops = fine_grid
    np.testing.assert_allclose(ops["TFbar"] @ ops["TF"], np.eye(n), atol=1e-11)
    np.testing.assert_allclose(ops["TBbar"] @ ops["TB"], np.eye(n), atol=1e-11)
    assert np.linalg.cond(ops["TF"]) < 1e4 and np.linalg.cond(ops["TB"]) < 1e4


def test_value_at_beta_minus_exact_for_polynomials():
    beta, n = 3.0, 11
    tau = grid.tau_nodes(beta, n)
    r = grid.value_at_beta_minus(n)
    for p in range(n):
        assert abs(r @ (tau / beta) ** p - 1.0) < 1e-12


def test_workload_index_sets_are_well_conditioned():
    from paper_2405_09494_gb300 import configs

    for name in ("c1", "c2"):
        cfg = configs.get(name)
        TF = grid.forward_map(cfg.mats_f, cfg.beta, cfg.ntau, "F")
        TB = grid.forward_map(cfg.mats_b, cfg.beta, cfg.ntau, "B")
        assert len(cfg.mats_f) == cfg.ntau and len(cfg.mats_b) == cfg.ntau + 1
        assert np.linalg.cond(TF) < 1e3 and np.linalg.cond(TB) < 1e3
