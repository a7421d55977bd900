"""Pins of the oracle's GW step against closed forms, identities and special cases.

What fixes each oracle function (none of these re-types the function itself):

* g0_tau: the jump G(0+) + G(beta-) = -S^{-1}; particle number from the Fermi sum;
  Dyson with Sigma = 0 (Eq. (dyson)) on a fine grid.
* polarization (Eq. (P0)): the Lindhard closed form in Matsubara space built
  from the eigenvectors; Hermiticity; P0^{-q}(tau) = P0^q(beta - tau)^T;
  P0(i Omega_0) <= 0 with the physical loop sign.
* screened_interaction (Eq. (P02P)): the Neumann series at weak coupling;
  [P, P0] = 0 per frequency; Hermiticity in tau.
* self_energy (Eq. (sigma)): the trace identity
  sum_k Tr[Sigma^(2)k(tau) G^k(-tau)] = -(1/s) sum_q sum_QQ' P0^q_QQ'(tau) P0^{-q}_QQ'(tau)
  that ties its index structure to the pinned P0; Hermiticity; real inputs at
  n_k = 1 give real results (Sec. 5.1).
* hartree_fock (Eq. (sigma_hf)): the explicit four-index U = sum_Q V V route (Eq. (U_decompose)).
* dyson / mu search / energy: reduce to the closed-form non-interacting values.

The planted-mistake tests at the end show that plausible slips fail these pins.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import grid, gw
from tests.conftest import random_system

NK = (2, 2, 2)
S_SPIN = 2


def _fermi(x, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * x))


@pytest.fixture(scope="module")
def small(fine_grid):
    beta, n, ops = fine_grid
    H, S, V = random_system(NK, 3, 5, seed=11)
    mu = gw.mu_noninteracting(H, S, beta, 3.0)
    G = gw.g0_tau(H, S, mu, beta, ops["tau"])
    return dict(beta=beta, n=n, ops=ops, H=H, S=S, V=V, mu=mu, G=G)


# ---------------------------------------------------------------- G0, mu, Dyson
def test_g0_jump_condition(small):
    n = small["n"]
    C = grid.cheb_values_to_coeffs(n)
    sgn = (-1.0) ** np.arange(n)
    c = np.einsum("lt,ktij->klij", C, small["G"])
    g0p = np.einsum("l,klij->kij", sgn, c)  # x = -1
    gbm = c.sum(axis=1)  # x = +1
    for k in range(small["H"].shape[0]):
        np.testing.assert_allclose(g0p[k] + gbm[k], -np.linalg.inv(small["S"][k]), atol=1e-12)


def test_g0_particle_number_matches_fermi_sum(small):
    H, S, beta, mu = small["H"], small["S"], small["beta"], small["mu"]
    eps = np.concatenate([scipy.linalg.eigh(H[k], S[k], eigvals_only=True) for k in range(H.shape[0])])
    n_ref = S_SPIN / H.shape[0] * _fermi(eps - mu, beta).sum()
    assert abs(n_ref - 3.0) < 1e-10
    gam = gw.density_matrix(small["G"])
    assert abs(gw.particle_number(gam, S) - n_ref) < 1e-10


def test_dyson_without_self_energy_is_g0(small):
    H, S, ops = small["H"], small["S"], small["ops"]
    Nk, n = H.shape[0], small["n"]
    zero_t = np.zeros((Nk, n, 3, 3), complex)
    G, mu = gw.dyson(H, S, np.zeros((Nk, 3, 3), complex), zero_t, small["mu"], ops)
    np.testing.assert_allclose(G, small["G"], atol=1e-10)
    _, mu_s = gw.dyson(H, S, np.zeros((Nk, 3, 3), complex), zero_t, 0.0, ops, n_elec=3.0, search_mu=True)
    assert abs(mu_s - small["mu"]) < 1e-8


def _interacting_sigma(small, scale=0.05, seed=5):
    """A Hermitian, tau-even self-energy pair (Sigma_HF, Sigma~(tau)) to make the Dyson step non-trivial."""
    rng = np.random.default_rng(seed)
    Nk, n = small["H"].shape[0], small["n"]
    X = rng.normal(size=(Nk, 3, 3)) + 1j * rng.normal(size=(Nk, 3, 3))
    Shf = scale * (X + X.conj().transpose(0, 2, 1))
    Y = rng.normal(size=(Nk, 1, 3, 3)) + 1j * rng.normal(size=(Nk, 1, 3, 3))
    Y = Y + Y.conj().transpose(0, 1, 3, 2)
    tau = small["ops"]["tau"]
    shape = np.exp(-3.0 * tau / small["beta"]) + np.exp(-3.0 * (small["beta"] - tau) / small["beta"])
    return Shf, -scale * shape[None, :, None, None] * Y


def test_particle_number_slope_is_the_derivative(small):
    H, S, ops = small["H"], small["S"], small["ops"]
    Shf, Sig = _interacting_sigma(small)
    for mu in (-0.3, 0.1, 0.4):
        n, dn = gw.particle_number_and_slope(H, S, Shf, Sig, mu, ops)
        h = 1e-5
        fd = (gw.particle_number_and_slope(H, S, Shf, Sig, mu + h, ops)[0]
              - gw.particle_number_and_slope(H, S, Shf, Sig, mu - h, ops)[0]) / (2 * h)
        assert dn > 0
        assert abs(dn - fd) < 1e-6 * max(1.0, abs(fd)), (mu, dn, fd)


def test_mu_search_finds_the_root_from_any_start(small):
    H, S, ops = small["H"], small["S"], small["ops"]
    Shf, Sig = _interacting_sigma(small)
    # brute force: plain bisection on N(mu) to a width of 1e-14
    lo, hi = -20.0, 20.0
    while hi - lo > 1e-14:
        mid = 0.5 * (lo + hi)
        if gw.particle_number_and_slope(H, S, Shf, Sig, mid, ops)[0] > 3.0:
            hi = mid
        else:
            lo = mid
    root = 0.5 * (lo + hi)
    slope = gw.particle_number_and_slope(H, S, Shf, Sig, root, ops)[1]
    for start in (0.0, root + 0.3, -19.0, 25.0):
        _, mu = gw.dyson(H, S, Shf, Sig, start, ops, n_elec=3.0, search_mu=True)
        n = gw.particle_number_and_slope(H, S, Shf, Sig, mu, ops)[0]
        assert abs(n - 3.0) <= 1e-11
        assert abs(mu - root) <= 2e-11 / slope + 1e-13


def test_energy_without_interaction_is_band_energy(small):
    H, S, beta, mu = small["H"], small["S"], small["beta"], small["mu"]
    Nk, n = H.shape[0], small["n"]
    eps = np.concatenate([scipy.linalg.eigh(H[k], S[k], eigvals_only=True) for k in range(Nk)])
    e_ref = S_SPIN / Nk * np.sum(_fermi(eps - mu, beta) * eps)
    zero = np.zeros((Nk, 3, 3), complex)
    E = gw.energy(H, S, small["G"], zero, np.zeros((Nk, n, 3, 3), complex), beta)
    assert abs(E[0] - e_ref) < 1e-10


# ---------------------------------------------------------------- P0
def test_polarization_matches_lindhard(small):
    H, S, V, beta, mu, ops = small["H"], small["S"], small["V"], small["beta"], small["mu"], small["ops"]
    Nk = H.shape[0]
    P0 = gw.polarization(small["G"], V, NK)
    P0w = gw.to_matsubara(P0, ops["TB"])
    eig = [scipy.linalg.eigh(H[k], S[k]) for k in range(Nk)]
    nu = ops["nu_b"]
    for q in range(Nk):
        ref = np.zeros((nu.size, 5, 5), complex)
        for k in range(Nk):
            kq = gw.kadd(NK, k, q)
            ec, Cc = eig[k]
            ea, Ca = eig[kq]
            M = np.einsum("dc,Qde,ea->Qca", Cc.conj(), V[k, kq], Ca)  # C^{k dagger} V^{k,k+q} C^{k+q}
            fc, fa = _fermi(ec - mu, beta), _fermi(ea - mu, beta)
            for m, W in enumerate(nu):
                num = fc[:, None] - fa[None, :]
                den = 1j * W + ec[:, None] - ea[None, :]
                deg = np.abs(den) < 1e-12
                w = np.where(deg, -beta * fc[:, None] * (1 - fc[:, None]), num / np.where(deg, 1.0, den))
                ref[m] += np.einsum("Qca,Rca,ca->QR", M, M.conj(), w)
        ref *= S_SPIN / Nk
        np.testing.assert_allclose(P0w[q], ref, atol=1e-10)


def test_polarization_hermitian_reflection_and_sign(small):
    P0 = gw.polarization(small["G"], small["V"], NK)
    np.testing.assert_allclose(P0, P0.conj().transpose(0, 1, 3, 2), atol=1e-14)
    n = small["n"]
    for q in range(P0.shape[0]):
        mq = gw.ksub(NK, 0, q)
        np.testing.assert_allclose(P0[mq], P0[q][::-1].transpose(0, 2, 1), atol=1e-14)
    P0w = gw.to_matsubara(P0, small["ops"]["TB"])
    i0 = small["ops"]["mats_b"].index(0)
    for q in range(P0.shape[0]):
        assert np.linalg.eigvalsh(P0w[q, i0]).max() < 1e-12


# ---------------------------------------------------------------- P (W solve)
def test_screened_interaction_neumann_series(small):
    ops = small["ops"]
    P0 = gw.polarization(small["G"], small["V"] * 0.05, NK)
    P, P0w, Pw = gw.screened_interaction(P0, ops["TB"], ops["TBbar"])
    ref = np.zeros_like(P0w)
    term = np.broadcast_to(np.eye(5), P0w.shape).copy()
    for _ in range(14):
        term = term @ P0w
        ref += term
    np.testing.assert_allclose(Pw, ref, atol=1e-15, rtol=1e-12)
    np.testing.assert_allclose(Pw @ P0w, P0w @ Pw, atol=1e-15)
    np.testing.assert_allclose(P, P.conj().transpose(0, 1, 3, 2), atol=1e-12)


# ---------------------------------------------------------------- Sigma
def _trace_identity_residual(G, P0, Sig):
    Gm = gw.g_minus_tau(G)
    lhs = np.einsum("ktij,ktji->t", Sig, Gm)
    rhs = np.zeros_like(lhs)
    for q in range(P0.shape[0]):
        rhs += np.einsum("tQR,tQR->t", P0[q], P0[gw.ksub(NK, 0, q)])
    rhs *= -1.0 / S_SPIN
    return np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))


def test_self_energy_trace_identity_with_bare_bubble(small):
    P0 = gw.polarization(small["G"], small["V"], NK)
    Sig = gw.self_energy(small["G"], P0, small["V"], NK)
    assert _trace_identity_residual(small["G"], P0, Sig) < 1e-13
    np.testing.assert_allclose(Sig, Sig.conj().transpose(0, 1, 3, 2), atol=1e-13)


def test_real_inputs_at_gamma_only_give_real_results(fine_grid):
    beta, n, ops = fine_grid
    H, S, V = random_system((1, 1, 1), 4, 6, seed=5, real=True)
    mu = gw.mu_noninteracting(H, S, beta, 4.0)
    G = gw.g0_tau(H, S, mu, beta, ops["tau"])
    P0 = gw.polarization(G, V, (1, 1, 1))
    P, _, _ = gw.screened_interaction(P0, ops["TB"], ops["TBbar"])
    Sig = gw.self_energy(G, P, V, (1, 1, 1))
    assert np.abs(G.imag).max() < 1e-14 and np.abs(P0.imag).max() < 1e-14
    assert np.abs(P.imag).max() < 1e-11 and np.abs(Sig.imag).max() < 1e-11


# ---------------------------------------------------------------- HF
def test_hartree_fock_against_four_index_interaction():
    nk = (1, 1, 2)
    H, S, V = random_system(nk, 2, 3, seed=3)
    rng = np.random.default_rng(4)
    gam = rng.normal(size=(2, 2, 2)) + 1j * rng.normal(size=(2, 2, 2))
    gam = gam + gam.conj().transpose(0, 2, 1)
    # U^{k1 k2 k3 k4}_{ijkl} = sum_Q V^{k1k2}_ij(Q) V^{k3k4}_kl(Q)
    U = np.einsum("abQij,cdQkl->abcdijkl", V, V)
    J = np.zeros((2, 2, 2), complex)
    K = np.zeros((2, 2, 2), complex)
    for k in range(2):
        for kp in range(2):
            J[k] += S_SPIN / 2 * np.einsum("ijba,ab->ij", U[k, k, kp, kp], gam[kp])
            K[k] -= 1 / 2 * np.einsum("iabj,ab->ij", U[k, kp, kp, k], gam[kp])
    _, Jo, Ko = gw.hartree_fock(gam, V, nk)
    np.testing.assert_allclose(Jo, J, atol=1e-13)
    np.testing.assert_allclose(Ko, K, atol=1e-13)


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistakes_fail_the_pins(small):
    """Each pin above rejects a plausible slip planted into a copy of the oracle's inputs/calls."""
    ops = small["ops"]
    V = small["V"]
    # (1) k1/k2 of V swapped inside the bubble -> Lindhard fails
    bad = gw.polarization(small["G"], lambda a, b: V[b, a], NK)
    good = gw.polarization(small["G"], V, NK)
    assert np.abs(gw.to_matsubara(bad, ops["TB"]) - gw.to_matsubara(good, ops["TB"])).max() > 1e-3
    # (2) literal (unphysical) loop sign -> P0(i Omega_0) is no longer <= 0
    lit = gw.polarization(small["G"], V, NK, loop_sign=-1)
    i0 = ops["mats_b"].index(0)
    assert max(np.linalg.eigvalsh(gw.to_matsubara(lit, ops["TB"])[q, i0]).max() for q in range(8)) > 1e-3
    # (3) P attached with Q and Q' exchanged in Sigma -> the trace identity fails
    Sig_bad = gw.self_energy(small["G"], good.transpose(0, 1, 3, 2), V, NK)
    assert _trace_identity_residual(small["G"], good, Sig_bad) > 1e-3
    # (4) orbital indices of V transposed in Sigma -> the trace identity fails
    Sig_bad2 = gw.self_energy(small["G"], good, lambda a, b: V[a, b].transpose(0, 2, 1), NK)
    assert _trace_identity_residual(small["G"], good, Sig_bad2) > 1e-3
    # (5) dG/dmu taken as -G G (the overlap dropped) -> the slope is no longer the derivative
    H, S = small["H"], small["S"]
    Shf, Sig = _interacting_sigma(small)
    Sw = gw.to_matsubara(Sig, ops["TF"])
    wgt = -(grid.value_at_beta_minus(ops["TF"].shape[1]) @ ops["TFbar"])
    Gw = gw.dyson_matsubara(H, S, Shf, Sw, 0.1, ops["nu_f"])
    slip = gw.particle_number(-np.einsum("m,kmij,kmjl->kil", wgt, Gw, Gw), S)
    h = 1e-5
    fd = (gw.particle_number_and_slope(H, S, Shf, Sig, 0.1 + h, ops)[0]
          - gw.particle_number_and_slope(H, S, Shf, Sig, 0.1 - h, ops)[0]) / (2 * h)
    assert abs(slip - fd) > 1e-3 * abs(fd)
