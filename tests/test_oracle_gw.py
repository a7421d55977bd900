"""Pins of the oracle's GW step against closed forms, identities and special cases.

What fixes each oracle function (none of these re-types the function itself):

* g0_tau: the jump G(0+) + G(beta-) = -S^{-1}; particle number from the Fermi sum;
  Dyson with Sigma = 0 (Eq. (dyson)) on a fine grid.
* polarization (Eq. (P0)): the Lindhard closed form in Matsubara space built
  from the eigenvectors; Hermiticity; P0^{-q}(tau) = P0^q(beta - tau)^T;
  P0(i Omega_0) <= 0 with the physical loop sign.
* screened_interaction (Eq. (P02P)): the Neumann series at weak coupling;
  [P, P0] = 0 per frequency; Hermiticity in tau; the values at -Omega_n are the adjoints of those
  at Omega_n on a closed frequency set.
* self_energy (Eq. (sigma)): the trace identity
  sum_k Tr[Sigma^(2)k(tau) G^k(-tau)] = -(1/s) sum_q sum_QQ' P0^q_QQ'(tau) P0^{-q}_QQ'(tau)
  that ties its index structure to the pinned P0; Hermiticity; real inputs at
  n_k = 1 give real results (Sec. 5.1).
* hartree_fock (Eq. (sigma_hf)): the explicit four-index U = sum_Q V V route (Eq. (U_decompose)).
* dyson / mu search / energy: reduce to the closed-form non-interacting values; with a static
  Sigma_HF, to the closed form of (H0 + Sigma_HF, S); with a pole self-energy
  Sigma~(i w) = v (i w + mu - E)^{-1} v^dagger, to the orbital block of the closed-form G of the
  embedded quadratic system [[H0 + Sigma_HF, v], [v^dagger, E]] with overlap S + identity
  (a Schur complement), whose particle number fixes mu and whose hybridization fixes E_c;
  the E_hf term of the energy to the interaction energy of the determinant of gamma written
  with the four-index U = sum_Q V V and Wick's theorem.

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


def _gen_eigh(A, B):
    """Generalised eigenpairs A C = B C eps with C^dagger B C = I (scipy, independent of the oracle)."""
    eps, C = scipy.linalg.eigh(A, B)
    return eps, C


def _free_fermion_tau(xi, beta, tau):
    """g(tau) = -exp(-xi tau) / (1 + exp(-beta xi)): the transform of 1 / (i w - xi), 0 < tau < beta."""
    return -np.exp(-xi * tau - np.logaddexp(0.0, -beta * xi))


def _closed_form_g(Hs, Ss, mu, beta, tau):
    """-C diag(g_{eps - mu}(tau)) C^dagger per k for the generalised problem (Hs, Ss)."""
    out = []
    for H, S in zip(Hs, Ss):
        eps, C = _gen_eigh(H, S)
        g = np.stack([_free_fermion_tau(e - mu, beta, tau) for e in eps], axis=1)  # (t, a)
        out.append(np.einsum("ia,ta,ja->tij", C, g, C.conj()))
    return np.stack(out)


def _closed_form_gamma(Hs, Ss, mu, beta):
    return np.stack([(lambda e, C: (C * _fermi(e - mu, beta)) @ C.conj().T)(*_gen_eigh(H, S)) for H, S in zip(Hs, Ss)])


def _static_sigma(small, seed=21, scale=0.3):
    rng = np.random.default_rng(seed)
    Nk = small["H"].shape[0]
    X = rng.normal(size=(Nk, 3, 3)) + 1j * rng.normal(size=(Nk, 3, 3))
    return scale * (X + X.conj().transpose(0, 2, 1))


def _pole_system(small, seed=31):
    """Two poles per k: E^k = diag(e1, e2), couplings v^k (3 x 2), and the embedded (H, S)."""
    rng = np.random.default_rng(seed)
    H, S = small["H"], small["S"]
    Nk = H.shape[0]
    E = rng.uniform(-1.0, 1.0, size=(Nk, 2))
    v = 0.3 * (rng.normal(size=(Nk, 3, 2)) + 1j * rng.normal(size=(Nk, 3, 2)))
    Shf = _static_sigma(small)
    Hemb = np.zeros((Nk, 5, 5), complex)
    Semb = np.zeros((Nk, 5, 5), complex)
    for k in range(Nk):
        Hemb[k, :3, :3] = H[k] + Shf[k]
        Hemb[k, :3, 3:] = v[k]
        Hemb[k, 3:, :3] = v[k].conj().T
        Hemb[k, 3:, 3:] = np.diag(E[k])
        Semb[k, :3, :3] = S[k]
        Semb[k, 3:, 3:] = np.eye(2)
    return E, v, Shf, Hemb, Semb


def _pole_sigma_tau(E, v, mu, beta, tau):
    """Sigma~^k(tau) = v diag(g_{E - mu}(tau)) v^dagger."""
    g = np.stack([[_free_fermion_tau(e - mu, beta, tau) for e in Ek] for Ek in E])  # (k, p, t)
    return np.einsum("kip,kpt,kjp->ktij", v, g, v.conj())


def _bisect(f, target, lo=-20.0, hi=20.0, width=1e-14):
    while hi - lo > width:
        mid = 0.5 * (lo + hi)
        if f(mid) > target:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def _static_pin(small, mu=0.2):
    """Residuals of Dyson with Sigma_HF only against G0 of (H0 + Sigma_HF, S): (G at mu, mu of the search)."""
    H, S, ops, beta = small["H"], small["S"], small["ops"], small["beta"]
    Nk, n = H.shape[0], small["n"]
    Shf = _static_sigma(small)
    zero_t = np.zeros((Nk, n, 3, 3), complex)
    G, _ = gw.dyson(H, S, Shf, zero_t, mu, ops)
    Gref = _closed_form_g(H + Shf, S, mu, beta, ops["tau"])
    _, mus = gw.dyson(H, S, Shf, zero_t, 0.0, ops, n_elec=3.0, search_mu=True)
    eps = np.concatenate([_gen_eigh(a, b)[0] for a, b in zip(H + Shf, S)])
    muref = _bisect(lambda m: S_SPIN / Nk * _fermi(eps - m, beta).sum(), 3.0)
    return np.abs(G - Gref).max(), abs(mus - muref)


def _pole_pin(small, mu=0.1):
    """Residuals of Dyson with a two-pole Sigma~ against the embedded closed form: (G at mu, mu of the search)."""
    H, S, ops, beta = small["H"], small["S"], small["ops"], small["beta"]
    Nk = H.shape[0]
    E, v, Shf, Hemb, Semb = _pole_system(small)
    G, _ = gw.dyson(H, S, Shf, _pole_sigma_tau(E, v, mu, beta, ops["tau"]), mu, ops)
    Gref = _closed_form_g(Hemb, Semb, mu, beta, ops["tau"])[:, :, :3, :3]
    # the search: the pole self-energy is built at the trial mu, so the root is that of the
    # embedded system's orbital-block particle number (s/N_k) sum_k Tr[gamma_oo S]
    def n_emb(m):
        gam = _closed_form_gamma(Hemb, Semb, m, beta)[:, :3, :3]
        return float(np.real(S_SPIN / Nk * np.einsum("kij,kji->", gam, S)))

    muref = _bisect(n_emb, 3.0)
    _, mus = gw.dyson(H, S, Shf, _pole_sigma_tau(E, v, muref, beta, ops["tau"]), 0.0, ops, n_elec=3.0,
                      search_mu=True)
    return np.abs(G - Gref).max(), abs(mus - muref)


def test_dyson_with_static_self_energy_is_g0_of_the_shifted_hamiltonian(small):
    rg, rmu = _static_pin(small)
    assert rg < 1e-10 and rmu < 1e-9, (rg, rmu)


def test_dyson_with_pole_self_energy_is_the_embedded_green_function(small):
    rg, rmu = _pole_pin(small)
    assert rg < 1e-10 and rmu < 1e-9, (rg, rmu)


def _slater_interaction(gam, V, Nk):
    """<U> in the determinant of gamma (per cell): U_{ij,kl} = sum_Q V_ij(Q) V_kl(Q) (Eq. (U_decompose)),
    <c+_i c+_k c_l c_j> = gamma_ji gamma_lk s^2 - gamma_li gamma_jk s (Wick, spin sums), momenta conserved."""
    U = np.einsum("abQij,cdQkl->abcdijkl", V, V)
    e = 0.0
    for k in range(Nk):
        for kp in range(Nk):
            e += S_SPIN ** 2 * np.einsum("ijkl,ji,lk->", U[k, k, kp, kp], gam[k], gam[kp])
            e -= S_SPIN * np.einsum("ijkl,li,jk->", U[k, kp, kp, k], gam[k], gam[kp])
    return 0.5 * e / Nk ** 2


def _ehf_pin(fine_grid, energy=None):
    energy = energy or gw.energy
    beta, n, ops = fine_grid
    nk = (1, 1, 2)
    H, S, V = random_system(nk, 2, 3, seed=7)
    mu = gw.mu_noninteracting(H, S, beta, 2.0)
    G = gw.g0_tau(H, S, mu, beta, ops["tau"])
    gam = gw.density_matrix(G)
    Shf, _, _ = gw.hartree_fock(gam, V, nk)
    E = energy(H, S, G, Shf, np.zeros_like(G), beta)
    return abs(E[2] - _slater_interaction(gam, V, 2))


def _ec_pin(small, energy=None):
    energy = energy or gw.energy
    H, S, ops, beta = small["H"], small["S"], small["ops"], small["beta"]
    Nk, mu = H.shape[0], 0.1
    E, v, Shf, Hemb, Semb = _pole_system(small)
    G = _closed_form_g(Hemb, Semb, mu, beta, ops["tau"])[:, :, :3, :3]
    Sig = _pole_sigma_tau(E, v, mu, beta, ops["tau"])
    gam = _closed_form_gamma(Hemb, Semb, mu, beta)
    # (1/beta) sum_n Tr[G Sigma~](i w_n) = Tr[G_oe v^dagger] at equal time = Tr[gamma_oe v^dagger]
    ec_ref = S_SPIN / (2 * Nk) * np.einsum("kip,kip->", gam[:, :3, 3:], v.conj())
    Ec = energy(H, S, G, Shf, Sig, beta)[3]
    return abs(Ec - ec_ref), abs(ec_ref)


def test_energy_hartree_fock_term_is_the_interaction_of_the_determinant(fine_grid):
    assert _ehf_pin(fine_grid) < 1e-12


def test_energy_correlation_term_is_half_the_pole_hybridization(small):
    res, scale = _ec_pin(small)
    assert scale > 1e-2 and res < 1e-10 * max(1.0, scale), (res, scale)


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
    # brute force: bisection on N(mu) to a width of 1e-14 (the oracle's search stops at |N - N_e| <= 1e-11)
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


def test_screened_interaction_at_mirrored_frequencies_is_the_adjoint(small):
    """With Hermitian P0(tau) blocks and a bosonic set closed under Omega -> -Omega, P0 and the
    solve [I - P0]^{-1} P0 at -Omega_n are the adjoints of their values at Omega_n: a solver may
    handle the non-negative frequencies and fill the rest.  An anti-Hermitian part in P0(tau)
    breaks it."""
    ops = small["ops"]
    P0 = gw.polarization(small["G"], small["V"], NK)
    mb = list(ops["mats_b"])
    mirror = [mb.index(-n) for n in mb]

    def residuals(P0_tau):
        _, P0w, Pw = gw.screened_interaction(P0_tau, ops["TB"], ops["TBbar"])
        r0 = np.abs(P0w[:, mirror] - P0w.conj().transpose(0, 1, 3, 2)).max() / np.abs(P0w).max()
        r1 = np.abs(Pw[:, mirror] - Pw.conj().transpose(0, 1, 3, 2)).max() / np.abs(Pw).max()
        return r0, r1

    r0, r1 = residuals(P0)
    assert r0 < 1e-13 and r1 < 1e-12, (r0, r1)
    rng = np.random.default_rng(3)
    H = rng.standard_normal(P0.shape) + 1j * rng.standard_normal(P0.shape)
    H = 0.5 * (H + H.conj().transpose(0, 1, 3, 2))
    s0, s1 = residuals(P0 + 1e-3 * np.abs(P0).max() * 1j * H)  # i H is anti-Hermitian
    assert s0 > 1e-5 and s1 > 1e-5, (s0, s1)


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


def test_planted_dyson_and_energy_slips_fail_the_pins(small, fine_grid, monkeypatch):
    """Slips planted into the oracle's Dyson step and energy are caught by the new pins."""
    good = gw.dyson_matsubara

    def sigma_sign(H0, S, Shf, Sw, mu, nu):  # + Sigma in place of - Sigma
        return good(H0, S, -Shf, -Sw, mu, nu)

    def mu_times_identity(H0, S, Shf, Sw, mu, nu):  # (i w + mu) S -> i w S + mu I
        Nk, nao = H0.shape[0], H0.shape[1]
        shift = mu * (S - np.eye(nao)[None])
        return good(H0 + shift, S, Shf, Sw, mu, nu)

    for slip in (sigma_sign, mu_times_identity):
        monkeypatch.setattr(gw, "dyson_matsubara", slip)
        rg_s, _ = _static_pin(small)
        rg_p, _ = _pole_pin(small)
        monkeypatch.setattr(gw, "dyson_matsubara", good)
        assert max(rg_s, rg_p) > 1e-4, slip.__name__
    # a dropped pole sign only (Sigma~ with the wrong sign, Sigma_HF right) fails the pole pin
    monkeypatch.setattr(gw, "dyson_matsubara", lambda H0, S, Shf, Sw, mu, nu: good(H0, S, Shf, -Sw, mu, nu))
    rg_p, _ = _pole_pin(small)
    monkeypatch.setattr(gw, "dyson_matsubara", good)
    assert rg_p > 1e-4

    # energy: E_hf without the factor 1/2, E_c with the wrong sign, E_c without the mirror beta - tau
    def ehf_double(H0, S, G, Shf, Sig, beta, s=2):
        E = gw.energy(H0, S, G, Shf, Sig, beta, s)
        return E[0] + E[2], E[1], 2 * E[2], E[3]

    def ec_flipped(H0, S, G, Shf, Sig, beta, s=2):
        E = gw.energy(H0, S, G, Shf, Sig, beta, s)
        return E[0] - 2 * E[3], E[1], E[2], -E[3]

    def ec_no_mirror(H0, S, G, Shf, Sig, beta, s=2):
        return gw.energy(H0, S, G, Shf, Sig[:, ::-1], beta, s)

    assert _ehf_pin(fine_grid, ehf_double) > 1e-3
    assert _ec_pin(small, ec_flipped)[0] > 1e-3
    assert _ec_pin(small, ec_no_mirror)[0] > 1e-4
