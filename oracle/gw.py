"""Full-Brillouin-zone finite-temperature GW step of the oracle (complex128).

TEST INFRASTRUCTURE ONLY: the plain, slow CPU definition the CUDA library is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the
library; it knows nothing of symmetry: every k and q of the mesh, AO basis.

Conventions (interface shared with the library through the input data only)
--------------------------------------------------------------------------
* k mesh n1 x n2 x n3, Gamma centred; flat index (i1 * n2 + i2) * n3 + i3,
  fractional coordinate (i1/n1, i2/n2, i3/n3) in the reciprocal basis.
* ``H0, S``: [Nk][nao][nao].  ``V(k1, k2)`` returns V^{k1,k2}_{Q,ij} as
  [naux][nao][nao] (``V`` may be a callable or a full [Nk][Nk][naux][nao][nao]
  array).
* ``G, Sigma``: [Nk][ntau][nao][nao]; ``P0, P``: [Nk(q)][ntau][naux][naux];
  tau on the Chebyshev nodes of ``oracle.grid``.
* spin-restricted closed shell, spin factor s = 2 (the spin reading below).

Readings of the paper
---------------------
* Sign of the bare bubble: Eq. (P0) is printed with -1/N_k; combined with
  G(-tau) = -G(beta - tau) that makes P0(i Omega_0) positive semidefinite and
  the geometric series of Eq. (P02P) anti-screening.  ``loop_sign = +1`` (the
  default) uses the physical sign, P0 = +(s/N_k) sum ..., which is <= 0 at
  Omega_0; ``loop_sign = -1`` is the literal print.
* Spin sums of Eqs. (P0) and (sigma_hf): G is spin diagonal; the closed loops
  (P0 and the Hartree term) carry s = 2, exchange and Sigma carry none.
* gamma = G(tau = 0^-) = -G(beta^-) (antiperiodicity), with G(beta^-) the value
  of the Chebyshev interpolant at x = 1.
* The number of electrons counts both spins: N_e = (s/N_k) sum_k Tr[gamma S].
* Total energy (not defined in the paper): Galitskii-Migdal form, see
  ``energy``.
"""
from __future__ import annotations

import numpy as np

from . import grid

__all__ = [
    "kmesh_size",
    "kindex",
    "kadd",
    "ksub",
    "fermi",
    "mu_noninteracting",
    "g0_tau",
    "g_minus_tau",
    "polarization",
    "to_matsubara",
    "screened_interaction",
    "self_energy",
    "density_matrix",
    "hartree_fock",
    "dyson_matsubara",
    "particle_number",
    "dyson",
    "energy",
    "scgw_iteration",
    "as_vfun",
]


# --------------------------------------------------------------------------
# k mesh bookkeeping
# --------------------------------------------------------------------------
def kmesh_size(nk) -> int:
    return int(nk[0] * nk[1] * nk[2])


def kindex(nk, i1, i2, i3) -> int:
    return ((i1 % nk[0]) * nk[1] + (i2 % nk[1])) * nk[2] + (i3 % nk[2])


def _kvec(nk, k):
    i3 = k % nk[2]
    i2 = (k // nk[2]) % nk[1]
    i1 = k // (nk[1] * nk[2])
    return i1, i2, i3


def kadd(nk, ka, kb) -> int:
    """Index of k_a + k_b, reduced to the mesh (momentum conservation modulo K)."""
    a, b = _kvec(nk, ka), _kvec(nk, kb)
    return kindex(nk, a[0] + b[0], a[1] + b[1], a[2] + b[2])


def ksub(nk, ka, kb) -> int:
    a, b = _kvec(nk, ka), _kvec(nk, kb)
    return kindex(nk, a[0] - b[0], a[1] - b[1], a[2] - b[2])


def as_vfun(V):
    """Accept V as a full [Nk][Nk][naux][nao][nao] array or as V(k1, k2)."""
    if callable(V):
        return V
    arr = np.asarray(V)
    return lambda k1, k2: arr[k1, k2]


# --------------------------------------------------------------------------
# non-interacting quantities
# --------------------------------------------------------------------------
def fermi(x, beta):
    """f(x) = 1 / (exp(beta x) + 1), evaluated without overflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x > 0
    e = np.exp(-beta * x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(beta * x[~pos]))
    return out


def _gen_eig(H, S):
    """Generalised Hermitian eigenproblem H C = S C eps with C^dagger S C = I."""
    L = np.linalg.cholesky(S)
    Linv = np.linalg.inv(L)
    Ht = Linv @ H @ Linv.conj().T
    Ht = 0.5 * (Ht + Ht.conj().T)
    eps, Y = np.linalg.eigh(Ht)
    return eps, Linv.conj().T @ Y


def mu_noninteracting(H0, S, beta, n_elec, s=2, tol=1e-13):
    """Chemical potential of the non-interacting system by bisection.

    (s/N_k) sum_{k,n} f(eps_kn - mu) = N_e (Sec. 4.1, the particle-number
    condition, with gamma of the non-interacting G).
    """
    Nk = H0.shape[0]
    eps = np.concatenate([_gen_eig(H0[k], S[k])[0] for k in range(Nk)])
    lo, hi = eps.min() - 10.0, eps.max() + 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        n = s / Nk * fermi(eps - mid, beta).sum()
        if n > n_elec:
            hi = mid
        else:
            lo = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def g0_tau(H0, S, mu, beta, tau):
    """Closed-form non-interacting G^k(tau), 0 < tau < beta.

    From Eq. (dyson) with Sigma = 0: G(i w) = C diag(1/(i w + mu - eps)) C^dagger,
    whose transform is G(tau) = -C diag(exp(-xi tau) / (1 + exp(-beta xi))) C^dagger,
    xi = eps - mu.  For xi < 0 the equal form -exp(xi (beta - tau)) / (exp(beta xi) + 1)
    is used so that no exponential overflows.
    """
    Nk, nao = H0.shape[0], H0.shape[1]
    tau = np.asarray(tau, dtype=np.float64)
    G = np.empty((Nk, tau.size, nao, nao), dtype=np.complex128)
    for k in range(Nk):
        eps, C = _gen_eig(H0[k], S[k])
        xi = eps - mu
        g = np.empty((tau.size, nao))
        for a, x in enumerate(xi):
            if x >= 0:
                g[:, a] = -np.exp(-x * tau) / (1.0 + np.exp(-beta * x))
            else:
                g[:, a] = -np.exp(x * (beta - tau)) / (np.exp(beta * x) + 1.0)
        G[k] = np.einsum("ia,ta,ja->tij", C, g, C.conj())
    return G


def g_minus_tau(G):
    """G(-tau_j) = -G(beta - tau_j) = -G(tau_{n-1-j}) (antiperiodicity, mirror nodes)."""
    return -G[:, ::-1]


# --------------------------------------------------------------------------
# P0, P, Sigma
# --------------------------------------------------------------------------
def polarization(G, V, nk, s=2, loop_sign=+1, qs=None, pairs=None, taus=None):
    """Bare bubble P0^q_{QQ'}(tau) of Eq. (P0) for every q of the mesh.

    P0^q_{QQ'}(tau) = loop_sign (s/N_k) sum_k sum_{abcd}
        V^{k,k+q}_{da}(Q) G^k_{cd}(-tau) G^{k+q}_{ab}(tau) V^{k+q,k}_{bc}(Q'),
    evaluated in the order of Algorithm 3:
        X1(Q)_{ca}  = sum_d G^k_{cd}(-tau) V^{k,k+q}_{da}(Q),
        X2(Q')_{ac} = sum_b G^{k+q}_{ab}(tau) V^{k+q,k}_{bc}(Q'),
        P0_{QQ'}   += sum_{ca} X1(Q)_{ca} X2(Q')_{ac}.
    ``qs`` restricts the evaluation to a list of q (other entries stay zero); ``pairs``, a set
    of (k, k + q), to the terms of those pairs (a partial sum over k, as one rank of a partition
    of the pairs computes it); ``taus``, to a list of tau indices (G is still needed at every
    tau: G(-tau_j) is read at the mirror node).
    """
    Vf = as_vfun(V)
    Nk, ntau, nao, _ = G.shape
    ts = np.arange(ntau) if taus is None else np.asarray(taus)
    nt = ts.size
    Gm = g_minus_tau(G)
    naux = Vf(0, 0).shape[0]
    P0 = np.zeros((Nk, ntau, naux, naux), dtype=np.complex128)
    for q in (range(Nk) if qs is None else qs):
        for k in range(Nk):
            kq = kadd(nk, k, q)
            if pairs is not None and (k, kq) not in pairs:
                continue
            Vkq = Vf(k, kq)  # [Q][d][a]
            Vqk = Vf(kq, k)  # [Q'][b][c]
            # X1[t][c][Q][a] = sum_d G^k(-tau)[t][c][d] V^{k,k+q}[Q][d][a]   (one GEMM over all t, Q)
            X1 = (Gm[k][ts].reshape(nt * nao, nao) @ Vkq.transpose(1, 0, 2).reshape(nao, naux * nao))
            X1 = X1.reshape(nt, nao, naux, nao)
            # X2[t][a][Q'][c] = sum_b G^{k+q}(tau)[t][a][b] V^{k+q,k}[Q'][b][c]
            X2 = (G[kq][ts].reshape(nt * nao, nao) @ Vqk.transpose(1, 0, 2).reshape(nao, naux * nao))
            X2 = X2.reshape(nt, nao, naux, nao)
            # P0[t][Q][Q'] += sum_{c,a} X1[t][c][Q][a] X2[t][a][Q'][c]
            A = X1.transpose(0, 2, 1, 3).reshape(nt, naux, nao * nao)  # [t][Q][(c,a)]
            B = X2.transpose(0, 2, 3, 1).reshape(nt, naux, nao * nao)  # [t][Q'][(c,a)]
            P0[q, ts] += np.matmul(A, B.transpose(0, 2, 1))
    P0 *= loop_sign * s / Nk
    return P0


def to_matsubara(F_tau, T):
    """Apply a (n_w x n_tau) map along the tau axis (axis 1): out[q, m] = sum_t T[m, t] F[q, t]."""
    return np.moveaxis(np.tensordot(T, F_tau, axes=(1, 1)), 0, 1)


def screened_interaction(P0_tau, TB, TBbar):
    """Eq. (P02P): P(i Omega) = [I - P0(i Omega)]^{-1} P0(i Omega), then back to tau.

    P0(i Omega_m) = sum_j TB[m, j] P0(tau_j) (forward bosonic map),
    P(tau_j) = sum_m TBbar[j, m] P(i Omega_m) (its least-squares inverse).
    """
    P0w = to_matsubara(P0_tau, TB)
    naux = P0w.shape[-1]
    I = np.eye(naux)
    Pw = np.linalg.solve(I[None, None] - P0w, P0w)  # one solve per (q, m)
    return to_matsubara(Pw, TBbar), P0w, Pw


def self_energy(G, P, V, nk, ks=None, pairs=None, taus=None):
    """Dynamic GW self-energy of Eq. (sigma) for every k of the mesh.

    Sigma^k_ij(tau) = -(1/N_k) sum_q sum_ab sum_QQ'
        G^{k-q}_ab(tau) V^{k,k-q}_ia(Q) P^q_QQ'(tau) V^{k-q,k}_bj(Q'),
    evaluated in the order of Algorithm 4:
        X1(Q)_{ib}  = sum_a V^{k,k-q}_{ia}(Q) G^{k-q}_{ab}(tau),
        X2(Q')_{ib} = sum_Q X1(Q)_{ib} P^q_{QQ'}(tau),
        Sigma_ij   += sum_{Q' b} X2(Q')_{ib} V^{k-q,k}_{bj}(Q').
    ``ks`` restricts the evaluation to a list of k (other entries stay zero); ``pairs``, a set
    of (k, k - q), to the terms of those pairs (a partial sum over q); ``taus``, to a list of tau
    indices (G and P are read at those only).
    """
    Vf = as_vfun(V)
    Nk, ntau, nao, _ = G.shape
    ts = np.arange(ntau) if taus is None else np.asarray(taus)
    nt = ts.size
    naux = P.shape[-1]
    Sig = np.zeros_like(G)
    for k in (range(Nk) if ks is None else ks):
        for q in range(Nk):
            kmq = ksub(nk, k, q)
            if pairs is not None and (k, kmq) not in pairs:
                continue
            V1 = Vf(k, kmq)  # [Q][i][a]
            V2 = Vf(kmq, k)  # [Q'][b][j]
            # X1[Q][i][t][b] = sum_a V^{k,k-q}[Q][i][a] G^{k-q}(tau)[t][a][b]   (one GEMM over all Q, t)
            X1 = V1.reshape(naux * nao, nao) @ G[kmq][ts].transpose(1, 0, 2).reshape(nao, nt * nao)
            X1 = X1.reshape(naux, nao, nt, nao).transpose(2, 0, 1, 3).reshape(nt, naux, nao * nao)
            # X2[t][Q'][(i,b)] = sum_Q P^q(tau)[t][Q][Q'] X1[t][Q][(i,b)]
            X2 = np.matmul(P[q][ts].transpose(0, 2, 1), X1)
            # Sigma[t][i][j] += sum_{Q',b} X2[t][Q'][i][b] V^{k-q,k}[Q'][b][j]
            X2 = X2.reshape(nt, naux, nao, nao).transpose(0, 2, 1, 3).reshape(nt, nao, naux * nao)
            Sig[k, ts] += np.matmul(X2, V2.reshape(naux * nao, nao))
    Sig *= -1.0 / Nk
    return Sig


# --------------------------------------------------------------------------
# density matrix, Hartree-Fock, Dyson, particle number
# --------------------------------------------------------------------------
def density_matrix(G):
    """gamma^k = G^k(0^-) = -G^k(beta^-), G(beta^-) from the Chebyshev interpolant."""
    r = grid.value_at_beta_minus(G.shape[1])
    return -np.einsum("t,ktij->kij", r, G)


def hartree_fock(gamma, V, nk, s=2, ks=None):
    """Sigma^(HF) = J + K of Eq. (sigma_hf).

    J^k_ij = (s/N_k) sum_{k'} sum_Q V^{kk}_ij(Q) sum_ab gamma^{k'}_ab V^{k'k'}_ba(Q)
    K^k_ij = -(1/N_k) sum_{k'} sum_Q sum_ab V^{kk'}_ia(Q) gamma^{k'}_ab V^{k'k}_bj(Q)
    ``ks`` restricts J and K to a list of k (other entries stay zero).
    """
    Vf = as_vfun(V)
    Nk = gamma.shape[0]
    naux = Vf(0, 0).shape[0]
    rho = np.zeros(naux, dtype=np.complex128)
    for kp in range(Nk):
        rho += np.einsum("ab,Qba->Q", gamma[kp], Vf(kp, kp))
    J = np.zeros_like(gamma)
    K = np.zeros_like(gamma)
    for k in (range(Nk) if ks is None else ks):
        J[k] = (s / Nk) * np.einsum("Qij,Q->ij", Vf(k, k), rho)
        for kp in range(Nk):
            K[k] -= (1.0 / Nk) * np.einsum("Qia,ab,Qbj->ij", Vf(k, kp), gamma[kp], Vf(kp, k), optimize=True)
    return J + K, J, K


def dyson_matsubara(H0, S, Sigma_hf, Sigma_w, mu, nu_f):
    """Eq. (dyson): G(i w_n) = [(i w_n + mu) S - H0 - Sigma_HF - Sigma~(i w_n)]^{-1}."""
    Nk, nw = Sigma_w.shape[0], Sigma_w.shape[1]
    Gw = np.empty_like(Sigma_w)
    for k in range(Nk):
        F = H0[k] + Sigma_hf[k]
        for m in range(nw):
            A = (1j * nu_f[m] + mu) * S[k] - F - Sigma_w[k, m]
            Gw[k, m] = np.linalg.inv(A)
    return Gw


def particle_number(gamma, S, s=2):
    """N = (s/N_k) sum_k Tr[gamma^k S^k] (Sec. 4.1, after Eq. (sigma_hf))."""
    Nk = gamma.shape[0]
    return float(np.real(s / Nk * np.einsum("kij,kji->", gamma, S)))


def dyson(H0, S, Sigma_hf, Sigma_tau, mu, grid_ops, n_elec=None, s=2, search_mu=False,
          mu_lo=-20.0, mu_hi=20.0, n_tol=1e-11, max_trials=200):
    """G(tau) from Eq. (dyson), optionally with the chemical-potential search.

    Sigma~(i w) = TF Sigma~(tau); G(i w) by inversion; G(tau) = TFbar G(i w).
    With search_mu, mu solves N(mu) = N_e (Sec. 4.1), N the particle number of
    gamma = -G(beta^-), by plain bisection of [mu_lo, mu_hi]: the midpoint is tried, the half
    that keeps the root is kept (N increases with mu), until |N(mu) - N_e| <= n_tol (the given mu
    is then not used).
    """
    TF, TFbar, nu_f = grid_ops["TF"], grid_ops["TFbar"], grid_ops["nu_f"]
    Sigma_w = to_matsubara(Sigma_tau, TF)
    wgt = -(grid.value_at_beta_minus(TF.shape[1]) @ TFbar)  # gamma = sum_m wgt[m] G(i w_m)

    def number(mu_):
        Gw = dyson_matsubara(H0, S, Sigma_hf, Sigma_w, mu_, nu_f)
        return particle_number(np.einsum("m,kmij->kij", wgt, Gw), S, s)

    if search_mu:
        lo, hi = mu_lo, mu_hi
        for _ in range(max_trials):
            mu = 0.5 * (lo + hi)
            n = number(mu)
            if abs(n - n_elec) <= n_tol:
                break
            if n > n_elec:
                hi = mu
            else:
                lo = mu
    Gw = dyson_matsubara(H0, S, Sigma_hf, Sigma_w, mu, nu_f)
    return to_matsubara(Gw, TFbar), mu


def particle_number_and_slope(H0, S, Sigma_hf, Sigma_tau, mu, grid_ops, s=2):
    """(N(mu), N'(mu)): the particle number of the Dyson solution at mu and its derivative,
    N'(mu) from differentiating Eq. (dyson), dG(i w)/dmu = -G(i w) S G(i w)."""
    TF, TFbar, nu_f = grid_ops["TF"], grid_ops["TFbar"], grid_ops["nu_f"]
    Sigma_w = to_matsubara(Sigma_tau, TF)
    wgt = -(grid.value_at_beta_minus(TF.shape[1]) @ TFbar)
    Gw = dyson_matsubara(H0, S, Sigma_hf, Sigma_w, mu, nu_f)
    gam = np.einsum("m,kmij->kij", wgt, Gw)
    dgam = -np.einsum("m,kmij,kjl,kmlp->kip", wgt, Gw, S, Gw)
    return particle_number(gam, S, s), particle_number(dgam, S, s)


def energy(H0, S, G_tau, Sigma_hf, Sigma_tau, beta, s=2):
    """Total energy in the Galitskii-Migdal form (not defined in the paper; a reading of this module).

    E = (s/N_k) sum_k Tr[gamma H0] + (s/2N_k) sum_k Tr[gamma Sigma_HF] + E_c,
    E_c = -(s/2N_k) sum_k int_0^beta Tr[G^k(tau) Sigma~^k(beta - tau)] dtau.
    The integral is n-point Gauss-Legendre on [0, beta] applied to the
    Chebyshev interpolants of G and Sigma~; the product has degree 2n - 2, so
    the rule is exact.  Returns (E, E_one_body, E_hf, E_c) as complex numbers.
    """
    Nk, nt = G_tau.shape[0], G_tau.shape[1]
    gam = density_matrix(G_tau)
    e1 = s / Nk * np.einsum("kij,kji->", gam, H0)
    ehf = s / (2 * Nk) * np.einsum("kij,kji->", gam, Sigma_hf)
    xg, wg = np.polynomial.legendre.leggauss(nt)
    C = grid.cheb_values_to_coeffs(nt)
    Tg = grid._cheb_T(nt, xg)  # (l, g)
    L = Tg.T @ C  # values at x_g from node values
    Gg = np.einsum("gt,ktij->kgij", L, G_tau)
    Sg = np.einsum("gt,ktij->kgij", L, Sigma_tau)[:, ::-1]  # beta - tau_g is the mirror node
    ec = -(s / (2 * Nk)) * 0.5 * beta * np.einsum("g,kgij,kgji->", wg, Gg, Sg)
    return e1 + ehf + ec, e1, ehf, ec


def scgw_iteration(H0, S, V, nk, G_tau, mu, grid_ops, n_elec, s=2, loop_sign=+1, search_mu=True,
                   Sigma_old=None, Sigma_hf_old=None, damping=1.0):
    """One self-consistency pass: G -> P0 -> P -> Sigma~, Sigma_HF -> damping -> Dyson (+ mu).

    Damping (reading, not in the paper): Sigma <- (1 - a) Sigma_old + a Sigma_new
    with a = ``damping``, applied to Sigma~(tau) and Sigma_HF alike.
    Returns a dict with every intermediate.
    """
    P0 = polarization(G_tau, V, nk, s, loop_sign)
    P, P0w, Pw = screened_interaction(P0, grid_ops["TB"], grid_ops["TBbar"])
    Sig = self_energy(G_tau, P, V, nk)
    gam = density_matrix(G_tau)
    Shf, J, K = hartree_fock(gam, V, nk, s)
    if Sigma_old is not None:
        Sig = (1.0 - damping) * Sigma_old + damping * Sig
        Shf = (1.0 - damping) * Sigma_hf_old + damping * Shf
    Gn, mu_n = dyson(H0, S, Shf, Sig, mu, grid_ops, n_elec, s, search_mu=search_mu)
    return dict(P0=P0, P0w=P0w, Pw=Pw, P=P, Sigma=Sig, Sigma_hf=Shf, J=J, K=K, gamma=gam, G_new=Gn, mu=mu_n)
