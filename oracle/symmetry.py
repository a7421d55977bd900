"""Space-group machinery of the oracle (Sec. 3 and Algorithm 1).

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).  Independent of the input
generator and of the library: the rotation matrices of the real spherical
harmonics come from the exponential of the angular-momentum generators (the
library and the generator fit them from sampled harmonics instead), and the
simultaneous diagonalisation refines subspaces character by character as the
paper describes (Sec. 3.4), rather than diagonalising one combination.

Contents
--------
* harmonic_rotation(l, R): D with Y_lm(R^{-1} u) = sum_m' Y_lm'(u) D[m', m]
  (Sec. 3.2: Wigner matrices, with (-1)^l for improper rotations).
* orbital_rep: O^k(alpha) of Eq. (basis_rot) for a crystal basis.
* stars / wedge of a k mesh (Sec. 4.2).
* projective representation and factor system, Eqs. (projrep), (factor).
* Dirac characters, Eq. (dirac) (second line; the averaged first line is used
  as the definition, which agrees with it).
* simultaneous diagonalisation -> U^k and block sizes (Sec. 3.4, Algorithm 1).

Pins (tests/test_oracle_symmetry.py): D for l = 1 is the permuted rotation
matrix; D is a homomorphism; wedge sizes equal Table 2; the projective rule
and the cocycle identity; lambda = 1 for symmorphic groups; Dirac characters
commute with D and with each other; U block-diagonalises covariant matrices;
the commutant dimension matches (1/h) sum_g |Tr D(g)|^2; covariance of the
synthetic inputs and equivariance of the oracle's self-energy.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg
from scipy.spatial.transform import Rotation


# ---------------------------------------------------------------------------
# real spherical harmonics: rotation matrices from the Lie algebra
# ---------------------------------------------------------------------------
def angular_momentum(l: int):
    """L_x, L_y, L_z in the complex basis |l m>, m = -l..l (Condon-Shortley ladder phases)."""
    m = np.arange(-l, l + 1)
    Lz = np.diag(m).astype(np.complex128)
    Lp = np.zeros((2 * l + 1, 2 * l + 1), dtype=np.complex128)
    for i, mm in enumerate(m[:-1]):
        Lp[i + 1, i] = np.sqrt(l * (l + 1) - mm * (mm + 1))
    Lm = Lp.conj().T
    return (Lp + Lm) / 2.0, (Lp - Lm) / 2.0j, Lz


def complex_to_real(l: int) -> np.ndarray:
    """C with Y_real[mu] = sum_m C[m, mu] Y_l^m (columns ordered mu = -l..l)."""
    C = np.zeros((2 * l + 1, 2 * l + 1), dtype=np.complex128)
    s2 = np.sqrt(0.5)
    for mu in range(-l, l + 1):
        c = mu + l
        if mu == 0:
            C[l, c] = 1.0
        elif mu > 0:
            C[l + mu, c] = s2 * (-1) ** mu
            C[l - mu, c] = s2
        else:
            a = -mu
            C[l + a, c] = s2 * (-1) ** a / 1j
            C[l - a, c] = -s2 / 1j
    return C


def harmonic_rotation(l: int, R: np.ndarray) -> np.ndarray:
    """Real-harmonic rotation matrix of the (possibly improper) orthogonal R."""
    R = np.asarray(R, dtype=np.float64)
    sign = 1.0
    if np.linalg.det(R) < 0:
        R = -R
        sign = (-1.0) ** l
    if l == 0:
        return np.array([[sign]])
    rv = Rotation.from_matrix(R).as_rotvec()
    Lx, Ly, Lz = angular_momentum(l)
    Dc = scipy.linalg.expm(-1j * (rv[0] * Lx + rv[1] * Ly + rv[2] * Lz))
    C = complex_to_real(l)
    Dr = C.conj().T @ Dc @ C
    assert np.abs(Dr.imag).max() < 1e-12
    return sign * Dr.real


# ---------------------------------------------------------------------------
# crystal, mesh and stars
# ---------------------------------------------------------------------------
class Crystal:
    """lattice: columns are the primitive vectors; ops: list of (R, v) Cartesian."""

    def __init__(self, lattice, positions, ops, shells):
        self.A = np.asarray(lattice, dtype=np.float64)
        self.Ai = np.linalg.inv(self.A)
        self.pos = np.asarray(positions, dtype=np.float64)
        self.ops = [(np.asarray(R, float), np.asarray(v, float)) for R, v in ops]
        self.shells = list(shells)
        self.per_atom = sum(2 * l + 1 for l in self.shells)
        self.n = self.per_atom * len(self.pos)
        # atom permutation and lattice translation T with R r_x + v = r_x' + T
        self.perm, self.trans = [], []
        for R, v in self.ops:
            p, t = [], []
            for x in range(len(self.pos)):
                rp = R @ self.pos[x] + v
                for y in range(len(self.pos)):
                    f = self.Ai @ (rp - self.pos[y])
                    if np.allclose(f, np.round(f), atol=1e-9):
                        p.append(y)
                        t.append(np.round(f))
                        break
                else:
                    raise ValueError("operation does not map the crystal onto itself")
            self.perm.append(p)
            self.trans.append(t)

    def k_action(self, iop: int) -> np.ndarray:
        """Matrix M with frac(R k) = M frac(k) (reciprocal basis)."""
        R = self.ops[iop][0]
        return self.A.T @ R @ self.Ai.T


def kgrid(nk):
    return np.array(list(itertools.product(range(nk[0]), range(nk[1]), range(nk[2]))))


def k_image(crystal: Crystal, nk, iop: int, k: int) -> int:
    iv = kgrid(nk)[k]
    M = crystal.k_action(iop)
    f = M @ (iv / np.asarray(nk, float))
    g = np.round(f * np.asarray(nk)).astype(int) % np.asarray(nk)
    return int((g[0] * nk[1] + g[1]) * nk[2] + g[2])


def stars(crystal: Crystal, nk):
    """Wedge representatives (first member of each star) and the star of each k."""
    Nk = nk[0] * nk[1] * nk[2]
    rep = -np.ones(Nk, dtype=int)
    reps = []
    for k in range(Nk):
        if rep[k] >= 0:
            continue
        reps.append(k)
        for o in range(len(crystal.ops)):
            rep[k_image(crystal, nk, o, k)] = len(reps) - 1
    return reps, rep


# ---------------------------------------------------------------------------
# representations
# ---------------------------------------------------------------------------
def orbital_rep(crystal: Crystal, iop: int, kfrac) -> np.ndarray:
    """O^k(alpha) of Eq. (basis_rot): column (x, s, m) -> row (x', s, m'), phase exp(-i (R k).T)."""
    R = crystal.ops[iop][0]
    kr = crystal.k_action(iop) @ np.asarray(kfrac, float)
    O = np.zeros((crystal.n, crystal.n), dtype=np.complex128)
    for x in range(len(crystal.pos)):
        xp = crystal.perm[iop][x]
        ph = np.exp(-2j * np.pi * kr @ crystal.trans[iop][x])
        off = 0
        for l in crystal.shells:
            D = harmonic_rotation(l, R)
            a = x * crystal.per_atom + off
            b = xp * crystal.per_atom + off
            O[b:b + 2 * l + 1, a:a + 2 * l + 1] = ph * D
            off += 2 * l + 1
    return O


def k_dot(crystal: Crystal, kfrac, w) -> float:
    """k . w for fractional k (reciprocal basis) and a Cartesian vector w."""
    return 2.0 * np.pi * np.asarray(kfrac, float) @ (crystal.Ai @ np.asarray(w, float))


def little_cogroup(crystal: Crystal, nk, k: int):
    return [o for o in range(len(crystal.ops)) if k_image(crystal, nk, o, k) == k]


def projective_rep(crystal: Crystal, iop: int, kfrac) -> np.ndarray:
    """D^k(alpha) = exp(i k . v(alpha)) O^k(alpha), Eq. (projrep)."""
    return np.exp(1j * k_dot(crystal, kfrac, crystal.ops[iop][1])) * orbital_rep(crystal, iop, kfrac)


def factor(crystal: Crystal, kfrac, ia: int, ib: int) -> complex:
    """lambda^k(alpha, beta) = exp{i k . [v(beta) - alpha v(beta)]}, Eq. (factor)."""
    Ra = crystal.ops[ia][0]
    vb = crystal.ops[ib][1]
    return np.exp(1j * k_dot(crystal, kfrac, vb - Ra @ vb))


def op_product(crystal: Crystal, ia: int, ib: int) -> int:
    P = crystal.ops[ia][0] @ crystal.ops[ib][0]
    for o, (R, _) in enumerate(crystal.ops):
        if np.allclose(R, P):
            return o
    raise ValueError("not closed")


def dirac_characters(crystal: Crystal, nk, k: int):
    """Omega_c = (n_c/h) sum_beta D(beta) D(gamma_c) D(beta)^{-1} over the little group, Eq. (dirac)."""
    kf = kgrid(nk)[k] / np.asarray(nk, float)
    G = little_cogroup(crystal, nk, k)
    D = {o: projective_rep(crystal, o, kf) for o in G}
    h = len(G)
    inv = {}
    for a in G:
        for b in G:
            if np.allclose(crystal.ops[a][0] @ crystal.ops[b][0], np.eye(3)):
                inv[a] = b
    seen, classes = set(), []
    for g in G:
        if g in seen:
            continue
        cl = sorted({op_product(crystal, op_product(crystal, b, g), inv[b]) for b in G})
        seen.update(cl)
        classes.append((g, cl))
    omegas = []
    for g, cl in classes:
        Om = sum(D[b] @ D[g] @ D[b].conj().T for b in G) * (len(cl) / h)
        omegas.append(Om)
    return omegas, D, G


def simultaneous_diagonalize(omegas, n: int, tol: float = 1e-8):
    """Common eigenvectors of commuting normal matrices by successive refinement (Sec. 3.4).

    Each relevant (non-zero) character contributes its Hermitian parts
    (Omega + Omega^dagger)/2 and (Omega - Omega^dagger)/(2i); every current
    block is split by the eigenvalue clusters of each part restricted to it.
    Returns U (columns grouped by block) and the block sizes.
    """
    blocks = [np.eye(n, dtype=np.complex128)]
    parts = []
    for Om in omegas:
        if np.abs(Om).max() < 1e-10:
            continue
        parts.append(0.5 * (Om + Om.conj().T))
        parts.append(0.5j * (Om.conj().T - Om))
    for H in parts:
        new = []
        for B in blocks:
            Hr = B.conj().T @ H @ B
            Hr = 0.5 * (Hr + Hr.conj().T)
            ev, Y = np.linalg.eigh(Hr)
            scale = max(1.0, np.abs(ev).max())
            start = 0
            for i in range(1, len(ev) + 1):
                if i == len(ev) or ev[i] - ev[i - 1] > tol * scale:
                    new.append(B @ Y[:, start:i])
                    start = i
        blocks = new
    U = np.hstack(blocks)
    return U, [b.shape[1] for b in blocks]
