"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module draws random numbers and shapes them into inputs; it computes no
step of the GW method.  To make the inputs of the symmetric workloads exactly
covariant it needs the action of the space-group operations on its own basis
functions, so it carries its own, independent description of that action
(atom permutation, lattice phase and real-spherical-harmonic rotation matrices
fitted at sample points).  The oracle and the library each derive the same
action from the crystal description in their own code; nothing is shared.

Conventions (the interface every side follows)
---------------------------------------------
* Conventional cubic lattice constant 1; FCC primitive vectors
  a1 = (0, 1/2, 1/2), a2 = (1/2, 0, 1/2), a3 = (1/2, 1/2, 0).
* k mesh: fractional (i1/n, i2/n, i3/n) in the reciprocal basis, flat index
  (i1 * n + i2) * n + i3.
* Basis order: atom, then shell (in the listed order), then m = -l..l.
  Real spherical harmonics: Y_{l0} = Y_l^0, Y_{l,m>0} = sqrt2 (-1)^m Re Y_l^m,
  Y_{l,m<0} = sqrt2 (-1)^m Im Y_l^{|m|} (Y_l^m with the Condon-Shortley phase);
  for l = 1 the order is (y, z, x).
* An operation {R|v} maps the function of atom x to the one at atom x' with
  R r_x + v = r_x' + T, and acts on Bloch sums with the phase exp(-i (R k).T).
* V(k1, k2) is [naux][nao][nao] with V^{k1,k2}_{Q,ij} = conj(V^{k2,k1}_{Q,ji}).

Value recipes
-------------
* no symmetry: H0^k = Q diag(eps) Q^dagger, Q Haar unitary, eps ~ U[-1, 1];
  S^k = I + 0.1 A / ||A||_2, A = B B^dagger, B complex Gaussian; V complex
  Gaussian / sqrt(naux), Hermitian paired.
* crystals: the same draws, group averaged (Reynolds projection over the point
  group, which is exact covariance), then H0 <- a H0 + b S so that the
  generalised spectrum of (H0, S) over the whole mesh spans exactly [-1, 1].
  V is drawn per orbit of momentum pairs under (point group) x (Hermitian
  swap): one Gaussian draw at the orbit's smallest pair, averaged over that
  pair's stabiliser, then carried to every pair of the orbit by the group
  action.  Every pair's value is therefore available on demand.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

from .configs import MASTER_SEED, Config

# --------------------------------------------------------------------------
# crystal and group
# --------------------------------------------------------------------------
FCC = 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]]).T  # columns a1 a2 a3


def _cubic_point_group():
    """The 48 signed permutation matrices (O_h), identity first."""
    ops = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            R = np.zeros((3, 3))
            for r, c in enumerate(perm):
                R[r, c] = signs[r]
            ops.append(R)
    ops.sort(key=lambda R: (not np.allclose(R, np.eye(3)),))
    return ops


def space_group(structure: str):
    """Coset representatives {R|v} of the space group (Cartesian R, v)."""
    oh = _cubic_point_group()
    if structure == "none":
        return [(np.eye(3), np.zeros(3))]
    if structure == "rocksalt":
        return [(R, np.zeros(3)) for R in oh]
    if structure == "diamond":
        # T_d: signed permutations with an even number of sign flips; the other
        # coset carries the fractional translation (1/4, 1/4, 1/4).
        td = [R for R in oh if int(np.sum(R < 0)) % 2 == 0]
        shift = np.full(3, 0.25)
        return [(R, np.zeros(3)) for R in td] + [(-R, shift.copy()) for R in td]
    raise ValueError(structure)


def atom_positions(structure: str):
    if structure == "rocksalt":
        return np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    if structure == "diamond":
        return np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]])
    return np.zeros((1, 3))


# --------------------------------------------------------------------------
# real spherical harmonics and their rotation matrices
# --------------------------------------------------------------------------
def _real_harmonics(l: int, xyz: np.ndarray) -> np.ndarray:
    from scipy.special import sph_harm_y

    r = np.linalg.norm(xyz, axis=1)
    theta = np.arccos(np.clip(xyz[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(xyz[:, 1], xyz[:, 0])
    out = np.empty((xyz.shape[0], 2 * l + 1))
    for m in range(-l, l + 1):
        if m == 0:
            out[:, l] = np.real(sph_harm_y(l, 0, theta, phi))
        elif m > 0:
            out[:, l + m] = np.sqrt(2.0) * (-1) ** m * np.real(sph_harm_y(l, m, theta, phi))
        else:
            out[:, l + m] = np.sqrt(2.0) * (-1) ** m * np.imag(sph_harm_y(l, -m, theta, phi))
    return out


_SAMPLE = np.random.default_rng(12345).normal(size=(64, 3))


@lru_cache(maxsize=None)
def _rot_matrix_cached(l: int, key: tuple) -> np.ndarray:
    R = np.array(key, dtype=np.float64).reshape(3, 3)
    A = _real_harmonics(l, _SAMPLE)
    B = _real_harmonics(l, _SAMPLE @ R)  # rows are R^{-1} u = R^T u
    D, *_ = np.linalg.lstsq(A, B, rcond=None)
    return D


def real_harmonic_rotation(l: int, R: np.ndarray) -> np.ndarray:
    """D with Y_lm(R^{-1} u) = sum_m' Y_lm'(u) D[m', m]."""
    return _rot_matrix_cached(l, tuple(np.round(R, 12).ravel()))


# --------------------------------------------------------------------------
# basis action on Bloch sums
# --------------------------------------------------------------------------
class _Action:
    """Action of each operation on one basis (orbital or auxiliary)."""

    def __init__(self, structure, shells, ops, lattice):
        self.pos = atom_positions(structure)
        self.nat = self.pos.shape[0]
        self.shells = list(shells)
        self.structure = structure
        self.ops = ops
        Ainv = np.linalg.inv(lattice)
        self.size_per_atom = sum(2 * l + 1 for l in self.shells) if structure != "none" else len(self.shells)
        self.n = self.nat * self.size_per_atom
        self.perm = []  # per op: atom -> atom'
        self.tvec = []  # per op: lattice translation (fractional integers) per atom
        for R, v in ops:
            perm, tv = [], []
            for x in range(self.nat):
                rp = R @ self.pos[x] + v
                for y in range(self.nat):
                    t = Ainv @ (rp - self.pos[y])
                    if np.allclose(t, np.round(t), atol=1e-9):
                        perm.append(y)
                        tv.append(np.round(t).astype(np.int64))
                        break
                else:
                    raise RuntimeError("operation does not map the crystal to itself")
            self.perm.append(perm)
            self.tvec.append(tv)
        off, o = [], 0
        for l in self.shells:
            off.append(o)
            o += 2 * l + 1 if structure != "none" else 1
        self.shell_off = off

    def dense(self, iop: int, kfrac_rot: np.ndarray) -> np.ndarray:
        """The n x n matrix of operation iop on Bloch sums whose rotated momentum is kfrac_rot."""
        n = self.n
        if self.structure == "none":
            return np.eye(n, dtype=np.complex128)
        O = np.zeros((n, n), dtype=np.complex128)
        R = self.ops[iop][0]
        for x in range(self.nat):
            xp = self.perm[iop][x]
            phase = np.exp(-2j * np.pi * float(kfrac_rot @ self.tvec[iop][x]))
            for s, l in enumerate(self.shells):
                D = real_harmonic_rotation(l, R)
                src = x * self.size_per_atom + self.shell_off[s]
                dst = xp * self.size_per_atom + self.shell_off[s]
                O[dst:dst + 2 * l + 1, src:src + 2 * l + 1] = phase * D
        return O

    def apply(self, iop: int, kfrac_rot: np.ndarray, X: np.ndarray, axis: int, conj: bool = False):
        """Return O X along ``axis`` (O of op iop at a k whose rotated image is kfrac_rot).

        With conj=True the conjugate matrix conj(O) is applied instead.
        """
        if self.structure == "none":
            return X.copy()
        O = self.dense(iop, kfrac_rot)
        if conj:
            O = O.conj()
        return np.moveaxis(np.tensordot(O, X, axes=(1, axis)), 0, axis)


class Mesh:
    def __init__(self, nk, lattice, ops):
        self.nk = tuple(int(n) for n in nk)
        self.N = self.nk[0] * self.nk[1] * self.nk[2]
        idx = np.array(list(itertools.product(range(self.nk[0]), range(self.nk[1]), range(self.nk[2]))))
        self.ivec = idx
        self.frac = idx / np.array(self.nk, dtype=np.float64)
        Ainv = np.linalg.inv(lattice)
        self.rotk = []  # per op: integer matrix acting on fractional k
        self.image = []  # per op: k -> index of R k
        for R, _ in ops:
            M = lattice.T @ R @ Ainv.T
            Mi = np.round(M).astype(np.int64)
            assert np.allclose(M, Mi, atol=1e-9)
            self.rotk.append(Mi)
            img = []
            for k in range(self.N):
                kk = Mi @ self.ivec[k]
                img.append(self.index(kk))
            self.image.append(np.array(img))

    def index(self, iv) -> int:
        n = self.nk
        return int(((iv[0] % n[0]) * n[1] + (iv[1] % n[1])) * n[2] + (iv[2] % n[2]))

    def rotated_frac(self, iop, k) -> np.ndarray:
        return (self.rotk[iop] @ self.ivec[k]) / np.array(self.nk, dtype=np.float64)

    def add(self, a, b):
        return self.index(self.ivec[a] + self.ivec[b])

    def sub(self, a, b):
        return self.index(self.ivec[a] - self.ivec[b])


# --------------------------------------------------------------------------
# the system
# --------------------------------------------------------------------------
def _rng(cfg: Config, *path) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([MASTER_SEED, cfg.index, *path]))


def _haar(rng, n):
    Z = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def _cgauss(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)


class System:
    """All inputs of one workload: H0, S and V(k1, k2) on demand.

    ``device`` (a torch device) moves the two-body work (group averaging and rotation of V) to
    PyTorch on that device; V(k1, k2) then returns torch tensors there.  The random draws are the
    same numpy draws either way; only the rounding of the averaging differs between backends, so
    one System instance must feed both sides of a comparison.
    """

    def __init__(self, cfg: Config, device=None):
        self.cfg = cfg
        self.device = device
        self.ops = space_group(cfg.structure)
        self.lattice = FCC if cfg.structure != "none" else np.eye(3)
        self.mesh = Mesh(cfg.nk, self.lattice, self.ops)
        self.ao = _Action(cfg.structure, cfg.ao_shells, self.ops, self.lattice)
        self.aux = _Action(cfg.structure, cfg.aux_shells, self.ops, self.lattice)
        self.nao, self.naux, self.Nk = cfg.nao, cfg.naux, self.mesh.N
        assert self.ao.n == self.nao and self.aux.n == self.naux
        self._make_one_body()
        self._vcache = {}
        self._stab = {}

    # ---- one-body ----------------------------------------------------------
    def _reynolds_matrices(self, X):
        """(1/|G|) sum_alpha O^k(alpha) X^k O^k(alpha)^dagger, placed at alpha k."""
        out = np.zeros_like(X)
        for iop in range(len(self.ops)):
            for k in range(self.Nk):
                kr = self.mesh.rotated_frac(iop, k)
                Y = self.ao.apply(iop, kr, X[k], 0)
                Y = self.ao.apply(iop, kr, Y, 1, conj=True)
                out[self.mesh.image[iop][k]] += Y
        return out / len(self.ops)

    def _make_one_body(self):
        cfg, nao, Nk = self.cfg, self.nao, self.Nk
        rng = _rng(cfg, 1)
        H = np.empty((Nk, nao, nao), dtype=np.complex128)
        A = np.empty_like(H)
        for k in range(Nk):
            Q = _haar(rng, nao)
            eps = rng.uniform(-1.0, 1.0, size=nao)
            H[k] = (Q * eps[None, :]) @ Q.conj().T
            B = _cgauss(rng, (nao, nao))
            A[k] = B @ B.conj().T
        if cfg.structure == "none":
            for k in range(Nk):
                A[k] /= np.linalg.norm(A[k], 2)
            self.S = np.eye(nao)[None] + 0.1 * A
            self.H0 = 0.5 * (H + H.conj().transpose(0, 2, 1))
            return
        H = self._reynolds_matrices(H)
        A = self._reynolds_matrices(A)
        A /= max(np.linalg.norm(A[k], 2) for k in range(Nk))
        S = np.eye(nao)[None] + 0.1 * A
        S = 0.5 * (S + S.conj().transpose(0, 2, 1))
        H = 0.5 * (H + H.conj().transpose(0, 2, 1))
        ev = []
        for k in range(Nk):
            L = np.linalg.cholesky(S[k])
            Li = np.linalg.inv(L)
            ev.append(np.linalg.eigvalsh(Li @ H[k] @ Li.conj().T))
        ev = np.concatenate(ev)
        a = 2.0 / (ev.max() - ev.min())
        b = -1.0 - a * ev.min()
        self.H0 = a * H + b * S
        self.S = S

    # ---- two-body ---------------------------------------------------------
    def _mat(self, O):
        if self.device is None:
            return O
        import torch

        return torch.from_numpy(O).to(self.device)

    def _act_pair(self, iop, swap, k1, k2, X):
        """Apply (alpha, swap) to V^{k1,k2}; return (new pair, tensor).

        V'(Q) = sum_Q' O_aux^q(alpha)[Q, Q'] O^{k1}(alpha) V(Q') O^{k2}(alpha)^dagger.
        """
        q = self.mesh.sub(k2, k1)
        a, b = self.mesh.image[iop][k1], self.mesh.image[iop][k2]
        if self.cfg.structure != "none":
            Oq = self._mat(self.aux.dense(iop, self.mesh.rotated_frac(iop, q)))
            O1 = self._mat(self.ao.dense(iop, self.mesh.rotated_frac(iop, k1)))
            O2 = self._mat(self.ao.dense(iop, self.mesh.rotated_frac(iop, k2)))
            naux, nao = self.naux, self.nao
            X = (Oq @ X.reshape(naux, nao * nao)).reshape(naux, nao, nao)
            X = O1 @ X @ O2.conj().T
        if swap:
            if self.device is not None:
                return (b, a), X.transpose(-1, -2).conj_physical().contiguous()
            return (b, a), np.conj(X).transpose(0, 2, 1)
        return (a, b), X

    def _canonical(self, k1, k2):
        """Smallest pair of the orbit, and one (op, swap) that maps (k1, k2) onto it."""
        best = None
        for iop in range(len(self.ops)):
            a, b = self.mesh.image[iop][k1], self.mesh.image[iop][k2]
            for swap in (0, 1):
                p = (b, a) if swap else (a, b)
                key = p[0] * self.Nk + p[1]
                if best is None or key < best[0]:
                    best = (key, p, iop, swap)
        return best[1], best[2], best[3]

    def _inverse_op(self, iop):
        R = self.ops[iop][0]
        Ri = R.T
        for j, (Rj, _) in enumerate(self.ops):
            if np.allclose(Rj, Ri):
                return j
        raise RuntimeError("group not closed")

    def _rep_value(self, p):
        if p in self._vcache:
            return self._vcache[p]
        cfg = self.cfg
        rng = _rng(cfg, 2, p[0], p[1])
        # optional coupling scale of the workload (cfg.extra["vscale"], default 1)
        X = _cgauss(rng, (self.naux, self.nao, self.nao)) * (cfg.extra.get("vscale", 1.0) / np.sqrt(self.naux))
        if self.device is not None:
            import torch

            X = torch.from_numpy(X).to(self.device)
            acc = torch.zeros_like(X)
        else:
            acc = np.zeros_like(X)
        n = 0
        for iop in range(len(self.ops)):
            a, b = self.mesh.image[iop][p[0]], self.mesh.image[iop][p[1]]
            for swap in (0, 1):
                # only the stabiliser of the pair contributes: skip the action of the other operations
                if ((b, a) if swap else (a, b)) != p:
                    continue
                q, Y = self._act_pair(iop, swap, p[0], p[1], X)
                acc += Y
                n += 1
        V = acc / n
        self._vcache[p] = V
        return V

    def V(self, k1, k2):
        p, iop, swap = self._canonical(k1, k2)
        Vp = self._rep_value(p)
        # (iop, swap) maps (k1,k2) onto p; the inverse maps p back to (k1,k2).
        pair, X = self._act_pair(self._inverse_op(iop), swap, p[0], p[1], Vp)
        assert pair == (k1, k2), (pair, (k1, k2))
        if self.device is not None:
            return X.resolve_conj().contiguous()
        return np.ascontiguousarray(X)

    def V_full(self):
        """Dense [Nk][Nk][naux][nao][nao] numpy array (small workloads only)."""
        out = np.empty((self.Nk, self.Nk, self.naux, self.nao, self.nao), dtype=np.complex128)
        for k1 in range(self.Nk):
            for k2 in range(self.Nk):
                v = self.V(k1, k2)
                out[k1, k2] = v if self.device is None else v.cpu().numpy()
        return out


@lru_cache(maxsize=4)
def system(name: str) -> System:
    from .configs import get

    return System(get(name))
