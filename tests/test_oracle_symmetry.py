"""Pins of the oracle's space-group code (Sec. 3, Algorithm 1) and of the symmetric inputs.

Expected values come from closed forms (the l = 1 harmonics are the
coordinates), group axioms (homomorphism, cocycle), the printed Table 2 wedge
sizes, Schur's lemma (commutant dimension) and the covariance that the
synthetic generator promises, checked with the oracle's independently built
representation matrices.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import symmetry as sy

HERE = os.path.dirname(os.path.abspath(__file__))


def _crystal(structure, shells):
    from paper_2405_09494_gb300 import synth

    return sy.Crystal(synth.FCC, synth.atom_positions(structure), synth.space_group(structure), shells)


def _td(shells):
    from paper_2405_09494_gb300 import synth

    ops = [(R, v) for R, v in synth.space_group("rocksalt") if int(np.sum(R < 0)) % 2 == 0]
    return sy.Crystal(synth.FCC, synth.atom_positions("diamond"), ops, shells)


def _rotations(n=12, seed=0):
    rs = Rotation.random(n, random_state=seed).as_matrix()
    return [R if i % 2 == 0 else -R for i, R in enumerate(rs)]


def test_l1_rotation_matrix_is_the_permuted_rotation():
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], float)  # (x, y, z) -> (y, z, x)
    for R in _rotations():
        np.testing.assert_allclose(sy.harmonic_rotation(1, R), P @ R @ P.T, atol=1e-13)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_rotation_matrices_form_an_orthogonal_representation(l):
    Rs = _rotations(8, seed=l)
    for a in Rs[:4]:
        for b in Rs[4:]:
            np.testing.assert_allclose(sy.harmonic_rotation(l, a @ b),
                                       sy.harmonic_rotation(l, a) @ sy.harmonic_rotation(l, b), atol=1e-12)
        D = sy.harmonic_rotation(l, a)
        np.testing.assert_allclose(D @ D.T, np.eye(2 * l + 1), atol=1e-12)


def test_wedge_sizes_match_table2():
    gold = json.load(open(os.path.join(HERE, "golden", "table2_wedge_sizes.json")))
    oh = _crystal("rocksalt", [0])
    td = _td([0])
    for n, expect in gold["O_h"].items():
        assert len(sy.stars(oh, (int(n),) * 3)[0]) == expect
    for n, expect in gold["T_d"].items():
        assert len(sy.stars(td, (int(n),) * 3)[0]) == expect


@pytest.mark.parametrize("structure", ["diamond", "rocksalt"])
def test_projective_rule_and_cocycle(structure):
    cr = _crystal(structure, [0, 1, 2])
    nk = (4, 4, 4)
    reps, _ = sy.stars(cr, nk)
    worst_rule, worst_cocycle, max_dev_from_one = 0.0, 0.0, 0.0
    for k in reps:
        kf = sy.kgrid(nk)[k] / 4.0
        G = sy.little_cogroup(cr, nk, k)
        D = {o: sy.projective_rep(cr, o, kf) for o in G}
        for a in G:
            for b in G:
                ab = sy.op_product(cr, a, b)
                lam = sy.factor(cr, kf, a, b)
                max_dev_from_one = max(max_dev_from_one, abs(lam - 1))
                worst_rule = max(worst_rule, np.abs(D[a] @ D[b] - lam * D[ab]).max())
        for a in G[:6]:
            for b in G[:6]:
                for c in G[:6]:
                    lhs = sy.factor(cr, kf, a, sy.op_product(cr, b, c)) * sy.factor(cr, kf, b, c)
                    rhs = sy.factor(cr, kf, sy.op_product(cr, a, b), c) * sy.factor(cr, kf, a, b)
                    worst_cocycle = max(worst_cocycle, abs(lhs - rhs))
    assert worst_rule < 1e-12 and worst_cocycle < 1e-12
    if structure == "rocksalt":
        assert max_dev_from_one < 1e-12  # symmorphic: lambda = 1 (Sec. 3.3)
    else:
        assert max_dev_from_one > 0.5  # non-symmorphic: a genuine factor system at the zone boundary


def test_dirac_characters_commute_and_blocks_are_irreducible_sums():
    cr = _crystal("diamond", [0, 1, 2])
    nk = (4, 4, 4)
    reps, _ = sy.stars(cr, nk)
    for k in reps:
        omegas, D, G = sy.dirac_characters(cr, nk, k)
        for Om in omegas:
            for g in G:
                assert np.abs(Om @ D[g] - D[g] @ Om).max() < 1e-11
            for Om2 in omegas:
                assert np.abs(Om @ Om2 - Om2 @ Om).max() < 1e-11
        U, sizes = sy.simultaneous_diagonalize(omegas, cr.n)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(cr.n), atol=1e-11)
        edges = np.cumsum([0] + sizes)
        mask = np.zeros((cr.n, cr.n), bool)
        for a, b in zip(edges[:-1], edges[1:]):
            mask[a:b, a:b] = True
        comm_dim = 0
        for g in G:
            Db = U.conj().T @ D[g] @ U
            assert np.abs(Db[~mask]).max() < 1e-10
        # Schur: sum over blocks of m_i^2 equals (1/h) sum_g |Tr D(g)|^2
        h = len(G)
        chi2 = sum(abs(np.trace(D[g])) ** 2 for g in G) / h
        for a, b in zip(edges[:-1], edges[1:]):
            blocks = [(U.conj().T @ D[g] @ U)[a:b, a:b] for g in G]
            n = b - a
            rows = [np.kron(np.eye(n), Dg.T) - np.kron(Dg, np.eye(n)) for Dg in blocks]
            M = np.vstack(rows)
            s = np.linalg.svd(M, compute_uv=False)
            comm_dim += int(np.sum(s < 1e-9 * max(1.0, s.max())))
        assert comm_dim == int(round(chi2))


def test_synthetic_inputs_are_covariant_under_the_oracle_representation():
    from paper_2405_09494_gb300 import configs, synth

    for name in ("t1",):
        cfg = configs.get(name)
        sysm = synth.System(cfg)
        ao = sy.Crystal(synth.FCC, synth.atom_positions(cfg.structure), synth.space_group(cfg.structure), cfg.ao_shells)
        aux = sy.Crystal(synth.FCC, synth.atom_positions(cfg.structure), synth.space_group(cfg.structure),
                         cfg.aux_shells)
        kg = sy.kgrid(cfg.nk) / np.asarray(cfg.nk, float)
        for o in range(len(ao.ops)):
            for k in range(cfg.nkpts):
                O = sy.orbital_rep(ao, o, kg[k])
                kk = sy.k_image(ao, cfg.nk, o, k)
                assert np.abs(O @ sysm.H0[k] @ O.conj().T - sysm.H0[kk]).max() < 1e-12
                assert np.abs(O @ sysm.S[k] @ O.conj().T - sysm.S[kk]).max() < 1e-12
        from oracle import gw

        for o in (3, 17, 40):
            for k1, k2 in ((0, 3), (5, 6), (7, 7)):
                q = gw.ksub(cfg.nk, k2, k1)
                Oq = sy.orbital_rep(aux, o, kg[q])
                O1 = sy.orbital_rep(ao, o, kg[k1])
                O2 = sy.orbital_rep(ao, o, kg[k2])
                V = sysm.V(k1, k2)
                rot = np.einsum("PQ,ia,Qab,jb->Pij", Oq, O1, V, O2.conj())
                a, b = sy.k_image(ao, cfg.nk, o, k1), sy.k_image(ao, cfg.nk, o, k2)
                assert np.abs(rot - sysm.V(a, b)).max() < 1e-12


@pytest.mark.parametrize("name", ["t1", "c1"])
def test_synthetic_inputs_are_seeded_hermitian_and_paired(name):
    """The input generator's promises that the method relies on: two instances draw the same inputs;
    H0 and S are Hermitian, and S is positive definite; and V^{k2,k1}_Q = (V^{k1,k2}_Q)^dagger for
    every Q.  That pairing is what makes P0^q(tau) = P0^{-q}(beta - tau)^T, the relation the tau
    reflection uses."""
    from paper_2405_09494_gb300 import configs, synth

    cfg = configs.get(name)
    a, b = synth.System(cfg), synth.System(cfg)
    assert np.array_equal(a.H0, b.H0) and np.array_equal(a.S, b.S)
    for k in range(cfg.nkpts):
        assert np.abs(a.H0[k] - a.H0[k].conj().T).max() < 1e-14
        assert np.abs(a.S[k] - a.S[k].conj().T).max() < 1e-14
        assert np.linalg.eigvalsh(a.S[k]).min() > 0
    for k1, k2 in ((0, 1), (2, 5), (3, 3), (7, 4)):
        V12, V21 = a.V(k1, k2), a.V(k2, k1)
        assert np.array_equal(V12, b.V(k1, k2))
        assert np.abs(V21 - V12.conj().transpose(0, 2, 1)).max() < 1e-13 * np.abs(V12).max()


def test_oracle_self_energy_and_polarization_are_equivariant():
    """Sigma^{alpha k} = O Sigma^k O^dagger and P0^{alpha q} = O_aux P0^q O_aux^dagger (Eqs. (mat_rot), (prot))."""
    from oracle import grid, gw
    from paper_2405_09494_gb300 import configs, synth

    cfg = configs.get("t1")
    sysm = synth.System(cfg)
    V = sysm.V_full()
    tau = grid.tau_nodes(cfg.beta, cfg.ntau)
    TB = grid.forward_map(cfg.mats_b, cfg.beta, cfg.ntau, "B")
    mu = gw.mu_noninteracting(sysm.H0, sysm.S, cfg.beta, cfg.n_elec)
    G = gw.g0_tau(sysm.H0, sysm.S, mu, cfg.beta, tau)
    P0 = gw.polarization(G, V, cfg.nk)
    P, _, _ = gw.screened_interaction(P0, TB, grid.backward_map(TB))
    Sig = gw.self_energy(G, P, V, cfg.nk)
    ao = sy.Crystal(synth.FCC, synth.atom_positions(cfg.structure), synth.space_group(cfg.structure), cfg.ao_shells)
    aux = sy.Crystal(synth.FCC, synth.atom_positions(cfg.structure), synth.space_group(cfg.structure), cfg.aux_shells)
    kg = sy.kgrid(cfg.nk) / np.asarray(cfg.nk, float)
    for o in (1, 9, 30, 47):
        for k in range(cfg.nkpts):
            kk = sy.k_image(ao, cfg.nk, o, k)
            O = sy.orbital_rep(ao, o, kg[k])
            Oa = sy.orbital_rep(aux, o, kg[k])
            assert np.abs(np.einsum("ia,tab,jb->tij", O, Sig[k], O.conj()) - Sig[kk]).max() < 1e-11
            assert np.abs(np.einsum("ia,tab,jb->tij", Oa, P0[k], Oa.conj()) - P0[kk]).max() < 1e-11
