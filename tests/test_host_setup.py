"""Host-side set-up of the library (no GPU): transform matrices and space-group analysis.

* The tau grid and the four Matsubara maps the library builds agree with the
  oracle's independent construction.
* The wedge sizes of the library's star analysis equal the printed n_ik column
  of Table 2 (tests/golden/table2_wedge_sizes.json).
* Block sizes at Gamma follow the textbook decomposition of the orbital
  representation (e.g. O_h: s -> A1g, p -> T1u, d -> Eg + T2g) and every
  partition covers the basis.
* Every workload's Matsubara sets are sorted and mirror-symmetric (the Hermitian shortcuts and the
  half-frequency W solve depend on it).
* The irrep dimension of every block, from the Dirac-character eigenvalues, equals the eigenvalue
  multiplicity of a group-averaged random operator on the oracle's block.
* In the partner-adapted bases every invariant operator is I_d (x) A on each block.
"""
import json
import os

import numpy as np
import pytest

from oracle import grid

HERE = os.path.dirname(os.path.abspath(__file__))


def _lib():
    from paper_2405_09494_gb300 import build, sgw

    if not os.path.exists(sgw.LIB_PATH):
        try:
            build.build()
        except RuntimeError as e:
            pytest.skip(str(e))
    return sgw


@pytest.mark.parametrize("name", ["c1", "c2", "t1"])
def test_library_grid_matches_oracle(name):
    sgw = _lib()
    from paper_2405_09494_gb300 import configs

    cfg = configs.get(name)
    tau, TF, TFb, TB, TBb = sgw.sgw_host_grid(cfg.nk, cfg.nao, cfg.naux, cfg.ntau, cfg.mats_f, cfg.mats_b, cfg.beta)
    oTF = grid.forward_map(cfg.mats_f, cfg.beta, cfg.ntau, "F")
    oTB = grid.forward_map(cfg.mats_b, cfg.beta, cfg.ntau, "B")

    def rel(a, b):
        return np.abs(a - b).max() / np.abs(b).max()

    assert np.abs(tau - grid.tau_nodes(cfg.beta, cfg.ntau)).max() < 1e-12
    assert rel(TF, oTF) < 1e-12 and rel(TB, oTB) < 1e-12
    assert rel(TFb, grid.backward_map(oTF)) < 1e-11 and rel(TBb, grid.backward_map(oTB)) < 1e-11


def _groups():
    from paper_2405_09494_gb300 import synth

    oh = synth.space_group("rocksalt")
    td = [(R, v) for R, v in oh if int(np.sum(R < 0)) % 2 == 0]
    return {"O_h": (oh, synth.atom_positions("rocksalt")), "T_d": (td, synth.atom_positions("diamond")),
            "Fd-3m": (synth.space_group("diamond"), synth.atom_positions("diamond"))}


def _analyse(ops, pos, n, aos, axs):
    sgw = _lib()
    from paper_2405_09494_gb300 import synth

    rot = np.stack([R for R, _ in ops])
    tra = np.stack([v for _, v in ops])
    nao = len(pos) * sum(2 * l + 1 for l in aos)
    naux = len(pos) * sum(2 * l + 1 for l in axs)
    return sgw.sgw_host_symmetry((n, n, n), nao, naux, synth.FCC, pos, rot, tra, aos, axs), nao, naux


def test_wedge_sizes_match_table2():
    gold = json.load(open(os.path.join(HERE, "golden", "table2_wedge_sizes.json")))
    groups = _groups()
    for gname in ("O_h", "T_d"):
        ops, pos = groups[gname]
        for n, expect in gold[gname].items():
            (nw, rep, _, _), _, _ = _analyse(ops, pos, int(n), (0,), (0,))
            assert nw == expect, (gname, n, nw)
    # the non-symmorphic diamond group has the same point group as O_h
    ops, pos = groups["Fd-3m"]
    for n, expect in gold["O_h"].items():
        (nw, _, _, _), _, _ = _analyse(ops, pos, int(n), (0,), (0,))
        assert nw == expect


def test_gamma_blocks_follow_the_irreducible_decomposition():
    ops, pos = _groups()["O_h"]
    (nw, rep, ao, ax), nao, naux = _analyse(ops, pos, 3, (0, 1, 2), (0, 1, 2, 3))
    # O_h on two O_h sites: s -> A1g (2), p -> T1u (2 x 3), d -> Eg (2 x 2) + T2g (2 x 3)
    assert sorted(ao[0]) == [2, 4, 6, 6]
    # aux adds f -> A2u + T1u + T2u: T1u gathers p and f copies (12)
    assert sorted(ax[0]) == [2, 2, 4, 6, 6, 12]
    ops, pos = _groups()["T_d"]
    (nw, rep, ao, ax), nao, naux = _analyse(ops, pos, 2, (0, 1, 2), (0,))
    # T_d: s -> A1 (2), p -> T2 (2 x 3), d -> E (2 x 2) + T2 (2 x 3)
    assert sorted(ao[0]) == [2, 4, 12]
    for g in ("O_h", "T_d", "Fd-3m"):
        ops, pos = _groups()[g]
        (nw, rep, ao, ax), nao, naux = _analyse(ops, pos, 4, (0, 1, 2), (0, 1, 2, 3, 4))
        assert all(sum(b) == nao for b in ao) and all(sum(b) == naux for b in ax)
        assert rep.min() == 0 and rep.max() == nw - 1


@pytest.mark.parametrize("structure", ["rocksalt", "diamond"])
def test_library_blocks_match_the_oracle_simultaneous_diagonalisation(structure):
    """Irrep block sizes are unique up to order: the library's (one Hermitian combination of the
    Dirac characters) and the oracle's (successive refinement) must agree at every wedge point."""
    from oracle import symmetry as sy
    from paper_2405_09494_gb300 import synth

    ops = synth.space_group(structure)
    pos = synth.atom_positions(structure)
    aos, axs = (0, 1, 2), (0, 1, 2, 3, 4)
    (nw, rep, ao, ax), nao, naux = _analyse(ops, pos, 4, aos, axs)
    for shells, lib_blocks in ((aos, ao), (axs, ax)):
        cr = sy.Crystal(synth.FCC, pos, ops, shells)
        reps, orep = sy.stars(cr, (4, 4, 4))
        assert len(reps) == nw and np.array_equal(orep, rep)
        for w, k in enumerate(reps):
            omegas, _, _ = sy.dirac_characters(cr, (4, 4, 4), k)
            _, sizes = sy.simultaneous_diagonalize(omegas, cr.n)
            assert sorted(sizes) == sorted(lib_blocks[w]), (structure, w, sizes, lib_blocks[w])


def test_largest_workload_grid_is_closed_and_well_conditioned():
    """c5 (200 tau, beta 500): both index sets are closed under w -> -w (so the Hermitian Gram
    shortcuts apply), the library's maps are well conditioned and invert, and sampled rows of
    the fermionic map agree with the oracle's quadrature."""
    sgw = _lib()
    from paper_2405_09494_gb300 import configs

    cfg = configs.get("c5")
    assert all(-n - 1 in cfg.mats_f for n in cfg.mats_f) and all(-n in cfg.mats_b for n in cfg.mats_b)
    tau, TF, TFb, TB, TBb = sgw.sgw_host_grid(cfg.nk, cfg.nao, cfg.naux, cfg.ntau, cfg.mats_f, cfg.mats_b, cfg.beta)
    assert np.linalg.cond(TF) < 2e3 and np.linalg.cond(TB) < 2e3
    assert np.abs(TFb @ TF - np.eye(cfg.ntau)).max() < 1e-11
    assert np.abs(TBb @ TB - np.eye(cfg.ntau)).max() < 1e-11
    rows = [0, 57, 100, 199]
    oTF = grid.forward_map([cfg.mats_f[i] for i in rows], cfg.beta, cfg.ntau, "F")
    assert np.abs(oTF - TF[rows]).max() < 1e-12 * np.abs(TF).max()


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4", "c5", "c3s", "t1"])
def test_every_workload_frequency_set_is_sorted_and_mirror_symmetric(name):
    """Each workload's Matsubara sets hold at least n_tau indices, ascend strictly, and are closed under
    w -> -w with mirrored positions: fermionic index m and -m - 1 at positions i and n_w - 1 - i,
    bosonic m and -m likewise (0 in the middle).  The Hermitian Gram stages need the closure.  The
    W solve over the non-negative bosonic frequencies, whose other half are adjoints, needs the
    bosonic order."""
    from paper_2405_09494_gb300 import configs

    cfg = configs.get(name)
    mf, mb = list(cfg.mats_f), list(cfg.mats_b)
    assert len(mf) >= cfg.ntau and len(mb) >= cfg.ntau
    assert all(a < b for a, b in zip(mf, mf[1:])) and all(a < b for a, b in zip(mb, mb[1:]))
    assert all(mf[len(mf) - 1 - i] == -mf[i] - 1 for i in range(len(mf)))
    assert all(mb[len(mb) - 1 - i] == -mb[i] for i in range(len(mb)))
    assert 0 in mb


@pytest.mark.parametrize("structure", ["rocksalt", "diamond"])
def test_library_irrep_dims_match_the_multiplicity_of_an_invariant_operator(structure):
    """The library's irrep dimension d of every block comes from its Dirac-character eigenvalues.
    Two things must hold at every wedge point of the 4x4x4 mesh.  d divides the block size.  And,
    matched by block size, d equals the eigenvalue multiplicity of a random Hermitian operator
    averaged over the little group and restricted to the oracle's block.  By Schur's lemma that
    operator is I_d (x) A on the block's d copies."""
    sgw = _lib()
    from oracle import symmetry as sy
    from paper_2405_09494_gb300 import synth

    ops = synth.space_group(structure)
    pos = synth.atom_positions(structure)
    aos, axs = (0, 1, 2), (0, 1, 2, 3, 4)
    rot = np.stack([R for R, _ in ops])
    tra = np.stack([v for _, v in ops])
    nao = len(pos) * sum(2 * l + 1 for l in aos)
    naux = len(pos) * sum(2 * l + 1 for l in axs)
    nw, _, ao, ax = sgw.sgw_host_symmetry((4, 4, 4), nao, naux, synth.FCC, pos, rot, tra, aos, axs)
    dao, dax = sgw.sgw_host_irrep_dims((4, 4, 4), nao, naux, synth.FCC, pos, rot, tra, aos, axs)
    assert len(dao) == len(dax) == nw
    rng = np.random.default_rng(5)
    for shells, lib_sizes, lib_dims in ((aos, ao, dao), (axs, ax, dax)):
        cr = sy.Crystal(synth.FCC, pos, ops, shells)
        reps, _ = sy.stars(cr, (4, 4, 4))
        for w, k in enumerate(reps):
            assert len(lib_dims[w]) == len(lib_sizes[w]), (structure, w)
            assert all(d > 0 and s % d == 0 for s, d in zip(lib_sizes[w], lib_dims[w])), (structure, w)
            omegas, D, G = sy.dirac_characters(cr, (4, 4, 4), k)
            U, sizes = sy.simultaneous_diagonalize(omegas, cr.n)
            R = rng.standard_normal((cr.n, cr.n)) + 1j * rng.standard_normal((cr.n, cr.n))
            R = R + R.conj().T
            H = sum(D[g] @ R @ D[g].conj().T for g in G) / len(G)
            pairs, st = [], 0
            for sz in sizes:
                B = U[:, st:st + sz]
                ev = np.linalg.eigvalsh(B.conj().T @ H @ B)
                distinct = 1 + int(np.sum(np.diff(ev) > 1e-8 * max(1.0, np.abs(ev).max())))
                pairs.append((sz, sz // distinct))
                st += sz
            assert sorted(pairs) == sorted(zip(lib_sizes[w], lib_dims[w])), (structure, w, pairs)


@pytest.mark.parametrize("structure", ["rocksalt", "diamond"])
def test_partner_basis_puts_invariant_operators_in_identical_copies(structure):
    """The partner-adapted bases (sgw_host_partner_basis) at every wedge point of a 4x4x4 mesh, for
    both families, are unitary.  In them, an operator commuting with the oracle's projective
    representation of the little group (a group-averaged random Hermitian operator) is block
    diagonal over the library's blocks.  On a block of irrep dimension d and multiplicity m it reads
    I_d (x) A: the d diagonal m x m blocks are equal, the rest vanish (Schur's lemma)."""
    sgw = _lib()
    from oracle import symmetry as sy
    from paper_2405_09494_gb300 import synth

    ops = synth.space_group(structure)
    pos = synth.atom_positions(structure)
    aos, axs = (0, 1, 2), (0, 1, 2, 3, 4)
    rot = np.stack([R for R, _ in ops])
    tra = np.stack([v for _, v in ops])
    nao = len(pos) * sum(2 * l + 1 for l in aos)
    naux = len(pos) * sum(2 * l + 1 for l in axs)
    args = ((4, 4, 4), nao, naux, synth.FCC, pos, rot, tra, aos, axs)
    _, _, ao, ax = sgw.sgw_host_symmetry(*args)
    dao, dax = sgw.sgw_host_irrep_dims(*args)
    rng = np.random.default_rng(9)
    for fam, shells, sizes, dims in ((0, aos, ao, dao), (1, axs, ax, dax)):
        U = sgw.sgw_host_partner_basis(*args, fam)
        cr = sy.Crystal(synth.FCC, pos, ops, shells)
        reps, _ = sy.stars(cr, (4, 4, 4))
        assert U.shape[0] == len(reps)
        for w, k in enumerate(reps):
            n = cr.n
            assert np.abs(U[w].conj().T @ U[w] - np.eye(n)).max() < 1e-12, (structure, fam, w)
            _, D, G = sy.dirac_characters(cr, (4, 4, 4), k)
            R = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
            H = sum(D[g] @ (R + R.conj().T) @ D[g].conj().T for g in G) / len(G)
            X = U[w].conj().T @ H @ U[w]
            scale = np.abs(X).max()
            st = 0
            for sz, d in zip(sizes[w], dims[w]):
                m = sz // d
                assert np.abs(X[st:st + sz, st + sz:]).max(initial=0.0) < 1e-11 * scale
                B = X[st:st + sz, st:st + sz]
                for i in range(d):
                    for j in range(d):
                        ref = B[:m, :m] if i == j else 0.0
                        err = np.abs(B[i * m:(i + 1) * m, j * m:(j + 1) * m] - ref).max()
                        assert err < 1e-11 * scale, (structure, fam, w, sz, d, i, j, err / scale)
                st += sz
