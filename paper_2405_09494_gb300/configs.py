"""Workload definitions: seeded synthetic systems shaped like the paper's solids.

Each entry fixes the sizes, the crystal, the tau grid and the finite Matsubara
index sets.  The index sets are plain input data (integers); the oracle and the
library each build their own transform matrices from them.  They were chosen
by the oracle's offline greedy volume search (``python -m oracle.choose_matsubara``)
so that the Chebyshev-node -> Matsubara map is well conditioned (cond 36 at
n_tau = 20, 140 at n_tau = 50).

Shell lists per atom (angular momenta) give the totals of the workloads:
rocksalt / diamond cells with two atoms, nao = 2 * sum(2l+1) over the shells.
"""
from __future__ import annotations

from dataclasses import dataclass, field

MASTER_SEED = 2405094940

F20 = [-24, -13, -9, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 8, 12, 23]
B20 = [-32, -15, -9, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 9, 15, 32]
F50 = [-136, -69, -46, -35, -28, -24, -21, -19, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7,
       -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 18, 20, 23,
       27, 34, 45, 68, 135]
B50 = [-196, -91, -54, -38, -30, -25, -21, -19, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7,
       -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 19, 21,
       25, 30, 38, 54, 91, 196]
F16 = [-15, -8, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 7, 14]
B16 = [-21, -10, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 10, 21]


@dataclass
class Config:
    name: str
    index: int
    structure: str  # "none" | "rocksalt" | "diamond"
    nk: tuple
    ao_shells: tuple  # angular momenta per atom ("none": nao s-like functions)
    aux_shells: tuple
    ntau: int
    beta: float
    mats_f: list
    mats_b: list
    spin: int = 2
    loop_sign: int = 1
    damping: float = 1.0
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nao(self) -> int:
        if self.structure == "none":
            return len(self.ao_shells)
        return 2 * sum(2 * l + 1 for l in self.ao_shells)

    @property
    def naux(self) -> int:
        if self.structure == "none":
            return len(self.aux_shells)
        return 2 * sum(2 * l + 1 for l in self.aux_shells)

    @property
    def nkpts(self) -> int:
        return self.nk[0] * self.nk[1] * self.nk[2]

    @property
    def n_elec(self) -> float:
        """Half filling: N_e = nao electrons per cell (both spins counted)."""
        return float(self.nao)


def _shells(counts: dict) -> tuple:
    out = []
    for l in sorted(counts):
        out += [l] * counts[l]
    return tuple(out)


CONFIGS = {
    "c1": Config(
        name="c1", index=0, structure="none", nk=(2, 2, 2), ao_shells=(0,) * 8, aux_shells=(0,) * 32,
        ntau=20, beta=100.0, mats_f=F20, mats_b=B20,
        description="plain step, no symmetry: 2x2x2 mesh, nao 8, naux 32, 20 tau, beta 100"),
    "c2": Config(
        name="c2", index=1, structure="rocksalt", nk=(3, 3, 3), ao_shells=_shells({0: 1, 1: 1, 2: 1}),
        aux_shells=_shells({0: 6, 1: 5, 2: 3, 3: 2}), ntau=50, beta=100.0, mats_f=F50, mats_b=B50,
        description="rocksalt Oh, 3x3x3 mesh (4 wedge points), nao 18, naux 100, 50 tau, beta 100"),
    # small rocksalt cell for the smoke run and the fast parity tests: 2x2x2 mesh (3 wedge points)
    "t1": Config(
        name="t1", index=10, structure="rocksalt", nk=(2, 2, 2), ao_shells=(0, 1), aux_shells=(0, 0, 1, 2),
        ntau=16, beta=10.0, mats_f=F16, mats_b=B16,
        description="rocksalt Oh, 2x2x2 mesh, nao 8, naux 20, 16 tau, beta 10"),
}


def get(name: str) -> Config:
    return CONFIGS[name]
