"""Workload definitions: seeded synthetic systems shaped like the paper's solids.

Each entry fixes the sizes, the crystal, the tau grid and the finite Matsubara
index sets.  The index sets are plain input data (integers); the oracle and the
library each build their own transform matrices from them.  They were chosen
by the oracle's offline greedy volume search (``python -m oracle.choose_matsubara``)
so that the Chebyshev-node -> Matsubara map is well conditioned (cond 36 at
n_tau = 20, 140 at n_tau = 50, about 1.1e3 at n_tau = 200, beta = 500).

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

F100 = [-529, -268, -177, -132, -106, -88, -76, -67, -60, -54, -50, -46, -43, -40, -38, -36, -34, -33, -32, -31, -30, -29, -28, -27, -26, -25, -24, -23, -22, -21, -20, -19, -18, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 35, 37, 39, 42, 45, 49, 53, 59, 66, 75, 87, 105, 131, 176, 267, 528]
B100 = [-775, -358, -212, -150, -116, -95, -81, -70, -62, -56, -51, -47, -44, -41, -39, -37, -35, -33, -32, -31, -30, -29, -28, -27, -26, -25, -24, -23, -22, -21, -20, -19, -18, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 35, 37, 39, 41, 44, 47, 51, 56, 62, 70, 81, 95, 116, 150, 212, 358, 775]
F150 = [-1174, -593, -392, -292, -233, -194, -166, -146, -130, -117, -107, -98, -91, -85, -80, -75, -71, -68, -65, -62, -59, -57, -55, -53, -52, -50, -49, -48, -47, -46, -45, -44, -43, -42, -41, -40, -39, -38, -37, -36, -35, -34, -33, -32, -31, -30, -29, -28, -27, -26, -25, -24, -23, -22, -21, -20, -19, -18, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 46, 47, 48, 49, 51, 52, 54, 56, 58, 61, 64, 67, 70, 74, 79, 84, 90, 97, 106, 116, 129, 145, 165, 193, 232, 291, 391, 592, 1173]
B150 = [-1735, -802, -474, -335, -259, -211, -179, -155, -137, -123, -111, -102, -94, -88, -82, -77, -73, -69, -66, -63, -60, -58, -56, -54, -52, -50, -49, -48, -47, -46, -45, -44, -43, -42, -41, -40, -39, -38, -37, -36, -35, -34, -33, -32, -31, -30, -29, -28, -27, -26, -25, -24, -23, -22, -21, -20, -19, -18, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 46, 47, 48, 49, 50, 52, 54, 56, 58, 60, 63, 66, 69, 73, 77, 82, 88, 94, 102, 111, 123, 137, 155, 179, 211, 259, 335, 474, 802, 1735]
F200 = [-2069, -1047, -691, -515, -410, -341, -292, -256, -228, -205, -187, -172, -159, -148, -138, -130, -123, -117, -111, -106, -101, -97, -93, -90, -87, -84, -81, -79, -77, -75, -73, -71, -69, -68, -66, -65, -64, -63, -62, -61, -60, -59, -58, -57, -56, -55, -54, -53, -52, -51, -50, -49, -48, -47, -46, -45, -44, -43, -42, -41, -40, -39, -38, -37, -36, -35, -34, -33, -32, -31, -30, -29, -28, -27, -26, -25, -24, -23, -22, -21, -20, -19, -18, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 46, 47, 48, 49, 50, 51, 52, 53, 54, 55, 56, 57, 58, 59, 60, 61, 62, 63, 64, 65, 67, 68, 70, 72, 74, 76, 78, 80, 83, 86, 89, 92, 96, 100, 105, 110, 116, 122, 129, 137, 147, 158, 171, 186, 204, 227, 255, 291, 340, 409, 514, 690, 1046, 2068]
B200 = [-3059, -1411, -834, -590, -456, -372, -314, -272, -240, -215, -195, -179, -165, -153, -143, -134, -126, -119, -113, -108, -103, -99, -95, -91, -88, -85, -82, -79, -77, -75, -73, -71, -69, -68, -66, -65, -64, -63, -62, -61, -60, -59, -58, -57, -56, -55, -54, -53, -52, -51, -50, -49, -48, -47, -46, -45, -44, -43, -42, -41, -40, -39, -38, -37, -36, -35, -34, -33, -32, -31, -30, -29, -28, -27, -26, -25, -24, -23, -22, -21, -20, -19, -18, -17, -16, -15, -14, -13, -12, -11, -10, -9, -8, -7, -6, -5, -4, -3, -2, -1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 46, 47, 48, 49, 50, 51, 52, 53, 54, 55, 56, 57, 58, 59, 60, 61, 62, 63, 64, 65, 66, 68, 69, 71, 73, 75, 77, 79, 82, 85, 88, 91, 95, 99, 103, 108, 113, 119, 126, 134, 143, 153, 165, 179, 195, 215, 240, 272, 314, 372, 456, 590, 834, 1411, 3059]


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
    # Sigma <- (1 - a) Sigma_old + a Sigma_new in the loop (not in the paper).  The crystal workloads
    # use a = 0.5: undamped, the rocksalt 3x3x3 loop alternates between two states
    # (max |Delta Sigma| about 1.3 Ha every pass), damped by 0.5 it converges (about 3.7x per pass).
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
        aux_shells=_shells({0: 6, 1: 5, 2: 3, 3: 2}), ntau=50, beta=100.0, mats_f=F50, mats_b=B50, damping=0.5,
        description="rocksalt Oh, 3x3x3 mesh (4 wedge points), nao 18, naux 100, 50 tau, beta 100"),
    "c3": Config(
        name="c3", index=2, structure="rocksalt", nk=(4, 4, 4), ao_shells=_shells({0: 4, 1: 4, 2: 2}),
        aux_shells=_shells({0: 10, 1: 10, 2: 11, 3: 4, 4: 3}), ntau=100, beta=200.0, mats_f=F100, mats_b=B100,
        damping=0.5,
        description="rocksalt Oh, 4x4x4 mesh (8 wedge points), nao 52, naux 300, 100 tau, beta 200"),
    "c4": Config(
        name="c4", index=3, structure="diamond", nk=(4, 4, 4), ao_shells=_shells({0: 4, 1: 4, 2: 2}),
        aux_shells=_shells({0: 10, 1: 10, 2: 11, 3: 4, 4: 3}), ntau=150, beta=200.0, mats_f=F150, mats_b=B150,
        damping=0.5,
        description="diamond Fd-3m (non-symmorphic), 4x4x4 mesh (8 wedge points), nao 52, naux 300, 150 tau, beta 200"),
    "c5": Config(
        name="c5", index=4, structure="rocksalt", nk=(4, 4, 4), ao_shells=_shells({0: 7, 1: 6, 2: 4, 3: 1}),
        aux_shells=_shells({0: 20, 1: 20, 2: 22, 3: 8, 4: 6}), ntau=200, beta=500.0, mats_f=F200, mats_b=B200,
        damping=0.5,
        # couplings scaled by 0.5: at unit scale the exchange term of its 52 occupied orbitals moves
        # Sigma by 20.7 Ha in the first pass and the mu root out of the search bracket [-20, 20]
        extra={"vscale": 0.5},
        description="rocksalt Oh, 4x4x4 mesh (8 wedge points), nao 104, naux 600, 200 tau, beta 500, "
                    "self-consistent loop with damping 0.5"),
    # c3's cell and shells (nao 52, naux 300: the same tiles and blocks per pair) on a 2x2x2 mesh with
    # 16 tau: a case small enough for full profiler captures of the c3/c4 kernels (operands of a few GB)
    "c3s": Config(
        name="c3s", index=12, structure="rocksalt", nk=(2, 2, 2), ao_shells=_shells({0: 4, 1: 4, 2: 2}),
        aux_shells=_shells({0: 10, 1: 10, 2: 11, 3: 4, 4: 3}), ntau=16, beta=10.0, mats_f=F16, mats_b=B16,
        damping=0.5,
        description="rocksalt Oh, 2x2x2 mesh, nao 52, naux 300, 16 tau, beta 10 (profiling case of c3's kernels)"),
    # small rocksalt cell for the smoke run and the fast parity tests: 2x2x2 mesh (3 wedge points)
    "t1": Config(
        name="t1", index=10, structure="rocksalt", nk=(2, 2, 2), ao_shells=(0, 1), aux_shells=(0, 0, 1, 2),
        ntau=16, beta=10.0, mats_f=F16, mats_b=B16,
        description="rocksalt Oh, 2x2x2 mesh, nao 8, naux 20, 16 tau, beta 10"),
}


def get(name: str) -> Config:
    return CONFIGS[name]
