"""Session: one library context for one workload, with its inputs loaded.

Marshalling only: it turns a workload description and the seeded synthetic
inputs into the C-ABI calls of :mod:`paper_2405_09494_gb300.sgw`, and
allocates the caller-owned device buffers with PyTorch.  Every step of the
method runs inside the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import sgw, synth
from .configs import Config


def structure_arrays(cfg: Config):
    """Crystal description for sgw_build_irrep_basis (from the workload definition)."""
    ops = synth.space_group(cfg.structure)
    rot = np.stack([R for R, _ in ops])
    tra = np.stack([v for _, v in ops])
    if cfg.structure == "none":
        return np.eye(3), np.zeros((1, 3)), rot, tra, [0] * cfg.nao, [0] * cfg.naux
    return synth.FCC, synth.atom_positions(cfg.structure), rot, tra, list(cfg.ao_shells), list(cfg.aux_shells)


class Session:
    def __init__(self, cfg: Config, precision: int = sgw.SGW_FP64, device: str = "cuda:0", system=None,
                 load_v: bool = True):
        import torch

        self.torch = torch
        self.cfg = cfg
        self.precision = precision
        self.device = torch.device(device)
        self.sys = system if system is not None else synth.System(cfg)
        self.ctx = sgw.sgw_create(cfg.nk, cfg.nao, cfg.naux, cfg.ntau, cfg.mats_f, cfg.mats_b, cfg.beta, cfg.n_elec,
                                  cfg.spin, cfg.loop_sign, precision)
        lat, pos, rot, tra, aos, axs = structure_arrays(cfg)
        self.layout = sgw.sgw_build_irrep_basis(self.ctx, lat, pos, rot, tra, aos, axs)
        L = self.layout
        self.wedge, self.rep, self.op = sgw.sgw_get_wedge(self.ctx, L.nkpts, L.nwedge)
        self.pairs = [sgw.sgw_get_pairs(self.ctx, w, L.npairs) for w in (0, 1)]
        H0 = torch.from_numpy(np.ascontiguousarray(self.sys.H0)).to(self.device)
        S = torch.from_numpy(np.ascontiguousarray(self.sys.S)).to(self.device)
        sgw.sgw_load_one_body(self.ctx, H0, S)
        if load_v:
            self.load_v()

    def load_v(self, chunk: int = 64):
        torch = self.torch
        cfg = self.cfg
        for which in (0, 1):
            k1, k2 = self.pairs[which]
            n = len(k1)
            for p0 in range(0, n, chunk):
                p1 = min(n, p0 + chunk)
                vs = [self.sys.V(int(a), int(b)) for a, b in zip(k1[p0:p1], k2[p0:p1])]
                if isinstance(vs[0], np.ndarray):
                    t = torch.from_numpy(np.stack(vs)).to(self.device)
                else:
                    t = torch.stack(vs).to(self.device).contiguous()
                sgw.sgw_load_v(self.ctx, which, p0, p1 - p0, t)
                torch.cuda.synchronize(self.device)
        del cfg

    # ---- buffers ----------------------------------------------------------
    def zeros(self, *shape):
        return self.torch.zeros(*shape, dtype=self.torch.complex128, device=self.device)

    def g_series(self, nt=None):
        return self.zeros(nt or self.cfg.ntau, self.layout.g_elems)

    def p_series(self, nt=None):
        return self.zeros(nt or self.cfg.ntau, self.layout.p_elems)

    # ---- steps --------------------------------------------------------------
    def g0(self):
        G = self.g_series()
        mu = sgw.sgw_g0(self.ctx, G)
        return G, mu

    def polarization(self, G, pairs=None):
        """P0(tau); with ``pairs`` = (begin, end), the partial sum over that range of the pair list."""
        P0 = self.p_series()
        if pairs is None:
            sgw.sgw_polarization(self.ctx, G, P0)
        else:
            sgw.sgw_polarization_pairs(self.ctx, G, P0, pairs[0], pairs[1])
        return P0

    def screened(self, P0):
        P = self.p_series()
        sgw.sgw_screened_interaction(self.ctx, P0, P)
        return P

    def self_energy(self, G, P, pairs=None):
        """Sigma~(tau); with ``pairs`` = (begin, end), the partial sum over that range of the pair list."""
        Sig = self.g_series()
        if pairs is None:
            sgw.sgw_self_energy(self.ctx, G, P, Sig)
        else:
            sgw.sgw_self_energy_pairs(self.ctx, G, P, Sig, pairs[0], pairs[1])
        return Sig

    def hartree_fock(self, G):
        H = self.zeros(self.layout.g_elems)
        sgw.sgw_hartree_fock(self.ctx, G, H)
        return H

    def dyson(self, Sig, Shf, mu, search_mu=True):
        G = self.g_series()
        mu = sgw.sgw_dyson(self.ctx, Sig, Shf, mu, search_mu, G)
        return G, mu

    def energy(self, G, Shf, Sig):
        return sgw.sgw_energy(self.ctx, G, Shf, Sig)

    def unfold(self, which, packed):
        nt = packed.shape[0] if packed.dim() == 2 else 1
        n = self.cfg.nao if which == 0 else self.cfg.naux
        out = self.zeros(self.layout.nkpts, nt, n, n)
        sgw.sgw_unfold(self.ctx, which, nt, packed, out)
        self.torch.cuda.synchronize(self.device)
        return out

    # ---- checkpoint / resume ------------------------------------------------
    def state_key(self) -> str:
        """Identity of the workload a saved loop state belongs to (configuration and precision)."""
        import hashlib
        import json

        desc = {k: (list(v) if isinstance(v, tuple) else v) for k, v in vars(self.cfg).items()}
        desc["precision"] = int(self.precision)
        return hashlib.sha256(json.dumps(desc, sort_keys=True, default=str).encode()).hexdigest()

    def save_state(self, path, G, Sig, Shf, mu, iteration=0, history=()):
        """Write the state of the self-consistency loop to ``path`` (.npz): packed G(tau),
        Sigma~(tau), Sigma_HF, mu and a JSON header (workload key, pass count, |Delta Sigma|
        history).  The library keeps nothing else between passes, so this is the whole state."""
        import json

        head = dict(key=self.state_key(), iteration=int(iteration), history=[float(x) for x in history],
                    g_elems=int(self.layout.g_elems), ntau=int(self.cfg.ntau))
        np.savez(path, G=G.cpu().numpy(), Sig=Sig.cpu().numpy(), Shf=Shf.cpu().numpy(), mu=np.float64(mu),
                 header=np.frombuffer(json.dumps(head).encode(), dtype=np.uint8))

    def load_state(self, path):
        """Read a state written by :meth:`save_state` for this workload: (G, Sig, Shf, mu, header)."""
        import json

        z = np.load(path)
        head = json.loads(bytes(z["header"]).decode())
        if head["key"] != self.state_key():
            raise ValueError("saved loop state belongs to another workload or precision")
        dev = self.device
        to = lambda a: self.torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        return to(z["G"]), to(z["Sig"]), to(z["Shf"]), float(z["mu"]), head

    def close(self):
        if self.ctx is not None:
            sgw.sgw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
