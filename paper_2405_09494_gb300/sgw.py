"""ctypes binding of the sgw C ABI (include/sgw.h): argument marshalling only.

Every function keeps the C name and forwards plain pointers.  Tensor arguments
may be torch tensors (their ``data_ptr()`` is passed) or integers (raw device
addresses).  Streams may be ``torch.cuda.Stream`` objects, integers or None
(the legacy default stream).  A failing call raises :class:`SGWError` with the
library's status text and detail message.  The library is the only compute
path: if ``libsgw.so`` is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsgw.so")

SGW_FP64 = 0
SGW_MIXED_FP32 = 1

STATUS = {0: "SGW_OK", 1: "SGW_ERR_ARG", 2: "SGW_ERR_CUDA", 3: "SGW_ERR_OOM", 4: "SGW_ERR_SINGULAR",
          5: "SGW_ERR_NOCONV", 6: "SGW_ERR_TIMEOUT", 7: "SGW_ERR_UNIMPLEMENTED", 8: "SGW_ERR_STATE"}

EXPORTS = [
    "sgw_create", "sgw_destroy", "sgw_status_str", "sgw_last_error", "sgw_sync", "sgw_build_irrep_basis",
    "sgw_get_wedge", "sgw_get_blocks", "sgw_get_pairs", "sgw_get_basis", "sgw_load_one_body", "sgw_load_v",
    "sgw_g0", "sgw_polarization", "sgw_screened_interaction", "sgw_self_energy", "sgw_hartree_fock", "sgw_dyson",
    "sgw_energy", "sgw_iterate", "sgw_unfold", "sgw_host_grid", "sgw_host_symmetry", "sgw_profile_enable",
    "sgw_profile_read", "sgw_screened_interaction_noalloc", "sgw_set_wait_limit", "sgw_polarization_pairs",
    "sgw_self_energy_pairs", "sgw_host_irrep_dims", "sgw_host_partner_basis",
]


class SGWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nk", ctypes.c_int * 3), ("nao", ctypes.c_int), ("naux", ctypes.c_int), ("ntau", ctypes.c_int),
                ("nw_f", ctypes.c_int), ("nw_b", ctypes.c_int), ("mats_f", ctypes.POINTER(ctypes.c_int)),
                ("mats_b", ctypes.POINTER(ctypes.c_int)), ("beta", ctypes.c_double), ("n_elec", ctypes.c_double),
                ("spin_factor", ctypes.c_int), ("loop_sign", ctypes.c_int), ("precision", ctypes.c_int)]


class Structure(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9), ("natom", ctypes.c_int),
                ("positions", ctypes.POINTER(ctypes.c_double)), ("nops", ctypes.c_int),
                ("rotations", ctypes.POINTER(ctypes.c_double)), ("translations", ctypes.POINTER(ctypes.c_double)),
                ("n_ao_shells", ctypes.c_int), ("ao_shells", ctypes.POINTER(ctypes.c_int)),
                ("n_aux_shells", ctypes.c_int), ("aux_shells", ctypes.POINTER(ctypes.c_int))]


class Layout(ctypes.Structure):
    _fields_ = [("nkpts", ctypes.c_int), ("nwedge", ctypes.c_int), ("g_elems", ctypes.c_longlong),
                ("p_elems", ctypes.c_longlong), ("npairs", ctypes.c_longlong), ("max_ao_block", ctypes.c_int),
                ("max_aux_block", ctypes.c_int)]


class IterStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("mu", ctypes.c_double), ("n_elec", ctypes.c_double),
                ("max_dsigma", ctypes.c_double), ("energy", ctypes.c_double * 4), ("energy_imag", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsgw.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"sgw CUDA library not found at {path}; build it with "
                           "`python -m paper_2405_09494_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    sig = {
        "sgw_create": ([ctypes.POINTER(Params), ctypes.POINTER(vp)], i),
        "sgw_destroy": ([vp], i),
        "sgw_status_str": ([i], ctypes.c_char_p),
        "sgw_last_error": ([vp, ctypes.c_char_p, ctypes.c_size_t], i),
        "sgw_sync": ([vp, vp], i),
        "sgw_build_irrep_basis": ([vp, ctypes.POINTER(Structure), ctypes.POINTER(Layout)], i),
        "sgw_get_wedge": ([vp, vp, vp, vp], i),
        "sgw_get_blocks": ([vp, i, i, ctypes.POINTER(i), vp], i),
        "sgw_get_pairs": ([vp, i, vp, vp], i),
        "sgw_get_basis": ([vp, i, vp, vp], i),
        "sgw_load_one_body": ([vp, vp, vp, vp], i),
        "sgw_load_v": ([vp, i, ll, ll, vp, vp], i),
        "sgw_g0": ([vp, ctypes.POINTER(d), vp, vp], i),
        "sgw_polarization": ([vp, vp, vp, vp], i),
        "sgw_polarization_pairs": ([vp, vp, vp, ll, ll, vp], i),
        "sgw_self_energy_pairs": ([vp, vp, vp, vp, ll, ll, vp], i),
        "sgw_screened_interaction": ([vp, vp, vp, vp], i),
        "sgw_self_energy": ([vp, vp, vp, vp, vp], i),
        "sgw_hartree_fock": ([vp, vp, vp, vp], i),
        "sgw_dyson": ([vp, vp, vp, ctypes.POINTER(d), i, vp, vp], i),
        "sgw_energy": ([vp, vp, vp, vp, ctypes.POINTER(d), vp], i),
        "sgw_iterate": ([vp, i, d, d, vp, vp, vp, ctypes.POINTER(d), ctypes.POINTER(IterStats), vp], i),
        "sgw_unfold": ([vp, i, i, vp, vp, vp], i),
        "sgw_host_grid": ([ctypes.POINTER(Params), vp, vp, vp, vp, vp], i),
        "sgw_host_symmetry": ([ctypes.POINTER(Params), ctypes.POINTER(Structure), ctypes.POINTER(i), vp, vp, vp], i),
        "sgw_host_irrep_dims": ([ctypes.POINTER(Params), ctypes.POINTER(Structure), ctypes.POINTER(i), vp, vp], i),
        "sgw_host_partner_basis": ([ctypes.POINTER(Params), ctypes.POINTER(Structure), i, ctypes.POINTER(i), vp], i),
        "sgw_screened_interaction_noalloc": ([vp, vp, vp, vp], i),
        "sgw_profile_enable": ([vp, i], i),
        "sgw_set_wait_limit": ([vp, ctypes.c_ulonglong], i),
        "sgw_profile_read": ([vp, i, ctypes.c_char_p, ctypes.POINTER(d), ctypes.POINTER(d),
                              ctypes.POINTER(ll), ctypes.POINTER(i), i], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status, ctx=None):
    if status != 0:
        lib = load_library()
        msg = lib.sgw_status_str(status).decode()
        if ctx is not None:
            buf = ctypes.create_string_buffer(512)
            lib.sgw_last_error(ctx, buf, 512)
            if buf.value:
                msg += ": " + buf.value.decode()
        raise SGWError(status, msg)


# ---------------------------------------------------------------------------
# one wrapper per C entry point
# ---------------------------------------------------------------------------
def _params(nk, nao, naux, ntau, mats_f, mats_b, beta, n_elec, spin_factor=2, loop_sign=1, precision=SGW_FP64):
    mf = (ctypes.c_int * len(mats_f))(*mats_f)
    mb = (ctypes.c_int * len(mats_b))(*mats_b)
    p = Params((ctypes.c_int * 3)(*nk), nao, naux, ntau, len(mats_f), len(mats_b), mf, mb, beta, n_elec, spin_factor,
               loop_sign, precision)
    p._keep = (mf, mb)
    return p


def _structure(lattice, positions, rotations, translations, ao_shells, aux_shells):
    import numpy as np

    lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.float64).reshape(-1))
    rot = np.ascontiguousarray(np.asarray(rotations, dtype=np.float64).reshape(-1))
    tra = np.ascontiguousarray(np.asarray(translations, dtype=np.float64).reshape(-1))
    aos = np.ascontiguousarray(np.asarray(ao_shells, dtype=np.int32))
    axs = np.ascontiguousarray(np.asarray(aux_shells, dtype=np.int32))
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    st = Structure((ctypes.c_double * 9)(*lat), pos.size // 3, pos.ctypes.data_as(dp), rot.size // 9,
                   rot.ctypes.data_as(dp), tra.ctypes.data_as(dp), aos.size, aos.ctypes.data_as(ip), axs.size,
                   axs.ctypes.data_as(ip))
    st._keep = (pos, rot, tra, aos, axs)
    return st


def sgw_create(nk, nao, naux, ntau, mats_f, mats_b, beta, n_elec, spin_factor=2, loop_sign=1, precision=SGW_FP64):
    lib = load_library()
    p = _params(nk, nao, naux, ntau, mats_f, mats_b, beta, n_elec, spin_factor, loop_sign, precision)
    out = ctypes.c_void_p()
    _check(lib.sgw_create(ctypes.byref(p), ctypes.byref(out)))
    return out


def sgw_destroy(ctx):
    _check(load_library().sgw_destroy(ctx))


def sgw_status_str(status: int) -> str:
    return load_library().sgw_status_str(status).decode()


def sgw_last_error(ctx) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(load_library().sgw_last_error(ctx, buf, 512))
    return buf.value.decode()


def sgw_sync(ctx, stream=None):
    _check(load_library().sgw_sync(ctx, _stream(stream)), ctx)


def sgw_build_irrep_basis(ctx, lattice, positions, rotations, translations, ao_shells, aux_shells) -> Layout:
    """lattice: 3x3 (columns = primitive vectors); rotations: [nops][3][3]; translations: [nops][3]."""
    st = _structure(lattice, positions, rotations, translations, ao_shells, aux_shells)
    lay = Layout()
    _check(load_library().sgw_build_irrep_basis(ctx, ctypes.byref(st), ctypes.byref(lay)), ctx)
    return lay


def sgw_get_wedge(ctx, nkpts, nwedge):
    import numpy as np

    wk = np.zeros(nwedge, np.int32)
    rep = np.zeros(nkpts, np.int32)
    op = np.zeros(nkpts, np.int32)
    _check(load_library().sgw_get_wedge(ctx, wk.ctypes.data, rep.ctypes.data, op.ctypes.data), ctx)
    return wk, rep, op


def sgw_get_blocks(ctx, which, w, nmax):
    import numpy as np

    n = ctypes.c_int()
    sizes = np.zeros(nmax, np.int32)
    _check(load_library().sgw_get_blocks(ctx, which, w, ctypes.byref(n), sizes.ctypes.data), ctx)
    return sizes[: n.value].copy()


def sgw_get_pairs(ctx, which, npairs):
    import numpy as np

    k1 = np.zeros(npairs, np.int32)
    k2 = np.zeros(npairs, np.int32)
    _check(load_library().sgw_get_pairs(ctx, which, k1.ctypes.data, k2.ctypes.data), ctx)
    return k1, k2


def sgw_get_basis(ctx, which, U, stream=None):
    _check(load_library().sgw_get_basis(ctx, which, _ptr(U), _stream(stream)), ctx)


def sgw_load_one_body(ctx, H0, S, stream=None):
    _check(load_library().sgw_load_one_body(ctx, _ptr(H0), _ptr(S), _stream(stream)), ctx)


def sgw_load_v(ctx, which, first, count, V, stream=None):
    _check(load_library().sgw_load_v(ctx, which, first, count, _ptr(V), _stream(stream)), ctx)


def sgw_g0(ctx, G_tau, stream=None) -> float:
    mu = ctypes.c_double()
    _check(load_library().sgw_g0(ctx, ctypes.byref(mu), _ptr(G_tau), _stream(stream)), ctx)
    return mu.value


def sgw_polarization(ctx, G_tau, P0_tau, stream=None):
    _check(load_library().sgw_polarization(ctx, _ptr(G_tau), _ptr(P0_tau), _stream(stream)), ctx)


def sgw_polarization_pairs(ctx, G_tau, P0_tau, pair_begin, pair_end, stream=None):
    _check(load_library().sgw_polarization_pairs(ctx, _ptr(G_tau), _ptr(P0_tau), int(pair_begin), int(pair_end),
                                                 _stream(stream)), ctx)


def sgw_screened_interaction(ctx, P0_tau, P_tau, stream=None):
    _check(load_library().sgw_screened_interaction(ctx, _ptr(P0_tau), _ptr(P_tau), _stream(stream)), ctx)


def sgw_screened_interaction_noalloc(ctx, P0_tau, P_tau, stream=None):
    """sgw_screened_interaction without any device allocation (scratch in a fixed 64 MiB library array).

    For callers that may not allocate device memory at call time; see include/sgw.h for the
    limits, the one-time set-up on each device and the rule that overlapping calls race.
    """
    _check(load_library().sgw_screened_interaction_noalloc(ctx, _ptr(P0_tau), _ptr(P_tau), _stream(stream)), ctx)


def sgw_self_energy(ctx, G_tau, P_tau, Sigma_tau, stream=None):
    _check(load_library().sgw_self_energy(ctx, _ptr(G_tau), _ptr(P_tau), _ptr(Sigma_tau), _stream(stream)), ctx)


def sgw_self_energy_pairs(ctx, G_tau, P_tau, Sigma_tau, pair_begin, pair_end, stream=None):
    _check(load_library().sgw_self_energy_pairs(ctx, _ptr(G_tau), _ptr(P_tau), _ptr(Sigma_tau), int(pair_begin),
                                                int(pair_end), _stream(stream)), ctx)


def sgw_hartree_fock(ctx, G_tau, Sigma_hf, stream=None):
    _check(load_library().sgw_hartree_fock(ctx, _ptr(G_tau), _ptr(Sigma_hf), _stream(stream)), ctx)


def sgw_dyson(ctx, Sigma_tau, Sigma_hf, mu, search_mu, G_tau, stream=None) -> float:
    m = ctypes.c_double(mu)
    _check(load_library().sgw_dyson(ctx, _ptr(Sigma_tau), _ptr(Sigma_hf), ctypes.byref(m), int(search_mu),
                                    _ptr(G_tau), _stream(stream)), ctx)
    return m.value


def sgw_energy(ctx, G_tau, Sigma_hf, Sigma_tau, stream=None):
    e = (ctypes.c_double * 5)()
    _check(load_library().sgw_energy(ctx, _ptr(G_tau), _ptr(Sigma_hf), _ptr(Sigma_tau), e, _stream(stream)), ctx)
    return list(e)


def sgw_iterate(ctx, max_iter, damping, tol, G_tau, Sigma_tau, Sigma_hf, mu, stream=None):
    m = ctypes.c_double(mu)
    stats = IterStats()
    _check(load_library().sgw_iterate(ctx, max_iter, damping, tol, _ptr(G_tau), _ptr(Sigma_tau), _ptr(Sigma_hf),
                                      ctypes.byref(m), ctypes.byref(stats), _stream(stream)), ctx)
    return m.value, stats


def sgw_unfold(ctx, which, nt, packed, ao_full, stream=None):
    _check(load_library().sgw_unfold(ctx, which, nt, _ptr(packed), _ptr(ao_full), _stream(stream)), ctx)


def sgw_set_wait_limit(ctx, ns):
    """Limit (ns) of each wait in the tensor-core pipeline kernel (2 s at creation; see sgw.h)."""
    _check(load_library().sgw_set_wait_limit(ctx, int(ns)), ctx)


def sgw_profile_enable(ctx, on=True):
    _check(load_library().sgw_profile_enable(ctx, int(bool(on))), ctx)


def sgw_profile_read(ctx, reset=False):
    """{kernel class: (ms, gflop, launches)} since the last reset."""
    n_max = 64
    names = ctypes.create_string_buffer(48 * n_max)
    ms = (ctypes.c_double * n_max)()
    gf = (ctypes.c_double * n_max)()
    ln = (ctypes.c_longlong * n_max)()
    n = ctypes.c_int()
    _check(load_library().sgw_profile_read(ctx, n_max, names, ms, gf, ln, ctypes.byref(n), int(bool(reset))), ctx)
    out = {}
    for k in range(min(n.value, n_max)):
        nm = names.raw[48 * k: 48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (ms[k], gf[k], ln[k])
    return out


def sgw_host_grid(nk, nao, naux, ntau, mats_f, mats_b, beta, n_elec=1.0):
    """Host-only: tau nodes and the four transform matrices the library builds."""
    import numpy as np

    p = _params(nk, nao, naux, ntau, mats_f, mats_b, beta, n_elec)
    tau = np.zeros(ntau)
    TF = np.zeros((len(mats_f), ntau), np.complex128)
    TFb = np.zeros((ntau, len(mats_f)), np.complex128)
    TB = np.zeros((len(mats_b), ntau), np.complex128)
    TBb = np.zeros((ntau, len(mats_b)), np.complex128)
    _check(load_library().sgw_host_grid(ctypes.byref(p), tau.ctypes.data, TF.ctypes.data, TFb.ctypes.data,
                                        TB.ctypes.data, TBb.ctypes.data))
    return tau, TF, TFb, TB, TBb


def sgw_host_irrep_dims(nk, nao, naux, lattice, positions, rotations, translations, ao_shells, aux_shells):
    """Host-only: the irrep dimension d of every block of sgw_host_symmetry, per wedge point (ao, aux)."""
    import numpy as np

    p = _params(nk, nao, naux, 2, [0, 1], [0, 1], 1.0, 1.0)
    st = _structure(lattice, positions, rotations, translations, ao_shells, aux_shells)
    Nk = nk[0] * nk[1] * nk[2]
    nw = ctypes.c_int()
    ao = np.zeros((Nk, nao + 1), np.int32)
    ax = np.zeros((Nk, naux + 1), np.int32)
    _check(load_library().sgw_host_irrep_dims(ctypes.byref(p), ctypes.byref(st), ctypes.byref(nw), ao.ctypes.data,
                                              ax.ctypes.data))
    n = nw.value
    dims = lambda row: [int(x) for x in row[: list(row).index(0)]]  # noqa: E731
    return [dims(ao[w]) for w in range(n)], [dims(ax[w]) for w in range(n)]


def sgw_host_partner_basis(nk, nao, naux, lattice, positions, rotations, translations, ao_shells, aux_shells, family):
    """Host-only: partner-adapted bases [nwedge][n][n] (complex) of one family (0 orbitals, 1 auxiliary)."""
    import numpy as np

    p = _params(nk, nao, naux, 2, [0, 1], [0, 1], 1.0, 1.0)
    st = _structure(lattice, positions, rotations, translations, ao_shells, aux_shells)
    Nk = nk[0] * nk[1] * nk[2]
    n = nao if family == 0 else naux
    nw = ctypes.c_int()
    U = np.zeros((Nk, n, n), np.complex128)
    _check(load_library().sgw_host_partner_basis(ctypes.byref(p), ctypes.byref(st), int(family), ctypes.byref(nw),
                                                 U.ctypes.data))
    return U[: nw.value]


def sgw_host_symmetry(nk, nao, naux, lattice, positions, rotations, translations, ao_shells, aux_shells):
    """Host-only space-group analysis: (nwedge, rep[nkpts], ao block sizes per wedge, aux block sizes per wedge)."""
    import numpy as np

    p = _params(nk, nao, naux, 2, [0, 1], [0, 1], 1.0, 1.0)
    st = _structure(lattice, positions, rotations, translations, ao_shells, aux_shells)
    Nk = nk[0] * nk[1] * nk[2]
    nw = ctypes.c_int()
    rep = np.zeros(Nk, np.int32)
    ao = np.zeros((Nk, nao + 1), np.int32)
    ax = np.zeros((Nk, naux + 1), np.int32)
    _check(load_library().sgw_host_symmetry(ctypes.byref(p), ctypes.byref(st), ctypes.byref(nw), rep.ctypes.data,
                                            ao.ctypes.data, ax.ctypes.data))
    n = nw.value
    blocks = lambda row: [int(x) for x in row[: list(row).index(0)]]  # noqa: E731
    return n, rep, [blocks(ao[w]) for w in range(n)], [blocks(ax[w]) for w in range(n)]
