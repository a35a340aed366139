"""Thin Python binding of libcdfci (include/cdfci.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays may be
numpy arrays (host memory) or torch tensors on the GPU (device memory); the
library detects which.  Nothing here computes any part of the method, and
there is no fallback: if libcdfci.so is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcdfci.so")

CDFCI_OK = 0
ERRORS = {-1: "ARG", -2: "NONFINITE", -3: "TABLE_FULL", -4: "TIMEOUT", -5: "CUDA", -6: "UNIMPLEMENTED",
          -7: "NOMEM", -8: "CAPACITY", -9: "NOT_NEGATIVE", -10: "INTERNAL"}


class cdfci_params(ctypes.Structure):
    _fields_ = [("num_coordinates", ctypes.c_int32), ("log2_capacity", ctypes.c_int32),
                ("z_threshold", ctypes.c_double), ("max_load", ctypes.c_double),
                ("dx_damping", ctypes.c_double), ("dx_threshold", ctypes.c_double),
                ("ref_alpha", ctypes.c_uint64), ("ref_beta", ctypes.c_uint64),
                ("block_threads", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("graph_chunk", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("num_states", ctypes.c_int32),
                ("z_threshold_search", ctypes.c_int32), ("max_memory", ctypes.c_double),
                ("integral_symmetry", ctypes.c_int32)]


class cdfci_optorb_params(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("bb_steps", ctypes.c_int32), ("inner_iterations", ctypes.c_int64),
                ("fci", cdfci_params)]


class cdfci_tune_report(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("chosen", ctypes.c_int32), ("m", ctypes.c_int32 * 16),
                ("grid_blocks", ctypes.c_int32 * 16), ("iterations", ctypes.c_int64 * 16),
                ("seconds", ctypes.c_double * 16), ("energy_drop", ctypes.c_double * 16),
                ("score", ctypes.c_double * 16)]


class cdfci_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("energy", ctypes.c_double), ("mu", ctypes.c_double),
                ("alpha", ctypes.c_double), ("dx", ctypes.c_double), ("nnz_c", ctypes.c_int64),
                ("n_slots", ctypes.c_int64), ("last_column", ctypes.c_int64), ("elements", ctypes.c_int64),
                ("applied", ctypes.c_int64), ("dropped", ctypes.c_int64), ("inserted", ctypes.c_int64),
                ("load", ctypes.c_double), ("status", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("reduced_iterations", ctypes.c_int64), ("grid_blocks", ctypes.c_int32),
                ("grid_wide", ctypes.c_int32), ("z_threshold", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class cdfci_checkpoint_header(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("N", ctypes.c_int32), ("n_alpha", ctypes.c_int32),
                ("n_beta", ctypes.c_int32), ("num_coordinates", ctypes.c_int32), ("have_prev", ctypes.c_int32),
                ("done", ctypes.c_int32), ("has_best", ctypes.c_int32), ("n_entries", ctypes.c_int64),
                ("mu", ctypes.c_double * 2), ("alpha", ctypes.c_double * 2), ("scale", ctypes.c_double * 2),
                ("dx", ctypes.c_double), ("energy", ctypes.c_double), ("last_gamma", ctypes.c_double),
                ("iterations", ctypes.c_int64), ("nnz_c", ctypes.c_int64), ("n_slots", ctypes.c_int64),
                ("elements", ctypes.c_int64), ("applied", ctypes.c_int64), ("dropped", ctypes.c_int64),
                ("inserted", ctypes.c_int64), ("last_column", ctypes.c_int64), ("reduced_iterations", ctypes.c_int64),
                ("prev_key", ctypes.c_uint64 * 2), ("prev_c", ctypes.c_double), ("prev_Hii", ctypes.c_double),
                ("prev_eta", ctypes.c_double), ("prev_mu_g", ctypes.c_double),
                ("best_key", ctypes.c_uint64 * 2), ("best_gbits", ctypes.c_uint64), ("best_b", ctypes.c_double),
                ("best_c", ctypes.c_double), ("gather", ctypes.c_double), ("pending", ctypes.c_int64 * 4),
                ("pending_err", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class CdfciError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libcdfci error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded libcdfci (raises if the CUDA library was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, u64p, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
        L.cdfci_default_params.argtypes = [ctypes.POINTER(cdfci_params)]
        L.cdfci_default_params.restype = None
        L.cdfci_create.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cdfci_params),
                                   ctypes.POINTER(vp)]
        L.cdfci_step.argtypes = [vp, i64, ctypes.POINTER(cdfci_stats)]
        L.cdfci_get_stats.argtypes = [vp, ctypes.POINTER(cdfci_stats)]
        L.cdfci_energy.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.cdfci_energy_with.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_double)]
        L.cdfci_get_column.argtypes = [vp, u64p, u64p, dp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.cdfci_export.argtypes = [vp, u64p, dp, dp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.cdfci_rdm.argtypes = [vp, dp, dp]
        L.cdfci_autotune.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cdfci_params),
                                     ctypes.c_double, ctypes.POINTER(cdfci_tune_report)]
        L.cdfci_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.cdfci_batch_step.argtypes = [vp, i64, ctypes.POINTER(cdfci_stats)]
        L.cdfci_batch_destroy.argtypes = [vp]
        L.cdfci_batch_destroy.restype = None
        L.cdfci_gradient.argtypes = [vp, dp, dp, dp]
        L.cdfci_last_step.argtypes = [vp, u64p, dp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.cdfci_column_noalloc.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, u64p, dp, i64,
                                           ctypes.POINTER(ctypes.c_int64), vp]
        L.cdfci_column_noalloc.restype = ctypes.c_int
        L.cdfci_set_initial.argtypes = [vp, u64p, dp, i64]
        L.cdfci_energies.argtypes = [vp, dp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.cdfci_time_kernels.argtypes = [vp, i64, dp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.cdfci_probe_slots.argtypes = [ctypes.c_void_p, ctypes.c_int, i64, ctypes.c_uint64, ctypes.c_void_p]
        L.cdfci_fcidump_header.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]
        L.cdfci_fcidump_read.argtypes = [ctypes.c_char_p, ctypes.c_double, ctypes.c_int, dp, dp,
                                         ctypes.POINTER(ctypes.c_double)]
        L.cdfci_get_entry.argtypes = [vp, u64p, u64p, ctypes.POINTER(ctypes.c_double)]
        L.cdfci_degenerate_set.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, i64, u64p,
                                           ctypes.POINTER(ctypes.c_int64)]
        L.cdfci_get_diagonal.argtypes = [vp, u64p, ctypes.POINTER(ctypes.c_double)]
        L.cdfci_create_hubbard_k.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(cdfci_params),
                                             ctypes.POINTER(vp)]
        L.cdfci_set_initial_degenerate.argtypes = [vp, ctypes.c_double, i64, ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.POINTER(ctypes.c_double)]
        L.cdfci_optorb.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                   ctypes.POINTER(cdfci_optorb_params), dp]
        L.cdfci_export_states.argtypes = [vp, u64p, dp, dp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.cdfci_checkpoint.argtypes = [vp, ctypes.POINTER(cdfci_checkpoint_header), u64p, dp, dp, ctypes.c_void_p, i64]
        L.cdfci_restore.argtypes = [vp, ctypes.POINTER(cdfci_checkpoint_header), u64p, dp, dp, ctypes.c_void_p]
        L.cdfci_destroy.argtypes = [vp]
        L.cdfci_destroy.restype = None
        L.cdfci_last_error.argtypes = []
        L.cdfci_last_error.restype = ctypes.c_char_p
        for name in ("cdfci_create", "cdfci_step", "cdfci_get_stats", "cdfci_energy", "cdfci_get_column",
                     "cdfci_export", "cdfci_last_step"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != CDFCI_OK:
        raise CdfciError(rc, lib().cdfci_last_error().decode())


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def cdfci_default_params(**overrides) -> cdfci_params:
    p = cdfci_params()
    lib().cdfci_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def cdfci_create(h, g, N: int, n_alpha: int, n_beta: int, params: Optional[cdfci_params] = None) -> int:
    handle = ctypes.c_void_p()
    p = params if params is not None else cdfci_default_params()
    _check(lib().cdfci_create(_ptr(h), _ptr(g), N, n_alpha, n_beta, ctypes.byref(p), ctypes.byref(handle)))
    return handle.value


def cdfci_create_hubbard_k(shape, t: float, U: float, n_alpha: int, n_beta: int,
                           params: Optional[cdfci_params] = None) -> int:
    """The k-space Hubbard model built by the library (plane waves, momentum tables)."""
    dims = np.ascontiguousarray(shape, dtype=np.int32).reshape(-1)
    handle = ctypes.c_void_p()
    p = params if params is not None else cdfci_default_params()
    _check(lib().cdfci_create_hubbard_k(dims.ctypes.data, len(dims), float(t), float(U), int(n_alpha), int(n_beta),
                                        ctypes.byref(p), ctypes.byref(handle)))
    return handle.value


def cdfci_degenerate_set(eps, n_alpha: int, n_beta: int, tol: float = 0.0, cap: int = 0) -> np.ndarray:
    """The determinants of lowest one-body energy (host only): (n, 2) keys {A, B} in the library's order."""
    e = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1)
    n = ctypes.c_int64(0)
    cap = int(cap) if cap > 0 else 1024
    keys = np.zeros((cap, 2), dtype=np.uint64)
    _check(lib().cdfci_degenerate_set(e.ctypes.data, len(e), int(n_alpha), int(n_beta), float(tol), cap,
                                      keys.ctypes.data, ctypes.byref(n)))
    return keys[:n.value].copy()


def cdfci_get_entry(handle: int, row_key, col_key) -> float:
    """H_{row, col} (Eq. entry), the get_entry of the Hamiltonian interface."""
    r = np.ascontiguousarray(np.asarray(row_key, dtype=np.uint64).reshape(2))
    c = np.ascontiguousarray(np.asarray(col_key, dtype=np.uint64).reshape(2))
    v = ctypes.c_double()
    _check(lib().cdfci_get_entry(handle, r.ctypes.data, c.ctypes.data, ctypes.byref(v)))
    return v.value


def cdfci_get_diagonal(handle: int, key) -> float:
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    v = ctypes.c_double()
    _check(lib().cdfci_get_diagonal(handle, k.ctypes.data, ctypes.byref(v)))
    return v.value


def cdfci_step(handle: int, n_iter: int) -> dict:
    s = cdfci_stats()
    _check(lib().cdfci_step(handle, int(n_iter), ctypes.byref(s)))
    return s.as_dict()


def cdfci_get_stats(handle: int) -> dict:
    s = cdfci_stats()
    _check(lib().cdfci_get_stats(handle, ctypes.byref(s)))
    return s.as_dict()


def cdfci_energy_with(handle: int, h, g) -> float:
    """Exact Rayleigh quotient of the stored vector under the integrals h, g (same space)."""
    h = np.ascontiguousarray(h, dtype=np.float64) if isinstance(h, np.ndarray) else h
    g = np.ascontiguousarray(g, dtype=np.float64) if isinstance(g, np.ndarray) else g
    E = ctypes.c_double()
    _check(lib().cdfci_energy_with(handle, _ptr(h), _ptr(g), ctypes.byref(E)))
    return E.value


def cdfci_energy(handle: int, mode: int = 0) -> float:
    e = ctypes.c_double()
    _check(lib().cdfci_energy(handle, int(mode), ctypes.byref(e)))
    return e.value


def cdfci_get_column(handle: int, key, cap: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray]:
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    n = ctypes.c_int64()
    if cap is None:
        rc = lib().cdfci_get_column(handle, _ptr(k), None, None, 0, ctypes.byref(n))
        if rc not in (CDFCI_OK, -8):
            _check(rc)
        cap = n.value
    keys = np.zeros((max(cap, 1), 2), dtype=np.uint64)
    vals = np.zeros(max(cap, 1))
    _check(lib().cdfci_get_column(handle, _ptr(k), _ptr(keys), _ptr(vals), cap, ctypes.byref(n)))
    return keys[:n.value], vals[:n.value]


def cdfci_export(handle: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    n = ctypes.c_int64()
    rc = lib().cdfci_export(handle, None, None, None, 0, ctypes.byref(n))
    if rc not in (CDFCI_OK, -8):
        _check(rc)
    cap = n.value
    keys = np.zeros((max(cap, 1), 2), dtype=np.uint64)
    c = np.zeros(max(cap, 1))
    b = np.zeros(max(cap, 1))
    _check(lib().cdfci_export(handle, _ptr(keys), _ptr(c), _ptr(b), cap, ctypes.byref(n)))
    return keys[:n.value], c[:n.value], b[:n.value]


def cdfci_optorb(h, g, M: int, N: int, n_alpha: int, n_beta: int, U0=None, outer: int = 4, bb_steps: int = 20,
                 inner_iterations: int = 20000, **fci) -> Tuple[np.ndarray, np.ndarray]:
    """OptOrbFCI (Algorithm 4): returns the final U (M x N) and E_0 of each outer iteration."""
    p = cdfci_optorb_params()
    p.outer, p.bb_steps, p.inner_iterations = outer, bb_steps, inner_iterations
    p.fci = cdfci_default_params(**fci)
    U = np.ascontiguousarray(np.eye(M)[:, :N] if U0 is None else U0, dtype=np.float64).copy()
    E = np.zeros(outer)
    h = np.ascontiguousarray(h, dtype=np.float64) if isinstance(h, np.ndarray) else h
    g = np.ascontiguousarray(g, dtype=np.float64) if isinstance(g, np.ndarray) else g
    _check(lib().cdfci_optorb(_ptr(h), _ptr(g), M, N, n_alpha, n_beta, _ptr(U), ctypes.byref(p), _ptr(E)))
    return U, E


def cdfci_set_initial_degenerate(handle: int, tol: float = 0.0, cap: int = 0) -> Tuple[int, float]:
    """Degenerate-subspace start; returns (number of degenerate determinants, lowest eigenvalue on them)."""
    n = ctypes.c_int64(0)
    E = ctypes.c_double(0.0)
    _check(lib().cdfci_set_initial_degenerate(handle, float(tol), int(cap), ctypes.byref(n), ctypes.byref(E)))
    return int(n.value), float(E.value)


MC_KERNELS = ["gkeys", "hist", "collect", "sortsel", "prepare", "eigen", "scatter", "finalize"]


def cdfci_fcidump_header(path: str) -> Tuple[int, int, int]:
    """(NORB, NELEC, MS2) of an FCIDUMP file's header."""
    n, ne, m2 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().cdfci_fcidump_header(os.fsencode(path), ctypes.byref(n), ctypes.byref(ne), ctypes.byref(m2)))
    return n.value, ne.value, m2.value


def cdfci_fcidump_read(path: str, threshold: float = 0.0) -> dict:
    """An FCIDUMP file as {h, g, N, n_alpha, n_beta, e_core} (values below `threshold` in magnitude
    stored as 0)."""
    N, ne, m2 = cdfci_fcidump_header(path)
    h = np.zeros((N, N))
    g = np.zeros((N, N, N, N))
    core = ctypes.c_double()
    _check(lib().cdfci_fcidump_read(os.fsencode(path), float(threshold), N, h.ctypes.data, g.ctypes.data,
                                    ctypes.byref(core)))
    return {"h": h, "g": g, "N": N, "n_alpha": (ne + m2) // 2, "n_beta": (ne - m2) // 2, "e_core": core.value}


def cdfci_probe_slots(table, log2_slots: int, n_ops: int, seed: int = 1, stream: int = 0) -> None:
    """Queue the random-slot probe on `stream` over the caller's device table (measurement only)."""
    _check(lib().cdfci_probe_slots(_ptr(table), int(log2_slots), int(n_ops), int(seed), stream))


def cdfci_time_kernels(handle: int, n_iter: int) -> dict:
    """Milliseconds per launch of the mCDFCI iteration, summed over n_iter iterations (which advance the solve)."""
    ms = np.zeros(len(MC_KERNELS), dtype=np.float64)
    n = ctypes.c_int32(0)
    _check(lib().cdfci_time_kernels(handle, int(n_iter), _ptr(ms), len(MC_KERNELS), ctypes.byref(n)))
    return dict(zip(MC_KERNELS, ms.tolist()))


def cdfci_energies(handle: int, cap: int = 8) -> np.ndarray:
    """The K + 1 energies of an xCDFCI handle (ascending); one for other handles."""
    E = np.zeros(cap)
    n = ctypes.c_int32()
    _check(lib().cdfci_energies(handle, _ptr(E), cap, ctypes.byref(n)))
    return E[:n.value].copy()


def cdfci_export_states(handle: int, k1: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Keys (n, 2) and rows C, B (n, k1) of every stored determinant."""
    n = ctypes.c_int64()
    rc = lib().cdfci_export_states(handle, None, None, None, 0, ctypes.byref(n))
    if rc not in (CDFCI_OK, -8):
        _check(rc)
    cap = n.value
    keys = np.zeros((max(cap, 1), 2), dtype=np.uint64)
    C = np.zeros((max(cap, 1), k1))
    B = np.zeros((max(cap, 1), k1))
    _check(lib().cdfci_export_states(handle, _ptr(keys), _ptr(C), _ptr(B), cap, ctypes.byref(n)))
    return keys[:n.value], C[:n.value], B[:n.value]


def cdfci_set_initial(handle: int, keys, c) -> None:
    """Start vector: keys (n, 2) uint64 {A, B}, c (n,) float64 (host arrays or device tensors)."""
    if isinstance(keys, np.ndarray):
        keys = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    if isinstance(c, np.ndarray):
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
    n = int(c.shape[0])
    _check(lib().cdfci_set_initial(handle, _ptr(keys), _ptr(c), n))


def cdfci_checkpoint(handle: int) -> dict:
    """The state between steps: {"header": cdfci_checkpoint_header, "keys", "c", "b", "flags"} (c, b as stored)."""
    hdr = cdfci_checkpoint_header()
    rc = lib().cdfci_checkpoint(handle, ctypes.byref(hdr), None, None, None, None, 0)
    if rc not in (CDFCI_OK, -8):
        _check(rc)
    n = int(hdr.n_entries)
    keys = np.zeros((max(n, 1), 2), dtype=np.uint64)
    c = np.zeros(max(n, 1))
    b = np.zeros(max(n, 1))
    flags = np.zeros(max(n, 1), dtype=np.uint8)
    _check(lib().cdfci_checkpoint(handle, ctypes.byref(hdr), _ptr(keys), _ptr(c), _ptr(b), _ptr(flags), n))
    return {"header": hdr, "keys": keys[:n], "c": c[:n], "b": b[:n], "flags": flags[:n]}


def cdfci_restore(handle: int, ckpt: dict) -> None:
    keys = np.ascontiguousarray(ckpt["keys"], dtype=np.uint64)
    c = np.ascontiguousarray(ckpt["c"], dtype=np.float64)
    b = np.ascontiguousarray(ckpt["b"], dtype=np.float64)
    flags = ckpt.get("flags")
    flags = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
    hdr = ckpt["header"]
    _check(lib().cdfci_restore(handle, ctypes.byref(hdr), _ptr(keys), _ptr(c), _ptr(b), _ptr(flags)))


def save_checkpoint(path: str, ckpt: dict) -> None:
    """Writes a checkpoint as .npz: the header's raw bytes and the rows."""
    np.savez(path, header=np.frombuffer(bytes(ckpt["header"]), dtype=np.uint8), keys=ckpt["keys"], c=ckpt["c"],
             b=ckpt["b"], flags=ckpt["flags"])


def load_checkpoint(path: str) -> dict:
    with np.load(path) as z:
        raw = z["header"].tobytes()
        if len(raw) != ctypes.sizeof(cdfci_checkpoint_header):
            raise ValueError("checkpoint header has the wrong size")
        hdr = cdfci_checkpoint_header.from_buffer_copy(raw)
        return {"header": hdr, "keys": z["keys"].copy(), "c": z["c"].copy(), "b": z["b"].copy(),
                "flags": z["flags"].copy()}


def cdfci_autotune(h, g, N: int, n_alpha: int, n_beta: int, seconds: float = 2.0, **params) -> Tuple[dict, dict]:
    """Picks num_coordinates by the measured energy decrease per second; returns
    (the tuned params as a dict, the report)."""
    p = cdfci_default_params(**params)
    rep = cdfci_tune_report()
    h = np.ascontiguousarray(h, dtype=np.float64) if isinstance(h, np.ndarray) else h
    g = np.ascontiguousarray(g, dtype=np.float64) if isinstance(g, np.ndarray) else g
    _check(lib().cdfci_autotune(_ptr(h), _ptr(g), N, n_alpha, n_beta, ctypes.byref(p), float(seconds), ctypes.byref(rep)))
    tuned = dict(params, num_coordinates=p.num_coordinates, grid_blocks=p.grid_blocks)
    report = {"chosen_m": rep.m[rep.chosen], "chosen_grid_blocks": rep.grid_blocks[rep.chosen],
              "m": list(rep.m[:rep.n]), "grid_blocks": list(rep.grid_blocks[:rep.n]),
              "iterations": list(rep.iterations[:rep.n]),
              "seconds": list(rep.seconds[:rep.n]), "energy_drop": list(rep.energy_drop[:rep.n]),
              "score": list(rep.score[:rep.n])}
    return tuned, report


def cdfci_rdm(handle: int, N: int, two_body: bool = True) -> Tuple[np.ndarray, Optional[np.ndarray]]:
    """Spin-summed gamma (N, N) and Gamma (N, N, N, N) of the current vector."""
    g1 = np.zeros((N, N))
    g2 = np.zeros((N, N, N, N)) if two_body else None
    _check(lib().cdfci_rdm(handle, _ptr(g1), _ptr(g2) if two_body else None))
    return g1, g2


def cdfci_gradient(handle: int, N: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """dE/dh (N, N), dE/dg (N, N, N, N) and dE/dkappa (N, N) of the current vector."""
    dh, dg, dk = np.zeros((N, N)), np.zeros((N, N, N, N)), np.zeros((N, N))
    _check(lib().cdfci_gradient(handle, _ptr(dh), _ptr(dg), _ptr(dk)))
    return dh, dg, dk


def cdfci_last_step(handle: int, cap: int = 1024) -> Tuple[np.ndarray, np.ndarray]:
    keys = np.zeros((cap, 2), dtype=np.uint64)
    eta = np.zeros(cap)
    m = ctypes.c_int64()
    _check(lib().cdfci_last_step(handle, _ptr(keys), _ptr(eta), cap, ctypes.byref(m)))
    return keys[:m.value], eta[:m.value]


def cdfci_column_noalloc(h, g, N: int, n_alpha: int, n_beta: int, key, keys_out, vals_out, cap: int,
                         stream: int = 0) -> int:
    """get_column for callers that cannot allocate device memory: h, g, keys_out and
    vals_out are device tensors the caller owns; returns the column length."""
    n = ctypes.c_int64()
    _check(lib().cdfci_column_noalloc(_ptr(h), _ptr(g), N, n_alpha, n_beta, _ptr(key), _ptr(keys_out),
                                      _ptr(vals_out), int(cap), ctypes.byref(n), stream))
    return n.value


def cdfci_destroy(handle: int) -> None:
    if handle:
        lib().cdfci_destroy(handle)


def cdfci_last_error() -> str:
    return lib().cdfci_last_error().decode()


class Solver:
    """Owning wrapper around a handle (convenience for tests and the benchmark)."""

    def __init__(self, h, g, N, n_alpha, n_beta, **params):
        self.N = N
        self.p = cdfci_default_params(**params)
        self.handle = cdfci_create(np.ascontiguousarray(h, dtype=np.float64) if isinstance(h, np.ndarray) else h,
                                   np.ascontiguousarray(g, dtype=np.float64) if isinstance(g, np.ndarray) else g,
                                   N, n_alpha, n_beta, self.p)

    @classmethod
    def hubbard_k(cls, shape, n_alpha: int, n_beta: int, t: float = 1.0, U: float = 4.0, **params) -> "Solver":
        """A solver of the k-space Hubbard model built by the library (cdfci_create_hubbard_k)."""
        self = cls.__new__(cls)
        self.N = int(np.prod(shape))
        self.p = cdfci_default_params(**params)
        self.handle = cdfci_create_hubbard_k(shape, t, U, n_alpha, n_beta, self.p)
        return self

    def step(self, n: int) -> dict:
        return cdfci_step(self.handle, n)

    def stats(self) -> dict:
        return cdfci_get_stats(self.handle)

    def energy(self, mode: int = 0) -> float:
        return cdfci_energy(self.handle, mode)

    def energy_with(self, h, g) -> float:
        return cdfci_energy_with(self.handle, h, g)

    def entry(self, row_key, col_key) -> float:
        return cdfci_get_entry(self.handle, row_key, col_key)

    def diagonal(self, key) -> float:
        return cdfci_get_diagonal(self.handle, key)

    def column(self, key):
        return cdfci_get_column(self.handle, key)

    def export(self):
        return cdfci_export(self.handle)

    def last_step(self):
        return cdfci_last_step(self.handle)

    def rdm(self, two_body: bool = True):
        return cdfci_rdm(self.handle, self.N, two_body)

    def set_initial(self, keys, c):
        cdfci_set_initial(self.handle, keys, c)

    def energies(self) -> np.ndarray:
        return cdfci_energies(self.handle)

    def time_kernels(self, n_iter: int) -> dict:
        return cdfci_time_kernels(self.handle, n_iter)

    def set_initial_degenerate(self, tol: float = 0.0, cap: int = 0) -> Tuple[int, float]:
        return cdfci_set_initial_degenerate(self.handle, tol, cap)

    def export_states(self):
        return cdfci_export_states(self.handle, max(1, int(self.p.num_states)))

    def checkpoint(self) -> dict:
        return cdfci_checkpoint(self.handle)

    def restore(self, ckpt: dict):
        cdfci_restore(self.handle, ckpt)

    def gradient(self):
        return cdfci_gradient(self.handle, self.N)

    def close(self):
        if self.handle:
            cdfci_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many solvers stepped together (cdfci_batch_*): the m = 1 ones in one persistent launch, the
    m > 1 ones as branches of one graph; does not own them."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[sv.handle for sv in self.solvers])
        out = ctypes.c_void_p()
        _check(lib().cdfci_batch_create(arr, len(self.solvers), ctypes.byref(out)))
        self.handle = out.value

    def step(self, n: int):
        st = (cdfci_stats * len(self.solvers))()
        _check(lib().cdfci_batch_step(self.handle, int(n), st))
        return [x.as_dict() for x in st]

    def close(self):
        if self.handle:
            lib().cdfci_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

