"""CPU oracle for the CDFCI column update (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never calls it.

The numerical core is ``cdfci_oracle.c`` (plain serial C, FP64 with binary128
scalars), loaded with ctypes:

  * ``column_literal``  - <D'|H|D> by literal ladder-operator application of
    Eq. (general-ham); the definition of a column.
  * ``column_sc``       - the Slater-Condon rules of Eq. (entry).
  * ``dense_H`` / ``sparse_H`` - H on a whole FCI space.
  * ``ground_energy``   - smallest eigenvalue of H (LAPACK ``eigh`` on the dense
    matrix, or ARPACK ``eigsh`` on the sparse one: library eigensolvers used
    as one step).
  * ``degenerate_start`` - the lowest eigenvector of H on the degenerate
    lowest one-body configurations (the k-space Hubbard start).
  * ``CDFCI``           - Algorithm 1 (m = 1) and Algorithm 2 (m > 1), serial.
  * ``line_search``     - the appendix's Cardano + Newton step.
  * ``rdm``             - spin-summed 1- and 2-RDMs by literal operator
    application (Sec. "Optimal Orbital Selections").
  * ``rotate_integrals`` / ``orbital_gradient`` - h, g in rotated orbitals
    U = exp(kappa) and the energy's derivative with respect to kappa, from
    the RDMs (Sec. "Optimal Orbital Selections", the rotated-integral energy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdfci_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

c_dp = ctypes.POINTER(ctypes.c_double)
c_u64p = ctypes.POINTER(ctypes.c_uint64)
c_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle's C core into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_column_literal.restype = ctypes.c_int64
        L.orc_column_literal.argtypes = [ctypes.c_int, c_dp, c_dp, ctypes.c_uint64, ctypes.c_uint64, c_u64p, c_dp, ctypes.c_int64]
        L.orc_column_sc.restype = ctypes.c_int64
        L.orc_column_sc.argtypes = L.orc_column_literal.argtypes
        L.orc_diag.restype = ctypes.c_double
        L.orc_diag.argtypes = [ctypes.c_int, c_dp, c_dp, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_fci_dim.restype = ctypes.c_int64
        L.orc_fci_dim.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_fci_dets.restype = ctypes.c_int
        L.orc_fci_dets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_u64p]
        L.orc_fci_index.restype = ctypes.c_int64
        L.orc_fci_index.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_dense_H.restype = ctypes.c_int
        L.orc_dense_H.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_dp, c_dp]
        L.orc_sparse_H.restype = ctypes.c_int64
        L.orc_sparse_H.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_dp, c_i64p, c_i64p, c_dp, ctypes.c_int64]
        L.orc_line_search.restype = ctypes.c_double
        L.orc_line_search.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_sym_eig.restype = ctypes.c_int
        L.orc_sym_eig.argtypes = [ctypes.c_int, c_dp, c_dp, c_dp]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_dp, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_double]
        L.orc_destroy.restype = None
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_energy.restype = ctypes.c_double
        L.orc_energy.argtypes = [ctypes.c_void_p]
        L.orc_info.restype = None
        L.orc_info.argtypes = [ctypes.c_void_p, c_dp]
        L.orc_export.restype = ctypes.c_int64
        L.orc_export.argtypes = [ctypes.c_void_p, c_u64p, c_dp, c_dp, ctypes.c_int64]
        L.orc_last_step.restype = ctypes.c_int64
        L.orc_last_step.argtypes = [ctypes.c_void_p, c_u64p, c_dp, ctypes.c_int64]
        L.orc_candidates.restype = ctypes.c_int64
        L.orc_candidates.argtypes = [ctypes.c_void_p, c_u64p, ctypes.c_int64]
        L.orc_step_choice.restype = ctypes.c_int
        L.orc_step_choice.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, c_dp, c_dp]
        L.orx_create.restype = ctypes.c_void_p
        L.orx_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_dp, c_u64p, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double]
        L.orx_destroy.restype = None
        L.orx_destroy.argtypes = [ctypes.c_void_p]
        L.orx_step.restype = ctypes.c_int
        L.orx_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orx_energies.restype = ctypes.c_int
        L.orx_energies.argtypes = [ctypes.c_void_p, c_dp]
        L.orx_info.restype = None
        L.orx_info.argtypes = [ctypes.c_void_p, c_dp, c_dp, c_dp]
        L.orx_export.restype = ctypes.c_int64
        L.orx_export.argtypes = [ctypes.c_void_p, c_u64p, c_dp, c_dp, ctypes.c_int64]
        L.orx_last_step.restype = None
        L.orx_last_step.argtypes = [ctypes.c_void_p, c_u64p, c_dp]
        L.orx_quartic.restype = None
        L.orx_quartic.argtypes = [ctypes.c_int, c_dp, c_dp, c_dp, ctypes.c_double, c_dp]
        L.orc_set_initial.restype = ctypes.c_int
        L.orc_set_initial.argtypes = [ctypes.c_void_p, c_u64p, c_dp, ctypes.c_int64]
        L.orc_rdm.restype = ctypes.c_int
        L.orc_rdm.argtypes = [ctypes.c_int, ctypes.c_int64, c_u64p, c_dp, c_dp, c_dp]
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(c_dp)


def _u(a: np.ndarray):
    return a.ctypes.data_as(c_u64p)


def _ints(h, g):
    h = np.ascontiguousarray(h, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    return h, g


def _column(fn, N, h, g, key) -> Tuple[np.ndarray, np.ndarray]:
    h, g = _ints(h, g)
    cap = 1 << 12
    while True:
        keys = np.zeros((cap, 2), dtype=np.uint64)
        vals = np.zeros(cap)
        n = fn(N, _d(h), _d(g), int(key[0]), int(key[1]), _u(keys), _d(vals), cap)
        if n >= 0:
            return keys[:n].copy(), vals[:n].copy()
        if n == -1:
            raise MemoryError("oracle column failed")
        cap = -n


def column_literal(N, h, g, key):
    """All (D', <D'|H|D>) with a nonzero value, by literal operator application."""
    return _column(lib().orc_column_literal, N, h, g, key)


def column_sc(N, h, g, key):
    """All (D', H_{D'D}) with a nonzero value, by the Slater-Condon rules of Eq. (entry)."""
    return _column(lib().orc_column_sc, N, h, g, key)


def diag(N, h, g, key) -> float:
    h, g = _ints(h, g)
    return lib().orc_diag(N, _d(h), _d(g), int(key[0]), int(key[1]))


def fci_dim(N, na, nb) -> int:
    return int(lib().orc_fci_dim(N, na, nb))


def fci_dets(N, na, nb) -> np.ndarray:
    dim = fci_dim(N, na, nb)
    keys = np.zeros((dim, 2), dtype=np.uint64)
    lib().orc_fci_dets(N, na, nb, _u(keys))
    return keys


def fci_index(N, na, nb, key) -> int:
    return int(lib().orc_fci_index(N, na, nb, int(key[0]), int(key[1])))


def dense_H(N, na, nb, h, g) -> np.ndarray:
    h, g = _ints(h, g)
    dim = fci_dim(N, na, nb)
    H = np.zeros((dim, dim))
    if lib().orc_dense_H(N, na, nb, _d(h), _d(g), _d(H)):
        raise MemoryError("oracle dense_H failed")
    return H


def sparse_H(N, na, nb, h, g):
    import scipy.sparse as sp
    h, g = _ints(h, g)
    dim = fci_dim(N, na, nb)
    cap = max(1024, dim * 64)
    while True:
        rows = np.zeros(cap, dtype=np.int64)
        cols = np.zeros(cap, dtype=np.int64)
        vals = np.zeros(cap)
        n = lib().orc_sparse_H(N, na, nb, _d(h), _d(g), rows.ctypes.data_as(c_i64p),
                               cols.ctypes.data_as(c_i64p), _d(vals), cap)
        if n >= 0:
            return sp.csr_matrix((vals[:n], (rows[:n], cols[:n])), shape=(dim, dim))
        if n == -1:
            raise MemoryError("oracle sparse_H failed")
        cap = -n


def ground_energy(N, na, nb, h, g, dense_limit: int = 2500) -> float:
    """Smallest eigenvalue of H over the FCI space (dense LAPACK or sparse ARPACK)."""
    dim = fci_dim(N, na, nb)
    if dim <= dense_limit:
        return float(np.linalg.eigvalsh(dense_H(N, na, nb, h, g))[0])
    from scipy.sparse.linalg import eigsh
    Hs = sparse_H(N, na, nb, h, g)
    w = eigsh(Hs, k=1, which="SA", tol=1e-14, ncv=min(dim - 1, 64), maxiter=100000,
              v0=np.ones(dim) / np.sqrt(dim))[0]
    return float(w[0])


def degenerate_start(N, na, nb, h, g, tol: float = 1e-10, cap: int = 1024):
    """The degenerate-subspace start of the paper's k-space Hubbard example (numerical section, 4x4
    lattice: the configurations of lowest one-body energy, the Hamiltonian restricted to them, its
    lowest eigenvector).  Per spin the orbitals below the ne-th lowest level h_pp are filled and
    every choice of the remaining electrons in that level's shell (levels within tol * max(1, |level|))
    is listed.  S = alpha x beta choices ordered by the 128-bit key (B << 64) | A; H_SS from
    column_sc; its eigenpairs from numpy's eigh.  When the lowest eigenvalue is degenerate (the 4x4
    lattice: 4-fold, over two total-momentum sectors) "the" eigenvector is any vector of its
    eigenspace; the start is the projection onto that eigenspace of the ramp r_s = 1 + s / |S|, which
    has a component in every sector of it (an arbitrary basis vector can lie in one sector only, and H
    conserves momentum).  The vector normalised, its largest component positive (ties: the first in
    S).  Returns (keys (|S|, 2), c, lowest eigenvalue)."""
    import itertools
    eps = np.diag(np.asarray(h, dtype=np.float64))

    def strings(ne):
        if ne == 0:
            return [0]
        top = sorted(eps)[ne - 1]
        band = tol * max(1.0, abs(top))
        below = [p for p in range(N) if eps[p] < top - band]
        shell = [p for p in range(N) if top - band <= eps[p] <= top + band]
        r = ne - len(below)
        base = sum(1 << p for p in below)
        return [base | sum(1 << p for p in pick) for pick in itertools.combinations(shell, r)]

    sa, sb = strings(na), strings(nb)
    if len(sa) * len(sb) > cap:
        raise ValueError(f"degenerate set of {len(sa) * len(sb)} determinants exceeds cap = {cap}")
    S = sorted((b, a) for a in sa for b in sb)
    index = {k: i for i, k in enumerate(S)}
    n = len(S)
    H = np.zeros((n, n))
    for i, (b, a) in enumerate(S):
        keys, vals = column_sc(N, h, g, (a, b))
        for (ka, kb), v in zip(keys, vals):
            j = index.get((int(kb), int(ka)))
            if j is not None:
                H[j, i] = v
    H = 0.5 * (H + H.T)
    w, V = np.linalg.eigh(H)
    # the lowest eigenvalue's whole eigenspace (eigenvalues within 1e-9 of it, relative): the start
    # is the projection onto it of the ramp r_s = 1 + s / |S| (s = position in S); for a simple
    # eigenvalue that is the eigenvector itself
    lo = w[0]
    k = int(np.sum(w <= lo + 1e-9 * max(1.0, abs(lo))))
    ramp = 1.0 + np.arange(n) / n
    v = V[:, :k] @ (V[:, :k].T @ ramp)
    v = v / np.linalg.norm(v)
    big = int(np.argmax(np.abs(v)))
    if v[big] < 0:
        v = -v
    keys = np.array([[a, b] for (b, a) in S], dtype=np.uint64)
    return keys, v, float(lo)


def line_search(v1: float, v2: float, v3: float) -> float:
    """argmin_eta eta^4 + v3 eta^3 + v2 eta^2 + v1 eta (appendix: Cardano + Newton)."""
    return float(lib().orc_line_search(v1, v2, v3))


def sym_eig(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib().orc_sym_eig(n, _d(A), _d(w), _d(V))
    return w, V


def rdm(N: int, keys: np.ndarray, c: np.ndarray):
    """Spin-summed gamma[p,q] = sum_s <a+_ps a_qs> / c.c and
    Gamma[p,q,r,s] = sum_{st} <a+_ps a+_rt a_st a_qs> / c.c (chemists' index order,
    so that E = sum h gamma + 1/2 sum (pq|rs) Gamma)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    g1 = np.zeros((N, N))
    g2 = np.zeros((N, N, N, N))
    if lib().orc_rdm(N, len(c), _u(keys), _d(c), _d(g1), _d(g2)):
        raise MemoryError("oracle rdm failed")
    return g1, g2


class CDFCI:
    """Serial Algorithm 1 (m = 1) / Algorithm 2 (m > 1)."""

    def __init__(self, N, na, nb, h, g, ref=(0, 0), tau=0.0, m=1, theta=0.9):
        self.h, self.g = _ints(h, g)
        self.N, self.na, self.nb, self.m = N, na, nb, m
        self._p = lib().orc_create(N, na, nb, _d(self.h), _d(self.g), int(ref[0]), int(ref[1]),
                                   float(tau), int(m), float(theta))
        if not self._p:
            raise ValueError("oracle create failed")

    def step(self, n: int = 1):
        r = lib().orc_step(self._p, int(n))
        if r:
            raise RuntimeError(f"oracle step failed ({r})")

    def set_initial(self, keys, c):
        """Start vector sum_k c_k e_{keys k}, applied in order as steps with the given c_k (from c = 0)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
        r = lib().orc_set_initial(self._p, keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _d(c), len(c))
        if r:
            raise RuntimeError(f"oracle set_initial failed ({r})")

    def step_choice(self, key):
        """One Algorithm-1 step on the given coordinate; returns (|g| of it, max |g|) before the step."""
        gc = ctypes.c_double()
        gm = ctypes.c_double()
        r = lib().orc_step_choice(self._p, int(key[0]), int(key[1]), ctypes.byref(gc), ctypes.byref(gm))
        if r:
            raise RuntimeError(f"oracle step_choice failed ({r})")
        return gc.value, gm.value

    def energy(self) -> float:
        return float(lib().orc_energy(self._p))

    def info(self) -> dict:
        out = np.zeros(10)
        lib().orc_info(self._p, _d(out))
        k = ["mu", "alpha", "dx", "iterations", "entries", "nnz_c", "elements", "applied", "dropped",
             "degenerate_steps"]
        return {a: (float(v) if a in ("mu", "alpha", "dx") else int(v)) for a, v in zip(k, out)}

    def export(self):
        n = self.info()["entries"]
        keys = np.zeros((n, 2), dtype=np.uint64)
        c = np.zeros(n)
        b = np.zeros(n)
        lib().orc_export(self._p, _u(keys), _d(c), _d(b), n)
        return keys, c, b

    def last_step(self):
        cap = max(self.m, 1)
        keys = np.zeros((cap, 2), dtype=np.uint64)
        eta = np.zeros(cap)
        m = lib().orc_last_step(self._p, _u(keys), _d(eta), cap)
        return keys[:m].copy(), eta[:m].copy()

    def candidates(self):
        cap = 1 << 16
        while True:
            keys = np.zeros((cap, 2), dtype=np.uint64)
            n = lib().orc_candidates(self._p, _u(keys), cap)
            if n >= 0:
                return keys[:n].copy()
            cap = -n

    def close(self):
        if self._p:
            lib().orc_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rotate_integrals(h: np.ndarray, g: np.ndarray, kappa: np.ndarray):
    """Integrals in the orbitals (phi) = (psi) U with U = exp(kappa), kappa
    antisymmetric: h'_pq = sum_ab U_ap h_ab U_bq and
    g'_pqrs = sum_abcd U_ap U_bq U_cr U_ds g_abcd (Sec. "Optimal Orbital
    Selections"; the exponential is the library's matrix exponential)."""
    from scipy.linalg import expm
    U = expm(np.asarray(kappa, dtype=np.float64))
    h2 = U.T @ h @ U
    g2 = np.einsum("ap,bq,cr,ds,abcd->pqrs", U, U, U, U, g, optimize=True)
    return h2, g2


def orbital_gradient(h: np.ndarray, g: np.ndarray, g1: np.ndarray, g2: np.ndarray) -> np.ndarray:
    """dE/dkappa at kappa = 0 for E = sum h' gamma + 1/2 sum g' Gamma with the
    integrals rotated by U = exp(kappa): the antisymmetric 2 (F - F^T), with
    F_pq = sum_r h_pr gamma_qr + sum_rst (pr|st) Gamma_qrst, so that
    dE = 1/2 sum_pq G_pq dkappa_pq for an antisymmetric dkappa."""
    F = h @ g1.T + np.einsum("prst,qrst->pq", g, g2)
    return 2.0 * (F - F.T)


def xcd_quartic(c, g, S, Hii) -> np.ndarray:
    """w0..w4 of h(eta) = f(C + eta e_i g) - f(C) from the oracle (w0 = 0)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    w = np.zeros(5)
    lib().orx_quartic(len(c), _d(c), _d(g), _d(S), float(Hii), _d(w))
    return w


class XCDFCI:
    """Serial Algorithm 3 (xCDFCI) for k1 = K + 1 states from start determinants keys (k1, 2)."""

    def __init__(self, N, na, nb, h, g, keys, tau=0.0, theta=0.9):
        self.h, self.g = _ints(h, g)
        self.N, self.k1 = N, len(keys)
        self._keys = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
        self._p = lib().orx_create(N, na, nb, _d(self.h), _d(self.g),
                                   self._keys.ctypes.data_as(c_u64p), self.k1, float(tau), float(theta))
        if not self._p:
            raise ValueError("oracle xCDFCI create failed")

    def step(self, n: int = 1):
        r = lib().orx_step(self._p, int(n))
        if r:
            raise RuntimeError(f"oracle xCDFCI step failed ({r})")

    def energies(self) -> np.ndarray:
        E = np.zeros(self.k1)
        if lib().orx_energies(self._p, _d(E)):
            raise RuntimeError("S is not positive definite")
        return E

    def info(self) -> dict:
        S = np.zeros((self.k1, self.k1))
        M = np.zeros((self.k1, self.k1))
        out = np.zeros(6)
        lib().orx_info(self._p, _d(S), _d(M), _d(out))
        return {"S": S, "M": M, "dx": out[0], "iterations": int(out[1]), "entries": int(out[2]),
                "elements": int(out[3]), "applied": int(out[4]), "dropped": int(out[5])}

    def export(self):
        n = self.info()["entries"]
        keys = np.zeros((n, 2), dtype=np.uint64)
        C = np.zeros((n, self.k1))
        B = np.zeros((n, self.k1))
        lib().orx_export(self._p, keys.ctypes.data_as(c_u64p), _d(C), _d(B), n)
        return keys, C, B

    def last_step(self):
        k = np.zeros(2, dtype=np.uint64)
        e = ctypes.c_double()
        lib().orx_last_step(self._p, k.ctypes.data_as(c_u64p), ctypes.byref(e))
        return k, e.value

    def close(self):
        if self._p:
            lib().orx_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# OptOrbFCI (Algorithm 4): the orbital subproblem and the outer loop
# ---------------------------------------------------------------------------
def optorb_transform(h: np.ndarray, g: np.ndarray, U: np.ndarray):
    """Integrals in the orbitals (phi) = (psi) U, U of size M x N with orthonormal
    columns (Sec. "Optimal Orbital Selections"): h' = U^T h U, g'_pqrs = sum U_ap U_bq U_cr U_ds g_abcd."""
    return U.T @ h @ U, np.einsum("ap,bq,cr,ds,abcd->pqrs", U, U, U, U, g, optimize=True)


def optorb_objective(h, g, U, g1, g2) -> float:
    """P4(U) of the subproblem (eq. subopt) in the RDM convention E = sum h gamma + 1/2 sum (pq|rs) Gamma."""
    h2, gg = optorb_transform(h, g, U)
    return float(np.sum(h2 * g1) + 0.5 * np.sum(gg * g2))


def optorb_gradient(h, g, U, g1, g2) -> np.ndarray:
    """Euclidean gradient of P4 with respect to U (M x N): 2 h U gamma + 2 sum g''_pbcd Gamma_abcd,
    g''_pbcd = sum_jkl g_pjkl U_jb U_kc U_ld (the symmetries of g and Gamma make the four
    positions of U contribute alike)."""
    g3 = np.einsum("pjkl,jb,kc,ld->pbcd", g, U, U, U, optimize=True)
    return 2.0 * h @ U @ g1 + 2.0 * np.einsum("pbcd,abcd->pa", g3, g2, optimize=True)


def polar(X: np.ndarray) -> np.ndarray:
    """orth(X): the orthonormal factor of the polar decomposition (closest matrix with orthonormal columns)."""
    W, _, Vt = np.linalg.svd(X, full_matrices=False)
    return W @ Vt


def optorb_subproblem(h, g, U, g1, g2, steps: int):
    """Projected gradient with alternating Barzilai-Borwein steps (Algorithm 4, eq. projBB):
    U <- orth(U - t_k grad P4(U)), t_k = <S,S>/|<S,Y>| on odd and |<S,Y>|/<Y,Y> on even k
    (S, Y the last differences of U and of the gradient), t_0 = 0.1 / max(1, ||grad||_F).
    Returns the U with the lowest P4 met and the P4 history."""
    best_U, best_P = U, optorb_objective(h, g, U, g1, g2)
    hist = [best_P]
    G = optorb_gradient(h, g, U, g1, g2)
    t = 0.1 / max(1.0, np.linalg.norm(G))
    Uo, Go = None, None
    for k in range(steps):
        if Uo is not None:
            S, Y = U - Uo, G - Go
            ss, sy, yy = np.sum(S * S), np.sum(S * Y), np.sum(Y * Y)
            if abs(sy) > 0.0 and yy > 0.0:
                t = ss / abs(sy) if k % 2 == 1 else abs(sy) / yy
            t = min(max(t, 1e-10), 1e10)
        Uo, Go = U, G
        U = polar(U - t * G)
        G = optorb_gradient(h, g, U, g1, g2)
        P = optorb_objective(h, g, U, g1, g2)
        hist.append(P)
        if P < best_P:
            best_U, best_P = U, P
    return best_U, hist


def optorb_run(h, g, M: int, N: int, na: int, nb: int, outer: int, bb_steps: int, U0=None):
    """Algorithm 4 with the exact FCI solution of each basis (dense diagonalisation):
    returns the energies E_0 per outer iteration and the final U."""
    U = np.eye(M)[:, :N] if U0 is None else np.asarray(U0, dtype=np.float64)
    dets = fci_dets(N, na, nb)
    energies = []
    for _ in range(outer):
        h2, g2 = optorb_transform(h, g, U)
        w, V = np.linalg.eigh(dense_H(N, na, nb, h2, g2))
        energies.append(float(w[0]))
        r1, r2 = rdm(N, dets, V[:, 0].copy())
        U, _ = optorb_subproblem(h, g, U, r1, r2, bb_steps)
    return np.array(energies), U
