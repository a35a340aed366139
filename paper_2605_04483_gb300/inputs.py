"""Seeded synthetic workloads: one- and two-electron integrals and start determinants.

This module only draws and lays out inputs.  It evaluates no Hamiltonian
element, no step and no energy, so both the CUDA path and the CPU oracle can
take their inputs from it.

Layout (both sides read the same arrays):
  h : float64 (N, N), symmetric, h[p, q] = h_pq  (Eq. 1int)
  g : float64 (N, N, N, N), chemists' order g[p, q, r, s] = (pq|rs), exactly
      8-fold symmetric (every image of an element holds the same double), so
      that the physicists' v_pqrs = (pr|qs) of Eq. (2int) is well defined.
  A determinant is a pair of 64-bit words (A, B): bit p of A is spatial
  orbital p occupied with spin alpha, bit p of B with spin beta.

Workloads:
  * Hubbard lattices (Sec. "Hamiltonian Representations", Hubbard example):
    real-space site basis, h_ij = -t per bond, (ii|ii) = U.  A lattice
    dimension is periodic only when its extent is at least 3 (so that no bond
    appears twice).
  * Synthetic ab initio integrals: a diagonally dominant random h and a
    positive semidefinite Cholesky-type g = sum_k L^k (x) L^k, as a stand-in
    for the paper's molecular FCIDUMP integrals, which are not available.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    n_alpha: int
    n_beta: int
    h: np.ndarray
    g: np.ndarray
    ref: Tuple[int, int]          # (A, B); (0, 0) = let each side choose (aufbau on h_pp)
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def fci_dim(self) -> int:
        return math.comb(self.N, self.n_alpha) * math.comb(self.N, self.n_beta)


# ---------------------------------------------------------------------------
# Hubbard
# ---------------------------------------------------------------------------

def lattice_bonds(shape: Sequence[int], periodic: bool | Sequence[bool] = True) -> List[Tuple[int, int]]:
    """Nearest-neighbour bonds (i < j) of an orthogonal lattice, row-major site order."""
    shape = tuple(int(s) for s in shape)
    if isinstance(periodic, bool):
        periodic = [periodic] * len(shape)
    n_sites = int(np.prod(shape))
    bonds = set()
    for site in range(n_sites):
        coord = list(np.unravel_index(site, shape))
        for d, L in enumerate(shape):
            nxt = list(coord)
            if coord[d] + 1 < L:
                nxt[d] = coord[d] + 1
            elif periodic[d] and L >= 3:
                nxt[d] = 0
            else:
                continue
            j = int(np.ravel_multi_index(nxt, shape))
            a, b = min(site, j), max(site, j)
            if a != b:
                bonds.add((a, b))
    return sorted(bonds)


def hubbard_integrals(shape: Sequence[int], t: float, U: float,
                      periodic: bool | Sequence[bool] = True) -> Tuple[np.ndarray, np.ndarray]:
    N = int(np.prod(shape))
    h = np.zeros((N, N))
    for i, j in lattice_bonds(shape, periodic):
        h[i, j] = -t
        h[j, i] = -t
    g = np.zeros((N, N, N, N))
    for i in range(N):
        g[i, i, i, i] = U
    return h, g


def neel_reference(shape: Sequence[int], n_alpha: int, n_beta: int) -> Tuple[int, int]:
    """Checkerboard start: alpha fills even-parity sites first, beta odd-parity sites first."""
    N = int(np.prod(shape))
    parity = [int(sum(np.unravel_index(s, shape))) % 2 for s in range(N)]
    even = [s for s in range(N) if parity[s] == 0]
    odd = [s for s in range(N) if parity[s] == 1]
    A = 0
    for s in (even + odd)[:n_alpha]:
        A |= 1 << s
    B = 0
    for s in (odd + even)[:n_beta]:
        B |= 1 << s
    return A, B


def hubbard(shape: Sequence[int], n_alpha: int, n_beta: int, t: float = 1.0, U: float = 4.0,
            periodic: bool | Sequence[bool] = True, name: str | None = None) -> Workload:
    h, g = hubbard_integrals(shape, t, U, periodic)
    return Workload(name or f"hubbard{'x'.join(map(str, shape))}_U{U:g}", int(np.prod(shape)),
                    n_alpha, n_beta, h, g, neel_reference(shape, n_alpha, n_beta),
                    dict(kind="hubbard", shape=list(shape), t=t, U=U, periodic=periodic))


def momenta(shape: Sequence[int]) -> np.ndarray:
    """Integer momentum indices n (row-major, one row per plane wave); k_d = 2 pi n_d / L_d."""
    return np.array(list(np.ndindex(*tuple(int(x) for x in shape))), dtype=np.int64).reshape(-1, len(shape))


def hubbard_k_integrals(shape: Sequence[int], t: float, U: float) -> Tuple[np.ndarray, np.ndarray]:
    """The periodic Hubbard model in the plane-wave basis phi_k(x) = exp(i k.x) / sqrt(L), one orbital per
    momentum (the row order of momenta()).  h is diagonal: eps_k = sum_xy conj(phi_k(x)) h_xy phi_k(y) of the
    real-space hopping (so a length-2 direction keeps its single bond); the on-site U gives
    (pq|rs) = sum_x U conj(phi_p) phi_q conj(phi_r) phi_s = (U/L) delta(k_q - k_p + k_s - k_r), real, with
    only the symmetries (pq|rs) = (rs|pq) = (qp|sr)."""
    shape = tuple(int(x) for x in shape)
    L = int(np.prod(shape))
    n = momenta(shape)
    hr, _ = hubbard_integrals(shape, t, U, True)
    x = momenta(shape)                                  # site coordinates, same row-major order
    phase = 2.0 * np.pi * (x / np.array(shape, dtype=float)) @ n.T     # [site, k]
    P = np.exp(1j * phase) / np.sqrt(L)
    hk = P.conj().T @ hr @ P
    off = hk - np.diag(np.diag(hk))
    if np.max(np.abs(off)) > 1e-12 or np.max(np.abs(hk.imag)) > 1e-12:
        raise AssertionError("the hopping is not diagonal in the plane waves")
    # eps_k in closed form (-2t cos k_d per direction of extent >= 3, -t cos k_d for extent 2, the single
    # bond), equal to the transform above; rounded to 12 decimals so that equal levels (the degenerate
    # shells) are exactly equal
    eps = np.zeros(L)
    for d, Ld in enumerate(shape):
        k = 2.0 * np.pi * n[:, d] / Ld
        if Ld >= 3:
            eps += -2.0 * t * np.cos(k)
        elif Ld == 2:
            eps += -t * np.cos(k)
    if np.max(np.abs(eps - np.diag(hk).real)) > 1e-12:
        raise AssertionError("closed-form band differs from the transformed hopping")
    h = np.diag(np.round(eps, 12) + 0.0)
    dk = (-n[:, None, None, None, :] + n[None, :, None, None, :] - n[None, None, :, None, :]
          + n[None, None, None, :, :]) % np.array(shape)
    g = np.where(np.all(dk == 0, axis=-1), U / L, 0.0)
    return h, g


def hubbard_k(shape: Sequence[int], n_alpha: int, n_beta: int, t: float = 1.0, U: float = 4.0,
              name: str | None = None) -> Workload:
    """The k-space Hubbard model (HamiltonianHubbardK, periodic boundaries); a handle needs
    integral_symmetry = 4.  Start: aufbau on eps_k, or the degenerate-subspace start."""
    h, g = hubbard_k_integrals(shape, t, U)
    return Workload(name or f"hubbardk_{'x'.join(map(str, shape))}_U{U:g}", int(np.prod(shape)),
                    n_alpha, n_beta, h, g, (0, 0),
                    dict(kind="hubbard_k", shape=list(shape), t=t, U=U, periodic=True, integral_symmetry=4))


def config3_k(U: float = 4.0, n_alpha: int = 8, n_beta: int = 8) -> Workload:
    """The paper's own Hubbard setting: 4x4 periodic lattice in momentum space, t = 1 (half filling: 8 + 8)."""
    return hubbard_k((4, 4), n_alpha, n_beta, t=1.0, U=U, name=f"hubbardk_4x4_pbc_U{U:g}_{n_alpha}a{n_beta}b")


# ---------------------------------------------------------------------------
# Synthetic ab initio integrals
# ---------------------------------------------------------------------------

def _pair_index(N: int) -> np.ndarray:
    """P[p, q] = index of the unordered pair {p, q} among N(N+1)/2 pairs."""
    P = np.zeros((N, N), dtype=np.int64)
    k = 0
    for p in range(N):
        for q in range(p + 1):
            P[p, q] = P[q, p] = k
            k += 1
    return P


def synthetic_integrals(N: int, rng: np.random.Generator, n_chol: int = 48,
                        h_diag_mean: float = 2.0, h_diag_sd: float = 0.5, h_off_sd: float = 0.05,
                        l_sd: float = 0.1, l_decay: float = 6.0) -> Tuple[np.ndarray, np.ndarray]:
    """Draw order: h diagonal, h upper off-diagonal (row-major), then each L^k's upper triangle
    including the diagonal (row-major).  g is built from unique elements so that all eight
    index permutations hold bitwise-identical doubles."""
    h = np.zeros((N, N))
    x = rng.normal(h_diag_mean, h_diag_sd, size=N)
    for p in range(N):
        h[p, p] = -x[p] * (1.0 + p / N)
    iu = np.triu_indices(N, 1)
    off = rng.normal(0.0, h_off_sd, size=len(iu[0]))
    h[iu] = off
    h[(iu[1], iu[0])] = off
    iu0 = np.triu_indices(N, 0)
    decay = np.exp(-np.abs(iu0[0] - iu0[1]) / l_decay)
    n_pairs = N * (N + 1) // 2
    P = _pair_index(N)
    # L^k as a vector over unordered pairs (p <= q)
    M = np.zeros((n_chol, n_pairs))
    pair_of_upper = P[iu0]
    for k in range(n_chol):
        M[k, pair_of_upper] = rng.normal(0.0, l_sd, size=len(iu0[0])) * decay
    G = np.zeros((n_pairs, n_pairs))
    for k in range(n_chol):
        G += np.multiply.outer(M[k], M[k])      # exactly symmetric: same products, same order
    g = G[P[:, :, None, None], P[None, None, :, :]]
    return h, np.ascontiguousarray(g)


def ab_initio(N: int, n_alpha: int, n_beta: int, seed: int, n_chol: int = 48,
              name: str | None = None) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    h, g = synthetic_integrals(N, rng, n_chol=n_chol)
    return Workload(name or f"abinitio_N{N}_{n_alpha}a{n_beta}b_s{seed}", N, n_alpha, n_beta, h, g,
                    (0, 0), dict(kind="ab_initio", seed=seed, n_chol=n_chol))


# ---------------------------------------------------------------------------
# The five workload configurations
# ---------------------------------------------------------------------------

def config1() -> Workload:
    """1D Hubbard chain, 8 sites, open boundary, 4+4 electrons, t=1, U=4 (FCI dim 4,900)."""
    return hubbard((8,), 4, 4, t=1.0, U=4.0, periodic=False, name="hubbard_chain8_obc_U4")


def config2() -> Workload:
    """Synthetic ab initio N=24, 6+6 electrons, seed 2, 48 Cholesky vectors."""
    return ab_initio(24, 6, 6, seed=2, name="abinitio_N24_6a6b_seed2")


def config3(U: float = 8.0) -> Workload:
    """2D Hubbard 4x4 periodic, 8+8 electrons, t=1 (FCI dim 165,636,900)."""
    return hubbard((4, 4), 8, 8, t=1.0, U=U, periodic=True, name=f"hubbard_4x4_pbc_U{U:g}")


def config5() -> Workload:
    """Synthetic ab initio N=16, 5+5 electrons, seed 5."""
    return ab_initio(16, 5, 5, seed=5, name="abinitio_N16_5a5b_seed5")


HUBBARD_SHAPES = [(6,), (7,), (8,), (9,), (10,), (11,), (12,), (13,), (14,), (15,), (16,),
                  (2, 3), (2, 4), (2, 5), (3, 4), (2, 7), (4, 4)]


def config4_instances(n_ab: int = 64, n_hub: int = 32) -> List[Workload]:
    """Uneven batch: n_ab ab initio instances (N ~ U[12,32], n_alpha = n_beta ~ U[3,8],
    seed 1000+i; N and n are the first two draws of that seed's generator) and n_hub
    Hubbard instances (seed 2000+i picks shape, U/t in {2,4,8}; half filling)."""
    out = []
    for i in range(n_ab):
        rng = np.random.Generator(np.random.PCG64(1000 + i))
        N = int(rng.integers(12, 33))
        n = int(rng.integers(3, 9))
        h, g = synthetic_integrals(N, rng)
        out.append(Workload(f"c4_ab{i}_N{N}_{n}a{n}b", N, n, n, h, g, (0, 0),
                            dict(kind="ab_initio", seed=1000 + i)))
    for i in range(n_hub):
        rng = np.random.Generator(np.random.PCG64(2000 + i))
        shape = HUBBARD_SHAPES[int(rng.integers(0, len(HUBBARD_SHAPES)))]
        U = float([2.0, 4.0, 8.0][int(rng.integers(0, 3))])
        N = int(np.prod(shape))
        na = N // 2
        nb = N - na
        out.append(hubbard(shape, na, nb, t=1.0, U=U, periodic=True,
                           name=f"c4_hub{i}_{'x'.join(map(str, shape))}_U{U:g}"))
    return out


def random_determinants(N: int, n_alpha: int, n_beta: int, count: int, seed: int) -> np.ndarray:
    """(count, 2) uint64 array of uniformly drawn determinants."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((count, 2), dtype=np.uint64)
    for k in range(count):
        a = rng.choice(N, size=n_alpha, replace=False)
        b = rng.choice(N, size=n_beta, replace=False)
        out[k, 0] = np.uint64(sum(1 << int(p) for p in a))
        out[k, 1] = np.uint64(sum(1 << int(p) for p in b))
    return out


def write_fcidump(path: str, w: Workload, e_core: float = 0.0, fortran: bool = False) -> None:
    """w's integrals as FCIDUMP text (Knowles-Handy format): the namelist header, one line per
    unique nonzero (ij|kl) with i >= j, k >= l, (i, j) >= (k, l) (1-based), one per h_ij with
    i >= j, then the core energy.  Values are written with 17 significant digits, so they read
    back to the same doubles; `fortran` writes D exponents."""
    N = w.N
    ms2 = w.n_alpha - w.n_beta

    def fmt(x: float) -> str:
        t = f"{x:.16E}"
        return t.replace("E", "D") if fortran else t

    lines = [f" &FCI NORB={N:3d},NELEC={w.n_alpha + w.n_beta:3d},MS2={ms2:2d},",
             "  ORBSYM=" + ",".join(["1"] * N) + ",", "  ISYM=1,", " &END"]
    for i in range(N):
        for j in range(i + 1):
            for k in range(N):
                for l in range(k + 1):
                    if i * (i + 1) // 2 + j < k * (k + 1) // 2 + l:
                        continue
                    v = float(w.g[i, j, k, l])
                    if v != 0.0:
                        lines.append(f"{fmt(v)} {i + 1:3d} {j + 1:3d} {k + 1:3d} {l + 1:3d}")
    for i in range(N):
        for j in range(i + 1):
            v = float(w.h[i, j])
            if v != 0.0:
                lines.append(f"{fmt(v)} {i + 1:3d} {j + 1:3d}   0   0")
    lines.append(f"{fmt(e_core)}   0   0   0   0")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
