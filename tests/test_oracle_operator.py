"""Pins for the oracle's definition layer (Eq. general-ham, Eq. 2int, Eq. entry).

Each check is independent of the oracle's own code: a Jordan-Wigner Fock-space
matrix built from Kronecker products, orbital-rotation invariance of the
spectrum, closed forms, and the non-interacting limit.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def _colmap(keys, vals):
    return {(int(k[0]), int(k[1])): float(v) for k, v in zip(keys, vals)}


# --------------------------------------------------------------------------
# Jordan-Wigner Fock-space matrix: an independent construction of H
# --------------------------------------------------------------------------

def _jw_annihilators(M):
    """a_P = Z x ... x Z x s x I x ... x I (P leading Z factors), s = |0><1|."""
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    s = np.array([[0.0, 1.0], [0.0, 0.0]])
    ops = []
    for P in range(M):
        op = np.array([[1.0]])
        for k in range(M):
            op = np.kron(op, Z if k < P else (s if k == P else I))
        ops.append(op)
    return ops


def _fock_index(key, N):
    """Kronecker index of an occupation string: spin-orbital P is factor P (most significant first)."""
    M = 2 * N
    idx = 0
    for P in range(M):
        occ = (int(key[0]) >> P) & 1 if P < N else (int(key[1]) >> (P - N)) & 1
        idx |= occ << (M - 1 - P)
    return idx


def _fock_H(N, h, g):
    M = 2 * N
    a = _jw_annihilators(M)
    ad = [x.T for x in a]
    H = np.zeros((2 ** M, 2 ** M))
    spin = [0] * N + [1] * N
    orb = list(range(N)) * 2
    for P in range(M):
        for Q in range(M):
            if spin[P] == spin[Q] and h[orb[P], orb[Q]] != 0:
                H += h[orb[P], orb[Q]] * ad[P] @ a[Q]
    # 1/2 sum v_PQRS a+_P a+_Q a_S a_R with v_PQRS = <PQ|RS> = (pr|qs) for matching spins
    for P, Q, R, S in itertools.product(range(M), repeat=4):
        if spin[P] != spin[R] or spin[Q] != spin[S]:
            continue
        v = g[orb[P], orb[R], orb[Q], orb[S]]
        if v != 0:
            H += 0.5 * v * ad[P] @ ad[Q] @ a[S] @ a[R]
    return H


@pytest.mark.parametrize("N,na,nb,seed", [(3, 1, 1, 1), (3, 2, 1, 2), (3, 1, 2, 3), (3, 2, 2, 4)])
def test_literal_matches_jordan_wigner_fock_matrix(N, na, nb, seed):
    w = inputs.ab_initio(N, na, nb, seed=seed)
    HF = _fock_H(N, w.h, w.g)
    dets = oracle.fci_dets(N, na, nb)
    sel = [_fock_index(d, N) for d in dets]
    H_jw = HF[np.ix_(sel, sel)]
    H_lit = oracle.dense_H(N, na, nb, w.h, w.g)
    assert np.abs(H_lit - H_jw).max() < 1e-12
    # the sector is closed: no amplitude leaks to other particle numbers
    others = [i for i in range(HF.shape[0]) if i not in set(sel)]
    assert np.abs(HF[np.ix_(others, sel)]).max() < 1e-12


def test_slater_condon_matches_literal_all_pairs_small():
    for (N, na, nb, seed) in [(4, 2, 1, 11), (4, 2, 2, 12), (5, 2, 2, 13), (6, 3, 2, 14)]:
        w = inputs.ab_initio(N, na, nb, seed=seed)
        for d in oracle.fci_dets(N, na, nb):
            k1, v1 = oracle.column_literal(N, w.h, w.g, d)
            k2, v2 = oracle.column_sc(N, w.h, w.g, d)
            m1, m2 = _colmap(k1, v1), _colmap(k2, v2)
            assert set(m1) == set(m2)
            for k in m1:
                assert abs(m1[k] - m2[k]) <= 1e-13 * max(1.0, abs(m1[k]))


@pytest.mark.parametrize("N,na,nb", [(8, 3, 3), (12, 4, 3), (24, 6, 6)])
def test_slater_condon_matches_literal_random_dets(N, na, nb):
    w = inputs.ab_initio(N, na, nb, seed=100 + N)
    for d in inputs.random_determinants(N, na, nb, 3 if N > 12 else 10, seed=N):
        m1 = _colmap(*oracle.column_literal(N, w.h, w.g, d))
        m2 = _colmap(*oracle.column_sc(N, w.h, w.g, d))
        assert set(m1) == set(m2)
        # column size: 1 + singles + doubles (random integrals have no structural zeros)
        va, vb = N - na, N - nb
        nh = 1 + na * va + nb * vb + math.comb(na, 2) * math.comb(va, 2) + \
            math.comb(nb, 2) * math.comb(vb, 2) + na * va * nb * vb
        assert len(m1) == nh
        for k in m1:
            assert abs(m1[k] - m2[k]) <= 1e-12 * max(1.0, abs(m1[k]))


def test_hermitian_and_number_conserving():
    w = inputs.ab_initio(6, 3, 2, seed=21)
    H = oracle.dense_H(6, 3, 2, w.h, w.g)
    assert np.abs(H - H.T).max() < 1e-13
    for d in oracle.fci_dets(6, 3, 2)[:50]:
        keys, _ = oracle.column_literal(6, w.h, w.g, d)
        for k in keys:
            assert bin(int(k[0])).count("1") == 3 and bin(int(k[1])).count("1") == 2


def test_closed_form_two_site_and_free_chains():
    gold = golden("closed_forms.txt")
    for U in (4, 1, 8):
        h, g = inputs.hubbard_integrals((2,), 1.0, float(U), periodic=False)
        assert abs(oracle.ground_energy(2, 1, 1, h, g) - gold[f"two_site_U{U}"]) < 1e-13
    h, g = inputs.hubbard_integrals((8,), 1.0, 0.0, periodic=False)
    assert abs(oracle.ground_energy(8, 4, 4, h, g) - gold["chain8_obc_U0"]) < 1e-11
    h, g = inputs.hubbard_integrals((6,), 1.0, 0.0, periodic=True)
    assert abs(oracle.ground_energy(6, 3, 3, h, g) - gold["ring6_U0"]) < 1e-11


def test_non_interacting_limit_is_orbital_filling():
    """g = 0: E0 = sum of the lowest n_alpha plus the lowest n_beta eigenvalues of h."""
    w = inputs.ab_initio(8, 3, 2, seed=31)
    eps = np.linalg.eigvalsh(w.h)
    E = oracle.ground_energy(8, 3, 2, w.h, np.zeros_like(w.g))
    assert abs(E - (eps[:3].sum() + eps[:2].sum())) < 1e-11


def test_constant_coulomb_shift():
    """(pq|rs) = J delta_pq delta_rs adds J n(n-1)/2 to every state (two-body term of Eq. general-ham)."""
    w = inputs.ab_initio(6, 2, 2, seed=41)
    N, J = 6, 0.37
    g = np.zeros((N,) * 4)
    for p in range(N):
        for r in range(N):
            g[p, p, r, r] = J
    n = 4
    H0 = oracle.dense_H(N, 2, 2, w.h, np.zeros_like(g))
    H1 = oracle.dense_H(N, 2, 2, w.h, g)
    assert np.abs(H1 - H0 - 0.5 * J * n * (n - 1) * np.eye(len(H0))).max() < 1e-12


def test_spectrum_invariant_under_orbital_rotation():
    """Eq. (1int)/(2int) transform as h' = U^T h U, (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd);
    the FCI spectrum must not change.  This checks that h and g enter as tensor
    contractions over the right orbitals (a wrong stride or a mixed spin/space
    index breaks it); the choice of (pq|rs) -> v_pqrs is pinned by the diagonal,
    constant-Coulomb and atomic-limit tests."""
    w = inputs.ab_initio(5, 2, 2, seed=51)
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.normal(size=(5, 5)))
    h2 = U.T @ w.h @ U
    g2 = np.einsum("ap,bq,cr,ds,abcd->pqrs", U, U, U, U, w.g, optimize=True)
    # restore exact 8-fold symmetry of the rotated tensor
    g2 = (g2 + g2.transpose(1, 0, 2, 3) + g2.transpose(0, 1, 3, 2) + g2.transpose(1, 0, 3, 2)) / 4
    g2 = (g2 + g2.transpose(2, 3, 0, 1)) / 2
    e1 = np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, w.h, w.g))
    e2 = np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, h2, g2))
    assert np.abs(e1 - e2).max() < 1e-11


def test_extended_hubbard_atomic_limit():
    """t = 0, two sites, on-site U, inter-site Coulomb V = (00|11) and exchange
    K = (01|10) (with its 8-fold images).  Two alpha electrons: E = V - K.  One
    alpha + one beta: K flips spins between the two covalent states and moves
    the pair between the two ionic states, so the exact spectrum is
    {V - K, V + K, U - K, U + K}.  These values depend on reading (pq|rs) as
    the physicists' v_prqs of Eq. (2int); a transposed mapping gives others."""
    N, U, V, K = 2, 3.0, 0.7, 0.2
    h = np.zeros((N, N))
    g = np.zeros((N, N, N, N))
    g[0, 0, 0, 0] = g[1, 1, 1, 1] = U
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = V
    for (p, q, r, s) in [(0, 1, 1, 0), (1, 0, 0, 1), (0, 1, 0, 1), (1, 0, 1, 0)]:
        g[p, q, r, s] = K
    # two alpha electrons: |1_0a 1_1a> has E = V - K (Coulomb minus exchange)
    E_aa = np.linalg.eigvalsh(oracle.dense_H(N, 2, 0, h, g))
    assert np.abs(E_aa - (V - K)).max() < 1e-14
    # one alpha + one beta: basis (A, B) in {(0,0),(0,1),(1,0),(1,1)} as site indices
    H = oracle.dense_H(N, 1, 1, h, g)
    w = np.sort(np.linalg.eigvalsh(H))
    # exact: ionic pair {U - K, U + K}, covalent pair {V - K (triplet m_s=0), V + K (singlet)}
    assert np.abs(w - np.sort([U - K, U + K, V - K, V + K])).max() < 1e-13


def test_alpha_beta_exchange_symmetry():
    w = inputs.ab_initio(6, 3, 2, seed=61)
    e1 = np.linalg.eigvalsh(oracle.dense_H(6, 3, 2, w.h, w.g))
    e2 = np.linalg.eigvalsh(oracle.dense_H(6, 2, 3, w.h, w.g))
    assert np.abs(e1 - e2).max() < 1e-11


def test_diagonal_is_textbook_determinant_energy():
    """<D|H|D> = sum_i h_ii + 1/2 sum_ij [(ii|jj) - delta_{s_i s_j} (ij|ji)] over occupied spin-orbitals."""
    w = inputs.ab_initio(8, 3, 4, seed=71)
    for d in inputs.random_determinants(8, 3, 4, 10, seed=3):
        occ = [(p, 0) for p in range(8) if (int(d[0]) >> p) & 1] + [(p, 1) for p in range(8) if (int(d[1]) >> p) & 1]
        e = sum(w.h[p, p] for p, _ in occ)
        for (p, s), (q, t) in itertools.product(occ, occ):
            e += 0.5 * (w.g[p, p, q, q] - (w.g[p, q, q, p] if s == t else 0.0))
        lit = _colmap(*oracle.column_literal(8, w.h, w.g, d))
        assert abs(lit[(int(d[0]), int(d[1]))] - e) < 1e-12
        assert abs(oracle.diag(8, w.h, w.g, d) - e) < 1e-12


def test_hubbard_column_structure():
    """Real-space Hubbard: a column is the diagonal U * (doubly occupied sites) plus +-t hops."""
    w = inputs.config1()
    for d in oracle.fci_dets(8, 4, 4)[::97]:
        m = _colmap(*oracle.column_literal(8, w.h, w.g, d))
        A, B = int(d[0]), int(d[1])
        assert m.get((A, B), 0.0) == 4.0 * bin(A & B).count("1")
        hops = 0
        for X in (A, B):
            for i in range(8):
                for j in (i - 1, i + 1):
                    if 0 <= j < 8 and (X >> i) & 1 and not (X >> j) & 1:
                        hops += 1
        assert len(m) - (1 if (A, B) in m else 0) == hops
        assert all(abs(v) == 1.0 for k, v in m.items() if k != (A, B))


def test_fci_ranking_roundtrip():
    dets = oracle.fci_dets(7, 3, 2)
    assert len(dets) == math.comb(7, 3) * math.comb(7, 2)
    for i, d in enumerate(dets):
        assert oracle.fci_index(7, 3, 2, d) == i
    assert len({(int(a), int(b)) for a, b in dets}) == len(dets)
