"""The k-space Hubbard model (HamiltonianHubbardK of Sec. "The Hamiltonian Class") in the
oracle: plane-wave integrals, their symmetry, the spectrum against the real-space lattice
(unitarily equivalent), momentum conservation, and the degenerate-subspace start of the
paper's 4x4 example (numerical section, "2D Hubbard Model")."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs


def momentum(shape, key):
    n = inputs.momenta(shape)
    tot = np.zeros(len(shape), dtype=np.int64)
    for word in key:
        w = int(word)
        for p in range(len(n)):
            if (w >> p) & 1:
                tot += n[p]
    return tuple(tot % np.array(shape))


def test_plane_wave_integrals():
    """h diagonal; (pq|rs) = U/L exactly when k_q - k_p + k_s - k_r = 0, else 0; the 4-fold
    symmetries hold exactly and the 8-fold one does not."""
    shape, U = (4, 4), 4.0
    w = inputs.config3_k(U)
    L = 16
    assert np.count_nonzero(w.h - np.diag(np.diag(w.h))) == 0
    g = w.g
    assert set(np.unique(g)) <= {0.0, U / L}
    n = inputs.momenta(shape)
    for p, q, r, s in [(0, 0, 0, 0), (1, 2, 3, 4), (5, 1, 3, 7), (2, 6, 9, 13)]:
        cons = np.all((n[q] - n[p] + n[s] - n[r]) % np.array(shape) == 0)
        assert g[p, q, r, s] == (U / L if cons else 0.0)
    assert np.array_equal(g, g.transpose(2, 3, 0, 1)) and np.array_equal(g, g.transpose(1, 0, 3, 2))
    assert not np.array_equal(g, g.transpose(1, 0, 2, 3))


def test_4x4_levels_match_the_paper():
    """The paper's 4x4 example: 5 one-body levels below zero, 6 at zero, 5 above (t = 1)."""
    eps = np.diag(inputs.config3_k(4.0).h)
    assert (np.sum(eps < 0), np.sum(eps == 0), np.sum(eps > 0)) == (5, 6, 5)
    assert sorted(eps)[0] == -4.0 and sorted(eps)[-1] == 4.0


@pytest.mark.parametrize("shape,na,nb,U", [((4,), 2, 2, 4.0), ((6,), 3, 3, 4.0), ((2, 3), 3, 2, 2.0),
                                           ((2, 2), 2, 2, 4.0), ((5,), 2, 3, 8.0)])
def test_spectrum_equals_the_real_space_lattice(shape, na, nb, U):
    """Plane waves are a unitary change of orbitals: the same ground energy as the site basis."""
    wk = inputs.hubbard_k(shape, na, nb, U=U)
    wr = inputs.hubbard(shape, na, nb, U=U, periodic=True)
    ek = oracle.ground_energy(wk.N, na, nb, wk.h, wk.g)
    er = oracle.ground_energy(wr.N, na, nb, wr.h, wr.g)
    assert abs(ek - er) <= 1e-10 * max(1.0, abs(er))


def test_noninteracting_closed_form():
    """U = 0: the lowest eigenvalue is the sum of the lowest one-body levels of each spin."""
    w = inputs.hubbard_k((2, 3), 3, 2, U=0.0)
    eps = np.sort(np.diag(w.h))
    assert abs(oracle.ground_energy(w.N, 3, 2, w.h, w.g) - (eps[:3].sum() + eps[:2].sum())) <= 1e-12


def test_columns_conserve_momentum_and_sc_matches_literal():
    """Every entry of a column has the column's total momentum; no singles appear; the
    Slater-Condon rules give the literal operator's values (both sides round a true zero on
    the diagonal differently, so entries below 1e-12 are compared as zero)."""
    shape = (2, 3)
    w = inputs.hubbard_k(shape, 3, 2, U=2.0)
    dets = oracle.fci_dets(w.N, 3, 2)
    for d in dets[::9]:
        kl, vl = oracle.column_literal(w.N, w.h, w.g, d)
        ks, vs = oracle.column_sc(w.N, w.h, w.g, d)
        ml = {(int(a), int(b)): v for (a, b), v in zip(kl, vl) if abs(v) > 1e-12}
        ms = {(int(a), int(b)): v for (a, b), v in zip(ks, vs) if abs(v) > 1e-12}
        assert set(ml) == set(ms)
        assert max(abs(ml[k] - ms[k]) for k in ml) <= 1e-13
        for (a, b) in ms:
            assert momentum(shape, (a, b)) == momentum(shape, d)
            da, db = bin(a ^ int(d[0])).count("1"), bin(b ^ int(d[1])).count("1")
            assert (da, db) in {(0, 0), (2, 2)}            # diagonal or an opposite-spin double


def test_degenerate_start_4x4_half_filling():
    """The paper's count: C(6, 3)^2 = 400 configurations share the lowest one-body energy at
    half filling; the start is an eigenvector of H on them (residual) below their diagonal."""
    w = inputs.config3_k(4.0)
    keys, c, E = oracle.degenerate_start(w.N, 8, 8, w.h, w.g)
    assert len(keys) == math.comb(6, 3) ** 2 == 400
    eps = np.diag(w.h)
    e_one = [sum(eps[p] for p in range(16) if (int(a) >> p) & 1) + sum(eps[p] for p in range(16) if (int(b) >> p) & 1)
             for a, b in keys]
    assert max(e_one) - min(e_one) == 0.0 and min(e_one) == -24.0          # (-4 - 4 x 2 + 3 x 0) per spin
    idx = {(int(a), int(b)): i for i, (a, b) in enumerate(keys)}
    H = np.zeros((400, 400))
    for i, k in enumerate(keys):
        ck, cv = oracle.column_sc(w.N, w.h, w.g, k)
        for (a, b), v in zip(ck, cv):
            j = idx.get((int(a), int(b)))
            if j is not None:
                H[j, i] = v
    assert np.max(np.abs(H - H.T)) <= 1e-14
    assert np.linalg.norm(H @ c - E * c) <= 1e-10 and abs(np.linalg.norm(c) - 1.0) <= 1e-14
    assert E <= np.min(np.diag(H)) and c[np.argmax(np.abs(c))] > 0
    # the lowest eigenvalue is 4-fold degenerate over total momenta (0, 0) and (pi, pi); the start
    # (the ramp projected onto the eigenspace) has a component in both sectors
    ev = np.linalg.eigvalsh(H)
    assert np.sum(ev <= E + 1e-9 * abs(E)) == 4
    km = inputs.momenta((4, 4))
    weight = {}
    for (a, b), x in zip(keys, c):
        K = sum(km[p] for p in range(16) if (int(a) >> p) & 1) + sum(km[p] for p in range(16) if (int(b) >> p) & 1)
        weight[tuple(int(q) for q in np.asarray(K) % 4)] = weight.get(tuple(int(q) for q in np.asarray(K) % 4), 0.0) + x * x
    assert set(k for k, v in weight.items() if v > 1e-12) == {(0, 0), (2, 2)}
    assert min(v for v in weight.values() if v > 1e-12) > 0.1


def test_degenerate_start_small_and_unique():
    """A 6-site ring with 2 + 2 electrons: the level -1 (k = +-pi/3) holds one electron of two
    per spin, so 2 x 2 = 4 configurations; the start's energy is an eigenvalue of H on them."""
    w = inputs.hubbard_k((6,), 2, 2, U=4.0)
    keys, c, E = oracle.degenerate_start(w.N, 2, 2, w.h, w.g)
    assert len(keys) == 4
    assert list(map(tuple, keys.tolist())) == sorted(map(tuple, keys.tolist()), key=lambda k: (k[1], k[0]))
    assert abs(np.linalg.norm(c) - 1.0) <= 1e-14 and E >= oracle.ground_energy(w.N, 2, 2, w.h, w.g) - 1e-12
