"""The Algorithm-3 (xCDFCI) oracle against the definition f(C) = ||H + C C^T||_F^2,
dense algebra on a small FCI space, Algorithm 1 (K + 1 = 1) and exact
diagonalisation (the K + 1 lowest eigenvalues)."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs


def small_problem(seed=8):
    N, na, nb = 6, 2, 2
    w = inputs.ab_initio(N, na, nb, seed=seed)
    dets = oracle.fci_dets(N, na, nb)
    H = oracle.dense_H(N, na, nb, w.h, w.g)
    return w, dets, H


def lowest_diagonal(dets, H, k):
    d = np.diag(H)
    order = sorted(range(len(dets)), key=lambda i: (d[i], int(dets[i][1]), int(dets[i][0])))
    return dets[order[:k]]


def test_quartic_coefficients_match_the_definition():
    """h(eta) = f(C + eta e_i g) - f(C) along g = G_i = 4 B_i + 4 C_i S is the oracle's
    w1 eta + w2 eta^2 + w3 eta^3 + w4 eta^4 (in particular w1 = ||g||^2, the directional derivative)."""
    _, dets, H = small_problem()
    rng = np.random.default_rng(0)
    n = len(dets)
    for k1 in (1, 2, 4):
        for trial in range(3):
            C = rng.normal(size=(n, k1)) * 0.1
            B = H @ C
            S = C.T @ C
            i = int(rng.integers(n))
            g = 4.0 * B[i] + 4.0 * C[i] @ S
            w = oracle.xcd_quartic(C[i], g, S, H[i, i])
            scale = 1.0 / np.sqrt(g @ g)
            etas = np.array([-2.0, -1.0, 1.0, 2.0]) * scale
            hv = []
            for eta in etas:
                X = C.copy()
                X[i] += eta * g
                D = X @ X.T - C @ C.T
                hv.append(2.0 * np.sum((H + C @ C.T) * D) + np.sum(D * D))
            A = np.vander(etas, 5, increasing=True)[:, 1:]
            fit = np.linalg.solve(A, np.array(hv))
            assert abs(w[1] - g @ g) <= 1e-14 * (g @ g)
            for p in range(4):
                assert abs(fit[p] - w[p + 1]) <= 1e-7 * max(1.0, abs(w[p + 1])) * scale ** -(p + 1), (k1, p, fit[p], w[p + 1])


def test_rows_and_small_matrices_follow_dense_algebra():
    """tau = 0: after 60 steps B = H C on every stored row, S = C^T C, M = C^T H C
    (the eta^2 terms are the outer product g^T g)."""
    w, dets, H = small_problem()
    start = lowest_diagonal(dets, H, 3)
    o = oracle.XCDFCI(6, 2, 2, w.h, w.g, start, tau=0.0)
    o.step(60)
    keys, C, B = o.export()
    index = {(int(a), int(b)): t for t, (a, b) in enumerate(dets)}
    Cd = np.zeros((len(dets), 3))
    for (a, b), row in zip(keys, C):
        Cd[index[(int(a), int(b))]] = row
    HC = H @ Cd
    for (a, b), row in zip(keys, B):
        assert np.abs(row - HC[index[(int(a), int(b))]]).max() <= 1e-11 * max(1.0, np.abs(HC).max())
    info = o.info()
    assert np.abs(info["S"] - Cd.T @ Cd).max() <= 1e-12 * max(1.0, np.abs(info["S"]).max())
    assert np.abs(info["M"] - Cd.T @ HC).max() <= 1e-11 * max(1.0, np.abs(info["M"]).max())
    assert info["iterations"] == 60
    o.close()


def test_one_state_is_algorithm_1():
    """K + 1 = 1: the same trajectory as Algorithm 1 (C_i += eta G_i is c_i += eta', eta' = eta G_i)."""
    w, dets, H = small_problem(seed=3)
    a = oracle.CDFCI(6, 2, 2, w.h, w.g, w.ref, 1e-4, 1)
    k, c, _ = a.export()
    ref = k[np.argmax(np.abs(c))]
    x = oracle.XCDFCI(6, 2, 2, w.h, w.g, ref[None, :], tau=1e-4)
    assert abs(x.energies()[0] - a.energy()) <= 1e-14 * abs(a.energy())
    for _ in range(200):
        a.step(1)
        x.step(1)
        assert np.array_equal(x.last_step()[0], a.last_step()[0][0])
    assert abs(x.energies()[0] - a.energy()) <= 1e-11 * abs(a.energy())
    a.close(); x.close()


@pytest.mark.parametrize("k1", [2, 3])
def test_converges_to_the_lowest_eigenvalues(k1):
    w, dets, H = small_problem(seed=11)
    exact = np.linalg.eigvalsh(H)[:k1]
    assert exact[-1] < 0
    o = oracle.XCDFCI(6, 2, 2, w.h, w.g, lowest_diagonal(dets, H, k1), tau=0.0)
    o.step(40000)
    E = o.energies()
    assert np.abs(E - exact).max() < 1e-8, (E, exact)
    o.close()
