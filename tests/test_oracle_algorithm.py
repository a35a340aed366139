"""Pins for the oracle's algorithm layer: Algorithm 1, Algorithm 2, the appendix's
step size, and the RDMs.  Every check compares with a definition evaluated
directly (f(c) = ||H + c c^T||_F^2 on a dense H, library root finders and
minimisers, finite differences), not with the oracle's own formulas."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs


def quartic_global_min(v1, v2, v3):
    """Global minimiser of eta^4 + v3 eta^3 + v2 eta^2 + v1 eta via numpy.roots of the derivative."""
    r = np.roots([4.0, 3.0 * v3, 2.0 * v2, v1])
    r = r[np.abs(r.imag) < 1e-9 * max(1.0, np.abs(r).max())].real
    hv = r ** 4 + v3 * r ** 3 + v2 * r ** 2 + v1 * r
    return r[np.argmin(hv)], np.sort(r)


def test_line_search_is_global_minimiser():
    rng = np.random.default_rng(0)
    n_three = 0
    for _ in range(3000):
        v1, v2, v3 = rng.normal(size=3) * rng.choice([1e-6, 1e-2, 1.0, 10.0], size=3)
        eta = oracle.line_search(v1, v2, v3)
        ref, roots = quartic_global_min(v1, v2, v3)
        n_three += len(roots) == 3
        h = lambda x: x ** 4 + v3 * x ** 3 + v2 * x ** 2 + v1 * x
        # same point, or a point with the same (minimal) value
        assert abs(eta - ref) <= 1e-9 * max(1.0, abs(ref)) or abs(h(eta) - h(ref)) <= 1e-13 * max(1.0, abs(h(ref)))
        assert abs(((4 * eta + 3 * v3) * eta + 2 * v2) * eta + v1) <= 1e-10 * max(1.0, abs(v1), abs(v2), abs(v3))
    assert n_three > 300  # the three-real-root branch was exercised


def test_line_search_three_roots_picks_the_far_root():
    """Delta < 0: of x1 < x2 < x3 the root farther from x2 minimises the quartic
    (appendix); h(x3) - h(x1) has the sign of (x1 + x3)/2 - x2."""
    for roots in [(-2.0, -0.4, 1.0), (-2.0, -0.6, 1.0), (-1.0, 0.3, 0.5), (-3.0, -2.9, 4.0), (0.1, 0.2, 5.0)]:
        x1, x2, x3 = roots
        # 4 (x - x1)(x - x2)(x - x3) = 4x^3 + 3 v3 x^2 + 2 v2 x + v1
        c = 4.0 * np.poly(roots)
        v3, v2, v1 = c[1] / 3.0, c[2] / 2.0, c[3]
        eta = oracle.line_search(v1, v2, v3)
        far = x1 if (x2 - x1) > (x3 - x2) else x3
        assert abs(eta - far) < 1e-12


def test_line_search_symmetric_tie_goes_to_the_smaller_root():
    """A coordinate that is the only nonzero one (c_i = 1, mu = 1, b_i = H_ii):
    the quartic is symmetric about eta = -1, its minima -1 -+ sqrt(-H_ii) have
    equal values, and the tie goes to the smaller root x1 whatever the rounding
    of the depressed cubic."""
    for H in (-5.0, -2.5, -30.25, -53.1, -4.235806999129704):
        v1, v2, v3 = 4.0 * H + 4.0, 2.0 * H + 6.0, 4.0
        eta = oracle.line_search(v1, v2, v3)
        assert abs(eta - (-1.0 - np.sqrt(-H))) <= 1e-12 * (1.0 + np.sqrt(-H)), (H, eta)
    for roots in [(-2.0, 0.0, 2.0), (-3.5, -1.0, 1.5), (-0.75, 0.5, 1.75)]:
        c = 4.0 * np.poly(roots)
        v3, v2, v1 = c[1] / 3.0, c[2] / 2.0, c[3]
        eta = oracle.line_search(v1, v2, v3)
        assert abs(eta - roots[0]) < 1e-12, (roots, eta)


def test_line_search_small_gradient():
    """Near convergence v1 -> 0 and eta ~ -v1 / (2 v2) to first order."""
    for v1 in (1e-8, -1e-10, 3e-13):
        eta = oracle.line_search(v1, 5.0, 0.7)
        assert abs(eta - (-v1 / 10.0)) <= 1e-6 * abs(v1)
        assert abs(((4 * eta + 2.1) * eta + 10.0) * eta + v1) <= 1e-15 * abs(v1)


def _dense(w):
    H = oracle.dense_H(w.N, w.n_alpha, w.n_beta, w.h, w.g)
    dets = oracle.fci_dets(w.N, w.n_alpha, w.n_beta)
    idx = {(int(a), int(b)): i for i, (a, b) in enumerate(dets)}
    return H, idx


def _vec(idx, keys, vals, n):
    v = np.zeros(n)
    for k, x in zip(keys, vals):
        v[idx[(int(k[0]), int(k[1]))]] = x
    return v


def f_obj(H, c):
    """Eq. (optimization): ||H + c c^T||_F^2."""
    return float(np.sum((H + np.outer(c, c)) ** 2))


def test_cdfci_step_matches_direct_definition():
    """Each step of Algorithm 1 (tau = 0): i is the argmax of |grad f| (grad by finite
    differences of f) over the previous column; eta minimises f(c + eta e_i)
    (quartic recovered by interpolating f); b = Hc, mu = c.c, alpha = c.Hc."""
    w = inputs.ab_initio(5, 2, 2, seed=3)
    H, idx = _dense(w)
    n = len(H)
    s = oracle.CDFCI(w.N, 2, 2, w.h, w.g, (0, 0), 0.0, 1)
    fprev = None
    for it in range(60):
        keys, c, b = s.export()
        cv = _vec(idx, keys, c, n)
        cand = s.candidates()
        s.step(1)
        (sel,), (eta,) = s.last_step()
        i = idx[(int(sel[0]), int(sel[1]))]
        # gradient by central differences of f
        cand_i = [idx[(int(k[0]), int(k[1]))] for k in cand]
        grad = []
        for j in cand_i:
            e = np.zeros(n)
            e[j] = 1e-4
            grad.append((f_obj(H, cv + e) - f_obj(H, cv - e)) / 2e-4)
        grad = np.abs(grad)
        assert grad[cand_i.index(i)] >= grad.max() * (1 - 1e-6)
        # quartic in eta by interpolation at 5 points, then its global minimiser
        ts = np.array([-2.0, -1.0, 0.0, 1.0, 2.0]) * max(1.0, abs(eta))
        vals = []
        for t in ts:
            e = np.zeros(n)
            e[i] = t
            vals.append(f_obj(H, cv + e))
        coef = np.polyfit(ts, vals, 4)
        assert abs(coef[0] - 1.0) < 1e-6
        ref, _ = quartic_global_min(coef[3], coef[2], coef[1])
        assert abs(eta - ref) < 1e-6 * max(1.0, abs(ref))
        keys, c, b = s.export()
        cv = _vec(idx, keys, c, n)
        bv = _vec(idx, keys, b, n)
        info = s.info()
        assert np.abs(bv - H @ cv).max() < 1e-12
        assert abs(info["mu"] - cv @ cv) < 1e-12
        assert abs(info["alpha"] - cv @ H @ cv) < 1e-11
        f = f_obj(H, cv)
        if fprev is not None:
            assert f <= fprev + 1e-10
        fprev = f


@pytest.mark.parametrize("m", [2, 4])
def test_mcdfci_step_is_block_minimiser(m):
    """Algorithm 2: (gamma, eta) minimises f(gamma c + E_I eta) over R^{m+1}
    (checked with scipy BFGS from the oracle's point and from random starts) and
    the new c is gamma c + E_I eta; b = Hc, mu, alpha exact."""
    from scipy.optimize import minimize
    w = inputs.ab_initio(5, 2, 2, seed=4)
    H, idx = _dense(w)
    n = len(H)
    s = oracle.CDFCI(w.N, 2, 2, w.h, w.g, (0, 0), 0.0, m)
    rng = np.random.default_rng(1)
    for it in range(25):
        keys, c, b = s.export()
        c0 = _vec(idx, keys, c, n)
        s.step(1)
        sel, eta = s.last_step()
        I = [idx[(int(k[0]), int(k[1]))] for k in sel]
        keys, c, b = s.export()
        c1 = _vec(idx, keys, c, n)
        # recover gamma from an entry outside I (if any)
        out = [j for j in range(n) if j not in I and c0[j] != 0]
        gamma = c1[out[0]] / c0[out[0]] if out else 1.0
        assert np.abs(c1 - (gamma * c0 + np.bincount(I, weights=eta, minlength=n))).max() < 1e-12

        def obj(x):
            return f_obj(H, x[0] * c0 + np.bincount(I, weights=x[1:], minlength=n))
        x_or = np.concatenate([[gamma], eta])
        best = obj(x_or)
        for start in [x_or + 1e-3 * rng.normal(size=len(x_or))] + [rng.normal(size=len(x_or)) for _ in range(3)]:
            r = minimize(obj, start, method="BFGS", options=dict(gtol=1e-10))
            assert best <= r.fun + 1e-9
        bv = _vec(idx, keys, b, n)
        assert np.abs(bv - H @ c1).max() < 1e-11
        info = s.info()
        assert abs(info["mu"] - c1 @ c1) < 1e-11
        assert abs(info["alpha"] - c1 @ H @ c1) < 1e-10


def test_reduced_problem_identity():
    """f(Q z; H) = ||H||^2 + 2 z^T Q^T H Q z + ||z||^4 for orthonormal Q (Sec. mCDFCI)."""
    rng = np.random.default_rng(2)
    A = rng.normal(size=(12, 12))
    H = A + A.T
    Q, _ = np.linalg.qr(rng.normal(size=(12, 4)))
    z = rng.normal(size=4)
    lhs = f_obj(H, Q @ z)
    rhs = np.sum(H ** 2) + 2 * z @ Q.T @ H @ Q @ z + (z @ z) ** 2
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_cdfci_converges_to_exact_diagonalisation_config1():
    """Config 1 (8-site open chain, U = 4, 4+4): Algorithm 1 reaches the dense ED energy."""
    w = inputs.config1()
    E0 = oracle.ground_energy(8, 4, 4, w.h, w.g, dense_limit=5000)
    s = oracle.CDFCI(8, 4, 4, w.h, w.g, w.ref, 0.0, 1)
    s.step(260000)
    assert abs(s.energy() - E0) < 1e-10
    info = s.info()
    assert abs(info["mu"] + E0) < 1e-8          # minimisers are +-sqrt(-E0) v0 (Eq. optimization)


def test_mcdfci_converges_ab_initio():
    w = inputs.ab_initio(6, 3, 2, seed=7)
    E0 = oracle.ground_energy(6, 3, 2, w.h, w.g)
    s = oracle.CDFCI(6, 3, 2, w.h, w.g, (0, 0), 0.0, 8)
    s.step(1500)
    assert abs(s.energy() - E0) < 1e-9
    s1 = oracle.CDFCI(6, 3, 2, w.h, w.g, (0, 0), 0.0, 1)
    s1.step(40000)
    assert abs(s1.energy() - E0) < 1e-9


def test_compression_rule():
    """tau > 0 (Sec. CDFCI, compression): b_j is updated iff c_j != 0 or |eta H_ji| >= tau.
    Hence every j with c_j != 0 keeps b_j = (Hc)_j exactly (it was recalculated when
    selected and has received every update since); mu = c.c is unaffected; alpha
    follows Eq. (update-var) with the stored pre-update b_i."""
    w = inputs.ab_initio(6, 2, 2, seed=9)
    H, idx = _dense(w)
    n = len(H)
    s = oracle.CDFCI(6, 2, 2, w.h, w.g, (0, 0), 2e-3, 1)
    for it in range(300):
        keys, c, b = s.export()
        bmap = {(int(k[0]), int(k[1])): (x, y) for k, x, y in zip(keys, c, b)}
        a0 = s.info()["alpha"]
        s.step(1)
        (sel,), (eta,) = s.last_step()
        c_i, b_i = bmap[(int(sel[0]), int(sel[1]))]
        ii = idx[(int(sel[0]), int(sel[1]))]
        Hii = H[ii, ii]
        assert abs(s.info()["alpha"] - (a0 + 2 * eta * b_i + eta * eta * Hii)) < 1e-12
    info = s.info()
    assert info["dropped"] > 0
    keys, c, b = s.export()
    cv = _vec(idx, keys, c, n)
    bv = _vec(idx, keys, b, n)
    nz = cv != 0
    assert np.abs((bv - H @ cv)[nz]).max() < 1e-12
    assert abs(info["mu"] - cv @ cv) < 1e-12
    # entries that were never applied are absent: every stored j was inserted by an update >= tau
    assert info["entries"] < n


def test_rdm_identities_and_hellmann_feynman():
    w = inputs.ab_initio(5, 2, 2, seed=12)
    H, idx = _dense(w)
    evals, evecs = np.linalg.eigh(H)
    c = evecs[:, 0]
    dets = oracle.fci_dets(5, 2, 2)
    g1, g2 = oracle.rdm(5, dets, c)
    n = 4
    assert abs(np.trace(g1) - n) < 1e-12
    assert abs(np.einsum("pprr->", g2) - n * (n - 1)) < 1e-11
    E = np.sum(w.h * g1) + 0.5 * np.sum(w.g * g2)
    assert abs(E - evals[0]) < 1e-11
    # Hellmann-Feynman: dE0/dh along a symmetric direction = sum D gamma
    rng = np.random.default_rng(3)
    D = rng.normal(size=(5, 5))
    D = D + D.T
    eps = 1e-5
    Ep = np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, w.h + eps * D, w.g))[0]
    Em = np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, w.h - eps * D, w.g))[0]
    assert abs((Ep - Em) / (2 * eps) - np.sum(D * g1)) < 1e-7


def test_orbital_gradient_matches_finite_differences_of_exact_energy():
    """dE/dkappa from the RDMs (the rotated-integral energy of Sec. "Optimal
    Orbital Selections") against a central difference, step 1e-5, of the
    exact ground energy of the rotated integrals; the rotation itself is
    pinned by the invariance of the spectrum."""
    w = inputs.ab_initio(5, 2, 2, seed=12)
    H, idx = _dense(w)
    evals, evecs = np.linalg.eigh(H)
    dets = oracle.fci_dets(5, 2, 2)
    g1, g2 = oracle.rdm(5, dets, evecs[:, 0])
    G = oracle.orbital_gradient(w.h, w.g, g1, g2)
    assert np.abs(G + G.T).max() < 1e-14
    rng = np.random.default_rng(8)
    K = rng.normal(size=(5, 5))
    K = K - K.T
    # a full rotation of the orbitals leaves the spectrum of H unchanged
    hr, gr = oracle.rotate_integrals(w.h, w.g, 0.7 * K)
    assert np.abs(np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, hr, gr)) - evals).max() < 1e-10
    eps = 1e-5
    Ep = np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, *oracle.rotate_integrals(w.h, w.g, eps * K)))[0]
    Em = np.linalg.eigvalsh(oracle.dense_H(5, 2, 2, *oracle.rotate_integrals(w.h, w.g, -eps * K)))[0]
    fd = (Ep - Em) / (2 * eps)
    assert abs(fd - 0.5 * np.sum(G * K)) < 1e-7 * max(1.0, abs(fd))
    # a wrong transpose in F (the classic slip) breaks the same check
    F_bad = w.h @ g1 + np.einsum("prst,rqst->pq", w.g, g2)
    assert abs(fd - np.sum((F_bad - F_bad.T) * K)) > 1e-6 or np.allclose(F_bad, F_bad.T)

