"""The adjoint at the configured size (Sec. "Optimal Orbital Selections"): synthetic ab initio N = 16,
5 + 5, seed 5 (FCI dim 19,079,424, column 4,236), Algorithm 2 with m = 512.

The derivatives cdfci_gradient returns are those of the variational energy of the stored vector c,
E(h, g) = c^T H(h, g) c / c^T c, which at the minimum is the ground-state energy's (Hellmann-Feynman).
They are checked against central differences (step 1e-5) of that energy along random symmetric
directions of h, 8-fold symmetric directions of g and antisymmetric orbital rotations kappa, each
energy the library's exact Rayleigh quotient of the same vector under the perturbed integrals
(cdfci_energy_with: fresh columns and table lookups, a code path independent of the RDM kernels).
Re-converging a 1.9e7-dimensional problem to the 1e-12 Ha such a difference needs per energy is not
feasible in a test; the converged-energy differences run on the small case in test_gpu_rdm.py.
dE/dkappa is also compared with the oracle's contraction of the oracle's RDMs on the leading part of
the vector."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def sym8(G):
    return (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2) +
            G.transpose(2, 3, 0, 1) + G.transpose(3, 2, 0, 1) + G.transpose(2, 3, 1, 0) + G.transpose(3, 2, 1, 0)) / 8


def rotated(h, g, kappa):
    """h' = U^T h U, g'_pqrs = sum U_ap U_bq U_cr U_ds g_abcd with U = exp(kappa); g' symmetrised
    (the einsum's rounding breaks the 8-fold symmetry in the last bits)."""
    U = scipy.linalg.expm(kappa)
    h2 = U.T @ h @ U
    g2 = np.einsum("ap,bq,cr,ds,abcd->pqrs", U, U, U, U, g, optimize=True)
    return 0.5 * (h2 + h2.T), sym8(g2)


def test_adjoint_config5_against_central_differences_and_the_oracle():
    require_gpu()
    from paper_2605_04483_gb300 import api
    w = inputs.config5()
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, num_coordinates=512, log2_capacity=25,
                   ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))
    try:
        st = s.step(8000)
        E = s.energy(1)
        assert abs(E - st["energy"]) < 1e-9 * abs(E) and st["nnz_c"] > 1_000_000
        dh, dg, dk = s.gradient()
        rng = np.random.default_rng(55)
        eps = 1e-5
        worst = 0.0
        for _ in range(2):
            D = rng.normal(size=(16, 16))
            D = D + D.T
            fd = (s.energy_with(w.h + eps * D, w.g) - s.energy_with(w.h - eps * D, w.g)) / (2 * eps)
            an = float(np.sum(D * dh))
            worst = max(worst, abs(fd - an) / max(1.0, abs(fd)))
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)), ("h", fd, an)
            G = sym8(rng.normal(size=(16, 16, 16, 16)))
            fd = (s.energy_with(w.h, w.g + eps * G) - s.energy_with(w.h, w.g - eps * G)) / (2 * eps)
            an = float(np.sum(G * dg))
            worst = max(worst, abs(fd - an) / max(1.0, abs(fd)))
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)), ("g", fd, an)
            K = rng.normal(size=(16, 16))
            K = K - K.T
            hp, gp = rotated(w.h, w.g, eps * K)
            hm, gm = rotated(w.h, w.g, -eps * K)
            fd = (s.energy_with(hp, gp) - s.energy_with(hm, gm)) / (2 * eps)
            an = 0.5 * float(np.sum(dk * K))
            worst = max(worst, abs(fd - an) / max(1.0, abs(fd)))
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)), ("kappa", fd, an)
        print(f"[config 5] E = {E:.10f} after 8000 iterations of m = 512, {st['nnz_c']} nonzeros; "
              f"largest relative difference gradient vs central difference {worst:.2e}")
        # the leading 2000 coefficients as a vector of their own: library RDM derivatives against
        # the oracle's literal-operator RDMs and its kappa contraction
        keys, c, _ = s.export()
    finally:
        s.close()
    top = np.argsort(-np.abs(c))[:2000]
    kt, ct = keys[top], c[top]
    t = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=23, z_threshold=1e-3,
                   ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))
    try:
        t.set_initial(kt, ct)
        th, tg, tk = t.gradient()
    finally:
        t.close()
    o1, o2 = oracle.rdm(w.N, kt, ct)
    assert np.abs(th - o1).max() < 1e-12
    assert np.abs(tg - 0.5 * sym8(o2)).max() < 1e-12
    Go = oracle.orbital_gradient(w.h, w.g, o1, o2)
    assert np.abs(tk - Go).max() < 1e-11 * max(1.0, np.abs(Go).max())
