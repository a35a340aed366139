"""The OptOrbFCI (Algorithm 4) oracle: the subproblem's objective equals the
FCI energy of the rotated basis, its gradient matches finite differences, a
full orbital space stays put, and the outer loop descends monotonically above
the full-space FCI energy."""
import numpy as np

import oracle
from paper_2605_04483_gb300 import inputs


def problem(M=8, na=2, nb=2, seed=4):
    w = inputs.ab_initio(M, na, nb, seed=seed)
    return w.h, w.g


def random_stiefel(M, N, seed):
    return oracle.polar(np.random.default_rng(seed).normal(size=(M, N)))


def test_objective_is_the_fci_energy_of_the_rotated_basis():
    h, g = problem()
    U = random_stiefel(8, 6, 1)
    h2, g2 = oracle.optorb_transform(h, g, U)
    w, V = np.linalg.eigh(oracle.dense_H(6, 2, 2, h2, g2))
    r1, r2 = oracle.rdm(6, oracle.fci_dets(6, 2, 2), V[:, 0].copy())
    assert abs(oracle.optorb_objective(h, g, U, r1, r2) - w[0]) <= 1e-11 * abs(w[0])


def test_gradient_matches_finite_differences():
    h, g = problem()
    rng = np.random.default_rng(2)
    U = random_stiefel(8, 6, 3)
    h2, g2 = oracle.optorb_transform(h, g, U)
    _, V = np.linalg.eigh(oracle.dense_H(6, 2, 2, h2, g2))
    r1, r2 = oracle.rdm(6, oracle.fci_dets(6, 2, 2), V[:, 0].copy())
    G = oracle.optorb_gradient(h, g, U, r1, r2)
    for _ in range(4):
        D = rng.normal(size=U.shape)
        eps = 1e-5
        fd = (oracle.optorb_objective(h, g, U + eps * D, r1, r2) - oracle.optorb_objective(h, g, U - eps * D, r1, r2)) / (2 * eps)
        assert abs(fd - np.sum(G * D)) <= 1e-7 * max(1.0, abs(fd))


def test_full_orbital_space_stays_put():
    """M = N: full CI is invariant under rotations, so the FCI state's orbital gradient vanishes
    and the subproblem keeps U = I; the energy does not change."""
    h, g = problem(M=6)
    E, U = oracle.optorb_run(h, g, 6, 6, 2, 2, outer=2, bb_steps=10)
    assert abs(E[1] - E[0]) <= 1e-11 * abs(E[0])
    assert np.abs(U - np.eye(6)).max() <= 1e-8


def test_outer_loop_descends_above_the_full_space_energy():
    h, g = problem()
    E_full = oracle.ground_energy(8, 2, 2, h, g)
    E, U = oracle.optorb_run(h, g, 8, 6, 2, 2, outer=6, bb_steps=20)
    assert np.all(np.diff(E) <= 1e-12 * abs(E[0])), E
    assert E[-1] < E[0] - 1e-6                                      # the orbitals do improve
    assert np.all(E >= E_full - 1e-10)
    assert np.abs(U.T @ U - np.eye(6)).max() <= 1e-13
