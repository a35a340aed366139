"""GPU RDMs and energy derivatives (Sec. "Optimal Orbital Selections") against
the oracle's literal operator application, and the derivatives against
central finite differences of converged energies."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def solver(w, **kw):
    from paper_2605_04483_gb300 import api
    kw.setdefault("log2_capacity", 16)
    return api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]), **kw)


def sym8(G):
    return (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2) +
            G.transpose(2, 3, 0, 1) + G.transpose(3, 2, 0, 1) + G.transpose(2, 3, 1, 0) + G.transpose(3, 2, 1, 0)) / 8


@pytest.mark.parametrize("case,m,n_iter", [("abinitio", 1, 300), ("abinitio", 8, 40), ("hubbard", 1, 200),
                                           ("hubbard", 4, 30), ("abinitio_4_3", 1, 150)])
def test_rdm_matches_oracle_on_the_stored_vector(case, m, n_iter):
    """Any vector will do (no convergence needed): the RDMs of the exported
    (keys, c) by literal operator application against the GPU's."""
    w = {"abinitio": lambda: inputs.ab_initio(7, 3, 3, seed=4), "hubbard": inputs.config1,
         "abinitio_4_3": lambda: inputs.ab_initio(7, 4, 3, seed=9)}[case]()
    s = solver(w, num_coordinates=m)
    try:
        s.step(n_iter)
        keys, c, _ = s.export()
        g1, g2 = s.rdm()
        E_rq = s.energy(1)
    finally:
        s.close()
    o1, o2 = oracle.rdm(w.N, keys, c)
    assert np.abs(g1 - o1).max() <= 1e-12 * max(1.0, np.abs(o1).max())
    assert np.abs(g2 - o2).max() <= 1e-12 * max(1.0, np.abs(o2).max())
    n = w.n_alpha + w.n_beta
    assert abs(np.trace(g1) - n) < 1e-12
    assert abs(np.einsum("pprr->", g2) - n * (n - 1)) < 1e-10
    E = np.sum(w.h * g1) + 0.5 * np.sum(w.g * g2)
    assert abs(E - E_rq) < 1e-10 * max(1.0, abs(E_rq))


def test_gradient_entries_match_the_oracle_contractions():
    w = inputs.ab_initio(7, 3, 2, seed=6)
    s = solver(w, num_coordinates=1)
    try:
        s.step(400)
        keys, c, _ = s.export()
        dh, dg, dk = s.gradient()
    finally:
        s.close()
    o1, o2 = oracle.rdm(w.N, keys, c)
    assert np.abs(dh - o1).max() < 1e-12
    assert np.abs(dg - 0.5 * sym8(o2)).max() < 1e-12
    G = oracle.orbital_gradient(w.h, w.g, o1, o2)
    assert np.abs(dk - G).max() < 1e-11 * max(1.0, np.abs(G).max())
    assert np.abs(dk + dk.T).max() < 1e-14


def _energy(h, g, w, n_iter=20000):
    from paper_2605_04483_gb300.autograd import CDFCIEnergy
    return CDFCIEnergy.apply(h, g, w.N, w.n_alpha, w.n_beta, n_iter,
                             dict(log2_capacity=14, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1])))


def test_adjoint_matches_central_differences():
    """CDFCIEnergy.backward (the library's RDMs) against central differences,
    step 1e-5, of converged GPU energies along random symmetric directions of
    h and 8-fold symmetric directions of g, and along an orbital rotation."""
    w = inputs.ab_initio(6, 2, 2, seed=3)
    E0 = oracle.ground_energy(6, 2, 2, w.h, w.g)
    h = torch.tensor(w.h, requires_grad=True)
    g = torch.tensor(w.g, requires_grad=True)
    E = _energy(h, g, w)
    assert abs(E.item() - E0) < 1e-11
    dh, dg = torch.autograd.grad(E, (h, g))
    rng = np.random.default_rng(21)
    eps = 1e-5
    for _ in range(3):
        D = rng.normal(size=(6, 6)); D = D + D.T
        Ep = _energy(torch.tensor(w.h + eps * D), torch.tensor(w.g), w).item()
        Em = _energy(torch.tensor(w.h - eps * D), torch.tensor(w.g), w).item()
        fd = (Ep - Em) / (2 * eps)
        assert abs(fd - np.sum(D * dh.numpy())) <= 1e-7 * max(1.0, abs(fd)), (fd, np.sum(D * dh.numpy()))
        Gd = sym8(rng.normal(size=(6, 6, 6, 6)))
        Ep = _energy(torch.tensor(w.h), torch.tensor(w.g + eps * Gd), w).item()
        Em = _energy(torch.tensor(w.h), torch.tensor(w.g - eps * Gd), w).item()
        fd = (Ep - Em) / (2 * eps)
        assert abs(fd - np.sum(Gd * dg.numpy())) <= 1e-7 * max(1.0, abs(fd)), (fd, np.sum(Gd * dg.numpy()))
    # orbital rotation: dE = 1/2 sum G_pq dkappa_pq
    from paper_2605_04483_gb300.autograd import dE_dkappa, _solve
    s = _solve(h, g, 6, 2, 2, 20000, dict(log2_capacity=14, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1])))
    try:
        Gk = dE_dkappa(s).numpy()
    finally:
        s.close()
    K = rng.normal(size=(6, 6)); K = K - K.T
    hp, gp = oracle.rotate_integrals(w.h, w.g, eps * K)
    hm, gm = oracle.rotate_integrals(w.h, w.g, -eps * K)
    fd = (_energy(torch.tensor(hp), torch.tensor(gp), w).item() - _energy(torch.tensor(hm), torch.tensor(gm), w).item()) / (2 * eps)
    assert abs(fd - 0.5 * np.sum(Gk * K)) <= 1e-7 * max(1.0, abs(fd)), (fd, 0.5 * np.sum(Gk * K))
