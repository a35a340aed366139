"""Batches of independent problems of different sizes: m = 1 problems in one launch follow exactly
the trajectory they follow alone; m > 1 problems (Algorithm 2, one graph branch each) follow theirs up
to the order of the FP64 atomics on b; every problem converges to the oracle's exact energy."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def problems():
    return [inputs.ab_initio(6, 2, 2, seed=31), inputs.ab_initio(8, 3, 2, seed=32), inputs.config1(),
            inputs.ab_initio(10, 3, 3, seed=11), inputs.ab_initio(7, 3, 3, seed=33),
            inputs.hubbard((2, 3), 3, 3, U=8.0)]


def make(ws, grid_blocks=1, **kw):
    from paper_2605_04483_gb300 import api
    return [api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=16, grid_blocks=grid_blocks,
                       ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]), **kw) for w in ws]


@pytest.mark.parametrize("grid_blocks", [1, 2])
def test_batched_trajectories_equal_the_single_ones(grid_blocks):
    from paper_2605_04483_gb300 import api
    ws = problems()
    alone = make(ws, grid_blocks)
    batched = make(ws, grid_blocks)
    b = api.Batch(batched)
    try:
        for n in (1, 7, 300):
            st_b = b.step(n)
            st_a = [s.step(n) for s in alone]
            for k, (x, y) in enumerate(zip(st_a, st_b)):
                for f in ("iterations", "energy", "mu", "alpha", "dx", "nnz_c", "n_slots", "elements", "applied"):
                    assert x[f] == y[f], (k, f, x[f], y[f])
        # the handles stay usable on their own after batched steps
        x, y = alone[0].step(5), batched[0].step(5)
        assert x["energy"] == y["energy"] and x["iterations"] == y["iterations"]
        for sa, sb in zip(alone[:3], batched[:3]):
            ka, ca, _ = sa.export()
            kb, cb, _ = sb.export()
            oa, ob = np.lexsort(ka.T[::-1]), np.lexsort(kb.T[::-1])
            assert np.array_equal(ka[oa], kb[ob]) and np.array_equal(ca[oa], cb[ob])
    finally:
        b.close()
        for s in alone + batched:
            s.close()


def test_batch_converges_every_problem():
    from paper_2605_04483_gb300 import api
    ws = problems()[:5]
    ss = make(ws)
    b = api.Batch(ss)
    try:
        st = b.step(300000)                   # the 8-site Hubbard chain needs about 3e5 at m = 1
        for w, x in zip(ws, st):
            E0 = oracle.ground_energy(w.N, w.n_alpha, w.n_beta, w.h, w.g, dense_limit=5000)
            assert abs(x["energy"] - E0) < 1e-8, (w.N, x["energy"] - E0)
    finally:
        b.close()
        for s in ss:
            s.close()


def test_batch_rejects_invalid_sets():
    from paper_2605_04483_gb300 import api
    ws = problems()[:2]
    a = make(ws[:1])[0]
    g2 = make(ws[1:2], grid_blocks=2)[0]
    x2 = api.Solver(ws[1].h, ws[1].g, ws[1].N, ws[1].n_alpha, ws[1].n_beta, num_states=2, log2_capacity=14)
    try:
        with pytest.raises(api.CdfciError):
            api.Batch([a, g2])                        # m = 1 solvers with different CTAs per problem
        with pytest.raises(api.CdfciError):
            api.Batch([a, a])
        with pytest.raises(api.CdfciError):
            api.Batch([a, x2])                        # excited states
    finally:
        for s in (a, g2, x2):
            s.close()


def block_problems():
    """Ab initio problems without exact ties of |g| (the chosen blocks do not depend on rounding)."""
    return [inputs.ab_initio(6, 2, 2, seed=31), inputs.ab_initio(8, 3, 2, seed=32),
            inputs.ab_initio(10, 3, 3, seed=11), inputs.ab_initio(7, 3, 3, seed=33),
            inputs.ab_initio(12, 3, 3, seed=2)]


def test_block_batch_follows_the_single_runs():
    """m > 1 problems with different m and sizes in one graph: the same chosen blocks (element counts)
    and energies as alone, below, at and above the graph chunk of 8 iterations; m = 1 problems in
    the same batch follow theirs exactly."""
    from paper_2605_04483_gb300 import api
    ws = block_problems()
    ms = [4, 16, 8, 32, 64]
    alone = [make([w], num_coordinates=m)[0] for w, m in zip(ws, ms)] + make(problems()[2:3])
    batched = [make([w], num_coordinates=m)[0] for w, m in zip(ws, ms)] + make(problems()[2:3])
    b = api.Batch(batched)
    try:
        for n in (3, 8, 21, 40):
            st_b = b.step(n)
            st_a = [s.step(n) for s in alone]
            for k, (x, y) in enumerate(zip(st_a, st_b)):
                assert x["iterations"] == y["iterations"], k
                assert x["elements"] == y["elements"], (k, x["elements"], y["elements"])
                assert abs(x["energy"] - y["energy"]) <= 1e-10 * abs(x["energy"]), (k, x["energy"], y["energy"])
                if k == len(ws):                          # the m = 1 problem: bit for bit
                    for f in ("energy", "mu", "alpha", "dx", "nnz_c", "n_slots", "applied"):
                        assert x[f] == y[f], (f, x[f], y[f])
        x, y = alone[0].step(8), batched[0].step(8)       # a batched handle goes on alone
        assert abs(x["energy"] - y["energy"]) <= 1e-10 * abs(x["energy"])
    finally:
        b.close()
        for s in alone + batched:
            s.close()


def test_block_batch_converges_every_problem():
    from paper_2605_04483_gb300 import api
    ws = block_problems()[:4] + [inputs.config1()]
    ms = [8, 16, 64, 64, 128]
    ss = [make([w], num_coordinates=m)[0] for w, m in zip(ws, ms)]
    b = api.Batch(ss)
    try:
        st = b.step(12000)
        for w, x in zip(ws, st):
            E0 = oracle.ground_energy(w.N, w.n_alpha, w.n_beta, w.h, w.g, dense_limit=5000)
            assert abs(x["energy"] - E0) < 1e-8, (w.N, x["energy"] - E0)
    finally:
        b.close()
        for s in ss:
            s.close()
