"""xCDFCI (Algorithm 3, num_states = K + 1) on the GPU against the oracle:
start rows, step-by-step choices and energies, rows of C and B, convergence
to the lowest eigenvalues, determinism and error paths."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def solver(w, k1, **kw):
    from paper_2605_04483_gb300 import api
    kw.setdefault("log2_capacity", 16)
    return api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, num_states=k1, ref_alpha=int(w.ref[0]),
                      ref_beta=int(w.ref[1]), **kw)


def start_keys(g, k1):
    """The start rows D_k are the rows with C = e_k after cdfci_create."""
    keys, C, _ = g.export_states()
    out = []
    for k in range(k1):
        e = np.zeros(k1)
        e[k] = 1.0
        hit = [i for i in range(len(keys)) if np.array_equal(C[i], e)]
        assert len(hit) == 1
        out.append(keys[hit[0]])
    return np.array(out, dtype=np.uint64)


def rows_by_key(keys, R):
    return {(int(a), int(b)): R[i] for i, (a, b) in enumerate(keys)}


def compare_rows(g, o, tol=1e-11):
    kg, Cg, Bg = g.export_states()
    ko, Co, Bo = o.export()
    cg, bg, co, bo = rows_by_key(kg, Cg), rows_by_key(kg, Bg), rows_by_key(ko, Co), rows_by_key(ko, Bo)
    assert set(cg) == set(co)
    scale = max(1.0, max(np.abs(v).max() for v in bo.values()))
    for k in co:
        assert np.abs(cg[k] - co[k]).max() <= tol * max(1.0, np.abs(co[k]).max()), k
        assert np.abs(bg[k] - bo[k]).max() <= tol * scale, k


@pytest.mark.parametrize("k1, tau", [(3, 0.0), (2, 1e-4), (4, 3e-4)])
def test_trajectory_matches_oracle(k1, tau):
    w = inputs.ab_initio(8, 3, 3, seed=7)
    g = solver(w, k1, z_threshold=tau)
    keys = start_keys(g, k1)
    o = oracle.XCDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, keys, tau=tau)
    assert np.abs(g.energies() - o.energies()).max() <= 1e-11 * np.abs(o.energies()).max()
    compare_rows(g, o)
    for it in range(150):
        g.step(1)
        o.step(1)
        (kg,), _ = g.last_step()
        ko, _ = o.last_step()
        assert (int(kg[0]), int(kg[1])) == (int(ko[0]), int(ko[1])), it
        Eg, Eo = g.energies(), o.energies()
        assert np.abs(Eg - Eo).max() <= 1e-11 * np.abs(Eo).max(), (it, Eg, Eo)
        if (it + 1) % 50 == 0:
            compare_rows(g, o)
    st = g.stats()
    info = o.info()
    assert st["iterations"] == 150 and st["n_slots"] == info["entries"]
    assert st["elements"] == info["elements"] and st["applied"] == info["applied"] and st["dropped"] == info["dropped"]
    g.close(); o.close()


@pytest.mark.parametrize("k1", [2, 3])
def test_converges_to_the_lowest_eigenvalues(k1):
    w = inputs.ab_initio(6, 2, 2, seed=11)
    H = oracle.dense_H(6, 2, 2, w.h, w.g)
    exact = np.linalg.eigvalsh(H)[:k1]
    g = solver(w, k1)
    g.step(40000)
    E = g.energies()
    assert np.abs(E - exact).max() < 1e-8, (E, exact)
    g.close()


def test_graph_steps_equal_single_steps():
    w = inputs.ab_initio(10, 3, 3, seed=11)
    a = solver(w, 3, z_threshold=1e-5)
    b = solver(w, 3, z_threshold=1e-5)
    a.step(203)
    for _ in range(203):
        b.step(1)
    assert np.array_equal(a.energies(), b.energies())
    ka, Ca, _ = a.export_states()
    kb, Cb, _ = b.export_states()
    ra, rb = rows_by_key(ka, Ca), rows_by_key(kb, Cb)
    assert set(ra) == set(rb) and all(np.array_equal(ra[k], rb[k]) for k in ra)
    a.close(); b.close()


def test_errors():
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(8, 3, 3, seed=7)
    for kw in ({"num_states": 9}, {"num_states": 2, "num_coordinates": 4}):
        with pytest.raises(api.CdfciError) as e:
            api.Solver(w.h, w.g, 8, 3, 3, **kw)
        assert e.value.code == -1
    g = solver(w, 2)
    for call in (lambda: g.rdm(), lambda: g.export(), lambda: g.energy(1), lambda: g.checkpoint()):
        with pytest.raises(api.CdfciError) as e:
            call()
        assert e.value.code == -6
    g.close()
