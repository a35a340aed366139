"""Start vectors (cdfci_set_initial) against the oracle, and checkpoint /
restore (cdfci_checkpoint, cdfci_restore): a restored handle continues the
writer's trajectory."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu, vec_by_key

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def solver(w, **kw):
    from paper_2605_04483_gb300 import api
    kw.setdefault("log2_capacity", 16)
    return api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]), **kw)


def start_vector(w, n, seed):
    """n distinct determinants of the space (a seeded draw) with normal coefficients."""
    rng = np.random.default_rng(seed)
    keys = set()
    while len(keys) < n:
        a = rng.choice(w.N, size=w.n_alpha, replace=False)
        b = rng.choice(w.N, size=w.n_beta, replace=False)
        keys.add((int(sum(1 << int(x) for x in a)), int(sum(1 << int(x) for x in b))))
    keys = np.array(sorted(keys), dtype=np.uint64)
    return keys[rng.permutation(len(keys))], rng.normal(size=n)


def assert_same_vectors(g, o, tol=1e-11):
    kg, cg, bg = g.export()
    ko, co, bo = o.export()
    mc_g, mb_g, mc_o, mb_o = vec_by_key(kg, cg), vec_by_key(kg, bg), vec_by_key(ko, co), vec_by_key(ko, bo)
    assert set(mc_g) == set(mc_o)
    scale = max(1.0, max(abs(v) for v in mb_o.values()))
    for k in mc_o:
        assert abs(mc_g[k] - mc_o[k]) <= tol * max(1.0, abs(mc_o[k]))
        assert abs(mb_g[k] - mb_o[k]) <= tol * scale, (k, mb_g[k], mb_o[k])


@pytest.mark.parametrize("grid_blocks", [2, 24])
def test_single_entry_start_equals_create(grid_blocks):
    """set_initial(e_ref) reproduces the handle cdfci_create starts (bitwise, m = 1)."""
    w = inputs.ab_initio(10, 4, 4, seed=9)
    a = solver(w, grid_blocks=grid_blocks)
    b = solver(w, grid_blocks=grid_blocks)
    ka, ca, _ = a.export()
    b.step(50)
    b.set_initial(ka[np.argmax(np.abs(ca))][None, :], np.array([1.0]))
    assert b.stats()["iterations"] == 0
    sa, sb = a.step(300), b.step(300)
    assert sa["energy"] == sb["energy"] and sa["iterations"] == sb["iterations"]
    ka, ca, ba = a.export()
    kb, cb, bb = b.export()
    assert vec_by_key(ka, ca) == vec_by_key(kb, cb) and vec_by_key(ka, ba) == vec_by_key(kb, bb)
    a.close(); b.close()


@pytest.mark.parametrize("tau", [0.0, 3e-4])
def test_start_vector_trajectory_matches_oracle(tau):
    """A 25-determinant start vector: the same stored set, c and b as the oracle,
    then 150 steps of Algorithm 1 along the oracle's trajectory."""
    w = inputs.ab_initio(10, 4, 4, seed=8)
    keys, c = start_vector(w, 25, seed=1)
    g = solver(w, z_threshold=tau)
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, w.ref, tau, 1)
    g.set_initial(keys, c)
    o.set_initial(keys, c)
    st = g.stats()
    assert abs(st["energy"] - o.energy()) <= 1e-11 * abs(o.energy())
    assert st["iterations"] == 0 and st["nnz_c"] == 25
    assert_same_vectors(g, o)
    for it in range(150):
        g.step(1)
        (kg,), (eg,) = g.last_step()
        gc, gm = o.step_choice(kg)
        assert gc >= gm * (1 - 1e-12), (it, gc, gm)
        assert abs(g.stats()["energy"] - o.energy()) <= 1e-11 * abs(o.energy()), it
    assert_same_vectors(g, o)
    g.close(); o.close()


def test_start_vector_block_matches_oracle():
    """m = 8: a start of 8 entries as one-coordinate block steps, then 12 block iterations."""
    w = inputs.ab_initio(9, 4, 3, seed=17)
    keys, c = start_vector(w, 8, seed=2)
    g = solver(w, num_coordinates=8, z_threshold=1e-4)
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, w.ref, 1e-4, 8)
    g.set_initial(keys, c)
    o.set_initial(keys, c)
    assert abs(g.stats()["energy"] - o.energy()) <= 1e-11 * abs(o.energy())
    assert_same_vectors(g, o, tol=1e-11)
    g.step(12)
    o.step(12)
    assert abs(g.stats()["energy"] - o.energy()) <= 1e-9 * abs(o.energy())
    g.close(); o.close()


def test_start_vector_errors():
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(8, 3, 3, seed=7)
    g = solver(w)
    keys, c = start_vector(w, 5, seed=3)
    for bad_keys, bad_c in [(keys[[0, 1, 0]], c[:3]),                                   # repeated key
                            (np.array([[0b1111, 0b111]], dtype=np.uint64), np.ones(1)),  # 4 alpha electrons
                            (np.array([[0b111, 1 << 9 | 3]], dtype=np.uint64), np.ones(1)),  # orbital 9 >= N
                            (keys, np.zeros(5)),                                           # all zero
                            (keys[:1], np.array([np.nan]))]:
        with pytest.raises(api.CdfciError) as e:
            g.set_initial(bad_keys, bad_c)
        assert e.value.code == -1
    g.close()


def test_start_vector_longer_than_the_block():
    """m = 4 with a start of 5 entries: the candidates of all start columns fit the list
    (its capacity bounds every write on the device), the state matches the oracle's."""
    w = inputs.ab_initio(8, 3, 3, seed=7)
    keys, c = start_vector(w, 5, seed=3)
    h4 = solver(w, num_coordinates=4)
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, w.ref, 0.0, 4)
    h4.set_initial(keys, c)
    o.set_initial(keys, c)
    assert abs(h4.stats()["energy"] - o.energy()) <= 1e-11 * abs(o.energy())
    assert_same_vectors(h4, o, tol=1e-11)
    h4.step(10)
    o.step(10)
    assert abs(h4.stats()["energy"] - o.energy()) <= 1e-9 * abs(o.energy())
    h4.close(); o.close()


@pytest.mark.parametrize("grid_a, grid_b", [(24, 24), (4, 4), (24, 4)])
def test_checkpoint_restore_continues_the_trajectory(grid_a, grid_b, tmp_path):
    """m = 1: 300 steps, checkpoint (through a file), 200 more; a new handle restored from the
    checkpoint takes the same 200 steps: bitwise on the same grid, to 1e-12 on another."""
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(12, 4, 4, seed=3)
    a = solver(w, grid_blocks=grid_a, z_threshold=1e-5, log2_capacity=18)
    a.step(300)
    ck = a.checkpoint()
    assert ck["header"].have_prev == 1 and ck["header"].n_entries == a.stats()["n_slots"]
    api.save_checkpoint(str(tmp_path / "a.npz"), ck)
    sa = a.step(200)
    ka, ca, ba = a.export()
    trail_a = a.last_step()
    b = solver(w, grid_blocks=grid_b, z_threshold=1e-5, log2_capacity=17)
    b.step(7)                                         # a different state that restore replaces
    b.restore(api.load_checkpoint(str(tmp_path / "a.npz")))
    s0 = b.stats()
    assert s0["iterations"] == 300 and s0["n_slots"] == ck["header"].n_entries
    sb = b.step(200)
    kb, cb, bb = b.export()
    assert sb["iterations"] == sa["iterations"]
    if grid_a == grid_b:
        assert sb["energy"] == sa["energy"]
        assert vec_by_key(ka, ca) == vec_by_key(kb, cb) and vec_by_key(ka, ba) == vec_by_key(kb, bb)
        assert np.array_equal(trail_a[0], b.last_step()[0])
    else:
        assert abs(sb["energy"] - sa["energy"]) <= 1e-12 * abs(sa["energy"])
        mc_a, mc_b = vec_by_key(ka, ca), vec_by_key(kb, cb)
        assert set(mc_a) == set(mc_b)
        assert max(abs(mc_a[k] - mc_b[k]) for k in mc_a) <= 1e-10
    a.close(); b.close()


def test_checkpoint_restore_block():
    """m = 16: restore continues the block trajectory (FP64 atomics: agreement to the last bits)."""
    w = inputs.ab_initio(12, 4, 4, seed=3)
    a = solver(w, num_coordinates=16, z_threshold=1e-5, log2_capacity=18)
    a.step(40)
    ck = a.checkpoint()
    assert ck["flags"].sum() > 0                      # the candidates of the next selection travel along
    sa = a.step(25)
    b = solver(w, num_coordinates=16, z_threshold=1e-5, log2_capacity=18)
    b.restore(ck)
    assert b.stats()["iterations"] == 40
    sb = b.step(25)
    assert sb["iterations"] == sa["iterations"]
    assert abs(sb["energy"] - sa["energy"]) <= 1e-9 * abs(sa["energy"])
    a.close(); b.close()


def test_restore_errors():
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(10, 4, 4, seed=9)
    a = solver(w)
    a.step(20)
    ck = a.checkpoint()
    other = inputs.ab_initio(10, 3, 4, seed=9)
    b = solver(other)
    with pytest.raises(api.CdfciError) as e:
        b.restore(ck)                                   # electron counts differ
    assert e.value.code == -1
    m4 = solver(w, num_coordinates=4)
    with pytest.raises(api.CdfciError) as e:
        m4.restore(ck)                                  # m = 1 checkpoint on an m > 1 handle
    assert e.value.code == -1
    small = solver(w, log2_capacity=5, z_threshold=1e3)     # the reference column stores nothing else
    with pytest.raises(api.CdfciError) as e:
        small.restore(ck)                               # more rows than max_load of 32 slots
    assert e.value.code == -3
    for s in (a, b, m4, small):
        s.close()


def test_restore_grows_the_candidate_list():
    """A checkpoint whose candidate list is longer than one iteration makes (a start vector of 12
    columns at m = 4) restored into a fresh m = 4 handle: the restore grows the handle's list to hold
    every flagged candidate, and the continuation follows the writer's and the oracle's."""
    w = inputs.ab_initio(8, 3, 3, seed=7)
    keys, c = start_vector(w, 12, seed=5)
    a = solver(w, num_coordinates=4)
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, w.ref, 0.0, 4)
    a.set_initial(keys, c)
    o.set_initial(keys, c)
    ck = a.checkpoint()
    n_h = 1 + 2 * 3 * 5 + 2 * 3 * 10 + 15 * 15              # column length of N = 8, 3 + 3
    assert ck["flags"].sum() > 4 * n_h + 4 + 64               # more than a fresh m = 4 handle's list
    b = solver(w, num_coordinates=4)
    b.restore(ck)
    assert b.stats()["energy"] == a.stats()["energy"]
    sa, sb = a.step(12), b.step(12)
    o.step(12)
    assert sa["iterations"] == sb["iterations"]
    assert abs(sb["energy"] - sa["energy"]) <= 1e-10 * abs(sa["energy"])
    assert abs(sb["energy"] - o.energy()) <= 1e-9 * abs(o.energy())
    a.close(); b.close(); o.close()
