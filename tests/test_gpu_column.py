"""GPU column enumeration (get_column) against the oracle: the key set (excitations,
hence determinants) bit-exact, signs exact, values within 1e-12 relative of the oracle's."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import ElementCheck, colmap, order_tol, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def check_columns(w, dets, literal=False):
    from paper_2605_04483_gb300 import api
    chk = ElementCheck(f"get_column N={w.N} {w.n_alpha}+{w.n_beta}")
    va, vb = w.N - w.n_alpha, w.N - w.n_beta
    nh = 1 + w.n_alpha * va + w.n_beta * vb + math.comb(w.n_alpha, 2) * math.comb(va, 2) + \
        math.comb(w.n_beta, 2) * math.comb(vb, 2) + w.n_alpha * va * w.n_beta * vb
    log2cap = max(10, int(math.ceil(math.log2(2 * nh))))     # the start column must fit at load <= 0.79
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=log2cap, ref_alpha=int(dets[0][0]),
                   ref_beta=int(dets[0][1]))
    try:
        for d in dets:
            k1, v1 = s.column(d)
            m1 = colmap(k1, v1)
            assert len(m1) == len(k1), "duplicate determinant in a GPU column"
            m2 = colmap(*oracle.column_sc(w.N, w.h, w.g, d))
            assert set(m1) == set(m2), f"key sets differ for det {d}: {len(set(m1) ^ set(m2))} keys"
            for k, v in m2.items():
                chk(w, m1[k], v, k)
                assert np.sign(m1[k]) == np.sign(v)
            if literal:                  # the definition itself: keys and signs exact, values to the order bound
                m3 = colmap(*oracle.column_literal(w.N, w.h, w.g, d))
                assert set(m1) == set(m3)
                for k, v in m3.items():
                    assert abs(m1[k] - v) <= order_tol(w, v), (k, m1[k], v)
                    assert np.sign(m1[k]) == np.sign(v)
    finally:
        s.close()
    chk.report()


def test_column_config1_hubbard_chain():
    w = inputs.config1()
    dets = oracle.fci_dets(8, 4, 4)[::7]
    check_columns(w, dets, literal=True)


def test_column_all_dets_small_ab_initio():
    w = inputs.ab_initio(8, 3, 3, seed=7)
    check_columns(w, oracle.fci_dets(8, 3, 3), literal=False)
    check_columns(w, oracle.fci_dets(8, 3, 3)[::50], literal=True)


def test_column_config2_size():
    """N = 24, 6 + 6 (config 2): column length 16,471."""
    w = inputs.config2()
    dets = inputs.random_determinants(24, 6, 6, 4, seed=5)
    check_columns(w, dets, literal=False)
    check_columns(w, dets[:1], literal=True)
    from paper_2605_04483_gb300 import api
    s = api.Solver(w.h, w.g, 24, 6, 6, log2_capacity=16)
    k, v = s.column(dets[0])
    s.close()
    assert len(k) == 1 + 2 * 6 * 18 + 2 * math.comb(6, 2) * math.comb(18, 2) + (6 * 18) ** 2 == 16471


def test_column_largest_batch_instance():
    """N = 32, 8 + 8: the largest instance of the uneven batch (52,705 elements)."""
    w = inputs.ab_initio(32, 8, 8, seed=1234)
    check_columns(w, inputs.random_determinants(32, 8, 8, 2, seed=6), literal=False)


def test_column_hubbard_4x4():
    w = inputs.config3(U=8.0)
    check_columns(w, inputs.random_determinants(16, 8, 8, 20, seed=7), literal=False)


@pytest.mark.parametrize("N,na,nb", [(6, 0, 3), (6, 3, 0), (5, 5, 2), (5, 2, 5), (1, 1, 1), (2, 1, 1),
                                     (40, 2, 1), (63, 1, 1)])
def test_column_edge_shapes(N, na, nb):
    w = inputs.ab_initio(N, na, nb, seed=N * 10 + na, n_chol=8)
    dets = inputs.random_determinants(N, na, nb, 3, seed=N)
    check_columns(w, dets, literal=(N <= 6))


def test_column_device_key_and_outputs():
    """Device-resident key and output buffers (torch tensors) give the same column."""
    import torch
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(10, 4, 3, seed=3)
    s = api.Solver(w.h, w.g, 10, 4, 3, log2_capacity=10)
    d = inputs.random_determinants(10, 4, 3, 1, seed=1)[0]
    k1, v1 = s.column(d)
    kd = torch.tensor(d.astype(np.int64), device="cuda")
    ko = torch.zeros((len(k1), 2), dtype=torch.int64, device="cuda")
    vo = torch.zeros(len(k1), dtype=torch.float64, device="cuda")
    import ctypes
    n = ctypes.c_int64()
    rc = api.lib().cdfci_get_column(s.handle, kd.data_ptr(), ko.data_ptr(), vo.data_ptr(), len(k1), ctypes.byref(n))
    assert rc == 0 and n.value == len(k1)
    m1 = colmap(k1, v1)
    m2 = colmap(ko.cpu().numpy().astype(np.uint64), vo.cpu().numpy())
    assert m1 == m2
    s.close()

