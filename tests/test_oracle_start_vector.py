"""Start vectors in the oracle (the reading behind cdfci_set_initial) and the
checkpoint file format, without a GPU."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs


def ref_key(o):
    k, c, _ = o.export()
    return k[np.argmax(np.abs(c))]


@pytest.mark.parametrize("m", [1, 4])
def test_single_entry_start_is_the_reference_start(m):
    """c = 1 e_ref through set_initial is exactly the initialisation of Algorithms 1 and 2."""
    w = inputs.ab_initio(7, 3, 2, seed=5)
    a = oracle.CDFCI(7, 3, 2, w.h, w.g, w.ref, 1e-3, m)
    b = oracle.CDFCI(7, 3, 2, w.h, w.g, w.ref, 1e-3, m)
    b.set_initial(ref_key(a)[None, :], np.array([1.0]))
    for o in (a, b):
        o.step(15)
    ka, ca, ba = a.export()
    kb, cb, bb = b.export()
    assert a.energy() == b.energy()
    da = {tuple(k): (x, y) for k, x, y in zip(map(tuple, ka), ca, ba)}
    db = {tuple(k): (x, y) for k, x, y in zip(map(tuple, kb), cb, bb)}
    assert da == db
    a.close(); b.close()


def test_start_vector_without_compression_gives_b_equal_Hc():
    """tau = 0: after the start steps b = H c on every stored determinant, every
    nonzero of H c is stored, mu = c.c and alpha = c.H c (dense H of the FCI space)."""
    N, na, nb = 6, 2, 2
    w = inputs.ab_initio(N, na, nb, seed=8)
    dets = oracle.fci_dets(N, na, nb)
    H = oracle.dense_H(N, na, nb, w.h, w.g)
    rng = np.random.default_rng(4)
    pick = rng.choice(len(dets), size=15, replace=False)
    cvals = rng.normal(size=15)
    cvals[3] = 0.0                                   # a zero entry is allowed
    o = oracle.CDFCI(N, na, nb, w.h, w.g, w.ref, 0.0, 1)
    o.set_initial(dets[pick], cvals)
    cfull = np.zeros(len(dets))
    cfull[pick] = cvals
    Hc = H @ cfull
    index = {(int(a), int(b)): i for i, (a, b) in enumerate(dets)}
    k, c, b = o.export()
    stored = {index[(int(x), int(y))] for x, y in k}
    assert {i for i in range(len(dets)) if Hc[i] != 0.0 or cfull[i] != 0.0} <= stored
    for (x, y), cv, bv in zip(k, c, b):
        i = index[(int(x), int(y))]
        assert cv == cfull[i]
        assert abs(bv - Hc[i]) <= 1e-12 * max(1.0, np.abs(Hc).max())
    info = o.info()
    assert abs(info["mu"] - cvals @ cvals) <= 1e-13 * (cvals @ cvals)
    assert abs(info["alpha"] - cfull @ Hc) <= 1e-12 * max(1.0, abs(cfull @ Hc))
    assert info["iterations"] == 0
    o.close()


def test_start_vector_rejects_a_repeated_key():
    w = inputs.ab_initio(6, 2, 2, seed=8)
    dets = oracle.fci_dets(6, 2, 2)
    o = oracle.CDFCI(6, 2, 2, w.h, w.g, w.ref, 0.0, 1)
    with pytest.raises(RuntimeError):
        o.set_initial(dets[[3, 5, 3]], np.array([1.0, 0.5, 0.25]))
    o.close()


def test_checkpoint_file_round_trip(tmp_path):
    """The .npz checkpoint keeps the header bytes and the rows unchanged."""
    from paper_2605_04483_gb300 import api
    hdr = api.cdfci_checkpoint_header()
    hdr.version = 1; hdr.N = 24; hdr.n_alpha = 6; hdr.n_beta = 6; hdr.num_coordinates = 1
    hdr.n_entries = 3; hdr.mu[0] = 1.25; hdr.mu[1] = 1e-17; hdr.prev_key[0] = 0x3f; hdr.gather = -0.5
    hdr.pending[2] = 7
    ck = {"header": hdr, "keys": np.array([[1, 2], [3, 4], [5, 6]], dtype=np.uint64), "c": np.array([0.5, 0.0, -1.0]),
          "b": np.array([1.0, 2.0, 3.0]), "flags": np.array([1, 0, 1], dtype=np.uint8)}
    p = tmp_path / "ck.npz"
    api.save_checkpoint(str(p), ck)
    back = api.load_checkpoint(str(p))
    assert bytes(back["header"]) == bytes(hdr)
    for k in ("keys", "c", "b", "flags"):
        assert np.array_equal(back[k], ck[k]) and back[k].dtype == ck[k].dtype
