"""Single matrix elements (cdfci_get_entry / cdfci_get_diagonal, the get_entry and get_diagonal of
Sec. "The Hamiltonian Class") against the oracle's columns."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import ElementCheck, colmap, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()



@pytest.mark.parametrize("kind", ["ab_initio", "hubbard_k"])
def test_entry_and_diagonal_match_the_oracle(kind):
    """get_entry / get_diagonal of Sec. "The Hamiltonian Class": the oracle's column values for
    pairs inside a column (either key order: H is symmetric), 0.0 beyond a double excitation, and
    the diagonal; for the 8-fold ab initio integrals and the 4-fold k-space ones."""
    from paper_2605_04483_gb300 import api
    if kind == "ab_initio":
        w, sym = inputs.ab_initio(10, 4, 3, seed=3), 8
    else:
        w, sym = inputs.hubbard_k((2, 3), 3, 2, U=2.0), 4
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=12, integral_symmetry=sym)
    chk = ElementCheck(f"get_entry/get_diagonal {kind}")
    try:
        dets = oracle.fci_dets(w.N, w.n_alpha, w.n_beta)
        rng = np.random.default_rng(4)
        for d in dets[rng.choice(len(dets), 5, replace=False)]:
            ko, vo = oracle.column_sc(w.N, w.h, w.g, d)
            col = colmap(ko, vo)
            dv = col.get((int(d[0]), int(d[1])), 0.0)
            chk(w, s.diagonal(d), dv, "diagonal")
            for k in list(col)[:: max(1, len(col) // 10)]:
                kk = np.array(k, dtype=np.uint64)
                chk(w, s.entry(kk, d), col[k], k)
                chk(w, s.entry(d, kk), col[k], k)
        ref = dets[0]
        far = [x for x in dets if bin(int(x[0]) ^ int(ref[0])).count("1") + bin(int(x[1]) ^ int(ref[1])).count("1") > 4]
        assert far and s.entry(ref, far[0]) == 0.0
        with pytest.raises(api.CdfciError) as e:
            s.entry(ref, np.array([1, 1], dtype=np.uint64))        # wrong electron counts
        assert e.value.code == -1
    finally:
        s.close()
    chk.report()
