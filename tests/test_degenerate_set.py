"""The library's degenerate set (cdfci_degenerate_set, host only: the configurations of the
k-space Hubbard start, reading of the paper's 4x4 example) against the oracle's independent
construction (no GPU needed)."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_04483_gb300 import api
    return api


@pytest.mark.parametrize("eps,na,nb,count", [
    (None, 8, 8, 400),                                   # the paper's 4x4 lattice: C(6, 3)^2
    ([0.0, 0.0, 0.0, 1.0, 1.0, 2.0], 2, 1, 9),           # one shell of 3 for both spins
    ([-1.0, 0.5, 0.5, 0.5, 0.5, 3.0], 3, 1, 6),          # alpha: 2 of 4 at 0.5; beta: the lowest alone
    ([-2.0, -1.0, -1.0, 1.0, 1.0, 2.0], 3, 3, 1),        # closed shells: one configuration
    ([0.3, 0.1, 0.2, 0.1, 0.9, 0.1], 0, 2, 3),           # no alpha electrons; 2 of the 3 at 0.1
])
def test_degenerate_set_matches_the_oracle(api, eps, na, nb, count):
    if eps is None:
        w = inputs.config3_k(4.0)
        h, g = w.h, w.g
    else:
        h = np.diag(eps)
        g = np.zeros((len(eps),) * 4)
    keys = api.cdfci_degenerate_set(np.diag(h), na, nb)
    ko, _, _ = oracle.degenerate_start(len(h), na, nb, h, g)
    assert len(keys) == count
    assert np.array_equal(keys, ko)
    # every member has the same, lowest one-body energy
    e = np.diag(h)
    one = [sum(e[p] for p in range(len(e)) if (int(a) >> p) & 1) + sum(e[p] for p in range(len(e)) if (int(b) >> p) & 1)
           for a, b in keys]
    assert max(one) == min(one)


def test_degenerate_set_errors(api):
    eps = np.diag(inputs.config3_k(4.0).h)
    with pytest.raises(api.CdfciError) as e:
        api.cdfci_degenerate_set(eps, 8, 8, cap=100)             # 400 > cap
    assert e.value.code == -8
    bad = eps.copy()
    bad[3] = np.nan
    with pytest.raises(api.CdfciError) as e:
        api.cdfci_degenerate_set(bad, 8, 8)
    assert e.value.code == -1
    with pytest.raises(api.CdfciError) as e:
        api.cdfci_degenerate_set(eps, 17, 8)
    assert e.value.code == -1
