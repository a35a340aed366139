"""OptOrbFCI (Algorithm 4) through cdfci_optorb against the oracle's outer loop
(exact FCI per basis): energies per outer iteration, the final basis, the
invariance of a full orbital space, argument errors."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_matches_the_oracle_outer_loop():
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(8, 2, 2, seed=4)
    E_o, U_o = oracle.optorb_run(w.h, w.g, 8, 6, 2, 2, outer=4, bb_steps=12)
    U, E = api.cdfci_optorb(w.h, w.g, 8, 6, 2, 2, outer=4, bb_steps=12, inner_iterations=40000, log2_capacity=12)
    assert np.abs(E - E_o).max() < 1e-8, (E, E_o)
    assert np.all(np.diff(E) <= 1e-10 * abs(E[0]))
    assert np.abs(U.T @ U - np.eye(6)).max() < 1e-13
    assert np.abs(U - U_o).max() < 1e-6


def test_full_space_is_invariant():
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(6, 2, 2, seed=4)
    U, E = api.cdfci_optorb(w.h, w.g, 6, 6, 2, 2, outer=2, bb_steps=6, inner_iterations=40000, log2_capacity=12)
    assert abs(E[1] - E[0]) < 1e-10 * abs(E[0])
    assert np.abs(U - np.eye(6)).max() < 1e-7


def test_errors():
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(8, 2, 2, seed=4)
    for args, kw in [((8, 9, 2, 2), {}),                                    # N > M
                     ((8, 6, 2, 2), {"U0": np.ones((8, 6))}),               # not orthonormal
                     ((8, 6, 2, 2), {"num_states": 2})]:
        with pytest.raises(api.CdfciError) as e:
            api.cdfci_optorb(w.h, w.g, *args, outer=1, bb_steps=1, inner_iterations=10, **kw)
        assert e.value.code == -1
