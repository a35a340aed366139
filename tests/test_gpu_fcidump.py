"""Algorithm 1 from an FCIDUMP file (Sec. "Example Usage"): the integrals the library reads drive the
GPU solver, and its trajectory matches the oracle run on the generator's integrals (which the CPU
round-trip test shows to be the same doubles)."""
import numpy as np
import pytest

import oracle
from paper_2605_04483_gb300 import inputs
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_cdfci_from_fcidump_matches_the_oracle(tmp_path):
    require_gpu()
    from paper_2605_04483_gb300 import api
    w = inputs.ab_initio(10, 3, 3, seed=31)
    p = tmp_path / "w.FCIDUMP"
    inputs.write_fcidump(str(p), w, e_core=3.25)
    r = api.cdfci_fcidump_read(str(p))
    s = api.Solver(r["h"], r["g"], r["N"], r["n_alpha"], r["n_beta"], log2_capacity=16,
                   ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, (int(w.ref[0]), int(w.ref[1])), 0.0, 1)
    try:
        for _ in range(5):
            st = s.step(60)
            o.step(60)
            assert abs(st["energy"] - o.energy()) < 1e-11, (st["energy"], o.energy())
        assert r["e_core"] == 3.25
    finally:
        s.close()
        o.close()
