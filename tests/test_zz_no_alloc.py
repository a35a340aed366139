"""cdfci_column_noalloc, the get_column entry point for callers that cannot call
cudaMalloc (code inside a memory pool or allocator it does not own, or a
framework that forbids allocation on its hot path), against the handle-based
cdfci_get_column.  Collected last so that a failure here does not stop the
other GPU tests; it also runs alone in a fresh process."""
import numpy as np
import pytest

from gpu_util import colmap, element_tol, require_gpu

pytestmark = pytest.mark.gpu


def _reference_column(api, w, det):
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=17,
                   ref_alpha=int(det[0]), ref_beta=int(det[1]))
    try:
        return s.column(det)
    finally:
        s.close()


def test_column_noalloc_matches_get_column_on_two_calls():
    require_gpu()
    import torch
    from paper_2605_04483_gb300 import api, inputs

    # a large problem first, then a small one: the shared scratch keeps the
    # first call's tables, which must not leak into the second call
    cases = [(inputs.config2(), inputs.random_determinants(24, 6, 6, 1, seed=11)[0]),
             (inputs.ab_initio(8, 3, 2, seed=5), inputs.random_determinants(8, 3, 2, 1, seed=12)[0])]
    for w, det in cases:
        k_ref, v_ref = _reference_column(api, w, det)
        h = torch.tensor(w.h, device="cuda")
        g = torch.tensor(w.g, device="cuda")
        cap = len(k_ref)
        keys = torch.zeros((cap, 2), dtype=torch.int64, device="cuda")
        vals = torch.zeros(cap, dtype=torch.float64, device="cuda")
        n = api.cdfci_column_noalloc(h, g, w.N, w.n_alpha, w.n_beta, np.ascontiguousarray(det, dtype=np.uint64),
                                     keys, vals, cap)
        assert n == cap
        m_ref = colmap(k_ref, v_ref)
        m_new = colmap(keys.cpu().numpy().astype(np.uint64), vals.cpu().numpy())
        assert set(m_new) == set(m_ref)
        for k, v in m_ref.items():
            assert abs(m_new[k] - v) <= element_tol(w, v), (k, m_new[k], v)


def test_column_noalloc_rejects_sizes_beyond_the_scratch_limit():
    require_gpu()
    import torch
    from paper_2605_04483_gb300 import api
    h = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(api.CdfciError) as e:
        api.cdfci_column_noalloc(h, h, 64, 1, 1, np.array([1, 1], dtype=np.uint64), out, out, 2)
    assert e.value.code == -1 and "scratch limit" in str(e.value)
