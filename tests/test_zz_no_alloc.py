"""cdfci_column_noalloc, the get_column entry point for callers that cannot call
cudaMalloc (code inside a memory pool or allocator it does not own, or a
framework that forbids allocation on its hot path): against the oracle's
Slater-Condon columns and the handle-based cdfci_get_column, on two calls in a
row; no device memory taken by repeated calls; a capturing stream refused.
Collected last so that a failure here does not stop the other GPU tests; it
also runs alone in a fresh process."""
import numpy as np
import pytest

import oracle
from gpu_util import ElementCheck, colmap, require_gpu

pytestmark = pytest.mark.gpu


def _reference_column(api, w, det):
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=17,
                   ref_alpha=int(det[0]), ref_beta=int(det[1]))
    try:
        return s.column(det)
    finally:
        s.close()


def _noalloc(api, torch, w, det, cap, h=None, g=None):
    h = torch.tensor(w.h, device="cuda") if h is None else h
    g = torch.tensor(w.g, device="cuda") if g is None else g
    keys = torch.zeros((cap, 2), dtype=torch.int64, device="cuda")
    vals = torch.zeros(cap, dtype=torch.float64, device="cuda")
    n = api.cdfci_column_noalloc(h, g, w.N, w.n_alpha, w.n_beta, np.ascontiguousarray(det, dtype=np.uint64),
                                 keys, vals, cap)
    return n, keys, vals


def test_column_noalloc_matches_get_column_and_the_oracle_on_two_calls():
    require_gpu()
    import torch
    from paper_2605_04483_gb300 import api, inputs

    # a large problem first, then a small one: the shared scratch keeps the
    # first call's tables, which must not leak into the second call
    cases = [(inputs.config2(), inputs.random_determinants(24, 6, 6, 1, seed=11)[0]),
             (inputs.ab_initio(8, 3, 2, seed=5), inputs.random_determinants(8, 3, 2, 1, seed=12)[0])]
    chk_ref, chk_orc = ElementCheck("noalloc vs get_column"), ElementCheck("noalloc vs oracle")
    for w, det in cases:
        k_ref, v_ref = _reference_column(api, w, det)
        cap = len(k_ref)
        n, keys, vals = _noalloc(api, torch, w, det, cap)
        assert n == cap
        m_new = colmap(keys.cpu().numpy().astype(np.uint64), vals.cpu().numpy())
        m_ref = colmap(k_ref, v_ref)
        m_orc = colmap(*oracle.column_sc(w.N, w.h, w.g, det))
        assert set(m_new) == set(m_ref) == set(m_orc)
        for k, v in m_ref.items():
            chk_ref(w, m_new[k], v, k)
        for k, v in m_orc.items():
            chk_orc(w, m_new[k], v, k)
            assert np.sign(m_new[k]) == np.sign(v)
    chk_ref.report()
    chk_orc.report()


def test_column_noalloc_takes_no_device_memory():
    """After a first call, further calls leave the device's free memory unchanged."""
    require_gpu()
    import torch
    from paper_2605_04483_gb300 import api, inputs
    w = inputs.ab_initio(16, 5, 4, seed=21)
    dets = inputs.random_determinants(16, 5, 4, 6, seed=22)
    h = torch.tensor(w.h, device="cuda")
    g = torch.tensor(w.g, device="cuda")
    cap = 8192
    keys = torch.zeros((cap, 2), dtype=torch.int64, device="cuda")
    vals = torch.zeros(cap, dtype=torch.float64, device="cuda")
    key = np.ascontiguousarray(dets[0], dtype=np.uint64)
    api.cdfci_column_noalloc(h, g, w.N, w.n_alpha, w.n_beta, key, keys, vals, cap)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for d in dets[1:]:
        api.cdfci_column_noalloc(h, g, w.N, w.n_alpha, w.n_beta, np.ascontiguousarray(d, dtype=np.uint64),
                                 keys, vals, cap)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_column_noalloc_refuses_a_capturing_stream():
    """The call waits on its stream, so on a stream under capture it returns CDFCI_ERR_ARG without
    queuing anything; the capture then ends normally."""
    require_gpu()
    import torch
    from paper_2605_04483_gb300 import api, inputs
    w = inputs.ab_initio(8, 3, 2, seed=5)
    det = np.ascontiguousarray(inputs.random_determinants(8, 3, 2, 1, seed=12)[0], dtype=np.uint64)
    h = torch.tensor(w.h, device="cuda")
    g = torch.tensor(w.g, device="cuda")
    keys = torch.zeros((512, 2), dtype=torch.int64, device="cuda")
    vals = torch.zeros(512, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(st):
        graph.capture_begin()
        try:
            api.cdfci_column_noalloc(h, g, w.N, w.n_alpha, w.n_beta, det, keys, vals, 512, stream=st.cuda_stream)
        except api.CdfciError as e:
            err = e
        finally:
            graph.capture_end()
    assert err is not None and err.code == -1 and "captured" in str(err)
    # the stream is usable afterwards and the next call works
    n = api.cdfci_column_noalloc(h, g, w.N, w.n_alpha, w.n_beta, det, keys, vals, 512, stream=st.cuda_stream)
    assert n > 0


def test_column_noalloc_rejects_sizes_beyond_the_scratch_limit():
    require_gpu()
    import torch
    from paper_2605_04483_gb300 import api
    h = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(api.CdfciError) as e:
        api.cdfci_column_noalloc(h, h, 64, 1, 1, np.array([1, 1], dtype=np.uint64), out, out, 2)
    assert e.value.code == -1 and "scratch limit" in str(e.value)
