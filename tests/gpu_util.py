"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

EPS = np.finfo(np.float64).eps


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def colmap(keys, vals):
    return {(int(k[0]), int(k[1])): float(v) for k, v in zip(keys, vals)}


_scale_cache = {}


def element_tol(w, v):
    """|gpu - oracle| bound for one column element.  A single is a sum of
    1 + 2n terms (n electrons) each bounded by S = max|h| + max|g|; two
    summation orders differ by at most 2 (2n+1) eps sum|terms| (recursive
    summation bound).  Doubles are one subtraction of the same two doubles on
    both sides.  Plus 1e-12 relative."""
    n = w.n_alpha + w.n_beta
    key = id(w)
    if key not in _scale_cache or _scale_cache[key][0] is not w:
        _scale_cache[key] = (w, np.abs(w.h).max() + (2 * n + 1) * np.abs(w.g).max())
    S = _scale_cache[key][1]
    return 1e-12 * abs(v) + 2 * (2 * n + 1) * EPS * S


def vec_by_key(keys, vals):
    return {(int(k[0]), int(k[1])): float(v) for k, v in zip(keys, vals)}
