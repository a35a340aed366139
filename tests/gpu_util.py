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


def order_tol(w, v):
    """|gpu - literal| bound against the oracle's literal operator application, which sums a single
    excitation's 1 + 2n terms (n electrons, each bounded by S = max|h| + max|g|) in another order than
    Eq. (entry): recursive summation bound 2 (2n+1) eps S, plus 1e-12 relative.  The 1e-12 relative
    parity itself is against the oracle's Slater-Condon columns (ElementCheck)."""
    n = w.n_alpha + w.n_beta
    S = np.abs(w.h).max() + (2 * n + 1) * np.abs(w.g).max()
    return 1e-12 * abs(v) + 2 * (2 * n + 1) * EPS * S


REL_TOL = 1e-12          # matrix elements: relative bound of the contract, no absolute floor

_scale_cache = {}


def zero_bound(w):
    """Bound for an entry whose oracle value is exactly 0.0 (only a diagonal can be one: off-diagonal
    zeros are not in a column).  The diagonal is a sum of 1 + n + n^2 terms, each bounded by
    S = max|h| + (2n+1) max|g|, summed in another order on the device: recursive summation bound
    2 (n^2 + n + 1) eps S."""
    n = w.n_alpha + w.n_beta
    key = id(w)
    if key not in _scale_cache or _scale_cache[key][0] is not w:
        _scale_cache[key] = (w, np.abs(w.h).max() + (2 * n + 1) * np.abs(w.g).max())
    return 2 * (n * n + n + 1) * EPS * _scale_cache[key][1]


class ElementCheck:
    """|gpu - oracle| <= 1e-12 |oracle| for every element with a nonzero oracle value (the zero_bound
    for an exactly-zero one); keeps the largest relative error seen, which the tests print."""

    def __init__(self, name):
        self.name, self.max_rel, self.n = name, 0.0, 0

    def __call__(self, w, gpu, ref, what=""):
        self.n += 1
        if ref == 0.0:
            assert abs(gpu) <= zero_bound(w), (what, gpu, ref)
            return
        rel = abs(gpu - ref) / abs(ref)
        self.max_rel = max(self.max_rel, rel)
        assert rel <= REL_TOL, (what, gpu, ref, rel)

    def report(self):
        print(f"[{self.name}] {self.n} elements, max |gpu - oracle| / |oracle| = {self.max_rel:.3e} "
              f"(bound {REL_TOL:g})")


def vec_by_key(keys, vals):
    return {(int(k[0]), int(k[1])): float(v) for k, v in zip(keys, vals)}
