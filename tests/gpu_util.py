"""Helpers for the GPU parity tests (test infrastructure)."""

from __future__ import annotations

import numpy as np

import oracle

U2 = 2.0**-106          # u^2, u = 2^-53
DD_BOUND = 4 * 2.0**-104   # times l |A||B|
QD_BOUND = 4 * 2.0**-208


def dev(x: np.ndarray):
    import torch
    if x.dtype == np.uint32:
        x = x.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t, mp=False) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a.view(np.uint32) if mp else a


def sample_indices(m, n, count, seed=0):
    """Row 0, column 0, the four corners and `count` random entries."""
    rng = np.random.default_rng(seed)
    ii = list(rng.integers(0, m, count)) + [0] * 8 + list(rng.integers(0, m, 8)) + [0, 0, m - 1, m - 1]
    jj = list(rng.integers(0, n, count)) + list(rng.integers(0, n, 8)) + [0] * 8 + [0, n - 1, 0, n - 1]
    return np.array(ii, dtype=np.int64), np.array(jj, dtype=np.int64)


def bound_ratio(A, B, C, ii, jj, rel):
    """max over samples of |c - c_exact| / (rel * l * sum|a||b|)."""
    l = A.shape[2]
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    return float(np.max(err / (rel * l * absab)))
