"""Helpers shared by the GPU parity tests (host-side marshalling only)."""

import numpy as np


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def c64(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def rel(a, b):
    """||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrel(a, b):
    """max |a - b| / max |b| (element-wise, complex magnitude)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# Per-element companion of the relative-Frobenius gates: max |a - b| <= PEAK_FACTOR * tol *
# max |b|. An error confined to a few elements (one tail column, one boundary frame, one ragged
# tile) is diluted in the norm of the whole array; relative to the array's peak it is not.
PEAK_FACTOR = 10.0


def assert_close(a, b, tol, what=""):
    """The relative-Frobenius gate ||a - b|| / ||b|| < tol and the per-element bound
    max |a - b| < PEAK_FACTOR * tol * max |b|."""
    e, m = rel(a, b), maxrel(a, b)
    assert e < tol, f"{what} relative error {e:.3e} >= {tol:.1e}"
    assert m < PEAK_FACTOR * tol, f"{what} peak-relative element error {m:.3e} >= {PEAK_FACTOR * tol:.1e}"
    return e, m


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def npair_index(a, b, M):
    return a * (2 * M - a + 1) // 2 + (b - a)


def pairs_from_full(S_full):
    """(M, M, P, Q) -> (npair, P, Q) upper triangle in the library's pair order."""
    M = S_full.shape[0]
    out = []
    for a in range(M):
        for b in range(a, M):
            out.append(S_full[a, b])
    return np.stack(out)


def lags_pairs(lag_full):
    """(M, M, L1, L2) -> (npair, L1, L2)."""
    return pairs_from_full(lag_full)
