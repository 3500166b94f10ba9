"""The oracle's pins catch plausible mistakes: each case plants one in a copy of an oracle
function (conjugate on the wrong side, a transposed block, a reversed frame index, a wrong sign
or exponent) and checks that the pin it targets fails. Planted on the CPU, never in the CUDA path.
"""

import numpy as np
import pytest

from oracle import slr


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _pair_products_wrong_conj(x, M):
    T = x.shape[0]
    k = T - M + 1
    q = np.zeros((M, M) + x.shape[1:], dtype=np.complex128)
    for m in range(M):
        for mp in range(M):
            for j in range(k):
                q[m, mp] += x[j + M - 1 - m] * np.conj(x[j + M - 1 - mp])
    return q


def _diag_sums_transposed(H, N1, N2, M):
    L1, L2 = 2 * N1 - 1, 2 * N2 - 1
    d = np.zeros((M, M, L1, L2), dtype=np.complex128)
    for a in range(M):
        for b in range(M):
            for l1 in range(N1):
                for l2 in range(N2):
                    for lp1 in range(N1):
                        for lp2 in range(N2):
                            d[a, b, l1 - lp1 + N1 - 1, l2 - lp2 + N2 - 1] += \
                                H[slr.col_index(lp1, lp2, a, N1, N2), slr.col_index(l1, l2, b, N1, N2)]
    return d


def _apply_W_reversed_frames(x, S):
    M = S.shape[0]
    k = x.shape[0] - M + 1
    out = np.zeros_like(x)
    for j in range(k):
        v = np.stack([x[j + m] for m in range(M)])
        w = np.einsum("abpq,bpq->apq", S, v)
        for a in range(M):
            out[j + a] += w[a]
    return out


_weight_S_orig = slr.weight_S


def _weight_S_wrong_sign(d, P, Q):
    return np.conj(_weight_S_orig(np.conj(d), P, Q))   # e^{+2 pi i d.r} instead of e^{-2 pi i d.r}


def _sos_residual(rng):
    T, P, Q, N1, N2, M = 5, 6, 8, 3, 2, 3
    xw = _crandn(rng, T, P, Q)
    x = _crandn(rng, T, P, Q)
    G = slr.gram_fft(xw, N1, N2, M)
    eps = 0.01 * np.linalg.eigvalsh(G)[-1]
    H, _ = slr.weight_H(G, eps, 0.0)
    S = slr.weight_S(slr.diag_sums(H, N1, N2, M), P, Q)
    direct = slr.penalty_filters(x, slr.filters_from_H(G, eps, 0.0), N1, N2, M)
    return abs(np.vdot(x, slr.apply_W(x, S)) - direct) / direct


def _gram_residual(rng):
    T, P, Q, N1, N2, M = 4, 8, 6, 3, 2, 2
    x = _crandn(rng, T, P, Q)
    Gb = slr.gram_brute(x, N1, N2, M)
    return np.linalg.norm(slr.gram_fft(x, N1, N2, M) - Gb) / np.linalg.norm(Gb)


@pytest.mark.parametrize("target,replacement,check", [
    ("pair_products", _pair_products_wrong_conj, _gram_residual),
    ("diag_sums", _diag_sums_transposed, _sos_residual),
    ("apply_W", _apply_W_reversed_frames, _sos_residual),
    ("weight_S", _weight_S_wrong_sign, _sos_residual),
])
def test_planted_mistake_is_caught(rng, monkeypatch, target, replacement, check):
    assert check(np.random.default_rng(5)) < 1e-10          # unmodified oracle passes
    monkeypatch.setattr(slr, target, replacement)
    assert check(np.random.default_rng(5)) > 1e-3           # the planted mistake is visible
