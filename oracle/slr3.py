"""FP64 oracle of the method on 3-D image volumes (TEST INFRASTRUCTURE ONLY).

The same IRLS (Sec. III, Algorithm 1) with a third spatial axis: the unknown x has shape
(T, R, P, Q) (frames, depth, rows, columns), F is the unitary 3-D DFT of each volume, the filter
support is N1 x N2 x N3 spatial taps (rows, columns, depth) times M frame taps, s = N1 N2 N3 M,
and the lifting is circular in all three spatial axes and valid in time (the hybrid form of
Sec. III-A with one more circular axis). Every formula is the 2-D one of oracle/slr.py with the
extra axis carried along; with R = N3 = 1 the functions reduce to it (tests/test_oracle_3d.py).
A column of the lifted matrix is indexed ((m N3 + l3) N1 + l1) N2 + l2.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it.
"""

from __future__ import annotations

import numpy as np

from . import slr

AX = (-3, -2, -1)


def F3(x: np.ndarray) -> np.ndarray:
    """Unitary forward 3-D DFT over the last three axes (sign e^{-2 pi i k.r})."""
    return np.fft.fftn(x, axes=AX, norm="ortho")


def F3H(y: np.ndarray) -> np.ndarray:
    return np.fft.ifftn(y, axes=AX, norm="ortho")


def A3(x: np.ndarray, masks: np.ndarray) -> np.ndarray:
    """A x = mask * F x, volume by volume."""
    return masks * F3(x)


def AH3(b: np.ndarray, masks: np.ndarray) -> np.ndarray:
    return F3H(masks * b)


def col_index3(l1: int, l2: int, l3: int, m: int, N1: int, N2: int, N3: int) -> int:
    return ((m * N3 + l3) * N1 + l1) * N2 + l2


def _taps(N1, N2, N3):
    for l3 in range(N3):
        for l1 in range(N1):
            for l2 in range(N2):
                yield l1, l2, l3


def lift3(x_hat: np.ndarray, N1: int, N2: int, N3: int, M: int) -> np.ndarray:
    """Hybrid lifting: spatially circular in 3-D, temporally valid (k = T - M + 1 windows).
    Row (j, c), c over the R x P x Q grid; column (l, m): x_hat[j + M - 1 - m][c - l]."""
    T = x_hat.shape[0]
    vox = int(np.prod(x_hat.shape[1:]))
    k = T - M + 1
    Tm = np.zeros((k * vox, N1 * N2 * N3 * M), dtype=np.complex128)
    for j in range(k):
        rows = slice(j * vox, (j + 1) * vox)
        for m in range(M):
            vol = x_hat[j + M - 1 - m]
            for l1, l2, l3 in _taps(N1, N2, N3):
                Tm[rows, col_index3(l1, l2, l3, m, N1, N2, N3)] = \
                    np.roll(vol, (l3, l1, l2), axis=(0, 1, 2)).ravel()
    return Tm


def gram_brute3(x: np.ndarray, N1: int, N2: int, N3: int, M: int) -> np.ndarray:
    Tm = lift3(F3(x), N1, N2, N3, M)
    return Tm.conj().T @ Tm


def gram_lags3(x: np.ndarray, N1: int, N2: int, N3: int, M: int) -> np.ndarray:
    """lag[m, m', i1, i2, i3] = sum_r q[m, m'](r) e^{-2 pi i (d1 r1/P + d2 r2/Q + d3 r3/R)},
    d = i - (N - 1), read out of the unnormalised 3-D FFT of the pair products."""
    R, P, Q = x.shape[1:]
    g = np.fft.fftn(slr.pair_products(x, M), axes=AX)
    L1, L2, L3 = 2 * N1 - 1, 2 * N2 - 1, 2 * N3 - 1
    lag = np.zeros((M, M, L1, L2, L3), dtype=np.complex128)
    for i1 in range(L1):
        for i2 in range(L2):
            for i3 in range(L3):
                lag[:, :, i1, i2, i3] = g[:, :, (i3 - (N3 - 1)) % R, (i1 - (N1 - 1)) % P,
                                          (i2 - (N2 - 1)) % Q]
    return lag


def gram_fft3(x: np.ndarray, N1: int, N2: int, N3: int, M: int) -> np.ndarray:
    """G[(l, m), (l', m')] = lag[m, m'](l - l')."""
    lag = gram_lags3(x, N1, N2, N3, M)
    s = N1 * N2 * N3 * M
    G = np.zeros((s, s), dtype=np.complex128)
    taps = list(_taps(N1, N2, N3))
    for m in range(M):
        for mp in range(M):
            for l1, l2, l3 in taps:
                for p1, p2, p3 in taps:
                    G[col_index3(l1, l2, l3, m, N1, N2, N3), col_index3(p1, p2, p3, mp, N1, N2, N3)] = \
                        lag[m, mp, l1 - p1 + N1 - 1, l2 - p2 + N2 - 1, l3 - p3 + N3 - 1]
    return G


def diag_sums3(H: np.ndarray, N1: int, N2: int, N3: int, M: int) -> np.ndarray:
    """d[a, b, i1, i2, i3] = sum_{l - l' = d} H[(l', b), (l, a)]."""
    L1, L2, L3 = 2 * N1 - 1, 2 * N2 - 1, 2 * N3 - 1
    d = np.zeros((M, M, L1, L2, L3), dtype=np.complex128)
    taps = list(_taps(N1, N2, N3))
    for a in range(M):
        for b in range(M):
            for l1, l2, l3 in taps:
                for p1, p2, p3 in taps:
                    d[a, b, l1 - p1 + N1 - 1, l2 - p2 + N2 - 1, l3 - p3 + N3 - 1] += \
                        H[col_index3(p1, p2, p3, b, N1, N2, N3), col_index3(l1, l2, l3, a, N1, N2, N3)]
    return d


def weight_S3(d: np.ndarray, R: int, P: int, Q: int) -> np.ndarray:
    """S[a, b](r) = sum_d d[a, b, d] e^{-2 pi i (d1 r1/P + d2 r2/Q + d3 r3/R)}: the lags placed on
    the R x P x Q grid and transformed by an unnormalised 3-D FFT. Shape (M, M, R, P, Q)."""
    M, _, L1, L2, L3 = d.shape
    N1, N2, N3 = (L1 + 1) // 2, (L2 + 1) // 2, (L3 + 1) // 2
    pad = np.zeros((M, M, R, P, Q), dtype=np.complex128)
    for i1 in range(L1):
        for i2 in range(L2):
            for i3 in range(L3):
                pad[:, :, (i3 - (N3 - 1)) % R, (i1 - (N1 - 1)) % P, (i2 - (N2 - 1)) % Q] += \
                    d[:, :, i1, i2, i3]
    return np.fft.fftn(pad, axes=AX)


def apply_W3(x: np.ndarray, S: np.ndarray) -> np.ndarray:
    """(W x)(r) = sum_j E_j^T S(r) E_j x(r), per voxel (as slr.apply_W)."""
    M = S.shape[0]
    T = x.shape[0]
    k = T - M + 1
    out = np.zeros_like(x)
    for j in range(k):
        v = np.stack([x[j + M - 1 - m] for m in range(M)])
        w = np.einsum("ab...,b...->a...", S, v)
        for a in range(M):
            out[j + M - 1 - a] += w[a]
    return out


def penalty_filters3(x: np.ndarray, Hh: np.ndarray, N1: int, N2: int, N3: int, M: int) -> float:
    Tm = lift3(F3(x), N1, N2, N3, M)
    return float(sum(np.sum(np.abs(Tm @ h.conj()) ** 2) for h in Hh))


def normal_op3(x: np.ndarray, masks: np.ndarray, S: np.ndarray, lam: float) -> np.ndarray:
    return AH3(A3(x, masks), masks) + lam * apply_W3(x, S)


def weight_from_x3(x, N1, N2, N3, M, eps, p):
    G = gram_fft3(x, N1, N2, N3, M)
    H, _ = slr.weight_H(G, eps, p)
    return weight_S3(diag_sums3(H, N1, N2, N3, M), *x.shape[1:])


def initial_eps3(x0, N1, N2, N3, M, frac=0.01):
    return frac * float(np.linalg.eigvalsh(gram_fft3(x0, N1, N2, N3, M))[-1])


def irls3(kspace, masks, N1, N2, N3, M, lam, p, n_irls, n_cg, gamma=1.4, eps_frac=0.01):
    """Algorithm 1 on volumes: x0 = A^H b, eps0 = lambda_max / 100, eps <- eps / gamma."""
    rhs = AH3(kspace, masks)
    x = rhs.copy()
    eps = initial_eps3(x, N1, N2, N3, M, eps_frac)
    for _ in range(n_irls):
        S = weight_from_x3(x, N1, N2, N3, M, eps, p)
        x = slr.cg(lambda v: normal_op3(v, masks, S, lam), rhs, x, n_cg)
        eps = eps / gamma
    return x
