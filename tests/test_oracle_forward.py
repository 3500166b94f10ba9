"""Pins of the oracle's forward model and lifting against definitions that do not share its code.

- F2 against the O(N^2) DFT sum written out (unitary, sign e^{-2 pi i}).
- A / A^H adjoint identity and Parseval (Sec. II-A).
- The hybrid lifting against the convolution it stands for, computed another way (FFT circular
  convolution in space + direct linear sum over frames; Sec. III-A hybrid convolution).
- Exact rows of the linear lifting are rows of the hybrid one (Sec. II-B valid shifts).
- Annihilation (Eq. annihilation-1D / annihilation-3D) and the null-space / rank bounds
  (Eq. dim-ker / rank-bound of Sec. II-C) on signals where they hold exactly.
"""

import numpy as np
import pytest

from oracle import slr


def _dft_direct(x):
    P, Q = x.shape
    out = np.zeros((P, Q), dtype=np.complex128)
    for k1 in range(P):
        for k2 in range(Q):
            acc = 0j
            for r1 in range(P):
                for r2 in range(Q):
                    acc += x[r1, r2] * np.exp(-2j * np.pi * (k1 * r1 / P + k2 * r2 / Q))
            out[k1, k2] = acc
    return out / np.sqrt(P * Q)


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_f2_matches_direct_dft(rng):
    x = _crandn(rng, 6, 5)
    assert np.allclose(slr.F2(x), _dft_direct(x), rtol=0, atol=1e-12)
    assert np.allclose(slr.F2H(slr.F2(x)), x, atol=1e-13)


def test_adjoint_identity_and_parseval(rng):
    T, P, Q = 3, 8, 6
    x = _crandn(rng, T, P, Q)
    y = _crandn(rng, T, P, Q)
    m = (rng.random((T, P, Q)) < 0.4).astype(np.uint8)
    lhs = np.vdot(slr.A(x, m), y)
    rhs = np.vdot(x, slr.AH(y, m))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.isclose(np.linalg.norm(slr.F2(x)), np.linalg.norm(x), rtol=1e-13)


@pytest.mark.parametrize("dims", [(4, 6, 5, 3, 2, 2), (5, 8, 8, 2, 3, 3), (3, 4, 4, 4, 4, 1)])
def test_lift_is_hybrid_convolution(rng, dims):
    T, P, Q, N1, N2, M = dims
    xh = _crandn(rng, T, P, Q)
    d = _crandn(rng, M, N1, N2)
    Tm = slr.lift(xh, N1, N2, M)
    dvec = np.zeros(N1 * N2 * M, dtype=np.complex128)
    for m in range(M):
        for l1 in range(N1):
            for l2 in range(N2):
                dvec[slr.col_index(l1, l2, m, N1, N2)] = d[m, l1, l2]
    got = (Tm @ dvec).reshape(T - M + 1, P, Q)
    # circular 2-D convolution in space by FFT, linear (valid) convolution over frames
    dpad = np.zeros((M, P, Q), dtype=np.complex128)
    dpad[:, :N1, :N2] = d
    Dk = np.fft.fft2(dpad)
    want = np.zeros((T - M + 1, P, Q), dtype=np.complex128)
    for n_out in range(M - 1, T):
        for m in range(M):
            want[n_out - (M - 1)] += np.fft.ifft2(np.fft.fft2(xh[n_out - m]) * Dk[m])
    assert np.allclose(got, want, atol=1e-11)


def test_linear_lifting_rows_are_hybrid_rows(rng):
    T, P, Q, N1, N2, M = 4, 7, 6, 3, 2, 2
    xh = _crandn(rng, T, P, Q)
    Tc = slr.lift(xh, N1, N2, M)
    Tl = slr.lift_linear(xh, N1, N2, M)
    k = T - M + 1
    nr1, nr2 = P - N1 + 1, Q - N2 + 1
    for j in range(k):
        for i1 in range(nr1):
            for i2 in range(nr2):
                c1, c2 = i1 + N1 - 1, i2 + N2 - 1
                assert np.array_equal(Tl[(j * nr1 + i1) * nr2 + i2], Tc[(j * P + c1) * Q + c2])


def test_annihilation_constant_decay(rng):
    """rho[r, n] = alpha(r) beta^n with beta constant: the 1x1x2 filter (1, -beta) nulls the
    lifted matrix (Eq. annihilation-1D with a spatially constant filter)."""
    T, P, Q, N1, N2, M = 6, 8, 8, 3, 3, 2
    beta = 0.83 * np.exp(0.2j)
    alpha = _crandn(rng, P, Q)
    x = np.stack([alpha * beta ** n for n in range(T)])
    Tm = slr.lift(slr.F2(x), N1, N2, M)
    d = np.zeros(N1 * N2 * M, dtype=np.complex128)
    d[slr.col_index(0, 0, 0, N1, N2)] = 1.0
    d[slr.col_index(0, 0, 1, N1, N2)] = -beta
    assert np.linalg.norm(Tm @ d) <= 1e-12 * np.linalg.norm(Tm)


@pytest.mark.parametrize("L", [1, 2])
def test_rank_constant_decays(rng, L):
    """L exponentials with spatially constant decays and generic amplitudes: every spatial tap
    position spans exactly L directions, so rank = N1*N2*L (M >= L)."""
    T, P, Q, N1, N2, M = 7, 8, 8, 2, 3, 3
    betas = [0.9, 0.6 * np.exp(0.4j)][:L]
    x = sum(np.stack([a * b ** n for n in range(T)]) for a, b in
            zip([_crandn(rng, P, Q) for _ in range(L)], betas))
    Tm = slr.lift(slr.F2(x), N1, N2, M)
    sv = np.linalg.svd(Tm, compute_uv=False)
    rank = int(np.sum(sv > 1e-10 * sv[0]))
    assert rank == N1 * N2 * L


def test_nullspace_bound_smooth_decay(rng):
    """One exponential whose decay is a trigonometric polynomial in space,
    beta(r) = b0 + b1 cos(2 pi r1 / P): its k-space support is 3 x 1, so the minimal filter
    Theta is 3 x 1 x 2 and on the circular grid the annihilation is exact. Eq. dim-ker then gives
    dim ker >= |Lambda:Theta| = (N1-2) * N2 * (M-1)."""
    T, P, Q, N1, N2, M = 6, 10, 8, 4, 3, 3
    r1 = np.arange(P)[:, None] * np.ones((1, Q))
    beta = 0.7 + 0.2 * np.cos(2 * np.pi * r1 / P)
    alpha = _crandn(rng, P, Q)
    x = np.stack([alpha * beta ** n for n in range(T)])
    Tm = slr.lift(slr.F2(x), N1, N2, M)
    sv = np.linalg.svd(Tm, compute_uv=False)
    nullity = int(np.sum(sv <= 1e-10 * sv[0])) + (Tm.shape[1] - len(sv))
    assert nullity >= (N1 - 3 + 1) * (N2 - 1 + 1) * (M - 2 + 1)
    # and a generic signal of the same shape has no null space at all
    sv_rand = np.linalg.svd(slr.lift(_crandn(rng, T, P, Q), N1, N2, M), compute_uv=False)
    assert sv_rand[-1] > 1e-6 * sv_rand[0]
