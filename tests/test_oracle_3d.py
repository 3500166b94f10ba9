"""Pins of the 3-D oracle (oracle/slr3.py): volumes (T, R, P, Q), taps N1 x N2 x N3 x M.

Against what the mathematics fixes: the explicit 3-D lifting (brute-force Gram T^H T and the
sum-of-squares identity sum_i ||T h_i||^2 = Re <x, W x>, which ties the summed diagonals, the
S(r) placement and the banded W to the lifting), the adjoint identity of the 3-D forward model,
the reduction to the 2-D oracle when R = N3 = 1, and planted mistakes in the depth axis.
"""

import numpy as np
import pytest

from oracle import slr, slr3


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_forward_model_adjoint_and_unitarity():
    rng = np.random.default_rng(0)
    x = _crandn(rng, 3, 4, 6, 5)
    y = _crandn(rng, 3, 4, 6, 5)
    masks = (rng.random((3, 4, 6, 5)) < 0.5).astype(np.uint8)
    lhs = np.vdot(slr3.A3(x, masks).ravel(), y.ravel())
    rhs = np.vdot(x.ravel(), slr3.AH3(y, masks).ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert np.isclose(np.linalg.norm(slr3.F3(x)), np.linalg.norm(x), rtol=1e-13)


@pytest.mark.parametrize("dims", [(4, 4, 6, 5, 2, 3, 2, 2), (5, 3, 4, 4, 3, 2, 3, 3),
                                  (3, 4, 4, 4, 4, 1, 2, 1)])
def test_gram3_equals_brute_force(dims):
    T, R, P, Q, N1, N2, N3, M = dims
    rng = np.random.default_rng(1)
    x = _crandn(rng, T, R, P, Q)
    G = slr3.gram_fft3(x, N1, N2, N3, M)
    Gb = slr3.gram_brute3(x, N1, N2, N3, M)
    assert np.linalg.norm(G - Gb) <= 1e-12 * np.linalg.norm(Gb)


def test_reduces_to_2d_when_depth_is_one():
    rng = np.random.default_rng(2)
    T, P, Q, N1, N2, M = 5, 8, 6, 3, 2, 2
    x2 = _crandn(rng, T, P, Q)
    x3 = x2[:, None]
    G2 = slr.gram_fft(x2, N1, N2, M)
    G3 = slr3.gram_fft3(x3, N1, N2, 1, M)
    assert np.allclose(G3, G2, atol=1e-10 * np.abs(G2).max())
    eps = 0.01 * np.linalg.eigvalsh(G2)[-1]
    S2 = slr.weight_from_x(x2, N1, N2, M, eps, 0.0)
    S3 = slr3.weight_from_x3(x3, N1, N2, 1, M, eps, 0.0)
    assert np.allclose(S3[:, :, 0], S2, atol=1e-10 * np.abs(S2).max())
    v = _crandn(rng, T, P, Q)
    assert np.allclose(slr3.apply_W3(v[:, None], S3)[:, 0], slr.apply_W(v, S2),
                       atol=1e-10 * np.abs(S2).max())


def _weight3(rng, x, N1, N2, N3, M, p):
    G = slr3.gram_fft3(x, N1, N2, N3, M)
    eps = 0.05 * np.linalg.eigvalsh(G)[-1]
    return G, eps


@pytest.mark.parametrize("p", [0.0, 0.5])
def test_sum_of_squares_identity_3d(p):
    rng = np.random.default_rng(3)
    T, R, P, Q, N1, N2, N3, M = 4, 4, 5, 4, 2, 2, 3, 2
    xw = _crandn(rng, T, R, P, Q)
    x = _crandn(rng, T, R, P, Q)
    G, eps = _weight3(rng, xw, N1, N2, N3, M, p)
    H, _ = slr.weight_H(G, eps, p)
    S = slr3.weight_S3(slr3.diag_sums3(H, N1, N2, N3, M), R, P, Q)
    direct = slr3.penalty_filters3(x, slr.filters_from_H(G, eps, p), N1, N2, N3, M)
    quad = np.vdot(x, slr3.apply_W3(x, S))
    assert abs(quad.imag) <= 1e-10 * abs(quad.real)
    assert abs(quad.real - direct) <= 1e-10 * direct


def test_planted_depth_mistakes_are_caught(monkeypatch):
    rng = np.random.default_rng(4)
    T, R, P, Q, N1, N2, N3, M = 4, 4, 4, 5, 2, 2, 2, 2
    xw = _crandn(rng, T, R, P, Q)
    x = _crandn(rng, T, R, P, Q)
    G, eps = _weight3(rng, xw, N1, N2, N3, M, 0.0)
    H, _ = slr.weight_H(G, eps, 0.0)
    direct = slr3.penalty_filters3(x, slr.filters_from_H(G, eps, 0.0), N1, N2, N3, M)
    d = slr3.diag_sums3(H, N1, N2, N3, M)
    # depth lags placed with the wrong sign
    S_bad = slr3.weight_S3(d[:, :, :, :, ::-1], R, P, Q)
    assert abs(np.vdot(x, slr3.apply_W3(x, S_bad)).real - direct) > 1e-6 * direct
    # Gram read out with the depth lag taken along the row axis
    lag = slr3.gram_lags3(xw, N1, N2, N3, M)
    orig = slr3.gram_lags3
    monkeypatch.setattr(slr3, "gram_lags3", lambda *a: np.swapaxes(orig(*a), 2, 4)
                        if N1 == N3 else orig(*a))
    Gb = slr3.gram_brute3(xw, N1, N2, N3, M)
    assert np.linalg.norm(slr3.gram_fft3(xw, N1, N2, N3, M) - Gb) > 1e-6 * np.linalg.norm(Gb)
    assert lag.shape == (M, M, 2 * N1 - 1, 2 * N2 - 1, 2 * N3 - 1)


def test_irls3_reduces_to_2d():
    rng = np.random.default_rng(5)
    T, P, Q, N1, N2, M = 6, 8, 8, 3, 3, 2
    x = np.exp(-np.arange(T)[:, None, None] / 3.0) * _crandn(rng, 1, P, Q)
    masks = (rng.random((T, P, Q)) < 0.5).astype(np.uint8)
    b = slr.A(x, masks)
    x2 = slr.irls(b, masks, N1, N2, M, 1e-3, 0.0, 3, 5)
    x3 = slr3.irls3(b[:, None], masks[:, None], N1, N2, 1, M, 1e-3, 0.0, 3, 5)
    assert np.allclose(x3[:, 0], x2, atol=1e-10 * np.abs(x2).max())


def test_volume_generator_properties():
    import synth
    w = synth.workload("vol_128x128x64x12", P=32, Q=32, depth=8, T=4,
                       times_ms=(10.0, 20.0, 30.0, 40.0))
    prob = synth.make_problem(w)
    m = prob["masks"]
    assert m.shape == (4, 8, 32, 32)
    assert all(int(m[n].sum()) == round(8 * 32 * 32 / w.R) for n in range(4))
    assert m[:, 0, 0, 0].all()                                   # DC sampled
    clean = m * slr3.F3(prob["x_true"])
    snr = 20 * np.log10(np.linalg.norm(clean) / np.linalg.norm(prob["kspace"] - clean))
    assert abs(snr - w.snr_db) < 1e-9


@pytest.mark.slow
def test_irls3_improves_on_the_adjoint():
    import synth
    w = synth.workload("vol_128x128x64x12", P=32, Q=32, depth=8, T=6,
                       times_ms=tuple(10.0 * (n + 1) for n in range(6)), N1=3, N2=3, N3=2, M=2,
                       n_irls=6, n_cg=10)
    prob = synth.make_problem(w)
    x0 = slr3.AH3(prob["kspace"], prob["masks"])
    x = slr3.irls3(prob["kspace"], prob["masks"], w.N1, w.N2, w.N3, w.M, w.lam, w.p, w.n_irls,
                   w.n_cg)
    xt = prob["x_true"]
    assert np.linalg.norm(x - xt) < 0.9 * np.linalg.norm(x0 - xt)
