"""The split length-128 column DFT of the volume CG operator (128 x 128 slices of depth 64), replayed
in numpy with the kernels' row layout, against the plain DFT (definition of the DFT, Cooley-Tukey
with 128 = 16 x 8).

The row pass stores, for column q, Y[k1][p2] = w128^(p2 k1) sum_p1 x[8 p1 + p2] w16^(p1 k1) at row
8 k1 + p2; the depth pass reads rows 8 k1 + p2 (one k1, all p2), forms X[k1 + 16 k2] by the 8-point
DFT over p2, and after the masked depth transforms stores Z[k1][p2] = w128^(-p2 k1) sum_k2
X[k1 + 16 k2] w8^(-p2 k2) at row 8 k1 + p2 again; the last pass runs the 16-point IDFT over k1 of
rows 8 k1 + p2 and stores x[p2 + 8 p1] at row 8 p1 + p2. A wrong twiddle sign, index or row
mapping in that chain shows here without a GPU.
"""
import numpy as np

N, N1, N2 = 128, 16, 8


def w(n, e):
    return np.exp(-2j * np.pi * e / n)


def row_pass_stage(x):
    """Rows p of x (N x C) -> the buffer after the row pass: row 8 k1 + p2 holds Y[k1][p2]."""
    out = np.empty_like(x)
    for p2 in range(N2):
        rows = x[p2::N2]  # x[8 p1 + p2], p1 = 0..15
        for k1 in range(N1):
            y = sum(rows[p1] * w(N1, p1 * k1) for p1 in range(N1))
            out[N2 * k1 + p2] = w(N, p2 * k1) * y
    return out


def depth_pass_forward(buf):
    """X[k1 + 16 k2] from rows 8 k1 + p2 (the 8-point DFT over p2)."""
    X = np.empty_like(buf)
    for k1 in range(N1):
        rows = buf[N2 * k1:N2 * k1 + N2]
        for k2 in range(N2):
            X[k1 + N1 * k2] = sum(rows[p2] * w(N2, p2 * k2) for p2 in range(N2))
    return X


def depth_pass_inverse(X):
    """Rows 8 k1 + p2 <- Z[k1][p2] (8-point IDFT over k2, twiddle w128^(-p2 k1))."""
    buf = np.empty_like(X)
    for k1 in range(N1):
        for p2 in range(N2):
            z = sum(X[k1 + N1 * k2] * w(N2, -p2 * k2) for k2 in range(N2))
            buf[N2 * k1 + p2] = w(N, -p2 * k1) * z
    return buf


def last_pass(buf):
    """Row 8 p1 + p2 <- x[p2 + 8 p1] = sum_k1 w16^(-p1 k1) Z[k1][p2] (in place by rows)."""
    out = np.empty_like(buf)
    for p2 in range(N2):
        Z = buf[p2::N2]  # Z[k1][p2] at rows 8 k1 + p2
        for p1 in range(N1):
            out[N2 * p1 + p2] = sum(Z[k1] * w(N1, -p1 * k1) for k1 in range(N1))
    return out


def test_split_forward_is_the_dft():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    X = depth_pass_forward(row_pass_stage(x))
    assert np.allclose(X, np.fft.fft(x, axis=0), rtol=0, atol=1e-10 * np.abs(X).max())


def test_split_inverse_is_the_unnormalised_idft():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    x = last_pass(depth_pass_inverse(X))
    assert np.allclose(x, N * np.fft.ifft(X, axis=0), rtol=0, atol=1e-10 * np.abs(x).max())


def test_split_round_trip_with_a_mask():
    """Forward, a mask in the DFT domain, inverse: the column part of A^H A (up to the scale)."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    mask = rng.random((N, 2)) < 0.3
    y = last_pass(depth_pass_inverse(mask * depth_pass_forward(row_pass_stage(x)))) / N
    ref = np.fft.ifft(mask * np.fft.fft(x, axis=0), axis=0)
    assert np.allclose(y, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_a_wrong_twiddle_sign_is_caught():
    """The pin fails for a plausible mistake: the inverse twiddle taken with the forward sign."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((N, 1)) + 1j * rng.standard_normal((N, 1))
    buf = np.empty_like(X)
    for k1 in range(N1):
        for p2 in range(N2):
            z = sum(X[k1 + N1 * k2] * w(N2, -p2 * k2) for k2 in range(N2))
            buf[N2 * k1 + p2] = w(N, p2 * k1) * z  # wrong sign
    assert not np.allclose(last_pass(buf), N * np.fft.ifft(X, axis=0), atol=1e-6)
