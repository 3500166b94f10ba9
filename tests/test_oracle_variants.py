"""Pins of the comparison-method oracle (oracle/variants.py): GIRAF fully circulant, HLR-Voxel and
IRLS-direct.

Each variant is tied to something other than itself: the explicit lifted matrices (brute-force
Gram, sum-of-squares identities that tie the weight operator to the explicit filters), adjoint
identities, special cases in which two methods coincide by construction (M = 1 for GIRAF, a 1 x 1
image for HLR-Voxel, a 1 x 1 spatial filter for IRLS-direct), invariants that only the fully
circulant lifting has, dense solves, and planted mistakes. The last tests check the paper's
qualitative claims on synthetic exponential data (Sec. IV-A): IRLS-direct and the proposed
method reach about the same error, GIRAF a clearly larger one.
"""

import numpy as np
import pytest

import synth
from oracle import slr, variants as V


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _hermitian_pd(rng, s, shift=1.0):
    B = _crandn(rng, s, s)
    return B @ B.conj().T / s + shift * np.eye(s)


# ---- GIRAF (fully circulant) -----------------------------------------------------------------

@pytest.mark.parametrize("dims", [(5, 6, 4, 2, 2, 2), (4, 5, 5, 3, 1, 3), (6, 4, 4, 1, 2, 4)])
def test_giraf_gram_equals_brute_force(dims):
    T, P, Q, N1, N2, M = dims
    x = _crandn(np.random.default_rng(0), T, P, Q)
    Tm = V.lift_circ(slr.F2(x), N1, N2, M)
    Gb = Tm.conj().T @ Tm
    assert np.linalg.norm(V.gram_circ(x, N1, N2, M) - Gb) <= 1e-12 * np.linalg.norm(Gb)


def test_giraf_sum_of_squares_identity_and_planted_window():
    rng = np.random.default_rng(1)
    T, P, Q, N1, N2, M = 5, 6, 5, 2, 3, 3
    xw, x = _crandn(rng, T, P, Q), _crandn(rng, T, P, Q)
    G = V.gram_circ(xw, N1, N2, M)
    eps = 0.05 * np.linalg.eigvalsh(G)[-1]
    H, _ = slr.weight_H(G, eps, 0.0)
    S = slr.weight_S(slr.diag_sums(H, N1, N2, M), P, Q)
    Tm = V.lift_circ(slr.F2(x), N1, N2, M)
    direct = sum(float(np.sum(np.abs(Tm @ h.conj()) ** 2))
                 for h in slr.filters_from_H(G, eps, 0.0))
    quad = np.vdot(x, V.apply_W_circ(x, S))
    assert abs(quad.real - direct) <= 1e-10 * direct and abs(quad.imag) <= 1e-10 * direct
    # the valid-window W of the proposed method does not give the circulant penalty
    assert abs(np.vdot(x, slr.apply_W(x, S)).real - direct) > 1e-3 * direct


def test_giraf_pair_products_are_shift_invariant_in_time():
    """Full circulance: q[a, b] depends on a - b only; the hybrid (valid) products do not."""
    x = _crandn(np.random.default_rng(2), 7, 4, 4)
    M = 3
    qc, qh = V.pair_products_circ(x, M), slr.pair_products(x, M)
    assert np.allclose(qc[1, 2], qc[0, 1], atol=1e-12) and np.allclose(qc[2, 2], qc[0, 0], atol=1e-12)
    assert not np.allclose(qh[1, 2], qh[0, 1], atol=1e-3)


def test_giraf_equals_proposed_for_one_frame_tap():
    rng = np.random.default_rng(3)
    x = _crandn(rng, 4, 6, 6)
    assert np.allclose(V.gram_circ(x, 3, 2, 1), slr.gram_fft(x, 3, 2, 1), atol=1e-10)
    S = _crandn(rng, 1, 1, 6, 6)
    assert np.allclose(V.apply_W_circ(x, S), slr.apply_W(x, S), atol=1e-12)


# ---- HLR-Voxel -------------------------------------------------------------------------------

def test_voxel_grams_are_the_explicit_toeplitz_grams():
    x = _crandn(np.random.default_rng(4), 7, 3, 4)
    M = 3
    Gv = V.voxel_grams(x, M)
    for r in [(0, 0), (1, 3), (2, 1)]:
        Tr = V.voxel_toeplitz(x, M, r)
        assert Tr.shape == (5, 3)
        assert np.allclose(Gv[r], Tr.conj().T @ Tr, atol=1e-12)


@pytest.mark.parametrize("p", [0.0, 0.5])
def test_voxel_sum_of_squares_identity_and_planted_transpose(p):
    rng = np.random.default_rng(5)
    T, P, Q, M = 6, 3, 4, 3
    xw, x = _crandn(rng, T, P, Q), _crandn(rng, T, P, Q)
    Gv = V.voxel_grams(xw, M)
    eps = V.voxel_initial_eps(xw, M, 0.05)
    Hv = V.voxel_weights(Gv, eps, p)
    pen = V.voxel_penalty(x, Hv, M)
    quad = np.vdot(x, slr.apply_W(x, V.voxel_S(Hv)))
    assert abs(quad.real - pen) <= 1e-10 * pen and abs(quad.imag) <= 1e-10 * pen
    S_bad = np.moveaxis(Hv, (2, 3), (0, 1))   # H_r instead of H_r^T
    assert abs(np.vdot(x, slr.apply_W(x, S_bad)).real - pen) > 1e-6 * pen


def test_voxel_initial_eps_is_one_value_from_the_largest_pixel_singular_value():
    """eps^(0) of HLR-Voxel is one number for the whole penalty: eps0_frac times the largest
    lambda_max(G_r) over the pixels, i.e. the square of the largest singular value of any
    pixel's explicit k x M Toeplitz matrix (Sec. III-C schedule)."""
    rng = np.random.default_rng(11)
    T, P, Q, M = 7, 3, 5, 3
    x = _crandn(rng, T, P, Q)
    x[:, 1, 2] *= 4.0                      # one bright pixel sets the value
    smax = max(np.linalg.svd(V.voxel_toeplitz(x, M, (r1, r2)), compute_uv=False)[0]
               for r1 in range(P) for r2 in range(Q))
    eps = V.voxel_initial_eps(x, M, 0.01)
    assert np.ndim(eps) == 0
    assert abs(eps - 0.01 * smax ** 2) <= 1e-12 * eps


def test_voxel_weight_closed_form_p0():
    rng = np.random.default_rng(6)
    Gv = np.stack([_hermitian_pd(rng, 3) for _ in range(6)]).reshape(2, 3, 3, 3)
    eps = rng.random((2, 3)) + 0.1
    Hv = V.voxel_weights(Gv, eps, 0.0)
    for i in range(2):
        for j in range(3):
            assert np.allclose(Hv[i, j], np.linalg.inv(Gv[i, j] + eps[i, j] * np.eye(3)), atol=1e-12)


def test_voxel_equals_proposed_on_a_single_pixel():
    """A 1 x 1 image: F is the identity and the proposed Gram with a 1 x 1 filter is the pixel's
    Toeplitz Gram, so both IRLS runs coincide."""
    rng = np.random.default_rng(7)
    T, M = 10, 3
    x_true = (np.exp(-np.arange(T) / 4.0) * (1 + 0.5j))[:, None, None]
    masks = (rng.random((T, 1, 1)) < 0.7).astype(np.uint8)
    masks[0] = 1
    b = slr.A(x_true + 0.01 * _crandn(rng, T, 1, 1), masks)
    a = slr.irls(b, masks, 1, 1, M, 0.1, 0.0, 4, 6)
    v = V.irls_hlr_voxel(b, masks, M, 0.1, 0.0, 4, 6)
    assert np.allclose(a, v, atol=1e-12 * np.abs(a).max())


# ---- IRLS-direct -----------------------------------------------------------------------------

def test_direct_unlift_is_the_adjoint_of_lift():
    rng = np.random.default_rng(8)
    T, P, Q, N1, N2, M = 5, 7, 6, 3, 2, 2
    xh = _crandn(rng, T, P, Q)
    Tm = V.lift_direct(xh, N1, N2, M)
    Y = _crandn(rng, *Tm.shape)
    lhs = np.vdot(Tm.ravel(), Y.ravel())
    rhs = np.vdot(xh.ravel(), V.unlift_direct(Y, T, P, Q, N1, N2, M).ravel())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert Tm.shape == (4 * 5 * 5, N1 * N2 * M)


@pytest.mark.parametrize("p", [0.0, 0.5])
def test_direct_sum_of_squares_identity_and_planted_transpose(p):
    rng = np.random.default_rng(9)
    T, P, Q, N1, N2, M = 5, 6, 6, 2, 3, 2
    xw, x = _crandn(rng, T, P, Q), _crandn(rng, T, P, Q)
    G = V.gram_direct(xw, N1, N2, M)
    eps = 0.05 * np.linalg.eigvalsh(G)[-1]
    H, _ = slr.weight_H(G, eps, p)
    Tm = V.lift_direct(V.centred_kspace(x), N1, N2, M)
    pen = sum(float(np.sum(np.abs(Tm @ h.conj()) ** 2)) for h in slr.filters_from_H(G, eps, p))
    quad = np.vdot(x, V.apply_W_direct(x, H, N1, N2, M))
    assert abs(quad.real - pen) <= 1e-10 * pen and abs(quad.imag) <= 1e-10 * pen
    assert abs(np.vdot(x, V.apply_W_direct(x, H.T, N1, N2, M)).real - pen) > 1e-6 * pen


def test_direct_equals_proposed_for_a_one_pixel_filter():
    """N1 = N2 = 1: every spatial position is a valid row, so the exact and the hybrid liftings
    are the same matrix."""
    rng = np.random.default_rng(10)
    T, P, Q, M = 6, 5, 4, 3
    x = _crandn(rng, T, P, Q)
    G = V.gram_direct(x, 1, 1, M)
    assert np.allclose(G, slr.gram_fft(x, 1, 1, M), atol=1e-10 * np.abs(G).max())
    H, _ = slr.weight_H(G, 0.1 * np.linalg.eigvalsh(G)[-1], 0.0)
    S = slr.weight_S(slr.diag_sums(H, 1, 1, M), P, Q)
    assert np.allclose(V.apply_W_direct(x, H, 1, 1, M), slr.apply_W(x, S), atol=1e-10)


def test_direct_lifting_is_taken_on_the_centred_kspace():
    """The exact Gram equals T^H T of the valid lifting of fftshift(F x), and differs from that
    of the natural-order k-space (the valid lifting is not shift invariant)."""
    x = _crandn(np.random.default_rng(12), 4, 8, 6)
    Tc = V.lift_direct(np.fft.fftshift(np.fft.fft2(x, norm="ortho"), axes=(1, 2)), 3, 2, 2)
    G = V.gram_direct(x, 3, 2, 2)
    assert np.allclose(G, Tc.conj().T @ Tc, atol=1e-12)
    Tn = V.lift_direct(slr.F2(x), 3, 2, 2)
    assert not np.allclose(G, Tn.conj().T @ Tn, atol=1e-3)


def test_direct_cg_reaches_the_dense_solution():
    rng = np.random.default_rng(11)
    T, P, Q, N1, N2, M = 3, 4, 4, 2, 2, 2
    masks = (rng.random((T, P, Q)) < 0.6).astype(np.uint8)
    H = _hermitian_pd(rng, N1 * N2 * M, 0.5)
    lam = 0.3
    op = lambda v: V.normal_op_direct(v, masks, H, lam, N1, N2, M)
    n = T * P * Q
    dense = np.stack([op(e.reshape(T, P, Q)).ravel() for e in np.eye(n, dtype=complex)], axis=1)
    assert np.allclose(dense, dense.conj().T, atol=1e-12)
    rhs = _crandn(rng, T, P, Q)
    x_dense = np.linalg.solve(dense, rhs.ravel()).reshape(T, P, Q)
    x_cg = slr.cg(op, rhs, np.zeros_like(rhs), 3 * n)
    assert np.linalg.norm(x_cg - x_dense) < 1e-8 * np.linalg.norm(x_dense)


# ---- the paper's qualitative claims (Sec. IV-A, Fig. 2 / Fig. 3) ------------------------------

@pytest.mark.slow
def test_direct_matches_proposed_and_giraf_breaks_down():
    w = synth.workload("tiny_32x32x8", n_irls=10, n_cg=8)
    prob = synth.make_problem(w)
    b, m, xt = prob["kspace"], prob["masks"], prob["x_true"]
    err = lambda x: np.linalg.norm(x - xt) / np.linalg.norm(xt)
    e_prop = err(slr.irls(b, m, w.N1, w.N2, w.M, w.lam, w.p, w.n_irls, w.n_cg))
    e_dir = err(V.irls_direct(b, m, w.N1, w.N2, w.M, w.lam, w.p, w.n_irls, w.n_cg))
    e_gir = err(V.irls_giraf(b, m, w.N1, w.N2, w.M, w.lam, w.p, w.n_irls, w.n_cg))
    e_adj = err(slr.AH(b, m))
    print(f"\nNRMSE proposed {e_prop:.4f} direct {e_dir:.4f} GIRAF {e_gir:.4f} adjoint {e_adj:.4f}")
    assert abs(e_dir - e_prop) < 0.15 * e_prop
    assert e_gir > 1.2 * e_prop


def test_uniform_mask_generator():
    """The comparison workload's sampling: exactly round(PQ/R) samples, DC included, seeded, no
    preference for low frequencies (compare the inner and outer halves of the k-space radius)."""
    m1 = synth.uniform_mask(128, 128, 1 / 0.3, np.random.default_rng(5))
    m2 = synth.uniform_mask(128, 128, 1 / 0.3, np.random.default_rng(5))
    assert np.array_equal(m1, m2)
    assert int(m1.sum()) == round(128 * 128 * 0.3) and m1[0, 0] == 1
    k = np.fft.fftfreq(128) * 128
    rad = np.hypot(*np.meshgrid(k, k, indexing="ij"))
    inner = rad < np.median(rad)
    assert abs(m1[inner].mean() - m1[~inner].mean()) < 0.03
