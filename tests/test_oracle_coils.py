"""Pins of the oracle's multi-coil forward model (Eq. measurement-ij with coil sensitivities).

b[c, n] = mask_n * F (C_c x_n); A^H b = sum_c conj(C_c) F^H (mask_n b[c, n]). Checked against
what the mathematics fixes: the adjoint identity, the single-coil special case C = 1, full
sampling with sum_c |C_c|^2 = 1 (A^H A = I), CG against a dense solve of the coil normal
equations, and a planted mistake (a missing conjugate) that the adjoint identity catches.
"""

import numpy as np
import pytest

import synth
from oracle import slr


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _coils(rng, nc, P, Q):
    return synth.coil_maps(nc, P, Q, rng)


def test_coil_maps_are_normalised_and_seeded():
    C1 = synth.coil_maps(6, 32, 24, np.random.default_rng(3))
    C2 = synth.coil_maps(6, 32, 24, np.random.default_rng(3))
    assert np.array_equal(C1, C2)
    assert np.allclose((np.abs(C1) ** 2).sum(0), 1.0, atol=1e-12)


def test_coil_adjoint_identity():
    rng = np.random.default_rng(0)
    T, P, Q, nc = 3, 16, 12, 4
    C = _coils(rng, nc, P, Q)
    masks = (rng.random((T, P, Q)) < 0.4).astype(np.uint8)
    x = _crandn(rng, T, P, Q)
    y = _crandn(rng, nc, T, P, Q)
    lhs = np.vdot(slr.A_coils(x, masks, C).ravel(), y.ravel())
    rhs = np.vdot(x.ravel(), slr.AH_coils(y, masks, C).ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_single_unit_coil_is_the_single_coil_model():
    rng = np.random.default_rng(1)
    T, P, Q = 2, 8, 8
    masks = (rng.random((T, P, Q)) < 0.5).astype(np.uint8)
    x = _crandn(rng, T, P, Q)
    C = np.ones((1, P, Q), dtype=complex)
    assert np.allclose(slr.A_coils(x, masks, C)[0], slr.A(x, masks), atol=1e-13)
    b = _crandn(rng, 1, T, P, Q)
    assert np.allclose(slr.AH_coils(b, masks, C), slr.AH(b[0], masks), atol=1e-13)


def test_full_sampling_with_normalised_coils_is_identity():
    rng = np.random.default_rng(2)
    T, P, Q, nc = 2, 16, 16, 5
    C = _coils(rng, nc, P, Q)
    masks = np.ones((T, P, Q), dtype=np.uint8)
    x = _crandn(rng, T, P, Q)
    assert np.allclose(slr.AH_coils(slr.A_coils(x, masks, C), masks, C), x, atol=1e-12)


def test_coil_cg_reaches_the_dense_solution():
    rng = np.random.default_rng(4)
    T, P, Q, nc, M = 3, 4, 4, 3, 2
    C = _coils(rng, nc, P, Q)
    masks = (rng.random((T, P, Q)) < 0.6).astype(np.uint8)
    S = _crandn(rng, M, M, P, Q) * 0.1
    S = 0.5 * (S + np.conj(np.transpose(S, (1, 0, 2, 3))))
    S = S + 2.0 * np.eye(M)[:, :, None, None]          # Hermitian positive definite per pixel
    lam = 0.3
    n = T * P * Q
    op = lambda v: slr.normal_op(v, masks, S, lam, C)
    dense = np.stack([op(e.reshape(T, P, Q)).ravel() for e in np.eye(n, dtype=complex)], axis=1)
    rhs = _crandn(rng, T, P, Q)
    x_dense = np.linalg.solve(dense, rhs.ravel()).reshape(T, P, Q)
    x_cg = slr.cg(op, rhs, np.zeros_like(rhs), 3 * n)
    assert np.linalg.norm(x_cg - x_dense) < 1e-8 * np.linalg.norm(x_dense)


def test_missing_conjugate_is_caught():
    rng = np.random.default_rng(5)
    T, P, Q, nc = 2, 8, 8, 3
    C = _coils(rng, nc, P, Q)
    masks = (rng.random((T, P, Q)) < 0.5).astype(np.uint8)
    x = _crandn(rng, T, P, Q)
    y = _crandn(rng, nc, T, P, Q)
    wrong_ah = sum(C[c][None] * slr.F2H(masks * y[c]) for c in range(nc))  # no conj
    lhs = np.vdot(slr.A_coils(x, masks, C).ravel(), y.ravel())
    rhs = np.vdot(x.ravel(), wrong_ah.ravel())
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)


@pytest.mark.slow
def test_coil_irls_improves_on_the_adjoint():
    w = synth.workload("coils_128x128x12", P=32, Q=32, T=8, n_coils=4,
                       times_ms=tuple(10.0 * (n + 1) for n in range(8)), N1=5, N2=5, M=2,
                       n_irls=8, n_cg=10, lam=0.1)
    prob = synth.make_problem(w)
    C, masks = prob["coils"], prob["masks"]
    x0 = slr.AH_coils(prob["kspace"], masks, C)
    x = slr.irls(prob["kspace"], masks, w.N1, w.N2, w.M, w.lam, w.p, w.n_irls, w.n_cg, coils=C)
    xt = prob["x_true"]
    assert np.linalg.norm(x - xt) < 0.8 * np.linalg.norm(x0 - xt)
