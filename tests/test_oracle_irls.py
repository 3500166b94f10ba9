"""Oracle checks at workload scale: the synthetic generator's stated properties, the T2 fitter on
exact data, and the IRLS sanity report (reconstruction beats zero filling; Algorithm 1 on the
32x32x8 workload). The complete IRLS trajectory has no printed values in the paper: its parity is
unpinned, only its steps are (see the other oracle tests)."""

import numpy as np
import pytest

import synth
from oracle import slr, t2fit


def test_generator_properties():
    w = synth.workload("tiny_32x32x8")
    prob = synth.make_problem(w)
    m, b, x = prob["masks"], prob["kspace"], prob["x_true"]
    assert m.shape == b.shape == x.shape == (8, 32, 32) and m.dtype == np.uint8
    assert all(int(m[n].sum()) == 256 for n in range(8))          # exactly N / R samples
    assert m[:, 0, 0].all() and m[:, -1, -1].all()                # DC block fully sampled
    assert not np.any(b[m == 0])                                  # unsampled entries are zero
    clean = m * slr.F2(x)
    snr = 20 * np.log10(np.linalg.norm(clean) / np.linalg.norm(b - clean))
    assert abs(snr - 30.0) < 1e-9
    again = synth.make_problem(w)
    assert np.array_equal(again["kspace"], b)                     # seeded


def test_t2_fit_exact_on_noise_free_monoexponential(rng):
    P, Q = 6, 7
    t2 = rng.uniform(20, 120, size=(P, Q))
    amp = rng.uniform(0.5, 1.0, size=(P, Q))
    times = 5.0 + 5.0 * np.arange(8)
    x = amp[None] * np.exp(-times[:, None, None] / t2[None])
    est = t2fit.fit_t2(x, times, fg=np.ones((P, Q), bool))
    assert np.allclose(est, t2, rtol=1e-9)


def test_irls_beats_zero_filling_tiny():
    w = synth.workload("tiny_32x32x8")
    prob = synth.make_problem(w)
    x_zf = slr.AH(prob["kspace"], prob["masks"])
    x = slr.irls(prob["kspace"], prob["masks"], w.N1, w.N2, w.M, w.lam, w.p, w.n_irls, w.n_cg)
    snr_zf = slr.snr_db(prob["x_true"], x_zf)
    snr_rec = slr.snr_db(prob["x_true"], x)
    assert snr_rec > snr_zf + 3.0, (snr_zf, snr_rec)


def _irls_carried_residual(kspace, masks, N1, N2, M, lam, p, n_irls, n_cg, gamma=1.4):
    """Algorithm 1 with the CG warm-start residual carried between IRLS iterations:
    r0^(1) = -lam W^(1) x0 (because A^H A A^H b = A^H b for 0/1 masks) and
    r0^(n+1) = r_end^(n) + lam (W^(n) - W^(n+1)) x^(n). This is the CUDA path's formulation:
    identical in exact arithmetic, but free of the cancellation in A^H b - (A^H A + lam W) x."""
    rhs = slr.AH(kspace, masks)
    x = rhs.copy()
    eps = slr.initial_eps(x, N1, N2, M)
    S_old, r = None, None
    for _ in range(n_irls):
        S = slr.weight_from_x(x, N1, N2, M, eps, p)
        if r is None:
            r = -lam * slr.apply_W(x, S)
        else:
            r = r + lam * (slr.apply_W(x, S_old) - slr.apply_W(x, S))
        pvec = r.copy()
        rr = slr.vdot(r, r).real
        for _ in range(n_cg):
            q = slr.normal_op(pvec, masks, S, lam)
            alpha = rr / slr.vdot(pvec, q).real
            x = x + alpha * pvec
            r = r - alpha * q
            rr_new = slr.vdot(r, r).real
            pvec = r + (rr_new / rr) * pvec
            rr = rr_new
        S_old = S
        eps /= gamma
    return x


def test_carried_residual_equals_recomputed():
    w = synth.workload("tiny_32x32x8", n_irls=8)
    prob = synth.make_problem(w)
    args = (prob["kspace"], prob["masks"], w.N1, w.N2, w.M, w.lam, w.p, w.n_irls, w.n_cg)
    ref = slr.irls(*args)
    got = _irls_carried_residual(*args)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
