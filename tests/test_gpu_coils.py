"""Multi-coil path (Eq. measurement-ij with coil sensitivities) through the C ABI against the
FP64 oracle's A_coils / AH_coils / normal_op(..., coils) / irls(..., coils).

Tolerances as for the single-coil parity tests: adjoint 2e-6, normal operator 1e-5 (FP32
transforms, one per coil, summed over coils), full IRLS 1e-4 on the final image.
"""

import numpy as np
import pytest

import synth
from oracle import slr

from gpu_util import assert_close, c64, crandn, pairs_from_full, rel, to_dev

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04511_gb300 import recon
    ctx = recon.Context(0)
    yield recon, ctx
    ctx.close()


def _small(**kw):
    base = dict(P=32, Q=64, T=6, n_coils=4, times_ms=tuple(10.0 * (n + 1) for n in range(6)),
                N1=5, N2=3, M=2, n_irls=6, n_cg=8)
    base.update(kw)
    w = synth.workload("coils_128x128x12", **base)
    return w, synth.make_problem(w)


CASES = [("32x64x6-4coils", {}),
         ("256x64x4-3coils", dict(P=256, Q=64, T=4, n_coils=3,
                                  times_ms=(10.0, 20.0, 30.0, 40.0))),
         ("128x128x12-12coils", None)]


def _case(kw):
    if kw is None:
        w = synth.workload("coils_128x128x12")
        return w, synth.make_problem(w)
    return _small(**kw)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_coil_adjoint_parity(R, case):
    recon, ctx = R
    w, prob = _case(case[1])
    C, masks = prob["coils"], prob["masks"]
    b = c64(prob["kspace"])
    x = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    recon.recon_adjoint_coils(ctx.h, to_dev(b), to_dev(masks), to_dev(c64(C)), x)
    ref = slr.AH_coils(b.astype(np.complex128), masks, c64(C).astype(np.complex128))
    err, peak = assert_close(x.cpu().numpy(), ref, 2e-6, "coil adjoint")
    print(f"\n[coil adjoint {case[0]}] rel. error {err:.2e} (peak-relative element {peak:.2e})")


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_coil_normal_operator_parity(R, case):
    recon, ctx = R
    w, prob = _case(case[1])
    C = c64(prob["coils"]).astype(np.complex128)
    masks = prob["masks"]
    rng = np.random.default_rng(11)
    x0 = slr.AH_coils(prob["kspace"], masks, C)
    S = slr.weight_from_x(x0, w.N1, w.N2, w.M, 0.01 * np.linalg.eigvalsh(
        slr.gram_fft(x0, w.N1, w.N2, w.M))[-1], 0.0)
    S = S.astype(np.complex64).astype(np.complex128)
    v = c64(crandn(rng, *masks.shape))
    y = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    lam = w.lam
    recon.recon_apply_normal_coils(ctx.h, to_dev(masks), to_dev(c64(C)), (w.N1, w.N2, w.M),
                                   to_dev(c64(pairs_from_full(S))), lam, to_dev(v), y)
    ref = slr.normal_op(v.astype(np.complex128), masks, S, lam, C)
    err, peak = assert_close(y.cpu().numpy(), ref, 1e-5, "coil normal operator")
    print(f"\n[coil normal operator {case[0]}] rel. error {err:.2e} (peak-relative element {peak:.2e})")


def _check_solve(recon, ctx, w, prob, tag):
    C = c64(prob["coils"])
    masks = prob["masks"]
    out = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    recon.recon_solve_coils(ctx.h, to_dev(c64(prob["kspace"])), to_dev(masks), to_dev(C),
                            (w.N1, w.N2, w.M), w.lam, w.p, w.n_irls, w.n_cg, out)
    x_gpu = out.cpu().numpy()
    x_ref = slr.irls(c64(prob["kspace"]).astype(np.complex128), masks, w.N1, w.N2, w.M, w.lam,
                     w.p, w.n_irls, w.n_cg, coils=C.astype(np.complex128))
    xt = prob["x_true"]
    err, peak = assert_close(x_gpu, x_ref, 1e-4, f"coil solve {tag}")
    x0 = slr.AH_coils(prob["kspace"], masks, C.astype(np.complex128))
    print(f"\n[coil solve {tag}] |x_gpu - x_oracle| / |x_oracle| = {err:.2e} (peak-relative "
          f"element {peak:.2e}); NRMSE gpu {rel(x_gpu, xt):.5f} oracle {rel(x_ref, xt):.5f} adjoint "
          f"{rel(x0, xt):.5f}")
    assert rel(x_gpu, xt) < rel(x0, xt)


def test_coil_solve_parity_small(R):
    recon, ctx = R
    w, prob = _small()
    _check_solve(recon, ctx, w, prob, "32x64x6 4 coils 6 x 8")


@pytest.mark.slow
def test_coil_solve_parity_128x128x12(R):
    recon, ctx = R
    w = synth.workload("coils_128x128x12")
    _check_solve(recon, ctx, w, synth.make_problem(w), "128x128x12 12 coils 20 x 10")


def test_unit_single_coil_matches_single_coil_solve(R):
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=4)
    prob = synth.make_problem(w)
    masks = to_dev(prob["masks"])
    b = to_dev(c64(prob["kspace"]))
    out1 = torch.empty(prob["masks"].shape, dtype=torch.complex64, device="cuda")
    out2 = torch.empty_like(out1)
    recon.recon_solve(ctx.h, b, masks, (w.N1, w.N2, w.M), w.lam, w.p, w.n_irls, w.n_cg, out1)
    ones = torch.ones((1, w.P, w.Q), dtype=torch.complex64, device="cuda")
    recon.recon_solve_coils(ctx.h, b.unsqueeze(0).contiguous(), masks, ones, (w.N1, w.N2, w.M),
                            w.lam, w.p, w.n_irls, w.n_cg, out2)
    assert rel(out2.cpu().numpy(), out1.cpu().numpy()) < 1e-5


def test_coil_errors(R):
    recon, ctx = R
    w, prob = _small()
    masks = to_dev(prob["masks"])
    b = to_dev(c64(prob["kspace"]))
    out = torch.empty(prob["masks"].shape, dtype=torch.complex64, device="cuda")
    no_coils = torch.empty((0, w.P, w.Q), dtype=torch.complex64, device="cuda")
    with pytest.raises(recon.ReconError) as e:
        recon.recon_solve_coils(ctx.h, b, masks, no_coils, (w.N1, w.N2, w.M), w.lam, w.p, 2, 2,
                                out)
    assert e.value.code == recon.RECON_EINVAL
