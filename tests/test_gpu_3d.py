"""Volumes (T, R, P, Q) through the C ABI against the FP64 3-D oracle (oracle/slr3.py).

Every stage the 3-D solve runs is compared with its oracle counterpart on the same seeded inputs:
the unitary 3-D DFT, the adjoint, the Gram matrix and its lags, the weight (summed diagonals and
S for p = 0 by the sweep inverse and p = 0.5 by the eigendecomposition), the normal operator and
the whole IRLS. Sizes: small cases the oracle finishes in seconds (several column tiles, more
rows than one wave of the row kernel), and the 128 x 128 x 64 x 12 volume series with its
7 x 7 x 3 x 2 filter in the launch shapes the benchmark times (operator, Gram, adjoint, and a
short solve). Tolerances follow the 2-D parity tests: transforms 2e-6, Gram 1e-5, S 1e-5,
normal operator 1e-5, solve 1e-4 (FP32 transforms and CG, FP64 weight).
"""

import numpy as np
import pytest

import synth
from oracle import slr, slr3

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
    base = dict(P=16, Q=32, depth=16, T=6, times_ms=tuple(10.0 * (n + 1) for n in range(6)),
                N1=3, N2=3, N3=2, M=2, n_irls=5, n_cg=8, lam=1e-2)
    base.update(kw)
    w = synth.workload("vol_128x128x64x12", **base)
    return w, synth.make_problem(w)


SMALL = [("16x16x32x6", {}),
         ("32x32x64x5-M3", dict(P=32, Q=64, depth=32, T=5, N1=5, N2=3, N3=3, M=3,
                                times_ms=(10.0, 20.0, 30.0, 40.0, 50.0)))]


def _case(kw):
    if kw is None:
        w = synth.workload("vol_128x128x64x12")
        return w, synth.make_problem(w)
    return _small(**kw)


CASES = SMALL + [("128x128x64x12", None)]
# 128 x 128 slices of depth 64: the shapes whose length-P DFT is split between the row pass and
# the depth pass of the CG operator (two column launches instead of three)
FOLD = ("128x128x64x4-M3", dict(P=128, Q=128, depth=64, T=4, N1=3, N2=3, N3=2, M=3,
                                times_ms=(10.0, 20.0, 30.0, 40.0)))


def _filt(w):
    return (w.N1, w.N2, w.N3, w.M)


def _lags_pairs3(lag):
    """oracle lag[m, m', i1, i2, i3] -> library layout (npair, L3, L1, L2)."""
    return np.transpose(pairs_from_full(lag), (0, 3, 1, 2))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fft3_parity(R, case):
    recon, ctx = R
    w, prob = _case(case[1])
    rng = np.random.default_rng(3)
    x = c64(crandn(rng, *prob["masks"].shape))
    xd = to_dev(x)
    y = torch.empty_like(xd)
    recon.recon_fft3(ctx.h, xd, y, inverse=False)
    ef = rel(y.cpu().numpy(), slr3.F3(x.astype(np.complex128)))
    recon.recon_fft3(ctx.h, xd, y, inverse=True)
    ei = rel(y.cpu().numpy(), slr3.F3H(x.astype(np.complex128)))
    print(f"\n[fft3 {case[0]}] forward {ef:.2e} inverse {ei:.2e}")
    assert ef < 2e-6 and ei < 2e-6


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_adjoint3_parity(R, case):
    recon, ctx = R
    w, prob = _case(case[1])
    masks = prob["masks"]
    b = c64(prob["kspace"])
    x = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    recon.recon_adjoint3(ctx.h, to_dev(b), to_dev(masks), x)
    err, peak = assert_close(x.cpu().numpy(), slr3.AH3(b.astype(np.complex128), masks), 2e-6,
                          "adjoint3")
    print(f"\n[adjoint3 {case[0]}] rel. error {err:.2e} (peak-relative element {peak:.2e})")


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gram3_parity(R, case):
    recon, ctx = R
    w, prob = _case(case[1])
    x0 = c64(slr3.AH3(prob["kspace"], prob["masks"]))
    s = w.N1 * w.N2 * w.N3 * w.M
    npair = w.M * (w.M + 1) // 2
    G = torch.empty((s, s), dtype=torch.complex128, device="cuda")
    lags = torch.empty((npair, 2 * w.N3 - 1, 2 * w.N1 - 1, 2 * w.N2 - 1), dtype=torch.complex128,
                       device="cuda")
    recon.recon_gram3(ctx.h, to_dev(x0), _filt(w), G, lags)
    xr = x0.astype(np.complex128)
    G_ref = slr3.gram_fft3(xr, w.N1, w.N2, w.N3, w.M)
    eg = rel(G.cpu().numpy().T, G_ref)
    el = rel(lags.cpu().numpy(), _lags_pairs3(slr3.gram_lags3(xr, w.N1, w.N2, w.N3, w.M)))
    print(f"\n[gram3 {case[0]}] G {eg:.2e} lags {el:.2e}")
    assert eg < 1e-5 and el < 1e-5


def test_gram3_brute_force_tiny(R):
    """Against the explicit lifted matrix T^H T (no FFT on the oracle side)."""
    recon, ctx = R
    rng = np.random.default_rng(8)
    T, D, P, Q, N1, N2, N3, M = 4, 16, 16, 16, 2, 3, 2, 2
    x = c64(crandn(rng, T, D, P, Q))
    s = N1 * N2 * N3 * M
    G = torch.empty((s, s), dtype=torch.complex128, device="cuda")
    recon.recon_gram3(ctx.h, to_dev(x), (N1, N2, N3, M), G)
    Gb = slr3.gram_brute3(x.astype(np.complex128), N1, N2, N3, M)
    assert rel(G.cpu().numpy().T, Gb) < 1e-5


@pytest.mark.parametrize("p", [0.0, 0.5])
@pytest.mark.parametrize("case", SMALL + [("128x128x64x12", None)],
                         ids=[c[0] for c in SMALL] + ["128x128x64x12"])
def test_weight3_parity(R, case, p):
    recon, ctx = R
    w, prob = _case(case[1])
    x0 = slr3.AH3(prob["kspace"], prob["masks"])
    G = slr3.gram_fft3(x0, w.N1, w.N2, w.N3, w.M)
    eps = 0.01 * float(np.linalg.eigvalsh(G)[-1])
    T, D, P, Q = prob["masks"].shape
    npair = w.M * (w.M + 1) // 2
    S = torch.empty((npair, D, P, Q), dtype=torch.complex64, device="cuda")
    dsum = torch.empty((npair, 2 * w.N3 - 1, 2 * w.N1 - 1, 2 * w.N2 - 1), dtype=torch.complex128,
                       device="cuda")
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).cuda()  # column-major
    recon.recon_weight3(ctx.h, (T, D, P, Q), _filt(w), Gd, eps, p, S, dsum)
    H, _ = slr.weight_H(G, eps, p)
    d_ref = slr3.diag_sums3(H, w.N1, w.N2, w.N3, w.M)
    S_ref = slr3.weight_S3(d_ref, D, P, Q)
    ed = rel(dsum.cpu().numpy(), _lags_pairs3(d_ref))
    es = rel(S.cpu().numpy(), pairs_from_full(S_ref))
    print(f"\n[weight3 {case[0]} p={p}] dsum {ed:.2e} S {es:.2e}")
    assert ed < 1e-8 and es < 1e-5


@pytest.mark.parametrize("case", CASES + [FOLD], ids=[c[0] for c in CASES + [FOLD]])
def test_normal3_operator_parity(R, case):
    recon, ctx = R
    w, prob = _case(case[1])
    masks = prob["masks"]
    rng = np.random.default_rng(11)
    x0 = slr3.AH3(prob["kspace"], masks)
    G = slr3.gram_fft3(x0, w.N1, w.N2, w.N3, w.M)
    S = slr3.weight_from_x3(x0, w.N1, w.N2, w.N3, w.M, 0.01 * np.linalg.eigvalsh(G)[-1], 0.0)
    S = S.astype(np.complex64).astype(np.complex128)
    v = c64(crandn(rng, *masks.shape))
    y = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    # lambda chosen so that both terms of the operator carry weight
    lam = float(np.linalg.norm(slr3.AH3(slr3.A3(v, masks), masks)) /
                np.linalg.norm(slr3.apply_W3(v.astype(np.complex128), S)))
    recon.recon_apply_normal3(ctx.h, to_dev(masks), _filt(w), to_dev(c64(pairs_from_full(S))), lam,
                              to_dev(v), y)
    ref = slr3.normal_op3(v.astype(np.complex128), masks, S, lam)
    err, peak = assert_close(y.cpu().numpy(), ref, 1e-5, "normal3")
    print(f"\n[normal3 {case[0]}] rel. error {err:.2e} (peak-relative element {peak:.2e}; lambda "
          f"{lam:.3g})")


def _check_solve(recon, ctx, w, prob, tag, n_irls, n_cg):
    masks = prob["masks"]
    out = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    b = c64(prob["kspace"])
    recon.recon_solve3(ctx.h, to_dev(b), to_dev(masks), _filt(w), w.lam, w.p, n_irls, n_cg, out)
    x_gpu = out.cpu().numpy()
    x_ref = slr3.irls3(b.astype(np.complex128), masks, w.N1, w.N2, w.N3, w.M, w.lam, w.p, n_irls,
                       n_cg)
    xt = prob["x_true"]
    x0 = slr3.AH3(b.astype(np.complex128), masks)
    err, peak = assert_close(x_gpu, x_ref, 1e-4, f"solve3 {tag}")
    print(f"\n[solve3 {tag}] |x_gpu - x_oracle| / |x_oracle| = {err:.2e} (peak-relative element "
          f"{peak:.2e}); NRMSE gpu {rel(x_gpu, xt):.5f} oracle {rel(x_ref, xt):.5f} adjoint "
          f"{rel(x0, xt):.5f}")
    return x_gpu, x0, xt


def test_solve3_parity_small(R):
    recon, ctx = R
    w, prob = _small()
    x_gpu, x0, xt = _check_solve(recon, ctx, w, prob, "16x16x32x6 5 x 8", w.n_irls, w.n_cg)
    assert rel(x_gpu, xt) < rel(x0, xt)


def test_solve3_parity_m3(R):
    recon, ctx = R
    w, prob = _small(**SMALL[1][1])
    _check_solve(recon, ctx, w, prob, "32x32x64x5 M=3 3 x 6", 3, 6)


def test_solve3_parity_fold(R):
    """A 128 x 128 x 64 volume series (the split length-P DFT in every CG step), 2 x 4."""
    recon, ctx = R
    w, prob = _small(**FOLD[1])
    _check_solve(recon, ctx, w, prob, "128x128x64x4 M=3 2 x 4", 2, 4)


def test_solve3_eig_path_matches(R):
    """p = 0 through the eigendecomposition gives the sweep-inverse solve (same weight)."""
    recon, ctx = R
    w, prob = _small()
    masks = to_dev(prob["masks"])
    b = to_dev(c64(prob["kspace"]))
    a = torch.empty(prob["masks"].shape, dtype=torch.complex64, device="cuda")
    e = torch.empty_like(a)
    recon.recon_solve3(ctx.h, b, masks, _filt(w), w.lam, 0.0, 3, 6, a)
    recon.recon_solve3(ctx.h, b, masks, _filt(w), w.lam, 0.0, 3, 6, e,
                       weight_method=recon.RECON_WEIGHT_EIG)
    assert rel(e.cpu().numpy(), a.cpu().numpy()) < 1e-5


@pytest.mark.slow
def test_solve3_parity_128x128x64x12_short(R):
    """The full-size volume series in the benchmark's launch shapes, 2 IRLS x 3 CG (the oracle
    then finishes in tens of seconds)."""
    recon, ctx = R
    w = synth.workload("vol_128x128x64x12")
    _check_solve(recon, ctx, w, synth.make_problem(w), "128x128x64x12 2 x 3", 2, 3)


def test_depth_one_equals_2d(R):
    """R = N3 = 1 through the volume entry points is the 2-D method."""
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=3, n_cg=5)
    prob = synth.make_problem(w)
    b = to_dev(c64(prob["kspace"]))
    m = to_dev(prob["masks"])
    out2 = torch.empty(prob["masks"].shape, dtype=torch.complex64, device="cuda")
    out3 = torch.empty_like(out2)
    recon.recon_solve(ctx.h, b, m, (w.N1, w.N2, w.M), w.lam, w.p, w.n_irls, w.n_cg, out2)
    recon.recon_solve3(ctx.h, b.unsqueeze(1).contiguous(), m.unsqueeze(1).contiguous(),
                       (w.N1, w.N2, 1, w.M), w.lam, w.p, w.n_irls, w.n_cg, out3.unsqueeze(1))
    assert torch.equal(out2, out3)


def test_volume_errors(R):
    recon, ctx = R
    w, prob = _small()
    masks = to_dev(prob["masks"])
    b = to_dev(c64(prob["kspace"]))
    out = torch.empty(prob["masks"].shape, dtype=torch.complex64, device="cuda")
    for filt in [(3, 3, 17, 2), (3, 3, 0, 2)]:  # N3 > R, N3 < 1
        with pytest.raises(recon.ReconError) as e:
            recon.recon_solve3(ctx.h, b, masks, filt, w.lam, w.p, 2, 2, out)
        assert e.value.code == recon.RECON_EINVAL
    bad = torch.empty((6, 24, 16, 32), dtype=torch.complex64, device="cuda")  # R = 24 unsupported
    with pytest.raises(recon.ReconError) as e:
        recon.recon_fft3(ctx.h, bad, bad)
    assert e.value.code == recon.RECON_EINVAL


def test_solve3_bf16_kspace(R):
    """Volumes with k-space stored as bfloat16 pairs (FP32 transforms and CG, FP64 weight): the
    oracle gets the same bfloat16-rounded k-space, so the gate measures the solver."""
    recon, ctx = R
    w, prob = _small()
    bt = torch.view_as_real(torch.from_numpy(c64(prob["kspace"]))).to(torch.bfloat16).contiguous()
    b_rounded = torch.view_as_complex(bt.float()).numpy().astype(np.complex128)
    masks = prob["masks"]
    out = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    recon.recon_solve3(ctx.h, bt.cuda(), to_dev(masks), _filt(w), w.lam, w.p, w.n_irls, w.n_cg, out)
    x_ref = slr3.irls3(b_rounded, masks, w.N1, w.N2, w.N3, w.M, w.lam, w.p, w.n_irls, w.n_cg)
    err, peak = assert_close(out.cpu().numpy(), x_ref, 1e-4, "solve3 bf16 k-space")
    print(f"\n[solve3 bf16 k-space] {err:.2e} (peak-relative element {peak:.2e}); NRMSE "
          f"{rel(out.cpu().numpy(), prob['x_true']):.5f}")
