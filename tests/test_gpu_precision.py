"""Precision report: the stored k-space in complex64 or bfloat16 pairs, FP32 transforms and CG,
FP64 weight, against the FP64 oracle on the same stored k-space (so the numbers measure the
solver, not the storage), on the 32x32x8 parity series (20 x 10) and the 256x256x16 benchmark
series (30 x 15, bfloat16; its complex64 run is test_gpu_parity.test_solve_parity_perf).

Per case: the Gram matrix of x0 = A^H b (relative Frobenius error), the final image (relative
error and the difference of the NRMSE against the ground truth) and the mono-exponential T2 map
(relative L2 over the foreground), each against its gate: Gram 1e-5, NRMSE difference 1e-4,
T2 map 0.5 %. The storage's own cost is printed beside it (NRMSE of the bfloat16 solve minus
that of the complex64 solve, both from the oracle).
"""

import numpy as np
import pytest

import synth
from oracle import slr, t2fit

from gpu_util import c64, rel, to_dev

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


def _stored(kspace, bf16):
    """(device tensor as stored, the same values as complex128 for the oracle)."""
    if bf16:
        bt = torch.view_as_real(torch.from_numpy(c64(kspace))).to(torch.bfloat16).contiguous()
        return bt.cuda(), torch.view_as_complex(bt.float()).numpy().astype(np.complex128)
    return to_dev(c64(kspace)), c64(kspace).astype(np.complex128)


CASES = [("tiny_32x32x8", False), ("tiny_32x32x8", True), ("perf_256x256x16", True)]


@pytest.mark.parametrize("name,bf16", CASES, ids=[f"{n}-{'bf16' if b else 'c64'}" for n, b in CASES])
def test_precision_report(R, name, bf16):
    recon, ctx = R
    w = synth.workload(name)
    prob = synth.make_problem(w)
    masks, xt = prob["masks"], prob["x_true"]
    b_dev, b_ref = _stored(prob["kspace"], bf16)
    m_dev = to_dev(masks)
    filt = (w.N1, w.N2, w.M)
    # Gram of x0 (the GPU adjoint's output, the same input on both sides)
    x0 = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    recon.recon_adjoint(ctx.h, b_dev, m_dev, x0)
    s = w.N1 * w.N2 * w.M
    G = torch.empty((s, s), dtype=torch.complex128, device="cuda")
    recon.recon_gram(ctx.h, x0, filt, G)
    G_ref = slr.gram_fft(x0.cpu().numpy().astype(np.complex128), *filt)
    e_gram = rel(G.cpu().numpy().T, G_ref)
    # the reconstruction and its T2 map
    out = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
    recon.recon_solve(ctx.h, b_dev, m_dev, filt, w.lam, w.p, w.n_irls, w.n_cg, out)
    x_gpu = out.cpu().numpy()
    x_ref = slr.irls(b_ref, masks, *filt, w.lam, w.p, w.n_irls, w.n_cg)
    nrmse_gpu, nrmse_ref = rel(x_gpu, xt), rel(x_ref, xt)
    fg = t2fit.foreground(xt)
    t2_err = t2fit.t2_rel_l2(t2fit.fit_t2(x_ref, w.times_ms, fg), t2fit.fit_t2(x_gpu, w.times_ms, fg))
    line = (f"\n[precision {name} {'bf16' if bf16 else 'c64'} k-space, {w.n_irls} x {w.n_cg}] "
            f"Gram {e_gram:.2e}; image vs oracle {rel(x_gpu, x_ref):.2e}; NRMSE gpu {nrmse_gpu:.6f} "
            f"oracle {nrmse_ref:.6f} (diff {abs(nrmse_gpu - nrmse_ref):.1e}); T2 map {t2_err:.2e}")
    if bf16 and name == "tiny_32x32x8":
        x_c64 = slr.irls(c64(prob["kspace"]).astype(np.complex128), masks, *filt, w.lam, w.p,
                         w.n_irls, w.n_cg)
        line += f"; storage cost (oracle NRMSE bf16 - c64) {nrmse_ref - rel(x_c64, xt):+.1e}"
    print(line)
    assert e_gram < 1e-5
    assert abs(nrmse_gpu - nrmse_ref) < 1e-4
    assert t2_err < 5e-3
