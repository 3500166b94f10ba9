"""The column-tile autotuner (RECON_OPT_AUTOTUNE, recon_tile_cache): the tuned launch shapes give
bitwise the same reconstructions as the built-in ones, the choices are cached per context, and
a cache file written by one context is read back by another."""

import numpy as np
import pytest

import synth

from gpu_util import c64, to_dev

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def recon():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04511_gb300 import recon
    return recon


CASES = [("128x128x12", "coils_128x128x12", dict(n_coils=1, n_irls=3, n_cg=4)),
         ("64x64x8", "tiny_32x32x8", dict(P=64, Q=64, n_irls=3, n_cg=4)),
         ("vol-32x32x16x6", "vol_128x128x64x12",
          dict(P=32, Q=32, depth=16, T=6, times_ms=tuple(10.0 * (n + 1) for n in range(6)),
               N1=3, N2=3, N3=2, M=2, n_irls=2, n_cg=3))]


def _solve(recon, ctx, w, prob, out):
    b = to_dev(c64(prob["kspace"]))
    m = to_dev(prob["masks"])
    if w.depth > 1:
        recon.recon_solve3(ctx.h, b, m, (w.N1, w.N2, w.N3, w.M), w.lam, w.p, w.n_irls, w.n_cg, out)
    else:
        recon.recon_solve(ctx.h, b, m, (w.N1, w.N2, w.M), w.lam, w.p, w.n_irls, w.n_cg, out)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tuned_tiles_give_identical_results(recon, case, tmp_path):
    _, name, kw = case
    w = synth.workload(name, **kw)
    prob = synth.make_problem(w)
    shape = prob["masks"].shape
    cache = tmp_path / "tiles.txt"
    ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(ref)
    with recon.Context(0) as ctx:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_AUTOTUNE, 0)
        _solve(recon, ctx, w, prob, ref)
        assert recon.recon_tile_choice(ctx.h, shape) == (0, 0)
    with recon.Context(0) as ctx:
        recon.recon_tile_cache(ctx.h, cache)
        _solve(recon, ctx, w, prob, out)
        choice = recon.recon_tile_choice(ctx.h, shape)
        _solve(recon, ctx, w, prob, out)          # second solve reuses the cached choice
        assert recon.recon_tile_choice(ctx.h, shape) == choice
    print(f"\n[autotune {case[0]}] tiles (column, depth) = {choice}")
    assert torch.equal(out, ref)
    assert choice[0] in (0, 8, 16, 32) and choice[1] in (0, 8, 16, 32)
    with recon.Context(0) as ctx:                 # a new context reads the file
        recon.recon_tile_cache(ctx.h, cache)
        assert recon.recon_tile_choice(ctx.h, shape) == choice


def test_malformed_cache_is_rejected(recon, tmp_path):
    bad = tmp_path / "bad.txt"
    bad.write_text("128 128 12 1 1 7 0\n")
    with recon.Context(0) as ctx:
        with pytest.raises(recon.ReconError) as e:
            recon.recon_tile_cache(ctx.h, bad)
        assert e.value.code == recon.RECON_EINVAL
