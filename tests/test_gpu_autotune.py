"""The column-pass autotuner (RECON_OPT_AUTOTUNE, recon_tile_cache): the tuned tile widths give
bitwise the same reconstructions as the built-in ones, the choices are cached per context, and
a cache file written by one context is read back by another. The radix schedules of the
Stockham column passes (RECON_OPT_AUTOTUNE_FFT, RECON_OPT_FFT_SCHEDULE) change the FP32
arithmetic: each schedule is checked against the FP64 oracle, operator and whole solve."""

import numpy as np
import pytest

import synth
from oracle import slr, slr3

from gpu_util import assert_close, c64, crandn, pairs_from_full, rel, to_dev

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


def test_cache_lines_with_and_without_schedules(recon, tmp_path):
    f = tmp_path / "tiles.txt"
    f.write_text("64 64 8 1 1 16 0\n192 192 6 1 1 8 0 1 0\n")
    with recon.Context(0) as ctx:
        recon.recon_tile_cache(ctx.h, f)
        assert recon.recon_tile_choice(ctx.h, (8, 64, 64)) == (16, 0)
        assert recon.recon_fft_schedule_choice(ctx.h, (8, 64, 64)) == (0, 0)
        assert recon.recon_fft_schedule_choice(ctx.h, (6, 192, 192)) == (1, 0)
        assert recon.recon_fft_schedule_choice(ctx.h, (6, 32, 32)) == (-1, -1)
    bad = tmp_path / "bad.txt"
    bad.write_text("64 64 8 1 1 16 0 2 0\n")
    with recon.Context(0) as ctx:
        with pytest.raises(recon.ReconError):
            recon.recon_tile_cache(ctx.h, bad)


SCHED_OPS = [("64x64x8", dict(P=64, Q=64, T=8, N1=5, N2=5, M=2)),
             ("192x192x6", dict(P=192, Q=192, T=6, N1=5, N2=5, M=2)),
             ("32x16x10-M3", dict(P=32, Q=16, T=10, N1=3, N2=3, M=3))]


def _times(T):
    return tuple(5.0 + 6.0 * n for n in range(T))


@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("case", SCHED_OPS, ids=[c[0] for c in SCHED_OPS])
def test_radix_schedule_operator_parity(recon, case, sched):
    """(A^H A + lambda W) with the column passes' Stockham transforms in each radix schedule."""
    kw = dict(case[1], times_ms=_times(case[1]["T"]))
    w = synth.workload("tiny_32x32x8", **kw)
    prob = synth.make_problem(w)
    masks = prob["masks"]
    rng = np.random.default_rng(31)
    npair = w.M * (w.M + 1) // 2
    S_full = np.zeros((w.M, w.M, w.P, w.Q), dtype=np.complex128)
    for a in range(w.M):
        for b in range(a, w.M):
            v = crandn(rng, w.P, w.Q) * (0.3 if a != b else 1.0)
            S_full[a, b] = v if a != b else np.abs(v)
            S_full[b, a] = np.conj(S_full[a, b])
    S_full = S_full.astype(np.complex64).astype(np.complex128)
    v = c64(crandn(rng, *masks.shape))
    with recon.Context(0) as ctx:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_FFT_SCHEDULE, sched)
        y = torch.empty(masks.shape, dtype=torch.complex64, device="cuda")
        recon.recon_apply_normal(ctx.h, to_dev(masks), (w.N1, w.N2, w.M),
                                 to_dev(c64(pairs_from_full(S_full))), 0.05, to_dev(v), y)
        ref = slr.normal_op(v.astype(np.complex128), masks, S_full, 0.05)
        e, _ = assert_close(y.cpu().numpy(), ref, 1e-5, f"schedule {sched}")
    print(f"\n[radix schedule {sched}, {case[0]}] operator {e:.2e}")


@pytest.mark.parametrize("sched", [0, 1])
def test_radix_schedule_solve_parity(recon, sched):
    """A whole solve at 64x64x8 (Stockham column passes) with each radix schedule forced."""
    w = synth.workload("tiny_32x32x8", P=64, Q=64, n_irls=6, n_cg=6)
    prob = synth.make_problem(w)
    out = torch.empty(prob["masks"].shape, dtype=torch.complex64, device="cuda")
    with recon.Context(0) as ctx:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_FFT_SCHEDULE, sched)
        _solve(recon, ctx, w, prob, out)
    x_ref = slr.irls(c64(prob["kspace"]).astype(np.complex128), prob["masks"], w.N1, w.N2, w.M,
                     w.lam, w.p, w.n_irls, w.n_cg)
    e, _ = assert_close(out.cpu().numpy(), x_ref, 1e-4, f"schedule {sched}")
    print(f"\n[radix schedule {sched}, solve 64x64x8] {e:.2e}")


def test_radix_schedule_autotune_volume(recon):
    """The tuner picks a (tile, schedule) pair for the length-P and depth passes of a volume;
    the solve with that choice matches the FP64 volume oracle, and the choice is cached."""
    kw = dict(P=32, Q=32, depth=16, T=6, times_ms=tuple(10.0 * (n + 1) for n in range(6)),
              N1=3, N2=3, N3=2, M=2, n_irls=2, n_cg=3)
    w = synth.workload("vol_128x128x64x12", **kw)
    prob = synth.make_problem(w)
    shape = prob["masks"].shape
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    with recon.Context(0) as ctx:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_AUTOTUNE_FFT, 1)
        _solve(recon, ctx, w, prob, out)
        sched = recon.recon_fft_schedule_choice(ctx.h, shape)
        tiles = recon.recon_tile_choice(ctx.h, shape)
    assert sched[0] in (0, 1) and sched[1] in (0, 1)
    x_ref = slr3.irls3(c64(prob["kspace"]).astype(np.complex128), prob["masks"], w.N1, w.N2, w.N3,
                       w.M, w.lam, w.p, w.n_irls, w.n_cg)
    e, _ = assert_close(out.cpu().numpy(), x_ref, 1e-4, "tuned volume")
    print(f"\n[autotune with schedules, volume 32x32x16x6] tiles {tiles} schedules {sched}: {e:.2e}")
