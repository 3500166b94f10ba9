"""recon_solve_batch: concurrent independent solves (one stream each) give exactly the results
of solving each problem alone (fixed launch shapes and reduction orders), on both weight paths."""

import numpy as np
import pytest

import synth

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


def _inputs(w, seeds):
    ks, ms = [], []
    for sd in seeds:
        prob = synth.make_problem(synth.workload(w.name, seed=sd, n_irls=w.n_irls, p=w.p))
        ks.append(torch.from_numpy(np.ascontiguousarray(prob["kspace"], dtype=np.complex64)).cuda())
        ms.append(torch.from_numpy(prob["masks"]).cuda())
    return ks, ms


@pytest.mark.parametrize("p,method", [(0.0, 0), (0.7, 0), (0.0, 1)])
def test_batch_equals_solo(R, p, method):
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=5, p=p)
    seeds = [0, 1, 2]
    ks, ms = _inputs(w, seeds)
    filt = (w.N1, w.N2, w.M)
    solo = []
    for k, m in zip(ks, ms):
        out = torch.empty(tuple(m.shape), dtype=torch.complex64, device="cuda")
        recon.recon_solve(ctx.h, k, m, filt, w.lam, w.p, w.n_irls, w.n_cg, out, weight_method=method)
        solo.append(out.cpu().numpy())
    outs = [torch.full(tuple(m.shape), float("nan"), dtype=torch.complex64, device="cuda") for m in ms]
    recon.recon_solve_batch(ctx.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, outs,
                            weight_method=method)
    for a, b in zip(outs, solo):
        assert np.array_equal(a.cpu().numpy(), b)
    # the problems differ, so the slots did not share state
    assert not np.array_equal(solo[0], solo[1])


@pytest.mark.parametrize("group", [1, 2, 3, 4])
def test_lockstep_batch_equals_solo(R, group):
    """Lockstep batches (RECON_OPT_BATCH_GROUP): the Lanczos, eps and sweep launches of each group
    serve all of its solves at once (group 2 over three solves leaves a ragged group of one;
    group 1 gives three groups whose weight launches take turns). Every result is bitwise the
    solo one, also on a second replay of the captured batch graph."""
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=5)
    ks, ms = _inputs(w, [0, 1, 2])
    filt = (w.N1, w.N2, w.M)
    solo = []
    for k, m in zip(ks, ms):
        out = torch.empty(tuple(m.shape), dtype=torch.complex64, device="cuda")
        recon.recon_solve(ctx.h, k, m, filt, w.lam, w.p, w.n_irls, w.n_cg, out)
        solo.append(out.cpu().numpy())
    recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, group)
    try:
        outs = [torch.full(tuple(m.shape), float("nan"), dtype=torch.complex64, device="cuda")
                for m in ms]
        for _ in range(2):
            recon.recon_solve_batch(ctx.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, outs)
            for a, b in zip(outs, solo):
                assert np.array_equal(a.cpu().numpy(), b)
            for o in outs:
                o.fill_(float("nan"))
    finally:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 0)


def test_lockstep_batch_perf_size(R):
    """Four 256x256x16 solves (s = 243) in one group: one sweep launch per IRLS iteration for
    the four, results bitwise the solo ones."""
    recon, ctx = R
    w = synth.workload("perf_256x256x16", n_irls=3)
    ks, ms = _inputs(w, [0, 5, 6, 7])
    filt = (w.N1, w.N2, w.M)
    solo = []
    for k, m in zip(ks, ms):
        out = torch.empty(tuple(m.shape), dtype=torch.complex64, device="cuda")
        recon.recon_solve(ctx.h, k, m, filt, w.lam, w.p, w.n_irls, w.n_cg, out)
        solo.append(out.cpu().numpy())
    recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 4)
    try:
        outs = [torch.empty(tuple(ms[0].shape), dtype=torch.complex64, device="cuda") for _ in ms]
        recon.recon_solve_batch(ctx.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, outs)
        for a, b in zip(outs, solo):
            assert np.array_equal(a.cpu().numpy(), b)
    finally:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 0)


UNEVEN = [(32, 8, (5, 5, 2)), (64, 12, (9, 9, 3)), (16, 6, (3, 3, 1)), (32, 10, (7, 5, 3)),
          (64, 8, (5, 7, 2))]


@pytest.mark.parametrize("group", [0, 2, 5])
def test_uneven_batch_equals_solo(R, group):
    """recon_solve_many: five problems of different grids, frame counts and filters (s = 50,
    243, 9, 105 and 70). Independent slots (group 0), and lockstep groups whose shared sweep and
    Lanczos launches mix matrices of different sizes; every result bitwise the solo one."""
    recon, ctx = R
    ks, ms, filts, solo = [], [], [], []
    for i, (P, T, filt) in enumerate(UNEVEN):
        w = synth.workload("tiny_32x32x8", P=P, Q=P, T=T, N1=filt[0], N2=filt[1], M=filt[2],
                           n_irls=4, n_cg=5, times_ms=tuple(5.0 + 4.0 * n for n in range(T)),
                           seed=40 + i)
        prob = synth.make_problem(w)
        ks.append(torch.from_numpy(np.ascontiguousarray(prob["kspace"], dtype=np.complex64)).cuda())
        ms.append(torch.from_numpy(prob["masks"]).cuda())
        filts.append(filt)
        out = torch.empty((T, P, P), dtype=torch.complex64, device="cuda")
        recon.recon_solve(ctx.h, ks[-1], ms[-1], filt, w.lam, w.p, w.n_irls, w.n_cg, out)
        solo.append(out.cpu().numpy())
    recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, group)
    try:
        outs = [torch.full(tuple(m.shape), float("nan"), dtype=torch.complex64, device="cuda")
                for m in ms]
        for _ in range(2):  # capture, then replay of the batch graph
            recon.recon_solve_many(ctx.h, ks, ms, filts, w.lam, w.p, w.n_irls, w.n_cg, outs)
            for a, b in zip(outs, solo):
                assert np.array_equal(a.cpu().numpy(), b)
            for o in outs:
                o.fill_(float("nan"))
    finally:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 0)


def test_batch_perf_size_two_slots(R):
    recon, ctx = R
    w = synth.workload("perf_256x256x16", n_irls=2)
    ks, ms = _inputs(w, [0, 5])
    filt = (w.N1, w.N2, w.M)
    solo = torch.empty(tuple(ms[1].shape), dtype=torch.complex64, device="cuda")
    recon.recon_solve(ctx.h, ks[1], ms[1], filt, w.lam, w.p, w.n_irls, w.n_cg, solo)
    outs = [torch.empty_like(solo) for _ in ms]
    recon.recon_solve_batch(ctx.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, outs)
    assert np.array_equal(outs[1].cpu().numpy(), solo.cpu().numpy())


def test_batch_errors(R):
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=1)
    ks, ms = _inputs(w, [0])
    out = [torch.empty(tuple(ms[0].shape), dtype=torch.complex64, device="cuda")]
    with pytest.raises(recon.ReconError) as e:
        recon.recon_solve_batch(ctx.h, ks * 17, ms * 17, (5, 5, 2), w.lam, w.p, 1, 1, out * 17)
    assert e.value.code == recon.RECON_EINVAL


def test_graph_replay_matches_direct_launches(R):
    """A solve replayed from its captured CUDA graph equals the directly launched one, also on
    a second replay and after the output buffer changes (re-capture)."""
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=6)
    ks, ms = _inputs(w, [3])
    filt = (w.N1, w.N2, w.M)

    def run(out):
        recon.recon_solve(ctx.h, ks[0], ms[0], filt, w.lam, w.p, w.n_irls, w.n_cg, out)
        return out.cpu().numpy()

    shape = tuple(ms[0].shape)
    recon.recon_set_option(ctx.h, recon.RECON_OPT_GRAPHS, 0)
    direct = run(torch.empty(shape, dtype=torch.complex64, device="cuda"))
    recon.recon_set_option(ctx.h, recon.RECON_OPT_GRAPHS, 1)
    o1 = torch.empty(shape, dtype=torch.complex64, device="cuda")
    first = run(o1)
    o1.fill_(float("nan"))
    second = run(o1)                       # replay of the cached graph
    third = run(torch.empty(shape, dtype=torch.complex64, device="cuda"))   # re-capture
    for got in (first, second, third):
        assert np.array_equal(got, direct)


def test_batch_over_budget_fails_cleanly(R):
    """A batch whose later slots do not fit the context's memory budget: the call reports
    RECON_ENOMEM after the first slots' work was queued, waits for that work before returning,
    and the context then solves as before (bitwise the result of a fresh context)."""
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=3)
    ks, ms = _inputs(w, [0, 1, 2, 3])
    filt = (w.N1, w.N2, w.M)
    need = recon.recon_bytes_needed(tuple(ms[0].shape), filt)
    ref = torch.empty(tuple(ms[0].shape), dtype=torch.complex64, device="cuda")
    recon.recon_solve(ctx.h, ks[0], ms[0], filt, w.lam, w.p, w.n_irls, w.n_cg, ref)
    small = recon.Context(0, mem_budget_bytes=int(2.5 * need))
    try:
        outs = [torch.empty(tuple(m.shape), dtype=torch.complex64, device="cuda") for m in ms]
        with pytest.raises(recon.ReconError) as e:
            recon.recon_solve_batch(small.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, outs)
        assert e.value.code == recon.RECON_ENOMEM
        torch.cuda.synchronize()
        out = torch.empty_like(ref)
        recon.recon_solve(small.h, ks[0], ms[0], filt, w.lam, w.p, w.n_irls, w.n_cg, out)
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    finally:
        small.close()


@pytest.mark.parametrize("pinned,group,bf16", [(True, 0, False), (False, 0, False),
                                               (True, 2, False), (True, 0, True)])
def test_host_batch_equals_device_batch(R, pinned, group, bf16):
    """recon_solve_batch_host (k-space, masks and images in host memory, copied per slot on the
    slot's own stream) gives bitwise the images of recon_solve_batch on device copies of the same
    inputs: page-locked and pageable host memory, independent slots and a lockstep group, and
    k-space stored as bfloat16 pairs (half the bytes copied)."""
    recon, ctx = R
    w = synth.workload("tiny_32x32x8", n_irls=4)
    ks, ms = _inputs(w, [0, 1, 2])
    if bf16:
        ks = [torch.view_as_real(k).to(torch.bfloat16).contiguous() for k in ks]
    filt = (w.N1, w.N2, w.M)
    shape = tuple(ms[0].shape)
    ref = [torch.empty(shape, dtype=torch.complex64, device="cuda") for _ in ms]
    recon.recon_solve_batch(ctx.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, ref)
    hk = [k.cpu() for k in ks]
    hm = [m.cpu() for m in ms]
    ho = [torch.full(shape, float("nan"), dtype=torch.complex64) for _ in ms]
    if pinned:
        hk = [t.pin_memory() for t in hk]
        hm = [t.pin_memory() for t in hm]
        ho = [t.pin_memory() for t in ho]
    recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, group)
    try:
        for _ in range(2):  # the second call replays the slots' graphs
            recon.recon_solve_batch_host(ctx.h, hk, hm, filt, w.lam, w.p, w.n_irls, w.n_cg, ho)
            for a, b in zip(ho, ref):
                assert np.array_equal(a.numpy(), b.cpu().numpy())
            for o in ho:
                o.fill_(float("nan"))
    finally:
        recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 0)
    with pytest.raises(ValueError):
        recon.recon_solve_batch_host(ctx.h, ks, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, ho)
