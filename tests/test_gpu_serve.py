"""Continuous batching: requests of different sizes served concurrently through
recon_submit / recon_poll give exactly the result of solving each alone, also when a tight
memory budget forces the server to wait for completions before admitting the next request."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SHAPES = [(32, 8, 5, 2), (64, 10, 7, 3), (32, 12, 5, 3), (64, 8, 5, 2), (128, 9, 7, 2)]


def _requests(serve, spacing_s):
    reqs = []
    for i, (P, T, N, M) in enumerate(SHAPES):
        w = synth.workload("tiny_32x32x8", P=P, Q=P, T=T, N1=N, N2=N, M=M, n_irls=4, n_cg=6,
                           times_ms=tuple(5.0 + 5.0 * n for n in range(T)), seed=300 + i)
        prob = synth.make_problem(w)
        k = torch.from_numpy(np.ascontiguousarray(prob["kspace"], dtype=np.complex64)).cuda()
        m = torch.from_numpy(prob["masks"]).cuda()
        out = torch.full(tuple(m.shape), float("nan"), dtype=torch.complex64, device="cuda")
        reqs.append(serve.Request(arrival_s=spacing_s * i, kspace=k, masks=m, out=out,
                                  filt=(N, N, M), lam=w.lam, p=w.p, irls=w.n_irls, cg=w.n_cg))
    return reqs


def _solo(recon, reqs):
    ctx = recon.Context(0)
    try:
        outs = []
        for r in reqs:
            o = torch.empty_like(r.out)
            recon.recon_solve(ctx.h, r.kspace, r.masks, r.filt, r.lam, r.p, r.irls, r.cg, o)
            outs.append(o.cpu().numpy())
        return outs
    finally:
        ctx.close()


@pytest.mark.parametrize("budget_mb", [0, 7])
def test_served_results_equal_solo(budget_mb):
    """budget 0: staggered arrivals, unlimited memory. budget 7 MB: every request arrives at
    once and the workspaces of the first three already fill the budget, so later ones are
    admitted only as earlier ones complete."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04511_gb300 import recon, serve
    reqs = _requests(serve, 0.0 if budget_mb else 0.002)
    solo = _solo(recon, reqs)
    srv = serve.Server(0, mem_budget_bytes=budget_mb << 20, max_inflight=4)
    try:
        stats = srv.run(reqs)
    finally:
        srv.close()
    assert stats["requests"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    if budget_mb:
        assert stats["busy_refusals"] > 0        # admission had to wait for memory
    for r, ref in zip(reqs, solo):
        assert r.done_s >= r.submitted_s >= r.arrival_s - 1e-3
        assert np.array_equal(r.out.cpu().numpy(), ref)
