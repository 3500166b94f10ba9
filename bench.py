#!/usr/bin/env python
"""Benchmark of the IRLS reconstruction (Algorithm 1) on the 256x256x16 workload.

One step = one complete reconstruction through the C ABI: x0 = A^H b, then 30 IRLS iterations
(Gram, FP64 eigendecomposition, weight, S(r), residual carry, 15 CG steps each) of a seeded
two-component T2 phantom, 8x variable-density mask, 9x9x3 filter, lambda = 1e-3, p = 0.
Metric: IRLS iterations per second (whole job: all ranks' iterations / max rank time).

Prints one JSON line (rank 0). `--impl reference` times the FP64 NumPy oracle instead, on the
host cores, on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IRLS iterations/s, 256x256x16 series, 9x9x3 filter, 15 CG steps per iteration"
UNIT = "IRLS iter/s"
WORKLOAD = "perf_256x256x16"
COIL_WORKLOAD = "coils_128x128x12"
VOL_WORKLOAD = "vol_128x128x64x12"
CMP_WORKLOAD = "cmp_128x128x12"

# kernels launched per profiled scope (eig is the cuSOLVER library call and is not counted;
# diag_sums is one kernel on the p = 0 path, two after the eigendecomposition)
KERNELS_PER_SCOPE = {"adjoint": 2, "gram": 2, "eps": 1, "diag_sums": 1, "weight_S": 2,
                     "resid_carry": 1, "cg_row_fwd": 1, "cg_col_mask": 1, "cg_row_inv_w": 1,
                     "cg_update": 1, "lanczos": 1, "hpd_inverse": 1}


def alg_bytes(kind: str, w, n_cg: int) -> float:
    """Algorithmic bytes per launch (complex64 elements E = T*P*Q, pixels N = P*Q; volumes:
    E = T*D*P*Q, N = D*P*Q). For volumes the column class holds two or three launches (the
    masked depth pass and the column transforms); its algorithmic bytes stay those of the
    operation."""
    D = getattr(w, "depth", 1)
    E = w.T * w.P * w.Q * D
    N = w.P * w.Q * D
    npair = w.M * (w.M + 1) // 2
    if kind == "cg_row_fwd":      # read r (+ p), write p and t
        return (24.0 * E + 32.0 * E * (n_cg - 1)) / n_cg
    if kind == "cg_col_mask":     # read t, mask; write t
        return 17.0 * E
    if kind == "cg_row_inv_w":    # read t, p, S; write q
        return 24.0 * E + 8.0 * npair * N
    if kind == "cg_update":       # read x, r, p, q; write x, r
        return 48.0 * E
    if kind == "resid_carry":     # read x, r, S_old, S_new; write r (first: no r, S_old)
        return 24.0 * E + 16.0 * npair * N
    if kind == "gram":            # read x
        return 8.0 * E
    if kind == "adjoint":         # read b, mask, write t; read t, write x
        return 33.0 * E
    return 0.0


FP64_NOMINAL_GFLOPS = 1250.0   # GB300 dense FP64, nominal (a probe here measured ~1056)
ALU_KINDS = ("hpd_inverse", "lanczos")
# DRAM bytes (read + write) per launch from one ncu capture of the launch class's kernel at the
# benchmark workload (full-set captures, caches flushed before each pass: the first sweep of the
# bench's first solve, profiles/hpd_sweep_kernel_s243.md; a CG pass of it,
# profiles/cg_kernels_perf_256x256x16.md, which give the commands). Only for the kernel versions
# those captures measured: drop an entry when its kernel changes.
TRAFFIC_BYTES = {"hpd_inverse": 563968, "cg_row_inv_w": 19943168}
# steps of the batch, after the timed region, whose dominant-class launches are timed by events
DOM_STEPS = 3


def alg_flops(kind: str, w) -> float:
    """Algorithmic FP64 FLOPs per launch of the FP64 kernels (complex FMA = 8 flops)."""
    s = w.N1 * w.N2 * w.M
    if kind == "hpd_inverse":
        # the method's work for the inverse of a Hermitian s x s matrix: s^3 / 2 complex FMA
        # (the kernel's padded tile sweep does more; that excess is not counted)
        return 8.0 * s ** 3 / 2.0
    if kind == "lanczos":
        # at most 64 Lanczos steps, one Hermitian matrix-vector product (s^2 complex FMA) each
        return 8.0 * 64 * s * s
    return 0.0


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        t0 = time.time()  # let the first sample arrive before the timed region starts
        while not self.lines and time.time() - t0 < 2.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def whole_job_rate(local_ms: float, units_per_rank: float, dist=None, device=None):
    """Max of the per-rank timed milliseconds over all ranks and the whole-job rate
    (units of every rank / that time). Replicas: each rank does units_per_rank."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    tmax = float(t.item())
    return tmax, world * units_per_rank / (tmax / 1000.0)


def cpu_oracle_rate(w, prob, budget_s: float = 12.0, max_iters: int = 6):
    """FP64 oracle IRLS iterations/s on the host cores (bounded sample)."""
    import numpy as np
    from oracle import slr
    b = prob["kspace"].astype(np.complex64).astype(np.complex128)
    masks = prob["masks"]
    rhs = slr.AH(b, masks)
    x = rhs.copy()
    eps = slr.initial_eps(x, w.N1, w.N2, w.M)
    n = 0
    t0 = time.perf_counter()
    while n < max_iters:
        S = slr.weight_from_x(x, w.N1, w.N2, w.M, eps, w.p)
        x = slr.cg(lambda v: slr.normal_op(v, masks, S, w.lam), rhs, x, w.n_cg)
        eps /= 1.4
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return n / dt, n, dt, cores


def cpu_oracle_one_thread(budget_s: float = 6.0):
    """The same oracle sample with one BLAS / OpenMP thread, in a child process (the thread count
    is fixed when NumPy loads); None if the child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench, synth; w = synth.workload(bench.WORKLOAD); "
            "p = synth.make_problem(w); r = bench.cpu_oracle_rate(w, p, budget_s=%r, max_iters=3); "
            "print(json.dumps(r[0]))" % budget_s)
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                             text=True, timeout=300)
        return float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except Exception:
        return None


def run_coils(steps: int, device: int) -> dict:
    """The multi-coil workload (128x128x12, 12 coils): whole solves, device-resident inputs,
    timed with CUDA events."""
    import numpy as np
    import torch
    import synth
    from paper_1704_04511_gb300 import recon
    w = synth.workload(COIL_WORKLOAD)
    prob = synth.make_problem(w)
    dev = torch.device("cuda", device)
    b = torch.from_numpy(prob["kspace"].astype(np.complex64)).to(dev)
    m = torch.from_numpy(prob["masks"]).to(dev)
    C = torch.from_numpy(prob["coils"].astype(np.complex64)).to(dev)
    out = torch.empty(tuple(m.shape), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = recon.Context(device, cuda_stream=stream.cuda_stream)
    try:
        def solve():
            recon.recon_solve_coils(ctx.h, b, m, C, (w.N1, w.N2, w.M), w.lam, w.p, w.n_irls,
                                    w.n_cg, out)
        for _ in range(2):
            solve()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            solve()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
    finally:
        ctx.close()
    return {"workload": COIL_WORKLOAD, "n_coils": w.n_coils, "irls": w.n_irls, "cg": w.n_cg,
            "filter": [w.N1, w.N2, w.M], "ms_per_solve": round(ms, 3),
            "irls_iters_per_s": round(1000.0 * w.n_irls / ms, 1),
            "note": "recon_solve_coils on device-resident k-space (12 coil series), one solve at "
                    "a time; the k-space of every coil stays in HBM/L2 between steps"}


def run_vol(steps: int, device: int) -> dict:
    """The volume workload (128x128x64 voxels x 12 frames, 7x7x3x2 filter, 25 IRLS x 15 CG):
    whole solves through recon_solve3 on device-resident k-space (working set ~0.6 GB, beyond
    L2, so every CG pass streams from HBM), one profiled solve for the per-class device times."""
    import numpy as np
    import torch
    import synth
    from paper_1704_04511_gb300 import recon
    w = synth.workload(VOL_WORKLOAD)
    prob = synth.make_problem(w)
    dev = torch.device("cuda", device)
    b = torch.from_numpy(prob["kspace"].astype(np.complex64)).to(dev)
    m = torch.from_numpy(prob["masks"]).to(dev)
    out = torch.empty(tuple(m.shape), dtype=torch.complex64, device=dev)
    filt = (w.N1, w.N2, w.N3, w.M)
    stream = torch.cuda.current_stream(dev)
    ctx = recon.Context(device, cuda_stream=stream.cuda_stream)
    try:
        def solve():
            recon.recon_solve3(ctx.h, b, m, filt, w.lam, w.p, w.n_irls, w.n_cg, out)
        solve()
        torch.cuda.synchronize(dev)
        recon.recon_profile(ctx.h, recon.PROF_ALL)
        solve()
        torch.cuda.synchronize(dev)
        prof = {recon.recon_profile_name(k): recon.recon_profile_read(ctx.h, k)
                for k in range(recon.PROF_KINDS)}
        recon.recon_profile(ctx.h, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            solve()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        need = recon.recon_bytes_needed3(tuple(m.shape), filt)
        tiles = recon.recon_tile_choice(ctx.h, tuple(m.shape))
    finally:
        ctx.close()
    peak, peak_src = load_peaks()
    tot = sum(v[0] for v in prof.values())
    classes = {}
    for k, (ms_k, n_k) in prof.items():
        if not n_k:
            continue
        ent = {"ms_per_solve": round(ms_k, 3), "launches": n_k,
               "share": round(ms_k / tot, 4) if tot else None,
               "avg_launch_us": round(1000.0 * ms_k / n_k, 2)}
        ab = alg_bytes(k, w, w.n_cg)
        if ab:
            gbs = ab / (ms_k / n_k / 1000.0) / 1e9
            ent.update({"alg_bytes_per_launch": ab, "achieved_GBs": round(gbs, 1),
                        "frac_of_hbm": round(gbs / peak, 4)})
        classes[k] = ent
    T, D, P, Q = m.shape
    s = w.N1 * w.N2 * w.N3 * w.M
    rows_lifted = (w.T - w.M + 1) * D * P * Q
    return {"workload": VOL_WORKLOAD, "T": T, "D": D, "P": P, "Q": Q, "filter": list(filt),
            "irls": w.n_irls, "cg": w.n_cg, "ms_per_solve": round(ms, 2),
            "irls_iters_per_s": round(1000.0 * w.n_irls / ms, 2),
            "voxel_frame_cg_steps_per_s": round(T * D * P * Q * w.n_irls * w.n_cg / (ms / 1000.0), 1),
            "hbm_peak_GBs": peak, "hbm_peak_source": peak_src, "classes": classes,
            "column_tiles": {"length_P": tiles[0], "depth": tiles[1]},
            "footprint": {"workspace_bytes": int(need),
                          "lifted_matrix_bytes_complex64": int(rows_lifted * s * 8),
                          "gram_bytes_complex128": int(s * s * 16)},
            "note": "recon_solve3, device-resident k-space, solves back to back (CUDA events); "
                    "per-class times from one profiled solve before the timed ones"}


def run_variants(steps: int, device: int) -> dict:
    """The comparison methods of Sec. IV on the 128x128x12 series from 30 % uniform random samples
    (9x9x3 filter, 20 IRLS x 10 CG; HLR-Voxel: 1x1x3): ms per solve (CUDA events, after one
    untimed solve) and NRMSE of each reconstruction against the ground truth."""
    import numpy as np
    import torch
    import synth
    from paper_1704_04511_gb300 import recon
    w = synth.workload(CMP_WORKLOAD)
    prob = synth.make_problem(w)
    dev = torch.device("cuda", device)
    b = torch.from_numpy(prob["kspace"].astype(np.complex64)).to(dev)
    m = torch.from_numpy(prob["masks"]).to(dev)
    out = torch.empty(tuple(m.shape), dtype=torch.complex64, device=dev)
    xt = prob["x_true"]
    stream = torch.cuda.current_stream(dev)
    ctx = recon.Context(device, cuda_stream=stream.cuda_stream)
    res = {}
    try:
        for name, variant, filt in (("proposed", recon.RECON_VARIANT_PROPOSED, (w.N1, w.N2, w.M)),
                                    ("giraf", recon.RECON_VARIANT_GIRAF, (w.N1, w.N2, w.M)),
                                    ("hlr_voxel", recon.RECON_VARIANT_HLR_VOXEL, (1, 1, w.M)),
                                    ("direct", recon.RECON_VARIANT_DIRECT, (w.N1, w.N2, w.M))):
            def solve():
                recon.recon_solve_variant(ctx.h, b, m, filt, w.lam, w.p, w.n_irls, w.n_cg, out,
                                          variant)
            solve()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                solve()
            e1.record(stream)
            e1.synchronize()
            x = out.cpu().numpy().astype(np.complex128)
            res[name] = {"ms_per_solve": round(e0.elapsed_time(e1) / steps, 2),
                         "nrmse": round(float(np.linalg.norm(x - xt) / np.linalg.norm(xt)), 5),
                         "filter": list(filt)}
    finally:
        ctx.close()
    x0 = np.fft.ifft2(prob["masks"] * prob["kspace"], norm="ortho")
    return {"workload": CMP_WORKLOAD, "irls": w.n_irls, "cg": w.n_cg, "lambda": w.lam,
            "sampling": "30 % uniform random per frame", "methods": res,
            "nrmse_adjoint": round(float(np.linalg.norm(x0 - xt) / np.linalg.norm(xt)), 5),
            "direct_over_proposed_time": round(res["direct"]["ms_per_solve"] /
                                               res["proposed"]["ms_per_solve"], 1),
            "note": "recon_solve_variant, one problem at a time, device-resident k-space"}


def run_served(n_requests: int, device: int) -> dict:
    """Continuous batching over the served mix: n requests, Poisson arrivals at 20/s, sizes
    {64, 128, 192, 256}^2, 8-24 frames, filters 5-9 x 2-3, 30 IRLS x 15 CG each."""
    import numpy as np
    import torch

    import synth
    from paper_1704_04511_gb300 import serve
    mix = synth.served_mix(n_requests, rate_hz=20.0, seed=0)
    reqs = []
    for arrival, w in mix:
        pr = synth.make_problem(w)
        k = torch.from_numpy(np.ascontiguousarray(pr["kspace"], dtype=np.complex64)).cuda(device)
        m = torch.from_numpy(pr["masks"]).cuda(device)
        out = torch.empty(tuple(m.shape), dtype=torch.complex64, device=f"cuda:{device}")
        reqs.append(serve.Request(arrival_s=arrival, kspace=k, masks=m, out=out,
                                  filt=(w.N1, w.N2, w.M), lam=w.lam, p=w.p, irls=w.n_irls,
                                  cg=w.n_cg))
    srv = serve.Server(device, mem_budget_bytes=8 << 30, max_inflight=8)
    try:
        stats = srv.run(reqs)
    finally:
        srv.close()
    stats["arrival_rate_hz"] = 20.0
    stats["mix"] = "sizes {64,128,192,256}^2, T 8-24, filter {5,7,9}^2 x {2,3}, 30 IRLS x 15 CG"
    stats["max_inflight"] = 8
    return stats


def run_p07(steps: int, device: int) -> dict:
    """The 256x256x16 workload at the paper's own operating point p = 0.7 (Sec. IV): the weight
    (G + eps I)^(0.35 - 1) needs the eigenvalues, so every IRLS iteration runs the FP64
    eigendecomposition (library zheevd) instead of the sweep inverse. Whole solves on
    device-resident k-space; per-class times from one profiled solve."""
    import numpy as np
    import torch
    import synth
    from paper_1704_04511_gb300 import recon
    w = synth.workload(WORKLOAD, p=0.7)
    prob = synth.make_problem(w)
    dev = torch.device("cuda", device)
    b = torch.from_numpy(prob["kspace"].astype(np.complex64)).to(dev)
    m = torch.from_numpy(prob["masks"]).to(dev)
    out = torch.empty(tuple(m.shape), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = recon.Context(device, cuda_stream=stream.cuda_stream)
    try:
        def solve():
            recon.recon_solve(ctx.h, b, m, (w.N1, w.N2, w.M), w.lam, w.p, w.n_irls, w.n_cg, out)
        solve()
        torch.cuda.synchronize(dev)
        recon.recon_profile(ctx.h, recon.PROF_ALL)
        solve()
        torch.cuda.synchronize(dev)
        eig_ms, eig_n = recon.recon_profile_read(ctx.h, 2)
        recon.recon_profile(ctx.h, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            solve()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
    finally:
        ctx.close()
    return {"workload": WORKLOAD, "p": w.p, "irls": w.n_irls, "cg": w.n_cg,
            "ms_per_solve": round(ms, 2), "irls_iters_per_s": round(1000.0 * w.n_irls / ms, 1),
            "eig_ms_per_solve": round(eig_ms, 2), "eig_calls": eig_n,
            "eig_share": round(eig_ms / ms, 3) if ms else None,
            "note": "p > 0 needs the eigenvalues: FP64 eigendecomposition per IRLS iteration "
                    "(cuSOLVER zheevd, s = 243), direct launches (no graph)"}


def run_many(n: int, steps: int, device: int) -> dict:
    """recon_solve_many on the first n requests of the served mix (uneven grids, frame counts and
    filters, shared parameters): aggregate IRLS iterations/s of the independent slots and of
    lockstep groups whose sweep launches mix the requests' matrices, and the shared sweep's
    per-launch time."""
    import numpy as np
    import torch
    import synth
    from paper_1704_04511_gb300 import recon
    mix = synth.served_mix(n, rate_hz=20.0, seed=0)
    dev = torch.device("cuda", device)
    ks, ms, outs, filts = [], [], [], []
    for _, w in mix:
        pr = synth.make_problem(w)
        ks.append(torch.from_numpy(np.ascontiguousarray(pr["kspace"], dtype=np.complex64)).to(dev))
        ms.append(torch.from_numpy(pr["masks"]).to(dev))
        outs.append(torch.empty(tuple(ms[-1].shape), dtype=torch.complex64, device=dev))
        filts.append((w.N1, w.N2, w.M))
    w0 = mix[0][1]
    stream = torch.cuda.current_stream(dev)
    ctx = recon.Context(device, cuda_stream=stream.cuda_stream)
    inv_kind = [recon.recon_profile_name(k) for k in range(recon.PROF_KINDS)].index("hpd_inverse")
    res = {}
    try:
        def solve():
            recon.recon_solve_many(ctx.h, ks, ms, filts, w0.lam, w0.p, w0.n_irls, w0.n_cg, outs)
        for g in (0, 4, n):
            recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, g)
            solve()
            torch.cuda.synchronize(dev)
            recon.recon_profile(ctx.h, 1 << inv_kind)
            solve()
            torch.cuda.synchronize(dev)
            inv_ms, inv_n = recon.recon_profile_read(ctx.h, inv_kind)
            recon.recon_profile(ctx.h, 0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                solve()
            e1.record(stream)
            e1.synchronize()
            ms_step = e0.elapsed_time(e1) / steps
            res[str(g)] = {"ms_per_batch": round(ms_step, 2),
                           "irls_iters_per_s": round(n * w0.n_irls / (ms_step / 1000.0), 1),
                           "sweep_launches": inv_n,
                           "sweep_us_per_launch": round(1000.0 * inv_ms / inv_n, 1) if inv_n else None}
        recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 0)
    finally:
        ctx.close()
    return {"requests": n, "shapes": [list(m.shape) for m in ms], "filters": filts,
            "groups": res,
            "note": "recon_solve_many over the first requests of the served mix; group 0 = "
                    "independent slots, g > 0 = lockstep groups of g sharing one sweep launch of "
                    "matrices of different sizes per IRLS iteration"}


def run_reference(args, rank: int):
    import synth
    if rank != 0:
        return
    w = synth.workload(WORKLOAD)
    prob = synth.make_problem(w)
    for _ in range(args.warmup):
        cpu_oracle_rate(w, prob, budget_s=0.0, max_iters=1)
    rates, times = [], []
    cores = 1
    for _ in range(args.steps):
        r, n, dt, cores = cpu_oracle_rate(w, prob, budget_s=0.0, max_iters=1)
        rates.append(r)
        times.append(dt)
    value = len(times) / sum(times)
    sample = (f"{WORKLOAD}: 1 IRLS iteration per step (Gram + eigh + weight + {w.n_cg} CG), "
              "FP64 NumPy oracle; numpy.fft single-threaded, eigh on the BLAS threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "irls": 1, "cg": w.n_cg, "filter": [w.N1, w.N2, w.M]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--irls", type=int, default=None, help="override IRLS iterations (testing)")
    ap.add_argument("--batch", type=int, default=4,
                    help="independent problems solved concurrently per step (1 = single solve)")
    ap.add_argument("--coil-steps", type=int, default=3,
                    help="solves of the 12-coil 128x128x12 workload to time (0 = skip)")
    ap.add_argument("--variant-steps", type=int, default=1,
                    help="solves per comparison method on the 128x128x12 30 %% uniform series "
                         "(0 = skip)")
    ap.add_argument("--only-vol", action="store_true",
                    help="time only the volume workload and print {\"vol\": ...} (profiling)")
    ap.add_argument("--vol-steps", type=int, default=2,
                    help="solves of the 128x128x64x12 volume workload to time (0 = skip)")
    ap.add_argument("--many", type=int, default=8,
                    help="served-mix requests solved as one uneven batch (recon_solve_many), 0 = skip")
    ap.add_argument("--p07-steps", type=int, default=1,
                    help="solves of the 256x256x16 workload at p = 0.7 to time (0 = skip)")
    ap.add_argument("--batch-modes", type=int, default=3,
                    help="steps timed per lockstep group size (RECON_OPT_BATCH_GROUP), 0 = skip")
    ap.add_argument("--served", type=int, default=512,
                    help="requests of the served mix (Poisson 20/s, mixed sizes) to serve after "
                         "the timed steps, reported as p50/p99 latency; 0 = skip, 512 = full mix")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.only_vol:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"vol": run_vol(max(args.vol_steps, 1), local_rank)}), flush=True)
        return

    import numpy as np
    import torch

    import synth
    from paper_1704_04511_gb300 import recon

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = synth.workload(WORKLOAD)
    if args.irls is not None:
        w = synth.workload(WORKLOAD, n_irls=args.irls)
    B = args.batch
    probs = [synth.make_problem(synth.workload(w.name, n_irls=w.n_irls, seed=100 * rank + sd))
             for sd in range(B)]
    prob = probs[0]
    b_host = [torch.from_numpy(np.ascontiguousarray(pr["kspace"], dtype=np.complex64)).pin_memory()
              for pr in probs]
    m_host = [torch.from_numpy(np.ascontiguousarray(pr["masks"])).pin_memory() for pr in probs]
    bs = [t.to(dev) for t in b_host]
    ms = [t.to(dev) for t in m_host]
    outs = [torch.empty(tuple(ms[0].shape), dtype=torch.complex64, device=dev) for _ in range(B)]
    out_host = [torch.empty(tuple(ms[0].shape), dtype=torch.complex64).pin_memory() for _ in range(B)]
    stream = torch.cuda.current_stream(dev)
    ctx = recon.Context(local_rank, cuda_stream=stream.cuda_stream)
    filt = (w.N1, w.N2, w.M)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def solve_one():
        recon.recon_solve(ctx.h, bs[0], ms[0], filt, w.lam, w.p, w.n_irls, w.n_cg, outs[0])

    def solve_batch():
        recon.recon_solve_batch(ctx.h, bs, ms, filt, w.lam, w.p, w.n_irls, w.n_cg, outs)

    step = solve_batch if B > 1 else solve_one

    def timed(fn, k):
        tot = 0.0
        for _ in range(k):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot

    for _ in range(args.warmup):
        solve_one()
        if B > 1:
            solve_batch()
    torch.cuda.synchronize(dev)

    # ---- one untimed profiled solve: per-class device time and launch counts per solve
    recon.recon_profile(ctx.h, recon.PROF_ALL)
    solve_one()
    torch.cuda.synchronize(dev)
    prof1 = {}
    for k in range(recon.PROF_KINDS):
        ms_, n_ = recon.recon_profile_read(ctx.h, k)
        prof1[recon.recon_profile_name(k)] = (ms_, n_)
    recon.recon_profile(ctx.h, 0)
    mine1 = {k: v for k, v in prof1.items() if k in KERNELS_PER_SCOPE}
    dom = max(mine1, key=lambda k: mine1[k][0])
    dom_kind = [recon.recon_profile_name(k) for k in range(recon.PROF_KINDS)].index(dom)

    # ---- the single-solve path (the comparison baseline), K device-resident solves
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    single_ms = timed(solve_one, args.steps)

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(gpu_id) if rank == 0 else None

    # ---- timed region: K steps of B concurrent solves replayed from their captured graphs, no
    # instrumentation inside; L2 flushed before each step (outside the events). One untimed step
    # first captures the graphs.
    recon.recon_profile(ctx.h, 0)
    step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    total_ms = timed(step, args.steps)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    # ---- the dominant launch class timed live on the same batch right after the timed region:
    # CUDA events around each of its launches (event nodes in the solve graphs, on the slots'
    # streams), read from the last of DOM_STEPS steps under the same conditions. Not inside the
    # timed region: event nodes around each launch of a CG pass (hundreds per solve) cut the
    # programmatic-dependent-launch overlap and slowed the step by a third.
    recon.recon_profile(ctx.h, 1 << dom_kind)
    step()
    torch.cuda.synchronize(dev)
    timed(step, DOM_STEPS)
    torch.cuda.synchronize(dev)
    batch_dom_ms, batch_dom_n = recon.recon_profile_read(ctx.h, dom_kind)
    # and on the plain single solve, where no other solve's kernels share the GPU while it runs
    # (inside the batch a launch's duration includes the time-sharing with three other solves);
    # the totals restart here (same mask)
    recon.recon_profile(ctx.h, 1 << dom_kind)
    solve_one()
    torch.cuda.synchronize(dev)
    timed(solve_one, DOM_STEPS)
    torch.cuda.synchronize(dev)
    dom_ms, dom_n = recon.recon_profile_read(ctx.h, dom_kind)
    recon.recon_profile(ctx.h, 0)
    step()  # recapture the graphs without event nodes for the sections below
    torch.cuda.synchronize(dev)
    t_max_ms, value = whole_job_rate(total_ms, args.steps * B * w.n_irls, dist, dev)
    single_max_ms, single_value = whole_job_rate(single_ms, args.steps * w.n_irls, dist, dev)
    if dist:
        dist.barrier()

    # ---- end to end: the public host-buffer call on pinned host buffers, copies inside the timed
    # region (each slot copies its own k-space and masks in and its image out on its own stream);
    # every step under the same conditions as the device-timed steps (L2 flushed before it,
    # outside its events; one event pair per step). One untimed call first captures the slots'
    # graphs on the host-buffer path.
    def e2e_step():
        recon.recon_solve_batch_host(ctx.h, b_host, m_host, filt, w.lam, w.p, w.n_irls, w.n_cg,
                                     out_host)

    e2e_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e2e_ms = timed(e2e_step, args.steps)
    _, e2e_value = whole_job_rate(e2e_ms, args.steps * B * w.n_irls, dist, dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    # ---- lockstep batches (RECON_OPT_BATCH_GROUP): the same B solves as one graph whose groups
    # share their FP64 weight launches; IRLS iterations/s per group size (same conditions as the
    # timed steps) and the shared sweep launch timed inside the step (event nodes of the graph)
    lockstep = None
    if B > 1 and args.batch_modes > 0:
        lockstep = {"groups": {}}
        inv_kind = [recon.recon_profile_name(k) for k in range(recon.PROF_KINDS)].index("hpd_inverse")
        for g in sorted({1, 2, B}):
            recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, g)
            recon.recon_profile(ctx.h, 1 << inv_kind)
            step()
            torch.cuda.synchronize(dev)
            g_ms = timed(step, args.batch_modes)
            inv_ms, inv_n = recon.recon_profile_read(ctx.h, inv_kind)
            recon.recon_profile(ctx.h, 0)
            per_launch_us = 1000.0 * inv_ms / inv_n if inv_n else None
            mats = min(g, B)
            ent = {"irls_iters_per_s": round(args.batch_modes * B * w.n_irls / (g_ms / 1000.0), 1),
                   "sweep_launches_per_step": inv_n, "matrices_per_sweep_launch": mats}
            if per_launch_us:
                gfl = mats * alg_flops("hpd_inverse", w) / (per_launch_us * 1e-6) / 1e9
                ent.update({"sweep_us_per_launch": round(per_launch_us, 1),
                            "sweep_us_per_matrix": round(per_launch_us / mats, 1),
                            "sweep_GFLOPs": round(gfl, 1),
                            "sweep_frac_of_fp64_nominal": round(gfl / FP64_NOMINAL_GFLOPS, 4)})
            lockstep["groups"][str(g)] = ent
        recon.recon_set_option(ctx.h, recon.RECON_OPT_BATCH_GROUP, 0)
        lockstep["note"] = ("recon_solve_batch with RECON_OPT_BATCH_GROUP = g: per IRLS iteration "
                            "one Lanczos / eps / sweep launch per group of g solves; the headline "
                            "value runs the independent slots (g = 0), measured faster")

    # ---- T2 maps of the reconstructed series (recon_t2fit), timed alone with events
    t2_map = torch.empty(tuple(outs[0].shape[1:]), dtype=torch.float32, device=dev)
    t2_reps = 20
    for _ in range(3):
        recon.recon_t2fit(ctx.h, outs[0], w.times_ms, t2_map)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(t2_reps):
        recon.recon_t2fit(ctx.h, outs[0], w.times_ms, t2_map)
    e1.record(stream)
    e1.synchronize()
    t2_us = 1000.0 * e0.elapsed_time(e1) / t2_reps
    t2_fg = int(torch.isfinite(t2_map).sum().item())

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return

    # dominant kernel of this library (the largest class of the profiled single solve, timed live
    # on the batch right after the timed region); per-class shares from the profiled solve
    DOM_NOTE = (f"CUDA events around every launch of the class in the last of {DOM_STEPS} plain "
                "single solves of the workload run right after the timed region (L2 flushed "
                "before each); in_batch_avg_launch_us: the same inside the last of "
                f"{DOM_STEPS} steps of the {B}-solve batch, where the launch shares the GPU")
    batch_us = round(1000.0 * batch_dom_ms / batch_dom_n, 3) if batch_dom_n else None
    peak, peak_src = load_peaks()
    if dom in ALU_KINDS:
        work = alg_flops(dom, w)
        achieved = work / (dom_ms / dom_n / 1000.0) / 1e9 if dom_n else 0.0
        roof = {"kernel": dom, "bound": "alu", "achieved": round(achieved, 1),
                "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s (FP64)",
                "frac": round(achieved / FP64_NOMINAL_GFLOPS, 4),
                "peak_source": "nominal FP64 rate of the part (no measured FP64 peak provided)",
                "alg_flops_per_launch": work,
                "avg_launch_us": round(1000.0 * dom_ms / dom_n, 3) if dom_n else None,
                "in_batch_avg_launch_us": batch_us, "timed": DOM_NOTE,
                "traffic": TRAFFIC_BYTES.get(dom)}
    else:
        work = alg_bytes(dom, w, w.n_cg)
        achieved = work / (dom_ms / dom_n / 1000.0) / 1e9 if dom_n else 0.0
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "alg_bytes_per_launch": work,
                "avg_launch_us": round(1000.0 * dom_ms / dom_n, 3) if dom_n else None,
                "in_batch_avg_launch_us": batch_us, "timed": DOM_NOTE,
                "traffic": TRAFFIC_BYTES.get(dom)}
    # the memory-bound CG passes (per-launch time from the profiled solve)
    cg_roof = {}
    for k in ("cg_row_fwd", "cg_col_mask", "cg_row_inv_w",
              "cg_update"):
        ms_k, n_k = prof1.get(k, (0.0, 0))
        if n_k:
            gbs = alg_bytes(k, w, w.n_cg) / (ms_k / n_k / 1000.0) / 1e9
            cg_roof[k] = {"avg_launch_us": round(1000.0 * ms_k / n_k, 3), "achieved_GBs": round(gbs, 1),
                          "frac_of_hbm": round(gbs / peak, 4)}
    launches = args.steps * B * sum(n * KERNELS_PER_SCOPE[k] for k, (ms, n) in mine1.items())
    step_ms_profiled = sum(ms for ms, n in prof1.values())
    phase = {k: {"ms_per_step": round(ms, 4), "launches_per_step": n,
                 "share": round(ms / step_ms_profiled, 4) if step_ms_profiled else None}
             for k, (ms, n) in prof1.items() if n}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
        "single_solve": {"value": single_value, "unit": UNIT,
                         "ms_per_solve": single_max_ms / args.steps,
                         "note": "the plain single-solve path; value above is B concurrent solves"},
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (eigensolver and weight in f64)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": w.T, "P": w.P, "Q": w.Q,
                   "filter": [w.N1, w.N2, w.M], "irls": w.n_irls, "cg": w.n_cg,
                   "lambda": w.lam, "p": w.p, "undersampling": w.R,
                   "batch": B, "parallelism": f"replicas x{world}, {B} concurrent solves per GPU",
                   "l2": "256 MiB buffer written before every timed step (outside the events)"},
        "roofline": roof,
        "roofline_cg_passes": cg_roof,
        "phases": phase,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(B * (bs[0].numel() * 8 + ms[0].numel())),
                "d2h_bytes_per_step": int(B * outs[0].numel() * 8),
                "note": "recon_solve_batch_host on pinned host inputs and outputs (each slot "
                        "copies its own k-space and masks in and its image out on its own "
                        "stream); each step timed like the device-timed ones (L2 flushed before "
                        "it, outside its events) including its host-device copies"},
        "clocks": clocks,
        "lockstep_batch": lockstep,
        "t2fit": {"us_per_map": round(t2_us, 2), "pixels": int(t2_map.numel()),
                  "foreground_pixels": t2_fg, "gauss_newton_steps": 20,
                  "note": "mono-exponential T2 map of one reconstructed series, synchronous call "
                          "(max |x_0| pass + per-pixel fit), outside the timed region"},
    }
    if args.served > 0:
        line["served"] = run_served(args.served, local_rank)
    if args.coil_steps > 0:
        line["coils"] = run_coils(args.coil_steps, local_rank)
    if args.vol_steps > 0:
        line["vol"] = run_vol(args.vol_steps, local_rank)
    if args.p07_steps > 0:
        line["p07"] = run_p07(args.p07_steps, local_rank)
    if args.many > 0:
        line["uneven_batch"] = run_many(args.many, 2, local_rank)
    if args.variant_steps > 0:
        line["variants"] = run_variants(args.variant_steps, local_rank)
    if not args.no_cpu_baseline:
        rate, n, dt, cores = cpu_oracle_rate(w, prob)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} IRLS iterations of {WORKLOAD} (Gram + eigh + weight + {w.n_cg} CG) "
                      f"in {dt:.1f} s, FP64 NumPy; numpy.fft single-threaded, eigh on BLAS threads"}
        one = cpu_oracle_one_thread()
        if one is not None:
            line["cpu_baseline"]["value_1_thread"] = one
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
