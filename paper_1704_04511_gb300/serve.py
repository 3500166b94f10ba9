"""Continuous-batching request loop over recon_submit / recon_poll.

Requests (reconstructions of different grid sizes, frame counts and filter supports) arrive over
time; each one is admitted as soon as a request slot is free and its workspace fits the
context's memory budget, runs on its own stream overlapping the others, and its latency is
measured from arrival to completion. All arithmetic runs in librecon.so; this module only
schedules calls.
"""

from __future__ import annotations

import collections
import dataclasses
import time

from . import recon


@dataclasses.dataclass
class Request:
    arrival_s: float           # arrival time relative to the start of the run
    kspace: object             # device tensor (T, P, Q) complex64 or (T, P, Q, 2) bfloat16
    masks: object              # device tensor (T, P, Q) uint8
    out: object                # device tensor (T, P, Q) complex64, receives the image series
    filt: tuple                # (N1, N2, M)
    lam: float
    p: float
    irls: int
    cg: int
    submitted_s: float = -1.0
    done_s: float = -1.0

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class Server:
    """Admits requests into the context's request slots and polls them to completion."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_inflight: int = 8):
        if not 1 <= max_inflight <= 16:
            raise ValueError("max_inflight must be in 1..16")
        self.ctx = recon.Context(device, mem_budget_bytes)
        self.max_inflight = max_inflight

    def close(self):
        self.ctx.close()

    def run(self, requests: list, idle_sleep_s: float = 20e-6) -> dict:
        """Serve every request (arrival times relative to now). Returns latency statistics."""
        order = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting = collections.deque()
        inflight = {}
        t0 = time.perf_counter()
        busy_refusals = 0
        while order or waiting or inflight:
            now = time.perf_counter() - t0
            progressed = False
            while order and order[0].arrival_s <= now:
                waiting.append(order.popleft())
            while waiting and len(inflight) < self.max_inflight:
                rq = waiting[0]
                ticket = recon.recon_submit(self.ctx.h, rq.kspace, rq.masks, rq.filt, rq.lam,
                                            rq.p, rq.irls, rq.cg, rq.out)
                if ticket is None:          # no slot or budget free: wait for a completion
                    busy_refusals += 1
                    break
                rq.submitted_s = time.perf_counter() - t0
                inflight[ticket] = rq
                waiting.popleft()
                progressed = True
            for ticket in list(inflight):
                if recon.recon_poll(self.ctx.h, ticket):
                    rq = inflight.pop(ticket)
                    rq.done_s = time.perf_counter() - t0
                    progressed = True
            if not progressed:
                if order and not waiting and not inflight:
                    time.sleep(max(0.0, min(order[0].arrival_s - now, 1e-3)))
                else:
                    time.sleep(idle_sleep_s)
        makespan = time.perf_counter() - t0
        lat = sorted(r.latency_s for r in requests)

        def pct(q):
            return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]

        iters = sum(r.irls for r in requests)
        return {"requests": len(requests), "p50_ms": 1000.0 * pct(0.50),
                "p99_ms": 1000.0 * pct(0.99), "max_ms": 1000.0 * lat[-1],
                "makespan_s": makespan, "irls_iters_per_s": iters / makespan,
                "busy_refusals": busy_refusals}
