"""Continuous-batching serving loop over the C ABI engine (iffd_engine_*).

Requests arrive over time (inputs.serving_requests); the host loop admits
them in arrival order while their workspace fits the engine's device budget
(admission control) and, optionally, while the DoFs in flight stay under a
cap (so that one engine step stays short), allocates each admitted request's
right-hand side and solution on the device, and steps the engine, which initialises newly
admitted requests and advances every active one. Requests that arrive while
others are iterating join at the next step; finished requests free their
workspace for the queue. Per request the loop records the latency from
arrival to completion (queueing included).
"""

from __future__ import annotations

import collections
import time

import numpy as np

from . import IFFDEngine, inputs


class Server:
    def __init__(self, budget_bytes: int, precision: str = "fp32", iterations_per_step: int = 2,
                 rtol: float = 1e-8, rhs_seed: int = 4, keep_results: bool = False,
                 max_inflight_dofs: int | None = None):
        self.engine = IFFDEngine(budget_bytes, precision=precision, rtol=rtol)
        self.k = iterations_per_step
        self.max_inflight_dofs = max_inflight_dofs
        self.rhs_seed = rhs_seed
        self.keep_results = keep_results
        self.results = {}  # request index -> (f, u, info) when keep_results

    def run(self, requests, max_wall_s: float, stop_arrivals_at: float | None = None) -> dict:
        """Serve `requests` (sorted by arrival time) in real time for at most
        `max_wall_s` seconds. Returns latency / throughput statistics."""
        import torch
        eng = self.engine
        queue = collections.deque()
        inflight = {}
        lat, dofs_done, iters = [], 0, []
        refused = 0
        inflight_dofs = 0
        step_s, step_active, step_dofs = [], [], []
        nxt = 0
        start = time.perf_counter()
        last_arrival = requests[-1].t if requests else 0.0
        if stop_arrivals_at is not None:
            last_arrival = min(last_arrival, stop_arrivals_at)
        while True:
            now = time.perf_counter() - start
            while nxt < len(requests) and requests[nxt].t <= now and requests[nxt].t <= last_arrival:
                queue.append(requests[nxt])
                nxt += 1
            while queue:  # FIFO admission while the head fits the budget
                r = queue[0]
                if (self.max_inflight_dofs is not None and inflight
                        and inflight_dofs + r.N > self.max_inflight_dofs):
                    break
                f = inputs.device_rhs(r.N, self.rhs_seed * 1_000_003 + r.index)
                u = torch.empty_like(f)
                rid = eng.submit(r.d, r.n, r.p, f, u)
                if rid is None:
                    refused += 1
                    del f, u
                    break
                inflight[rid] = (r, f, u)
                inflight_dofs += r.N
                queue.popleft()
            if inflight:
                t0 = time.perf_counter()
                step_active.append(len(inflight))
                step_dofs.append(inflight_dofs)
                eng.step(self.k)
                t_done = time.perf_counter() - start
                step_s.append(t_done + start - t0)
                for rid, info in eng.poll():
                    r, f, u = inflight.pop(rid)
                    inflight_dofs -= r.N
                    lat.append(t_done - r.t)
                    dofs_done += r.N
                    iters.append(info["iters"])
                    if self.keep_results:
                        self.results[r.index] = (f, u, info)
            elif nxt < len(requests) and requests[nxt].t <= last_arrival:
                time.sleep(max(0.0, min(requests[nxt].t - now, 0.01)))
            else:
                break
            if time.perf_counter() - start > max_wall_s:
                break
        wall = time.perf_counter() - start
        arrived = nxt
        lat = np.array(lat) if lat else np.zeros(0)
        return {
            "wall_s": wall,
            "arrived": arrived,
            "completed": int(lat.size),
            "in_flight_at_stop": len(inflight),
            "queued_at_stop": len(queue),
            "admission_refusals": refused,
            "dofs_solved": int(dofs_done),
            "dof_per_s": dofs_done / wall if wall > 0 else 0.0,
            "offered_dof_per_s": sum(r.N for r in requests[:arrived]) / max(min(wall, last_arrival), 1e-9),
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_iters": float(np.mean(iters)) if iters else None,
            "steps": len(step_s),
            "mean_step_s": float(np.mean(step_s)) if step_s else None,
            "mean_active": float(np.mean(step_active)) if step_active else None,
            "mean_inflight_dofs": float(np.mean(step_dofs)) if step_dofs else None,
            "max_inflight_dofs": self.max_inflight_dofs,
            "engine": eng.stats(),
        }
