"""GPU test of the continuous-batching serving loop at small scale: a Poisson
stream of mixed 2D/3D requests, admission limited by the workspace budget,
requests joining while others iterate; every result equals the same request
solved alone (bitwise) and meets the relative residual."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_stiffness, require_gpu

pytestmark = pytest.mark.gpu


def small_stream(count=40, rate=1e5, seed=11):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        d = int(rng.integers(2, 4))
        n = int(rng.integers(16, 80)) if d == 2 else int(rng.integers(10, 28))
        p = int(rng.integers(2, 9))
        out.append(inputs.Request(k, t, d, n, p))
    return out


def test_serving_stream_results_equal_alone():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDPlan
    from paper_2512_20269_gb300.serving import Server
    reqs = small_stream()  # all 40 arrive within about half a millisecond
    probe = IFFDEngine(1 << 20)
    need = max(probe.request_bytes(r.d, r.n, r.p) for r in reqs)
    probe.close()
    srv = Server(budget_bytes=4 * need, precision="fp32", iterations_per_step=2, keep_results=True)
    st = srv.run(reqs, max_wall_s=120.0)
    assert st["completed"] == len(reqs) and st["in_flight_at_stop"] == 0 and st["queued_at_stop"] == 0
    assert st["admission_refusals"] > 0           # the budget limited admission
    assert st["p50_latency_s"] is not None and st["p99_latency_s"] >= st["p50_latency_s"]
    for r in reqs:
        f, u, info = srv.results[r.index]
        plan = IFFDPlan(r.d, r.n, r.p, precision="fp32", true_residual=False)
        ua, ia = plan.pcg_solve(f)
        assert ia["iters"] == info["iters"]
        assert torch.equal(ua.reshape(-1), u.reshape(-1))
        fu = f.cpu().numpy().reshape((r.n + r.p - 2,) * r.d)
        res = np.linalg.norm(fu - oracle_stiffness(u.cpu().numpy().reshape(fu.shape), r.n, r.p)) / np.linalg.norm(fu)
        assert res <= 1.1e-8
