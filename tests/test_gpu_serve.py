"""Continuous batching on the GPU: requests arrive while others run, join as memory
frees up, and each result equals the same request run alone (bitwise, and so within
the 1e-5 tolerance)."""
import math

import numpy as np
import pytest

from paper_2502_10640_gb300 import capi, serve, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def make_requests():
    out = []
    sizes = [2048, 3000, 5000, 1500, 8192, 2500, 4000, 6000]
    for k, n in enumerate(sizes):
        R = 5e-6 * (1 + k % 3)
        w = 30.0 + 10 * k
        pos = wl.uniform_sphere(n, R, 700 + k)
        dt = 0.01 / math.sqrt(2 * wl.explosion_rate(n, w, R))
        out.append(serve.ServeRequest(k, 0.002 * k, n, w, dt, 1e-3 * R, 6 + 5 * k, pos))
    return out


def alone(r):
    with capi.Batch(8 << 30) as b:
        s = b.add(r.positions, r.w, r.dt, r.softening)
        b.step(r.steps)
        return b.state(s, r.n)


def test_served_results_equal_the_requests_run_alone():
    reqs = make_requests()
    # room for about three of these bunches at a time: later arrivals must queue and join
    budget = sum(sorted(capi.pp_batch_footprint(r.n) for r in reqs)[-3:])
    srv = serve.Server(budget, block_steps=4)
    try:
        rep = srv.run(reqs)
    finally:
        srv.close()
    assert rep["completed"] == len(reqs) and rep["rejected"] == 0
    assert rep["blocks"] > 3
    assert any(r.queueing > 0 for r in srv.results)          # someone waited for memory
    assert rep["p50_latency_s"] <= rep["p99_latency_s"]
    for res in srv.results:
        r = reqs[res.rid]
        assert res.steps == r.steps
        ref = alone(r)
        for got, want in zip((res.positions, res.velocities, res.accelerations), ref[:3]):
            assert np.array_equal(got, want)
        d = np.linalg.norm(res.positions - ref[0]) / np.linalg.norm(ref[0])
        assert d <= 1e-5


def test_served_trace_at_specified_sizes_against_the_oracle():
    """Requests from the serving trace at the specified sizes (uniform spheres of 4096 to
    524288 macro-electrons, R = 50 um, 1 nC, softening 5 nm), step counts shortened:
    each served result's final accelerations (the Eq. B field at its final positions)
    agree with the oracle's on 256 sampled targets within 1e-5."""
    import oracle
    trace = wl.serve_trace(6)
    reqs = serve.requests_from_trace(trace, n_scale=1.0, steps_scale=0.004)
    srv = serve.Server(150 << 30, block_steps=4)
    try:
        rep = srv.run(reqs)
    finally:
        srv.close()
    assert rep["completed"] == len(reqs)
    qm = -oracle.constants()["e"] / oracle.constants()["me"]
    for res in srv.results:
        r = reqs[res.rid]
        idx = np.linspace(0, r.n - 1, 256).astype(np.int64)
        ref = qm * oracle.fields_subset(res.positions, r.w, r.softening, idx)
        err = np.linalg.norm(res.accelerations[idx] - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (r.n, err)
