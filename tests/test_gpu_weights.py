"""Per-particle weights and warm (moving) bunches against the oracle, which takes
per-particle weights natively."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_10640_gb300 import capi, workloads as wl
from tests._bounds import field_error_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def weights(n, seed, lo=0.5, hi=4.0):
    return lo + (hi - lo) * wl.uniform(seed, 3, n)


@pytest.mark.parametrize("n", [777, 5000, 40000])
def test_weighted_fields(n):
    pos = wl.uniform_sphere(n, 10e-6, seed=300 + n)
    w = 20.0 * weights(n, 300 + n)
    eps = 1e-3 * 10e-6
    ref = oracle.fields(pos, w, eps)
    with capi.Simulation(n, 20.0, 1e-15, eps) as sim:
        sim.set_weights(w)
        sim.load(pos)
        E = sim.fields()
    assert rel(E, ref) <= 1e-5
    c = oracle.constants()
    bound = field_error_bound(pos, w.max(), eps, np.arange(0, n, max(1, n // 500)), c["k"] * c["e"])
    err = np.linalg.norm(E - ref, axis=1)[::max(1, n // 500)]
    assert np.all(err <= bound)


def test_weights_set_after_load_recompute_acceleration():
    n = 3000
    pos = wl.gaussian_bunch(n, 3e-6, seed=310)
    w = 5.0 * weights(n, 310)
    ref_a = oracle.accel(pos, w, 1e-8)
    with capi.Simulation(n, 5.0, 1e-15, 1e-8) as sim:
        sim.load(pos)
        sim.set_weights(w)
        _, _, a, step, _ = sim.state()
    assert step == 0 and rel(a, ref_a) <= 1e-5


def test_weighted_warm_run_matches_oracle():
    """Unequal weights and a thermal velocity spread, 40 steps."""
    n, R = 2500, 5e-6
    pos = wl.uniform_sphere(n, R, seed=320)
    w = 50.0 * weights(n, 320)
    vel = wl.gaussian_bunch(n, 2e4, seed=321)            # m/s per coordinate
    eps = 1e-3 * R
    dt = 0.01 / math.sqrt(2 * wl.explosion_rate(n, float(w.mean()), R))
    steps = 40
    pr, vr, ar = oracle.vv_run(pos, vel, None, w, eps, dt, steps)
    with capi.Simulation(n, 50.0, dt, eps) as sim:
        sim.set_weights(w)
        sim.load(pos, vel)
        sim.step(steps)
        p, v, a, _, _ = sim.state()
        d = sim.diagnostics(with_pe=True)
    assert rel(p - pos, pr - pos) <= 1e-5
    assert rel(v - vel, vr - vel) <= 1e-5
    dr = oracle.diagnostics(pr, vr, w)
    assert abs(d["ke"] / dr["ke"] - 1) <= 1e-5
    scale = oracle.constants()["me"] * np.sum(w * np.linalg.norm(vr, axis=1))
    for k in ("px", "py", "pz"):
        assert abs(d[k] - dr[k]) <= 1e-9 * scale
    assert abs(d["pe"] / oracle.potential_energy(pr, w, eps) - 1) <= 1e-5


def test_weight_validation_and_reset():
    n = 100
    pos = wl.gaussian_bunch(n, 1e-6, seed=330)
    with capi.Simulation(n, 1.0, 1e-15, 0.0) as sim:
        bad = np.ones(n)
        bad[7] = -1.0
        with pytest.raises(capi.PPError) as e:
            sim.set_weights(bad)
        assert e.value.status == capi.PP_ERR_ARG
        sim.set_weights(np.full(n, 2.0))
        with pytest.raises(capi.PPError):
            sim.set_option(capi.PP_OPT_ACC, capi.PP_ACC_KAHAN)
        sim.load(pos)
        E2 = sim.fields()
        sim.set_weights(None)                       # back to the common weight 1.0
        E1 = sim.fields()
    assert rel(E2, 2.0 * E1) <= 1e-6
