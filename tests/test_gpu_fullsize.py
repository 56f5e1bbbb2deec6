"""Full-size runs in the benchmark's launch plan, checked where the oracle cannot follow
the whole run: sampled oracle forces on the GPU's own late-time state, the all-FP64 GPU
path (within 1e-12 of the oracle's fields) over the whole run, conservation laws, and the
closed-form expansion of a cold uniform ball.  The two whole-run tests are marked slow
(about 3 and 6 minutes of GPU time)."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_10640_gb300 import capi, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def shell_scale(t, K):
    """s(t) of a cold uniform ball: s'' = K / s^2, s(0) = 1, s'(0) = 0 (no shell crossing)."""
    from scipy.optimize import brentq
    tau = t * math.sqrt(2 * K)
    f = lambda s: math.sqrt(s * (s - 1)) + math.log(math.sqrt(s) + math.sqrt(s - 1)) - tau
    return 1.0 if tau == 0 else brentq(f, 1.0, 1e6, xtol=1e-14)


@pytest.mark.slow
def test_sphere_1m_full_run_both_folds():
    """2^20 particles, R = 50 um, 1 nC, all 500 steps of 2e-14 s, with the FP64 fold and
    with the compensated FP32 fold: at step 500 each run's fields on 4096 sampled targets
    (against all sources, on that run's own state) are within 1e-5 of the oracle, the two
    runs' RMS radii agree within 1e-5, the radius follows the homologous expansion of a
    cold uniform ball (continuum limit, sampling noise ~1e-3), and momentum stays at the
    FP32 summation noise level."""
    b = wl.SPHERE_1M
    pos0 = b.positions()
    idx = np.sort(np.unique((wl.uniform(79, 0, 4096) * b.n).astype(np.int64)))
    K = wl.explosion_rate(b.n, b.w, b.scale)
    s = shell_scale(b.steps * b.dt, K)
    assert s > 20
    radius = {}
    for acc in (capi.PP_ACC_FP64FOLD, capi.PP_ACC_KAHAN):
        with capi.Simulation(b.n, b.w, b.dt, b.eps, acc=acc) as sim:
            sim.load(pos0)
            d0 = sim.diagnostics(with_pe=False)
            sim.step(b.steps)
            d1 = sim.diagnostics(with_pe=False)
            p, v, a, step, _ = sim.state()
            E = sim.fields()
        assert step == b.steps
        radius[acc] = d1["rms_radius"]
        assert abs(d1["rms_radius"] / d0["rms_radius"] / s - 1) < 0.01
        pmag = math.sqrt(d1["px"] ** 2 + d1["py"] ** 2 + d1["pz"] ** 2)
        pscale = oracle.constants()["me"] * b.w * np.linalg.norm(v, axis=1).sum()
        assert pmag <= 1e-6 * pscale
        assert rel(E[idx], oracle.fields_subset(p, b.w, b.eps, idx)) <= 1e-5, acc
    assert abs(radius[capi.PP_ACC_KAHAN] / radius[capi.PP_ACC_FP64FOLD] - 1) <= 1e-5


@pytest.mark.slow
def test_gaussian_65536_full_run_against_the_fp64_gpu_path():
    """All 2000 steps of the N = 65536 Gaussian bunch with FP32 pair math (default
    configuration) and with the all-FP64 path (itself within 1e-12 of the oracle's
    fields): RMS radius within 1e-5, velocities and displacements within 1e-5 in
    relative L2; energy and momentum conserved; sampled oracle forces on the final
    state within 1e-5."""
    b = wl.GAUSSIAN_65536
    pos0 = b.positions()
    out = {}
    for acc in (capi.PP_ACC_FP64FOLD, capi.PP_ACC_FP64_FULL):
        with capi.Simulation(b.n, b.w, b.dt, b.eps, acc=acc) as sim:
            sim.load(pos0)
            d0 = sim.diagnostics(with_pe=True)
            sim.step(b.steps)
            d1 = sim.diagnostics(with_pe=acc == capi.PP_ACC_FP64FOLD)
            p, v, a, step, _ = sim.state()
            E = sim.fields() if acc == capi.PP_ACC_FP64FOLD else None
        assert step == b.steps
        out[acc] = (d0, d1, p, v, E)
    (d0a, d1a, pa, va, Ea), (d0b, d1b, pb, vb, _) = out[capi.PP_ACC_FP64FOLD], out[capi.PP_ACC_FP64_FULL]
    assert abs(d1a["rms_radius"] / d1b["rms_radius"] - 1) <= 1e-5
    assert rel(va, vb) <= 1e-5
    assert rel(pa - pos0, pb - pos0) <= 1e-5
    e0 = d0a["ke"] + d0a["pe"]
    e1 = d1a["ke"] + d1a["pe"]
    assert d1a["ke"] > 0.3 * d0a["pe"]               # a large part of the energy converted
    assert abs(e1 / e0 - 1) < 1e-3
    pmag = math.sqrt(d1a["px"] ** 2 + d1a["py"] ** 2 + d1a["pz"] ** 2)
    assert pmag <= 1e-6 * oracle.constants()["me"] * b.w * np.linalg.norm(va, axis=1).sum()
    idx = np.sort(np.unique((wl.uniform(80, 0, 512) * b.n).astype(np.int64)))
    assert rel(Ea[idx], oracle.fields_subset(pa, b.w, b.eps, idx)) <= 1e-5


def test_paper_lattice_experiment_series_matches_oracle():
    """The 16^3 lattice of Sec. 2.1 at dt = 1e-13 s: the emittance and moment series of the
    experiment driver against the oracle run for the first 1000 steps."""
    from paper_2502_10640_gb300 import experiments
    run = experiments.run_lattice(16, 1e-13, 1e-10, records=4)
    assert run["steps"] == 1000 and len(run["series"]["emit_x"]) == 5
    assert run["resident"]                       # the small-N default path ran
    assert abs(run["energy_drift"]) <= 1e-7      # measured: 8e-9
    b = wl.PAPER_LATTICE
    pos = b.positions()
    p, v, a = pos, np.zeros_like(pos), None
    for k in range(4):
        p, v, a = oracle.vv_run(p, v, a, b.w, 0.0, b.dt, 250)
        d = oracle.diagnostics(p, v, b.w)
        for key in ("emit_x", "x_rms", "vx_rms", "rms_radius"):
            got = run["series"][key][k + 1]
            assert abs(got / d[key] - 1) <= 1e-5, (k, key, got, d[key])
        assert abs(run["series"]["x_max"][k + 1] / d["x_max"] - 1) <= 1e-6


def test_lattice_energy_error_is_second_order_in_dt():
    """Velocity Verlet (Eq. G/H) is second order: on the 16^3 lattice run to 1e-8 s, the
    relative change of kinetic + Coulomb energy grows by about 100 when dt grows tenfold
    (measured: 2.1e-4 at dt = 1e-11 s, 2.4e-2 at 1e-10 s)."""
    from paper_2502_10640_gb300 import experiments
    fine = experiments.run_lattice(16, 1e-11, 1e-8, records=2)
    coarse = experiments.run_lattice(16, 1e-10, 1e-8, records=2)
    ratio = coarse["energy_drift"] / fine["energy_drift"]
    assert 70.0 <= ratio <= 140.0, ratio
