"""Resident small-N stepping: all steps of a pp_step call in one cooperative launch, a
grid-wide barrier between steps and the staged sources bulk-copied after it.  Checked against the FP64 oracle (runs of Velocity Verlet,
Eq. G/H, on the Eq. B forces), against the per-launch kernels, for bitwise reproducibility
(independent of how steps are grouped into calls and of checkpoints), and for its bounded
barrier wait."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_10640_gb300 import capi, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


# Single FP32 staging unless a test says otherwise: most tests here are about the
# resident kernel's single-staging forms, which PP_POS_AUTO (the default) would leave
# for hi/lo staging on inputs with very close pairs.
SINGLE = capi.PP_POS_SINGLE


def run(pos, vel, w, eps, dt, steps, resident, chunks=None, positions=SINGLE):
    n = pos.shape[0]
    with capi.Simulation(n, w, dt, eps, positions=positions) as sim:
        sim.set_option(capi.PP_OPT_RESIDENT, resident)
        sim.load(pos, vel)
        active = sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE)
        for k in (chunks or [steps]):
            sim.step(k)
        p, v, a, step, _ = sim.state()
    assert step == steps
    return p, v, a, active


def dt_for(n, w, radius, courant=0.02):
    return courant / math.sqrt(2 * wl.explosion_rate(n, w, radius))


# both CTA sizes (256 threads below N = 3072, 512 from there), odd and even N, one and
# several source chunks per thread, up to the largest N that fits shared memory
SIZES = [1, 2, 3, 63, 64, 65, 511, 1000, 1025, 3001, 3072, 4096, 8192, 12288]


@pytest.mark.parametrize("n", SIZES)
def test_resident_run_matches_oracle(n):
    radius = 3e-6
    pos = wl.gaussian_bunch(n, radius, seed=900 + n)
    vel = wl.gaussian_bunch(n, 2e3, seed=950 + n)
    w, eps = 4.0, 1e-9
    dt = dt_for(n, w, radius)
    steps = 6
    p, v, a, active = run(pos, vel, w, eps, dt, steps, capi.PP_RESIDENT_ON)
    assert active == 1
    pr, vr, ar = oracle.vv_run(pos, vel, None, w, eps, dt, steps)
    if n == 1:
        assert np.all(a == 0.0) and np.array_equal(v, vel)
        assert rel(p, pr) <= 1e-15 and rel(v, vr) <= 1e-15
        return
    assert rel(p - pos, pr - pos) <= TOL
    assert rel(v - vel, vr - vel) <= TOL
    assert rel(a, ar) <= TOL


def test_resident_and_per_launch_kernels_agree():
    n = 3001
    pos = wl.uniform_sphere(n, 5e-6, seed=71)
    dt = dt_for(n, 10.0, 5e-6)
    on = run(pos, None, 10.0, 2e-9, dt, 25, capi.PP_RESIDENT_ON)
    off = run(pos, None, 10.0, 2e-9, dt, 25, capi.PP_RESIDENT_OFF)
    assert on[3] == 1 and off[3] == 0
    for x, y in zip(on[:3], off[:3]):
        assert rel(x, y) <= TOL


def test_resident_is_bitwise_reproducible_across_call_grouping_and_checkpoints():
    n = 2500
    pos = wl.gaussian_bunch(n, 2e-6, seed=72)
    dt = dt_for(n, 3.0, 2e-6)
    one = run(pos, None, 3.0, 0.0, dt, 30, capi.PP_RESIDENT_AUTO)
    again = run(pos, None, 3.0, 0.0, dt, 30, capi.PP_RESIDENT_AUTO)
    grouped = run(pos, None, 3.0, 0.0, dt, 30, capi.PP_RESIDENT_AUTO, chunks=[1, 7, 2, 20])
    assert one[3] == 1
    for x, y, z in zip(one[:3], again[:3], grouped[:3]):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    with capi.Simulation(n, 3.0, dt, 0.0, positions=SINGLE) as sim:
        sim.load(pos)
        sim.step(11)
        state = sim.state()
    with capi.Simulation(n, 3.0, dt, 0.0, positions=SINGLE) as sim:
        sim.set_state(*state)
        sim.step(19)
        resumed = sim.state()
    for x, y in zip(one[:3], resumed[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n", [700, 5000])
def test_resident_weighted_run_matches_oracle_and_per_launch(n):
    """Per-particle weights (each source term scaled by w_j / W): both CTA sizes, against
    the oracle (which takes weights natively) and against the per-launch kernels."""
    radius = 4e-6
    pos = wl.uniform_sphere(n, radius, seed=960 + n)
    w = 30.0 * (0.5 + 3.5 * wl.uniform(961 + n, 3, n))
    eps = 1e-3 * radius
    dt = dt_for(n, float(w.mean()), radius)
    steps = 12
    out = {}
    for mode in (capi.PP_RESIDENT_AUTO, capi.PP_RESIDENT_OFF):
        with capi.Simulation(n, 30.0, dt, eps, positions=SINGLE) as sim:
            sim.set_option(capi.PP_OPT_RESIDENT, mode)
            sim.set_weights(w)
            sim.load(pos)
            assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == (mode == capi.PP_RESIDENT_AUTO)
            sim.step(steps)
            out[mode] = sim.state()[:3]
    pr, vr, ar = oracle.vv_run(pos, np.zeros_like(pos), None, w, eps, dt, steps)
    p, v, a = out[capi.PP_RESIDENT_AUTO]
    assert rel(p - pos, pr - pos) <= TOL and rel(v, vr) <= TOL and rel(a, ar) <= TOL
    for x, y in zip(out[capi.PP_RESIDENT_AUTO], out[capi.PP_RESIDENT_OFF]):
        assert rel(x, y) <= TOL


@pytest.mark.parametrize("n", [1500, 4099, 6144])
def test_resident_split_positions_on_close_pairs(n):
    """Hi/lo staging in the resident kernel (both CTA sizes, up to the largest N whose
    two staged copies fit shared memory): on a 1 nm-softened ball whose closest pairs sit
    ~1e3 times closer than its radius, where single FP32 staging loses ~3e-5, the run
    stays within 1e-5 of the oracle."""
    radius, w, eps = 20e-6, 10.0, 1e-9
    pos = wl.uniform_sphere(n, radius, seed=7 + n)
    dt = dt_for(n, w, radius)
    steps = 4
    with capi.Simulation(n, w, dt, eps, positions=capi.PP_POS_SPLIT) as sim:
        sim.load(pos)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1
        sim.step(steps)
        p, v, a, step, _ = sim.state()
    pr, vr, ar = oracle.vv_run(pos, np.zeros_like(pos), None, w, eps, dt, steps)
    assert step == steps
    assert rel(a, ar) <= TOL
    assert rel(v, vr) <= TOL
    assert rel(p - pos, pr - pos) <= TOL


def test_resident_compensated_fold():
    """PP_ACC_KAHAN on the resident kernel: the resident kernel keeps all its partial sums
    in compensated FP32 in both accumulation modes, so the runs are bitwise equal, at
    one tile per thread (N = 3000) and at four (N = 12288), and within 1e-5 of the
    oracle's fields."""
    n = 3000
    pos = wl.gaussian_bunch(n, 2e-6, seed=80)
    dt = dt_for(n, 2.0, 2e-6)
    out = {}
    for acc in (capi.PP_ACC_FP64FOLD, capi.PP_ACC_KAHAN):
        with capi.Simulation(n, 2.0, dt, 1e-9, acc=acc, positions=SINGLE) as sim:
            sim.load(pos)
            assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1
            sim.step(7)
            out[acc] = sim.state()[:3]
    for x, y in zip(out[capi.PP_ACC_FP64FOLD], out[capi.PP_ACC_KAHAN]):
        assert np.array_equal(x, y)
    n = 12288
    pos = wl.gaussian_bunch(n, 3e-6, seed=81)
    dt = dt_for(n, 2.0, 3e-6)
    acc_out = {}
    for acc in (capi.PP_ACC_FP64FOLD, capi.PP_ACC_KAHAN):
        with capi.Simulation(n, 2.0, dt, 1e-9, acc=acc, positions=SINGLE) as sim:
            sim.load(pos)
            assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1
            sim.step(2)
            acc_out[acc] = sim.state()[2]
    ar = oracle.vv_run(pos, np.zeros_like(pos), None, 2.0, 1e-9, dt, 2)[2]
    for acc, a in acc_out.items():
        assert rel(a, ar) <= TOL, acc
    assert rel(acc_out[capi.PP_ACC_KAHAN], acc_out[capi.PP_ACC_FP64FOLD]) <= 1e-12


def test_resident_paper_lattice_without_softening():
    """The 16^3 cube lattice of Sec. 2.1 (eps = 0: the self pair is skipped by the floor on
    s, a coincident pair contributes zero), 20 steps of dt = 1e-13 s, against the oracle."""
    b = wl.PAPER_LATTICE
    pos = b.positions()
    pos[100] = pos[7]                 # a coincident pair
    p, v, a, active = run(pos, None, b.w, 0.0, b.dt, 20, capi.PP_RESIDENT_AUTO)
    assert active == 1
    pr, vr, ar = oracle.vv_run(pos, np.zeros_like(pos), None, b.w, 0.0, b.dt, 20)
    assert rel(p - pos, pr - pos) <= TOL
    assert rel(v, vr) <= TOL
    assert rel(a, ar) <= TOL


def test_resident_selection_rules():
    pos = wl.gaussian_bunch(3000, 2e-6, seed=73)
    with capi.Simulation(3000, 1.0, 1e-15, 1e-9, positions=SINGLE) as sim:
        sim.load(pos)
        assert sim.get_option(capi.PP_OPT_RESIDENT) == capi.PP_RESIDENT_AUTO
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1
        sim.set_option(capi.PP_OPT_RESIDENT, capi.PP_RESIDENT_OFF)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0
        sim.set_option(capi.PP_OPT_RESIDENT, capi.PP_RESIDENT_AUTO)
        sim.set_option(capi.PP_OPT_ACC, capi.PP_ACC_KAHAN)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1          # compensated form
        sim.set_option(capi.PP_OPT_ACC, capi.PP_ACC_FP64_FULL)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0          # FP64 pair math
        sim.set_option(capi.PP_OPT_ACC, capi.PP_ACC_FP64FOLD)
        sim.set_option(capi.PP_OPT_POSITIONS, capi.PP_POS_SPLIT)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1          # hi/lo form
        sim.set_option(capi.PP_OPT_POSITIONS, capi.PP_POS_SINGLE)
        sim.set_option(capi.PP_OPT_VARIANT, capi.variants().index("f32x2.fold64.t64r1k128"))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1          # same staging
        sim.set_option(capi.PP_OPT_VARIANT, capi.variants().index("f32.fold64.t128r2k128"))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0          # float4 staging
        sim.set_option(capi.PP_OPT_VARIANT, -1)
        sim.set_weights(np.full(3000, 1.0))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1          # weighted form
        sim.set_option(capi.PP_OPT_POSITIONS, capi.PP_POS_SPLIT)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0          # weighted hi/lo: per launch
        sim.set_weights(None)
        sim.set_option(capi.PP_OPT_ACC, capi.PP_ACC_KAHAN)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0          # compensated hi/lo: per launch
        sim.set_option(capi.PP_OPT_ACC, capi.PP_ACC_FP64FOLD)
        with pytest.raises(capi.PPError) as e:
            sim.set_option(capi.PP_OPT_RESIDENT, 3)
        assert e.value.status == capi.PP_ERR_ARG
    with capi.Simulation(12288, 1.0, 1e-15, 1e-9, positions=SINGLE) as sim:
        sim.load(wl.gaussian_bunch(12288, 2e-6, seed=74))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1          # the largest that fits
    with capi.Simulation(6145, 1.0, 1e-15, 1e-9, positions=capi.PP_POS_SPLIT) as sim:
        sim.load(wl.gaussian_bunch(6145, 2e-6, seed=79))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0          # hi/lo does not fit
    with capi.Simulation(12289, 1.0, 1e-15, 1e-9, positions=SINGLE) as sim:
        sim.set_option(capi.PP_OPT_RESIDENT, capi.PP_RESIDENT_ON)
        sim.load(wl.gaussian_bunch(12289, 2e-6, seed=75))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0          # does not fit


@pytest.mark.parametrize("steps", [1, 5])
def test_resident_barrier_wait_reports_timeout_and_context_recovers(steps):
    """CTA 0 withholds its first barrier arrival: every CTA's bounded wait runs out,
    the call returns PP_ERR_TIMEOUT (no fault, no hang) and a reload makes the context
    usable again."""
    n = 3000
    pos = wl.gaussian_bunch(n, 2e-6, seed=76)
    with capi.Simulation(n, 1.0, 1e-15, 1e-9, positions=SINGLE) as sim:
        sim.set_option(capi.PP_OPT_TIMEOUT_NS, 20_000_000)
        sim.load(pos)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1
        sim.set_option(capi.PP_OPT_TEST_SKIP_COPY, 1)
        with pytest.raises(capi.PPError) as e:
            sim.step(steps)
        assert e.value.status == capi.PP_ERR_TIMEOUT
        with pytest.raises(capi.PPError) as e:
            sim.step(1)
        assert e.value.status == capi.PP_ERR_STATE
        sim.load(pos)
        sim.step(3)
        p, v, a, step, _ = sim.state()
    pr, vr, ar = oracle.vv_run(pos, np.zeros_like(pos), None, 1.0, 1e-9, 1e-15, 3)
    assert step == 3 and rel(a, ar) <= TOL


def test_autotune_keeps_small_n_steps_resident():
    """At small N the autotuner only times variants whose staging layout the resident
    kernel reads, so after tuning the steps still run resident and the results stay
    within tolerance of the oracle."""
    n = 1500
    pos = wl.gaussian_bunch(n, 2e-6, seed=77)
    dt = dt_for(n, 2.0, 2e-6)
    with capi.Simulation(n, 2.0, dt, 1e-9, positions=SINGLE) as sim:
        sim.load(pos)
        res = sim.autotune()
        assert res["candidates"] >= 2
        assert res["variant_name"].startswith(("f32x2.", "f32x2cl"))
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 1
        sim.step(5)
        a = sim.state()[2]
    ar = oracle.vv_run(pos, np.zeros_like(pos), None, 2.0, 1e-9, dt, 5)[2]
    assert rel(a, ar) <= TOL


def test_resident_calls_longer_than_one_launch():
    """A call of more steps than one cooperative launch takes (4096) is split into several
    launches; the staging parity carries across them: 9000 steps in one call, in calls of
    4500, and in calls of 1000 agree bitwise."""
    n = 200
    pos = wl.gaussian_bunch(n, 1e-6, seed=78)
    dt = dt_for(n, 1.0, 1e-6, courant=0.002)
    one = run(pos, None, 1.0, 1e-9, dt, 9000, capi.PP_RESIDENT_AUTO)
    two = run(pos, None, 1.0, 1e-9, dt, 9000, capi.PP_RESIDENT_AUTO, chunks=[4500, 4500])
    many = run(pos, None, 1.0, 1e-9, dt, 9000, capi.PP_RESIDENT_AUTO, chunks=[1000] * 9)
    assert one[3] == 1
    for x, y, z in zip(one[:3], two[:3], many[:3]):
        assert np.array_equal(x, y) and np.array_equal(x, z)
