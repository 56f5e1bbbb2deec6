"""Guarded staging on spatially sorted sources (the tile-box test of pp_order.cu and
tile_boxed) against the FP64 oracle, through the C ABI.

Each force pass sorts the staged sources along a Morton curve, tests each (target, tile)
against the tile's bounding box and sums the tiles that may hold a close pair with hi/lo
separations.  Results must meet the same bars as the per-pair guard: rel-L2 <= 1e-5 and
every particle inside the a-priori single-staging bound; on the hard ball several times
more accurate than single staging; bitwise reproducible across runs, CUDA-graph blocks
and a checkpoint and resume (the order is a function of the positions alone).
"""
import math

import numpy as np
import pytest

import oracle
from tests._bounds import field_error_bound
from paper_2502_10640_gb300 import capi, workloads as wl

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
K_E = oracle.constants()["k"] * oracle.constants()["e"]
GUARDED = capi.PP_POS_GUARDED


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def box_variants():
    names = capi.variants()
    out = [i for i, nm in enumerate(names) if nm.startswith("f32x2bguard.")]
    assert len(out) >= 3
    return out


def weighted_box_variants():
    names = capi.variants()
    out = [i for i, nm in enumerate(names) if nm.startswith("f32x2wbguard.")]
    assert len(out) >= 1
    return out


def fields_with(pos, w, eps, variant=None, acc=None, positions=GUARDED):
    with capi.Simulation(pos.shape[0], w, 1e-15, eps, acc=acc, positions=positions) as sim:
        if variant is not None:
            sim.set_option(capi.PP_OPT_VARIANT, variant)
        sim.load(pos)
        E = sim.fields()
        if variant is not None:
            assert sim.get_option(capi.PP_OPT_VARIANT) == variant
        return E


def check(E, ref, pos, w, eps, idx=None):
    assert np.all(np.isfinite(E))
    r = rel_l2(E, ref)
    assert r <= FORCE_TOL, r
    idx = np.arange(pos.shape[0]) if idx is None else idx
    bound = field_error_bound(pos, w, eps, idx, K_E)
    err = np.linalg.norm(E[idx] - ref[idx], axis=1)
    assert float(np.max(err / bound)) <= 1.0
    return r


# ragged sizes around the 256- and 512-source tiles, one source, and a multi-tile ball
@pytest.mark.parametrize("n", [1, 2, 3, 255, 257, 511, 1023, 1025, 4099, 9000])
def test_every_box_variant_matches_oracle(n):
    pos = wl.uniform_sphere(n, 5e-6, seed=300 + n)
    eps = 1e-9
    ref = oracle.fields(pos, 10.0, eps)
    for v in box_variants():
        name = capi.variants()[v]
        acc = capi.PP_ACC_KAHAN if ".kahan." in name else capi.PP_ACC_FP64FOLD
        E = fields_with(pos, 10.0, eps, variant=v, acc=acc)
        if n == 1:
            assert np.all(E == 0.0)
            continue
        check(E, ref, pos, 10.0, eps)


@pytest.mark.parametrize("n", [2, 1025, 9000])
def test_weighted_box_variant_matches_oracle(n):
    """Per-particle weights (sources scaled by w_j / W, gathered with the positions) on the
    sorted kernel."""
    pos = wl.uniform_sphere(n, 5e-6, seed=400 + n)
    wts = 10.0 * (0.5 + wl.uniform(93, 3, n))
    eps = 1e-9
    ref = oracle.fields(pos, wts, eps)
    for v in weighted_box_variants():
        with capi.Simulation(n, 10.0, 1e-15, eps, positions=GUARDED) as sim:
            sim.set_option(capi.PP_OPT_VARIANT, v)
            sim.set_weights(wts)
            sim.load(pos)
            E = sim.fields()
            assert sim.get_option(capi.PP_OPT_VARIANT) == v
        assert np.all(np.isfinite(E))
        assert rel_l2(E, ref) <= FORCE_TOL


def test_box_guard_on_the_hard_ball():
    """The 40000-particle ball with 1 nm softening, where single staging misses 1e-5:
    the tile-box guard meets it and is several times more accurate than single staging."""
    n, R, eps = 40000, 20e-6, 1e-9
    pos = wl.uniform_sphere(n, R, seed=7 + n)
    ref = oracle.fields(pos, 10.0, eps)
    v = capi.variants().index("f32x2bguard.sfold64.t128r4k512s2m4u2")
    E = fields_with(pos, 10.0, eps, variant=v)
    idx = np.linspace(0, n - 1, 4096).astype(np.int64)
    r = rel_l2(E, ref)
    assert r <= FORCE_TOL, r
    bound = field_error_bound(pos, 10.0, eps, idx, K_E)
    assert float(np.max(np.linalg.norm(E[idx] - ref[idx], axis=1) / bound)) <= 1.0
    E1 = fields_with(pos, 10.0, eps, positions=capi.PP_POS_SINGLE)
    assert 4 * r <= rel_l2(E1, ref), (r, rel_l2(E1, ref))


def test_coincident_sources_and_no_softening():
    """Two particles at one place, eps = 0: the pair adds nothing (non-finite check)."""
    pos = wl.gaussian_bunch(3000, 1e-6, seed=34)
    pos[17] = pos[3]
    pos[2999] = pos[0]
    ref = oracle.fields(pos, 1.0, 0.0)
    v = capi.variants().index("f32x2bguard.sfold64.t128r4k256m4u1")
    E = fields_with(pos, 1.0, 0.0, variant=v)
    check(E, ref, pos, 1.0, 0.0)


def test_large_n_default_plan_sorts_and_matches_sampled_oracle():
    """At N = 131072 guarded staging takes the sorted tile-box kernel by default;
    sampled targets against the oracle, and the same fields bitwise on a second run."""
    n, R, eps = 131072, 50e-6, 5e-9
    pos = wl.uniform_sphere(n, R, seed=123)
    names = capi.variants()
    outs = []
    for _ in range(2):
        with capi.Simulation(n, 1.0, 1e-15, eps, positions=GUARDED) as sim:
            sim.load(pos)
            assert names[sim.get_option(capi.PP_OPT_VARIANT)].startswith("f32x2bguard.")
            outs.append(sim.fields())
    assert np.array_equal(outs[0], outs[1])
    idx = np.linspace(0, n - 1, 2048).astype(np.int64)
    ref = oracle.fields_subset(pos, 1.0, eps, idx)
    assert rel_l2(outs[0][idx], ref) <= FORCE_TOL
    bound = field_error_bound(pos, 1.0, eps, idx, K_E)
    assert float(np.max(np.linalg.norm(outs[0][idx] - ref, axis=1) / bound)) <= 1.0


def test_steps_graphs_and_resume_are_bitwise():
    """Per-launch steps on the sorted kernel: with and without CUDA-graph blocks, and
    across a checkpoint and resume, the state is bitwise the same."""
    n, w, eps = 131072, 1.0, 5e-9
    pos0 = wl.uniform_sphere(n, 50e-6, seed=124)
    dt = 0.02 / math.sqrt(2 * wl.explosion_rate(n, w, 50e-6))
    runs = []
    for gb in (0, 4):
        with capi.Simulation(n, w, dt, eps, positions=GUARDED) as sim:
            sim.set_option(capi.PP_OPT_GRAPH_BLOCK, gb)
            sim.load(pos0)
            sim.step(3)
            mid = sim.state()
            sim.step(5)
            runs.append((mid, sim.state()))
    for x, y in zip(runs[0][1][:3], runs[1][1][:3]):
        assert np.array_equal(x, y)
    mid = runs[0][0]
    with capi.Simulation(n, w, dt, eps, positions=GUARDED) as sim:
        sim.set_state(*mid)
        sim.step(5)
        resumed = sim.state()
    for x, y in zip(runs[0][1][:3], resumed[:3]):
        assert np.array_equal(x, y)


def test_box_guard_run_matches_oracle():
    """A softened ball stepped 40 times on the sorted kernel against the oracle's run."""
    n, R, w, eps = 6000, 5e-6, 50.0, 1e-9
    pos0 = wl.uniform_sphere(n, R, seed=36)
    dt = 0.02 / math.sqrt(2 * wl.explosion_rate(n, w, R))
    steps = 40
    p_ref, v_ref, a_ref = oracle.vv_run(pos0, np.zeros_like(pos0), None, w, eps, dt, steps)
    v = capi.variants().index("f32x2bguard.sfold64.t128r4k512s2m4u2")
    with capi.Simulation(n, w, dt, eps, positions=GUARDED) as sim:
        sim.set_option(capi.PP_OPT_VARIANT, v)
        sim.load(pos0)
        assert sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE) == 0
        sim.step(steps)
        p, vel, a, _, _ = sim.state()
    assert rel_l2(p - pos0, p_ref - pos0) <= FORCE_TOL
    assert rel_l2(vel, v_ref) <= FORCE_TOL
    assert rel_l2(a, a_ref) <= FORCE_TOL


def sort_launches(npad):
    """Launches of one spatial sort: bounding box (2), keys, the shared-memory sort of
    2048-key blocks, then per merge size k above 2048 one global step per j >= 2048 and
    one shared-memory pass; gather and tile boxes."""
    nkeys = 2
    while nkeys < npad:
        nkeys *= 2
    L = min(nkeys, 2048)
    count, k = 6, 2 * L
    while k <= nkeys:
        count += int(math.log2(k // L)) + 1
        k *= 2
    return count


@pytest.mark.parametrize("n,mode,sorted_", [(1 << 20, GUARDED, True), (131072, GUARDED, True), (65536, GUARDED, False),
                                             (20000, GUARDED, False),
                                             (1 << 20, capi.PP_POS_SINGLE, False)])
def test_launches_per_pass(n, mode, sorted_):
    """PP_OPT_LAUNCHES_PER_PASS: the force launch, plus the sort's launches where the plan
    sorts (the bench multiplies it by the timed steps)."""
    with capi.Simulation(n, 1.0, 1e-15, 0.0, positions=mode) as sim:
        got = sim.get_option(capi.PP_OPT_LAUNCHES_PER_PASS)
        name = capi.variants()[sim.get_option(capi.PP_OPT_VARIANT)]
    assert name.startswith(("f32x2bguard.", "f32x2wbguard.")) == sorted_, name
    assert got == (1 + sort_launches(n) if sorted_ else 1), (got, name)
    if n == 1 << 20 and sorted_:
        assert got == 61


def test_autotune_under_guarded_staging():
    """The autotuner times the sorted variants with their sort included; its choice keeps
    the state and meets the tolerance on the hard ball."""
    n, R, eps = 40000, 20e-6, 1e-9
    pos = wl.uniform_sphere(n, R, seed=7 + n)
    idx = np.arange(0, n, 37)
    ref = oracle.fields_subset(pos, 10.0, eps, idx)
    with capi.Simulation(n, 10.0, 1e-15, eps, positions=GUARDED) as sim:
        sim.load(pos)
        before = sim.state()
        res = sim.autotune()
        after = sim.state()
        for x, y in zip(before[:3], after[:3]):
            assert np.array_equal(x, y)
        assert res["variant_name"].startswith(("f32x2guard.", "f32x2bguard.")), res
        assert res["candidates"] >= 4
        E = sim.fields()
    assert rel_l2(E[idx], ref) <= FORCE_TOL


def test_box_guard_just_above_a_power_of_two():
    """N = 131073: the sort pads its keys to 262144, the staged array to the next tile;
    sampled targets (the first and last particles included) against the oracle."""
    n, R, eps = 131073, 50e-6, 5e-9
    pos = wl.uniform_sphere(n, R, seed=125)
    with capi.Simulation(n, 1.0, 1e-15, eps, positions=GUARDED) as sim:
        sim.load(pos)
        assert capi.variants()[sim.get_option(capi.PP_OPT_VARIANT)].startswith("f32x2bguard.")
        E = sim.fields()
    idx = np.unique(np.concatenate([np.linspace(0, n - 1, 1024).astype(np.int64),
                                    np.arange(n - 8, n)]))
    ref = oracle.fields_subset(pos, 1.0, eps, idx)
    assert np.all(np.isfinite(E))
    assert rel_l2(E[idx], ref) <= FORCE_TOL
    bound = field_error_bound(pos, 1.0, eps, idx, K_E)
    assert float(np.max(np.linalg.norm(E[idx] - ref, axis=1) / bound)) <= 1.0
