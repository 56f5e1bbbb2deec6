"""Batch contexts (many bunches, one persistent launch per step) vs the oracle, and the
batching guarantees: a bunch's result is bitwise the same alone and in any mix, with or
without CUDA graphs, and when bunches join or leave between step blocks."""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bunch(n, kind, scale, w, eps_frac, seed, courant=0.01):
    pos = wl.gaussian_bunch(n, scale, seed) if kind == "g" else wl.uniform_sphere(n, scale, seed)
    dt = courant / math.sqrt(2 * wl.explosion_rate(n, w, scale))
    return {"pos": pos, "w": w, "eps": eps_frac * scale, "dt": dt, "n": n}


BUNCHES = [bunch(700, "g", 2e-6, 5.0, 1e-3, 61), bunch(1600, "s", 5e-6, 50.0, 2e-3, 62),
           bunch(3000, "g", 3e-6, 20.0, 1e-3, 63), bunch(5001, "s", 8e-6, 200.0, 1e-3, 64)]
BIG = 64 << 30


def test_batch_runs_match_oracle():
    steps = 30
    with capi.Batch(BIG) as b:
        slots = [b.add(x["pos"], x["w"], x["dt"], x["eps"]) for x in BUNCHES]
        b.step(steps)
        for x, s in zip(BUNCHES, slots):
            p, v, a, k = b.state(s, x["n"])
            assert k == steps
            pr, vr, ar = oracle.vv_run(x["pos"], np.zeros_like(x["pos"]), None, x["w"], x["eps"],
                                       x["dt"], steps)
            assert rel(p - x["pos"], pr - x["pos"]) <= TOL
            assert rel(v, vr) <= TOL
            assert rel(a, ar) <= TOL
            d = b.diagnostics(s, with_pe=True)
            dr = oracle.diagnostics(pr, vr, x["w"])
            assert abs(d["rms_radius"] / dr["rms_radius"] - 1) <= TOL
            assert abs(d["ke"] / dr["ke"] - 1) <= TOL
            assert abs(d["pe"] / oracle.potential_energy(pr, x["w"], x["eps"]) - 1) <= TOL


def _run(members, steps, graph_block=0, add_order=None):
    out = {}
    with capi.Batch(BIG, graph_block=graph_block) as b:
        order = add_order or list(range(len(members)))
        slots = {}
        for i in order:
            x = members[i]
            slots[i] = b.add(x["pos"], x["w"], x["dt"], x["eps"])
        b.step(steps)
        for i, s in slots.items():
            out[i] = b.state(s, members[i]["n"])
    return out


def test_bunch_is_bitwise_the_same_alone_and_in_the_mix():
    steps = 12
    mix = _run(BUNCHES, steps)
    for i in range(len(BUNCHES)):
        alone = _run([BUNCHES[i]], steps)[0]
        for x, y in zip(alone[:3], mix[i][:3]):
            assert np.array_equal(x, y)
    shuffled = _run(BUNCHES, steps, add_order=[3, 1, 0, 2])
    for i in range(len(BUNCHES)):
        for x, y in zip(shuffled[i][:3], mix[i][:3]):
            assert np.array_equal(x, y)


def test_graph_blocks_are_bitwise_equal_to_plain_launches():
    a = _run(BUNCHES[:2], 20, graph_block=0)
    b = _run(BUNCHES[:2], 20, graph_block=8)
    for i in a:
        for x, y in zip(a[i][:3], b[i][:3]):
            assert np.array_equal(x, y)


def test_join_and_leave_between_step_blocks():
    x0, x1, x2 = BUNCHES[0], BUNCHES[1], BUNCHES[2]
    with capi.Batch(BIG, graph_block=4) as b:
        s0 = b.add(x0["pos"], x0["w"], x0["dt"], x0["eps"])
        s1 = b.add(x1["pos"], x1["w"], x1["dt"], x1["eps"])
        b.step(5)
        s2 = b.add(x2["pos"], x2["w"], x2["dt"], x2["eps"])     # joins late
        b.step(3)
        b.remove(s0)                                             # leaves
        b.step(6)
        late = b.state(s2, x2["n"])
        early = b.state(s1, x1["n"])
        assert b.info()["active"] == 2
        assert late[3] == 9 and early[3] == 14
    ref_late = _run([x2], 9)[0]
    ref_early = _run([x1], 14)[0]
    for got, ref in ((late, ref_late), (early, ref_early)):
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x, y)


def test_admission_by_memory_budget_and_slot_reuse():
    x0, x1 = BUNCHES[0], BUNCHES[3]
    f0 = capi.pp_batch_footprint(x0["n"])
    f1 = capi.pp_batch_footprint(x1["n"])
    assert f1 > f0 > 9 * 8 * x0["n"]
    with capi.Batch(f0 + f1 - 1) as b:
        s0 = b.add(x0["pos"], x0["w"], x0["dt"], x0["eps"])
        with pytest.raises(capi.PPError) as e:
            b.add(x1["pos"], x1["w"], x1["dt"], x1["eps"])
        assert e.value.status == capi.PP_ERR_NOMEM
        assert b.info() == {"active": 1, "bytes_used": f0, "budget": f0 + f1 - 1}
        b.remove(s0)
        s1 = b.add(x1["pos"], x1["w"], x1["dt"], x1["eps"])
        assert s1 == s0                                          # the freed slot is reused
        assert b.info()["bytes_used"] == f1


def test_hard_ball_in_a_mix_meets_the_field_tolerance():
    """A uniform ball of 40000 particles with softening 1e-4 R (the batched workload's
    rule), whose closest pairs sit ~1e3 times closer than its radius, in a mix: the
    default staging rule moves it off single staging (to guarded or hi/lo staging)
    from its own positions, its initial accelerations (the Eq. B field of the added
    positions) are within 1e-5 of the oracle, and it steps bitwise the same alone and
    in the mix."""
    n, R, w = 40000, 20e-6, 10.0
    hard = bunch(n, "s", R, w, 1e-4, 47)
    members = BUNCHES[:2] + [hard]
    with capi.Batch(BIG) as b:
        slots = [b.add(x["pos"], x["w"], x["dt"], x["eps"]) for x in members]
        assert b.get_option(capi.PP_OPT_POSITIONS) == capi.PP_POS_AUTO
        assert b.get_option(capi.PP_OPT_POSITIONS, slots[2]) in (capi.PP_POS_GUARDED,
                                                                  capi.PP_POS_SPLIT)
        a0 = b.state(slots[2], n)[2]
        b.step(4)
        mix = b.state(slots[2], n)
    assert rel(a0, oracle.accel(hard["pos"], w, hard["eps"])) <= TOL
    alone = _run([hard], 4)[0]
    for x, y in zip(alone[:3], mix[:3]):
        assert np.array_equal(x, y)


def test_hi_lo_staged_batch_runs_match_oracle():
    """Every bunch on hi/lo staging (PP_OPT_POSITIONS = PP_POS_SPLIT): 256-target blocks
    and half-size tiles of the batch kernel, against the oracle's runs."""
    steps = 12
    with capi.Batch(BIG, positions=capi.PP_POS_SPLIT) as b:
        slots = [b.add(x["pos"], x["w"], x["dt"], x["eps"]) for x in BUNCHES]
        for s in slots:
            assert b.get_option(capi.PP_OPT_POSITIONS, s) == capi.PP_POS_SPLIT
        b.step(steps)
        for x, s in zip(BUNCHES, slots):
            p, v, a, k = b.state(s, x["n"])
            pr, vr, ar = oracle.vv_run(x["pos"], np.zeros_like(x["pos"]), None, x["w"], x["eps"],
                                       x["dt"], steps)
            assert rel(p - x["pos"], pr - x["pos"]) <= TOL
            assert rel(v, vr) <= TOL
            assert rel(a, ar) <= TOL


def test_guarded_batch_runs_match_oracle():
    """Every bunch on guarded staging (PP_OPT_POSITIONS = PP_POS_GUARDED): single-staging
    pair loop in 512-target blocks, close-pair and self-pair tiles summed with hi/lo
    separations; against the oracle's runs."""
    steps = 12
    with capi.Batch(BIG, positions=capi.PP_POS_GUARDED) as b:
        slots = [b.add(x["pos"], x["w"], x["dt"], x["eps"]) for x in BUNCHES]
        for s in slots:
            assert b.get_option(capi.PP_OPT_POSITIONS, s) == capi.PP_POS_GUARDED
        b.step(steps)
        for x, s in zip(BUNCHES, slots):
            p, v, a, k = b.state(s, x["n"])
            pr, vr, ar = oracle.vv_run(x["pos"], np.zeros_like(x["pos"]), None, x["w"], x["eps"],
                                       x["dt"], steps)
            assert rel(p - x["pos"], pr - x["pos"]) <= TOL
            assert rel(v, vr) <= TOL
            assert rel(a, ar) <= TOL


def test_every_kernel_shape_gives_bitwise_the_same_results_and_the_autotuner_picks_one():
    """The compiled shapes (threads per CTA, register budget, unrolling) change no
    addition order, so a mix of guarded, single and hi/lo bunches steps bitwise
    identically in each; the autotuner keeps one of them and leaves the states
    untouched."""
    members = BUNCHES[:3]
    names = capi.batch_shapes()
    assert len(names) >= 4
    results = []
    for k in range(len(names)):
        with capi.Batch(BIG) as b:
            b.set_option(capi.PP_OPT_VARIANT, k)
            assert b.get_option(capi.PP_OPT_VARIANT) == k
            b.set_option(capi.PP_OPT_POSITIONS, capi.PP_POS_GUARDED)
            slots = [b.add(members[0]["pos"], members[0]["w"], members[0]["dt"],
                           members[0]["eps"])]
            b.set_option(capi.PP_OPT_POSITIONS, capi.PP_POS_SINGLE)
            slots.append(b.add(members[1]["pos"], members[1]["w"], members[1]["dt"],
                               members[1]["eps"]))
            b.set_option(capi.PP_OPT_POSITIONS, capi.PP_POS_SPLIT)
            slots.append(b.add(members[2]["pos"], members[2]["w"], members[2]["dt"],
                               members[2]["eps"]))
            b.step(6)
            results.append([b.state(s, x["n"]) for s, x in zip(slots, members)])
    for other in results[1:]:
        for got, ref in zip(other, results[0]):
            for x, y in zip(got[:3], ref[:3]):
                assert np.array_equal(x, y)
    with capi.Batch(BIG) as b:
        slots = [b.add(x["pos"], x["w"], x["dt"], x["eps"]) for x in members]
        before = [b.state(s, x["n"]) for s, x in zip(slots, members)]
        res = b.autotune()
        assert res["candidates"] == len(names) and res["ms_per_pass"] > 0
        assert b.get_option(capi.PP_OPT_VARIANT) == res["shape"]
        after = [b.state(s, x["n"]) for s, x in zip(slots, members)]
        for got, ref in zip(after, before):
            for x, y in zip(got[:3], ref[:3]):
                assert np.array_equal(x, y)
        b.step(6)
        tuned = [b.state(s, x["n"]) for s, x in zip(slots, members)]
    with capi.Batch(BIG) as b:
        slots = [b.add(x["pos"], x["w"], x["dt"], x["eps"]) for x in members]
        b.step(6)
        plain = [b.state(s, x["n"]) for s, x in zip(slots, members)]
    for got, ref in zip(tuned, plain):
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x, y)


def test_batch_rejects_bad_input():
    with capi.Batch(BIG) as b:
        bad = np.zeros((10, 3))
        bad[2, 2] = np.inf
        with pytest.raises(capi.PPError) as e:
            b.add(bad, 1.0, 1e-15, 0.0)
        assert e.value.status == capi.PP_ERR_ARG
        assert b.info()["active"] == 0 and b.info()["bytes_used"] == 0
        with pytest.raises(capi.PPError) as e:
            b.remove(3)
        assert e.value.status == capi.PP_ERR_ARG


def test_batch_bounded_wait_reports_timeout():
    """A withheld tile copy in the persistent batch kernel: the step returns PP_ERR_TIMEOUT
    (no fault, no hang), the bunches' states are reported unspecified, and the batch accepts
    and steps new bunches afterwards."""
    x = BUNCHES[1]
    with capi.Batch(BIG) as b:
        b.set_option(capi.PP_OPT_TIMEOUT_NS, 20_000_000)
        s0 = b.add(x["pos"], x["w"], x["dt"], x["eps"])
        b.set_option(capi.PP_OPT_TEST_SKIP_COPY, 1)
        with pytest.raises(capi.PPError) as e:
            b.step(2)
        assert e.value.status == capi.PP_ERR_TIMEOUT
        with pytest.raises(capi.PPError) as e:
            b.state(s0, x["n"])
        assert e.value.status == capi.PP_ERR_STATE
        b.remove(s0)
        s1 = b.add(x["pos"], x["w"], x["dt"], x["eps"])
        b.step(3)
        got = b.state(s1, x["n"])
    ref = _run([x], 3)[0]
    for a, c in zip(got[:3], ref[:3]):
        assert np.array_equal(a, c)
