"""The seeded input generators: SplitMix64 against its published output sequence, the
uniform and Gaussian draws' basic statistics, and the structure of the paper's lattice
and of the batch and serving workloads (all on the CPU)."""
import math

import numpy as np

from paper_2502_10640_gb300 import workloads as wl


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 started from state 0 (state advanced by the golden gamma before mixing)
    got = [int(x) for x in wl.splitmix64(np.arange(3, dtype=np.uint64))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_are_in_range_and_streams_differ():
    u = wl.uniform(5, 1, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    v = wl.uniform(5, 2, 200000)
    assert not np.array_equal(u, v)
    assert np.array_equal(u, wl.uniform(5, 1, 200000))


def test_gaussian_bunch_is_centred_with_the_given_sigma():
    pos = wl.gaussian_bunch(100000, 2e-6, seed=9)
    assert pos.shape == (100000, 3) and pos.flags.c_contiguous
    assert np.allclose(pos.mean(axis=0), 0.0, atol=1e-20)
    assert np.allclose(pos.std(axis=0), 2e-6, rtol=0.01)


def test_uniform_sphere_radius_and_density():
    pos = wl.uniform_sphere(100000, 5e-6, seed=10)
    r = np.linalg.norm(pos - pos.mean(axis=0), axis=1)
    assert r.max() <= 5e-6 * (1 + 1e-2)          # re-centring moves the ball by ~R/sqrt(N)
    # uniform density: the fraction inside half the radius is 1/8
    assert abs(np.mean(r < 2.5e-6) - 0.125) < 0.005


def test_paper_lattice_is_cell_centred_with_the_printed_spacing():
    b = wl.PAPER_LATTICE
    pos = b.positions()
    assert pos.shape == (4096, 3)
    xs = np.unique(np.round(pos[:, 0] / 1e-9)) * 1e-9
    assert len(xs) == 16
    assert np.allclose(np.diff(xs), 1e-4 / 16)
    assert math.isclose(xs[0], -1e-4 / 2 + 1e-4 / 32, rel_tol=1e-9)
    assert math.isclose(b.w, 5e16 * (1e-4) ** 3 / 4096, rel_tol=1e-12)


def test_batch_mix_and_serving_trace_shapes():
    mix = wl.batch_mix()
    assert len(mix) == 64
    ns = np.array([b.n for b in mix])
    assert ns.min() >= 1024 and ns.max() <= 131072
    trace = wl.serve_trace(16)
    arrivals = [r.arrival for r in trace]
    assert arrivals == sorted(arrivals) and len(trace) == 16
