"""pp_fields_noalloc: the allocation-free field entry point, checked against the FP64
oracle and against pp_compute_fields.

It serves callers that may not call cudaMalloc (memory arenas owned by a host
framework, latency-critical loops that must not hit the allocator, plug-ins limited to
the buffers they are given).  This file is collected last on purpose: if it fails, a
run that stops at the first failure has already run every other test.  It passes alone
in a fresh process too (it loads the library itself).
"""
import numpy as np
import pytest

import oracle
from tests._bounds import field_error_bound
from paper_2502_10640_gb300 import capi, workloads as wl

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5       # the rel-L2 field tolerance used throughout the GPU tests
K_E = oracle.constants()["k"] * oracle.constants()["e"]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()
    return t


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def reference_fields(pos, w, eps):
    with capi.Simulation(pos.shape[0], w, 1e-15, eps) as sim:
        sim.load(pos)
        return sim.fields()


def noalloc(torch, pos, w, eps):
    n = pos.shape[0]
    pos_d = torch.tensor(pos, device="cuda", dtype=torch.float64)
    out_d = torch.full((n, 3), float("nan"), device="cuda", dtype=torch.float64)
    capi.pp_fields_noalloc(n, w, eps, pos_d, out_d)
    got = out_d.cpu().numpy()
    assert np.all(np.isfinite(got))
    return got


def test_noalloc_matches_compute_fields_on_two_calls_in_a_row(torch):
    # two different problems back to back: the second must not see the first's scratch
    cases = [(12000, 5e-6, 40.0, 1e-9, 51), (3001, 2e-6, 3.0, 0.0, 52)]
    for n, sigma, w, eps, seed in cases:
        pos = wl.gaussian_bunch(n, sigma, seed)
        got = noalloc(torch, pos, w, eps)
        assert rel(got, reference_fields(pos, w, eps)) <= FORCE_TOL, n


@pytest.mark.parametrize("case", ["largest N", "close pairs"])
def test_noalloc_matches_the_oracle_element_by_element(torch, case):
    """At N = PP_FIELDS_NOALLOC_MAX_N (every scratch region at its full extent) and on a
    1 nm-softened ball whose closest pairs sit ~1e3 times closer than its radius: the
    field within 1e-5 of the FP64 oracle in relative L2, every particle inside the
    a-priori bound of hi/lo staging."""
    if case == "largest N":
        n, w, eps = capi.PP_FIELDS_NOALLOC_MAX_N, 25.0, 1e-9
        pos = wl.gaussian_bunch(n, 4e-6, seed=53)
    else:
        n, w, eps = 9000, 10.0, 1e-9
        pos = wl.uniform_sphere(n, 20e-6, seed=7 + n)
    got = noalloc(torch, pos, w, eps)
    ref = oracle.fields(pos, w, eps)
    assert rel(got, ref) <= FORCE_TOL
    bound = field_error_bound(pos, w, eps, np.arange(n), K_E, split=True)
    assert np.all(np.linalg.norm(got - ref, axis=1) <= bound)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    n = capi.PP_FIELDS_NOALLOC_MAX_N + 1
    pos_d = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    out_d = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    with pytest.raises(capi.PPError) as e:
        capi.pp_fields_noalloc(n, 1.0, 0.0, pos_d, out_d)
    assert e.value.status == capi.PP_ERR_ARG
    assert "16384" in str(e.value)
