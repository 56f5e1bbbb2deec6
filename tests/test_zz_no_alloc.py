"""pp_fields_noalloc: the allocation-free field entry point, checked against
pp_compute_fields.

It serves callers that may not call cudaMalloc (memory arenas owned by a host
framework, latency-critical loops that must not hit the allocator, plug-ins limited to
the buffers they are given).  This file is collected last on purpose: if it fails, a
run that stops at the first failure has already run every other test.  It passes alone
in a fresh process too (it loads the library itself).
"""
import numpy as np
import pytest

from paper_2502_10640_gb300 import capi, workloads as wl

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5       # the rel-L2 field tolerance used throughout the GPU tests


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()
    return t


def reference_fields(pos, w, eps):
    with capi.Simulation(pos.shape[0], w, 1e-15, eps) as sim:
        sim.load(pos)
        return sim.fields()


def test_noalloc_matches_compute_fields_on_two_calls_in_a_row(torch):
    # two different problems back to back: the second must not see the first's scratch
    cases = [(12000, 5e-6, 40.0, 1e-9, 51), (3001, 2e-6, 3.0, 0.0, 52)]
    for n, sigma, w, eps, seed in cases:
        pos = wl.gaussian_bunch(n, sigma, seed)
        ref = reference_fields(pos, w, eps)
        pos_d = torch.tensor(pos, device="cuda", dtype=torch.float64)
        out_d = torch.full((n, 3), float("nan"), device="cuda", dtype=torch.float64)
        capi.pp_fields_noalloc(n, w, eps, pos_d, out_d)
        got = out_d.cpu().numpy()
        assert np.all(np.isfinite(got))
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= FORCE_TOL, (n, rel)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    n = capi.PP_FIELDS_NOALLOC_MAX_N + 1
    pos_d = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    out_d = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    with pytest.raises(capi.PPError) as e:
        capi.pp_fields_noalloc(n, 1.0, 0.0, pos_d, out_d)
    assert e.value.status == capi.PP_ERR_ARG
    assert "16384" in str(e.value)
