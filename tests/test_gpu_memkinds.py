"""Where caller arrays live: host memory through the copy engine (PP_MEM_HOST), device
memory (PP_MEM_DEVICE) and mapped page-locked host memory read and written by the kernels
themselves (PP_MEM_HOST_MAPPED) give bitwise the same results; buffers that are not mapped
page-locked memory, or that run past their allocation, are refused on the host before any
kernel could touch them."""
import numpy as np
import pytest

from paper_2502_10640_gb300 import capi, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def _pinned(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t


def _device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


N = 5003          # several 1024-particle pads, a ragged tail


def _bunch():
    pos = wl.gaussian_bunch(N, 4e-6, seed=501)
    vel = wl.gaussian_bunch(N, 1e3, seed=502)
    return pos, vel


@pytest.mark.parametrize("kind", ["host", "device", "mapped"])
def test_load_fields_steps_state_agree_bitwise(kind):
    pos, vel = _bunch()
    out = {}
    for k in ("host", kind):
        cv = {"host": lambda a: a.copy(), "device": _device, "mapped": _pinned}[k]
        with capi.Simulation(N, 7.0, 2e-15, 1e-9) as sim:
            sim.load(cv(pos), cv(vel))
            E = cv(np.zeros((N, 3)))
            sim.fields(E)
            sim.step(7)
            bufs = [cv(np.zeros((N, 3))) for _ in range(3)]
            _, _, _, step, frame = capi.pp_get_state(sim.ctx, *bufs)
            # round trip: set the state back from the same kind of buffers and step on
            sim.set_state(*bufs, step, frame)
            sim.step(3)
            fin = [cv(np.zeros((N, 3))) for _ in range(3)]
            capi.pp_get_state(sim.ctx, *fin)
        host = lambda t: t.cpu().numpy() if hasattr(t, "cpu") else t
        out[k] = [host(E)] + [host(b) for b in bufs] + [host(b) for b in fin]
    assert step == 7
    for a, b in zip(out["host"], out[kind]):
        assert np.array_equal(a, b)


def test_mapped_check_refuses_what_the_kernels_must_not_touch():
    import torch
    pinned = torch.empty(1 << 17, dtype=torch.float64, pin_memory=True)   # 1 MiB
    base = pinned.data_ptr()
    capi.pp_check_mapped(base, pinned.numel() * 8)                      # the whole tensor
    capi.pp_check_mapped(base + 8 * 1000, 8 * 3000)                      # a range inside it
    pageable = np.zeros(1 << 17)
    with pytest.raises(capi.PPError) as e:
        capi.pp_check_mapped(pageable.ctypes.data, pageable.nbytes)
    assert e.value.status == capi.PP_ERR_ARG
    device = torch.zeros(1 << 17, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.PPError) as e:
        capi.pp_check_mapped(device.data_ptr(), 8 * device.numel())
    assert e.value.status == capi.PP_ERR_ARG
    # a range that starts inside a page-locked allocation and runs 1 GiB past its end
    with pytest.raises(capi.PPError) as e:
        capi.pp_check_mapped(base + 8 * 1000, 1 << 30)
    assert e.value.status == capi.PP_ERR_ARG
    with pytest.raises(capi.PPError):
        capi.pp_check_mapped(base, 0)


def test_mapped_kind_with_pageable_memory_is_refused_before_any_kernel():
    pos, _ = _bunch()
    lib = capi.load()
    with capi.Simulation(N, 7.0, 2e-15, 1e-9) as sim:
        st = lib.pp_load_particles(sim.ctx, pos.ctypes.data, None, capi.PP_MEM_HOST_MAPPED)
        assert st == capi.PP_ERR_ARG
        sim.load(pos)                                     # the context stays usable
        E = np.empty((N, 3))
        assert lib.pp_compute_fields(sim.ctx, E.ctypes.data, capi.PP_MEM_HOST_MAPPED) == capi.PP_ERR_ARG
        assert lib.pp_compute_fields(sim.ctx, E.ctypes.data, 3) == capi.PP_ERR_ARG
        assert lib.pp_get_state(sim.ctx, E.ctypes.data, None, None, None, None, -1) == capi.PP_ERR_ARG
        sim.fields()


def test_batch_accepts_every_kind_and_refuses_others():
    pos, vel = _bunch()
    lib = capi.load()
    with capi.Batch(8 << 30) as b:
        s0 = b.add(pos, 7.0, 2e-15, 1e-9, vel)
        slot = capi.ctypes.c_int(-1)
        pp = _pinned(pos)
        pv = _pinned(vel)
        st = lib.pp_batch_add(b.b, N, 7.0, 2e-15, 1e-9, pp.data_ptr(), pv.data_ptr(),
                              capi.PP_MEM_HOST_MAPPED, capi.ctypes.byref(slot))
        assert st == capi.PP_OK
        assert lib.pp_batch_add(b.b, N, 7.0, 2e-15, 1e-9, pos.ctypes.data, None, 5,
                                capi.ctypes.byref(slot)) == capi.PP_ERR_ARG
        b.step(4)
        a = b.state(s0, N)
        c = b.state(slot.value, N)
        for x, y in zip(a[:3], c[:3]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("kind", ["device", "mapped"])
def test_set_state_refuses_non_finite_device_side_input(kind):
    """The one-pass state import checks finiteness on the device: a NaN velocity in a
    device or mapped buffer is refused with PP_ERR_ARG and a reload recovers."""
    pos, vel = _bunch()
    conv = {"device": _device, "mapped": _pinned}[kind]
    with capi.Simulation(N, 7.0, 2e-15, 1e-9) as sim:
        sim.load(pos, vel)
        p, v, a, step, frame = sim.state()
        v[123, 1] = np.nan
        with pytest.raises(capi.PPError) as e:
            sim.set_state(conv(p), conv(v), conv(a), step, frame)
        assert e.value.status == capi.PP_ERR_ARG
        with pytest.raises(capi.PPError) as e:
            sim.step(1)
        assert e.value.status == capi.PP_ERR_STATE
        sim.load(pos, vel)
        sim.step(2)
