"""ctypes binding of the C ABI in include/pp.h (same function names).

Argument marshalling only: every step of the computation runs in the CUDA library.
Arrays may be numpy arrays (host memory, on_device = 0) or CUDA torch tensors (device
memory, on_device = 1); both must be float64 with shape [N][3].  Non-OK statuses raise
PPError carrying the status and the library's message.  If the compiled library is
missing and cannot be built, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PP_OK = 0
PP_ERR_ARG = -1
PP_ERR_NOMEM = -2
PP_ERR_CUDA = -3
PP_ERR_TIMEOUT = -4
PP_ERR_STATE = -5
STATUS_NAMES = {0: "PP_OK", -1: "PP_ERR_ARG", -2: "PP_ERR_NOMEM", -3: "PP_ERR_CUDA",
                -4: "PP_ERR_TIMEOUT", -5: "PP_ERR_STATE"}

PP_ACC_FP64FOLD = 0
PP_ACC_KAHAN = 1
PP_ACC_FP64_FULL = 2

PP_OPT_ACC = 1
PP_OPT_STREAM = 2
PP_OPT_SPLIT = 3
PP_OPT_GRAPH_BLOCK = 4
PP_OPT_TIMEOUT_NS = 5
PP_OPT_VARIANT = 6
PP_OPT_POSITIONS = 7
PP_OPT_RESIDENT = 8
PP_OPT_RESIDENT_ACTIVE = 9
PP_OPT_POSITIONS_AUTO = 10
PP_OPT_LAUNCHES_PER_PASS = 11

PP_POS_SINGLE = 0
PP_POS_SPLIT = 1
PP_POS_AUTO = 2
PP_POS_GUARDED = 3
PP_FRAME_LEN = 5
PP_OPT_TEST_SKIP_COPY = 99

PP_RESIDENT_OFF = 0
PP_RESIDENT_AUTO = 1
PP_RESIDENT_ON = 2

PP_MEM_HOST = 0
PP_MEM_DEVICE = 1
PP_MEM_HOST_MAPPED = 2


class PPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class pp_tune_result(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("split", ctypes.c_int),
                ("ms_per_pass", ctypes.c_double), ("candidates", ctypes.c_int)]


class pp_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_int64),
                ("rms_radius", ctypes.c_double), ("ke", ctypes.c_double), ("pe", ctypes.c_double),
                ("px", ctypes.c_double), ("py", ctypes.c_double), ("pz", ctypes.c_double),
                ("emit_x", ctypes.c_double), ("x_rms", ctypes.c_double),
                ("x_max", ctypes.c_double), ("vx_rms", ctypes.c_double),
                ("vx_max", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("cz", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_DP = ctypes.c_void_p
_I64 = ctypes.c_int64
_CTX = ctypes.c_void_p

# (name, restype, argtypes) of every exported symbol declared in include/pp.h
SIGNATURES = [
    ("pp_create", ctypes.c_int, [_I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(_CTX)]),
    ("pp_set_option", ctypes.c_int, [_CTX, ctypes.c_int, _I64]),
    ("pp_get_option", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.POINTER(_I64)]),
    ("pp_load_particles", ctypes.c_int, [_CTX, _DP, _DP, ctypes.c_int]),
    ("pp_check_mapped", ctypes.c_int, [ctypes.c_void_p, _I64]),
    ("pp_compute_fields", ctypes.c_int, [_CTX, _DP, ctypes.c_int]),
    ("pp_set_weights", ctypes.c_int, [_CTX, _DP, ctypes.c_int]),
    ("pp_step", ctypes.c_int, [_CTX, _I64]),
    ("pp_diagnostics", ctypes.c_int, [_CTX, ctypes.POINTER(pp_diag), ctypes.c_int]),
    ("pp_get_particles", ctypes.c_int, [_CTX, _DP, _DP, ctypes.c_int]),
    ("pp_get_state", ctypes.c_int, [_CTX, _DP, _DP, _DP, ctypes.POINTER(_I64),
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("pp_set_state", ctypes.c_int, [_CTX, _DP, _DP, _DP, _I64, ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_int]),
    ("pp_get_n", ctypes.c_int, [_CTX, ctypes.POINTER(_I64)]),
    ("pp_staging_check", ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    ("pp_destroy", ctypes.c_int, [_CTX]),
    ("pp_last_error", ctypes.c_char_p, [_CTX]),
    ("pp_version", ctypes.c_char_p, []),
    ("pp_variant_name", ctypes.c_char_p, [ctypes.c_int]),
    ("pp_pairs_per_step", ctypes.c_double, [_I64]),
    ("pp_autotune", ctypes.c_int, [_CTX, ctypes.POINTER(pp_tune_result)]),
    ("pp_batch_footprint", ctypes.c_int, [_I64, ctypes.POINTER(_I64)]),
    ("pp_batch_create", ctypes.c_int, [_I64, ctypes.POINTER(_CTX)]),
    ("pp_batch_set_option", ctypes.c_int, [_CTX, ctypes.c_int, _I64]),
    ("pp_batch_add", ctypes.c_int, [_CTX, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    _DP, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("pp_batch_remove", ctypes.c_int, [_CTX, ctypes.c_int]),
    ("pp_batch_step", ctypes.c_int, [_CTX, _I64]),
    ("pp_batch_get_state", ctypes.c_int, [_CTX, ctypes.c_int, _DP, _DP, _DP, ctypes.POINTER(_I64),
                                          ctypes.c_int]),
    ("pp_batch_diagnostics", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.POINTER(pp_diag),
                                            ctypes.c_int]),
    ("pp_batch_info", ctypes.c_int, [_CTX, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                     ctypes.POINTER(_I64)]),
    ("pp_batch_destroy", ctypes.c_int, [_CTX]),
    ("pp_batch_get_option", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_I64)]),
    ("pp_batch_shape_name", ctypes.c_char_p, [ctypes.c_int]),
    ("pp_batch_autotune", ctypes.c_int, [_CTX, ctypes.POINTER(pp_tune_result)]),
    ("pp_fields_noalloc", ctypes.c_int, [_I64, ctypes.c_double, ctypes.c_double, _DP, _DP, _VP]),
]

PP_FIELDS_NOALLOC_MAX_N = 16384


def library_path() -> str:
    return _build.LIB


def load():
    """Load (building first if needed) the compiled library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, ctx=None):
    if status != PP_OK:
        msg = load().pp_last_error(ctx)
        raise PPError(status, msg.decode() if msg else "")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _arg(x, n: int | None, writable: bool):
    """(pointer, memory kind, keepalive) for a numpy array or a torch tensor: CUDA tensors
    are PP_MEM_DEVICE, pinned CPU tensors (contiguous float64 of the right shape)
    PP_MEM_HOST_MAPPED, everything else PP_MEM_HOST."""
    if x is None:
        return None, PP_MEM_HOST, None
    if _is_torch(x):
        import torch
        if not x.is_cuda:
            if (x.is_pinned() and x.dtype == torch.float64 and x.is_contiguous()
                    and (n is None or tuple(x.shape) == (n, 3))):
                return x.data_ptr(), PP_MEM_HOST_MAPPED, x
            x = x.numpy()
        else:
            if x.dtype != torch.float64 or not x.is_contiguous():
                if writable:
                    raise ValueError("device output arrays must be contiguous float64")
                x = x.to(torch.float64).contiguous()
            if n is not None and tuple(x.shape) not in ((n, 3),):
                raise ValueError(f"expected shape ({n}, 3), got {tuple(x.shape)}")
            torch.cuda.current_stream(x.device).synchronize()
            return x.data_ptr(), PP_MEM_DEVICE, x
    a = x
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        if writable:
            raise ValueError("output arrays must be C-contiguous float64")
        a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape != (n, 3):
        raise ValueError(f"expected shape ({n}, 3), got {a.shape}")
    return a.ctypes.data, PP_MEM_HOST, a


def _same_kind(*ons):
    ons = [o for o in ons if o is not None]
    if len(set(ons)) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ons[0] if ons else 0


# ---- the ABI, function by function --------------------------------------------

def pp_version() -> str:
    return load().pp_version().decode()


def pp_variant_name(index: int):
    name = load().pp_variant_name(int(index))
    return name.decode() if name else None


def variants() -> list[str]:
    """Names of all compiled force-kernel variants, in index order."""
    out = []
    while (name := pp_variant_name(len(out))) is not None:
        out.append(name)
    return out


def pp_pairs_per_step(n: int) -> float:
    return load().pp_pairs_per_step(n)


def pp_create(n: int, w: float, dt: float, softening: float):
    ctx = _CTX()
    _check(load().pp_create(int(n), float(w), float(dt), float(softening), ctypes.byref(ctx)))
    return ctx


def pp_set_option(ctx, key: int, value: int) -> None:
    _check(load().pp_set_option(ctx, int(key), int(value)), ctx)


def pp_get_option(ctx, key: int) -> int:
    v = _I64()
    _check(load().pp_get_option(ctx, int(key), ctypes.byref(v)), ctx)
    return v.value


def pp_staging_check(ctx) -> dict:
    """The last PP_POS_AUTO decision's measured field differences (NaN: not measured)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().pp_staging_check(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return {"single_rel": a.value, "guarded_rel": b.value}


def pp_get_n(ctx) -> int:
    n = _I64()
    _check(load().pp_get_n(ctx, ctypes.byref(n)), ctx)
    return n.value


def pp_load_particles(ctx, pos, vel=None) -> None:
    n = pp_get_n(ctx)
    p, op, k1 = _arg(pos, n, False)
    v, ov, k2 = _arg(vel, n, False)
    on = _same_kind(op, ov if vel is not None else None)
    _check(load().pp_load_particles(ctx, p, v, on), ctx)


def pp_set_weights(ctx, w=None) -> None:
    """Per-particle weights ([N] float64, host array or CUDA tensor); None = equal weights."""
    if w is None:
        _check(load().pp_set_weights(ctx, None, 0), ctx)
        return
    n = pp_get_n(ctx)
    if _is_torch(w) and w.is_cuda:
        import torch
        w = w.to(torch.float64).contiguous()
        if tuple(w.shape) != (n,):
            raise ValueError(f"expected shape ({n},)")
        torch.cuda.current_stream(w.device).synchronize()
        _check(load().pp_set_weights(ctx, w.data_ptr(), 1), ctx)
        return
    a = np.ascontiguousarray(w, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError(f"expected shape ({n},)")
    _check(load().pp_set_weights(ctx, a.ctypes.data, 0), ctx)


def pp_compute_fields(ctx, out=None):
    """Field E [V/m], [N][3]; `out` may be a preallocated numpy array or CUDA tensor."""
    n = pp_get_n(ctx)
    if out is None:
        out = np.empty((n, 3), dtype=np.float64)
    p, on, keep = _arg(out, n, True)
    _check(load().pp_compute_fields(ctx, p, on), ctx)
    return out


def pp_step(ctx, nsteps: int) -> None:
    _check(load().pp_step(ctx, int(nsteps)), ctx)


def pp_diagnostics(ctx, with_pe: bool = True) -> dict:
    d = pp_diag()
    _check(load().pp_diagnostics(ctx, ctypes.byref(d), 1 if with_pe else 0), ctx)
    return d.as_dict()


def pp_get_particles(ctx, pos=None, vel=None):
    n = pp_get_n(ctx)
    if pos is None and vel is None:
        pos = np.empty((n, 3))
        vel = np.empty((n, 3))
    p, op, k1 = _arg(pos, n, True)
    v, ov, k2 = _arg(vel, n, True)
    on = _same_kind(op if pos is not None else None, ov if vel is not None else None)
    _check(load().pp_get_particles(ctx, p, v, on), ctx)
    return pos, vel


def pp_get_state(ctx, pos=None, vel=None, acc=None):
    """(pos, vel, acc, step, frame); frame = (cx, cy, cz, L0, staging) of the FP32 staging."""
    n = pp_get_n(ctx)
    if pos is None and vel is None and acc is None:
        pos, vel, acc = (np.empty((n, 3)) for _ in range(3))
    p, op, k1 = _arg(pos, n, True)
    v, ov, k2 = _arg(vel, n, True)
    a, oa, k3 = _arg(acc, n, True)
    on = _same_kind(*(o for o, x in ((op, pos), (ov, vel), (oa, acc)) if x is not None))
    step = _I64()
    frame = (ctypes.c_double * PP_FRAME_LEN)()
    _check(load().pp_get_state(ctx, p, v, a, ctypes.byref(step), frame, on), ctx)
    return pos, vel, acc, step.value, tuple(frame)


def pp_set_state(ctx, pos, vel, acc, step: int, frame=None) -> None:
    n = pp_get_n(ctx)
    p, op, k1 = _arg(pos, n, False)
    v, ov, k2 = _arg(vel, n, False)
    a, oa, k3 = _arg(acc, n, False)
    on = _same_kind(op, ov, oa)
    if frame is not None and len(frame) != PP_FRAME_LEN:
        raise ValueError(f"frame must hold {PP_FRAME_LEN} values (cx, cy, cz, L0, staging)")
    fr = None if frame is None else (ctypes.c_double * PP_FRAME_LEN)(*[float(x) for x in frame])
    _check(load().pp_set_state(ctx, p, v, a, int(step), fr, on), ctx)


def pp_check_mapped(ptr: int, nbytes: int) -> None:
    """Raise PPError unless the nbytes at address ptr may be passed as PP_MEM_HOST_MAPPED
    (host-side check only; nothing runs on the device)."""
    _check(load().pp_check_mapped(ctypes.c_void_p(int(ptr)), int(nbytes)))


def pp_autotune(ctx) -> dict:
    """Time the fitting kernel variants and j-splits; keep the fastest on ctx."""
    r = pp_tune_result()
    _check(load().pp_autotune(ctx, ctypes.byref(r)), ctx)
    return {"variant": r.variant, "variant_name": pp_variant_name(r.variant), "split": r.split,
            "ms_per_pass": r.ms_per_pass, "candidates": r.candidates}


def pp_destroy(ctx) -> None:
    if ctx:
        _check(load().pp_destroy(ctx))


def pp_fields_noalloc(n: int, w: float, softening: float, pos, out, stream=None) -> None:
    """Field [V/m] of n particles at device positions `pos` into device `out` ([n][3],
    CUDA float64 tensors), using no device allocation (fixed scratch, n <= 16384).

    `stream` is a torch.cuda.Stream (default: the current stream of pos's device)."""
    import torch
    for x in (pos, out):
        if not (_is_torch(x) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
                and tuple(x.shape) == (n, 3)):
            raise ValueError("pos and out must be contiguous CUDA float64 tensors of shape (n, 3)")
    if out.device != pos.device:
        raise ValueError(f"pos is on {pos.device} but out is on {out.device}")
    s = stream if stream is not None else torch.cuda.current_stream(pos.device)
    if s.device != pos.device:
        raise ValueError(f"the stream belongs to {s.device}, the tensors to {pos.device}")
    # the library works on the current device: make it the tensors' device
    with torch.cuda.device(pos.device):
        _check(load().pp_fields_noalloc(int(n), float(w), float(softening), pos.data_ptr(),
                                         out.data_ptr(), s.cuda_stream))


def pp_last_error(ctx=None) -> str:
    m = load().pp_last_error(ctx)
    return m.decode() if m else ""


def pp_batch_footprint(n: int) -> int:
    b = _I64()
    _check(load().pp_batch_footprint(int(n), ctypes.byref(b)))
    return b.value


def batch_shapes() -> list[str]:
    """Names of the compiled batch-kernel shapes (index = PP_OPT_VARIANT of a batch)."""
    out, k = [], 0
    while True:
        nm = load().pp_batch_shape_name(k)
        if nm is None:
            return out
        out.append(nm.decode())
        k += 1


class Batch:
    """Owning wrapper of a batch context (pp_batch_*): many bunches stepped together."""

    def __init__(self, budget_bytes: int, graph_block: int | None = None,
                 positions: int | None = None):
        self.b = _CTX()
        _check(load().pp_batch_create(int(budget_bytes), ctypes.byref(self.b)))
        if graph_block is not None:
            self.set_option(PP_OPT_GRAPH_BLOCK, graph_block)
        if positions is not None:
            self.set_option(PP_OPT_POSITIONS, positions)

    def set_option(self, key: int, value: int):
        _check(load().pp_batch_set_option(self.b, int(key), int(value)))

    def get_option(self, key: int, slot: int = -1) -> int:
        """An option of the batch (slot = -1) or of one bunch (its PP_OPT_POSITIONS)."""
        v = _I64()
        _check(load().pp_batch_get_option(self.b, int(slot), int(key), ctypes.byref(v)))
        return v.value

    def autotune(self) -> dict:
        """Time every compiled shape on the current bunches; keep the fastest."""
        r = pp_tune_result()
        _check(load().pp_batch_autotune(self.b, ctypes.byref(r)))
        return {"shape": r.variant, "shape_name": batch_shapes()[r.variant],
                "ms_per_pass": r.ms_per_pass, "candidates": r.candidates}

    def add(self, pos, w: float, dt: float, softening: float = 0.0, vel=None) -> int:
        n = int(pos.shape[0])
        p, op, k1 = _arg(pos, n, False)
        v, ov, k2 = _arg(vel, n, False)
        on = _same_kind(op, ov if vel is not None else None)
        slot = ctypes.c_int()
        _check(load().pp_batch_add(self.b, n, float(w), float(dt), float(softening), p, v, on,
                                   ctypes.byref(slot)))
        return slot.value

    def remove(self, slot: int):
        _check(load().pp_batch_remove(self.b, int(slot)))

    def step(self, nsteps: int = 1):
        _check(load().pp_batch_step(self.b, int(nsteps)))

    def state(self, slot: int, n: int):
        pos, vel, acc = (np.empty((n, 3)) for _ in range(3))
        step = _I64()
        _check(load().pp_batch_get_state(self.b, int(slot), pos.ctypes.data, vel.ctypes.data,
                                         acc.ctypes.data, ctypes.byref(step), 0))
        return pos, vel, acc, step.value

    def diagnostics(self, slot: int, with_pe: bool = False) -> dict:
        d = pp_diag()
        _check(load().pp_batch_diagnostics(self.b, int(slot), ctypes.byref(d),
                                           1 if with_pe else 0))
        return d.as_dict()

    def info(self) -> dict:
        a, u, g = _I64(), _I64(), _I64()
        _check(load().pp_batch_info(self.b, ctypes.byref(a), ctypes.byref(u), ctypes.byref(g)))
        return {"active": a.value, "bytes_used": u.value, "budget": g.value}

    def close(self):
        if self.b:
            _check(load().pp_batch_destroy(self.b))
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tune_cache_path() -> str:
    return os.environ.get("PP_TUNE_CACHE", os.path.join(_build.BUILD, "autotune.json"))


def _tune_key(n: int, acc: int, positions: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    bucket = 1 << max(0, int(n - 1).bit_length())          # next power of two
    return f"{p.name}|{p.multi_processor_count}|n<={bucket}|acc={acc}|pos={positions}"


class Simulation:
    """Owning wrapper: one context, destroyed with the object or on close().

    tune="cache" applies a cached autotuner choice for this device, N bucket and mode
    (running pp_autotune and storing its choice on a miss, once particles are loaded);
    tune="always" reruns the autotuner at every load; tune=None keeps the built-in plan.
    """

    def __init__(self, n: int, w: float, dt: float, softening: float = 0.0, acc: int | None = None,
                 positions: int | None = None, tune: str | None = None):
        self.ctx = pp_create(n, w, dt, softening)
        self.n = n
        self.acc = PP_ACC_FP64FOLD if acc is None else acc
        self.positions = PP_POS_AUTO if positions is None else positions
        self.tune = tune
        self.tuned = None
        if acc is not None:
            pp_set_option(self.ctx, PP_OPT_ACC, acc)
        if positions is not None:
            pp_set_option(self.ctx, PP_OPT_POSITIONS, positions)

    def _apply_tuning(self):
        import json
        path = _tune_cache_path()
        # keyed by the staging in force (what PP_POS_AUTO decided at this load)
        key = _tune_key(self.n, self.acc, pp_get_option(self.ctx, PP_OPT_POSITIONS))
        cache = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        hit = cache.get(key) if self.tune == "cache" else None
        names = variants()
        if hit and hit.get("variant_name") in names:
            pp_set_option(self.ctx, PP_OPT_VARIANT, names.index(hit["variant_name"]))
            pp_set_option(self.ctx, PP_OPT_SPLIT, 0)
            self.tuned = dict(hit, cached=True)
            return
        res = pp_autotune(self.ctx)
        # the split count is kept only for this N; the cache stores the kernel variant
        cache[key] = {"variant_name": res["variant_name"], "ms_per_pass": res["ms_per_pass"],
                      "n": self.n}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = f"{path}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
        self.tuned = dict(res, cached=False)

    def set_option(self, key, value):
        pp_set_option(self.ctx, key, value)

    def get_option(self, key) -> int:
        return pp_get_option(self.ctx, key)

    def staging_check(self) -> dict:
        return pp_staging_check(self.ctx)

    def load(self, pos, vel=None):
        pp_load_particles(self.ctx, pos, vel)
        if self.tune in ("cache", "always"):
            self._apply_tuning()

    def set_weights(self, w=None):
        pp_set_weights(self.ctx, w)

    def fields(self, out=None):
        return pp_compute_fields(self.ctx, out)

    def step(self, nsteps: int = 1):
        pp_step(self.ctx, nsteps)

    def autotune(self) -> dict:
        return pp_autotune(self.ctx)

    def diagnostics(self, with_pe: bool = True) -> dict:
        return pp_diagnostics(self.ctx, with_pe)

    def particles(self):
        return pp_get_particles(self.ctx)

    def state(self):
        return pp_get_state(self.ctx)

    def set_state(self, pos, vel, acc, step, frame=None):
        pp_set_state(self.ctx, pos, vel, acc, step, frame)

    def close(self):
        if self.ctx:
            pp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
