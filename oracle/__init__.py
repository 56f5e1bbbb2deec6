"""FP64 CPU oracle for the electrostatic PP electron-bunch model (arXiv 2502.10640, Sec. 2.1).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The GPU product path never imports this module.

The arithmetic lives in ``pp_oracle.c`` (plain C, FP64, OpenMP over the target particle);
this file only compiles it with gcc and marshals numpy arrays through ctypes.

Functions (each follows the passage named in its docstring):
  fields(pos, w, eps)                 Eq. B / Eq. E   field E_i [V/m]
  fields_subset(pos, w, eps, idx)     Eq. B / Eq. E   field at selected particles
  accel(pos, w, eps)                  Eq. D / Eq. F   a_i = (q_e/m_e) E_i
  vv_run(pos, vel, acc, w, eps, dt, n) Eq. G, Eq. H   Velocity Verlet
  potential_energy(pos, w, eps)       pairwise Coulomb energy, pairs once
  diagnostics(pos, vel, w)            Eq. I and the moments of Figs. 5-6
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libpp_oracle.so")
_lock = threading.Lock()
_lib = None

DIAG_KEYS = ("rms_radius", "ke", "px", "py", "pz", "emit_x", "x_rms", "x_max",
             "vx_rms", "vx_max", "cx", "cy", "cz")


def build(force: bool = False) -> str:
    """Compile pp_oracle.c into a shared library (gcc, -O2, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    i64p = ctypes.POINTER(ctypes.c_int64)
    for name in ("oracle_const_e", "oracle_const_me", "oracle_const_eps0", "oracle_const_k"):
        getattr(lib, name).restype = ctypes.c_double
        getattr(lib, name).argtypes = []
    lib.oracle_fields_subset.argtypes = [i64, dp, dp, ctypes.c_double, i64, i64p, dp]
    lib.oracle_fields_subset.restype = None
    lib.oracle_fields.argtypes = [i64, dp, dp, ctypes.c_double, dp]
    lib.oracle_fields.restype = None
    lib.oracle_accel.argtypes = [i64, dp, dp, ctypes.c_double, dp]
    lib.oracle_accel.restype = None
    lib.oracle_vv_run.argtypes = [i64, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                  i64, dp]
    lib.oracle_vv_run.restype = None
    lib.oracle_potential_energy.argtypes = [i64, dp, dp, ctypes.c_double]
    lib.oracle_potential_energy.restype = ctypes.c_double
    lib.oracle_diagnostics.argtypes = [i64, dp, dp, dp, dp]
    lib.oracle_diagnostics.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
        return _lib


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (used by tests that plant mistakes)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", "-std=c11", "-o", out_path, src, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class use_library:
    """Context manager: route the module functions to another compiled oracle library."""

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved = _lib
            _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pos(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("positions/velocities must be [N][3]")
    return a


def _weights(w, n: int) -> np.ndarray:
    if np.ndim(w) == 0:
        return np.full(n, float(w), dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.shape != (n,):
        raise ValueError("weights must be a scalar or [N]")
    return w


def constants() -> dict:
    """The oracle's CODATA 2018 constants: e [C], m_e [kg], eps0 [F/m], k = 1/(4 pi eps0)."""
    lib = _load()
    return {"e": lib.oracle_const_e(), "me": lib.oracle_const_me(),
            "eps0": lib.oracle_const_eps0(), "k": lib.oracle_const_k()}


def fields(pos, w, eps: float = 0.0) -> np.ndarray:
    """Eq. B / Eq. E: field [V/m] at every particle from all the others."""
    lib = _load()
    pos = _pos(pos)
    n = pos.shape[0]
    w = _weights(w, n)
    out = np.empty((n, 3), dtype=np.float64)
    lib.oracle_fields(n, _dp(pos), _dp(w), float(eps), _dp(out))
    return out


def fields_subset(pos, w, eps: float, idx) -> np.ndarray:
    """Eq. B / Eq. E at the particles idx (rows of the result follow idx)."""
    lib = _load()
    pos = _pos(pos)
    n = pos.shape[0]
    w = _weights(w, n)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise IndexError("subset index out of range")
    out = np.empty((idx.size, 3), dtype=np.float64)
    lib.oracle_fields_subset(n, _dp(pos), _dp(w), float(eps), idx.size,
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    return out


def accel(pos, w, eps: float = 0.0) -> np.ndarray:
    """Eq. D / Eq. F: acceleration [m/s^2] a_i = (q_e/m_e) E_i."""
    lib = _load()
    pos = _pos(pos)
    n = pos.shape[0]
    w = _weights(w, n)
    out = np.empty((n, 3), dtype=np.float64)
    lib.oracle_accel(n, _dp(pos), _dp(w), float(eps), _dp(out))
    return out


def vv_run(pos, vel, acc, w, eps: float, dt: float, nsteps: int):
    """Eq. G then Eq. H for nsteps steps.  acc=None computes a(r0) first.

    Returns new (pos, vel, acc) arrays; the inputs are not modified.
    """
    lib = _load()
    pos = _pos(pos).copy()
    vel = _pos(vel).copy()
    n = pos.shape[0]
    w = _weights(w, n)
    acc = accel(pos, w, eps) if acc is None else _pos(acc).copy()
    scratch = np.empty_like(pos)
    lib.oracle_vv_run(n, _dp(pos), _dp(vel), _dp(acc), _dp(w), float(eps), float(dt),
                      int(nsteps), _dp(scratch))
    return pos, vel, acc


def potential_energy(pos, w, eps: float = 0.0) -> float:
    """Coulomb potential energy [J], each pair once, softened like the field."""
    lib = _load()
    pos = _pos(pos)
    n = pos.shape[0]
    w = _weights(w, n)
    return float(lib.oracle_potential_energy(n, _dp(pos), _dp(w), float(eps)))


def diagnostics(pos, vel, w) -> dict:
    """Eq. I and the Fig. 5-6 moments; keys in DIAG_KEYS."""
    lib = _load()
    pos = _pos(pos)
    vel = _pos(vel)
    n = pos.shape[0]
    if n == 0:
        raise ValueError("diagnostics need at least one particle")
    w = _weights(w, n)
    out = np.empty(len(DIAG_KEYS), dtype=np.float64)
    lib.oracle_diagnostics(n, _dp(pos), _dp(vel), _dp(w), _dp(out))
    return dict(zip(DIAG_KEYS, out.tolist()))
