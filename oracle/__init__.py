"""FP64 CPU oracle for the two-component Shan-Chen D3Q19 evaporation step.

TEST INFRASTRUCTURE ONLY. The product library (the CUDA path behind the C ABI)
never imports, links or runs anything in this package; only the tests, the
smoke check and the CPU-baseline leg of the benchmark do. The numerics live in
``sc_oracle.c`` (plain FP64 loops, arXiv:1701.03637 Sec. II); the analytic laws
of Sec. III live in ``analytic.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsc_oracle.so")
SRC = os.path.join(HERE, "sc_oracle.c")
Q = 19

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, IEEE semantics, optional OpenMP)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "sc_oracle.h"))
    ):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("tau_r", C.c_double), ("tau_b", C.c_double), ("G", C.c_double), ("rho_H", C.c_double),
                ("geometry", C.c_int32), ("sink_z0", C.c_int32), ("sink_layers", C.c_int32),
                ("sphere_cx", C.c_double), ("sphere_cy", C.c_double), ("sphere_cz", C.c_double),
                ("R_H", C.c_double), ("wall_z0", C.c_int32), ("wall_thickness", C.c_int32),
                ("G_rr", C.c_double), ("G_bb", C.c_double)]


class Init(C.Structure):
    _fields_ = [("shape", C.c_int32), ("film_z", C.c_int32),
                ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double), ("radius", C.c_double),
                ("rho_hi", C.c_double), ("rho_lo", C.c_double), ("noise_amp", C.c_double),
                ("seed", C.c_uint64)]


class Diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("mass_r", C.c_double), ("mass_b", C.c_double),
                ("evaporated_mass", C.c_double), ("flux_last", C.c_double),
                ("interface_z", C.c_double), ("radius", C.c_double), ("droplet_sites", C.c_int64)]


def configure(L):
    """Declare the C signatures on a loaded oracle library (the built one, or a
    variant compiled from a modified copy of the source by a test)."""
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    L.orc_create.argtypes = [C.POINTER(Params), C.POINTER(C.c_void_p)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_threads.restype = C.c_int
    L.orc_init_shape.argtypes = [C.c_void_p, C.POINTER(Init)]
    L.orc_init_fields.argtypes = [C.c_void_p, dp, dp]
    L.orc_set_populations.argtypes = [C.c_void_p, dp]
    L.orc_get_populations.argtypes = [C.c_void_p, dp]
    L.orc_step.argtypes = [C.c_void_p, C.c_int64]
    L.orc_fields.argtypes = [C.c_void_p, dp, dp]
    L.orc_profile.argtypes = [C.c_void_p, dp]
    L.orc_diag_get.argtypes = [C.c_void_p, C.POINTER(Diag)]
    L.orc_flux_field.argtypes = [C.c_void_p, dp]
    L.orc_site_class.argtypes = [C.c_void_p, np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")]
    L.orc_lattice_tables.argtypes = [np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS"), dp,
                                     np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")]
    L.orc_feq.argtypes = [C.c_double, dp, dp]
    L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_uniform.restype = C.c_double
    return L


def compile_variant(src_text: str, out_dir: str, name: str = "variant") -> C.CDLL:
    """Compile source text with the oracle's flags into out_dir and load it. Used by
    the mutation tests, which plant a mistake in a copy of sc_oracle.c and check
    that the pins catch it; the built oracle is untouched."""
    src = os.path.join(out_dir, f"{name}.c")
    with open(src, "w") as fh:
        fh.write(src_text)
    for h in ("sc_oracle.h",):
        with open(os.path.join(HERE, h)) as fi, open(os.path.join(out_dir, h), "w") as fo:
            fo.write(fi.read())
    so = os.path.join(out_dir, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", src, "-o", so, "-lm"])
    return configure(C.CDLL(so))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = configure(C.CDLL(LIB_PATH))
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_threads())


def tables():
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q, np.float64)
    opp = np.zeros(Q, np.int32)
    lib().orc_lattice_tables(c, w, opp)
    return c, w, opp


def feq(rho: float, u) -> np.ndarray:
    out = np.zeros(Q, np.float64)
    lib().orc_feq(float(rho), np.ascontiguousarray(u, np.float64), out)
    return out


def splitmix64(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64(seed, k))


def uniform(seed: int, k: int) -> float:
    return float(lib().orc_uniform(seed, k))


_PARAM_DEFAULTS = dict(tau_r=1.0, tau_b=1.0, G=3.6, rho_H=0.03, geometry=0, sink_z0=0, sink_layers=1,
                       sphere_cx=0.0, sphere_cy=0.0, sphere_cz=0.0, R_H=0.0, wall_z0=0, wall_thickness=0,
                       G_rr=0.0, G_bb=0.0)
_INIT_DEFAULTS = dict(shape=0, film_z=0, cx=0.0, cy=0.0, cz=0.0, radius=0.0, rho_hi=1.0, rho_lo=0.03,
                      noise_amp=0.0, seed=0)


class Lattice:
    """One FP64 lattice. ``params`` is a dict with the fields of ``Params``."""

    def __init__(self, params: dict, library=None):
        self._L = library if library is not None else lib()
        p = dict(_PARAM_DEFAULTS)
        p.update({k: v for k, v in params.items() if k in dict(Params._fields_)})
        self.params = p
        self.shape = (p["nz"], p["ny"], p["nx"])
        self.n = p["nx"] * p["ny"] * p["nz"]
        self._p = Params(**p)
        h = C.c_void_p()
        rc = self._L.orc_create(C.byref(self._p), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle: invalid parameters ({rc})")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.orc_destroy(h)
            self._h = None

    def init_shape(self, init: dict) -> None:
        i = dict(_INIT_DEFAULTS)
        i.update({k: v for k, v in init.items() if k in dict(Init._fields_)})
        rc = self._L.orc_init_shape(self._h, C.byref(Init(**i)))
        if rc != 0:
            raise MemoryError("oracle init failed")

    def init_fields(self, rho_r: np.ndarray, rho_b: np.ndarray) -> None:
        self._L.orc_init_fields(self._h, np.ascontiguousarray(rho_r, np.float64).ravel(),
                              np.ascontiguousarray(rho_b, np.float64).ravel())

    def set_populations(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, np.float64).reshape(2 * Q * self.n)
        self._L.orc_set_populations(self._h, f)

    def populations(self) -> np.ndarray:
        out = np.zeros(2 * Q * self.n, np.float64)
        self._L.orc_get_populations(self._h, out)
        return out.reshape(2, Q, *self.shape)

    def step(self, n: int = 1) -> None:
        self._L.orc_step(self._h, int(n))

    def fields(self):
        rr = np.zeros(self.n, np.float64)
        rb = np.zeros(self.n, np.float64)
        self._L.orc_fields(self._h, rr, rb)
        return rr.reshape(self.shape), rb.reshape(self.shape)

    def profile(self) -> np.ndarray:
        out = np.zeros(self.params["nz"], np.float64)
        self._L.orc_profile(self._h, out)
        return out

    def diagnostics(self) -> dict:
        d = Diag()
        self._L.orc_diag_get(self._h, C.byref(d))
        return {k: getattr(d, k) for k, _ in Diag._fields_}

    def flux_field(self) -> np.ndarray:
        out = np.zeros(3 * self.n, np.float64)
        self._L.orc_flux_field(self._h, out)
        return out.reshape(3, *self.shape)

    def site_class(self) -> np.ndarray:
        out = np.zeros(self.n, np.int8)
        self._L.orc_site_class(self._h, out)
        return out.reshape(self.shape)
