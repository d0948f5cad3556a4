"""Build and load the sc_lbm CUDA library (sm_103a) and declare its C ABI.

Every numeric step of the method runs in the library's kernels; this module only
compiles, loads and marshals. Loading fails loudly when the library is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsc_lbm.so")
SOURCES = ["sc_lbm.cu"]
HEADERS = ["sc_kernels.cuh", "sc_batch.cuh", "sc_ncomp.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "sc_lbm.h")]
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library for sm_103a into the package's _build/ folder."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(f) for f in _inputs())
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    vscript = os.path.join(BUILD_DIR, "exports.map")
    with open(vscript, "w") as fh:
        fh.write("{ global: sc_*; local: *; };\n")
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    # device code optimisation split over the host's cores (one translation unit)
    cmd = [_nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", f"--split-compile={min(os.cpu_count() or 1, 16)}",
           "-Xcompiler", "-fPIC", "-shared",
           "-I", INCLUDE, "-Xlinker", f"--version-script={vscript}",
           *[os.path.join(CSRC, s) for s in SOURCES], "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("tau_r", C.c_double), ("tau_b", C.c_double), ("G", C.c_double), ("rho_H", C.c_double),
                ("geometry", C.c_int32), ("sink_z0", C.c_int32), ("sink_layers", C.c_int32),
                ("sphere_cx", C.c_double), ("sphere_cy", C.c_double), ("sphere_cz", C.c_double),
                ("R_H", C.c_double), ("wall_z0", C.c_int32), ("wall_thickness", C.c_int32),
                ("storage", C.c_int32), ("tile", C.c_int32), ("zchunk", C.c_int32),
                ("staging", C.c_int32), ("layout", C.c_int32), ("G_rr", C.c_double), ("G_bb", C.c_double)]


class Init(C.Structure):
    _fields_ = [("shape", C.c_int32), ("film_z", C.c_int32),
                ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double), ("radius", C.c_double),
                ("rho_hi", C.c_double), ("rho_lo", C.c_double), ("noise_amp", C.c_double),
                ("seed", C.c_uint64)]


MAX_COMP = 4


class NParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("ncomp", C.c_int32),
                ("tau", C.c_double * MAX_COMP), ("g", (C.c_double * MAX_COMP) * MAX_COMP),
                ("wall_z0", C.c_int32), ("wall_thickness", C.c_int32)]


class Diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("mass_r", C.c_double), ("mass_b", C.c_double),
                ("evaporated_mass", C.c_double), ("flux_last", C.c_double),
                ("interface_z", C.c_double), ("radius", C.c_double), ("droplet_sites", C.c_int64),
                ("status", C.c_int32), ("reserved", C.c_int32)]


# name -> (restype, argtypes): the declarations of include/sc_lbm.h
_VP = C.c_void_p
_SIGS = {
    "sc_last_error": (C.c_char_p, []),
    "sc_lattice_directions": (C.c_int, [_VP, _VP]),
    "sc_tile_list": (C.c_int, [C.POINTER(C.c_int32), _VP, _VP, C.c_int32]),
    "sc_lbm_required_bytes": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_size_t)]),
    "sc_lbm_create": (C.c_int, [C.POINTER(Params), _VP, C.POINTER(_VP)]),
    "sc_lbm_create_ext": (C.c_int, [C.POINTER(Params), _VP, _VP, C.c_size_t, C.POINTER(_VP)]),
    "sc_lbm_destroy": (None, [_VP]),
    "sc_lbm_set_stream": (C.c_int, [_VP, _VP]),
    "sc_lbm_sync": (C.c_int, [_VP]),
    "sc_lbm_init": (C.c_int, [_VP, C.POINTER(Init)]),
    "sc_lbm_init_fields": (C.c_int, [_VP, _VP, _VP]),
    "sc_lbm_step": (C.c_int, [_VP, C.c_int64]),
    "sc_lbm_read_fields": (C.c_int, [_VP, _VP, _VP]),
    "sc_lbm_read_fields_device": (C.c_int, [_VP, _VP, _VP]),
    "sc_lbm_read_populations": (C.c_int, [_VP, _VP]),
    "sc_lbm_write_populations": (C.c_int, [_VP, _VP]),
    "sc_lbm_set_counters": (C.c_int, [_VP, C.c_int64, C.c_double]),
    "sc_lbm_diagnostics": (C.c_int, [_VP, C.POINTER(Diag)]),
    "sc_lbm_profile": (C.c_int, [_VP, _VP]),
    "sc_lbm_flux_profile": (C.c_int, [_VP, _VP]),
    "sc_lbm_diag_bytes": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "sc_lbm_diagnostics_noalloc": (C.c_int, [_VP, _VP]),
    "sc_lbm_launch_info": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "sc_lbm_tune": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "sc_lbm_launch_count": (C.c_int, [_VP, C.c_int64, C.POINTER(C.c_int64)]),
    "sc_lbm_kernel_name": (C.c_char_p, [_VP]),
    "sc_lbm_set_wait": (C.c_int, [_VP, C.c_int64, C.c_int32]),
    "sc_lbm_persist_bands": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int32)]),
    "sc_slab_create": (C.c_int, [C.POINTER(Params), C.c_int32, C.c_int32, _VP, C.POINTER(_VP)]),
    "sc_slab_info": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_size_t)]),
    "sc_slab_pack": (C.c_int, [_VP, C.c_int32, _VP]),
    "sc_slab_unpack": (C.c_int, [_VP, C.c_int32, _VP]),
    "sc_ncomp_create": (C.c_int, [C.POINTER(NParams), _VP, C.POINTER(_VP)]),
    "sc_ncomp_destroy": (None, [_VP]),
    "sc_ncomp_write_populations": (C.c_int, [_VP, _VP]),
    "sc_ncomp_init_fields": (C.c_int, [_VP, _VP]),
    "sc_ncomp_read_populations": (C.c_int, [_VP, _VP]),
    "sc_ncomp_step": (C.c_int, [_VP, C.c_int64]),
    "sc_ncomp_sync": (C.c_int, [_VP]),
    "sc_batch_create": (C.c_int, [C.c_size_t, C.c_int32, _VP, C.POINTER(_VP)]),
    "sc_batch_destroy": (None, [_VP]),
    "sc_batch_add": (C.c_int, [_VP, C.POINTER(Params), C.POINTER(C.c_int32), C.POINTER(_VP)]),
    "sc_batch_lattice": (C.c_int, [_VP, C.c_int32, C.POINTER(_VP)]),
    "sc_batch_remove": (C.c_int, [_VP, C.c_int32]),
    "sc_batch_set_steps": (C.c_int, [_VP, C.c_int32, C.c_int64]),
    "sc_batch_remaining": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int64)]),
    "sc_batch_step": (C.c_int, [_VP, C.c_int64]),
    "sc_batch_configure": (C.c_int, [_VP, C.c_int32, C.c_int32]),
    "sc_batch_tune": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "sc_batch_info": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_size_t),
                                C.POINTER(C.c_size_t), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "sc_batch_sync": (C.c_int, [_VP]),
}


def declared_symbols():
    return sorted(_SIGS)


class ScError(RuntimeError):
    """A library call failed; ``code`` is its SC_E* return value."""

    def __init__(self, msg: str, code: int = 0):
        super().__init__(msg)
        self.code = code


def load(path: str | None = None):
    """Load the compiled library (building it first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            build()
        lib = C.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(rc: int) -> None:
    if rc != 0:
        msg = load().sc_last_error().decode(errors="replace")
        raise ScError(f"sc_lbm error {rc}: {msg}", rc)
