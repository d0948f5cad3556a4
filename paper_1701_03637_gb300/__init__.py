"""GB300 (sm_103a) two-component Shan-Chen D3Q19 lattice Boltzmann step with the
fixed-density evaporation boundary of arXiv:1701.03637.

``Lattice`` wraps one handle of the C ABI declared in ``include/sc_lbm.h``.
PyTorch supplies the device memory (``sc_lbm_create_ext`` on a torch buffer) and
the CUDA stream; every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native
from ._native import Diag, Init, Params, ScError, build, check

Q = 19
STORAGE = {"f32": 0, "f16": 1, "bf16": 2, "f16s": 3}
STAGING = {"auto": 0, "thread": 1, "rows": 2, "persistent": 3}
GEOMETRY = {"periodic": 0, "planar": 1, "sphere": 2}
LAYOUT = {"two": 0, "aa": 1}

__all__ = ["Lattice", "Batch", "ScError", "build", "lattice_directions", "tile_list", "required_bytes", "Q"]

_PARAM_DEFAULTS = dict(tau_r=1.0, tau_b=1.0, G=3.6, rho_H=0.03, geometry=0, sink_z0=0, sink_layers=1,
                       sphere_cx=0.0, sphere_cy=0.0, sphere_cz=0.0, R_H=0.0, wall_z0=0, wall_thickness=0,
                       storage=0, tile=0, zchunk=0, staging=0, layout=0, G_rr=0.0, G_bb=0.0)
_INIT_DEFAULTS = dict(shape=0, film_z=0, cx=0.0, cy=0.0, cz=0.0, radius=0.0, rho_hi=1.0, rho_lo=0.03,
                      noise_amp=0.0, seed=0)


def _lib():
    return _native.load()


def make_params(params: dict) -> Params:
    p = dict(_PARAM_DEFAULTS)
    p.update(params)
    if isinstance(p.get("storage"), str):
        p["storage"] = STORAGE[p["storage"]]
    if isinstance(p.get("geometry"), str):
        p["geometry"] = GEOMETRY[p["geometry"]]
    if isinstance(p.get("layout"), str):
        p["layout"] = LAYOUT[p["layout"]]
    if isinstance(p.get("staging"), str):
        p["staging"] = STAGING[p["staging"]]
    return Params(**{k: p[k] for k, _ in Params._fields_})


def make_init(init: dict) -> Init:
    i = dict(_INIT_DEFAULTS)
    i.update(init)
    return Init(**{k: i[k] for k, _ in Init._fields_})


def lattice_directions():
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q, np.float64)
    check(_lib().sc_lattice_directions(c.ctypes.data, w.ctypes.data))
    return c, w


def tile_list():
    n = C.c_int32()
    tx = np.zeros(16, np.int32)
    ty = np.zeros(16, np.int32)
    check(_lib().sc_tile_list(C.byref(n), tx.ctypes.data, ty.ctypes.data, 16))
    return [(int(tx[k]), int(ty[k])) for k in range(n.value)]


def required_bytes(params: dict) -> int:
    b = C.c_size_t()
    check(_lib().sc_lbm_required_bytes(C.byref(make_params(params)), C.byref(b)))
    return int(b.value)


def _current_stream_handle(device):
    import torch
    return torch.cuda.current_stream(device).cuda_stream


class Lattice:
    """One lattice on the current CUDA device.

    ``params``: dict with the fields of ``sc_params`` (``nx, ny, nz`` required);
    ``storage`` may be "f32", "f16", "bf16" or "f16s", ``geometry`` "periodic",
    "planar" or "sphere", ``layout`` "two" (two population lattices) or "aa" (one
    updated in place, half the memory, the same bits); ``G`` is the cross coupling
    of Eq. (3), ``G_rr``/``G_bb`` optional self couplings (the multiphase model).
    Device memory is a torch uint8 tensor lent to ``sc_lbm_create_ext`` (it must
    outlive the handle, which this object guarantees); the stream is torch's
    current stream unless ``stream`` (a ``torch.cuda.Stream``) is given.
    """

    def __init__(self, params: dict, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._p = make_params(params)
        self.params = {k: getattr(self._p, k) for k, _ in Params._fields_}
        self.nx, self.ny, self.nz = self._p.nx, self._p.ny, self._p.nz
        self.n = self.nx * self.ny * self.nz
        self.shape = (self.nz, self.ny, self.nx)
        nbytes = required_bytes(self.params)
        with torch.cuda.device(self.device):
            self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self._mem.data_ptr()
            aligned = (base + 255) & ~255
            self.stream = stream or torch.cuda.current_stream(self.device)
            h = C.c_void_p()
            check(_lib().sc_lbm_create_ext(C.byref(self._p), C.c_void_p(self.stream.cuda_stream),
                                           C.c_void_p(aligned), C.c_size_t(nbytes), C.byref(h)))
        self._h = h

    @classmethod
    def _member(cls, handle, params: Params, device, stream, owner):
        """A view of a lattice that a Batch owns (its memory is the batch's arena)."""
        self = cls.__new__(cls)
        import torch
        self.torch = torch
        self.device = device
        self._p = params
        self.params = {k: getattr(params, k) for k, _ in Params._fields_}
        self.nx, self.ny, self.nz = params.nx, params.ny, params.nz
        self.n = self.nx * self.ny * self.nz
        self.shape = (self.nz, self.ny, self.nx)
        self.stream = stream
        self._owner = owner
        self._h = handle
        return self

    # ------------------------------------------------------------ lifecycle
    def close(self):
        """Destroy the handle (after its stream has finished) and release its device
        memory to torch's allocator."""
        h = getattr(self, "_h", None)
        if h is not None and h.value and getattr(self, "_owner", None) is None:
            _lib().sc_lbm_destroy(h)
        self._h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self.stream = stream
        check(_lib().sc_lbm_set_stream(self._h, C.c_void_p(stream.cuda_stream)))

    def sync(self):
        check(_lib().sc_lbm_sync(self._h))

    # ------------------------------------------------------------ state
    def init(self, init: dict) -> None:
        check(_lib().sc_lbm_init(self._h, C.byref(make_init(init))))

    def init_fields(self, rho_r, rho_b) -> None:
        rr = np.ascontiguousarray(rho_r, np.float32).reshape(-1)
        rb = np.ascontiguousarray(rho_b, np.float32).reshape(-1)
        assert rr.size == self.n and rb.size == self.n
        check(_lib().sc_lbm_init_fields(self._h, rr.ctypes.data, rb.ctypes.data))

    def step(self, n: int = 1) -> None:
        check(_lib().sc_lbm_step(self._h, int(n)))

    def read_fields(self):
        rr = np.empty(self.n, np.float32)
        rb = np.empty(self.n, np.float32)
        check(_lib().sc_lbm_read_fields(self._h, rr.ctypes.data, rb.ctypes.data))
        return rr.reshape(self.shape), rb.reshape(self.shape)

    def read_fields_into(self, rr_host, rb_host) -> None:
        """Canonical densities into caller host buffers (numpy or pinned torch CPU tensors)."""
        pr = rr_host.data_ptr() if hasattr(rr_host, "data_ptr") else rr_host.ctypes.data
        pb = rb_host.data_ptr() if hasattr(rb_host, "data_ptr") else rb_host.ctypes.data
        check(_lib().sc_lbm_read_fields(self._h, pr, pb))

    def init_fields_from(self, rr_host, rb_host) -> None:
        pr = rr_host.data_ptr() if hasattr(rr_host, "data_ptr") else rr_host.ctypes.data
        pb = rb_host.data_ptr() if hasattr(rb_host, "data_ptr") else rb_host.ctypes.data
        check(_lib().sc_lbm_init_fields(self._h, pr, pb))

    def read_fields_device(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty((2, *self.shape), dtype=torch.float32, device=self.device)
        check(_lib().sc_lbm_read_fields_device(self._h, C.c_void_p(out[0].data_ptr()),
                                               C.c_void_p(out[1].data_ptr())))
        return out

    def read_populations(self) -> np.ndarray:
        f = np.empty(2 * Q * self.n, np.float64)
        check(_lib().sc_lbm_read_populations(self._h, f.ctypes.data))
        return f.reshape(2, Q, *self.shape)

    def write_populations(self, f) -> None:
        f = np.ascontiguousarray(f, np.float64).reshape(-1)
        assert f.size == 2 * Q * self.n
        check(_lib().sc_lbm_write_populations(self._h, f.ctypes.data))

    def set_counters(self, step: int, evaporated_mass: float) -> None:
        check(_lib().sc_lbm_set_counters(self._h, int(step), float(evaporated_mass)))

    def diagnostics(self) -> dict:
        d = Diag()
        check(_lib().sc_lbm_diagnostics(self._h, C.byref(d)))
        return {k: getattr(d, k) for k, _ in Diag._fields_ if k != "reserved"}

    def profile(self) -> np.ndarray:
        out = np.empty(self.nz, np.float64)
        check(_lib().sc_lbm_profile(self._h, out.ctypes.data))
        return out

    def flux_profile(self) -> np.ndarray:
        """Plane means of the relative flux rho^r (U^r - U) of Eqs. (flux) and (velw),
        shape (3, nz) (x, y, z components), computed on the device (tau = 1)."""
        out = np.empty(3 * self.nz, np.float64)
        check(_lib().sc_lbm_flux_profile(self._h, out.ctypes.data))
        return out.reshape(3, self.nz)

    def diag_bytes(self) -> int:
        b = C.c_size_t()
        check(_lib().sc_lbm_diag_bytes(self._h, C.byref(b)))
        return int(b.value)

    def tune(self, trials: int = 3) -> dict:
        """Time every tile shape and z-chunk length on this lattice and keep the fastest
        (the state and bookkeeping are unchanged)."""
        t, z = C.c_int32(), C.c_int32()
        check(_lib().sc_lbm_tune(self._h, int(trials), C.byref(t), C.byref(z)))
        return dict(tile=t.value, zchunk=z.value)

    def launch_count(self, steps: int) -> int:
        """Kernel launches that step(steps) issues in the current configuration."""
        n = C.c_int64()
        check(_lib().sc_lbm_launch_count(self._h, int(steps), C.byref(n)))
        return int(n.value)

    def kernel_name(self) -> str:
        return _lib().sc_lbm_kernel_name(self._h).decode()

    def launch_info(self) -> dict:
        tx, ty, zc, n, st = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
        check(_lib().sc_lbm_launch_info(self._h, C.byref(tx), C.byref(ty), C.byref(zc), C.byref(n), C.byref(st)))
        out = dict(tile_x=tx.value, tile_y=ty.value, zchunk=zc.value, ctas=n.value,
                   staging={1: "thread", 2: "rows", 3: "persistent"}.get(st.value, st.value))
        if out["staging"] == "persistent":
            out["bands"] = self.persist_bands()
        return out

    def persist_bands(self, request: int = -1) -> int:
        """Bands along x of the persistent in-place step: -1 reports the count in use,
        0 restores the automatic count, k >= 1 marches k bands (re-planning the tiles)."""
        b = C.c_int32()
        check(_lib().sc_lbm_persist_bands(self._h, int(request), C.byref(b)))
        return int(b.value)

    def set_wait(self, limit_ns: int, withhold_cta: int = -1) -> None:
        """Time limit of the persistent in-place step's progress waits; withhold_cta >= 0
        makes that CTA withhold its progress reports (a test of the failure path)."""
        check(_lib().sc_lbm_set_wait(self._h, int(limit_ns), int(withhold_cta)))


class Batch:
    """Many lattices advanced together by one persistent launch per time step.

    Members live in a device arena of ``arena_bytes`` that the library allocates;
    ``add`` fails with ``ScError`` (-2) when no free range fits the lattice, which
    is the admission test of a serving loop. Each member is a ``Lattice`` view for
    init, fields and diagnostics; ``step`` advances all members at once.
    """

    def __init__(self, arena_bytes: int, storage="f32", device=None, stream=None):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            b = C.c_void_p()
            check(_lib().sc_batch_create(C.c_size_t(int(arena_bytes)), self.storage,
                                         C.c_void_p(self.stream.cuda_stream), C.byref(b)))
        self._b = b
        self._members = {}

    def close(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            for lat in self._members.values():
                lat._h = None
            self._members = {}
            _lib().sc_batch_destroy(b)
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, params: dict):
        """Admit a lattice; returns (slot, Lattice view)."""
        p = make_params(dict(params, storage=self.storage))
        slot, h = C.c_int32(), C.c_void_p()
        check(_lib().sc_batch_add(self._b, C.byref(p), C.byref(slot), C.byref(h)))
        lat = Lattice._member(h, p, self.device, self.stream, self)
        self._members[slot.value] = lat
        return slot.value, lat

    def lattice(self, slot: int):
        return self._members[slot]

    def remove(self, slot: int) -> None:
        check(_lib().sc_batch_remove(self._b, int(slot)))
        lat = self._members.pop(slot, None)
        if lat is not None:
            lat._h = None

    def set_steps(self, slot: int, steps: int) -> None:
        check(_lib().sc_batch_set_steps(self._b, int(slot), int(steps)))

    def remaining(self, slot: int) -> int:
        v = C.c_int64()
        check(_lib().sc_batch_remaining(self._b, int(slot), C.byref(v)))
        return int(v.value)

    def step(self, n: int = 1) -> None:
        check(_lib().sc_batch_step(self._b, int(n)))

    def configure(self, tile: int = 0, zchunk: int = 0) -> None:
        check(_lib().sc_batch_configure(self._b, int(tile), int(zchunk)))

    def tune(self, trials: int = 3):
        t, z = C.c_int32(), C.c_int32()
        check(_lib().sc_batch_tune(self._b, int(trials), C.byref(t), C.byref(z)))
        return t.value, z.value

    def info(self) -> dict:
        m, it, fb, lf, t, z = C.c_int32(), C.c_int64(), C.c_size_t(), C.c_size_t(), C.c_int32(), C.c_int32()
        check(_lib().sc_batch_info(self._b, C.byref(m), C.byref(it), C.byref(fb), C.byref(lf), C.byref(t),
                                   C.byref(z)))
        return dict(members=m.value, items=it.value, free_bytes=fb.value, largest_free=lf.value, tile=t.value,
                    zchunk=z.value)

    def sync(self) -> None:
        check(_lib().sc_batch_sync(self._b))
