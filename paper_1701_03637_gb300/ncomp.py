"""More than two components (include/sc_lbm.h, sc_ncomp_*): Eq. (3) summed over every
other component on a periodic lattice with an optional solid slab. This module only
marshals; every step runs in the library's kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._native import MAX_COMP, NParams, check, load

Q = 19


class NLattice:
    """ncomp = len(tau) components (2 to 4) on the current CUDA device and stream;
    g[c][cbar] the couplings of Eq. (3)."""

    def __init__(self, nx, ny, nz, tau, g, wall_z0=0, wall_thickness=0, stream=None):
        import torch
        tau = list(map(float, tau))
        g = np.asarray(g, np.float64)
        self.ncomp = len(tau)
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        p = NParams(nx=nx, ny=ny, nz=nz, ncomp=self.ncomp, wall_z0=wall_z0, wall_thickness=wall_thickness)
        for c in range(min(self.ncomp, MAX_COMP)):
            p.tau[c] = tau[c]
            for b in range(min(self.ncomp, MAX_COMP)):
                p.g[c][b] = float(g[c, b])
        self.stream = stream or torch.cuda.current_stream()
        h = C.c_void_p()
        check(load().sc_ncomp_create(C.byref(p), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().sc_ncomp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def write_populations(self, f) -> None:
        f = np.ascontiguousarray(f, np.float64).reshape(-1)
        assert f.size == self.ncomp * Q * self.n
        check(load().sc_ncomp_write_populations(self._h, f.ctypes.data))

    def init_fields(self, rho) -> None:
        """Rest populations w_i rho^c from densities rho[c][z][y][x] (computed on the device)."""
        rho = np.ascontiguousarray(rho, np.float32).reshape(-1)
        assert rho.size == self.ncomp * self.n
        check(load().sc_ncomp_init_fields(self._h, rho.ctypes.data))

    def read_populations(self) -> np.ndarray:
        f = np.empty(self.ncomp * Q * self.n, np.float64)
        check(load().sc_ncomp_read_populations(self._h, f.ctypes.data))
        return f.reshape((self.ncomp, Q) + self.shape)

    def step(self, n: int = 1) -> None:
        check(load().sc_ncomp_step(self._h, int(n)))

    def sync(self) -> None:
        check(load().sc_ncomp_sync(self._h))
