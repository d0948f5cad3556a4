"""FP64 oracle of the N-component Shan-Chen D3Q19 step.

TEST INFRASTRUCTURE ONLY: the product library never imports or runs it; only the
tests use it. Plain numpy, written step by step in the order the paper states the
method (Sec. II), for any number of components: the paper calls the extension of
its two-component model to more components straightforward (Sec. I), and Eq. (3)
already sums the force over the other components cbar. The lattice is periodic
with an optional solid slab (halfway bounce-back, Psi = 0 at solid sites); the
paper states its evaporation boundary for two components only, so this model has
no sink.

Per step, for components c = 0..N-1:
  rho^c = sum_i f_i^c                                   (Sec. II A)
  Psi^c = 1 - exp(-rho^c)                                (Eq. 4, rho0 = 1)
  F^c = -Psi^c(x) sum_cbar g^{c cbar} sum_{i>=1} w_i Psi^cbar(x + e_i) e_i   (Eq. 3)
  u' = sum_c (m^c / tau_c) / sum_c (rho^c / tau_c)       (the common velocity)
  u^c_eq = u' + tau_c F^c / rho^c (u' where rho^c = 0)   (Sec. II B)
  f_i^c <- f_i^c - (f_i^c - f^eq_i(rho^c, u^c_eq)) / tau_c  at fluid sites (Eqs. 1, 2)
  streaming to x + e_i with periodic wrap; a population bound for a solid site
  returns to its source in the opposite direction.
State between steps: the canonical (post-stream) populations f[c][i][z][y][x].
"""
from __future__ import annotations

import numpy as np

Q = 19
# D3Q19 in the library's direction order: rest, +-x, +-y, +-z, then the 12 face
# diagonals in opposite pairs
E = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
              (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
              (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.int64)
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
OPP = np.array([int(np.flatnonzero((E == -e).all(axis=1))[0]) for e in E])
CS2 = 1.0 / 3.0


def _shift(a, e):
    """a(x - e) for an array whose last three axes are [z][y][x] (periodic)."""
    return np.roll(a, shift=(int(e[2]), int(e[1]), int(e[0])), axis=(-3, -2, -1))


def feq(rho, u):
    """Eq. (2): w_i rho (1 + c.u / c_s^2 + (c.u)^2 / (2 c_s^4) - u.u / (2 c_s^2)); u is [3][...]."""
    cu = np.tensordot(E.astype(np.float64), u, axes=([1], [0]))  # [19][...]
    uu = (u * u).sum(axis=0)
    return W.reshape((Q,) + (1,) * rho.ndim) * rho * (1.0 + cu / CS2 + 0.5 * (cu / CS2) ** 2 - 0.5 * uu / CS2)


class Lattice:
    """N components on an nx x ny x nz periodic lattice. tau: N relaxation times;
    g: N x N couplings g^{c cbar} of Eq. (3); solid planes z in [wall_z0, wall_z0 +
    wall_thickness)."""

    def __init__(self, nx, ny, nz, tau, g, wall_z0=0, wall_thickness=0):
        self.shape = (nz, ny, nx)
        self.tau = np.asarray(tau, np.float64)
        self.g = np.asarray(g, np.float64)
        self.n = len(self.tau)
        assert self.g.shape == (self.n, self.n)
        z = np.arange(nz)[:, None, None] * np.ones(self.shape, bool)
        self.solid = (z >= wall_z0) & (z < wall_z0 + wall_thickness)
        self.f = np.zeros((self.n, Q) + self.shape)

    def set_populations(self, f):
        self.f = np.array(f, np.float64).reshape((self.n, Q) + self.shape)
        self.f[:, :, self.solid] = 0.0

    def densities(self):
        rho = self.f.sum(axis=1)
        rho[:, self.solid] = 0.0
        return rho

    def step(self, steps: int = 1):
        for _ in range(int(steps)):
            self._step()

    def _step(self):
        f, n = self.f, self.n
        fluid = ~self.solid
        rho = self.densities()
        psi = np.where(self.solid, 0.0, 1.0 - np.exp(-rho))            # Eq. (4)
        # a^cbar = sum_i w_i Psi^cbar(x + e_i) e_i
        a = np.zeros((n, 3) + self.shape)
        for i in range(1, Q):
            for cb in range(n):
                nb = _shift(psi[cb], -E[i])                          # Psi(x + e_i)
                for d in range(3):
                    a[cb, d] += W[i] * nb * E[i, d]
        F = -psi[:, None] * np.einsum("cb,bd...->cd...", self.g, a)    # Eq. (3)
        m = np.tensordot(f, E.astype(np.float64), axes=([1], [0]))     # [c][...][3]
        m = np.moveaxis(m, -1, 1)                                      # [c][3][...]
        den = (rho / self.tau[:, None, None, None]).sum(axis=0)
        up = (m / self.tau[:, None, None, None, None]).sum(axis=0) / np.where(den > 0, den, 1.0)
        out = f.copy()
        for c in range(n):
            r = rho[c]
            shift = np.where(r > 0, self.tau[c] * F[c] / np.where(r > 0, r, 1.0), 0.0)
            ueq = up + shift
            post = f[c] - (f[c] - feq(r, ueq)) / self.tau[c]          # Eq. (1)
            out[c] = np.where(fluid, post, f[c])
        # streaming (push, periodic) with halfway bounce-back into solid sites
        new = np.zeros_like(out)
        for i in range(Q):
            moved = _shift(out[:, i], E[i])                            # at x: what left x - e_i
            blocked = _shift(self.solid, -E[i])                        # at x: is x + e_i solid
            new[:, i] += np.where(self.solid, 0.0, moved)
            new[:, OPP[i]] += np.where(blocked & fluid, out[:, i], 0.0)
        new[:, :, self.solid] = 0.0
        self.f = new
