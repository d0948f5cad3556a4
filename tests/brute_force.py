"""A second, literal FP64 evaluation of one time step (arXiv:1701.03637 Sec. II),
written independently of the oracle for tiny lattices: per-site Python loops,
its own D3Q19 table (lexicographic order of the velocity vectors, weights from
|e|^2), push streaming. Used only to pin the oracle.

State convention: canonical populations f[c, x, y, z, k] after streaming and
the sink reset, c = 0 (r), 1 (b); k indexes VELOCITIES.
"""
from __future__ import annotations

import math

import numpy as np

VELOCITIES = [(ex, ey, ez) for ex in (-1, 0, 1) for ey in (-1, 0, 1) for ez in (-1, 0, 1)
              if ex * ex + ey * ey + ez * ez <= 2]
WEIGHT = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
W = [WEIGHT[ex * ex + ey * ey + ez * ez] for ex, ey, ez in VELOCITIES]
OPPOSITE = [VELOCITIES.index((-ex, -ey, -ez)) for ex, ey, ez in VELOCITIES]
CS2 = 1.0 / 3.0


class BruteForce:
    def __init__(self, p: dict):
        self.p = p
        self.nx, self.ny, self.nz = p["nx"], p["ny"], p["nz"]
        self.evaporated = 0.0
        self.cls = {}
        for x in range(self.nx):
            for y in range(self.ny):
                for z in range(self.nz):
                    self.cls[(x, y, z)] = self._classify(x, y, z)

    def _classify(self, x, y, z):
        p = self.p
        t = p.get("wall_thickness", 0)
        if t and p["wall_z0"] <= z < p["wall_z0"] + t:
            return "solid"
        g = p.get("geometry", 0)
        if g == 1 and (z - p["sink_z0"]) % self.nz < p["sink_layers"]:
            return "sink"
        if g == 2:
            r2 = (x - p["sphere_cx"]) ** 2 + (y - p["sphere_cy"]) ** 2 + (z - p["sphere_cz"]) ** 2
            if r2 >= p["R_H"] ** 2:
                return "sink"
        return "fluid"

    def _wrap(self, x, y, z):
        return x % self.nx, y % self.ny, z % self.nz

    def step(self, f):
        p = self.p
        tau = (p["tau_r"], p["tau_b"])
        G, rho_H = p["G"], p["rho_H"]
        sites = list(self.cls)
        # densities and pseudopotential (Eq. (4), rho0 = 1); zero at solid sites
        rho = {s: [0.0, 0.0] for s in sites}
        psi = {s: [0.0, 0.0] for s in sites}
        for s in sites:
            if self.cls[s] == "solid":
                continue
            for c in (0, 1):
                rho[s][c] = math.fsum(f[c][s][k] for k in range(19))
                psi[s][c] = 1.0 - math.exp(-rho[s][c])
        post = {s: [list(f[0][s]), list(f[1][s])] for s in sites}
        for s in sites:
            if self.cls[s] != "fluid":
                continue  # sinks stream their reset values, solids hold nothing
            x, y, z = s
            # Eq. (3): F^c = -G psi^c(x) sum_i w_i psi^cbar(x + e_i) e_i
            F = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]
            for c in (0, 1):
                acc = [0.0, 0.0, 0.0]
                for k, e in enumerate(VELOCITIES):
                    n = self._wrap(x + e[0], y + e[1], z + e[2])
                    for d in range(3):
                        acc[d] += W[k] * psi[n][1 - c] * e[d]
                F[c] = [-G * psi[s][c] * a for a in acc]
            # common velocity weighted by rho^c / tau_c, then the force shift
            mom = [[sum(f[c][s][k] * VELOCITIES[k][d] for k in range(19)) for d in range(3)] for c in (0, 1)]
            den = rho[s][0] / tau[0] + rho[s][1] / tau[1]
            u_common = [(mom[0][d] / tau[0] + mom[1][d] / tau[1]) / den if den > 0 else 0.0 for d in range(3)]
            for c in (0, 1):
                if rho[s][c] > 0:
                    u = [u_common[d] + tau[c] * F[c][d] / rho[s][c] for d in range(3)]
                else:
                    u = list(u_common)
                uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
                for k, e in enumerate(VELOCITIES):
                    eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2]
                    feq = W[k] * rho[s][c] * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2))
                    post[s][c][k] = f[c][s][k] - (f[c][s][k] - feq) / tau[c]
        # push streaming with halfway bounce-back off solid sites
        new = {s: [[0.0] * 19, [0.0] * 19] for s in sites}
        for s in sites:
            if self.cls[s] == "solid":
                continue
            x, y, z = s
            for k, e in enumerate(VELOCITIES):
                n = self._wrap(x + e[0], y + e[1], z + e[2])
                for c in (0, 1):
                    if self.cls[n] == "solid":
                        new[s][c][OPPOSITE[k]] = post[s][c][k]
                    else:
                        new[n][c][k] = post[s][c][k]
        # evaporation boundary on the arrived populations (Sec. II C)
        flux = 0.0
        for s in sites:
            if self.cls[s] != "sink":
                continue
            rr = math.fsum(new[s][0])
            rb = math.fsum(new[s][1])
            flux += rr - rho_H
            for k in range(19):
                new[s][0][k] = W[k] * rho_H
                new[s][1][k] = W[k] * (rr + rb - rho_H)
        self.evaporated += flux
        return [{s: new[s][0] for s in sites}, {s: new[s][1] for s in sites}]

    # conversion from / to the oracle's array f[c, i, z, y, x] with direction table c_oracle
    def from_array(self, a, c_oracle):
        perm = [next(i for i in range(19) if tuple(c_oracle[i]) == v) for v in VELOCITIES]
        return [{(x, y, z): [float(a[c, perm[k], z, y, x]) for k in range(19)]
                 for x in range(self.nx) for y in range(self.ny) for z in range(self.nz)} for c in (0, 1)]

    def to_array(self, f, c_oracle):
        out = np.zeros((2, 19, self.nz, self.ny, self.nx))
        for i in range(19):
            k = VELOCITIES.index(tuple(int(v) for v in c_oracle[i]))
            for (x, y, z), vals in f[0].items():
                out[0, i, z, y, x] = vals[k]
                out[1, i, z, y, x] = f[1][(x, y, z)][k]
        return out
