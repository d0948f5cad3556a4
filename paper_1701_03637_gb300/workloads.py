"""Named synthetic workloads and seeded input generators.

This module holds parameters and random inputs only, none of the method's
arithmetic; both the CUDA path and the FP64 oracle are fed from it. The
geometries follow arXiv:1701.03637 Sec. III (planar film on a wall of
thickness 2 with an evaporation boundary at the far side; a floating droplet
with the boundary outside it).
"""
from __future__ import annotations

import numpy as np

Q = 19


def film_4x4x128(rho_hi=1.0, rho_lo=0.03, rho_H=0.03, seed=0, noise=1e-4, storage="f32"):
    """Planar film, 4x4x128 (x, y periodic): solid slab z in {0, 1} (the paper's wall of
    thickness 2), r-rich film for z < 32, evaporation sink plane z = 127."""
    params = dict(nx=4, ny=4, nz=128, tau_r=1.0, tau_b=1.0, G=3.6, rho_H=rho_H, geometry=1,
                  sink_z0=127, sink_layers=1, wall_z0=0, wall_thickness=2, storage=storage)
    init = dict(shape=0, film_z=32, rho_hi=rho_hi, rho_lo=rho_lo, noise_amp=noise, seed=seed)
    return params, init


def droplet(n, radius, seed, rho_hi=1.0, rho_lo=0.03, rho_H=0.03, noise=1e-4, storage="f32",
            spherical_sink=False):
    """Floating droplet in an n^3 box, x, y periodic. The sink is either the two
    z-boundary planes (z = n-1 and z = 0, i.e. two layers across the periodic seam)
    or the spherical exterior r >= n/2 - 2 (the paper's geometry)."""
    c = n / 2.0
    params = dict(nx=n, ny=n, nz=n, tau_r=1.0, tau_b=1.0, G=3.6, rho_H=rho_H, storage=storage)
    if spherical_sink:
        params.update(geometry=2, sphere_cx=c, sphere_cy=c, sphere_cz=c, R_H=n / 2.0 - 2.0)
    else:
        params.update(geometry=1, sink_z0=n - 1, sink_layers=2)
    init = dict(shape=1, cx=c, cy=c, cz=c, radius=radius, rho_hi=rho_hi, rho_lo=rho_lo, noise_amp=noise, seed=seed)
    return params, init


WORKLOADS = {
    "film_4x4x128": lambda **kw: film_4x4x128(**kw),
    "droplet_128": lambda **kw: droplet(128, 24.0, 1, **kw),
    "droplet_512": lambda **kw: droplet(512, 96.0, 2, **kw),
}


def random_populations(nx, ny, nz, seed, rho=(0.6, 0.1), spread=0.3):
    """Non-equilibrium populations f[c][i][z][y][x] = rho_c * U(1-spread, 1+spread) / 19,
    float64, seeded with numpy's PCG64."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(1.0 - spread, 1.0 + spread, (2, Q, nz, ny, nx)) / Q
    return f * np.asarray(rho, np.float64)[:, None, None, None, None]


def smooth_state(nx, ny, nz, seed, amp=0.05):
    """Density fields with a few long-wavelength modes (rho_r, rho_b), float64."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rr = np.full((nz, ny, nx), 0.5)
    rb = np.full((nz, ny, nx), 0.3)
    for _ in range(3):
        k = rng.integers(1, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        arg = 2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz)
        rr += amp * np.cos(arg + ph[0])
        rb += amp * np.sin(arg + ph[1])
    return rr, rb
