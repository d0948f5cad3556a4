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


def three_component_droplet(n, radius, seed, rho_hi=0.7, rho_lo=0.04, rho_third=0.1, noise=1e-4):
    """Three components in an n^3 periodic box: a droplet of component 0 (rho_hi inside
    the sphere, rho_lo outside) in component 1 (the complement), with component 2
    dissolved everywhere at rho_third; uniform noise of +-noise on every density
    (numpy's PCG64 with `seed`). g^{01} = 3.6 (the paper's G), g^{02} = g^{12} = 1.0,
    no self coupling, tau = 1. Returns (NLattice keyword arguments, rho[c][z][y][x])."""
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    inside = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 <= radius * radius
    rho = np.empty((3, n, n, n), np.float32)
    rho[0] = np.where(inside, rho_hi, rho_lo)
    rho[1] = np.where(inside, rho_lo, rho_hi)
    rho[2] = rho_third
    rng = np.random.default_rng(seed)
    rho += rng.uniform(-noise, noise, rho.shape).astype(np.float32)
    g = [[0.0, 3.6, 1.0], [3.6, 0.0, 1.0], [1.0, 1.0, 0.0]]
    return dict(nx=n, ny=n, nz=n, tau=[1.0, 1.0, 1.0], g=g), rho


WORKLOADS = {
    "film_4x4x128": lambda **kw: film_4x4x128(**kw),
    "droplet_128": lambda **kw: droplet(128, 24.0, 1, **kw),
    "droplet_256": lambda **kw: droplet(256, 48.0, 2, **kw),
    "droplet_512": lambda **kw: droplet(512, 96.0, 2, **kw),
    # the same recipe at 1024^3 (R/N = 0.1875): in FP32 it fits one GPU only in place
    "droplet_1024": lambda **kw: droplet(1024, 192.0, 2, **kw),
}


class SplitMix64:
    """Counter stream of SplitMix64 (Steele, Lea and Flood 2014), for drawing
    workload parameters; u() maps the top 53 bits to [0, 1)."""

    M = (1 << 64) - 1

    def __init__(self, seed: int):
        self.x = seed & self.M

    def next(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & self.M
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.M
        return z ^ (z >> 31)

    def u(self) -> float:
        return (self.next() >> 11) * 2.0 ** -53


def ensemble_member(k: int, rng: "SplitMix64", lo: float = 32.0, hi: float = 96.0, cubic: bool = False,
                    storage="f32"):
    """One lattice of a randomised ensemble: edges exp(U(ln lo, ln hi)) (per axis, or one
    for a cube), even k a planar film (wall z in {0, 1}, film below nz/4, sink plane
    z = nz-1), odd k a floating droplet (radius U(0.2, 0.35) x the shortest edge, sinks
    at the z-boundary planes); g ~ U(3.2, 3.8) and one tau ~ U(0.8, 1.2) for both
    components; init seed from the stream."""
    import math

    def edge():
        return int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * rng.u())))

    if cubic:
        nx = ny = nz = edge()
    else:
        nx, ny, nz = edge(), edge(), edge()
    G = 3.2 + 0.6 * rng.u()
    tau = 0.8 + 0.4 * rng.u()
    seed = rng.next()
    base = dict(nx=nx, ny=ny, nz=nz, tau_r=tau, tau_b=tau, G=G, rho_H=0.03, storage=storage)
    if k % 2 == 0:
        params = dict(base, geometry=1, sink_z0=nz - 1, sink_layers=1, wall_z0=0, wall_thickness=2)
        init = dict(shape=0, film_z=max(3, nz // 4), rho_hi=1.0, rho_lo=0.03, noise_amp=1e-4, seed=seed)
    else:
        r = (0.2 + 0.15 * rng.u()) * min(nx, ny, nz)
        params = dict(base, geometry=1, sink_z0=nz - 1, sink_layers=2)
        init = dict(shape=1, cx=nx / 2.0, cy=ny / 2.0, cz=nz / 2.0, radius=r, rho_hi=1.0, rho_lo=0.03,
                    noise_amp=1e-4, seed=seed)
    return params, init


def ensemble(count: int = 64, seed: int = 3, storage="f32"):
    """A batched ensemble: count lattices drawn by ensemble_member from one stream."""
    rng = SplitMix64(seed)
    return [ensemble_member(k, rng, storage=storage) for k in range(count)]


def shard(sizes, rank: int, world: int):
    """Indices of the ensemble members that `rank` of `world` ranks advances: the
    largest member first to the rank with the fewest sites so far (ties to the lower
    rank), so every member goes to exactly one rank and the ranks' site totals differ
    by at most the largest member. Deterministic: every rank computes the same split."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    order = sorted(range(len(sizes)), key=lambda k: (-sizes[k], k))
    load = [0] * world
    owner = [0] * len(sizes)
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += sizes[k]
    return [k for k in range(len(sizes)) if owner[k] == rank]


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


def request_stream(count: int, rate: float, seed: int = 4, lo: float = 32.0, hi: float = 160.0,
                   steps=(2000, 20000), storage="f16"):
    """A served request stream: Poisson arrivals at `rate` per second (exponential gaps),
    each request a cubic lattice (edge log-uniform in [lo, hi]) drawn like an ensemble
    member, with a step count uniform in [steps[0], steps[1]]. Returns a list of
    (arrival_s, params, init, nsteps)."""
    import math
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += -math.log(1.0 - rng.u()) / rate
        params, init = ensemble_member(k, rng, lo, hi, cubic=True, storage=storage)
        n = int(steps[0] + (steps[1] - steps[0]) * rng.u())
        out.append((t, params, init, n))
    return out
