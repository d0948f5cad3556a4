"""Experiments of arXiv:1701.03637 Sec. III run on the library's step.

These drive the CUDA path through the public API and record what the paper
compares with its laws: the densities inside and outside droplets of several
radii for the Laplace law (the sink closed), the radius of an evaporating
droplet with the spherical sink r >= R_H over time (Sec. III C), the interface
position of an evaporating planar film (Sec. III B), and the profiles and
relative flux of the diffusion column (Sec. III A). They only read fields,
diagnostics and the device-computed flux; every time step and every evaluation
of the method's formulas runs in the library. The equation of state that turns
densities into a pressure jump is the caller's (`pressure` arguments).
"""
from __future__ import annotations

import math

import numpy as np

from . import Lattice

def _droplet_params(n, G, tau, geometry=0, R_H=0.0, rho_H=0.03, storage="f32"):
    c = n / 2.0
    p = dict(nx=n, ny=n, nz=n, tau_r=tau, tau_b=tau, G=G, rho_H=rho_H, geometry=geometry, storage=storage)
    if geometry == 2:
        p.update(sphere_cx=c, sphere_cy=c, sphere_cz=c, R_H=R_H)
    return p


def _init(n, R, rho, seed):
    c = n / 2.0
    return dict(shape=1, cx=c, cy=c, cz=c, radius=R, rho_hi=rho[0], rho_lo=rho[1], noise_amp=1e-4, seed=seed)


def surface_tension(pressure, radii=(8.0, 12.0, 16.0), margin=12, steps=4000, G=3.6, tau=1.0, rho=(0.7, 0.04),
                    seed=5):
    """Laplace test with the sink closed: for each initial radius a droplet in a
    periodic box of edge 2 R + 2 margin equilibrates for `steps` steps; the
    pressure jump between the centre and the box corner, pressure(rho^r, rho^b, G)
    of the caller's equation of state, is fitted against 1/R (R from the droplet
    volume). Returns gamma = slope / 2 and the fit data."""
    inv_r, dp = [], []
    for R0 in radii:
        n = int(2 * R0 + 2 * margin)
        lat = Lattice(_droplet_params(n, G, tau))
        lat.init(_init(n, R0, rho, seed))
        lat.step(steps)
        rr, rb = lat.read_fields()
        d = lat.diagnostics()
        lat.close()
        m = n // 2
        inv_r.append(1.0 / d["radius"])
        dp.append(float(pressure(rr[m, m, m], rb[m, m, m], G) - pressure(rr[0, 0, 0], rb[0, 0, 0], G)))
    slope, icpt = np.polyfit(inv_r, dp, 1)
    return dict(gamma=slope / 2.0, intercept=icpt, inv_radius=inv_r, pressure_jump=dp)


def single_component_laplace(pressure, g, rho_l, rho_g, radii=(8.0, 12.0, 16.0), margin=12, steps=3000):
    """Laplace test of the multiphase pseudopotential model (component b absent,
    self coupling g^{rr} = g, no cross coupling): a liquid droplet (rho_l) in its
    vapour (rho_g) in a periodic box of edge 2 R + 2 margin settles for `steps`
    steps; R is the radius of the volume where rho > (rho_l + rho_g) / 2. Returns
    gamma = slope / 2 of the jump of pressure(rho^r, 0, 0, G_rr=g) (the caller's
    equation of state) against 1/R and the fit data."""
    inv_r, dp = [], []
    for R0 in radii:
        n = int(2 * R0 + 2 * margin)
        c = (n - 1) / 2.0
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        inside = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 < R0 * R0
        lat = Lattice(dict(nx=n, ny=n, nz=n, G=0.0, G_rr=g, geometry=0))
        lat.init_fields(np.where(inside, rho_l, rho_g).astype(np.float32), np.zeros((n, n, n), np.float32))
        lat.step(steps)
        rr, _ = lat.read_fields()
        lat.close()
        m = n // 2
        vol = float(np.count_nonzero(rr > 0.5 * (rho_l + rho_g)))
        inv_r.append(1.0 / equivalent_radius(vol))
        dp.append(float(pressure(rr[m, m, m], 0.0, 0.0, G_rr=g) - pressure(rr[0, 0, 0], 0.0, 0.0, G_rr=g)))
    slope, icpt = np.polyfit(inv_r, dp, 1)
    return dict(gamma=slope / 2.0, intercept=icpt, inv_radius=inv_r, pressure_jump=dp)


def evaporating_droplet(n, R0, rho_H=0.01, G=3.6, tau=1.0, rho=(0.7, 0.04), equilibrate=2000, steps=20000,
                        every=500, R_H=None, R_stop=4.0, seed=5, storage="f32", tune=False):
    """A droplet equilibrates with the sink closed, then evaporates through the
    spherical sink r >= R_H (default n/2 - 2) with rho^r = rho_H there. Returns
    the radius series R(t) (t counted from opening the sink), the coexistence
    densities at the start (rho^r at the centre, the r vapour density in the
    shell R + 4 < r < R + 6, rho^b far outside) and R_H. tune: let the step's
    autotuner pick the kernel configuration of the evaporation run (same bits)."""
    R_H = n / 2.0 - 2.0 if R_H is None else R_H
    eq = Lattice(_droplet_params(n, G, tau, storage=storage))
    eq.init(_init(n, R0, rho, seed))
    eq.step(equilibrate)
    f = eq.read_populations()
    rr, rb = eq.read_fields()
    R_start = eq.diagnostics()["radius"]
    eq.close()
    c, m = n / 2.0, n // 2
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    rho_ma0 = float(rr[m, m, m])
    rho_mi0 = float(rr[(r > R_start + 4) & (r < R_start + 6)].mean())
    rho_b_out = float(rb[0, 0, 0])
    ev = Lattice(_droplet_params(n, G, tau, geometry=2, R_H=R_H, rho_H=rho_H, storage=storage))
    ev.write_populations(f)
    if tune:
        ev.tune()
    ts, Rs, fluxes = [0], [R_start], [0.0]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        ev.step(k)
        done += k
        d = ev.diagnostics()
        if d["status"] != 0:
            raise RuntimeError(f"diagnostics status {d['status']} at step {done}")
        ts.append(done)
        Rs.append(d["radius"])
        fluxes.append(d["evaporated_mass"])
        if d["radius"] < R_stop:
            break
    ev.close()
    return dict(t=np.asarray(ts, np.float64), R=np.asarray(Rs), evaporated_mass=np.asarray(fluxes), R_H=R_H,
                rho_ma0=rho_ma0, rho_mi0=rho_mi0, rho_b_out=rho_b_out, rho_H=rho_H, G=G, n=n)


def radius_rate(t, R, t0, t1):
    """Mean dR/dt over [t0, t1] from a radius series (linear interpolation)."""
    return (float(np.interp(t1, t, R)) - float(np.interp(t0, t, R))) / (t1 - t0)


def equivalent_radius(droplet_sites: int) -> float:
    return (3.0 * droplet_sites / (4.0 * math.pi)) ** (1.0 / 3.0)


def evaporating_film(nz=128, film_z=32, nxy=4, rho=(0.70, 0.04), rho_H=0.02, G=3.6, tau=1.0, equilibrate=20000,
                     steps=1_000_000, every=10000, seed=0, storage="f32"):
    """The planar film of Sec. III B: a wall of thickness 2 at z in {0, 1}, the
    r-rich film below film_z, equilibrated with the sink closed, then evaporating
    through the sink plane z = nz - 1 (rho^r = rho_H there). Returns the
    interface position x_I(t) (t from opening the sink), the evaporated mass, the
    coexistence densities of the equilibrated profile (rho^r in the liquid and
    vapour plateaus, rho^b in the vapour) and x_H = nz - 1."""
    base = dict(nx=nxy, ny=nxy, nz=nz, tau_r=tau, tau_b=tau, G=G, rho_H=rho_H, wall_z0=0, wall_thickness=2,
                storage=storage)
    eq = Lattice(dict(base, geometry=0))
    eq.init(dict(shape=0, film_z=film_z, rho_hi=rho[0], rho_lo=rho[1], noise_amp=1e-4, seed=seed))
    eq.step(equilibrate)
    f = eq.read_populations()
    rr, rb = eq.read_fields()
    eq.close()
    pr, pb = rr.mean(axis=(1, 2)), rb.mean(axis=(1, 2))
    rho_ma = float(pr[4:film_z - 6].mean())
    rho_mi = float(pr[film_z + 10:nz - 6].mean())
    rho_b_vap = float(pb[film_z + 10:nz - 6].mean())
    ev = Lattice(dict(base, geometry=1, sink_z0=nz - 1, sink_layers=1))
    ev.write_populations(f)
    d = ev.diagnostics()
    ts, xs, em = [0], [d["interface_z"]], [0.0]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        ev.step(k)
        done += k
        d = ev.diagnostics()
        if d["status"] != 0:
            raise RuntimeError(f"diagnostics status {d['status']} at step {done}")
        ts.append(done)
        xs.append(d["interface_z"])
        em.append(d["evaporated_mass"])
    ev.close()
    return dict(t=np.asarray(ts, np.float64), x_I=np.asarray(xs), evaporated_mass=np.asarray(em), x_H=float(nz - 1),
                rho_ma=rho_ma, rho_mi=rho_mi, rho_b_vap=rho_b_vap, rho_H=rho_H, G=G)


def fick_column(nz=125, nxy=4, rho_cbar=0.7, rho_H=0.001, G=3.6, tau=1.0, times=(3000, 10000), storage="f32"):
    """The diffusion experiment of Sec. III A (the paper's 125 x 4 x 4 sites by
    default): a column of the other component (rho^b = rho_cbar, rho^r = 0) between
    the evaporation boundary z = 0, which holds rho^r = rho_H, and a wall of thickness
    2 at the far end (the last two planes). Returns, at each
    time, the xy-mean profiles of rho^r and rho^b and the z flux of r relative to
    the mixture, rho^r (U^r - U) of Eqs. (flux) and (velw) (tau = 1), evaluated on
    the device (sc_lbm_flux_profile)."""
    p = dict(nx=nxy, ny=nxy, nz=nz, tau_r=tau, tau_b=tau, G=G, rho_H=rho_H, geometry=1, sink_z0=0, sink_layers=1,
             wall_z0=nz - 2, wall_thickness=2, storage=storage)
    lat = Lattice(p)
    lat.init_fields(np.zeros((nz, nxy, nxy), np.float32), np.full((nz, nxy, nxy), rho_cbar, np.float32))
    out = []
    done = 0
    for T in times:
        lat.step(T - done)
        done = T
        rr, rb = lat.read_fields()
        out.append(dict(t=T, rho_r=rr.astype(np.float64).mean(axis=(1, 2)), rho_b=rb.astype(np.float64).mean(axis=(1, 2)),
                        flux=lat.flux_profile()[2]))
    lat.close()
    return out
