"""Pin: an evaporating droplet in the oracle follows the Laplace-pressure-
corrected radius law of Sec. III C (Eq. (drop-r-df4)), with the surface tension
measured by a Laplace test (sink closed, pressure jump against 1/R) and the
coexistence densities, vapour D^c (Sec. III A) and d0 = 2.5 from the film
section. The droplet (radius ~10 in a 40^3 box, spherical sink r >= 18 with
rho_H = 0.01) is equilibrated with the sink closed, the sink is opened, and the
radius change over a quasi-steady window (steps 1000-2000 after opening, after
the diffusive set-up of the vapour profile and before the final collapse) is
compared with the law integrated by RK4 from the simulated radius at the start
of the window."""
import math

import numpy as np

G = 3.6


def _radius(rr, rb):
    return (3.0 * int(np.sum(rr > rb)) / (4.0 * math.pi)) ** (1.0 / 3.0)


def _pressure(a, b):
    # bulk pressure of the two-component Shan-Chen fluid: c_s^2 (rho^r + rho^b) + g c_s^2 psi^r psi^b
    from oracle.analytic import psi
    return (a + b) / 3.0 + G / 3.0 * float(psi(a)) * float(psi(b))


def _droplet(oracle_mod, n, R, params=None):
    c = n / 2.0
    o = oracle_mod.Lattice(dict(nx=n, ny=n, nz=n, G=G, geometry=0, **(params or {})))
    o.init_shape(dict(shape=1, cx=c, cy=c, cz=c, radius=R, rho_hi=0.7, rho_lo=0.04, seed=5, noise_amp=1e-4))
    return o


def test_droplet_follows_the_laplace_corrected_radius_law(oracle_mod):
    from oracle import analytic as A
    # surface tension from the Laplace law: pressure jump = 2 gamma / R
    inv_r, dp = [], []
    for R, n in [(6, 24), (9, 30), (12, 36)]:
        o = _droplet(oracle_mod, n, R)
        o.step(1500)
        rr, rb = o.fields()
        m = n // 2
        inv_r.append(1.0 / _radius(rr, rb))
        dp.append(_pressure(rr[m, m, m], rb[m, m, m]) - _pressure(rr[0, 0, 0], rb[0, 0, 0]))
    slope, icpt = np.polyfit(inv_r, dp, 1)
    gamma = slope / 2.0
    assert gamma > 0 and abs(icpt) < 0.05 * slope * max(inv_r)  # a line through the origin

    n = 40
    o = _droplet(oracle_mod, n, 10.0)
    o.step(1000)
    f = o.populations()
    rr, rb = o.fields()
    c, m = n / 2.0, n // 2
    R0 = _radius(rr, rb)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    rho_ma0 = rr[m, m, m]
    rho_mi0 = rr[(r > R0 + 4) & (r < R0 + 6)].mean()
    rho_b_out = rb[0, 0, 0]
    R_H, rho_H, d0 = n / 2.0 - 2.0, 0.01, 2.5
    e = oracle_mod.Lattice(dict(nx=n, ny=n, nz=n, G=G, geometry=2, sphere_cx=c, sphere_cy=c, sphere_cz=c,
                                R_H=R_H, rho_H=rho_H))
    e.set_populations(f)
    e.step(1000)
    R1 = _radius(*e.fields())
    e.step(1000)
    R2 = _radius(*e.fields())
    D = float(A.diffusion_coefficient(rho_mi0, rho_b_out, G))

    def rhs(R):
        _, mi = A.laplace_densities(R, R0, gamma, rho_ma0, rho_mi0)
        return A.drop_mass_rate(R, R_H, d0, D, mi, rho_H) / A._dMdR(R, R_H, d0, rho_ma0, rho_mi0, rho_H,
                                                                      R0=R0, gamma=gamma)

    R, dt = R1, 10.0
    for _ in range(100):
        k1 = rhs(R)
        k2 = rhs(R + 0.5 * dt * k1)
        k3 = rhs(R + 0.5 * dt * k2)
        k4 = rhs(R + dt * k3)
        R += dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert R2 < R1 < R0  # evaporating
    assert abs((R2 - R1) - (R - R1)) < 0.05 * abs(R - R1), (R1, R2, R)
