"""Analytic laws of arXiv:1701.03637 Sec. III, written out in numpy.

TEST INFRASTRUCTURE ONLY (part of the oracle): the tests use these closed forms
and ODE solutions to check the simulated physics.

Readings where the printed formulas are garbled (each also listed in the design
notes):
  * Psi' in Eq. (diffu-t-1) is dPsi/drho = exp(-rho/rho0) (the "spatial
    derivative" wording cannot be meant: D must not depend on the gradient).
  * The mass derivative in Eqs. (mass_flux-2) and (mass-df1) is negative when
    rho_mi > rho_H (the film/droplet loses mass), so dx_I/dt and dR_I/dt carry
    a minus sign.
  * Eq. (xt) is the solution of Eq. (xit) only with x_H - d0 in place of the
    printed x_H + d0; ``film_xI`` integrates the ODE as stated and
    ``film_xI_printed`` keeps the printed form for comparison.
  * Eqs. (mass-df2)/(drop-mass-df4) are the R-derivatives of Eq. (drop-mass-1)
    (with the stray ``d`` read as d0); ``drop_mass`` implements Eq.
    (drop-mass-1) and the printed derivatives are kept for cross-checking.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def psi(rho):
    """Eq. (psifunc) with rho0 = 1."""
    return 1.0 - np.exp(-np.asarray(rho, dtype=np.float64))


def dpsi(rho):
    """dPsi/drho (reading of Psi' in Eq. (diffu-t-1))."""
    return np.exp(-np.asarray(rho, dtype=np.float64))


def diffusion_matrix(rho_c, rho_cb, g, tau=1.0):
    """(D^{cc}, D^{c cbar}) of Eq. (diffu-t-1), symmetric g^{c cbar} = g^{cbar c} = g."""
    rt = rho_c + rho_cb
    dcc = CS2 * (tau - 0.5) * rho_cb / rt - CS2 * rho_c * psi(rho_cb) * g * dpsi(rho_c) / rt
    dccb = -CS2 * (tau - 0.5) * rho_c / rt + CS2 * rho_cb * psi(rho_c) * g * dpsi(rho_cb) / rt
    return dcc, dccb


def diffusion_coefficient(rho_c, rho_cb, g, tau=1.0):
    """Small-gradient D^c of Sec. III A (Eq. (fick-simple) and the D^c below it)."""
    rt = rho_c + rho_cb
    return CS2 * (tau - 0.5) - CS2 / rt * (
        rho_cb * psi(rho_c) * g * dpsi(rho_cb) + rho_c * psi(rho_cb) * g * dpsi(rho_c))


# ---------------------------------------------------------------- planar film (Sec. III B)

def film_rate_constant(D, rho_ma, rho_mi, rho_H):
    """K = D (rho_mi - rho_H) / (rho_ma - rho_mi/2 - rho_H/2), from Eqs. (mass_flux-1), (xit)."""
    return D * (rho_mi - rho_H) / (rho_ma - 0.5 * rho_mi - 0.5 * rho_H)


def film_flux(D, rho_mi, rho_H, x_H, x_I, d0):
    """|j| of Eq. (fick-linear-0): linear vapour profile between x_I + d0 and x_H."""
    return D * (rho_mi - rho_H) / (x_H - x_I - d0)


def film_xI(t, x0, x_H, d0, D, rho_ma, rho_mi, rho_H):
    """x_I(t) solving Eq. (xit) (sign reading: evaporation lowers x_I) with x_I(0) = x0."""
    K = film_rate_constant(D, rho_ma, rho_mi, rho_H)
    t = np.asarray(t, dtype=np.float64)
    return x_H - d0 - np.sqrt((x_H - d0 - x0) ** 2 + 2.0 * K * t)


def film_xI_printed(t, x0, x_H, d0, D, rho_ma, rho_mi, rho_H):
    """Eq. (xt) exactly as printed (x_H + d0); kept only to report the difference."""
    K = film_rate_constant(D, rho_ma, rho_mi, rho_H)
    t = np.asarray(t, dtype=np.float64)
    return x_H + d0 - np.sqrt((x_H + d0 - x0) ** 2 + 2.0 * K * t)


def film_xI_rk4(t_end, dt, x0, x_H, d0, D, rho_ma, rho_mi, rho_H):
    """Eq. (xit) integrated with classic RK4 (independent of the closed form)."""
    K = film_rate_constant(D, rho_ma, rho_mi, rho_H)

    def rhs(x):
        return -K / (x_H - x - d0)

    x, t = float(x0), 0.0
    n = int(round(t_end / dt))
    for _ in range(n):
        k1 = rhs(x)
        k2 = rhs(x + 0.5 * dt * k1)
        k3 = rhs(x + 0.5 * dt * k2)
        k4 = rhs(x + dt * k3)
        x += dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    return x


# ---------------------------------------------------------------- droplet (Sec. III C)

def _int_r_times(b, a, c):
    """int_a^c r (b - r) dr."""
    return b * (c * c - a * a) / 2.0 - (c ** 3 - a ** 3) / 3.0


def drop_mass(R, R_H, d0, rho_ma, rho_mi, rho_H):
    """Eq. (drop-mass-1): total mass of c inside R_H, integrated in closed form."""
    a, b = R - d0, R + d0
    m1 = 4.0 * math.pi / 3.0 * a ** 3 * rho_ma
    m2 = 4.0 * math.pi / 3.0 * (b ** 3 - a ** 3) * rho_mi \
        - 4.0 * math.pi * (rho_mi - rho_ma) * a / (2.0 * d0) * _int_r_times(b, a, b)
    m3 = 4.0 * math.pi / 3.0 * (R_H ** 3 - b ** 3) * rho_H \
        - 4.0 * math.pi * (rho_H - rho_mi) * b / (R_H - b) * _int_r_times(R_H, b, R_H)
    return m1 + m2 + m3


def drop_dMdR_printed(R, R_H, d0, rho_ma, rho_mi, rho_H):
    """The bracket of Eq. (mass-df2) (dM/dt = this * dR/dt), as printed."""
    return 2.0 * math.pi / 3.0 * (
        R_H ** 2 * (-rho_H + rho_mi)
        + R_H * (-2 * R * rho_H + 2 * R * rho_mi - 2 * d0 * rho_H + 2 * d0 * rho_mi)
        + 6 * R ** 2 * rho_ma - 6 * R ** 2 * rho_mi - 2 * d0 ** 2 * rho_ma + 2 * d0 ** 2 * rho_mi)


def drop_mass_rate(R, R_H, d0, D, rho_mi, rho_H):
    """dM/dt of Eq. (mass-df1), sign reading: negative when rho_mi > rho_H."""
    return -4.0 * math.pi * D * (rho_mi - rho_H) * (R + d0) * R_H / (R_H - R - d0)


def laplace_densities(R, R0, gamma, rho_ma0, rho_mi0):
    """Eqs. (rho_ma) and (rho_mi)."""
    rho_ma = rho_ma0 - 2.0 * gamma / CS2 * (1.0 / R0 - 1.0 / R)
    return rho_ma, rho_mi0 * rho_ma / rho_ma0


def drop_dMdR_laplace_printed(R, R_H, d0, R0, gamma, rho_ma0, rho_mi0, rho_H):
    """The bracket of Eq. (drop-mass-df4), as printed (d read as d0)."""
    d = d0
    ma = rho_ma0 - 2.0 * gamma / CS2 * (1.0 / R0 - 1.0 / R)
    mi = rho_mi0 * ma / rho_ma0
    return 2.0 * math.pi / 3.0 * (
        (-R_H ** 2 - 2 * R * R_H - 2 * R_H * d0) * rho_H
        + (R_H ** 2 + 2 * R * R_H + 2 * R_H * d0 - 6 * R ** 2 + 2 * d ** 2) * mi
        + (R * R_H ** 2 + d * R_H ** 2 + R ** 2 * R_H + 2 * R * R_H * d0 + d0 ** 2 * R_H - 2 * R ** 3
           + 2 * R * d ** 2) * (-2.0 * gamma * rho_mi0 / (CS2 * rho_ma0) / R ** 2)
        + (6 * R ** 2 - 2 * d ** 2) * ma
        + (2 * R ** 3 - 2 * R * d ** 2) * (-2.0 * gamma / (CS2 * R ** 2)))


def _dMdR(R, R_H, d0, rho_ma, rho_mi, rho_H, R0=None, gamma=0.0):
    """Exact-in-float derivative of Eq. (drop-mass-1) by a 4-point central difference."""
    def M(r):
        if gamma:
            ma, mi = laplace_densities(r, R0, gamma, rho_ma, rho_mi)
        else:
            ma, mi = rho_ma, rho_mi
        return drop_mass(r, R_H, d0, ma, mi, rho_H)

    h = 1e-3 * max(1.0, abs(R))
    return (-M(R + 2 * h) + 8 * M(R + h) - 8 * M(R - h) + M(R - 2 * h)) / (12 * h)


def droplet_radius_rk4(R0, t_end, dt, R_H, d0, D, rho_ma, rho_mi, rho_H, gamma=0.0, R_stop=None):
    """R_I(t) from dM/dt (Eq. (mass-df1)) = dM/dR dR/dt, integrated with RK4.

    gamma = 0 gives Eq. (mass-dfsum-sim); gamma > 0 gives Eq. (drop-r-df4) with the
    Laplace-corrected densities of Eqs. (rho_ma), (rho_mi) in both the mass and
    the flux. Returns (t, R) arrays, stopping early when R < R_stop.
    """
    def rhs(R):
        if gamma:
            _, mi = laplace_densities(R, R0, gamma, rho_ma, rho_mi)
        else:
            mi = rho_mi
        return drop_mass_rate(R, R_H, d0, D, mi, rho_H) / _dMdR(
            R, R_H, d0, rho_ma, rho_mi, rho_H, R0=R0, gamma=gamma)

    n = int(round(t_end / dt))
    ts, Rs = [0.0], [float(R0)]
    R = float(R0)
    for k in range(n):
        k1 = rhs(R)
        k2 = rhs(R + 0.5 * dt * k1)
        k3 = rhs(R + 0.5 * dt * k2)
        k4 = rhs(R + dt * k3)
        R += dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        ts.append((k + 1) * dt)
        Rs.append(R)
        if R_stop is not None and R < R_stop:
            break
    return np.array(ts), np.array(Rs)


def erfc_profile(z, t, D, rho_H):
    """Dirichlet reservoir into an empty half space: rho = rho_H erfc(z / (2 sqrt(D t)))."""
    from scipy.special import erfc
    return rho_H * erfc(np.asarray(z, dtype=np.float64) / (2.0 * math.sqrt(D * t)))


def bulk_pressure(rho_r, rho_b, G, G_rr=0.0, G_bb=0.0):
    """Bulk pressure of the two-component Shan-Chen fluid with Psi = 1 - exp(-rho)
    (Sec. III C): c_s^2 (rho^r + rho^b) + G c_s^2 Psi^r Psi^b, the force of Eq. (3)
    expanded with sum_i w_i e_i e_i = c_s^2 I (the paper prints the interaction term
    with a factor 1/2 that this expansion does not give), plus g^{cc} c_s^2 (Psi^c)^2 / 2
    for self couplings."""
    cs2 = 1.0 / 3.0
    rr = np.asarray(rho_r, np.float64)
    rb = np.asarray(rho_b, np.float64)
    pr = psi(rr)
    pb = psi(rb)
    return cs2 * (rr + rb) + G * cs2 * pr * pb + 0.5 * cs2 * (G_rr * pr * pr + G_bb * pb * pb)
