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


# ---------------------------------------------------------------- diffusion column (Sec. III A)

def _fick2_operator(rc, rb, left_c, left_b, g, tau, closed_left):
    """Banded form of the spatial operator of Eq. (fick2) on sites 1..M (interleaved
    unknowns [c_1, b_1, c_2, b_2, ...]): d rho^a_i / dt = flux_in - flux_out with the
    face flux of Eq. (fick) F^a_{i+1/2} = -sum_b D^{ab}_{i+1/2} (rho^b_{i+1} - rho^b_i),
    D^{ab} of Eq. (diffu-t-1) at the mean of the two sites' densities. Site 0 holds the
    Dirichlet values (left_c, left_b) unless closed_left; the face past site M is closed
    (the halfway wall). Returns (ab, rhs0): ab the (7, 2M) band of the operator for
    scipy.linalg.solve_banded((3, 3), ...), rhs0 the Dirichlet contribution."""
    M = len(rc)
    c = np.concatenate([[left_c], rc])
    b = np.concatenate([[left_b], rb])
    cm, bm = 0.5 * (c[1:] + c[:-1]), 0.5 * (b[1:] + b[:-1])   # faces 1/2 .. M - 1/2
    dcc, dcb = diffusion_matrix(cm, bm, g, tau)     # equation of c: D^{cc}, D^{c cbar}
    dbb, dbc = diffusion_matrix(bm, cm, g, tau)     # equation of cbar: D^{cbar cbar}, D^{cbar c}
    if closed_left:
        dcc, dcb, dbb, dbc = (np.where(np.arange(M) == 0, 0.0, v) for v in (dcc, dcb, dbb, dbc))
    # coefficient of face k (between site k and k + 1, k = 0..M-1) per (equation, variable);
    # unknown 2 i + e is equation e at site i + 1, between faces i and i + 1 (the last closed)
    K = {(0, 0): dcc, (0, 1): dcb, (1, 1): dbb, (1, 0): dbc}
    n = 2 * M
    ab = np.zeros((7, n))
    rhs0 = np.zeros(n)
    for (e, v), Dk in K.items():
        Du = np.concatenate([Dk[1:], [0.0]])              # face above each site
        ab[3 + e - v, v::2] -= Dk + Du                    # the site's own variable
        ab[5 + e - v, v:n - 2:2] += Dk[1:]                # variable of the site below (rows 2..)
        ab[1 + e - v, v + 2::2] += Dk[1:]                 # variable of the site above
        rhs0[e] += Dk[0] * (left_c if v == 0 else left_b)  # the Dirichlet site 0
    return ab, rhs0


def fick2_column(M, times, rho_H, rho_cbar, g, tau=1.0, dt=2.0, rho_c0=None, rho_b0=None, closed_left=False,
                 tol=1e-15, max_iter=50):
    """Eq. (fick2) on the lattice sites of the diffusion column of Sec. III A: site 0 is
    the evaporation boundary (rho^c = rho_H, rho^cbar = rho_cbar - rho_H, the sink's
    complement of a total rho_cbar), sites 1..M hold the fluid (initially rho^c = 0,
    rho^cbar = rho_cbar unless rho_c0 / rho_b0 are given), and the face past site M is
    closed (halfway bounce-back at the wall). Eq. (fick2) is read as the divergence of
    the fluxes of Eq. (fick), d rho^a/dt = div(sum_b D^{ab} grad rho^b), with the
    coefficients of Eq. (diffu-t-1) at the local densities and the sign that makes it
    dissipative; this is the printed form where D is constant, and it conserves mass.
    Finite volumes of unit width, Crank-Nicolson in time with the coefficients at the
    mid-step state, Picard-iterated until the step changes by less than tol. With
    closed_left the face at site 0 is closed as well (site 0 then takes no part).
    Returns {t: (rho_c[1..M], rho_cbar[1..M])} for t in times (multiples of dt)."""
    from scipy.linalg import solve_banded
    rc = np.zeros(M) if rho_c0 is None else np.array(rho_c0, np.float64)
    rb = np.full(M, float(rho_cbar)) if rho_b0 is None else np.array(rho_b0, np.float64)
    lc, lb = float(rho_H), float(rho_cbar) - float(rho_H)
    out = {}
    t = 0.0
    want = sorted(times)
    for T in want:
        nsteps = int(round((T - t) / dt))
        for _ in range(nsteps):
            x0 = np.empty(2 * M)
            x0[0::2], x0[1::2] = rc, rb
            x = x0.copy()
            for _ in range(max_iter):
                mid = 0.5 * (x0 + x)
                ab, rhs0 = _fick2_operator(mid[0::2], mid[1::2], lc, lb, g, tau, closed_left)
                # (I - dt/2 L) x1 = (I + dt/2 L) x0 + dt * rhs0
                Lx0 = rhs0 * 0.0
                for d in range(-3, 4):
                    row = ab[3 - d]
                    if d >= 0:
                        Lx0[: 2 * M - d] += row[d:] * x0[d:]
                    else:
                        Lx0[-d:] += row[: 2 * M + d] * x0[: 2 * M + d]
                A = -0.5 * dt * ab
                A[3] += 1.0
                x1 = solve_banded((3, 3), A, x0 + 0.5 * dt * Lx0 + dt * rhs0)
                done = np.max(np.abs(x1 - x)) <= tol
                x = x1
                if done:
                    break
            rc, rb = x[0::2].copy(), x[1::2].copy()
        t += nsteps * dt
        out[T] = (rc.copy(), rb.copy())
    return out
