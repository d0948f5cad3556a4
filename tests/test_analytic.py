"""Pins for the analytic laws (oracle/analytic.py) against the formulas the paper
prints and against independent numerical solutions."""
import math

import numpy as np
import pytest

from oracle import analytic as A


def test_diffusion_coefficient_limits():
    # g = 0: D = cs^2 (tau - 1/2)
    assert abs(A.diffusion_coefficient(0.3, 0.4, 0.0, tau=1.0) - 1 / 6) < 1e-15
    assert abs(A.diffusion_coefficient(0.3, 0.4, 0.0, tau=0.8) - 0.1) < 1e-15
    # D^c = D^{cc} - D^{c cbar} (Sec. III A, grad rho^cbar = -grad rho^c)
    dcc, dccb = A.diffusion_matrix(0.036, 0.704, 3.6)
    assert abs((dcc - dccb) - A.diffusion_coefficient(0.036, 0.704, 3.6)) < 1e-15
    # an independent evaluation of the Sec. III A formula at the film's printed
    # equilibrium densities (0.036, 0.704)
    assert abs(A.diffusion_coefficient(0.036, 0.704, 3.6) - 0.11824) < 1e-5


def test_film_closed_form_solves_ode():
    args = dict(x0=64.0, x_H=128.0, d0=2.5, D=0.118, rho_ma=0.704, rho_mi=0.036, rho_H=0.02)
    for T in (1e4, 1e5, 1e6):
        x_ode = A.film_xI_rk4(T, 100.0, **args)
        assert abs(x_ode - A.film_xI(T, **args)) < 1e-8
    # the printed Eq. (xt) differs from the ODE solution by O(d0 K t / (x_H - x0)^2)
    assert abs(A.film_xI_printed(1e6, **args) - A.film_xI(1e6, **args)) > 0.1


@pytest.mark.parametrize("R", [8.0, 20.0, 40.0, 65.0])
def test_droplet_mass_derivative_matches_printed(R):
    """Eq. (mass-df2) is d/dR of Eq. (drop-mass-1)."""
    args = (126.0, 2.5, 0.712, 0.037, 0.03)
    assert abs(A._dMdR(R, *args) / A.drop_dMdR_printed(R, *args) - 1) < 1e-9


@pytest.mark.parametrize("R", [8.0, 20.0, 40.0, 65.0])
def test_droplet_laplace_mass_derivative_matches_printed(R):
    """Eq. (drop-mass-df4) is d/dR of Eq. (drop-mass-1) with Eqs. (rho_ma), (rho_mi)."""
    R_H, d0, R0, gam, ma0, mi0, rH = 126.0, 2.5, 65.0, 0.08, 0.712, 0.037, 0.03
    num = A._dMdR(R, R_H, d0, ma0, mi0, rH, R0=R0, gamma=gam)
    assert abs(num / A.drop_dMdR_laplace_printed(R, R_H, d0, R0, gam, ma0, mi0, rH) - 1) < 1e-9


def test_droplet_mass_closed_form_matches_quadrature():
    from scipy.integrate import quad
    R, R_H, d0, ma, mi, rH = 30.0, 100.0, 2.5, 0.712, 0.037, 0.02

    def dens(r):
        if r < R - d0:
            return ma
        if r < R + d0:
            return mi - (mi - ma) * (R + d0 - r) / (2 * d0) * (R - d0) / r
        return rH - (rH - mi) * (R_H - r) / (R_H - R - d0) * (R + d0) / r

    q = sum(quad(lambda r: 4 * math.pi * r * r * dens(r), a, b, epsabs=1e-10)[0]
            for a, b in ((0, R - d0), (R - d0, R + d0), (R + d0, R_H)))
    assert abs(A.drop_mass(R, R_H, d0, ma, mi, rH) / q - 1) < 1e-10


def test_droplet_rk4_step_size_converged_and_shrinks():
    kw = dict(R_H=126.0, d0=2.5, D=0.118, rho_ma=0.712, rho_mi=0.037, rho_H=0.02)
    t1, R1 = A.droplet_radius_rk4(65.0, 2e5, 100.0, **kw)
    t2, R2 = A.droplet_radius_rk4(65.0, 2e5, 50.0, **kw)
    assert abs(R1[-1] - R2[-1]) < 1e-6
    assert np.all(np.diff(R1) < 0)
    # Laplace pressure speeds up the late stage (Sec. III C)
    _, R3 = A.droplet_radius_rk4(65.0, 2e5, 100.0, gamma=0.08, **kw)
    assert R3[-1] < R1[-1]


def test_erfc_profile_boundary():
    assert A.erfc_profile(0.0, 100.0, 0.1, 0.001) == pytest.approx(0.001)
    assert A.erfc_profile(1e3, 100.0, 0.1, 0.001) < 1e-12
