"""Coexistence densities of the single-component pseudopotential fluid (test helper)."""
import numpy as np


def sc_coexistence(g):
    """Liquid and vapour densities of the single-component pseudopotential fluid with
    Psi = 1 - exp(-rho) (Eq. (4)) and p = c_s^2 rho + (g c_s^2 / 2) Psi^2 (the
    self-coupling force of Eq. (3) expanded to second order): p(rho_g) = p(rho_l) = p0
    and the integral of (p0 - p) Psi' / Psi^2 from rho_g to rho_l vanishes (Shan and
    Chen's mechanical-stability condition, which replaces Maxwell's equal areas for
    this force). Returns (rho_g, rho_l)."""
    from scipy import integrate, optimize
    cs2 = 1.0 / 3.0

    def psi(r):
        return -np.expm1(-r)

    def p(r):
        return cs2 * r + 0.5 * g * cs2 * psi(r) ** 2

    def eqs(v):
        rg, rl = v
        p0 = p(rg)
        area = integrate.quad(lambda r: (p0 - p(r)) * np.exp(-r) / psi(r) ** 2, rg, rl, epsabs=1e-13)[0]
        return [p(rl) - p0, area]

    return optimize.fsolve(eqs, [0.1, 2.0], xtol=1e-13)
