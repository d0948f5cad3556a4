"""Radius change predicted by the Laplace-corrected droplet law, Eq. (drop-r-df4),
integrated with classic RK4 from a measured state (test helper)."""


def law_dR(A, R_start, T, R0, gamma, run, d0=2.5, dt=10.0):
    """Radius change over T steps from R_start: dR/dt = (mass rate of Eq. (mass-df1)
    with the Laplace-corrected vapour density) / dM/dR of Eq. (drop-mass-1), the
    vapour D^c of Sec. III A at the corrected vapour density; gamma = 0 drops the
    Laplace correction. `run` carries the measured coexistence densities
    (rho_ma0, rho_mi0, rho_b_out), R_H, rho_H and G."""
    def rhs(R):
        _, mi = A.laplace_densities(R, R0, gamma, run["rho_ma0"], run["rho_mi0"])
        D = float(A.diffusion_coefficient(mi, run["rho_b_out"], run["G"]))
        return A.drop_mass_rate(R, run["R_H"], d0, D, mi, run["rho_H"]) / A._dMdR(
            R, run["R_H"], d0, run["rho_ma0"], run["rho_mi0"], run["rho_H"], R0=R0, gamma=gamma)

    R = R_start
    for _ in range(int(round(T / dt))):
        k1 = rhs(R)
        k2 = rhs(R + 0.5 * dt * k1)
        k3 = rhs(R + 0.5 * dt * k2)
        k4 = rhs(R + dt * k3)
        R += dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return R - R_start
