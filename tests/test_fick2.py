"""The numerical solution of Eq. (fick2) (oracle/analytic.py: fick2_column, finite
volumes on the lattice sites, Crank-Nicolson with Picard iteration) pinned to what
fixes it independently, then the oracle's lattice Boltzmann column of Sec. III A
compared with it.

Pins: with g = 0 the coefficients of Eq. (diffu-t-1) give a flux -c_s^2 (tau - 1/2)
grad rho^c at uniform total density, so the solution is the erfc of a Dirichlet
half space with D = 1/6; with both ends closed every component's mass is exact;
halving the time step changes nothing at second order; exchanging the two
components' initial profiles exchanges the solutions (the second equation uses
the coefficient matrix with the roles swapped)."""
import numpy as np
import pytest

from oracle import analytic as A


def test_g0_is_the_erfc_half_space():
    M, T, rH = 122, 2000, 0.001
    c, b = A.fick2_column(M, [T], rH, 0.7, 0.0, dt=2.0)[T]
    z = np.arange(1, M + 1)
    # the semi-discrete solution differs from the continuous erfc by O(dx^2 / (D t))
    assert np.max(np.abs(c - A.erfc_profile(z, T, 1.0 / 6.0, rH))) < 2e-4 * rH
    assert np.max(np.abs(c + b - 0.7)) < 1e-12  # the total stays uniform


@pytest.mark.parametrize("g", [0.0, 3.6])
def test_closed_column_conserves_each_mass(g):
    rng = np.random.default_rng(1)
    c0, b0 = rng.uniform(0, 0.01, 50), 0.7 + rng.uniform(-0.01, 0.01, 50)
    c1, b1 = A.fick2_column(50, [400], 0.001, 0.7, g, rho_c0=c0, rho_b0=b0, closed_left=True)[400]
    assert abs(c1.sum() - c0.sum()) < 1e-12 and abs(b1.sum() - b0.sum()) < 1e-12
    assert c1.std() < 0.2 * c0.std()  # and it diffuses


def test_time_step_convergence():
    a = A.fick2_column(122, [10000], 0.001, 0.7, 3.6, dt=2.0)[10000][0]
    b = A.fick2_column(122, [10000], 0.001, 0.7, 3.6, dt=1.0)[10000][0]
    assert np.max(np.abs(a - b)) < 1e-7 * 0.001


def test_exchanging_the_components_exchanges_the_solution():
    rng = np.random.default_rng(2)
    p, q = 0.3 + rng.uniform(0, 0.05, 30), 0.4 + rng.uniform(0, 0.05, 30)
    # g = 1.5 keeps D^c > 0 at these densities (g = 3.1 would put them inside the spinodal,
    # where D^c < 0 and Eq. (fick2) is ill-posed)
    c1, b1 = A.fick2_column(30, [200], 0.0, 0.7, 1.5, rho_c0=p, rho_b0=q, closed_left=True)[200]
    c2, b2 = A.fick2_column(30, [200], 0.0, 0.7, 1.5, rho_c0=q, rho_b0=p, closed_left=True)[200]
    assert np.max(np.abs(c1 - b2)) < 1e-14 and np.max(np.abs(b1 - c2)) < 1e-14
    assert np.max(np.abs(c1 - p)) > 1e-4  # the profiles did move


def _paper_column(oracle_mod, times, nz=125, nxy=4, rH=0.001, rb0=0.7, g=3.6):
    """The diffusion experiment of Sec. III A in the oracle: 125 x 4 x 4 sites, the
    evaporation boundary at site 0 (rho_H = 0.001), a wall of thickness 2 at the far end
    (sites 123 and 124), the column filled with rho^cbar = 0.7."""
    p = dict(nx=nxy, ny=nxy, nz=nz, tau_r=1.0, tau_b=1.0, G=g, rho_H=rH, geometry=1, sink_z0=0, sink_layers=1,
             wall_z0=nz - 2, wall_thickness=2)
    o = oracle_mod.Lattice(p)
    o.init_fields(np.zeros((nz, nxy, nxy)), np.full((nz, nxy, nxy), rb0))
    out, done = {}, 0
    for T in times:
        o.step(T - done)
        done = T
        rr, rb = o.fields()
        out[T] = (rr.mean(axis=(1, 2))[1:nz - 2], rb.mean(axis=(1, 2))[1:nz - 2])
    return out


def test_oracle_column_follows_fick2(oracle_mod):
    """The whole profile of the lattice Boltzmann column against the solution of Eq.
    (fick2) with the same boundary values, except the fluid site next to the wall: there
    the force of Eq. (3) sees Psi = 0 at the solid sites (the walls carry no
    pseudopotential), so the trace component is drawn onto the wall and that one site
    holds more of it than diffusion alone gives (+0.75% of rho_H at step 5000, +10% at
    10000)."""
    rH, times = 0.001, [3000, 10000]
    lb = _paper_column(oracle_mod, times)
    cn = A.fick2_column(122, times, rH, 0.7, 3.6, dt=2.0)
    tol = {3000: 1e-3, 10000: 5e-3}  # measured 6e-4 and 3.1e-3 of rho_H
    for T in times:
        (lc, lb_), (c, b) = lb[T], cn[T]
        assert np.max(np.abs(lc[:-1] - c[:-1])) < tol[T] * rH, T
        assert np.max(np.abs(lb_[:-1] - b[:-1])) < 2e-3, T
        assert lc[-1] > c[-1]  # the wall site's excess
        assert abs(lc.sum() - c.sum()) < 2e-3 * c.sum()  # the mass that entered agrees to 0.2%
