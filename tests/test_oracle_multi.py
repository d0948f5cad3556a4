"""Pins of the N-component oracle (oracle/multi.py, Eq. (3) summed over every
component cbar): with two components it is the two-component C oracle (a separate
implementation pinned in tests/test_oracle.py); an absent third component changes
nothing; each component's mass and, with symmetric couplings on a periodic
lattice, the total momentum are exact; relabelling the components relabels the
result."""
import numpy as np
import pytest

from oracle import multi

Q = 19


def _state(n, shape, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 0.6, (n,) + shape)
    f = rng.uniform(0.7, 1.3, (n, Q) + shape) / Q
    return f * rho[:, None]


def test_directions_match_the_two_component_oracle(oracle_mod):
    c, w, opp = oracle_mod.tables()
    assert np.array_equal(multi.E, c) and np.allclose(multi.W, w, rtol=0, atol=0)
    assert np.array_equal(multi.OPP, opp)


@pytest.mark.parametrize("wall", [0, 2])
def test_two_components_equal_the_c_oracle(oracle_mod, wall):
    nx, ny, nz = 5, 4, 9
    tau = (0.9, 1.15)
    g = np.array([[-0.8, 3.3], [3.3, 0.4]])
    f = _state(2, (nz, ny, nx), 3)
    m = multi.Lattice(nx, ny, nz, tau, g, wall_z0=3, wall_thickness=wall)
    o = oracle_mod.Lattice(dict(nx=nx, ny=ny, nz=nz, tau_r=tau[0], tau_b=tau[1], G=3.3, G_rr=-0.8, G_bb=0.4,
                                geometry=0, wall_z0=3, wall_thickness=wall))
    m.set_populations(f)
    o.set_populations(f)
    m.step(5)
    o.step(5)
    assert np.max(np.abs(m.f - o.populations())) < 1e-13


def test_absent_third_component_changes_nothing():
    nx, ny, nz = 4, 5, 6
    g2 = np.array([[0.3, 3.1], [3.1, -0.2]])
    g3 = np.array([[0.3, 3.1, 1.7], [3.1, -0.2, 2.2], [1.7, 2.2, -0.9]])
    f2 = _state(2, (nz, ny, nx), 4)
    f3 = np.concatenate([f2, np.zeros((1, Q, nz, ny, nx))])
    a = multi.Lattice(nx, ny, nz, (1.0, 0.8), g2)
    b = multi.Lattice(nx, ny, nz, (1.0, 0.8, 1.2), g3)
    a.set_populations(f2)
    b.set_populations(f3)
    a.step(4)
    b.step(4)
    assert np.max(np.abs(b.f[:2] - a.f)) < 1e-15 and not b.f[2].any()


@pytest.mark.parametrize("wall", [0, 2])
def test_mass_and_momentum(wall):
    nx, ny, nz = 5, 4, 8
    g = np.array([[-1.0, 2.5, 1.5], [2.5, 0.0, 3.0], [1.5, 3.0, -0.5]])  # symmetric
    m = multi.Lattice(nx, ny, nz, (0.9, 1.0, 1.3), g, wall_z0=2, wall_thickness=wall)
    m.set_populations(_state(3, (nz, ny, nx), 5))
    mass0 = m.densities().sum(axis=(1, 2, 3))
    mom = lambda: np.einsum("cizyx,id->d", m.f, multi.E.astype(np.float64))
    p0 = mom()
    m.step(6)
    assert np.max(np.abs(m.densities().sum(axis=(1, 2, 3)) - mass0)) < 1e-12
    if wall == 0:  # walls take momentum (bounce-back); the periodic lattice keeps it
        assert np.max(np.abs(mom() - p0)) < 1e-13


def test_relabelling_the_components_relabels_the_result():
    nx, ny, nz = 4, 4, 5
    g = np.array([[-0.5, 2.0, 1.0], [2.0, 0.3, 2.6], [1.0, 2.6, -1.1]])
    tau = np.array([0.95, 1.1, 0.85])
    f = _state(3, (nz, ny, nx), 6)
    perm = [2, 0, 1]
    a = multi.Lattice(nx, ny, nz, tau, g)
    b = multi.Lattice(nx, ny, nz, tau[perm], g[np.ix_(perm, perm)])
    a.set_populations(f)
    b.set_populations(f[perm])
    a.step(3)
    b.step(3)
    assert np.max(np.abs(b.f - a.f[perm])) < 1e-14
