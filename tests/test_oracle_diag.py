"""Pins for the oracle's observables of Sec. III: the interface position x_I of
the film (Sec. III B: where rho^c - rho^cbar = 0, here the first downward zero of
the plane mean phi(z) = <rho^r - rho^b>_xy above the liquid base, interpolated
linearly between the two planes around it) and the droplet radius of Sec. III C
(R = (3 V / 4 pi)^(1/3), V the number of sites with rho^r > rho^b).

Every state is built by hand as rest populations w_i rho^c(x) of prescribed
density fields, so the expected value is known in closed form: a zero of a
piecewise-linear profile, or a count of sites. The fields vary across x and y
with zero plane mean, so only the plane mean decides x_I.

The checks are functions of an oracle library so that tests/test_oracle_mutants.py
can run the same checks against copies of the oracle with a planted mistake.
"""
import math

import numpy as np
import pytest

Q = 19


def _weights(oracle_mod):
    _, w, _ = oracle_mod.tables()
    return w


def _state(oracle_mod, rho_r, rho_b):
    """Rest populations f_i^c = w_i rho^c of two (nz, ny, nx) density fields."""
    w = _weights(oracle_mod)
    f = np.empty((2, Q) + rho_r.shape)
    f[0] = w[:, None, None, None] * rho_r[None]
    f[1] = w[:, None, None, None] * rho_b[None]
    return f


def _film_fields(phi, nx=3, ny=2, seed=0):
    """Density fields with plane means rho^r - rho^b = phi(z): rho^r = 0.5 + phi/2 + d,
    rho^b = 0.5 - phi/2 + d', where d, d' vary over (x, y) with zero mean per plane."""
    rng = np.random.default_rng(seed)
    nz = len(phi)
    d = rng.uniform(-0.05, 0.05, (nz, ny, nx))
    d -= d.mean(axis=(1, 2), keepdims=True)
    e = rng.uniform(-0.05, 0.05, (nz, ny, nx))
    e -= e.mean(axis=(1, 2), keepdims=True)
    phi = np.asarray(phi, np.float64)[:, None, None]
    return 0.5 + 0.5 * phi + d, 0.5 - 0.5 * phi + e


def _interface(oracle_mod, phi, library=None, **geom):
    nz = len(phi)
    rr, rb = _film_fields(phi)
    p = dict(nx=rr.shape[2], ny=rr.shape[1], nz=nz, geometry=0)
    p.update(geom)
    o = oracle_mod.Lattice(p, library=library)
    o.set_populations(_state(oracle_mod, rr, rb))
    return o.diagnostics()["interface_z"]


def _pw_linear(nz, knots):
    """phi(z) linear between (z, value) knots, constant beyond the ends."""
    zs, vs = zip(*knots)
    return np.interp(np.arange(nz, dtype=np.float64), zs, vs)


# Each case: (profile, extra geometry, expected x_I). The expected values are the
# zeros of the piecewise-linear profiles, worked out by hand.
def _cases():
    nz = 64
    # a straight line through zero at z = 40.3 (slope -0.013): x_I = 40.3
    line = -0.013 * (np.arange(nz) - 40.3)
    # different slopes on the two sides of the crossing: phi(40) = 0.3, phi(41) = -0.1,
    # so x_I = 40 + 0.3 / 0.4 = 40.75 (the planes 39 and 42 lie off that line)
    kink = _pw_linear(nz, [(0, 0.7), (39, 0.7), (40, 0.3), (41, -0.1), (42, -0.6), (63, -0.6)])
    # an upward crossing first (between z = 4 and 5), then the downward one at
    # phi(30) = 0.12, phi(31) = -0.28: x_I = 30.3
    updown = _pw_linear(nz, [(0, -0.2), (4, -0.2), (5, 0.4), (29, 0.4), (30, 0.12), (31, -0.28), (63, -0.28)])
    # two downward crossings: phi(20) = 0.05, phi(21) = -0.15 (x_I = 20.25), and a
    # second one at phi(50) = 0.2, phi(51) = -0.2 (50.5) that must be ignored
    two = _pw_linear(nz, [(0, 0.5), (19, 0.5), (20, 0.05), (21, -0.15), (35, -0.15), (36, 0.3),
                          (50, 0.2), (51, -0.2), (63, -0.2)])
    # a wall z in {10, 11}: a downward crossing below it (phi(5) = 0.1, phi(6) = -0.3,
    # 5.25) lies under the liquid base z = 12 and is ignored; the next downward one,
    # phi(33) = 0.06, phi(34) = -0.34, gives 33.15
    walled = _pw_linear(nz, [(0, 0.3), (4, 0.3), (5, 0.1), (6, -0.3), (9, -0.3), (12, 0.5), (32, 0.5),
                             (33, 0.06), (34, -0.34), (63, -0.34)])
    # no downward crossing at all: -1
    none = np.full(nz, 0.25)
    return [
        ("line", line, {}, 40.3),
        ("kink", kink, {}, 40.75),
        ("upward_first", updown, {}, 30.3),
        ("two_downward", two, {}, 20.25),
        ("wall_below", walled, dict(wall_z0=10, wall_thickness=2), 33.15),
        ("none", none, {}, -1.0),
    ]


CASES = _cases()


def check_interface_cases(oracle_mod, library=None):
    """Returns the names of the cases whose x_I misses the hand-worked value."""
    bad = []
    for name, phi, geom, want in CASES:
        got = _interface(oracle_mod, phi, library=library, **geom)
        if not abs(got - want) <= 1e-12 * max(1.0, abs(want)):
            bad.append((name, got, want))
    return bad


def _droplet_state(oracle_mod, n=12, V=317, ties=40, seed=3):
    """A lattice with exactly V sites where rho^r > rho^b, `ties` sites where the two
    are equal (not counted: the inequality is strict) and the rest b-rich."""
    rng = np.random.default_rng(seed)
    N = n ** 3
    perm = rng.permutation(N)
    rr = rng.uniform(0.02, 0.05, N)
    rb = rng.uniform(0.6, 0.8, N)
    rich = perm[:V]
    rr[rich], rb[rich] = rng.uniform(0.6, 0.8, V), rng.uniform(0.02, 0.05, V)
    tie = perm[V:V + ties]
    rr[tie] = rb[tie] = rng.uniform(0.1, 0.5, ties)
    return rr.reshape(n, n, n), rb.reshape(n, n, n)


def check_radius(oracle_mod, library=None, V=317):
    n = 12
    rr, rb = _droplet_state(oracle_mod, n, V)
    o = oracle_mod.Lattice(dict(nx=n, ny=n, nz=n, geometry=0), library=library)
    o.set_populations(_state(oracle_mod, rr, rb))
    d = o.diagnostics()
    want = (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0)
    ok = d["droplet_sites"] == V and abs(d["radius"] - want) <= 1e-14 * want
    return ok, d["droplet_sites"], d["radius"], want


@pytest.mark.parametrize("case", [c[0] for c in CASES])
def test_interface_position_of_hand_built_profiles(oracle_mod, case):
    name, phi, geom, want = next(c for c in CASES if c[0] == case)
    got = _interface(oracle_mod, phi, **geom)
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (name, got, want)


def test_profile_is_the_plane_mean(oracle_mod):
    """phi(z) of the oracle equals the prescribed plane means (the per-site fields
    vary across the plane); all-solid planes are NaN."""
    name, phi, geom, _ = CASES[4]
    rr, rb = _film_fields(phi)
    o = oracle_mod.Lattice(dict(nx=rr.shape[2], ny=rr.shape[1], nz=len(phi), geometry=0, **geom))
    o.set_populations(_state(oracle_mod, rr, rb))
    got = o.profile()
    solid = np.zeros(len(phi), bool)
    solid[10:12] = True
    assert np.all(np.isnan(got[solid]))
    assert np.allclose(got[~solid], phi[~solid], rtol=0, atol=1e-14)


@pytest.mark.parametrize("V", [0, 1, 317, 1000])
def test_radius_of_a_known_site_count(oracle_mod, V):
    ok, got_v, got_r, want = check_radius(oracle_mod, V=V)
    assert ok, (got_v, V, got_r, want)
