"""Pin: the oracle's time step equals an independent literal evaluation of
Sec. II (tests/brute_force.py) on tiny lattices, after 1 and 10 steps, to FP64
rounding, for periodic, walled + planar-sink, spherical-sink and unequal-tau
cases."""
import numpy as np
import pytest

from tests.brute_force import BruteForce, VELOCITIES, W

CASES = {
    "periodic_3x3x3": dict(nx=3, ny=3, nz=3, tau_r=1.0, tau_b=1.0, G=3.6, rho_H=0.03, geometry=0),
    "wall_sink_unequal_tau_4x4x8": dict(nx=4, ny=4, nz=8, tau_r=0.85, tau_b=1.3, G=3.2, rho_H=0.05,
                                        geometry=1, sink_z0=7, sink_layers=1, wall_z0=0, wall_thickness=2),
    "seam_sink_4x3x5": dict(nx=4, ny=3, nz=5, tau_r=1.0, tau_b=1.0, G=3.6, rho_H=0.03, geometry=1,
                            sink_z0=4, sink_layers=2),
    "sphere_sink_5x5x5": dict(nx=5, ny=5, nz=5, tau_r=1.1, tau_b=0.9, G=2.5, rho_H=0.04, geometry=2,
                              sphere_cx=2.0, sphere_cy=2.0, sphere_cz=2.0, R_H=2.0),
}


def test_brute_force_table_is_d3q19():
    assert len(VELOCITIES) == 19
    assert abs(sum(W) - 1.0) < 1e-15
    for a in range(3):
        for b in range(3):
            m = sum(w * e[a] * e[b] for w, e in zip(W, VELOCITIES))
            assert abs(m - (1.0 / 3.0 if a == b else 0.0)) < 1e-15


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_equals_brute_force(oracle_mod, name):
    p = CASES[name]
    c_oracle, _, _ = oracle_mod.tables()
    o = oracle_mod.Lattice(p)
    rng = np.random.default_rng(sum(map(ord, name)))
    f = rng.uniform(0.7, 1.3, (2, 19, p["nz"], p["ny"], p["nx"])) / 19.0
    f[0] *= 0.8
    f[1] *= 0.25
    o.set_populations(f)
    state = o.populations()
    bf = BruteForce(p)
    g = bf.from_array(state, c_oracle)
    done = 0
    for target in (1, 10):
        o.step(target - done)
        while done < target:
            g = bf.step(g)
            done += 1
        got = o.populations()
        want = bf.to_array(g, c_oracle)
        assert np.max(np.abs(got - want)) < 1e-14, (name, target, np.max(np.abs(got - want)))
        d = o.diagnostics()
        assert abs(d["evaporated_mass"] - bf.evaporated) < 1e-13
