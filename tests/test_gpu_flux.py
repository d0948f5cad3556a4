"""The relative flux of Sec. III A computed on the device (sc_lbm_flux_profile:
j^r = rho^r (U^r - U) with the velocities of Eq. (velw), tau = 1, per-plane means)
against the oracle's evaluation (orc_flux_field) of the same canonical state:
the GPU's populations are read out and given to the oracle, so both evaluate the
definition in FP64 on the same state. They differ only where the oracle re-forms
the sink populations in FP64 from the GPU's FP32 reset values (about 1e-9 of a
density next to sinks), far inside the 1e-6 of the profile's scale allowed."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


def _oracle_profile(oracle_mod, params, f):
    o = oracle_mod.Lattice(params)
    o.set_populations(f)
    j = o.flux_field()  # [3][z][y][x], 0 at sink and solid sites
    return j.mean(axis=(2, 3))


@pytest.mark.parametrize("layout", ["two", "aa"])
@pytest.mark.parametrize("case", ["wall_and_sink", "self_couplings", "sphere_sink"])
def test_flux_profile_matches_the_oracle(sc, oracle_mod, case, layout):
    from paper_1701_03637_gb300.workloads import random_populations
    nx, ny, nz = 6, 5, 12
    p = dict(nx=nx, ny=ny, nz=nz, G=3.1, geometry=1, sink_z0=0, sink_layers=1, wall_z0=nz - 2, wall_thickness=2)
    if case == "self_couplings":
        p.update(G_rr=-0.7, G_bb=0.3)
    if case == "sphere_sink":
        p = dict(nx=9, ny=8, nz=10, G=3.4, geometry=2, sphere_cx=4.0, sphere_cy=4.0, sphere_cz=5.0, R_H=3.5)
        nx, ny, nz = 9, 8, 10
    g = sc.Lattice(dict(p, layout=layout))
    g.write_populations(random_populations(nx, ny, nz, seed=31, rho=(0.3, 0.6)))
    for steps in (0, 3):
        g.step(steps)
        got = g.flux_profile()
        want = _oracle_profile(oracle_mod, p, g.read_populations())
        scale = np.max(np.abs(want))
        assert scale > 1e-5, "a state with a real flux"
        assert np.max(np.abs(got - want)) <= 1e-6 * scale, (case, layout, steps, got - want)
    g.close()


def test_flux_profile_needs_tau_one(sc):
    g = sc.Lattice(dict(nx=4, ny=4, nz=8, tau_r=0.9, tau_b=0.9))
    with pytest.raises(sc.ScError, match="-1"):
        g.flux_profile()
    g.close()
