"""Pin of the oracle's relative flux of Eqs. (flux) and (velw): a literal numpy
writing of the definition (tests/flux_literal.py, on the canonical populations)
equals the oracle's own C evaluation (`orc_flux_field`) on the same state: two
independent writings of the paper's definition (tau = 1, cross coupling only)."""
import numpy as np


def test_paper_flux_matches_the_oracle(oracle_mod):
    from tests.flux_literal import paper_flux_z
    from paper_1701_03637_gb300.workloads import random_populations
    nx, ny, nz = 6, 5, 12
    p = dict(nx=nx, ny=ny, nz=nz, G=3.1, geometry=1, sink_z0=0, sink_layers=1, wall_z0=nz - 2, wall_thickness=2)
    o = oracle_mod.Lattice(p)
    o.set_populations(random_populations(nx, ny, nz, seed=31, rho=(0.3, 0.6)))
    o.step(3)
    f = o.populations()
    c, w, _ = oracle_mod.tables()
    j = paper_flux_z(f, c, w, p["G"])
    jo = o.flux_field()[2]
    fluid = np.ones((nz, ny, nx), bool)
    fluid[0] = False             # sink plane
    fluid[nz - 2:] = False       # wall
    assert np.array_equal(o.site_class() == 0, fluid)
    assert np.max(np.abs(j[fluid] - jo[fluid])) < 1e-14
    assert np.max(np.abs(jo[fluid])) > 1e-4  # a state with a real flux
