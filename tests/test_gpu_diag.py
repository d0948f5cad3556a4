"""The GPU diagnostics on hand-built states whose observables are known in closed
form (the states of tests/test_oracle_diag.py): the interface position x_I of
Sec. III B as the first downward zero of the plane mean of rho^r - rho^b above
the liquid base, linearly interpolated, and the droplet radius of Sec. III C from
the count of sites with rho^r > rho^b. Both the synchronous diagnostics and the
no-allocation entry point are checked, in both population layouts. The states
pass through FP32 storage, so x_I carries the FP32 rounding of the densities
(about 1e-8 of a density over a slope of 1e-2: the test allows 1e-5)."""
import ctypes as C
import math

import numpy as np
import pytest

import test_oracle_diag as cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


class _W:
    """Rest-population weights for the state builder (the library's own table)."""

    def __init__(self, sc):
        self.w = sc.lattice_directions()[1]

    def tables(self):
        return None, self.w, None


def _noalloc(lat):
    import torch
    from paper_1701_03637_gb300 import _native
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    _native.check(_native.load().sc_lbm_diagnostics_noalloc(lat.handle, C.c_void_p(out.data_ptr())))
    lat.sync()
    v = out.cpu().tolist()
    return {"interface_z": v[4], "radius": v[5], "droplet_sites": int(v[6])}


@pytest.mark.parametrize("layout", ["two", "aa"])
@pytest.mark.parametrize("case", [c[0] for c in cases.CASES])
def test_interface_position_of_hand_built_profiles(sc, case, layout):
    name, phi, geom, want = next(c for c in cases.CASES if c[0] == case)
    rr, rb = cases._film_fields(phi)
    p = dict(nx=rr.shape[2], ny=rr.shape[1], nz=len(phi), geometry=0, layout=layout, **geom)
    lat = sc.Lattice(p)
    lat.write_populations(cases._state(_W(sc), rr, rb))
    for got in (lat.diagnostics()["interface_z"], _noalloc(lat)["interface_z"]):
        if want < 0:
            assert got == -1.0
        else:
            assert abs(got - want) < 1e-5, (name, layout, got, want)
    lat.close()


@pytest.mark.parametrize("layout", ["two", "aa"])
@pytest.mark.parametrize("V", [0, 1, 317, 1000])
def test_radius_of_a_known_site_count(sc, V, layout):
    n = 12
    rr, rb = cases._droplet_state(None, n, V)
    lat = sc.Lattice(dict(nx=n, ny=n, nz=n, geometry=0, layout=layout))
    lat.write_populations(cases._state(_W(sc), rr, rb))
    want = (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0)
    for d in (lat.diagnostics(), _noalloc(lat)):
        assert d["droplet_sites"] == V
        assert math.isclose(d["radius"], want, rel_tol=1e-12, abs_tol=1e-15)
    lat.close()
