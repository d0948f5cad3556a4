"""The diagnostics entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (their allocator is owned by someone else,
or their memory budget is fixed before the library runs), so
sc_lbm_diagnostics_noalloc keeps its scratch in a file-scope device array and
writes its results into memory the caller already owns. This checks it, through
the C ABI, against sc_lbm_diagnostics on two calls in a row. It lives in a file
of its own that pytest collects last, and must pass alone in a fresh process as
well as after the other tests.
"""
import ctypes as C
import math

import pytest

pytestmark = pytest.mark.gpu

FIELDS = ["mass_r", "mass_b", "evaporated_mass", "flux_last", "interface_z", "radius", "droplet_sites", "status"]


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


def _noalloc(sc, lat, out):
    from paper_1701_03637_gb300 import _native
    rc = _native.load().sc_lbm_diagnostics_noalloc(lat.handle, C.c_void_p(out.data_ptr()))
    _native.check(rc)
    lat.sync()
    return dict(zip(FIELDS, out.cpu().tolist()))


def _close(a, b, rel):
    return abs(a - b) <= rel * max(1.0, abs(b))


@pytest.mark.parametrize("case,storage", [("droplet_sphere_sink", "f32"), ("film_wall_sink", "f32"),
                                          ("droplet_sphere_sink_in_place", "f32"), ("droplet_sphere_sink", "f16"),
                                          ("droplet_sphere_sink", "f16s"), ("droplet_sphere_sink", "bf16"),
                                          ("droplet_sphere_sink_in_place", "f16")])
def test_noalloc_matches_diagnostics_twice(sc, case, storage):
    import torch
    from paper_1701_03637_gb300.workloads import droplet, film_4x4x128
    if case.startswith("droplet_sphere_sink"):
        params, init = droplet(40, 9.0, 11, spherical_sink=True)
    else:
        params, init = film_4x4x128(rho_hi=0.7, rho_lo=0.04, rho_H=0.01)
    params["storage"] = storage
    if case.endswith("in_place"):
        params["layout"] = "aa"  # 40 steps: even form, 65 steps: odd form
    lat = sc.Lattice(params)
    lat.init(init)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (40, 25):
        lat.step(steps)
        got = _noalloc(sc, lat, out)
        ref = lat.diagnostics()
        # same partial sums, folded in the same order on the device: equal to
        # rounding (the cube root of the radius may differ in its last ulp)
        for k in ("mass_r", "mass_b", "evaporated_mass", "flux_last", "interface_z"):
            assert _close(got[k], ref[k], 1e-12), (k, got[k], ref[k])
        assert math.isclose(got["radius"], ref["radius"], rel_tol=1e-12, abs_tol=1e-12)
        assert int(got["droplet_sites"]) == ref["droplet_sites"]
        assert int(got["status"]) == ref["status"] == 0
    lat.close()


def test_noalloc_limit_is_nz_32768(sc):
    """One part per plane for nz >= 608, 8 doubles per part, 262144 doubles of
    scratch: nz = 32768 fits exactly, nz = 32769 is rejected."""
    import torch
    from paper_1701_03637_gb300 import _native
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    ok = sc.Lattice(dict(nx=1, ny=1, nz=32768))
    ok.init(dict(shape=0, film_z=100, rho_hi=0.7, rho_lo=0.04))
    got = _noalloc(sc, ok, out)
    ref = ok.diagnostics()
    assert _close(got["mass_r"], ref["mass_r"], 1e-12) and got["interface_z"] == ref["interface_z"]
    ok.close()
    lat = sc.Lattice(dict(nx=1, ny=1, nz=32769))
    rc = _native.load().sc_lbm_diagnostics_noalloc(lat.handle, C.c_void_p(out.data_ptr()))
    assert rc == -1
    assert b"limit" in _native.load().sc_last_error()
    lat.close()
