"""The z-slab decomposition on the GPU: 2, 3 and 5 slab handles of one lattice on one
device, exchanging their ghost planes through the library's pack/unpack and device
copies before every step, hold in their own planes exactly what one lattice stepped
by sc_lbm_step holds (walls, planar sinks across the periodic seam, the spherical
sink, self couplings, FP32, FP16, BF16 and scaled FP16 storage), from the seeded initial state of the
whole lattice; their diagnostics add up to the whole lattice's."""
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


def _cases():
    from paper_1701_03637_gb300.workloads import droplet, film_4x4x128
    out = {}
    p, i = film_4x4x128(rho_hi=0.7, rho_lo=0.04, rho_H=0.01)
    p.update(nx=8, ny=6, nz=40, sink_z0=39)
    i.update(film_z=12)
    out["film_wall_sink"] = (p, i)
    p, i = droplet(24, 6.0, 5)  # two-layer planar sink across the z seam
    p.update(nx=24, ny=20)
    out["droplet_seam_sink"] = (p, i)
    p, i = droplet(20, 5.0, 3, spherical_sink=True)
    p.update(G_rr=-0.9, G_bb=0.4, tau_r=0.95, tau_b=1.1)
    out["sphere_sink_self_couplings"] = (p, i)
    return out


CASES = _cases()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f16s"])
@pytest.mark.parametrize("parts", [2, 3, 5])
@pytest.mark.parametrize("case", list(CASES))
def test_slabs_equal_one_lattice(sc, case, parts, storage):
    from paper_1701_03637_gb300.slab import LocalSlabs
    params, init = CASES[case]
    params = dict(params, storage=storage)
    steps = 37
    whole = sc.Lattice(params)
    whole.init(init)
    whole.step(steps)
    f = whole.read_populations()
    d = whole.diagnostics()
    slabs = LocalSlabs(params, parts)
    slabs.init(init)
    slabs.step(steps)
    slabs.sync()  # the ghosts of the current buffer, before the state is read
    mass_r = mass_b = evap = 0.0
    sites = 0
    for s in slabs.slabs:
        fl = s.read_populations()
        assert np.array_equal(fl[:, :, s.own], f[:, :, s.z0:s.z1]), (case, parts, storage, s.z0)
        ds = s.diagnostics()
        mass_r += ds["mass_r"]
        mass_b += ds["mass_b"]
        evap += ds["evaporated_mass"]
        sites += ds["droplet_sites"]
        assert ds["status"] == 0
    assert sites == d["droplet_sites"]
    for got, want in ((mass_r, d["mass_r"]), (mass_b, d["mass_b"]), (evap, d["evaporated_mass"])):
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (got, want)
    slabs.close()
    whole.close()


def test_slab_validation(sc):
    from paper_1701_03637_gb300.slab import Slab
    params, _ = CASES["droplet_seam_sink"]
    for z0, z1 in ((-1, 4), (3, 4), (10, 25), (5, 5)):
        with pytest.raises(sc.ScError, match="-1"):
            Slab(params, z0, z1)
    with pytest.raises(sc.ScError, match="-1"):
        Slab(dict(params, layout="aa"), 0, 12)
