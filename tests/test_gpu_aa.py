"""The in-place (AA) layout: the time step of Sec. II on one population lattice
updated in place, by either of its two kernels: the persistent cooperative step
(one launch for many steps, CTAs ordered by bounded neighbour waits, the lattice
marched whole or in x-bands one after another) or the
two-pass step (Psi of every site, then stream + sink + force + collision). The
state either reaches after any number of steps -- in either of its two storage
forms -- is the two-lattice step's, bit for bit, for every storage type, geometry
(walls, planar and spherical sinks) and ragged extent; it also matches the FP64
oracle directly, and checkpoints taken in either form restore into either
layout."""
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
    """Lattices of different extents, parameters and geometries (with their inits)."""
    from paper_1701_03637_gb300.workloads import droplet, film_4x4x128
    out = {}
    out["film_wall_sink"] = film_4x4x128(rho_hi=0.7, rho_lo=0.04, rho_H=0.01)
    p, i = droplet(40, 9.0, 11, spherical_sink=True)
    p.update(nx=37, ny=33, nz=29, sphere_cx=18.0, sphere_cy=16.0, sphere_cz=14.0, R_H=12.0, G=3.4, rho_H=0.025)
    i.update(cx=18.0, cy=16.0, cz=14.0, radius=7.0)
    out["sphere_sink_ragged"] = (p, i)
    p, i = droplet(32, 8.0, 5)
    p.update(tau_r=0.9, tau_b=1.15, G=3.7)
    out["seam_sink_unequal_tau"] = (p, i)
    p, i = droplet(24, 6.0, 9)
    p.update(geometry=0, nx=130, ny=17, nz=21)  # two row segments, the second ragged
    i.update(cx=65.0, cy=8.0, cz=10.0)
    out["periodic_two_segments"] = (p, i)
    p, i = film_4x4x128(rho_hi=0.7, rho_lo=0.04, rho_H=0.02)
    p.update(nx=1, ny=3, nz=12, sink_z0=11, wall_z0=5, wall_thickness=1)
    i.update(film_z=4)
    out["thin_column_mid_wall"] = (p, i)
    p, i = droplet(20, 5.0, 3, spherical_sink=True)
    p.update(nx=20, ny=12, nz=16, sphere_cx=10.0, sphere_cy=6.0, sphere_cz=8.0, R_H=7.0, G_rr=-1.1, G_bb=0.5)
    i.update(cx=10.0, cy=6.0, cz=8.0, radius=4.0)
    out["self_couplings_sphere_sink"] = (p, i)
    return out


CASES = _cases()


STAGINGS = ["persistent", "thread"]


def _run(sc, params, init, steps, layout, staging="auto", bands=None):
    lat = sc.Lattice(dict(params, layout=layout, staging=staging if layout == "aa" else "auto"))
    if layout == "aa" and staging == "persistent":
        assert lat.launch_info()["staging"] == "persistent"
    if bands is not None:
        assert lat.persist_bands(bands) == bands
        assert lat.launch_info()["bands"] == bands
    lat.init(init)
    out = []
    done = 0
    for n in steps:
        lat.step(n - done)
        done = n
        out.append((lat.read_populations(), lat.read_fields(), lat.diagnostics()))
    lat.close()
    return out


def _same_diag(d, ref):
    # the evaporated mass is summed in another order (per row-segment CTA instead of
    # per tile column): equal to FP64 rounding
    for k in ("evaporated_mass", "flux_last"):
        assert abs(d[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, d[k], ref[k])
    for k in ("mass_r", "mass_b", "interface_z", "radius", "droplet_sites", "status", "step"):
        assert d[k] == ref[k], (k, d[k], ref[k])


@pytest.mark.parametrize("staging", STAGINGS)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f16s"])
@pytest.mark.parametrize("case", list(CASES))
def test_same_bits_as_two_lattices(sc, case, storage, staging):
    params, init = CASES[case]
    params = dict(params, storage=storage)
    steps = [1, 2, 7, 77, 150]  # odd and even forms; 64-step graphs replayed from both parities
    aa = _run(sc, params, init, steps, "aa", staging)
    two = _run(sc, params, init, steps, "two")
    for n, (fa, (ra, ba), da), (ft, (rt, bt), dt) in zip(steps, aa, two):
        assert np.array_equal(fa, ft), (case, storage, n)
        assert np.array_equal(ra, rt) and np.array_equal(ba, bt), (case, storage, n)
        _same_diag(da, dt)


# band counts dividing each case's nx (bands of 2 sites included)
BANDS = {"seam_sink_unequal_tau": [2, 4, 16], "periodic_two_segments": [2, 5, 65],
         "self_couplings_sphere_sink": [2, 5, 10], "film_wall_sink": [2]}


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f16s"])
@pytest.mark.parametrize("case,bands", [(c, b) for c, bs in BANDS.items() for b in bs])
def test_bands_same_bits_as_two_lattices(sc, case, bands, storage):
    """The persistent step marching the lattice in x-bands, one after another (halo
    Psi at a band edge saved by the band before or formed from the band after), gives
    the two-lattice step's bits."""
    params, init = CASES[case]
    params = dict(params, storage=storage)
    steps = [1, 2, 7, 77]
    aa = _run(sc, params, init, steps, "aa", "persistent", bands=bands)
    two = _run(sc, params, init, steps, "two")
    for n, (fa, (ra, ba), da), (ft, (rt, bt), dt) in zip(steps, aa, two):
        assert np.array_equal(fa, ft), (case, bands, storage, n)
        assert np.array_equal(ra, rt) and np.array_equal(ba, bt), (case, bands, storage, n)
        _same_diag(da, dt)


def test_band_requests(sc):
    params, init = CASES["seam_sink_unequal_tau"]
    lat = sc.Lattice(dict(params, layout="aa", staging="persistent"))
    assert lat.persist_bands() == 1  # a 32^2 plane is far below the automatic limit
    for bad in (3, 33, -2):  # not a divisor of nx = 32, bands under 2 sites, no such request
        with pytest.raises(sc.ScError, match="-1"):
            lat.persist_bands(bad)
    assert lat.persist_bands() == 1
    assert lat.persist_bands(8) == 8 and lat.launch_info()["tile_x"] <= 4
    assert lat.persist_bands(0) == 1
    lat.close()
    lat = sc.Lattice(dict(params, layout="aa", staging="thread"))
    assert lat.persist_bands() == 0
    with pytest.raises(sc.ScError, match="-1"):
        lat.persist_bands(2)
    lat.close()


@pytest.mark.parametrize("staging", STAGINGS)
@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("case", ["sphere_sink_ragged", "thin_column_mid_wall"])
def test_random_state_matches_oracle(sc, oracle_mod, case, steps, staging):
    """One and two in-place steps (the two forms) of a non-equilibrium state against
    the oracle, within 1e-6 of each population's scale as in the two-lattice tests."""
    from paper_1701_03637_gb300.workloads import random_populations
    params, _ = CASES[case]
    nx, ny, nz = params["nx"], params["ny"], params["nz"]
    _, w = sc.lattice_directions()
    f0 = random_populations(nx, ny, nz, seed=4242 + nx, rho=(0.55, 0.25))
    g = sc.Lattice(dict(params, layout="aa", staging=staging))
    o = oracle_mod.Lattice(params)
    g.write_populations(f0)
    o.set_populations(f0)
    g.step(steps)
    o.step(steps)
    fg, fo = g.read_populations(), o.populations()
    rho = np.abs(fo).sum(axis=1, keepdims=True)
    den = np.maximum(np.maximum(np.abs(fo), w[None, :, None, None, None] * rho), 1e-30)
    assert np.max(np.abs(fg - fo) / den) < 1e-6 * steps
    dg, do = g.diagnostics(), o.diagnostics()
    assert abs(dg["mass_r"] - do["mass_r"]) <= 1e-6 * abs(do["mass_r"])
    assert abs(dg["mass_b"] - do["mass_b"]) <= 1e-6 * abs(do["mass_b"])
    assert abs(dg["evaporated_mass"] - do["evaporated_mass"]) <= 1e-6 * max(1.0, abs(do["mass_r"]))
    g.close()


@pytest.mark.parametrize("staging", STAGINGS)
@pytest.mark.parametrize("case", ["sphere_sink_ragged", "film_wall_sink"])
def test_checkpoint_from_either_form_restores_into_either_layout(sc, case, staging):
    params, init = CASES[case]
    src = sc.Lattice(dict(params, layout="aa", staging=staging))
    src.init(init)
    for taken_at in (3, 8):  # odd form, then even form
        src.step(taken_at - src.diagnostics()["step"])
        f = src.read_populations()
        d = src.diagnostics()
        results = []
        for layout in ("aa", "two"):
            dst = sc.Lattice(dict(params, layout=layout, staging=staging if layout == "aa" else "auto"))
            dst.write_populations(f)
            dst.set_counters(d["step"], d["evaporated_mass"])
            dst.step(5)
            results.append((dst.read_populations(), dst.diagnostics()))
            dst.close()
        assert np.array_equal(results[0][0], results[1][0])
        _same_diag(results[0][1], results[1][1])
    src.close()


def test_init_returns_to_the_even_form(sc):
    params, init = CASES["seam_sink_unequal_tau"]
    a = sc.Lattice(dict(params, layout="aa"))
    a.init(init)
    a.step(3)  # odd form
    a.init(init)
    a.step(4)
    b = sc.Lattice(dict(params, layout="aa"))
    b.init(init)
    b.step(4)
    assert np.array_equal(a.read_populations(), b.read_populations())
    assert a.diagnostics()["step"] == b.diagnostics()["step"] == 4
    a.close()
    b.close()


def test_launch_info_and_tuner_report_the_in_place_step(sc):
    params, init = CASES["periodic_two_segments"]
    lat = sc.Lattice(dict(params, layout="aa", staging="thread"))
    lat.init(init)
    info = lat.launch_info()
    assert info["tile_y"] == 1 and info["zchunk"] == 1 and info["staging"] == "thread"
    assert info["tile_x"] == 128 and 1 <= info["ctas"] <= 2 * 17 * 21  # row segments of the lattice
    assert lat.launch_count(10) == 20
    before = lat.read_populations()
    assert lat.tune() == dict(tile=0, zchunk=1)
    assert np.array_equal(lat.read_populations(), before)
    lat.close()
    # the automatic choice in place: the two-pass step on small planes, the persistent
    # step (one CTA per tile column, the whole z extent) on planes of 2^17 sites or more
    lat = sc.Lattice(dict(params, layout="aa"))
    assert lat.launch_info()["staging"] == "thread"
    lat.close()
    big = dict(params, nx=512, ny=256, nz=4)
    lat = sc.Lattice(dict(big, layout="aa"))
    info = lat.launch_info()
    assert info["staging"] == "persistent" and info["zchunk"] == big["nz"] and info["bands"] == 1
    cols = -(-big["nx"] // info["tile_x"]) * -(-big["ny"] // info["tile_y"])
    assert info["ctas"] == cols
    assert lat.launch_count(10) == 1 and lat.launch_count(2049) == 3
    lat.close()
    # one band while its tiles fit the shared ring (512^2), two where they do not (1024^2)
    for n, bands in ((512, 1), (1024, 2)):
        lat = sc.Lattice(dict(big, nx=n, ny=n, nz=2, layout="aa"))
        info = lat.launch_info()
        assert info["staging"] == "persistent" and info["bands"] == bands, n
        assert info["ctas"] == -(-n // bands // info["tile_x"]) * -(-n // info["tile_y"])
        lat.close()


def test_batch_rejects_in_place_members(sc):
    params, _ = CASES["seam_sink_unequal_tau"]
    b = sc.Batch(1 << 28)
    with pytest.raises(sc.ScError, match="-1"):
        b.add(dict(params, layout="aa"))
    b.close()


@pytest.mark.parametrize("n", [128, 256])
def test_full_size_droplet_same_bits(sc, n):
    """The benchmark's droplet (planar sinks across the z seam) at 128^3 and 256^3,
    in place with either kernel: densities equal to the two-lattice step's after an
    odd and an even number of steps, compared on the device."""
    import torch
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(n, 24.0 * n / 128, 1)
    fields = {}
    for kind in ("aa", "aa_bands", "aa_thread", "two"):
        layout = "two" if kind == "two" else "aa"
        staging = {"aa": "persistent", "aa_bands": "persistent", "aa_thread": "thread", "two": "auto"}[kind]
        lat = sc.Lattice(dict(params, layout=layout, staging=staging))
        if kind == "aa_bands":
            assert lat.persist_bands(4) == 4
        lat.init(init)
        lat.step(9)
        f9 = lat.read_fields_device().clone()
        lat.step(11)
        f20 = lat.read_fields_device().clone()
        fields[kind] = (f9, f20, lat.diagnostics())
        lat.close()
        torch.cuda.synchronize()
    for kind in ("aa", "aa_bands", "aa_thread"):
        for k in (0, 1):
            assert torch.equal(fields[kind][k], fields["two"][k]), (kind, k)
        _same_diag(fields[kind][2], fields["two"][2])


def test_more_steps_than_one_persistent_launch(sc):
    """1031 steps are two persistent launches (1024 + 7), the second starting in the
    odd form: the same bits as the two-lattice step."""
    params, init = CASES["film_wall_sink"]
    aa = _run(sc, params, init, [1031], "aa", "persistent")
    two = _run(sc, params, init, [1031], "two")
    assert np.array_equal(aa[0][0], two[0][0])
    _same_diag(aa[0][2], two[0][2])
