"""Batched step: every member of a batch computes what the single-lattice path
computes for it (the method of Sec. II per lattice), bit for bit, whatever the
other members, their step limits, the kernel tile or the autotuner do."""
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


def _members():
    """Lattices of different extents, parameters and geometries (with their inits)."""
    from paper_1701_03637_gb300.workloads import droplet, film_4x4x128
    out = []
    p, i = film_4x4x128(rho_hi=0.7, rho_lo=0.04, rho_H=0.01)
    p.update(nx=6, ny=5, nz=48, sink_z0=47)
    i.update(film_z=14)
    out.append((p, i))
    p, i = droplet(40, 9.0, 11, spherical_sink=True)
    p.update(nx=37, ny=33, nz=29, sphere_cx=18.0, sphere_cy=16.0, sphere_cz=14.0, R_H=12.0, G=3.4, rho_H=0.025)
    i.update(cx=18.0, cy=16.0, cz=14.0, radius=7.0)
    out.append((p, i))
    p, i = droplet(32, 8.0, 5)
    p.update(tau_r=0.9, tau_b=1.15, G=3.7)
    out.append((p, i))
    p, i = droplet(24, 6.0, 9)
    p.update(geometry=0, nx=50, ny=17, nz=21, G_rr=-0.8, G_bb=0.4)  # with self couplings
    i.update(cx=25.0, cy=8.0, cz=10.0)
    out.append((p, i))
    p, i = droplet(33, 7.0, 13)
    p.update(nx=65, ny=9, nz=40, sink_z0=0, sink_layers=2, G=3.3, rho_H=0.035)
    i.update(cx=32.0, cy=4.0, cz=20.0, radius=4.0)
    out.append((p, i))
    return out


def _alone(sc, params, init, steps):
    g = sc.Lattice(params)
    g.init(init)
    g.step(steps)
    f = g.read_populations()
    d = g.diagnostics()
    g.close()
    return f, d


def _same_bookkeeping(d, ref):
    # the evaporated mass is summed over other partial sums (items, not CTA slots):
    # equal to FP64 rounding
    for k in ("evaporated_mass", "flux_last"):
        assert abs(d[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, d[k], ref[k])
    for k in ("mass_r", "mass_b", "interface_z", "radius", "droplet_sites", "status", "step"):
        assert d[k] == ref[k], (k, d[k], ref[k])


def test_members_match_the_lattices_stepped_alone(sc):
    members = _members()
    limits = [37, 100, 64, -1, 1]
    b = sc.Batch(1 << 30)
    lats = []
    for (p, i), lim in zip(members, limits):
        slot, lat = b.add(p)
        lat.init(i)
        b.set_steps(slot, lim)
        lats.append((slot, lat))
    b.step(70)   # a graph sequence of 32, a second, then 6 single launches
    b.step(30)
    for ((p, i), lim, (slot, lat)) in zip(members, limits, lats):
        n = 100 if lim < 0 else min(lim, 100)
        f_ref, d_ref = _alone(sc, p, i, n)
        assert np.array_equal(lat.read_populations(), f_ref), (p, lim)
        _same_bookkeeping(lat.diagnostics(), d_ref)
        assert b.remaining(slot) == (2 ** 63 - 1 if lim < 0 else lim - n)
    b.close()


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5])
def test_every_tile_gives_the_same_bits(sc, tile):
    members = _members()[1:4]
    b = sc.Batch(1 << 29)
    b.configure(tile=tile, zchunk=8)
    lats = []
    for p, i in members:
        _, lat = b.add(p)
        lat.init(i)
        lats.append(lat)
    b.step(41)
    assert b.info()["tile"] == tile
    for (p, i), lat in zip(members, lats):
        f_ref, _ = _alone(sc, p, i, 41)
        assert np.array_equal(lat.read_populations(), f_ref), (tile, p)
    b.close()


def test_tuner_leaves_the_state_untouched(sc):
    members = _members()
    b = sc.Batch(1 << 30)
    lats = []
    for p, i in members:
        _, lat = b.add(p)
        lat.init(i)
        lats.append(lat)
    b.step(5)
    before = [lat.read_populations() for lat in lats]
    dbefore = [lat.diagnostics() for lat in lats]
    tile, zc = b.tune(trials=2)
    assert 1 <= tile <= len(sc.tile_list()) and zc in (16, 32, 64)
    for lat, f, d in zip(lats, before, dbefore):
        assert np.array_equal(lat.read_populations(), f)
        assert lat.diagnostics() == d
    b.step(20)
    for (p, i), lat in zip(members, lats):
        f_ref, d_ref = _alone(sc, p, i, 25)
        assert np.array_equal(lat.read_populations(), f_ref)
        _same_bookkeeping(lat.diagnostics(), d_ref)
    b.close()


def test_admission_by_free_arena_and_reuse(sc):
    from paper_1701_03637_gb300.workloads import droplet
    p, i = droplet(32, 8.0, 5)
    need = sc.required_bytes(p)
    b = sc.Batch(2 * need + 4096)
    s0, l0 = b.add(p)
    s1, l1 = b.add(p)
    with pytest.raises(sc.ScError, match="-2"):
        b.add(p)
    assert b.info()["members"] == 2
    b.remove(s0)
    assert b.info()["largest_free"] >= need
    s2, l2 = b.add(p)
    l1.init(i)
    l2.init(i)
    b.step(12)
    f_ref, _ = _alone(sc, p, i, 12)
    assert np.array_equal(l1.read_populations(), f_ref)
    assert np.array_equal(l2.read_populations(), f_ref)
    b.close()


def test_members_join_and_leave_mid_run(sc):
    members = _members()
    b = sc.Batch(1 << 30)
    slots = []
    for p, i in members[:3]:
        s, lat = b.add(p)
        lat.init(i)
        slots.append(s)
    b.step(33)
    b.remove(slots[1])
    p, i = members[3]
    s3, l3 = b.add(p)
    l3.init(i)
    b.step(40)
    f_ref, _ = _alone(sc, *members[0], 73)
    assert np.array_equal(b.lattice(slots[0]).read_populations(), f_ref)
    f_ref, _ = _alone(sc, *members[2], 73)
    assert np.array_equal(b.lattice(slots[2]).read_populations(), f_ref)
    f_ref, _ = _alone(sc, p, i, 40)
    assert np.array_equal(l3.read_populations(), f_ref)
    # a member stepped on its own in between keeps in step with the batch
    l3.step(3)
    b.step(5)
    f_ref, _ = _alone(sc, p, i, 48)
    assert np.array_equal(l3.read_populations(), f_ref)
    b.close()


def test_member_matches_the_oracle(sc, oracle_mod):
    members = _members()
    p, i = members[2]
    b = sc.Batch(1 << 29)
    for q, j in members[1:4]:
        _, lat = b.add(q)
        lat.init(j)
        if q is p:
            mine = lat
    b.step(200)
    o = oracle_mod.Lattice(p)
    o.init_shape(i)
    o.step(200)
    gr, gb = mine.read_fields()
    orr, ob = o.fields()
    assert np.max(np.abs(gr - orr)) < 1e-4 and np.max(np.abs(gb - ob)) < 1e-4
    b.close()


@pytest.mark.parametrize("extent", [(64, 64, 2), (512, 288, 2)])
def test_thin_wide_member_books_every_item_in_its_own_slot(sc, extent):
    """A member with more tile columns of the batch's 8x4 tile than work items of
    its own step (64x64x2), or more than the single-lattice step's CTA cap of 4096
    (512x288x2): every (column, chunk) item still has an evaporated-mass slot of
    its own, so the evaporated mass equals the lone run's (to FP64 summation order)
    and is the same from run to run."""
    nx, ny, nz = extent
    p = dict(nx=nx, ny=ny, nz=nz, tau_r=1.0, tau_b=1.0, G=3.6, rho_H=0.01, geometry=1, sink_z0=1, sink_layers=1)
    i = dict(shape=0, film_z=1, rho_hi=0.7, rho_lo=0.04, noise_amp=1e-3, seed=21)
    runs = []
    for _ in range(2):
        b = sc.Batch(1 << 29)
        b.configure(tile=4, zchunk=1)  # the 8x4 tile: the most columns
        _, lat = b.add(p)
        lat.init(i)
        b.step(70)
        runs.append((lat.read_populations(), lat.diagnostics()))
        b.close()
    f_ref, d_ref = _alone(sc, p, i, 70)
    assert d_ref["evaporated_mass"] > 0
    for f, d in runs:
        assert np.array_equal(f, f_ref)
        _same_bookkeeping(d, d_ref)
    assert runs[0][1] == runs[1][1]
