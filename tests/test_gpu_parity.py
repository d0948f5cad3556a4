"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances: one FP32 step of any state is within 1e-6 relative per population,
relative to the population's own scale max(|f_oracle|, w_i rho^c(x)) (the
equilibrium value at that site, so an over-relaxed population that lands near
zero is not judged against zero); densities after 1000 steps are within 1e-4
absolute. Reduced-precision storage is judged against the oracle applied
to the same quantised input, within one storage ulp of the offset f - w_i.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

Q = 19


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


@pytest.fixture(scope="module")
def W(sc):
    _, w = sc.lattice_directions()
    return w


def _pair(sc, oracle_mod, params):
    return sc.Lattice(params), oracle_mod.Lattice(params)


def _rel_err(f_gpu, f_orc, w):
    rho = np.abs(f_orc).sum(axis=1, keepdims=True)  # per component and site
    den = np.maximum(np.maximum(np.abs(f_orc), w[None, :, None, None, None] * rho), 1e-30)
    return np.max(np.abs(f_gpu - f_orc) / den)


GEOMS = {
    "periodic": dict(),
    "wall_planar_sink": dict(geometry=1, sink_z0=7, sink_layers=1, wall_z0=0, wall_thickness=2, rho_H=0.03),
    "seam_sink_2layers": dict(geometry=1, sink_z0=-1, sink_layers=2, rho_H=0.02),
    "sphere_sink": dict(geometry=2, sphere_cx=10.0, sphere_cy=5.5, sphere_cz=4.0, R_H=4.5, rho_H=0.025),
    "unequal_tau": dict(tau_r=0.8, tau_b=1.3, G=2.5),
    "self_couplings": dict(G=2.0, G_rr=-1.3, G_bb=0.6, tau_r=0.9),  # Eq. (3) summed over cbar = c too
}
# nx not a multiple of 4: per-thread pulls; nx a multiple of 8: staged rows (FP32 and FP16/BF16)
SHAPES = [(37, 13, 11), (5, 3, 4), (1, 6, 9), (70, 9, 8), (33, 17, 5),
          (40, 13, 11), (8, 3, 4), (4, 6, 9), (72, 9, 8), (24, 17, 5)]


# step kernel tiles: 0 = automatic choice, k > 0 = entry k - 1 of the tile list (32x8, 32x4, 16x8, 8x4, 64x4)
KERNELS = [0, 1, 2, 4]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("geom", list(GEOMS))
def test_one_step_random_state(sc, oracle_mod, W, shape, geom, kernel):
    from paper_1701_03637_gb300.workloads import random_populations
    nx, ny, nz = shape
    p = dict(nx=nx, ny=ny, nz=nz, G=3.6, tile=kernel)
    p.update(GEOMS[geom])
    if p.get("geometry") == 1:
        p["sink_z0"] = p["sink_z0"] % nz
        if p.get("wall_thickness", 0) and nz < 8:
            p["wall_thickness"] = 0
        p["sink_layers"] = min(p["sink_layers"], nz)
    g, o = _pair(sc, oracle_mod, p)
    seed = nx * 10007 + ny * 101 + nz + 1000003 * list(GEOMS).index(geom)
    f0 = random_populations(nx, ny, nz, seed=seed, rho=(0.55, 0.25))
    g.write_populations(f0)
    o.set_populations(f0)
    # the written state is the oracle's (sink reset applied, solids zeroed) to FP32 rounding;
    # a sink site's complement is a 38-term FP32 sum, read back through a second reset
    assert _rel_err(g.read_populations(), o.populations(), W) < 2e-6
    g.step(1)
    o.step(1)
    assert _rel_err(g.read_populations(), o.populations(), W) < 1e-6
    dg, do = g.diagnostics(), o.diagnostics()
    assert dg["step"] == do["step"] == 1
    assert abs(dg["mass_r"] - do["mass_r"]) <= 1e-6 * abs(do["mass_r"])
    assert abs(dg["mass_b"] - do["mass_b"]) <= 1e-6 * abs(do["mass_b"])
    assert abs(dg["flux_last"] - do["flux_last"]) <= 1e-6 * max(1.0, abs(do["mass_r"]))
    assert dg["droplet_sites"] == do["droplet_sites"]


def test_init_shape_matches_oracle(sc, oracle_mod, W):
    """Device-side SplitMix64 noise and shape equal the oracle's definition."""
    for params, init in [
        (dict(nx=12, ny=10, nz=9, geometry=2, sphere_cx=6, sphere_cy=5, sphere_cz=4.5, R_H=4.0),
         dict(shape=1, cx=6.0, cy=5.0, cz=4.5, radius=3.0, rho_hi=0.7, rho_lo=0.04, noise_amp=1e-2, seed=12345)),
        (dict(nx=4, ny=4, nz=40, geometry=1, sink_z0=39, wall_thickness=2),
         dict(shape=0, film_z=10, rho_hi=1.0, rho_lo=0.03, noise_amp=1e-4, seed=0)),
    ]:
        g, o = _pair(sc, oracle_mod, params)
        g.init(init)
        o.init_shape(init)
        assert _rel_err(g.read_populations(), o.populations(), W) < 2e-6
        gr, gb = g.read_fields()
        orr, ob = o.fields()
        assert np.max(np.abs(gr - orr)) < 1e-6 and np.max(np.abs(gb - ob)) < 1e-6


# FP32 bookkeeping bound: every collided site rounds 2 x 19 products and sums per
# step; the residue is unbiased to first order but identical states round alike,
# so the conserved total M_r + E may drift by a fraction of an ulp per site and
# step. The bound below allows 2e-8 relative per step (a third of an FP32 ulp).
DRIFT_PER_STEP = 2e-8


def _check_bookkeeping(dg, do, steps):
    tol = DRIFT_PER_STEP * steps * do["mass_r"]
    assert abs(dg["evaporated_mass"] - do["evaporated_mass"]) < tol
    assert abs(dg["mass_r"] - do["mass_r"]) < tol
    assert abs(dg["flux_last"] - do["flux_last"]) < 1e-3 * abs(do["flux_last"]) + 1e-9 * do["mass_r"]


@pytest.mark.parametrize("kernel", [0, 3])
def test_film_1000_steps(sc, oracle_mod, kernel):
    """4x4x128 film (wall 2, sink plane z=127, rho_H = 0.03, g = 3.6, init 1.0/0.03 with
    1e-4 noise): densities within 1e-4 absolute after 1000 steps."""
    from paper_1701_03637_gb300.workloads import film_4x4x128
    params, init = film_4x4x128()
    g, o = sc.Lattice(dict(params, tile=kernel)), oracle_mod.Lattice(params)
    g.init(init)
    o.init_shape(init)
    g.step(1000)
    o.step(1000)
    gr, gb = g.read_fields()
    orr, ob = o.fields()
    assert np.max(np.abs(gr - orr)) < 1e-4
    assert np.max(np.abs(gb - ob)) < 1e-4
    dg, do = g.diagnostics(), o.diagnostics()
    assert abs(dg["interface_z"] - do["interface_z"]) < 1e-3
    _check_bookkeeping(dg, do, 1000)
    assert dg["status"] == 0


@pytest.mark.parametrize("kernel", [1, 2])
def test_droplet_48_500_steps(sc, oracle_mod, kernel):
    """Droplet with the spherical-exterior sink, 48^3, 500 steps: densities within 1e-4."""
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(48, 10.0, 7, spherical_sink=True)
    g, o = sc.Lattice(dict(params, tile=kernel)), oracle_mod.Lattice(params)
    g.init(init)
    o.init_shape(init)
    g.step(500)
    o.step(500)
    gr, gb = g.read_fields()
    orr, ob = o.fields()
    assert np.max(np.abs(gr - orr)) < 1e-4 and np.max(np.abs(gb - ob)) < 1e-4
    dg, do = g.diagnostics(), o.diagnostics()
    assert dg["droplet_sites"] == do["droplet_sites"]
    _check_bookkeeping(dg, do, 500)


@pytest.mark.parametrize("nx,stagings", [(41, (0,)), (40, (1, 2)), (8, (1, 2))])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_tiles_and_chunks_give_identical_bits(sc, nx, stagings, storage):
    """The per-site arithmetic does not depend on the tile shape, z-chunking, the
    staging of the pulls or graph replay (a wall and a spherical sink included)."""
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(40, 9.0, 3, spherical_sink=True)
    params.update(nx=nx, ny=23, nz=19, sphere_cx=nx / 2.0, sphere_cy=11.0, sphere_cz=9.0, R_H=9.0,
                  wall_z0=0, wall_thickness=2, storage=storage)
    init.update(cx=nx / 2.0, cy=11.0, cz=9.0, radius=min(6.0, nx / 2.0 - 1))
    if storage == "f16" and nx % 8:
        stagings = (0,)
    ref = None
    launches = [(st, tile, zc) for st in stagings
                for tile, zc in [(1, 0), (2, 3), (3, 1), (4, 19), (1, 5), (2, 0), (3, 7), (5, 0), (5, 4)]]
    for k, (st, tile, zc) in enumerate(launches):
        g = sc.Lattice(dict(params, tile=tile, zchunk=zc, staging=st))
        if st:
            assert g.launch_info()["staging"] == {1: "thread", 2: "rows"}[st]
        g.init(init)
        if k == 4:
            for _ in range(30):
                g.step(1)
        else:
            g.step(30)
        f = g.read_populations()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref), (st, tile, zc)


def test_tuner_keeps_state_and_bits(sc):
    """The single-lattice autotuner leaves state and bookkeeping untouched, and the
    configuration it picks computes the same bits."""
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(40, 9.0, 3)
    params.update(nx=40, ny=23, nz=19, wall_z0=0, wall_thickness=2)
    init.update(cx=20.0, cy=11.0, cz=9.0, radius=6.0)
    a, b = sc.Lattice(params), sc.Lattice(params)
    a.init(init)
    b.init(init)
    a.step(5)
    b.step(5)
    f, d = a.read_populations(), a.diagnostics()
    cfg = a.tune(trials=2)
    assert 1 <= cfg["tile"] <= len(sc.tile_list())
    assert np.array_equal(a.read_populations(), f) and a.diagnostics() == d
    a.step(20)
    b.step(20)
    assert np.array_equal(a.read_populations(), b.read_populations())
    da, db = a.diagnostics(), b.diagnostics()
    assert abs(da["evaporated_mass"] - db["evaporated_mass"]) <= 1e-12 * max(1.0, abs(db["evaporated_mass"]))


def test_checkpoint_restore(sc, oracle_mod):
    from paper_1701_03637_gb300.workloads import film_4x4x128
    params, init = film_4x4x128(rho_hi=0.7, rho_lo=0.04, rho_H=0.01)
    a = sc.Lattice(params)
    a.init(init)
    a.step(300)
    f = a.read_populations()
    d = a.diagnostics()
    b = sc.Lattice(params)
    b.write_populations(f)
    b.set_counters(d["step"], d["evaporated_mass"])
    a.step(300)
    b.step(300)
    ra, _ = a.read_fields()
    rb, _ = b.read_fields()
    # the restore recomputes the sink complement from FP32 sums: rounding-level drift only
    assert np.max(np.abs(ra - rb)) < 1e-5
    da, db = a.diagnostics(), b.diagnostics()
    assert da["step"] == db["step"] == 600
    assert abs(da["evaporated_mass"] - db["evaporated_mass"]) < 1e-6


def _storage_ulp(off, storage):
    mant = 7 if storage == "bf16" else 10
    ulp = np.exp2(np.floor(np.log2(np.maximum(off, 1e-30))) - mant)
    return np.maximum(ulp, 2.0 ** -133 if storage == "bf16" else 2.0 ** -24)


@pytest.mark.parametrize("nx", [37, 40])
@pytest.mark.parametrize("kernel", [1, 4])
@pytest.mark.parametrize("storage", ["f16", "bf16", "f16s"])
@pytest.mark.parametrize("with_sink", [False, True])
def test_reduced_precision_one_step(sc, oracle_mod, W, storage, with_sink, kernel, nx):
    """FP16/BF16 offset storage: one step equals the oracle on the same quantised input
    to within one storage ulp of the offset f - w_i plus the FP32 arithmetic bound of
    the FP32 one-step test (1e-6 relative; it dominates where f is within a few FP32
    ulps of w_i, whose offset has a tiny storage ulp). With a sink the oracle
    recomputes the sink's complement from the quantised input in FP64 while the GPU
    keeps it quantised, so sinks and their neighbours get three ulps."""
    from paper_1701_03637_gb300.workloads import random_populations
    ny, nz = 13, 11
    geom = dict(GEOMS["wall_planar_sink"])
    if not with_sink:
        geom.update(geometry=0)
    p = dict(nx=nx, ny=ny, nz=nz, G=3.6, storage=storage, tile=kernel, **geom)
    g = sc.Lattice(p)
    o = oracle_mod.Lattice(p)
    g.write_populations(random_populations(nx, ny, nz, seed=9, rho=(0.6, 0.3)))
    fq = g.read_populations()  # quantised state as the GPU holds it
    o.set_populations(fq)
    g.step(1)
    o.step(1)
    fg, fo = g.read_populations(), o.populations()
    w = W[None, :, None, None, None]
    if storage == "f16s":  # g = f / w stored: one FP16 ulp of g, times w
        ulp = w * _storage_ulp(np.abs(fo) / w, storage)
    else:
        ulp = _storage_ulp(np.abs(fo - w), storage)
    err = np.abs(fg - fo)
    k = np.full(fo.shape, 1.01)
    if with_sink:
        near = np.zeros(o.site_class().shape, bool)
        near[5:10] = True  # sink plane 7 and two planes either side
        k[:, :, near] = 3.0
    fluid = np.broadcast_to(o.site_class() == 0, fo.shape)
    ratio = np.where(fluid, err / (k * ulp + 1e-6 * np.abs(fo)), 0.0)
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio.max() <= 1.0, (float(ratio.max()), worst, float(fg[worst]), float(fo[worst]), float(ulp[worst]))


@pytest.mark.parametrize("n,radius,seed,tuned", [(128, 24.0, 1, False), (128, 24.0, 1, True), (512, 96.0, 2, True)])
def test_full_size_sampled_windows(sc, oracle_mod, n, radius, seed, tuned):
    """The 128^3 and 512^3 droplets in the benchmark's launch configuration (the
    autotuned one, as bench.py times it, and the automatic one): one GPU step,
    checked at sampled sites against the oracle run on a 7^3 window around each
    site (the step reaches two sites, so the window's own periodic seam cannot
    reach the centre)."""
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(n, radius, seed)
    g = sc.Lattice(params)
    g.init(init)
    if tuned:
        g.tune(trials=2)
    r0, b0 = g.read_fields()
    g.step(1)
    r1, b1 = g.read_fields()
    # total mass is conserved exactly by the sink's complement rule
    assert abs((r1.sum(dtype=np.float64) + b1.sum(dtype=np.float64)) /
               (r0.sum(dtype=np.float64) + b0.sum(dtype=np.float64)) - 1) < 1e-6
    rng = np.random.default_rng(5)
    h, R = n // 2, int(radius)
    pts = [(h, h, h), (h, h, h + R), (h + R, h, h), (10, n - 28, n - 2), (3, 5, n - 1), (7, 9, 0), (0, 0, 1),
           (n - 1, n - 1, n - 2)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(8)]
    for (X, Y, Z) in pts:
        xs = np.arange(X - 3, X + 4) % n
        ys = np.arange(Y - 3, Y + 4) % n
        zs = np.arange(Z - 3, Z + 4) % n
        wr = r0[np.ix_(zs, ys, xs)].astype(np.float64)
        wb = b0[np.ix_(zs, ys, xs)].astype(np.float64)
        wp = dict(nx=7, ny=7, nz=7, G=params["G"], rho_H=params["rho_H"])
        sink_planes = [k for k, z in enumerate(zs) if z in (n - 1, 0)]
        if sink_planes:
            wp.update(geometry=1, sink_z0=sink_planes[0], sink_layers=len(sink_planes))
        o = oracle_mod.Lattice(wp)
        o.init_fields(wr, wb)
        o.step(1)
        orr, ob = o.fields()
        assert abs(r1[Z, Y, X] - orr[3, 3, 3]) < 1e-6 * max(1.0, orr[3, 3, 3]), (X, Y, Z)
        assert abs(b1[Z, Y, X] - ob[3, 3, 3]) < 1e-6 * max(1.0, ob[3, 3, 3]), (X, Y, Z)


@pytest.mark.parametrize("layout", ["two", "aa"])
def test_close_releases_device_memory(sc, layout):
    """Lattice.close destroys the handle after its stream has finished and gives its
    device memory back to torch's allocator."""
    import torch
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(64, 12.0, 1)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    lat = sc.Lattice(dict(params, layout=layout))
    lat.init(init)
    lat.step(3)
    assert torch.cuda.memory_allocated() - before >= sc.required_bytes(dict(params, layout=layout))
    lat.close()
    assert torch.cuda.memory_allocated() == before
