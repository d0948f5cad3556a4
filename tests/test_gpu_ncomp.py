"""More than two components on the GPU (sc_ncomp_*): Eq. (3) summed over every other
component. Three and four components against the N-component FP64 oracle
(oracle/multi.py) from non-equilibrium states, with and without a solid slab, within
1e-6 of each population's scale per step (the two-component parity bar); two
components with self couplings bit for bit against sc_lbm_step; an absent third
component changes no bit of the other two."""
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


def _state(n, shape, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 0.6, (n,) + shape)
    return rng.uniform(0.7, 1.3, (n, Q) + shape) / Q * rho[:, None]


G3 = np.array([[-0.9, 2.8, 1.6], [2.8, 0.2, 3.1], [1.6, 3.1, -0.4]])
G4 = np.array([[-0.5, 2.2, 1.4, 0.8], [2.2, 0.1, 2.9, 1.1], [1.4, 2.9, -0.7, 2.0], [0.8, 1.1, 2.0, 0.3]])


@pytest.mark.parametrize("steps", [1, 4])
@pytest.mark.parametrize("n,wall", [(3, 0), (3, 2), (4, 0), (4, 2)])
def test_matches_the_n_component_oracle(sc, n, wall, steps):
    from oracle import multi
    from paper_1701_03637_gb300.ncomp import NLattice
    nx, ny, nz = 7, 5, 9
    tau = [0.9, 1.15, 1.0, 0.85][:n]
    g = (G3 if n == 3 else G4)
    f0 = _state(n, (nz, ny, nx), 11 + n)
    gl = NLattice(nx, ny, nz, tau, g, wall_z0=4, wall_thickness=wall)
    o = multi.Lattice(nx, ny, nz, tau, g, wall_z0=4, wall_thickness=wall)
    gl.write_populations(f0)
    o.set_populations(f0)
    gl.step(steps)
    o.step(steps)
    fg, fo = gl.read_populations(), o.f
    # each population's own scale max(|f|, w_i rho^c), as in the two-component parity tests
    rho = np.abs(fo).sum(axis=1, keepdims=True)
    den = np.maximum(np.maximum(np.abs(fo), multi.W[None, :, None, None, None] * rho), 1e-30)
    err = np.max(np.abs(fg - fo) / den)
    assert err < 1e-6 * steps, err
    gl.close()


@pytest.mark.parametrize("wall", [0, 2])
def test_two_components_are_the_two_component_step(sc, wall):
    from paper_1701_03637_gb300.ncomp import NLattice
    nx, ny, nz = 12, 6, 10
    f0 = _state(2, (nz, ny, nx), 21)
    g = np.array([[-0.7, 3.2], [3.2, 0.35]])
    a = NLattice(nx, ny, nz, [0.95, 1.1], g, wall_z0=3, wall_thickness=wall)
    a.write_populations(f0)
    b = sc.Lattice(dict(nx=nx, ny=ny, nz=nz, tau_r=0.95, tau_b=1.1, G=3.2, G_rr=-0.7, G_bb=0.35, geometry=0,
                        wall_z0=3, wall_thickness=wall))
    b.write_populations(f0)
    a.step(20)
    b.step(20)
    assert np.array_equal(a.read_populations(), b.read_populations())
    a.close()
    b.close()


def test_absent_third_component_changes_nothing(sc):
    from paper_1701_03637_gb300.ncomp import NLattice
    nx, ny, nz = 8, 5, 7
    f2 = _state(2, (nz, ny, nx), 31)
    f3 = np.concatenate([f2, np.zeros((1, Q, nz, ny, nx))])
    a = NLattice(nx, ny, nz, [1.0, 0.9], G3[:2, :2])
    b = NLattice(nx, ny, nz, [1.0, 0.9, 1.2], G3)
    a.write_populations(f2)
    b.write_populations(f3)
    a.step(15)
    b.step(15)
    fb = b.read_populations()
    assert np.array_equal(fb[:2], a.read_populations()) and not fb[2].any()
    a.close()
    b.close()


def test_invalid_parameters(sc):
    from paper_1701_03637_gb300.ncomp import NLattice
    for kw in (dict(tau=[1.0]), dict(tau=[1.0] * 5), dict(tau=[1.0, 0.5]), dict(g=np.full((2, 2), np.nan))):
        args = dict(tau=[1.0, 1.0], g=np.zeros((2, 2)))
        args.update(kw)
        g = args["g"] if args["g"].shape[0] >= len(args["tau"]) else np.zeros((len(args["tau"]),) * 2)
        with pytest.raises(sc.ScError, match="-1"):
            NLattice(4, 4, 4, args["tau"], g)


def test_init_fields_gives_rest_populations(sc):
    """sc_ncomp_init_fields: populations w_i rho^c (Eq. 2 at rest) of the given
    densities, FP32-rounded, solid sites 0."""
    from oracle import multi
    from paper_1701_03637_gb300.ncomp import NLattice
    from paper_1701_03637_gb300.workloads import three_component_droplet
    params, rho = three_component_droplet(12, 3.0, 4)
    lat = NLattice(**params, wall_z0=5, wall_thickness=2)
    lat.init_fields(rho)
    f = lat.read_populations()
    want = multi.W[None, :, None, None, None] * rho[:, None].astype(np.float64)
    solid = np.zeros(rho.shape[1:], bool)
    solid[5:7] = True
    want[:, :, solid] = 0.0
    # the library's FP32 weights sum to 1 exactly (w_1 = 1/18 - 1 ulp, w_0 = 1 - 12 w_1),
    # so w_0 is 1.2e-7 above 1/3; with the product's rounding (2^-24) the bound is 2.5e-7
    assert np.all(np.abs(f - want) <= 2.5e-7 * np.abs(want)), np.max(np.abs(f - want) / np.maximum(want, 1e-30))
    lat.close()
