"""Pins for the FP64 oracle: each test checks it against something other than
itself — lattice identities, textbook special cases, exact invariants of the
method, library routines, and numbers printed in arXiv:1701.03637."""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
Q = 19


def _golden(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split(None, 3))
    return rows


def _paper_value(key):
    for row in _golden("paper_values.txt"):
        if row[0] == key:
            return float(row[1]), float(row[2])
    raise KeyError(key)


def _random_state(nx, ny, nz, seed, rho=(0.6, 0.1), spread=0.3):
    rng = np.random.default_rng(seed)
    f = rng.uniform(1 - spread, 1 + spread, (2, Q, nz, ny, nx)) / Q
    return f * np.asarray(rho)[:, None, None, None, None]


# ---------------------------------------------------------------- tables and equilibrium

def test_d3q19_isotropy(oracle_mod):
    """Sec. II A weights: sum w = 1, odd moments vanish, sum w c c = cs^2 I and the
    4th-order tensor is cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)."""
    c, w, opp = oracle_mod.tables()
    c = c.astype(np.float64)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ c, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso, atol=1e-16)
    assert sorted(map(tuple, c.astype(int))) == sorted(
        {(a, b, e) for a in (-1, 0, 1) for b in (-1, 0, 1) for e in (-1, 0, 1) if abs(a) + abs(b) + abs(e) <= 2})
    assert np.array_equal(c[opp], -c)
    assert sorted(np.round(w * 36).astype(int).tolist()) == [1] * 12 + [2] * 6 + [12]


@pytest.mark.parametrize("rho,u", [(0.7, (0.01, -0.02, 0.03)), (0.036, (0.1, 0.0, -0.05)), (1.0, (0, 0, 0))])
def test_feq_moments(oracle_mod, rho, u):
    """Eq. (2): sum feq = rho, sum feq c = rho u, sum feq c c = rho (cs^2 I + u u)."""
    c, _, _ = oracle_mod.tables()
    c = c.astype(np.float64)
    u = np.array(u, np.float64)
    fe = oracle_mod.feq(rho, u)
    assert abs(fe.sum() - rho) < 1e-15
    assert np.allclose(fe @ c, rho * u, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", fe, c, c), rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_splitmix64_published_vectors(oracle_mod):
    for seed, k, val in _golden("splitmix64.txt"):
        assert oracle_mod.splitmix64(int(seed), int(k)) == int(val)
    u = oracle_mod.uniform(1234567, 1)
    assert u == (6457827717110365317 >> 11) * 2.0 ** -53


# ---------------------------------------------------------------- streaming and walls

def test_pure_streaming_is_periodic_roll(oracle_mod):
    """With g = 0 and tau -> infinity the step is pure streaming: each direction is
    numpy's periodic roll by e_i (Sec. II A, periodic boundaries)."""
    nx, ny, nz = 5, 4, 3
    L = oracle_mod.Lattice(dict(nx=nx, ny=ny, nz=nz, G=0.0, tau_r=1e15, tau_b=1e15))
    f = _random_state(nx, ny, nz, 1)
    L.set_populations(f)
    L.step(1)
    g = L.populations()
    c, _, _ = oracle_mod.tables()
    for i in range(Q):
        want = np.roll(f[:, i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(1, 2, 3))
        assert np.allclose(g[:, i], want, rtol=1e-12, atol=0)


def test_halfway_bounce_back(oracle_mod):
    """A population streaming into a solid site returns to its source with the
    opposite velocity (Sec. II A walls, Succi's simple bounce back)."""
    nx, ny, nz = 3, 3, 6
    L = oracle_mod.Lattice(dict(nx=nx, ny=ny, nz=nz, G=0.0, tau_r=1e15, tau_b=1e15, wall_z0=4, wall_thickness=2))
    f = _random_state(nx, ny, nz, 2)
    L.set_populations(f)
    f = L.populations()  # solid sites zeroed
    assert np.all(f[:, :, 4:] == 0)
    L.step(1)
    g = L.populations()
    c, _, opp = oracle_mod.tables()
    for i in range(Q):
        for z in range(4):
            zd = z + c[i, 2]
            if zd in (4, 5):
                # arrives at (x, y, z) in direction opp[i] from its own site
                assert np.allclose(g[:, opp[i], z], f[:, i, z], rtol=1e-12)
    assert np.all(g[:, :, 4:] == 0)
    # the exchange is a permutation: every component keeps its mass
    assert np.allclose(g.sum(axis=(1, 2, 3, 4)), f.sum(axis=(1, 2, 3, 4)), rtol=1e-14)


# ---------------------------------------------------------------- exact invariants

def test_component_mass_conserved_sink_closed(oracle_mod):
    nx, ny, nz = 6, 5, 8
    L = oracle_mod.Lattice(dict(nx=nx, ny=ny, nz=nz, G=3.6, wall_z0=0, wall_thickness=2))
    L.set_populations(_random_state(nx, ny, nz, 3))
    m0 = L.populations().sum(axis=(1, 2, 3, 4))
    L.step(40)
    m1 = L.populations().sum(axis=(1, 2, 3, 4))
    assert np.allclose(m1, m0, rtol=1e-13, atol=0)


def test_total_momentum_conserved_periodic(oracle_mod):
    """Sum_x F^r + F^b vanishes pairwise for Eq. (3), and the shifted-velocity collision
    adds sum_c F^c, so total momentum is exact on a fully periodic lattice."""
    nx, ny, nz = 6, 5, 7
    L = oracle_mod.Lattice(dict(nx=nx, ny=ny, nz=nz, G=3.6, tau_r=1.0, tau_b=0.8))
    L.set_populations(_random_state(nx, ny, nz, 4))
    c, _, _ = oracle_mod.tables()

    def mom():
        return np.einsum("cin,ia->a", L.populations().reshape(2, Q, -1), c.astype(np.float64))

    p0 = mom()
    L.step(30)
    assert np.allclose(mom(), p0, atol=1e-13)


def test_sink_reset_values_and_mass_balance(oracle_mod):
    """Sec. II C: after a step the sink holds f^r = w rho_H and f^b = w (rho_tot - rho_H);
    the complement rule keeps rho^r + rho^b, so M_r + E and M_r + M_b are constant."""
    nx, ny, nz = 4, 3, 10
    p = dict(nx=nx, ny=ny, nz=nz, G=3.6, rho_H=0.03, geometry=1, sink_z0=9, sink_layers=1,
             wall_z0=0, wall_thickness=2)
    L = oracle_mod.Lattice(p)
    L.set_populations(_random_state(nx, ny, nz, 5, rho=(0.5, 0.3)))
    _, w, _ = oracle_mod.tables()
    d0 = L.diagnostics()
    L.step(25)
    f = L.populations()
    rho_tot = f[:, :, 9].sum(axis=(0, 1))
    assert np.allclose(f[0, :, 9], w[:, None, None] * 0.03, rtol=1e-15)
    assert np.allclose(f[1, :, 9], w[:, None, None] * (rho_tot - 0.03), rtol=1e-13)
    d1 = L.diagnostics()
    assert abs((d1["mass_r"] + d1["evaporated_mass"]) - (d0["mass_r"] + d0["evaporated_mass"])) < 1e-12
    assert abs((d1["mass_r"] + d1["mass_b"]) - (d0["mass_r"] + d0["mass_b"])) < 1e-12
    assert d1["evaporated_mass"] != 0.0


def test_spherical_sink_classification(oracle_mod):
    L = oracle_mod.Lattice(dict(nx=9, ny=9, nz=9, geometry=2, sphere_cx=4, sphere_cy=4, sphere_cz=4, R_H=3.5))
    cls = L.site_class()
    z, y, x = np.meshgrid(np.arange(9), np.arange(9), np.arange(9), indexing="ij")
    want = ((x - 4) ** 2 + (y - 4) ** 2 + (z - 4) ** 2 >= 3.5 ** 2).astype(np.int8)
    assert np.array_equal(cls, want)


# ---------------------------------------------------------------- textbook special cases (g = 0)

def _mode_amplitude(d, axis_len):
    return np.abs(np.fft.rfft(d)[1])


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_binary_diffusion_g0(oracle_mod, tau):
    """g = 0: the concentration mode of a binary BGK mixture decays with
    D = cs^2 (tau - 1/2) (the g -> 0 limit of the paper's D^c)."""
    nx = 64
    L = oracle_mod.Lattice(dict(nx=nx, ny=1, nz=1, G=0.0, tau_r=tau, tau_b=tau))
    x = np.arange(nx)
    a = 1e-3 * np.cos(2 * np.pi * x / nx)
    L.init_fields((0.5 + a).reshape(1, 1, nx), (0.5 - a).reshape(1, 1, nx))
    r, b = L.fields()
    A0 = _mode_amplitude((r - b).ravel(), nx)
    T = 600
    L.step(T)
    r, b = L.fields()
    A1 = _mode_amplitude((r - b).ravel(), nx)
    D = -math.log(A1 / A0) / (T * (2 * math.pi / nx) ** 2)
    assert abs(D / ((tau - 0.5) / 3) - 1) < 5e-3


def test_shear_wave_viscosity(oracle_mod):
    """g = 0: a transverse shear wave decays as exp(-nu k^2 t), nu = cs^2 (tau - 1/2)
    (Sec. II A: nu = (2 tau - 1)/6)."""
    nx, tau = 64, 0.9
    L = oracle_mod.Lattice(dict(nx=nx, ny=1, nz=1, G=0.0, tau_r=tau, tau_b=tau))
    x = np.arange(nx)
    uy = 1e-3 * np.sin(2 * np.pi * x / nx)
    f = np.zeros((2, Q, 1, 1, nx))
    for s in range(nx):
        for cidx, rho in enumerate((0.6, 0.4)):
            f[cidx, :, 0, 0, s] = oracle_mod.feq(rho, (0.0, uy[s], 0.0))
    L.set_populations(f)
    c, _, _ = oracle_mod.tables()

    def amp():
        g = L.populations()
        jy = np.einsum("cin,i->n", g.reshape(2, Q, -1), c[:, 1].astype(np.float64))
        return np.abs(np.fft.rfft(jy)[1])

    A0 = amp()
    T = 500
    L.step(T)
    nu = -math.log(amp() / A0) / (T * (2 * math.pi / nx) ** 2)
    assert abs(nu / ((tau - 0.5) / 3) - 1) < 5e-3


# ---------------------------------------------------------------- the paper's diffusion law

@pytest.mark.parametrize("g", [0.5, 1.0, 1.5])
def test_shan_chen_diffusion_coefficient(oracle_mod, g):
    """Sec. III A: a symmetric mixture (rho^c = rho^cbar, so the concentration mode
    is decoupled from pressure) decays with the paper's D^c(rho, g)."""
    from oracle import analytic
    nx = 128
    L = oracle_mod.Lattice(dict(nx=nx, ny=1, nz=1, G=g))
    x = np.arange(nx)
    a = 1e-4 * np.cos(2 * np.pi * x / nx)
    L.init_fields((0.35 + a).reshape(1, 1, nx), (0.35 - a).reshape(1, 1, nx))
    r, b = L.fields()
    A0 = _mode_amplitude((r - b).ravel(), nx)
    T = 1500
    L.step(T)
    r, b = L.fields()
    D = -math.log(_mode_amplitude((r - b).ravel(), nx) / A0) / (T * (2 * math.pi / nx) ** 2)
    want = analytic.diffusion_coefficient(0.35, 0.35, g)
    assert abs(D / want - 1) < 3e-3, (D, want)


def test_fick_reservoir_profile_and_flux(oracle_mod):
    """Sec. III A experiment (component cbar at 0.7, rho_H = 0.001 at the evaporation
    boundary, g = 3.6, wall of thickness 2): at early times the profile is the
    erfc solution with the paper's D^c, and the measured flux rho^r (U^r - U)
    (Eqs. (flux), (velw)) equals -D^c grad rho^r (Eq. (fick-simple))."""
    from oracle import analytic
    rb0, _ = _paper_value("fick_rho_cbar")
    rH, _ = _paper_value("fick_rho_H")
    g, _ = _paper_value("fick_g")
    nz = 128
    L = oracle_mod.Lattice(dict(nx=4, ny=4, nz=nz, G=g, rho_H=rH, geometry=1, sink_z0=0, sink_layers=1,
                                wall_z0=nz - 2, wall_thickness=2))
    L.init_fields(np.zeros((nz, 4, 4)), np.full((nz, 4, 4), rb0))
    T = 3000
    L.step(T)
    r, b = L.fields()
    pr, pb = r.mean(axis=(1, 2)), b.mean(axis=(1, 2))
    D = analytic.diffusion_coefficient(rH / 2, rb0, g)
    an = analytic.erfc_profile(np.arange(nz), T, D, rH)
    assert np.max(np.abs(pr[:60] - an[:60])) < 0.01 * rH
    j = L.flux_field()[2].mean(axis=(1, 2))
    grad = np.gradient(pr)
    Dl = analytic.diffusion_coefficient(pr[2:30], pb[2:30], g)
    ratio = j[2:30] / (-Dl * grad[2:30])
    assert np.all(np.abs(ratio - 1) < 0.01), ratio


# ---------------------------------------------------------------- the paper's film experiment

@pytest.fixture(scope="module")
def equilibrated_film(oracle_mod):
    """Sec. III B film: 128 sites normal to the film, 4x4 cross-section, wall of
    thickness 2 at the bottom, init 0.70/0.04 with the interface at 64, g = 3.6."""
    L = oracle_mod.Lattice(dict(nx=4, ny=4, nz=128, G=3.6, wall_z0=0, wall_thickness=2))
    L.init_shape(dict(shape=0, film_z=64, rho_hi=0.70, rho_lo=0.04))
    L.step(20000)
    return L


def test_film_equilibrium_matches_paper(equilibrated_film):
    r, _ = equilibrated_film.fields()
    pr = r.mean(axis=(1, 2))
    rho_ma, tol_ma = _paper_value("film_rho_ma")
    rho_mi, tol_mi = _paper_value("film_rho_mi")
    width, tol_w = _paper_value("film_width_2d0")
    assert abs(pr[20:50].mean() - rho_ma) < tol_ma
    assert abs(pr[80:115].mean() - rho_mi) < tol_mi
    # interface width: sites between 10% and 90% of the density jump
    lo, hi = pr[80:115].mean(), pr[20:50].mean()
    frac = (pr[40:90] - lo) / (hi - lo)
    w = np.count_nonzero((frac > 0.1) & (frac < 0.9))
    assert abs(w - width) <= tol_w
    assert abs(equilibrated_film.diagnostics()["interface_z"] - 63.5) < 1.0


def test_film_evaporation_flux_law(oracle_mod):
    """Sec. III B: with the sink open the vapour profile becomes linear and the
    evaporation rate per area follows Eq. (fick-linear-0)."""
    from oracle import analytic
    nz = 64
    base = dict(nx=4, ny=4, nz=nz, G=3.6, wall_z0=0, wall_thickness=2)
    L = oracle_mod.Lattice(base)
    L.init_shape(dict(shape=0, film_z=24, rho_hi=0.70, rho_lo=0.04))
    L.step(10000)
    f = L.populations()
    r, b = L.fields()
    rho_mi = r.mean(axis=(1, 2))[36:50].mean()
    rho_b_ma = b.mean(axis=(1, 2))[40]
    D = analytic.diffusion_coefficient(rho_mi, rho_b_ma, 3.6)
    for rH in (0.01, 0.02):
        M = oracle_mod.Lattice(dict(base, geometry=1, sink_z0=nz - 1, sink_layers=1, rho_H=rH))
        M.set_populations(f)
        d0 = M.diagnostics()
        M.step(8000)
        d = M.diagnostics()
        j_th = analytic.film_flux(D, rho_mi, rH, nz - 1, d["interface_z"], 2.5)
        assert abs(d["flux_last"] / 16 / j_th - 1) < 0.08
        assert d["interface_z"] < d0["interface_z"]
        assert abs((d["mass_r"] + d["evaporated_mass"]) - (d0["mass_r"] + d0["evaporated_mass"])) < 1e-9


def test_total_momentum_conserved_with_self_couplings(oracle_mod):
    """With the self couplings of Eq. (3) (sum over cbar including c) the force still
    vanishes pairwise over a periodic lattice, so total momentum stays exact. Unequal
    g^{rr} and g^{bb} make a self term built from the wrong component's Psi break it."""
    nx, ny, nz = 6, 5, 7
    L = oracle_mod.Lattice(dict(nx=nx, ny=ny, nz=nz, G=2.0, G_rr=-1.3, G_bb=0.6, tau_r=1.0, tau_b=0.9))
    L.set_populations(_random_state(nx, ny, nz, 14))
    c, _, _ = oracle_mod.tables()

    def mom():
        return np.einsum("cin,ia->a", L.populations().reshape(2, Q, -1), c.astype(np.float64))

    p0 = mom()
    L.step(30)
    assert np.allclose(mom(), p0, atol=1e-13)


def _sc_coexistence(g):
    from tests.sc_eos import sc_coexistence
    return sc_coexistence(g)


@pytest.mark.parametrize("g", [-4.5, -5.0, -6.0])
def test_single_component_coexistence_matches_mechanical_stability(oracle_mod, g):
    """The multiphase pseudopotential model the paper names as an extension: component
    b absent, g^{rr} = g below the critical -4 (Psi = 1/2, rho = ln 2). A flat liquid
    slab in a periodic 1 x 1 x 80 column settles to the coexistence densities of the
    mechanical-stability condition (the lattice adds under 1%); b stays exactly zero."""
    rg, rl = _sc_coexistence(g)
    assert rg < np.log(2.0) < rl
    nz = 80
    z = np.arange(nz)
    rho = np.where((z >= 20) & (z < 60), rl, rg).reshape(nz, 1, 1).astype(np.float64)
    L = oracle_mod.Lattice(dict(nx=1, ny=1, nz=nz, G=0.0, G_rr=g, G_bb=0.0))
    L.init_fields(rho, np.zeros_like(rho))
    L.step(10000)
    rr, rb = L.fields()
    assert abs(rr[40, 0, 0] / rl - 1.0) < 2e-3
    assert abs(rr[0, 0, 0] / rg - 1.0) < 1e-2
    assert np.all(rb == 0.0)


def test_self_coupling_separates_phases_inside_the_spinodal(oracle_mod):
    """A 1% density wave about rho = ln 2 (inside the spinodal for g < -4) grows to the
    coexistence densities with g^{rr} = -5 and decays without self coupling."""
    nz = 64
    z = np.arange(nz)
    rho = (np.log(2.0) * (1.0 + 0.01 * np.cos(2 * np.pi * z / nz))).reshape(nz, 1, 1)
    rg, rl = _sc_coexistence(-5.0)
    out = {}
    for g in (-5.0, 0.0):
        L = oracle_mod.Lattice(dict(nx=1, ny=1, nz=nz, G=0.0, G_rr=g))
        L.init_fields(rho, np.zeros_like(rho))
        L.step(10000)
        out[g] = L.fields()[0]
    assert abs(out[-5.0].max() / rl - 1.0) < 5e-3 and abs(out[-5.0].min() / rg - 1.0) < 2e-2
    assert out[0.0].max() - out[0.0].min() < 1e-3 * np.log(2.0)
