"""Error of the stored-precision variants against the FP64 oracle on the same
seeded droplet (the floating droplet of Sec. III C; radius / box = 0.1875 as in
the 128^3 and 512^3 workloads): density L-infinity and L2 errors and the droplet
size after N steps, for FP32 populations and for FP16 / BF16 offsets
h_i = f_i - w_i rho0 (rho0 = 1) with FP32 arithmetic, and for FP16 of the
scaled populations g_i = f_i / w_i.

Bounds: FP32 carries ~1e-7 relative rounding per step (parity bar 1e-4 after
1000 steps). An FP16 offset store rounds h to 11 significant bits: |h| <= w_i
gives at most 2^-12 w_i absolute per store and per step, a random walk whose
density effect after n steps is of order 2^-12 sqrt(n) ~ 8e-3 at n = 1000 and
is damped where the dynamics is diffusive; BF16 has 8 significant bits (8x
FP16). The tests assert those orders and record the measured values.
"""
import os

import numpy as np
import pytest

from tests.results import save

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


def _study(sc, oracle_mod, n, steps):
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(n, 0.1875 * n, 1)
    o = oracle_mod.Lattice(params)
    o.init_shape(init)
    o.step(steps)
    orr, ob = o.fields()
    od = o.diagnostics()
    out = {}
    for st in ("f32", "f16", "bf16", "f16s"):
        g = sc.Lattice(dict(params, storage=st))
        g.init(init)
        g.step(steps)
        gr, gb = g.read_fields()
        d = g.diagnostics()
        g.close()
        e = np.concatenate([(gr - orr).ravel(), (gb - ob).ravel()])
        out[st] = dict(linf=float(np.max(np.abs(e))), l2=float(np.sqrt(np.mean(e * e))),
                       radius=d["radius"], radius_oracle=od["radius"],
                       droplet_sites=d["droplet_sites"], droplet_sites_oracle=od["droplet_sites"],
                       mass_r=d["mass_r"], mass_r_oracle=od["mass_r"])
    return out


def _record(name, out):
    save(f"precision_{name}.json", out)


def test_precision_vs_oracle_64(sc, oracle_mod):
    out = _study(sc, oracle_mod, 64, 1000)
    _record("64_1000", out)
    assert out["f32"]["linf"] < 1e-4
    assert out["f16"]["linf"] < 3e-2 and out["bf16"]["linf"] < 0.25 and out["f16s"]["linf"] < 3e-2
    assert out["f16"]["l2"] < 4e-3
    assert abs(out["f32"]["radius"] - out["f32"]["radius_oracle"]) < 1e-3
    assert abs(out["f16"]["radius"] - out["f16"]["radius_oracle"]) < 0.5


def test_film_interface_vs_oracle(sc, oracle_mod):
    """Interface position of the 4x4x128 film (paper densities 0.70 / 0.04,
    rho_H = 0.02) after 2000 steps in every storage against the FP64 oracle."""
    from paper_1701_03637_gb300.workloads import film_4x4x128
    params, init = film_4x4x128(rho_hi=0.70, rho_lo=0.04, rho_H=0.02)
    o = oracle_mod.Lattice(params)
    o.init_shape(init)
    o.step(2000)
    od = o.diagnostics()
    out = {}
    for st in ("f32", "f16", "bf16", "f16s"):
        g = sc.Lattice(dict(params, storage=st))
        g.init(init)
        g.step(2000)
        d = g.diagnostics()
        g.close()
        out[st] = dict(interface_z=d["interface_z"], interface_z_oracle=od["interface_z"],
                       error=abs(d["interface_z"] - od["interface_z"]),
                       evaporated_mass=d["evaporated_mass"], evaporated_mass_oracle=od["evaporated_mass"])
    _record("film_2000", out)
    assert out["f32"]["error"] < 1e-3
    assert out["f16"]["error"] < 0.5 and out["f16s"]["error"] < 0.5 and out["bf16"]["error"] < 2.0


@pytest.mark.slow
def test_precision_vs_oracle_128(sc, oracle_mod):
    """The 128^3 droplet (radius 24, the crop-equivalent of the 512^3 workload): the
    error of every storage type against the FP64 oracle after 1000 steps (about three
    minutes of oracle time on 16 cores)."""
    out = _study(sc, oracle_mod, 128, 1000)
    _record("128_1000", out)
    assert out["f32"]["linf"] < 1e-4
    assert abs(out["f32"]["radius"] - out["f32"]["radius_oracle"]) < 1e-3
    # the L-infinity error is the tail of the per-site error over 4.2M sites (it was 2.0e-2
    # over the 64^3 droplet's 262k): 3.4e-2 measured in FP16 offsets, 2.2e-2 in scaled FP16
    assert out["f16"]["linf"] < 6e-2 and out["f16s"]["linf"] < 6e-2 and out["bf16"]["linf"] < 0.25
    assert out["f16"]["l2"] < 4e-3 and out["f16s"]["l2"] < 4e-3
    assert abs(out["f16"]["radius"] - out["f16"]["radius_oracle"]) < 0.5


@pytest.mark.skipif(os.environ.get("SC_PAPER_SCALE") != "1",
                    reason="5000 oracle steps of a 128^3 lattice (about fifteen minutes): set SC_PAPER_SCALE=1")
def test_precision_vs_oracle_128_5000(sc, oracle_mod):
    """The same study over 5000 steps, the run length of the large-droplet precision
    case. Bounds scale the 1000-step ones: the FP32 rounding linearly in the steps
    (5x), the FP16 / BF16 store rounding as a random walk (sqrt(5) x)."""
    out = _study(sc, oracle_mod, 128, 5000)
    _record("128_5000", out)
    assert out["f32"]["linf"] < 5e-4
    assert abs(out["f32"]["radius"] - out["f32"]["radius_oracle"]) < 5e-3
    assert out["f16"]["linf"] < 0.14 and out["f16s"]["linf"] < 0.14 and out["bf16"]["linf"] < 0.56
    assert out["f16"]["l2"] < 9e-3 and out["f16s"]["l2"] < 9e-3
    assert abs(out["f16"]["radius"] - out["f16"]["radius_oracle"]) < 1.12
