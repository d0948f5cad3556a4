"""The evaporating planar film of Sec. III B on the GPU path over the paper's
10^6 steps: the interface must recede as Eq. (xit) predicts -- the quasi-steady
linear vapour profile between x_I + d0 and the sink plane x_H, whose flux moves
the interface -- integrated from the measured state (coexistence densities of
the equilibrated profile, vapour-state D^c of Sec. III A, d0 = 2.5). The law is
taken in the ODE's own closed form; the paper's printed Eq. (xt) (with x_H + d0)
is reported beside it. Paper densities 0.70 / 0.04; rho_H = 0.02 (10^6 steps)
and 0.01 (4 x 10^5 steps, before the film is gone). With rho_H = 0.03 the
driving difference rho_mi - rho_H is 0.007 and the film recedes ~20% slower than
the law: a 0.0015 shift of the vapour density at an evaporating interface from
its equilibrium value moves the rate by that much."""
import json
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


@pytest.mark.parametrize("rho_H,steps", [(0.02, 1_000_000), (0.01, 400_000)])
def test_film_interface_follows_the_evaporation_law(sc, rho_H, steps):
    from oracle import analytic as A
    from paper_1701_03637_gb300 import experiments as X
    run = X.evaporating_film(rho_H=rho_H, steps=steps, every=20000)
    t, x = run["t"], run["x_I"]
    D = float(A.diffusion_coefficient(run["rho_mi"], run["rho_b_vap"], run["G"]))
    t0 = 50000.0  # after the diffusive set-up of the vapour profile ((x_H - x_I)^2 / D ~ 8e4 at most)
    x0 = float(np.interp(t0, t, x))
    T = t[-1] - t0
    args = (run["x_H"], 2.5, D, run["rho_ma"], run["rho_mi"], rho_H)
    law = float(A.film_xI(T, x0, *args)) - x0
    printed = float(A.film_xI_printed(T, x0, *args)) - x0
    sim = float(x[-1]) - x0
    rec = dict(rho_H=rho_H, D=D, x0=x0, T=T, dx_sim=sim, dx_law=law, dx_printed=printed, rho_ma=run["rho_ma"],
               rho_mi=run["rho_mi"], rho_b_vap=run["rho_b_vap"], t=t.tolist(), x_I=x.tolist())
    save(f"film_law_{rho_H}.json", rec)
    print(json.dumps({k: v for k, v in rec.items() if k not in ("t", "x_I")}))
    assert sim < 0
    # measured: 3.5% (rho_H = 0.02), 6.7% (0.01; the vapour D^c rises towards the sink)
    assert abs(sim - law) < 0.10 * abs(law), (sim, law, printed)
