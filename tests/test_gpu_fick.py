"""The diffusion experiment of Sec. III A on the GPU path, at the paper's geometry:
component r enters an r-free 125 x 4 x 4 column of rho^b = 0.7 through the
evaporation boundary (rho_H = 0.001, g = 3.6) and a wall of thickness 2 closes the
far end. The whole profile follows the numerical solution of Eq. (fick2) with the
same boundary values (oracle/analytic.py), except the fluid site next to the wall,
where the force of Eq. (3) sees Psi = 0 at the solid sites and draws the trace
component onto the wall; the early profile is the erfc of Fick's law with the
paper's D^c, and the measured flux rho^r (U^r - U) (Eqs. (flux), (velw), evaluated
on the device) equals -D^c grad rho^r (Eq. (fick-simple)) with D^c at the local
densities."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TIMES = (3000, 10000, 30000)


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


@pytest.fixture(scope="module")
def column(sc):
    from paper_1701_03637_gb300 import experiments as X
    return X.fick_column(nz=125, rho_cbar=0.7, rho_H=0.001, G=3.6, times=TIMES)


def test_paper_column_follows_fick2(column):
    from oracle import analytic as A
    rH = 0.001
    cn = A.fick2_column(122, TIMES, rH, 0.7, 3.6, dt=2.0)
    # the oracle's column lies within 6e-4, 3.1e-3 and 1.2e-2 of rho_H of this solution
    tol = {3000: 1.5e-3, 10000: 6e-3, 30000: 2e-2}
    for rec in column:
        T = rec["t"]
        c, b = cn[T]
        lc, lb = rec["rho_r"][1:123], rec["rho_b"][1:123]  # fluid sites 1..122
        assert np.max(np.abs(lc[:-1] - c[:-1])) < tol[T] * rH, (T, np.max(np.abs(lc[:-1] - c[:-1])) / rH)
        assert np.max(np.abs(lb[:-1] - b[:-1])) < 2e-3, T
        assert abs(lc.sum() - c.sum()) < 5e-3 * c.sum(), T


def test_early_profile_and_flux(column):
    from oracle import analytic as A
    rH, rb0, g = 0.001, 0.7, 3.6
    D = float(A.diffusion_coefficient(rH / 2, rb0, g))
    for rec in column[:2]:
        z = np.arange(len(rec["rho_r"]))
        an = A.erfc_profile(z, rec["t"], D, rH)
        reach = int(min(100, 3 * np.sqrt(D * rec["t"])))
        assert np.max(np.abs(rec["rho_r"][:reach] - an[:reach])) < 0.01 * rH, rec["t"]
        grad = np.gradient(rec["rho_r"])
        Dl = A.diffusion_coefficient(rec["rho_r"][2:30], rec["rho_b"][2:30], g)
        ratio = rec["flux"][2:30] / (-Dl * grad[2:30])
        assert np.all(np.abs(ratio - 1) < 0.02), (rec["t"], ratio)
