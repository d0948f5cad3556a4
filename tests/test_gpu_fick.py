"""The diffusion experiment of Sec. III A on the GPU path: component r enters an
r-free column through the evaporation boundary (rho_H = 0.001, rho^b = 0.7,
g = 3.6). The profile follows the erfc solution of Fick's law with the paper's
D^c at 3000 and 10000 steps, and the measured flux rho^r (U^r - U) equals
-D^c grad rho^r (Eq. (fick-simple)) with D^c at the local densities."""
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


def test_fick_column_profile_and_flux(sc):
    from oracle import analytic as A
    from paper_1701_03637_gb300 import experiments as X
    rH, rb0, g = 0.001, 0.7, 3.6
    D = float(A.diffusion_coefficient(rH / 2, rb0, g))
    for rec in X.fick_column(rho_cbar=rb0, rho_H=rH, G=g, times=(3000, 10000)):
        z = np.arange(len(rec["rho_r"]))
        an = A.erfc_profile(z, rec["t"], D, rH)
        reach = int(min(100, 3 * np.sqrt(D * rec["t"])))
        assert np.max(np.abs(rec["rho_r"][:reach] - an[:reach])) < 0.01 * rH, rec["t"]
        grad = np.gradient(rec["rho_r"])
        Dl = A.diffusion_coefficient(rec["rho_r"][2:30], rec["rho_b"][2:30], g)
        ratio = rec["flux"][2:30] / (-Dl * grad[2:30])
        assert np.all(np.abs(ratio - 1) < 0.02), (rec["t"], ratio)
