"""A second, literal writing of the relative flux of Sec. III A (test helper):
j^r = rho^r (U^r - U) with the velocities of Eq. (velw) at tau = 1, in numpy on
canonical populations, used to pin the oracle's C evaluation (orc_flux_field)."""
import numpy as np


def paper_flux_z(f, c, w, G):
    """z flux of component r relative to the mixture, j^r = rho^r (U^r - U), with
    the velocities of Eq. (velw) at tau = 1: U = (m^r + m^b + (F^r + F^b) / 2) /
    (rho^r + rho^b) and U^r = (m^r + F^r + rho^r u') / (2 rho^r), u' the common
    velocity and F^c = -g Psi^c(x) sum_i w_i Psi^cbar(x + e_i) e_i (Eq. (3),
    periodic neighbours; solid sites have rho = Psi = 0; the paper's cross coupling
    only). f: canonical populations [2][19][z][y][x] (FP64); c, w: a direction table."""
    rho = f.sum(axis=1)
    m = np.tensordot(c.astype(np.float64).T, f, axes=([1], [1]))  # [3][2][z][y][x]
    psi = -np.expm1(-rho)
    acc = np.zeros((2, 3) + rho.shape[1:])
    for i in range(1, len(w)):
        e = c[i]
        for cc in (0, 1):
            pn = np.roll(psi[1 - cc], shift=(-int(e[2]), -int(e[1]), -int(e[0])), axis=(0, 1, 2))
            for d in range(3):
                if e[d]:
                    acc[cc, d] += w[i] * pn * e[d]
    F = -G * psi[:, None] * acc  # [2][3][...]
    rr, rb = rho[0], rho[1]
    rt = np.maximum(rr + rb, 1e-300)
    up = (m[2, 0] + m[2, 1]) / rt  # tau_r = tau_b: the common velocity is the mixture momentum / mass
    U = (m[2, 0] + m[2, 1] + 0.5 * (F[0, 2] + F[1, 2])) / rt
    with np.errstate(divide="ignore", invalid="ignore"):
        Ur = np.where(rr > 0, (m[2, 0] + F[0, 2] + rr * up) / (2.0 * rr), 0.0)
    return np.where(rr > 0, rr * (Ur - U), 0.0)
