"""The in-place (AA) addressing scheme as include/sc_lbm.h states it, checked on
the host against direct streaming (Sec. II A: population i moves to x + e_i, or
back to x in direction opp(i) where x + e_i is solid).

A numpy model keeps one slot array. In the even form population i arriving at x
sits at (i, x - e_i), or at (opp(i), x) where x - e_i is solid; in the odd form
at (opp(i), x). A step reads a site's arrived populations and writes its
post-collision f*_j into the slot population opp(j) was read from. With the
identity collision (f* = the arrived populations) the arrived populations after
every step must equal those of direct streaming, and the slots one site writes
must be exactly the slots it read, so no site's update touches another's."""
import numpy as np
import pytest

Q = 19


def _tables():
    from tests.brute_force import VELOCITIES
    e = np.asarray(VELOCITIES, np.int64)
    opp = np.array([int(np.flatnonzero((e == -e[i]).all(axis=1))[0]) for i in range(Q)])
    return e, opp


class Lattice:
    def __init__(self, nx, ny, nz, wall=()):
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        self.xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
        self.solid = np.isin(self.xyz[:, 2], list(wall))
        self.e, self.opp = _tables()

    def site(self, xyz):
        nz, ny, nx = self.shape
        x, y, z = xyz[..., 0] % nx, xyz[..., 1] % ny, xyz[..., 2] % nz
        return x + nx * (y + ny * z)

    def even_slot(self, s, i):
        """(direction, site) holding population i arriving at site s, even form."""
        src = self.site(self.xyz[s] - self.e[i])
        return (int(self.opp[i]), s) if self.solid[src] else (i, int(src))

    def odd_slot(self, s, i):
        return int(self.opp[i]), s

    def stream(self, arrived):
        """Direct streaming of post-collision values f* = arrived (identity collision):
        arrived'_i(x) = f*_i(x - e_i), or f*_opp(i)(x) where x - e_i is solid."""
        out = np.zeros_like(arrived)
        for s in np.flatnonzero(~self.solid):
            for i in range(Q):
                src = self.site(self.xyz[s] - self.e[i])
                out[i, s] = arrived[self.opp[i], s] if self.solid[src] else arrived[i, src]
        return out


def _aa_step(L, A, odd):
    """One in-place step on the slot array A (identity collision). Returns the new
    array and, per fluid site, the slots read and written."""
    slot = L.odd_slot if odd else L.even_slot
    B = A.copy()
    touched = {}
    for s in np.flatnonzero(~L.solid):
        reads = [slot(s, i) for i in range(Q)]
        f = [A[d, x] for d, x in reads]            # arrived populations of s
        writes = [reads[L.opp[j]] for j in range(Q)]  # f*_j into the slot opp(j) came from
        for j, (d, x) in enumerate(writes):
            B[d, x] = f[j]
        touched[int(s)] = (sorted(reads), sorted(writes))
    return B, touched


def _arrived(L, A, odd):
    slot = L.odd_slot if odd else L.even_slot
    out = np.zeros((Q, L.n))
    for s in np.flatnonzero(~L.solid):
        for i in range(Q):
            d, x = slot(s, i)
            out[i, s] = A[d, x]
    return out


@pytest.mark.parametrize("shape,wall", [((3, 3, 3), ()), ((4, 3, 6), (0, 1)), ((1, 2, 5), (2,)),
                                        ((5, 4, 4), (3,))])
def test_in_place_forms_follow_direct_streaming(shape, wall):
    L = Lattice(*shape, wall=wall)
    rng = np.random.default_rng(7)
    arrived = rng.uniform(0.1, 1.0, (Q, L.n))
    arrived[:, L.solid] = 0.0
    # load: the even form of the initial arrived populations
    A = np.zeros((Q, L.n))
    for s in np.flatnonzero(~L.solid):
        for i in range(Q):
            d, x = L.even_slot(s, i)
            A[d, x] = arrived[i, s]
    assert np.array_equal(_arrived(L, A, odd=False), arrived)
    odd = False
    owner = {}
    for step in range(6):
        A, touched = _aa_step(L, A, odd)
        odd = not odd
        arrived = L.stream(arrived)
        assert np.array_equal(_arrived(L, A, odd), arrived), step
        for s, (reads, writes) in touched.items():
            assert reads == writes  # a site writes exactly the slots it read
            for sl in reads:        # and no other site reads or writes them in this step
                assert owner.setdefault((step, sl), s) == s
    # six steps: back in the even form, where the two-lattice pull reads
    assert not odd
