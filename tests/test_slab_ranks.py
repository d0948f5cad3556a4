"""The z-slab decomposition's host logic on the CPU with 2 and 4 gloo ranks.

Each rank holds one slab of a periodic lattice (forces across every face, self
couplings, unequal tau) as an FP64 oracle lattice of its planes plus 2 ghost planes
per side; before every step the ranks exchange their 2 boundary planes through
paper_1701_03637_gb300.slab.exchange_ring (the same function that sends device
buffers over NCCL), and each rank's own planes must then equal the same planes of
the whole lattice stepped by the oracle, bit for bit (the oracle's step is per site
and deterministic, and the ghost planes give every own site the neighbourhood it has
in the whole lattice)."""
import os
import socket

import numpy as np
import pytest

Q = 19
PARAMS = dict(nx=5, ny=4, nz=13, tau_r=0.9, tau_b=1.15, G=3.3, G_rr=-0.6, G_bb=0.25, rho_H=0.03, geometry=0)
STEPS = 6


def _state():
    from paper_1701_03637_gb300.workloads import random_populations
    return random_populations(PARAMS["nx"], PARAMS["ny"], PARAMS["nz"], seed=77, rho=(0.45, 0.35))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1701_03637_gb300.slab import GHOSTS, exchange_ring, slab_ranges
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.set_threads(1)
        f = _state()
        nz = PARAMS["nz"]
        z0, z1 = slab_ranges(nz, world)[rank]
        idx = [(z - GHOSTS) % nz for z in range(z0, z1 + 2 * GHOSTS)]  # local planes: ghosts, own, ghosts
        local = oracle.Lattice(dict(PARAMS, nz=len(idx)))
        fl = f[:, :, idx].copy()
        face = fl[:, :, :GHOSTS].shape
        recv_low = torch.zeros(face, dtype=torch.float64)
        recv_high = torch.zeros(face, dtype=torch.float64)
        for _ in range(STEPS):
            send_low = torch.from_numpy(np.ascontiguousarray(fl[:, :, GHOSTS:2 * GHOSTS]))
            send_high = torch.from_numpy(np.ascontiguousarray(fl[:, :, -2 * GHOSTS:-GHOSTS]))
            exchange_ring(send_low, send_high, recv_low, recv_high, rank, world, dist)
            fl[:, :, :GHOSTS] = recv_low.numpy()
            fl[:, :, -GHOSTS:] = recv_high.numpy()
            local.set_populations(fl)
            local.step(1)
            fl = local.populations()
        whole = oracle.Lattice(PARAMS)
        whole.set_populations(f)
        whole.step(STEPS)
        want = whole.populations()[:, :, z0:z1]
        got = fl[:, :, GHOSTS:-GHOSTS]
        out.put((rank, bool(np.array_equal(got, want)), float(np.max(np.abs(got - want)))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slabs_over_gloo_ranks_equal_the_whole_lattice(oracle_mod, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, same, err in sorted(results):
        assert same, (world, rank, err)


def test_slab_ranges_cover_the_lattice_once():
    from paper_1701_03637_gb300.slab import slab_ranges
    for nz in (4, 13, 128, 512):
        for parts in (1, 2, 3, 4, 8):
            if nz < 2 * parts:
                with pytest.raises(ValueError):
                    slab_ranges(nz, parts)
                continue
            r = slab_ranges(nz, parts)
            assert r[0][0] == 0 and r[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [z1 - z0 for z0, z1 in r]
            assert min(sizes) >= 2 and max(sizes) - min(sizes) <= 1


def test_single_rank_is_its_own_neighbour():
    import torch
    from paper_1701_03637_gb300.slab import exchange_ring
    lo, hi = torch.arange(6.0), torch.arange(6.0) + 10
    rl, rh = torch.zeros(6), torch.zeros(6)
    exchange_ring(lo, hi, rl, rh, 0, 1)
    assert torch.equal(rl, hi) and torch.equal(rh, lo)
