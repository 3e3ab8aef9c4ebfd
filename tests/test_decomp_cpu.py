"""Sharding across ranks on the CPU (gloo, 2 and 4 processes): the replica timing reduction
and the domain decomposition of one grid with halo exchange.  The decomposed run steps each
rank's block with the FP64 reference and must equal the single-domain run bit for bit, for
periodic and no-flux boundaries, splits along x, along y and both, and halo widths 1 to 4
(a remainder block when K does not divide the step count)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import decomp, inputs

NX, NY = 20, 18
RATES = inputs.rates_from_sigma_mu(0.45, 0.2, 0.1, 0.01).as_tuple()
TAU = [oracle.tau_from_d(d) for d in (0.05, 0.05, 0.01, 0.05)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _state():
    st = inputs.random_state(NX, NY, 7)
    st[2] *= 0.05
    return st


def _worker(rank, world, port, px, py, bc, K, nsteps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dec = decomp.Decomposition(NX, NY, px, py, rank, bc)
        block = dec.local(_state())

        def step(ext, k, b):
            return oracle.sslbm_run(ext, TAU, RATES, 1.0, b, k)

        out = decomp.run_decomposed(dec, block, step, nsteps, K)
        full = dec.gather(out)
        t = decomp.max_over_ranks(float(rank + 1), world)
        if rank == 0:
            q.put((full, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, px, py, bc, K, nsteps):
    import torch.multiprocessing as mp
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, px, py, bc, K, nsteps, q)) for r in range(world)]
    for p in procs:
        p.start()
    full, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return full, t


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
@pytest.mark.parametrize("bc", [decomp.BC_PERIODIC, decomp.BC_NOFLUX])
@pytest.mark.parametrize("K", [1, 3])
def test_two_ranks_match_single_domain_bitwise(px, py, bc, K):
    nsteps = 7
    full, t = _run(2, px, py, bc, K, nsteps)
    ref = oracle.sslbm_run(_state(), TAU, RATES, 1.0, bc, nsteps)
    assert np.array_equal(full.view(np.uint64), ref.view(np.uint64))
    assert t == 2.0  # the maximum over ranks of (rank + 1)


@pytest.mark.parametrize("bc", [decomp.BC_PERIODIC, decomp.BC_NOFLUX])
def test_four_ranks_two_by_two_with_corners(bc):
    """A 2 x 2 layout: the corners of the halo come from the diagonal neighbour through the
    two-phase exchange; K = 4 > 1 needs them."""
    full, t = _run(4, 2, 2, bc, 4, 9)
    ref = oracle.sslbm_run(_state(), TAU, RATES, 1.0, bc, 9)
    assert np.array_equal(full.view(np.uint64), ref.view(np.uint64))
    assert t == 4.0


def test_split_and_layout_rules():
    assert decomp.split(10, 3) == [(0, 4), (4, 7), (7, 10)]
    with pytest.raises(ValueError):
        decomp.split(2, 3)
    d = decomp.Decomposition(NX, NY, 2, 2, 3, decomp.BC_NOFLUX)
    assert (d.ix, d.iy) == (1, 1)
    assert d.neighbour(0, 1) is None and d.neighbour(0, -1) == 2 and d.neighbour(1, -1) == 1
    assert d.halo(3) == (3, 0, 3, 0)
    p = decomp.Decomposition(NX, NY, 2, 1, 0, decomp.BC_PERIODIC)
    assert p.neighbour(0, -1) == 1 and p.neighbour(0, 1) == 1 and p.neighbour(1, 1) == 0
    with pytest.raises(ValueError):
        d.extend(np.zeros((5, 2, 2)), 3)
