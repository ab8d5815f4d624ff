"""A CPU model of the multi-GPU form the design leaves out (row strips with a
halo exchange, as the paper's Sec. 4 does with column strips over MPI): each
strip updates only its own rows from halo copies of its neighbours' edge rows.
Because the draws are keyed by site, any partition reproduces the unpartitioned
chain bit-exactly.  Single process with P strips, and two gloo ranks that
exchange halo rows with send/recv."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle


def strips(L, P):
    b = [L * p // P for p in range(P + 1)]
    return [(b[p], b[p + 1]) for p in range(P)]


@pytest.mark.parametrize("L,P", [(16, 2), (16, 4), (18, 3), (24, 5)])
def test_strip_partition_equals_full_lattice(L, P):
    seed, beta, n = 31, 0.43, 6
    full = oracle.init_hot(L, seed)
    local = [full.copy() for _ in range(P)]       # each strip's own copy of the lattice
    parts = strips(L, P)
    for t in range(1, n + 1):
        for c in (0, 1):
            oracle.half_sweep(full, seed, t, c, beta)
            # halo exchange: every strip receives its neighbours' edge rows
            for p, (i0, i1) in enumerate(parts):
                for q, (j0, j1) in enumerate(parts):
                    if q != p:
                        local[p][j0:j1] = local[q][j0:j1]
            for p, (i0, i1) in enumerate(parts):
                oracle.half_sweep_rows(local[p], seed, t, c, beta, i0, i1)
    merged = np.concatenate([local[p][i0:i1] for p, (i0, i1) in enumerate(parts)])
    np.testing.assert_array_equal(merged, full)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, L, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed, beta, n = 77, 0.44, 5
    i0, i1 = L * rank // world, L * (rank + 1) // world
    s = oracle.init_hot(L, seed)                  # every rank starts from the same lattice
    up, down = (rank - 1) % world, (rank + 1) % world
    for t in range(1, n + 1):
        for c in (0, 1):
            # ring exchange of the edge rows (the paper's blocking send/recv pattern)
            first = torch.from_numpy(s[i0].copy())
            last = torch.from_numpy(s[i1 - 1].copy())
            halo_above = torch.empty(L, dtype=torch.int8)
            halo_below = torch.empty(L, dtype=torch.int8)
            reqs = [dist.isend(first, up, tag=1), dist.isend(last, down, tag=2),
                    dist.irecv(halo_above, up, tag=2), dist.irecv(halo_below, down, tag=1)]
            for r in reqs:
                r.wait()
            s[(i0 - 1) % L] = halo_above.numpy()
            s[i1 % L] = halo_below.numpy()
            oracle.half_sweep_rows(s, seed, t, c, beta, i0, i1)
    out[rank] = s[i0:i1].copy()
    dist.barrier()
    dist.destroy_process_group()


def test_strip_partition_with_two_gloo_ranks():
    L, world = 20, 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, L, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        merged = np.concatenate([out[0], out[1]])
    full = oracle.init_hot(L, 77)
    oracle.run(full, 77, 0.44, 0, 5, 5)
    np.testing.assert_array_equal(merged, full)
