"""Row-range sharding across 2 ranks (gloo, CPU): partial fields of disjoint
row ranges, summed by all_reduce, equal the full-aperture field.  The partial
fields here come from the CPU oracle; on GPUs the same function sums
Plan.propagate_roi partials over NCCL."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2609_01978_gb300.shard import chord_weights, propagate_sharded
    g = O.Geometry(D=4e-3 / 4, f=20e-3 / 4, lam=632.8e-9, M=64, p=0.3e-6)
    dx2, R2 = g.dx * g.dx, g.R * g.R
    sR = int(R2 // dx2)
    while (sR + 1) * dx2 <= R2:
        sR += 1
    while sR * dx2 > R2:
        sR -= 1
    w = chord_weights(g.N, g.c, sR)

    def partial(j0, j1):
        U = O.field_czt(g, j0, j1) if j1 > j0 else np.zeros((g.M, g.M), complex)
        return torch.from_numpy(np.ascontiguousarray(U))

    U = propagate_sharded(partial, g.N, weights=w)
    if rank == 0:
        out.put(U.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_row_ranges_cover_and_balance():
    from paper_2609_01978_gb300.shard import row_ranges
    r = row_ranges(10, 3)
    assert r[0][0] == 0 and r[-1][1] == 10 and all(a[1] == b[0] for a, b in zip(r, r[1:]))
    w = [0, 0, 5, 5, 5, 5, 5, 5, 0, 0]
    rw = row_ranges(10, 2, w)
    assert sum(w[rw[0][0]:rw[0][1]]) == 15 and rw[-1][1] == 10 and rw[0][1] == rw[1][0]


def test_two_rank_gloo_sum_equals_full_field():
    import multiprocessing as mp
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    U = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g = O.Geometry(D=4e-3 / 4, f=20e-3 / 4, lam=632.8e-9, M=64, p=0.3e-6)
    ref = O.field_czt(g)
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-12


def test_chord_weights_count_the_aperture(oracle_mod):
    """The shard balance weights (samples of each row inside the disc) sum to
    the oracle's aperture count, and the weighted split gives each of four
    ranks close to a quarter of the open samples."""
    from paper_2609_01978_gb300.shard import chord_weights, row_ranges
    O = oracle_mod
    for D, f in [(4e-3, 20e-3), (0.05, 0.25)]:
        g = O.Geometry(D=D, f=f, lam=632.8e-9, M=64, p=0.3e-6)
        dx2, R2 = g.dx * g.dx, g.R * g.R
        sR = int(R2 // dx2)
        while (sR + 1) * dx2 <= R2:
            sR += 1
        while sR * dx2 > R2:
            sR -= 1
        w = chord_weights(g.N, g.c, sR)
        assert sum(w) == O.count_aperture(g)
        rr = row_ranges(g.N, 4, w)
        share = [sum(w[a:b]) / sum(w) for a, b in rr]
        assert rr[0][0] == 0 and rr[-1][1] == g.N
        assert max(abs(x - 0.25) for x in share) < 2.0 * max(w) / sum(w) + 1e-12
