"""Multi-rank partition on CPU (gloo, world size 2): the strong partition's
union equals the unsplit suspension, each rank's cells advanced by the
oracle match the unsplit run bitwise, and the weak partition gives each
rank its own suspension.  Timing follows the bench's rule (max over ranks)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1911_03062_gb300 import inputs as I
from paper_1911_03062_gb300.shard import cell_range, shard_groups


def test_cell_range_covers_exactly():
    for n in (0, 1, 7, 55000):
        for world in (1, 2, 3, 8):
            spans = [cell_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    try:
        _rank_body(rank, world, port, out)
    except BaseException as e:          # report instead of leaving the parent waiting
        out.put(("error", f"rank {rank}: {e!r}"))
        raise


def _rank_body(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    groups = shard_groups("rbc10k_plt1500", rank, world, "strong", scale=0.0008)   # 8 RBC + 1 PLT
    xs = []
    for g in groups:
        if g.n_cells == 0:
            xs.append(np.zeros((0, g.mtype.nV, 3)))
            continue
        T = O.OracleType.from_mesh_type(g.mtype)
        x, _ = T.step_cells(g.x0, g.v0, g.f_ext, K=10, m=5)
        xs.append(x)
    flat = torch.from_numpy(np.concatenate([x.ravel() for x in xs]))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([flat.numel()]))
    nmax = int(max(s.item() for s in sizes))
    padded = torch.zeros(nmax, dtype=torch.float64)
    padded[:flat.numel()] = flat
    buf = [torch.zeros(nmax, dtype=torch.float64) for _ in sizes]
    dist.all_gather(buf, padded)     # test-side gather of results (not on the solver's path)
    buf = [b[:int(s.item())] for b, s in zip(buf, sizes)]
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put(([b.numpy() for b in buf], float(t.item())))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_strong_partition_matches_unsplit():
    from oracle import oracle as O
    O.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=240)
    assert got[0] != "error", got[1]
    parts, tmax = got
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 2.0
    # unsplit reference, re-assembled in the ranks' order
    groups = [I.materialise(g) for g in I.workload_groups("rbc10k_plt1500", 0.0008)]
    per_rank = [[] for _ in range(world)]
    for g in groups:
        T = O.OracleType.from_mesh_type(g.mtype)
        x, _ = T.step_cells(g.x0, g.v0, g.f_ext, K=10, m=5)
        for r in range(world):
            lo, hi = cell_range(g.n_cells, r, world)
            per_rank[r].append(x[lo:hi].ravel())
    for r in range(world):
        assert np.array_equal(parts[r], np.concatenate(per_rank[r]))


def test_weak_partition_gives_distinct_suspensions():
    a = shard_groups("rbc1", 0, 2, "weak")
    b = shard_groups("rbc1", 1, 2, "weak")
    assert a[0].n_cells == b[0].n_cells == 1
    assert not np.allclose(a[0].x0, b[0].x0)
    c = shard_groups("rbc1", 1, 2, "weak")
    assert np.array_equal(b[0].f_ext, c[0].f_ext)
