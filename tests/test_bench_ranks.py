"""The multi-rank path of bench.py on CPU (gloo, world size 2, no GPU).

Weak scaling: every rank draws its own workload (seed 1 + rank) and the
only collective is the final reduction, the particle-steps summed and the
time maximised over the ranks, so value = all ranks' particle-steps / the
slowest rank's time."""
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # per-rank measurements: particle-steps and seconds
        psteps, secs = 1000.0 * (rank + 1), 0.5 + 0.25 * rank
        tot, mx = bench.combine_ranks([(psteps, "sum"), (secs, "max")])
        # each rank its own beam: the seeds, and so the momenta, differ
        bench.scale_workload(2000)
        w = bench.make_workload(seed=bench.rank_seed(rank))
        p = torch.tensor(w.particles[0][1][:, 0].copy())
        g = [torch.zeros_like(p) for _ in range(world)]
        tdist.all_gather(g, p)
        same = bool(torch.equal(g[0], g[1]))
        out[rank] = (tot, mx, tot / mx, same, bench.rank_seed(rank))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_reduce_and_draw_their_own_workloads():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        tot, mx, value, same, seed = res[r]
        assert tot == 3000.0 and mx == 0.75 and value == 4000.0
        assert not same and seed == r + 1


def test_one_rank_is_unchanged():
    import bench
    assert bench.combine_ranks([(5.0, "sum"), (2.0, "max")]) == [5.0, 2.0]
