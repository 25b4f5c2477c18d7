"""Host logic of the N > 1 benchmark path (replicas only: no collective on the
data path), run as two gloo ranks on the CPU: every rank draws its own noise,
the whole-job time is the slowest rank's and the bytes are summed over ranks,
and the reference arm runs on rank 0 alone."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from oracle import noise
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    ms, nbytes = bench.combine_ranks(dist, 10.0 + rank, 100.0 * (rank + 1), 'cpu')
    eta = noise.rademacher(bench.rank_seed(rank), 0, 64)
    gathered = [None] * world
    dist.all_gather_object(gathered, eta.tolist())
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, nbytes, gathered))


def test_two_replicas():
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, nbytes, gathered in res:
        assert ms == 11.0                  # the slowest rank's time
        assert nbytes == 300.0             # the bytes of all ranks
        a, b = np.array(gathered[0]), np.array(gathered[1])
        assert not np.array_equal(a, b)    # each replica draws its own noise


def test_reference_arm_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv('RANK', '1')
    monkeypatch.setenv('WORLD_SIZE', '2')

    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(Args())          # rank 1: no work, no line
    assert capsys.readouterr().out == ''
