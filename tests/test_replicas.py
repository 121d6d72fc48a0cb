"""The multi-process path of bench.py (N replicas, one per GPU, launched by
torchrun): rank discovery from the launcher's environment, the barrier and
the maximum over ranks of the timed region, and the reference arm that runs
on rank 0 only.  The coupled step does not shard (independent replicas, no
collective on the data path), so only this host logic runs on several
processes; here as CPU ranks over gloo, world size 2."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    ws, r, local = bench._dist()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench._barrier(ws)
        # each rank's timed region; the job's time is the slowest rank's
        m = bench._barrier_and_max(10.0 * (rank + 1), ws)
        out = io.StringIO()
        ran = None
        if rank == 1:
            # the reference arm prints from rank 0 only; other ranks leave at once
            args = bench.parse_args(["--impl", "reference", "--gpus", "2"])
            with contextlib.redirect_stdout(out):
                ran = bench.run_reference(args)
        bench._barrier(ws)
        q.put((rank, ws, r, local, m, out.getvalue(), ran))
    finally:
        dist.destroy_process_group()


def test_two_replicas_share_barrier_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r_rank, ws, r, local, m, out, ran) in enumerate(res):
        assert (r_rank, ws, r, local) == (rank, 2, rank, rank)
        assert m == 20.0
    assert res[1][5] == "" and res[1][6] is None
