"""The N > 1 path of bench.py on the CPU: the solve does not shard, so N GPUs run
N independent replicas. What remains for several ranks is host logic: the
whole-job rate from the slowest rank's time (an all-reduce over `gloo`
here, NCCL under the GPU bench) and the reference arm, which rank 0 alone runs
and prints under torchrun."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_worker(rank, world, port, ms_of_rank, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + bench.replica_rate(ms_of_rank[rank], 4, world, dist, "cpu"))
    finally:
        dist.destroy_process_group()


def test_replica_rate_max_over_ranks_gloo():
    """Two ranks that timed 4 units in 120 and 250 ms: both report the max
    (250 ms) and the job rate 2 x 4 / 0.25 s = 32 units/s."""
    import bench
    world, ms_of_rank = 2, [120.0, 250.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, world, port, ms_of_rank, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms in out:
        assert ms == 250.0, (rank, ms)
        assert abs(rate - 32.0) < 1e-12, (rank, rate)
    # one process: its own time, no reduction
    assert bench.replica_rate(250.0, 4, 1) == (16.0, 250.0)


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched as the driver launches N > 1: rank 0
    times the oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
