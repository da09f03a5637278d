"""The multi-process path of bench.py on CPU: two gloo ranks (world size 2).

Each rank of a run is an independent replica; bench.py takes the slowest rank's time (an
all-reduce MAX) and reports the whole job's molecule-steps over it. The reference arm runs on
rank 0 only. Rendezvous on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=ws, rank=rank)
    mx = bench._reduce_max(times[rank], ws, "cpu")
    val = bench._whole_job_value(4096, 300, ws, mx)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, mx, val))


def test_slowest_rank_sets_the_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [60.0, 75.5]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in got:
        assert mx == 75.5
        assert val == pytest.approx(4096 * 300 * 2 / 75.5e-3, rel=1e-15)


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._reduce_max(12.5, 1, "cpu") == 12.5
    assert bench._whole_job_value(10, 4, 1, 2.0) == pytest.approx(10 * 4 / 2e-3)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_runs_on_rank_zero_only(rank):
    """Launched as rank 1 of 2 the reference arm exits 0 without output; as rank 0 it prints one
    JSON line with impl = reference (a trimmed config-1 run of the oracle)."""
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    if rank == 1:
        assert lines == []
    else:
        d = json.loads(lines[-1])
        assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
