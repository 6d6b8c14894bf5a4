"""The benchmark's multi-rank path on the CPU: `--gpus N` starts N ranks (or fails clearly when N
GPUs are not visible), and inside the timed loop the ranks exchange their best candidates after
every step (gloo, world size 2, with a stand-in problem whose best is known per step)."""
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_torchrun_command_line():
    sys.path.insert(0, ROOT)
    import bench
    argv = bench.torchrun_argv(["--gpus", "4", "--steps", "5"], 4, 29555)
    assert argv[:3] == [sys.executable, "-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in argv and "--nnodes=1" in argv
    assert "--master-addr=127.0.0.1" in argv and "--master-port=29555" in argv
    assert argv[-5:] == [os.path.join(ROOT, "bench.py"), "--gpus", "4", "--steps", "5"]


def test_gpus_beyond_the_visible_devices_fail_clearly():
    import torch
    want = max(2, torch.cuda.device_count() + 1)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", str(want), "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300,
                       env={k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")})
    assert r.returncode == 2, (r.returncode, r.stderr[-2000:])
    assert f"needs {want} visible GPUs" in r.stderr


def test_world_size_must_match_gpus():
    env = dict(os.environ, WORLD_SIZE="3", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 2 and "WORLD_SIZE=3" in r.stderr


# per rank, per step: (F, t, restart) of the rank's best so far
BESTS = {0: [(-5, 50, 3), (-7, 100, 1), (-7, 100, 1)],
         1: [(-6, 50, 0), (-6, 50, 0), (-9, 150, 2)]}
EXPECT = [(-6, 50, 1, 0), (-7, 100, 0, 1), (-9, 150, 1, 2)]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        done = []

        def step():
            done.append(len(done))

        def best():
            F, t, r = BESTS[rank][len(done) - 1]
            return np.full(5, rank, np.uint8), F, t, r

        trace = bench.step_loop(3, step, best)
        out.put((rank, len(done), trace))
    finally:
        dist.destroy_process_group()


def test_step_loop_exchanges_the_best_after_every_step():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, world, port, out)) for k in range(world)]
    for p in procs:
        p.start()
    got = dict((r, (n, tr)) for r, n, tr in (out.get(timeout=180) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        n, trace = got[rank]
        assert n == 3
        assert [tuple(t) for t in trace] == EXPECT
