"""Host-side logic of bench.py's N > 1 path, as world_size-2 gloo ranks on CPU.

Frames are independent, so ranks share no data: each decodes its own seeded
batch and the only cross-rank step is the max over ranks of the timed region
(and of the end-to-end time).  The reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from workloads import ebch
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [812.5, 640.25][rank]
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        code = ebch("ebch_16_11")
        _, _, lch = bench.make_inputs(code, 9, bench.rank_seed(rank), 1)
        q.put((rank, slowest, float(np.abs(lch).sum()), bench.job_rate(world, 9, code.k * code.k, 3, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_decode_their_own_frames():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert [r[1] for r in res] == [812.5, 812.5]
    assert res[0][2] != res[1][2]  # distinct batches per rank
    # whole job: both ranks' frames over the slowest rank's time
    assert res[0][3] == res[1][3] == pytest.approx(2 * 9 * 121 * 3 / 0.8125)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.rank_seed(0) != bench.rank_seed(1)


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "1", "--ref-frames", "7"], capture_output=True, text=True, env=env,
                          timeout=600, cwd=ROOT)


def test_reference_arm_runs_on_rank_zero_only():
    r1 = _run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _run_reference({"RANK": "0", "WORLD_SIZE": "2"})
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "bits/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
