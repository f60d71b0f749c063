"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

With N > 1 ranks every rank runs its own replica; the timed region is closed
by a barrier, the step time is the maximum over the ranks and the work is the
sum over them, and only rank 0 prints. The reference arm runs on rank 0 alone
and the other ranks leave without work. Both are checked here with world size
2 and the gloo backend, without a GPU.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REDUCE = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_init()
bench.barrier(world)
out = dict(world=world, rank=rank, local=local,
           mx=bench.max_over_ranks(world, 10.0 * (rank + 1)),
           sm=bench.sum_over_ranks(world, 3.0 + rank))
bench.barrier(world)
import torch.distributed as dist
dist.destroy_process_group()
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(argv, world=2, timeout=240):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen(argv, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    try:
        for p in procs:
            o, e = p.communicate(timeout=timeout)
            assert p.returncode == 0, e[-2000:]
            outs.append(o)
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


def test_two_gloo_ranks_reduce_max_and_sum():
    pytest.importorskip("torch")
    outs = _launch([sys.executable, "-c", REDUCE.format(root=ROOT)])
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1]
    for d in res:
        assert d["world"] == 2
        assert d["mx"] == 20.0          # max over ranks of 10, 20
        assert d["sm"] == 7.0           # 3 + 4


def test_reference_arm_prints_on_rank_zero_only():
    pytest.importorskip("torch")
    outs = _launch([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--scale", "0.001",
                    "--steps", "1", "--warmup", "0"])
    lines = [[l for l in o.splitlines() if l.startswith("{")] for o in outs]
    assert len(lines[1]) == 0, "rank 1 must not print"
    assert len(lines[0]) == 1
    d = json.loads(lines[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
