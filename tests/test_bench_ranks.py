"""Host-side logic of bench.py's multi-process launch, on CPU with the gloo backend.

The build runs one replica of the solve per GPU (one process each, as torchrun starts them); the
replicas share only the barriers around the timed region and the max-over-ranks reduction of its
duration, and only rank 0 prints.  These tests run that logic with two gloo ranks on the host.
"""
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


_CHILD = r"""
import os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
world, rank, local, dist = bench._dist_init("gloo")
assert world == 2 and dist is not None
t = bench.max_over_ranks(1.0 + 2.0 * rank, dist, "cpu")
dist.barrier()
dist.destroy_process_group()
print(f"rank {rank} max {t}")
"""


def test_max_over_ranks_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r), BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", _CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("gloo rank did not finish")
        assert p.returncode == 0, err
        outs.append(out.strip())
    # both ranks see the slower rank's time (3.0)
    assert outs == ["rank 0 max 3.0", "rank 1 max 3.0"]


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
