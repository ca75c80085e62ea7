"""bench.py's multi-GPU mode runs independent replicas (the sweep of one instance is not
sharded): every rank times its own replica and the job takes as long as the slowest rank.  This
checks that bookkeeping with two gloo ranks on the CPU, and that the reference arm runs on rank
0 only."""
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


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
value, max_ms = bench.job_rate(local_ms, steps=10, world=world)
print(f"rank={{rank}} value={{value:.6f}} max_ms={{max_ms}}", flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _launch(code, world, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_job_rate_takes_the_slowest_replica():
    outs = _launch(WORKER.format(root=ROOT), 2)
    for out in outs:
        assert "max_ms=200.0" in out
        # 2 replicas x 10 sweeps in 0.2 s
        assert "value=100.000000" in out


def test_reference_arm_runs_on_rank_zero_only():
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.argv = ['bench.py', '--impl', "
            "'reference', '--steps', '1', '--warmup', '0', '--workload', 'tfim1d_L1_N16', "
            "'--gpus', '2']; import bench; bench.main()")
    outs = _launch(code, 2)
    assert '"impl": "reference"' in outs[0]
    assert outs[1].strip() == ""


@pytest.mark.parametrize("workload", ["sf_N20_L2", "lrtfim_N128_L1"])
def test_reference_arm_of_the_general_workloads(workload):
    # the oracle's Algorithm 5 (spin terms, or the fermionic relaxation) as the reference arm
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.argv = ['bench.py', '--impl', "
            f"'reference', '--steps', '1', '--warmup', '0', '--workload', {workload!r}]; "
            "import bench; bench.main()")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         timeout=240)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
