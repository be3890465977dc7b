"""The N > 1 path of bench.py on CPU (gloo, world size 2): independent replicas, rank r solving the
workload of seed + r, and the step time taken as the maximum over ranks."""
import json
import os
import socket
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_replicas_reduce_to_the_max_and_solve_different_images():
    tmp = tempfile.mkdtemp(prefix="replicas_")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "replica_worker.py"), tmp]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=240, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    recs = [json.load(open(os.path.join(tmp, f"rank_{r}.json"))) for r in range(2)]
    assert [r["rank"] for r in recs] == [0, 1]
    assert all(r["world"] == 2 and r["max"] == 20.0 for r in recs)
    assert recs[0]["void"] != recs[1]["void"] or recs[0]["mu"] != recs[1]["mu"]
