"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs its own replica with its own seed, and the job's figures are the
slowest rank's time and the sum of the ranks' units."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench, workload
    rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mx, sm = bench.rank_reducers(dist, "cpu")
    ms = 10.0 + 5.0 * rank            # this rank's timed region
    units = 1000.0 * (rank + 1)       # this rank's particle pushes
    class A:  # the bench's arguments that make_workload reads
        ppc = 1
        nx = "8,8,8"
        smooth = 0
    g, sps, _ = bench.make_workload(A, rank)
    x, u = workload.load_particles(g, sps[0], [0, 1, 2])
    out = {{"max": mx(ms), "sum": sm(units), "seed": sps[0].seed, "x": x.tolist(), "u": u.tolist()}}
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps(out))
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_like_the_bench():
    import json
    port = _free_port()
    code = WORKER.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 15.0           # the slowest rank's time
        assert o["sum"] == 3000.0         # units of both replicas
    assert outs[0]["seed"] != outs[1]["seed"]
    assert outs[0]["x"] == outs[1]["x"]   # the same lattice ...
    assert outs[0]["u"] != outs[1]["u"]   # ... with each replica's own thermal draw
