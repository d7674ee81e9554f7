"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would
launch them (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_* in the environment).

The solver shards as replicas only: each rank solves its own seeded system
and ranks meet only at the barriers and the max/sum of the timings, so these
helpers are the whole of the multi-GPU logic."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import bench
rank, world, local = bench.dist_setup(2)
assert world == 2 and local == rank
bench.barrier(world)
t = 10.0 + rank                      # per-rank "elapsed ms"
out = {{"rank": rank,
        "max": bench.max_over_ranks(t, world),
        "sum": bench.sum_over_ranks(1.0 + rank, world)}}
# the reference arm: rank 0 alone runs and prints; other ranks return at once
class A: steps = 1; warmup = 3; gpus = 2
if rank == 1:
    t0 = time.perf_counter()
    bench.reference_arm(A, rank, world)
    out["reference_rank1_s"] = time.perf_counter() - t0
bench.barrier(world)
print(json.dumps(out), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_timings_and_only_rank0_reports():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 11.0            # max over ranks of 10 + rank
        assert o["sum"] == 3.0             # 1 + 2
    r1 = [o for o in outs if o["rank"] == 1][0]
    assert r1["reference_rank1_s"] < 1.0   # no oracle work on rank 1


def test_replica_seeds_differ_per_rank():
    """Each rank's replica uses its own seed (host_sequence(seed_offset=rank))."""
    sys.path.insert(0, ROOT)
    import dataclasses
    import blackoil_synth as bs
    g = dataclasses.replace(bs.CONFIGS["20x20x5"])
    a = bs.jacobian(g)
    b = bs.jacobian(dataclasses.replace(g, seed=g.seed + 1))
    assert a.nb == b.nb and (a.rowptr == b.rowptr).all()
    assert not (a.val == b.val).all()
