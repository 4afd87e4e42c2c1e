"""Host logic of the benchmark on CPU: rank combination and the partition of
independent bodies over gloo ranks (world size 2), roofline bookkeeping and
the JSON contract of the reference arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
r = dist.get_rank()
t, u = bench.combine_over_ranks(1.0 + r, 10.0 * (r + 1))
assert (t, u) == (2.0, 30.0), (t, u)
bench.barrier()
dist.destroy_process_group()
print("ok", r)
'''


def test_combine_over_ranks_gloo_world2(tmp_path):
    w = tmp_path / "w.py"
    w.write_text(WORKER % ROOT)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT="29517", WORLD_SIZE="2")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, str(w)], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    assert "ok 0" in outs[0] and "ok 1" in outs[1]


def test_combine_identity_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(3.0, 7.0) == (3.0, 7.0)


def test_profile_traffic_requires_matching_source(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "s.md").write_text("traffic_bytes_per_launch: 1000\nunits_per_launch: 10\n"
                               "kernel_source_sha256_16: %s\n" % bench.source_digest(str(src)))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic(str(src), "s.md") == (1000.0, 10.0)
    src.write_text("kernel v2")
    assert bench.profile_traffic(str(src), "s.md") is None


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""


PARTITION_WORKER = r'''
import os, sys
sys.path.insert(0, %r)
import torch, torch.distributed as dist
import bench, sg_inputs as si
dist.init_process_group("gloo")
r, ws = dist.get_rank(), dist.get_world_size()
bodies = si.random_bodies(256, seed=1)
w = [t for _, _, t in bodies]
mine = bench.partition_bodies(w, ws)[r]
# every rank derives the same partition on its own; gather it to check
got = [None] * ws
dist.all_gather_object(got, mine)
flat = sorted(i for p in got for i in p)
assert flat == list(range(256)), "every body exactly once"
loads = [sum(w[i] for i in p) for p in got]
assert max(loads) <= sum(w) / ws + max(w) + 1e-9, loads
assert max(loads) / (sum(w) / ws) < 1.05, loads
# a rank's relaxation particles are its bodies' particles of the whole run
x, y, z, off = si.relax_particles(bodies[:12], 120000, seed=5, subset=[b for b in mine if b < 12])
xa, ya, za, offa = si.relax_particles(bodies[:12], 120000, seed=5)
k = 0
for b in [b for b in mine if b < 12]:
    n = offa[b + 1] - offa[b]
    assert off[k + 1] - off[k] == n
    assert (x[off[k]:off[k + 1]] == xa[offa[b]:offa[b + 1]]).all()
    k += 1
t, u = bench.combine_over_ranks(1.0 + r, float(len(mine)))
assert u == 256.0
dist.destroy_process_group()
print("ok", r)
'''


def test_partition_bodies_gloo_world2(tmp_path):
    w = tmp_path / "p.py"
    w.write_text(PARTITION_WORKER % ROOT)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT="29519", WORLD_SIZE="2")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, str(w)], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=180)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    assert "ok 0" in outs[0] and "ok 1" in outs[1]


def test_partition_bodies_single_and_many_ranks():
    sys.path.insert(0, ROOT)
    import bench
    w = [5.0, 1.0, 3.0, 3.0, 2.0]
    assert bench.partition_bodies(w, 1) == [[0, 1, 2, 3, 4]]
    # heaviest first: body 0 (5) -> r0, 2 (3) -> r1, 3 (3) -> r2, 4 (2) -> r1 (loads 3 = 3: the lower rank),
    # 1 (1) -> r2 (load 3 < 5)
    assert bench.partition_bodies(w, 3) == [[0], [2, 4], [1, 3]]
    parts = bench.partition_bodies([1.0] * 10, 4)
    assert sorted(len(p) for p in parts) == [2, 2, 3, 3]
