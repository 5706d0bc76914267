"""Host-side logic of bench.py, on CPU: max-over-ranks timing with two gloo
ranks, clock-sample parsing, the stale-traffic guard and the reference arm's
rank handling."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
d = bench.Dist(want_gpu=False)
v = d.max(float(10 + 5 * d.rank))
d.barrier()
print(json.dumps({{"rank": d.rank, "world": d.world, "max": v}}))
d.close()
"""


def test_dist_max_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["world"] == 2 and o["max"] == 15.0 for o in outs)


def test_clock_parsing(tmp_path):
    sys.path.insert(0, ROOT)
    import bench

    c = bench.Clocks(0)
    f = tmp_path / "c.csv"
    f.write_text("1965, 2070, 800.1, Not Active, Not Active, Not Active, Active\n"
                 "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active\n"
                 "1980, 2070, 850.0, Not Active, Not Active, Not Active, Not Active\n")

    class P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class F:
        name = str(f)

        def flush(self):
            pass

    c.proc, c.file = P(), F()
    out = c.stop()
    assert out["sm_mhz"] == 1980 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_clock_sampler_waits_for_its_first_sample(tmp_path, monkeypatch):
    """Clocks.start() returns only once the sampler has written a sample (its
    start-up must not overlap a timed region), and at most after about 3 s
    when none comes; stop() parses what it wrote.  A fake nvidia-smi on PATH
    stands in for the real one: it sleeps 0.4 s, then writes a sample every
    0.1 s."""
    sys.path.insert(0, ROOT)
    import time

    import bench

    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nsleep 0.4\nwhile true; do\n"
                    "  echo '2070, 2070, 900.0, Not Active, Not Active, Not Active, Not Active'\n"
                    "  sleep 0.1\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.Clocks(0)
    t0 = time.time()
    c.start()
    waited = time.time() - t0
    assert os.path.getsize(c.file.name) > 0 and 0.3 < waited < 3.5, waited
    time.sleep(0.3)
    out = c.stop()
    assert out["sm_mhz"] == 2070 and out["reasons"] == [] and out["samples"] >= 2

    # a sampler that never writes: start() gives up after about 3 s
    fake.write_text("#!/bin/sh\nsleep 30\n")
    c = bench.Clocks(0)
    t0 = time.time()
    c.start()
    assert 2.5 < time.time() - t0 < 5.0
    assert c.stop()["samples"] == 0

    # no nvidia-smi at all
    monkeypatch.setenv("PATH", str(tmp_path / "none"))
    c = bench.Clocks(0)
    c.start()
    assert c.proc is None and c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_guard_uses_source_hash():
    sys.path.insert(0, ROOT)
    import bench

    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    rec = json.load(open(path))["dslash_f32_nn_32^4"]
    got = bench.ncu_traffic("dslash_f32_nn_32^4")
    if rec["source_hash"] == bench.kernel_source_hash():
        assert got == rec["dram_bytes_per_launch"]
    else:
        assert got is None
    assert bench.ncu_traffic("no such kernel") is None


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""
