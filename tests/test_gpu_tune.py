"""Launch-shape autotuner (qex_tune, qex_tune_info): shapes change how sites
are spread over threads, never a per-site result."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import fieldgen as fg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C3 = -1.0 / 24.0


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02750_gb300 import build

    build.build()
    import paper_1612_02750_gb300 as mod

    mod.load()
    return mod


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 4, 10), (16, 16, 16, 16)])
@pytest.mark.parametrize("prec", ["f64", "f32r12h", "f32s16"])
@pytest.mark.parametrize("naik", [False, True])
def test_tuned_shapes_keep_dslash_bits(q, monkeypatch, dims, prec, naik):
    """The plain and normal-operator Dslash give bit-identical fields with the
    compiled default shapes and with the measured ones; the reported shapes
    are among the candidates."""
    import torch

    s = fg.rng_streams(31)
    u = fg.random_links(dims, "haar", s["links"])
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fat = fat64 if prec == "f64" else q.qex_convert_links(lat, "f64", fat64, prec)
    lng = None
    if naik:
        w = fg.random_links(dims, "gauss3", s["long_links"])
        lng = q.qex_pack_links(lat, q.qex_long_links_prec(prec), dev(w))
    inp = q.empty_field(lat, prec).normal_()
    monkeypatch.setenv("QEX_TUNE", "0")
    ref = q.qex_dslash(lat, prec, fat, lng, C3, 1, inp)
    ref_n = q.qex_normal_op(lat, prec, fat, lng, C3, 0.1, inp)
    assert q.qex_tune_info(lat, prec, naik)["source"] == "disabled"
    monkeypatch.delenv("QEX_TUNE")
    q.qex_tune(lat, prec, fat, lng)
    info = q.qex_tune_info(lat, prec, naik)
    assert info["source"] == "measured", info
    assert info["dslash_block"] in (64, 128, 256) and info["reduce_block"] in (64, 128, 256)
    assert 0 <= info["reduce_blocks_per_sm"] <= 16 and info["blas_blocks_per_sm"] in (2, 4, 8, 16)
    assert info["dslash_waves"] in (0, 2)
    got = q.qex_dslash(lat, prec, fat, lng, C3, 1, inp)
    got_n = q.qex_normal_op(lat, prec, fat, lng, C3, 0.1, inp)
    assert torch.equal(got, ref) and torch.equal(got_n, ref_n)


def test_forced_shapes_keep_cg_correct(q, oracle_mod):
    """A solve under measured shapes meets the oracle's true residual, and two
    solves under the same shapes give the same bits."""
    import torch

    dims = (8, 8, 8, 8)
    m = 0.1
    s = fg.rng_streams(32)
    u = fg.random_links(dims, "haar", s["links"])
    b = fg.gaussian_field(s["source"], dims)
    b[~fg.even_mask(dims)] = 0
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fat16 = q.qex_convert_links(lat, "f64", fat64, "f32r12h")
    q.qex_tune(lat, "f32r12h", fat16)
    q.qex_tune(lat, "f64", fat64)
    bh = q.qex_pack_field(lat, "f64", 0, dev(b))
    xs = []
    for _ in range(2):
        x = torch.zeros_like(bh)
        st, stats = q.qex_cg(lat, "f32r12h", fat64, None, fat16, None, 0.0, m, bh, x, tol=1e-10, delta=0.1)
        assert st == 0 and stats["converged"]
        xs.append(x)
    assert torch.equal(xs[0], xs[1])
    xf = q.qex_unpack_field(lat, "f64", 0, xs[0]).cpu().numpy()
    assert oracle_mod.true_residual(dims, u, b, xf, m) <= 1.05e-10


CHILD = r"""
import json, sys
import torch
import paper_1612_02750_gb300 as q
q.load()
lat = q.Lattice((8, 8, 8, 8))
fat = q.empty_links(lat, "f32").normal_()
inp = q.empty_field(lat, "f32").normal_()
q.qex_dslash(lat, "f32", fat, None, 0.0, 1, inp)
print(json.dumps(q.qex_tune_info(lat, "f32", False)))
"""


def test_tune_cache_file_round_trip(q, tmp_path):
    """The first process measures and appends a qex-tune-v1 line to the file
    named by QEX_TUNE_CACHE; the next one takes the same shapes from it."""
    path = tmp_path / "tune.txt"
    env = dict(os.environ, QEX_TUNE_CACHE=str(path), PYTHONPATH=ROOT)
    env.pop("QEX_TUNE", None)
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert runs[0]["source"] == "measured" and runs[1]["source"] == "cache"
    for k in ("dslash_block", "reduce_block", "reduce_blocks_per_sm", "dslash_waves"):
        assert runs[0][k] == runs[1][k]
    lines = [ln for ln in path.read_text().splitlines() if ln.startswith("qex-tune-v1 ")]
    assert len(lines) == 1 and "dims8x8x8x8" in lines[0] and "prec1 naik0" in lines[0]
    assert len(lines[0].split("|")[1].split()) == 5


CAPPED = r"""
import hashlib, json, sys
import torch
import paper_1612_02750_gb300 as q
q.load()
torch.manual_seed(5)
lat = q.Lattice((32, 32, 32, 32))
fat64 = q.empty_links(lat, "f64").normal_()
fat32 = q.qex_convert_links(lat, "f64", fat64, "f32")
fat16 = q.qex_convert_links(lat, "f64", fat64, "f32r12h")
inp = q.empty_field(lat, "f32r12h").normal_()
out = q.qex_dslash(lat, "f32r12h", fat16, None, 0.0, 1, inp)
b = q.empty_field(lat, "f64").normal_()
x = torch.zeros_like(b)
st, stats = q.qex_cg(lat, "f32", fat64, None, fat32, None, 0.0, 0.5, b, x, tol=1e-10, delta=0.1)
h = lambda t: hashlib.sha1(t.cpu().numpy().tobytes()).hexdigest()
print(json.dumps({"dslash": h(out), "x": h(x), "iters": stats["iters"], "status": st,
                  "waves": [q.qex_tune_info(lat, p)["dslash_waves"] for p in ("f32r12h", "f32")]}))
"""


def test_capped_grid_keeps_bits(q, tmp_path):
    """On 32^4 (a launch of ~3.4 resident waves) the plain Dslash and the
    mixed solve give the same bits with one thread per site and with the grid
    capped at two resident waves (sites taken grid-stride)."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    runs = []
    for waves in (0, 2):
        path = tmp_path / f"tune_{waves}.txt"
        path.write_text("".join(f"qex-tune-v1 sm{sms} dims32x32x32x32 ap1 prec{p} naik0 | 128 256 4 0 {w}\n"
                                for p, w in ((0, 0), (1, waves), (3, waves))))
        env = dict(os.environ, QEX_TUNE_CACHE=str(path), PYTHONPATH=ROOT)
        env.pop("QEX_TUNE", None)
        env.pop("QEX_CG_MODE", None)
        r = subprocess.run([sys.executable, "-c", CAPPED], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert runs[0]["waves"] == [0, 0] and runs[1]["waves"] == [2, 2]
    assert runs[0]["status"] == 0 and runs[0]["iters"] > 0
    for k in ("dslash", "x", "iters", "status"):
        assert runs[0][k] == runs[1][k], k


def test_tune_errors(q):
    lat = q.Lattice((2, 4, 4, 4))
    fat = q.empty_links(lat, "f64").zero_()
    with pytest.raises(q.QexError) as e:
        q.qex_tune(lat, "f64", None)
    assert e.value.status == 1
    with pytest.raises(q.QexError) as e:
        q.qex_tune(lat, "f64", fat, fat)  # Naik with an extent of 2
    assert e.value.status == 2
    assert q.qex_tune_info(lat, "f64")["source"] == "default"


def test_fma_rates_are_measured(q):
    """qex_fma_rates times FP64 and FP32 FMA chains on this GPU: both rates
    are positive and finite, and FP32 is the faster (on a GB300 FP64 is about
    1/60 of it)."""
    import math

    r = q.qex_fma_rates()
    assert all(math.isfinite(v) and v > 0 for v in r.values()), r
    assert r["fp32_gflops"] > 4 * r["fp64_gflops"], r
