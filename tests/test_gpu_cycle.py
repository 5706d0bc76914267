"""Bounded inner cycles of the mixed-precision CG.

A reliable update normally waits until the iterated residual has dropped by
delta since the last one.  At small mass that can take thousands of inner
iterations, and over such a cycle the recursion residual of the inner
precision drifts away from b - A x: the iteration goes on reducing a
residual that is no longer the true one and the solve stalls.  A mixed solve
therefore also makes a reliable update after a fixed number of inner
iterations (100 with 16-bit links, 500 with FP32 ones; QEX_RU_CYCLE=<n>
overrides, 0 turns the bound off).

The hard case here: 8^4, Haar links, m = 0.005, 16-bit two-row inner links,
delta = 0.01.  Without the bound it has not converged after 30,000
iterations; with it, it converges in about 11,000.  Every solve is checked
against the oracle's true residual of the returned x.
"""

import numpy as np
import pytest

import fieldgen as fg

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
MASS = 0.005
DELTA = 0.01
INNER = "f32r12h"


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


def _links(q, dims, seed):
    u, _, b = fg.make_inputs(dims, "haar", False, seed)
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fat16 = q.qex_convert_links(lat, "f64", fat64, INNER)
    return lat, u, b, fat64, fat16


def _solve(q, lat, fat64, fat16, b, maxiter=60000):
    import torch

    b64 = q.qex_pack_field(lat, "f64", 0, dev(b))
    x64 = torch.zeros_like(b64)
    st, stats = q.qex_cg(lat, INNER, fat64, None, fat16, None, 0.0, MASS, b64, x64, tol=1e-10, maxiter=maxiter,
                         delta=DELTA, check=False)
    return st, stats, q.qex_unpack_field(lat, "f64", 0, x64).cpu().numpy()


@pytest.mark.parametrize("mode", ["fused", "graph", "host"])
def test_bounded_cycle_converges_where_unbounded_stalls(q, oracle_mod, monkeypatch, mode):
    monkeypatch.setenv("QEX_CG_MODE", mode)
    lat, u, b, fat64, fat16 = _links(q, DIMS, 4)
    monkeypatch.delenv("QEX_RU_CYCLE", raising=False)
    st, stats, x = _solve(q, lat, fat64, fat16, b)
    assert st == 0 and stats["converged"], stats
    assert stats["iters"] < 20000, stats
    # no cycle is longer than 100 iterations
    assert stats["reliable_updates"] >= stats["iters"] // 100, stats
    tr = oracle_mod.true_residual(DIMS, u, b, x, MASS)
    assert tr <= 1.05e-10 and stats["true_rel_resid"] == pytest.approx(tr, rel=1e-3, abs=1e-13)

    # the override is read per solve: a 50-iteration bound gives at least twice as many updates
    monkeypatch.setenv("QEX_RU_CYCLE", "50")
    st50, stats50, x50 = _solve(q, lat, fat64, fat16, b)
    assert st50 == 0 and stats50["reliable_updates"] >= stats50["iters"] // 50, stats50
    assert oracle_mod.true_residual(DIMS, u, b, x50, MASS) <= 1.05e-10

    # without the bound the same solve stalls far above tol
    monkeypatch.setenv("QEX_RU_CYCLE", "0")
    st0, stats0, x0 = _solve(q, lat, fat64, fat16, b, maxiter=30000)
    assert st0 == 5 and not stats0["converged"] and stats0["iters"] == 30000, stats0
    assert stats0["reliable_updates"] < 30000 // 100
    assert oracle_mod.true_residual(DIMS, u, b, x0, MASS) > 1e-8


def test_graph_and_host_agree_bitwise_with_bounded_cycles(q, monkeypatch):
    """The bound is taken in the same kernel in both loops: identical bits."""
    lat, u, b, fat64, fat16 = _links(q, DIMS, 4)
    monkeypatch.setenv("QEX_CG_MODE", "graph")
    st_g, stats_g, x_g = _solve(q, lat, fat64, fat16, b)
    monkeypatch.setenv("QEX_CG_MODE", "host")
    st_h, stats_h, x_h = _solve(q, lat, fat64, fat16, b)
    assert st_g == st_h == 0
    assert (stats_g["iters"], stats_g["reliable_updates"]) == (stats_h["iters"], stats_h["reliable_updates"])
    assert np.array_equal(x_g, x_h)


def test_bounded_cycle_multi_rhs(q, oracle_mod):
    import torch

    lat, u, _, fat64, fat16 = _links(q, DIMS, 4)
    srcs = [fg.make_inputs(DIMS, "haar", False, 300 + k)[2] for k in range(3)]
    B = torch.cat([q.qex_pack_field(lat, "f64", 0, dev(s)) for s in srcs])
    X = torch.zeros_like(B)
    st, stats = q.qex_cg_mrhs(lat, INNER, fat64, None, fat16, None, 0.0, MASS, 3, B, X, tol=1e-10, maxiter=60000,
                              delta=DELTA, check=False)
    assert st == 0, stats
    n = B.numel() // 3
    for k, s in enumerate(stats):
        assert s["converged"] and s["iters"] < 20000, s
        assert s["reliable_updates"] >= max(t["iters"] for t in stats) // 100, s
        x = q.qex_unpack_field(lat, "f64", 0, X[k * n:(k + 1) * n]).cpu().numpy()
        assert oracle_mod.true_residual(DIMS, u, srcs[k], x, MASS) <= 1.05e-10


def test_bounded_cycle_batch(q, oracle_mod):
    import torch

    items, refs = [], []
    for k, dims in enumerate([DIMS, (8, 8, 4, 12), (6, 6, 6, 8)]):
        lat, u, b, fat64, fat16 = _links(q, dims, 40 + k)
        b64 = q.qex_pack_field(lat, "f64", 0, dev(b))
        items.append({"lat": lat, "fat64": fat64, "fat32": fat16, "mass": MASS, "b64": b64,
                      "x64": torch.zeros_like(b64)})
        refs.append((dims, u, b))
    st, stats = q.qex_cg_batch(items, INNER, tol=1e-10, maxiter=60000, delta=DELTA, check=False)
    assert st == 0, stats
    for it, s, (dims, u, b) in zip(items, stats, refs):
        assert s["converged"] and s["iters"] < 20000, s
        assert s["reliable_updates"] >= s["iters"] // 100, s
        x = q.qex_unpack_field(it["lat"], "f64", 0, it["x64"]).cpu().numpy()
        tr = oracle_mod.true_residual(dims, u, b, x, MASS)
        assert tr <= 1.05e-10 and s["true_rel_resid"] == pytest.approx(tr, rel=1e-3, abs=1e-13)
