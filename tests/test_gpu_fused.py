"""The mixed-precision solve with its inner iterations in one persistent
cooperative kernel (QEX_CG_MODE=fused) against the oracle and the graph
solve."""

import numpy as np
import pytest

import fieldgen as fg
from parity import assert_close

pytestmark = pytest.mark.gpu

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


def _setup(q, dims, naik, inner, seed):
    s = fg.rng_streams(seed)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    b = fg.gaussian_field(s["source"], dims)
    b[~fg.even_mask(dims)] = 0
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    lng64 = q.qex_pack_links(lat, "f64", dev(w)) if naik else None
    fati = q.qex_convert_links(lat, "f64", fat64, inner)
    lngi = q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec(inner)) if naik else None
    return lat, u, w, b, fat64, lng64, fati, lngi


def _solve(q, lat, inner, fat64, lng64, fati, lngi, c3, m, bh, **kw):
    import torch

    x = torch.zeros_like(bh)
    st, stats = q.qex_cg(lat, inner, fat64, lng64, fati, lngi, c3, m, bh, x, check=False, **kw)
    return st, stats, x


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 4, 10), (16, 8, 8, 8)])
@pytest.mark.parametrize("inner", ["f32", "f32r12h"])
@pytest.mark.parametrize("naik", [False, True])
def test_fused_solve_matches_oracle_and_graph(q, oracle_mod, monkeypatch, dims, inner, naik):
    """Same iterations (up to rounding-driven differences of a few) and a
    solution within 1e-7 of the graph solve's; the oracle's true residual of
    the fused solution is <= 1.05e-10."""
    m = 0.1
    c3 = C3 if naik else 0.0
    lat, u, w, b, fat64, lng64, fati, lngi = _setup(q, dims, naik, inner, 41)
    bh = q.qex_pack_field(lat, "f64", 0, dev(b))
    st_g, stats_g, x_g = _solve(q, lat, inner, fat64, lng64, fati, lngi, c3, m, bh, tol=1e-10, delta=0.1)
    monkeypatch.setenv("QEX_CG_MODE", "fused")
    st_f, stats_f, x_f = _solve(q, lat, inner, fat64, lng64, fati, lngi, c3, m, bh, tol=1e-10, delta=0.1)
    assert st_g == 0 and st_f == 0 and stats_f["converged"], stats_f
    assert abs(stats_f["iters"] - stats_g["iters"]) <= max(3, stats_g["iters"] // 50)
    xf = q.qex_unpack_field(lat, "f64", 0, x_f).cpu().numpy()
    xg = q.qex_unpack_field(lat, "f64", 0, x_g).cpu().numpy()
    ev = fg.even_mask(dims)
    assert_close(xf[ev], xg[ev], 1e-7, "fused against graph solve")
    assert oracle_mod.true_residual(dims, u, b, xf, m, w, c3) <= 1.05e-10


def test_fused_solve_edges(q, monkeypatch):
    """Iteration cap (status 5 with exactly maxiter iterations), a zero source
    (x = 0), and bit-identical repeated solves."""
    import torch

    dims = (8, 4, 6, 8)
    lat, u, w, b, fat64, lng64, fati, lngi = _setup(q, dims, False, "f32r12h", 42)
    bh = q.qex_pack_field(lat, "f64", 0, dev(b))
    monkeypatch.setenv("QEX_CG_MODE", "fused")
    st, stats, _ = _solve(q, lat, "f32r12h", fat64, None, fati, None, 0.0, 0.05, bh, tol=1e-12, maxiter=9,
                          delta=0.1)
    assert st == 5 and stats["iters"] == 9 and not stats["converged"]
    st, stats, x = _solve(q, lat, "f32r12h", fat64, None, fati, None, 0.0, 0.05, torch.zeros_like(bh), tol=1e-10)
    assert st == 0 and stats["converged"] and not x.any()
    runs = [_solve(q, lat, "f32r12h", fat64, None, fati, None, 0.0, 0.05, bh, tol=1e-10, delta=0.1)[2]
            for _ in range(2)]
    assert torch.equal(runs[0], runs[1])


def test_fused_barrier_limit_runs_out_and_the_lattice_recovers(q, oracle_mod, monkeypatch):
    """The persistent kernel's grid barriers give up after a limit of clock64
    cycles.  With the limit set to 100 cycles (a barrier of 32 blocks takes
    longer) some wait runs out: qex_cg returns QEX_ERR_TIMEOUT (6), every
    block has left the kernel, and the next solve on the same lattice, with
    the default limit of about a second, converges to the oracle's true
    residual."""
    import re

    dims = (8, 8, 8, 16)  # Vh = 4096: 32 blocks of 128 threads
    m = 0.1
    lat, u, w, b, fat64, lng64, fati, lngi = _setup(q, dims, False, "f32r12h", 81)
    bh = q.qex_pack_field(lat, "f64", 0, dev(b))
    monkeypatch.setenv("QEX_CG_MODE", "fused")
    monkeypatch.setenv("QEX_BARRIER_TIMEOUT_CYCLES", "100")
    st, stats, x = _solve(q, lat, "f32r12h", fat64, lng64, fati, lngi, 0.0, m, bh, tol=1e-10, delta=0.1)
    msg = q.qex_last_error()
    assert st == 6 and not stats["converged"], (st, stats, msg)
    left = re.search(r"\((\d+) of (\d+) blocks left", msg)
    assert left and left.group(1) == left.group(2) and int(left.group(2)) > 1, msg
    monkeypatch.delenv("QEX_BARRIER_TIMEOUT_CYCLES")
    st, stats, x = _solve(q, lat, "f32r12h", fat64, lng64, fati, lngi, 0.0, m, bh, tol=1e-10, delta=0.1)
    assert st == 0 and stats["converged"], stats
    xf = q.qex_unpack_field(lat, "f64", 0, x).cpu().numpy()
    assert oracle_mod.true_residual(dims, u, b, xf, m) <= 1.05e-10
