"""Float-float reliable updates (ru_ff.cu) and qex_true_residual.

The intermediate reliable updates of a mixed solve compute r = b - A x with
every real carried as an unevaluated sum of two FP32 numbers; the first
update and the one that may end the solve stay FP64.  These tests check
* qex_true_residual in both arithmetics against the oracle's FP64 true
  residual, with and without the Naik term, for a random x (residual of
  order 1) and for a near solution (residual 1e-10, where the float-float
  error has to stay far below the residual itself);
* that the float-float result does not depend on the scale of b and x (they
  are carried times 2^ff_k, a power of two taken from ||b||): b, x and
  2^+-90 b, 2^+-90 x give the same bits;
* exact zeros (identity links, a zero x);
* mixed solves with float-float updates (QEX_RU_FF=1; FP64 updates are the
  default) against the same solves with FP64 updates: the same iteration
  counts up to rounding, FP64 stopping test, the oracle's true residual of
  the returned x;
* that the updates give way to FP64 once their error (about 1e-13 of
  ||x|| + ||b||) would reach 1e-3 of the residual: at small mass on Haar
  links ||x|| is about 1400 ||b||, and with an update every 50 iterations
  float-float updates to the end stalled the solve near 5e-8.
"""

import numpy as np
import pytest

import fieldgen as fg

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


def _setup(q, dims, naik, seed, fat="haar"):
    s = fg.rng_streams(seed)
    u = fg.random_links(dims, fat, s["links"], 0.3)
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    ev = fg.even_mask(dims)
    b = fg.gaussian_field(s["source"], dims)
    b[~ev] = 0
    x = fg.gaussian_field(s["chi"], dims)
    x[~ev] = 0
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    lng64 = q.qex_pack_links(lat, "f64", dev(w)) if naik else None
    return lat, u, w, b, x, fat64, lng64


@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (6, 4, 8, 8)])
def test_true_residual_both_arithmetics_match_oracle(q, oracle_mod, naik, dims):
    mass = 0.1
    c3 = C3 if naik else 0.0
    lat, u, w, b, x, fat64, lng64 = _setup(q, dims, naik, 7)
    ref = oracle_mod.true_residual(dims, u, b, x, mass, w, c3)
    b64, x64 = q.qex_pack_field(lat, "f64", 0, dev(b)), q.qex_pack_field(lat, "f64", 0, dev(x))
    r64 = q.qex_true_residual(lat, fat64, lng64, c3, mass, b64, x64, "f64")
    rff = q.qex_true_residual(lat, fat64, lng64, c3, mass, b64, x64, "ff")
    assert ref > 0.5
    assert abs(r64 - ref) <= 1e-13 * ref, (r64, ref)
    # the norm of the FP32-rounded residual: 2^-24 relative a real
    assert abs(rff - ref) <= 1e-7 * ref, (rff, ref)


@pytest.mark.parametrize("naik", [False, True])
def test_true_residual_near_solution(q, oracle_mod, naik):
    """x from an FP64 solve to 1e-10.  An error e of the float-float residual
    vector, uncorrelated with r, moves the norm by about ||e||^2 / (2 ||r||):
    agreement to 1% of a 1e-10 residual bounds ||e|| by about 1.4e-11 ||b||
    (an FP32 residual would be off by about 1e-7 ||b||)."""
    import torch

    dims, mass = (8, 8, 4, 8), 0.05
    c3 = C3 if naik else 0.0
    lat, u, w, b, _, fat64, lng64 = _setup(q, dims, naik, 11)
    b64 = q.qex_pack_field(lat, "f64", 0, dev(b))
    x64 = torch.zeros_like(b64)
    st, stats = q.qex_cg(lat, "f64", fat64, lng64, None, None, c3, mass, b64, x64, tol=1e-10, maxiter=20000)
    assert st == 0
    x = q.qex_unpack_field(lat, "f64", 0, x64).cpu().numpy()
    ref = oracle_mod.true_residual(dims, u, b, x, mass, w, c3)
    assert 1e-12 < ref <= 1.05e-10
    rff = q.qex_true_residual(lat, fat64, lng64, c3, mass, b64, x64, "ff")
    r64 = q.qex_true_residual(lat, fat64, lng64, c3, mass, b64, x64, "f64")
    # FP64 in another summation order already moves a 1e-10 residual by about 1e-6 of itself
    assert abs(r64 - ref) <= 1e-4 * ref and abs(rff - ref) <= 1e-2 * ref, (r64, rff, ref)


@pytest.mark.parametrize("scale", [2.0 ** -90, 2.0 ** 90, 2.0 ** -20])
def test_float_float_residual_is_scale_free(q, scale):
    dims, mass = (8, 4, 6, 8), 0.1
    lat, u, w, b, x, fat64, lng64 = _setup(q, dims, True, 13)
    b64, x64 = q.qex_pack_field(lat, "f64", 0, dev(b)), q.qex_pack_field(lat, "f64", 0, dev(x))
    base = q.qex_true_residual(lat, fat64, lng64, C3, mass, b64, x64, "ff")
    got = q.qex_true_residual(lat, fat64, lng64, C3, mass, b64 * scale, x64 * scale, "ff")
    assert got == base


def test_float_float_residual_exact_zeros(q, oracle_mod):
    """Identity links (off-diagonal entries exactly 0) and x = 0 (r = b)."""
    import torch

    dims, mass = (6, 4, 4, 8), 0.2
    lat, u, w, b, x, _, _ = _setup(q, dims, False, 17)
    one = np.zeros_like(u)
    one[..., 0, 0] = one[..., 1, 1] = one[..., 2, 2] = 1.0
    fat64 = q.qex_pack_links(lat, "f64", dev(one))
    b64, x64 = q.qex_pack_field(lat, "f64", 0, dev(b)), q.qex_pack_field(lat, "f64", 0, dev(x))
    ref = oracle_mod.true_residual(dims, one, b, x, mass)
    rff = q.qex_true_residual(lat, fat64, None, 0.0, mass, b64, x64, "ff")
    assert abs(rff - ref) <= 1e-7 * ref, (rff, ref)
    z = q.qex_true_residual(lat, fat64, None, 0.0, mass, b64, torch.zeros_like(x64), "ff")
    assert abs(z - 1.0) <= 1e-7


def _solve(q, lat, fat64, lng64, fat_i, lng_i, c3, mass, b64, inner, delta=0.01):
    import torch

    x64 = torch.zeros_like(b64)
    st, stats = q.qex_cg(lat, inner, fat64, lng64, fat_i, lng_i, c3, mass, b64, x64, tol=1e-10, maxiter=60000,
                         delta=delta, check=False)
    return st, stats, q.qex_unpack_field(lat, "f64", 0, x64).cpu().numpy()


@pytest.mark.parametrize("mode", ["graph", "host", "fused"])
@pytest.mark.parametrize("naik", [False, True])
def test_solves_with_float_float_updates(q, oracle_mod, monkeypatch, mode, naik):
    dims, mass, inner = (8, 8, 8, 8), 0.02, "f32r12h"
    c3 = C3 if naik else 0.0
    lat, u, w, b, _, fat64, lng64 = _setup(q, dims, naik, 19, fat="exp")
    fat_i = q.qex_convert_links(lat, "f64", fat64, inner)
    lng_i = q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec(inner)) if naik else None
    b64 = q.qex_pack_field(lat, "f64", 0, dev(b))
    monkeypatch.setenv("QEX_CG_MODE", mode)
    monkeypatch.delenv("QEX_RU_FF", raising=False)  # default: FP64 updates
    st0, s0, x0 = _solve(q, lat, fat64, lng64, fat_i, lng_i, c3, mass, b64, inner)
    monkeypatch.setenv("QEX_RU_FF", "1")
    st1, s1, x1 = _solve(q, lat, fat64, lng64, fat_i, lng_i, c3, mass, b64, inner)
    assert st0 == st1 == 0 and s0["converged"] and s1["converged"]
    assert s0["ff_updates"] == 0 and 1 <= s1["ff_updates"] < s1["reliable_updates"], (s0, s1)
    assert abs(s1["iters"] - s0["iters"]) <= max(2, s0["iters"] // 50), (s0, s1)
    for x, s in ((x0, s0), (x1, s1)):
        tr = oracle_mod.true_residual(dims, u, b, x, mass, w, c3)
        assert tr <= 1.05e-10 and s["true_rel_resid"] == pytest.approx(tr, rel=1e-3, abs=1e-13)


def test_graph_and_host_agree_bitwise_with_float_float_updates(q, monkeypatch):
    dims, mass, inner = (8, 4, 6, 8), 0.05, "f32r12"
    lat, u, w, b, _, fat64, lng64 = _setup(q, dims, False, 23)
    fat_i = q.qex_convert_links(lat, "f64", fat64, inner)
    b64 = q.qex_pack_field(lat, "f64", 0, dev(b))
    monkeypatch.setenv("QEX_RU_FF", "1")
    monkeypatch.setenv("QEX_CG_MODE", "graph")
    st_g, s_g, x_g = _solve(q, lat, fat64, None, fat_i, None, 0.0, mass, b64, inner, delta=0.05)
    monkeypatch.setenv("QEX_CG_MODE", "host")
    st_h, s_h, x_h = _solve(q, lat, fat64, None, fat_i, None, 0.0, mass, b64, inner, delta=0.05)
    assert st_g == st_h == 0 and s_g["reliable_updates"] >= 3 and s_g["ff_updates"] >= 1
    assert (s_g["iters"], s_g["reliable_updates"]) == (s_h["iters"], s_h["reliable_updates"])
    assert np.array_equal(x_g, x_h)


def test_float_float_updates_give_way_at_small_mass(q, oracle_mod, monkeypatch):
    dims, mass, inner = (8, 8, 8, 8), 0.005, "f32r12h"
    u, _, b = fg.make_inputs(dims, "haar", False, 4)
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fat_i = q.qex_convert_links(lat, "f64", fat64, inner)
    b64 = q.qex_pack_field(lat, "f64", 0, dev(b))
    monkeypatch.setenv("QEX_RU_CYCLE", "50")
    monkeypatch.setenv("QEX_RU_FF", "1")
    st, s, x = _solve(q, lat, fat64, None, fat_i, None, 0.0, mass, b64, inner)
    assert st == 0 and s["converged"], s
    assert 1 <= s["ff_updates"] < s["reliable_updates"] - 10, s
    assert oracle_mod.true_residual(dims, u, b, x, mass) <= 1.05e-10
