"""Batched CG over independent lattices (qex_cg_batch) against the oracle."""

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


def _problem(q, dims, mass, seed, naik, inner, zero=False):
    s = fg.rng_streams(seed)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    b = fg.gaussian_field(s["source"], dims)
    b[~fg.even_mask(dims)] = 0
    if zero:
        b[...] = 0
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    lng64 = q.qex_pack_links(lat, "f64", dev(w)) if naik else None
    item = {"lat": lat, "fat64": fat64, "lng64": lng64, "mass": mass, "c_naik": C3 if naik else 0.0,
            "b64": q.qex_pack_field(lat, "f64", 0, dev(b))}
    if inner != "f64":
        item["fat32"] = q.qex_convert_links(lat, "f64", fat64, inner)
        item["lng32"] = q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec(inner)) if naik else None
    import torch

    item["x64"] = torch.zeros_like(item["b64"])
    return item, u, w, b


SPECS = [((4, 4, 4, 4), 0.1), ((6, 4, 4, 10), 0.05), ((8, 8, 4, 8), 0.2), ((8, 4, 6, 8), 0.08), ((4, 6, 4, 4), 0.3)]


@pytest.mark.parametrize("inner", ["f64", "f32", "f32r12", "f32r12h", "f32s16"])
@pytest.mark.parametrize("naik", [False, True])
def test_batch_matches_oracle_and_single(q, oracle_mod, inner, naik):
    """Five lattices of different extents and masses (one with a zero source)
    solved in one batch, in every inner format: each meets an
    oracle-recomputed true residual of 1.05e-10 and agrees with the oracle's
    1e-13 solve to 1e-7."""
    probs = [_problem(q, d, m, 70 + k, naik, inner, zero=(k == 3)) for k, (d, m) in enumerate(SPECS)]
    st, stats = q.qex_cg_batch([p[0] for p in probs], inner, tol=1e-10, delta=0.1)
    assert st == 0 and all(s["converged"] for s in stats), stats
    for k, (item, u, w, b) in enumerate(probs):
        dims = SPECS[k][0]
        lat = item["lat"]
        x = q.qex_unpack_field(lat, "f64", 0, item["x64"]).cpu().numpy()
        if k == 3:
            assert not x.any()
            continue
        tr = oracle_mod.true_residual(dims, u, b, x, item["mass"], w, item["c_naik"])
        assert tr <= 1.05e-10, (k, tr)
        xr, ok, _, _ = oracle_mod.cg(dims, u, b, item["mass"], w, item["c_naik"], tol=1e-13, maxiter=50000)
        assert ok
        ev = fg.even_mask(dims)
        assert_close(x[ev], xr[ev], 1e-7, ("x against the oracle's 1e-13 solve", k))


@pytest.mark.slow
def test_batch_multi_lattice_workload_full(q, oracle_mod):
    """The multi-lattice workload in full: eight lattices 8^4, 12^4, 16^4,
    16^3 x 32, 20^4, 24^4, 24^3 x 48, 32^4 (Haar links, seed 4 + 10k, masses
    m_k = 0.005 * 20^(k/7) in that order) in one batch with 16-bit inner links,
    delta = 0.01 and the tuned launch shape: every lattice converges and the
    oracle recomputes each true residual <= 1.05e-10."""
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (16, 16, 16, 32), (20, 20, 20, 20),
                 (24, 24, 24, 24), (24, 24, 24, 48), (32, 32, 32, 32)]
    masses = [0.005 * 20 ** (k / 7) for k in range(8)]
    probs = [_problem(q, d, m, 4 + 10 * k, False, "f32r12h") for k, (d, m) in enumerate(zip(dims_list, masses))]
    st, stats = q.qex_cg_batch([p[0] for p in probs], "f32r12h", tol=1e-10, maxiter=100000, delta=0.01)
    assert st == 0 and all(s["converged"] for s in stats), stats
    shape = q.qex_cg_batch_tune_info(probs[0][0]["lat"])
    assert shape["source"] in ("measured", "cache", "disabled"), shape
    for k, (item, u, w, b) in enumerate(probs):
        x = q.qex_unpack_field(item["lat"], "f64", 0, item["x64"]).cpu().numpy()
        assert oracle_mod.true_residual(dims_list[k], u, b, x, masses[k]) <= 1.05e-10, k


@pytest.mark.parametrize("inner,naik", [("f32r12h", True), ("f64", False)])
def test_batch_shapes_give_identical_bits(q, oracle_mod, inner, naik):
    """Every (blocks per SM, groups per work item) shape runs the same
    per-site arithmetic and the same per-256-site-group reductions: pinned
    shapes (1, 1), (3, 2), (2, 4) and the autotuner's choice give the same
    iteration counts and bit-identical solutions, which meet the oracle."""
    import torch

    runs = []
    for pin in ((1, 1), (3, 2), (2, 4), None):
        probs = [_problem(q, d, m, 110 + k, naik, inner) for k, (d, m) in enumerate(SPECS)]
        lead = probs[0][0]["lat"]
        if pin:
            q.qex_cg_batch_tune_set(lead, *pin)
        st, stats = q.qex_cg_batch([p[0] for p in probs], inner, tol=1e-10, delta=0.1)
        assert st == 0 and all(s["converged"] for s in stats), (pin, stats)
        info = q.qex_cg_batch_tune_info(lead)
        if pin:
            assert (info["blocks_per_sm"], info["groups_per_item"], info["source"]) == (pin[0], pin[1], "set")
        else:
            assert info["source"] in ("measured", "cache", "disabled")
        runs.append(([s["iters"] for s in stats], [p[0]["x64"].clone() for p in probs], probs))
    for its, xs, _ in runs[1:]:
        assert its == runs[0][0]
        for a, b in zip(xs, runs[0][1]):
            assert torch.equal(a, b)
    for k, (item, u, w, b) in enumerate(runs[0][2]):
        x = q.qex_unpack_field(item["lat"], "f64", 0, runs[0][1][k]).cpu().numpy()
        assert oracle_mod.true_residual(SPECS[k][0], u, b, x, item["mass"], w, item["c_naik"]) <= 1.05e-10


def test_batch_tuner_measures_once_per_key(q, monkeypatch):
    """A set of extents the process has not seen: the first batch measures
    the launch shape, the next batch with the same extents takes it from the
    process cache; a pin is reported as set and (0, 0) removes it."""
    monkeypatch.delenv("QEX_TUNE", raising=False)
    specs = [((4, 4, 6, 10), 0.2), ((6, 6, 4, 8), 0.15)]  # extents no other test batches
    sources = []
    for _ in range(2):
        probs = [_problem(q, d, m, 120 + k, False, "f32r12h") for k, (d, m) in enumerate(specs)]
        st, _ = q.qex_cg_batch([p[0] for p in probs], "f32r12h", tol=1e-10, delta=0.1)
        assert st == 0
        sources.append(q.qex_cg_batch_tune_info(probs[0][0]["lat"])["source"])
    assert sources == ["measured", "cache"]
    with pytest.raises(q.QexError) as e:
        q.qex_cg_batch_tune_set(probs[0][0]["lat"], 4, 1)
    assert e.value.status == 1
    with pytest.raises(q.QexError):
        q.qex_cg_batch_tune_set(probs[0][0]["lat"], 2, 3)
    q.qex_cg_batch_tune_set(probs[0][0]["lat"], 0, 0)


def test_batch_errors(q):
    a, _, _, _ = _problem(q, (4, 4, 4, 4), 0.1, 80, False, "f64")
    b, _, _, _ = _problem(q, (4, 4, 4, 4), 0.1, 81, True, "f64")
    with pytest.raises(q.QexError) as e:
        q.qex_cg_batch([a, b], "f64")  # Naik disagreement
    assert e.value.status == 1
    with pytest.raises(q.QexError) as e:
        q.qex_cg_batch([a, dict(a)], "f64")  # shared lattice object
    assert e.value.status == 1
    with pytest.raises(q.QexError) as e:
        q.qex_cg_batch([a], "f32r12h")  # no inner-precision links
    assert e.value.status == 1


@pytest.mark.parametrize("inner", ["f64", "f32r12h"])
def test_batch_graph_matches_host_loop(q, monkeypatch, inner):
    """The CUDA-graph batch loop and the host-driven loop run the same kernels
    in the same order: identical iteration counts and bitwise-equal solutions."""
    import torch

    runs = []
    for mode in ("graph", "host"):
        if mode == "host":
            monkeypatch.setenv("QEX_CG_MODE", "host")
        probs = [_problem(q, d, m, 90 + k, True, inner) for k, (d, m) in enumerate(SPECS)]
        st, stats = q.qex_cg_batch([p[0] for p in probs], inner, tol=1e-10, delta=0.1)
        assert st == 0
        runs.append(([s["iters"] for s in stats], [p[0]["x64"].clone() for p in probs]))
    assert runs[0][0] == runs[1][0]
    for a, b in zip(runs[0][1], runs[1][1]):
        assert torch.equal(a, b)


def test_batch_maxiter_stops_every_lattice(q):
    """A cap below what the lattices need: the solve stops at the cap with
    QEX_ERR_NOT_CONVERGED (status 5) and reports each lattice's count."""
    probs = [_problem(q, d, m, 100 + k, False, "f32r12h") for k, (d, m) in enumerate(SPECS[:3])]
    st, stats = q.qex_cg_batch([p[0] for p in probs], "f32r12h", tol=1e-12, maxiter=7, delta=0.1, check=False)
    assert st == 5
    assert [s["iters"] for s in stats] == [7, 7, 7] and not any(s["converged"] for s in stats)
