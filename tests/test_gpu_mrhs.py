"""Multi-right-hand-side Dslash and CG against the single-RHS path and the
oracle."""

import numpy as np
import pytest

import fieldgen as fg
from parity import assert_close

pytestmark = pytest.mark.gpu

C3 = -1.0 / 24.0
TOL = {"f64": 1e-14, "f32": 1e-6, "f32r12": 1e-6, "f32r12h": 1e-6, "f32s16": 1e-6}


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


@pytest.mark.parametrize("nrhs", [1, 3, 5, 16, 37])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32r12", "f32r12h", "f32s16"])
@pytest.mark.parametrize("naik", [False, True])
def test_dslash_mrhs_matches_single(q, nrhs, prec, naik):
    """Each output field of the batched operator equals the single-RHS
    operator on that field (same arithmetic order; ragged RHS groups and a
    ragged site tail)."""
    import torch

    dims = (6, 4, 4, 10)
    s = fg.rng_streams(61)
    u = fg.random_links(dims, "haar", s["links"])
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fat = fat64 if prec == "f64" else q.qex_convert_links(lat, "f64", fat64, prec)
    lng = None
    if naik:
        w = fg.random_links(dims, "gauss3", s["long_links"])
        lng = q.qex_pack_links(lat, q.qex_long_links_prec(prec), dev(w))
    n = q.qex_field_bytes(lat, prec) // (8 if prec == "f64" else 4)
    for out_p in (0, 1):
        inp = q.empty_fields(lat, prec, nrhs).normal_()
        out = q.qex_dslash_mrhs(lat, prec, fat, lng, C3, out_p, nrhs, inp)
        for r in range(nrhs):
            ref = q.qex_dslash(lat, prec, fat, lng, C3, out_p, inp[r * n:(r + 1) * n].contiguous())
            got = out[r * n:(r + 1) * n]
            assert torch.linalg.norm(got - ref).item() <= TOL[prec] * torch.linalg.norm(ref).item(), (out_p, r)


def test_dslash_mrhs_matches_oracle(q, oracle_mod):
    dims = (8, 4, 6, 8)
    s = fg.rng_streams(62)
    u = fg.random_links(dims, "exp", s["links"], 0.4)
    w = fg.random_links(dims, "gauss3", s["long_links"])
    lat = q.Lattice(dims)
    fat = q.qex_pack_links(lat, "f64", dev(u))
    lng = q.qex_pack_links(lat, "f64", dev(w))
    fields = [fg.gaussian_field(s["source"], dims) for _ in range(6)]
    inp = torch_cat(q, [q.qex_pack_field(lat, "f64", 1, dev(f)) for f in fields])
    out = q.qex_dslash_mrhs(lat, "f64", fat, lng, C3, 0, 6, inp)
    n = q.qex_field_bytes(lat, "f64") // 8
    ev = fg.even_mask(dims)
    for r, f in enumerate(fields):
        got = q.qex_unpack_field(lat, "f64", 0, out[r * n:(r + 1) * n].contiguous()).cpu().numpy()
        ref = oracle_mod.dslash_parity(dims, u, f, 0, w, C3)
        assert_close(got[ev], ref[ev], 1e-13, r)


# oracle tolerances of the formats (16-bit links: 1.5e-5 quantisation per real)
ORACLE_TOL = {"f32": 1e-5, "f32r12": 1e-5, "f32r12h": 1e-4, "f32s16": 1e-4}


@pytest.mark.parametrize("prec", ["f32", "f32r12", "f32r12h", "f32s16"])
@pytest.mark.parametrize("naik", [False, True])
def test_dslash_mrhs_fp32_formats_match_oracle(q, oracle_mod, prec, naik):
    """Every FP32-class format of the batched operator against the oracle on
    the unrounded FP64 inputs, element by element: 6 right-hand sides (a full
    group of 4 and a ragged group of 2), both output parities, a ragged site
    tail (Vh = 960)."""
    dims = (10, 6, 4, 8)
    s = fg.rng_streams(64)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    c3 = C3 if naik else 0.0
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fat = q.qex_convert_links(lat, "f64", fat64, prec)
    lng = None
    if naik:
        lng = q.qex_convert_links(lat, "f64", q.qex_pack_links(lat, "f64", dev(w)), q.qex_long_links_prec(prec))
    fields = [fg.gaussian_field(s["source"], dims) for _ in range(6)]
    n = q.qex_field_bytes(lat, prec) // 4
    ev = fg.even_mask(dims)
    for out_p in (0, 1):
        inp = torch_cat(q, [q.qex_pack_field(lat, prec, 1 - out_p, dev(f)) for f in fields])
        out = q.qex_dslash_mrhs(lat, prec, fat, lng, c3, out_p, 6, inp)
        mask = ev if out_p == 0 else ~ev
        for r, f in enumerate(fields):
            got = q.qex_unpack_field(lat, prec, out_p, out[r * n:(r + 1) * n].contiguous()).cpu().numpy()
            ref = oracle_mod.dslash_parity(dims, u, f, out_p, w, c3)
            assert_close(got[mask], ref[mask], ORACLE_TOL[prec], (prec, naik, out_p, r))


def torch_cat(q, parts):
    import torch

    return torch.cat(parts).contiguous()


@pytest.mark.parametrize("inner", ["f64", "f32", "f32r12", "f32r12h", "f32s16"])
@pytest.mark.parametrize("naik", [False, True])
def test_cg_mrhs(q, oracle_mod, inner, naik):
    """Five sources (one of them zero, the others 1e-2 .. 1e2 in size) solved
    together, in every inner format (long links in qex_long_links_prec):
    every solution has an oracle-recomputed true residual <= 1.05e-10 and
    agrees with the oracle's 1e-13 solve of the same source to 1e-7."""
    import torch

    dims = (8, 8, 4, 8)
    m = 0.1
    s = fg.rng_streams(63)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    c3 = C3 if naik else 0.0
    ev = fg.even_mask(dims)
    srcs = []
    for r in range(5):
        b = fg.gaussian_field(s["source"], dims) * (0.0 if r == 2 else 10.0 ** (r - 2))
        b[~ev] = 0
        srcs.append(b)
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    lng64 = q.qex_pack_links(lat, "f64", dev(w)) if naik else None
    fat32 = q.qex_convert_links(lat, "f64", fat64, inner) if inner != "f64" else None
    lng32 = q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec(inner)) if (naik and inner != "f64") else None
    B = torch_cat(q, [q.qex_pack_field(lat, "f64", 0, dev(b)) for b in srcs])
    X = torch.zeros_like(B)
    st, stats = q.qex_cg_mrhs(lat, inner, fat64, lng64, fat32, lng32, c3, m, 5, B, X, tol=1e-10, delta=0.1)
    assert st == 0 and all(x["converged"] for x in stats), stats
    n = q.qex_field_bytes(lat, "f64") // 8
    for r, b in enumerate(srcs):
        x = q.qex_unpack_field(lat, "f64", 0, X[r * n:(r + 1) * n].contiguous()).cpu().numpy()
        if r == 2:
            assert not x.any()
            continue
        tr = oracle_mod.true_residual(dims, u, b, x, m, w, c3)
        assert tr <= 1.05e-10, (r, tr)
        xr, ok, _, _ = oracle_mod.cg(dims, u, b, m, w, c3, tol=1e-13, maxiter=50000)
        assert ok
        assert_close(x[ev], xr[ev], 1e-7, ("x against the oracle's 1e-13 solve", r))


def test_cg_mrhs_errors(q):
    import torch

    lat = q.Lattice((4, 4, 4, 4))
    fat = q.empty_links(lat, "f64")
    B = q.empty_fields(lat, "f64", 2).zero_()
    X = torch.zeros_like(B)
    with pytest.raises(q.QexError) as e:
        q.qex_cg_mrhs(lat, "f64", fat, None, None, None, 0.0, 0.1, 0, B, X)
    assert e.value.status == 1
    with pytest.raises(q.QexError) as e:
        q.qex_cg_mrhs(lat, "f64", fat, None, None, None, 0.0, 0.1, 65, B, X)
    assert e.value.status == 1
    st, stats = q.qex_cg_mrhs(lat, "f64", fat, None, None, None, 0.0, 0.1, 2, B, X)  # zero sources
    assert st == 0 and all(s["converged"] for s in stats) and not X.any()


@pytest.mark.slow
def test_cg_mrhs_workload_24x24x24x24_16_sources(q, oracle_mod):
    """The multi-RHS workload in full: 24^4, Haar links (seed 4), 16 Gaussian
    even-site sources, m = 0.05, one batched mixed-precision solve (two-row
    FP32 inner links, FP64 reliable updates, delta = 0.01) to 1e-10: every
    source converges and the oracle recomputes each true residual."""
    import torch

    dims, nrhs, seed, m = (24, 24, 24, 24), 16, 4, 0.05
    st = fg.rng_streams(seed)
    u = fg.random_links(dims, "haar", st["links"])
    ev = fg.even_mask(dims)
    srcs = []
    for _ in range(nrhs):
        b = fg.gaussian_field(st["source"], dims)
        b[~ev] = 0
        srcs.append(b)
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fatr = q.qex_convert_links(lat, "f64", fat64, "f32r12")
    B = torch_cat(q, [q.qex_pack_field(lat, "f64", 0, dev(b)) for b in srcs])
    X = torch.zeros_like(B)
    status, stats = q.qex_cg_mrhs(lat, "f32r12", fat64, None, fatr, None, 0.0, m, nrhs, B, X, tol=1e-10,
                                  delta=0.01)
    assert status == 0 and all(s["converged"] for s in stats), stats
    n = q.qex_field_bytes(lat, "f64") // 8
    for r, b in enumerate(srcs):
        x = q.qex_unpack_field(lat, "f64", 0, X[r * n:(r + 1) * n].contiguous()).cpu().numpy()
        tr = oracle_mod.true_residual(dims, u, b, x, m)
        assert tr <= 1.05e-10, (r, tr)
        assert stats[r]["true_rel_resid"] == pytest.approx(tr, rel=1e-3)
