"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (norm-wise ||gpu - oracle|| / ||oracle|| per field, and the
largest element error against the largest |entry| within 5x that, see
parity.py): 1e-13 for FP64, 1e-5 for FP32 and two-row FP32 (inputs rounded to
FP32 on the device, oracle in FP64 on the unrounded inputs), 1e-4 for the
16-bit link formats.  Index work (neighbour tables, packing) is bit-exact.
Lattices span several 256-site blocks and a ragged tail.
"""

import numpy as np
import pytest

import fieldgen as fg
from parity import assert_close

pytestmark = pytest.mark.gpu

C3 = -1.0 / 24.0
# 16-bit fixed-point links: 1.5e-5 quantisation per real, ~3e-5 per entry of O(0.5)
TOL = {"f64": 1e-13, "f32": 1e-5, "f32r12": 1e-5, "f32r12h": 1e-4, "f32s16": 1e-4}
PRECS = ["f64", "f32", "f32r12", "f32r12h", "f32s16"]


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


def host(t):
    return t.cpu().numpy()


class Setup:
    """Packed links (F64 and F32) of one seeded input."""

    def __init__(self, q, dims, naik, seed=1, fat="haar", antiperiodic=True, a=0.3):
        self.q = q
        self.dims = dims
        s = fg.rng_streams(seed)
        self.u = fg.random_links(dims, fat, s["links"], a)
        self.w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
        self.psi = fg.gaussian_field(s["source"], dims)
        self.ap = antiperiodic
        self.lat = q.Lattice(dims, antiperiodic)
        self.fat = {"f64": q.qex_pack_links(self.lat, "f64", dev(self.u))}
        self.fat["f32"] = q.qex_convert_links(self.lat, "f64", self.fat["f64"], "f32")
        if fat in ("haar", "exp", "unit"):  # SU(3) links: two-row storage applies
            self.fat["f32r12"] = q.qex_convert_links(self.lat, "f64", self.fat["f64"], "f32r12")
            self.fat["f32r12h"] = q.qex_convert_links(self.lat, "f64", self.fat["f64"], "f32r12h")
        self.fat["f32s16"] = q.qex_convert_links(self.lat, "f64", self.fat["f64"], "f32s16")
        self.lng = {p: None for p in PRECS}
        if naik:
            self.lng["f64"] = q.qex_pack_links(self.lat, "f64", dev(self.w))
            self.lng["f32"] = q.qex_pack_links(self.lat, "f32", dev(self.w))
            self.lng["f32s16"] = q.qex_pack_links(self.lat, "f32s16", dev(self.w))
            for p in ("f32r12", "f32r12h"):  # long links are not unitary: never two-row
                self.lng[p] = self.lng[q.qex_long_links_prec(p)]

    def half(self, prec, parity, field):
        return self.q.qex_pack_field(self.lat, prec, parity, dev(field))

    def full(self, prec, parity, half):
        return host(self.q.qex_unpack_field(self.lat, prec, parity, half))


SHAPES = [(4, 4, 4, 4), (6, 4, 4, 10), (8, 4, 6, 4), (8, 8, 8, 12), (16, 8, 8, 8), (4, 6, 10, 8)]


@pytest.mark.parametrize("dims", SHAPES + [(2, 4, 2, 6)])
def test_neighbor_table_device_bit_exact(q, oracle_mod, dims):
    lat = q.Lattice(dims)
    for p in (0, 1):
        for mu in range(4):
            for hop in ((1, -1, 3, -3) if dims[mu] >= 4 else (1, -1)):
                got = host(q.qex_neighbor_table_device(lat, p, mu, hop))
                assert np.array_equal(got, oracle_mod.neighbor_table(dims, p, mu, hop))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 10)])
def test_pack_roundtrip_bit_exact(q, dims):
    s = fg.rng_streams(3)
    u = fg.random_links(dims, "haar", s["links"])
    lat = q.Lattice(dims)
    for prec, cast in (("f64", np.complex128), ("f32", np.complex64)):
        back = host(q.qex_unpack_links(lat, prec, q.qex_pack_links(lat, prec, dev(u))))
        assert np.array_equal(back, u.astype(cast).astype(np.complex128))
        f = fg.gaussian_field(s["source"], dims)
        ev = fg.even_mask(dims)
        for p in (0, 1):
            half = q.qex_pack_field(lat, prec, p, dev(f))
            out = dev(np.full_like(f, 7.0))
            q.qex_unpack_field(lat, prec, p, half, out)
            out = host(out)
            mine = ev if p == 0 else ~ev
            assert np.array_equal(out[mine], f.astype(cast).astype(np.complex128)[mine])
            assert np.all(out[~mine] == 7.0)
    l32 = q.qex_pack_links(lat, "f32", dev(u))
    l64 = q.qex_convert_links(lat, "f32", l32, "f64")
    assert np.array_equal(host(q.qex_unpack_links(lat, "f64", l64)), u.astype(np.complex64).astype(np.complex128))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 10), (10, 6, 4, 8)])
def test_pack_links_pair_equals_pack_then_convert(q, dims):
    """One pass from canonical links to the FP64 set and an FP32-class set
    gives the same bits as qex_pack_links to F64 followed by
    qex_convert_links, in every FP32 format (non-unitary Gaussian links for
    the scaled 16-bit one); an F64 second set and NULL buffers are refused."""
    import torch

    s = fg.rng_streams(5)
    lat = q.Lattice(dims)
    for second, kind in (("f32", "haar"), ("f32r12", "haar"), ("f32r12h", "haar"), ("f32s16", "gauss3")):
        u = fg.random_links(dims, kind, s["links"])
        ref64 = q.qex_pack_links(lat, "f64", dev(u))
        ref2 = q.qex_convert_links(lat, "f64", ref64, second)
        got64 = q.empty_links(lat, "f64").fill_(float("nan"))
        got2 = q.empty_links(lat, second).fill_(float("nan"))
        q.qex_pack_links_pair(lat, dev(u), second, got64, got2)
        # compared as bits: 16-bit words read as floats can be NaN patterns
        assert torch.equal(got64.view(torch.int64), ref64.view(torch.int64)), second
        assert torch.equal(got2.view(torch.int32), ref2.view(torch.int32)), second
    lib = q.load()
    assert lib.qex_pack_links_pair(lat.handle, dev(u).data_ptr(), got64.data_ptr(), 0, got2.data_ptr(), None) == 1
    assert lib.qex_pack_links_pair(lat.handle, None, got64.data_ptr(), 3, got2.data_ptr(), None) == 1


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 10)])
def test_convert_field_bit_exact(q, dims):
    """Half fields: F64 -> F32 rounds each real to nearest (numpy's cast),
    F32 -> F64 is exact, a conversion within FP64 or within the FP32-class
    formats (all of which keep FP32 vectors) copies; a NULL input is an
    argument error."""
    import torch

    s = fg.rng_streams(43)
    f = fg.gaussian_field(s["source"], dims)
    lat = q.Lattice(dims)
    ev = fg.even_mask(dims)
    rounded = f.astype(np.complex64).astype(np.complex128)
    for p in (0, 1):
        mine = ev if p == 0 else ~ev
        h64 = q.qex_pack_field(lat, "f64", p, dev(f))
        h32 = q.qex_convert_field(lat, "f64", h64, "f32")
        assert np.array_equal(host(q.qex_unpack_field(lat, "f32", p, h32))[mine], rounded[mine])
        assert torch.equal(h32, q.qex_pack_field(lat, "f32", p, dev(f)))
        back = q.qex_convert_field(lat, "f32", h32, "f64")
        assert np.array_equal(host(q.qex_unpack_field(lat, "f64", p, back))[mine], rounded[mine])
        assert torch.equal(q.qex_convert_field(lat, "f64", h64, "f64"), h64)
        for fmt in ("f32r12", "f32r12h", "f32s16"):
            assert torch.equal(q.qex_convert_field(lat, "f32", h32, fmt), h32)
    with pytest.raises(q.QexError) as e:
        q.qex_convert_field(lat, "f64", None, "f32")
    assert e.value.status == 1


@pytest.mark.parametrize("kind", ["haar", "exp"])
def test_two_row_links_roundtrip(q, kind):
    """SU(3) links stored as two FP32 rows come back with the third row rebuilt
    to FP32 accuracy; pack and convert from FP64 give the same bits."""
    dims = (6, 4, 4, 10)
    u = fg.random_links(dims, kind, fg.rng_streams(9)["links"])
    lat = q.Lattice(dims)
    r12 = q.qex_pack_links(lat, "f32r12", dev(u))
    assert r12.numel() * 4 == q.qex_links_bytes(lat, "f32r12") == int(np.prod(dims)) * 4 * 12 * 4
    back = host(q.qex_unpack_links(lat, "f32r12", r12))
    assert np.abs(back - u).max() <= 2e-6
    assert np.array_equal(back[..., :2, :], u[..., :2, :].astype(np.complex64).astype(np.complex128))
    via = q.qex_convert_links(lat, "f64", q.qex_pack_links(lat, "f64", dev(u)), "f32r12")
    assert np.array_equal(host(via), host(r12))


def test_fix16_links_roundtrip(q):
    """16-bit fixed-point two-row links: rows 0 and 1 come back as
    round(v * 32767) / 32767, row 2 rebuilt from them; pack and convert agree."""
    dims = (6, 4, 4, 10)
    u = fg.random_links(dims, "haar", fg.rng_streams(10)["links"])
    lat = q.Lattice(dims)
    h = q.qex_pack_links(lat, "f32r12h", dev(u))
    assert h.numel() * 4 == q.qex_links_bytes(lat, "f32r12h") == int(np.prod(dims)) * 4 * 12 * 2
    back = host(q.qex_unpack_links(lat, "f32r12h", h))
    rows = u[..., :2, :]
    quant = (np.round(rows.real * 32767) + 1j * np.round(rows.imag * 32767)) / 32767
    assert np.abs(back[..., :2, :] - quant).max() <= 1e-15
    assert np.abs(back - u).max() <= 1e-4
    via = q.qex_convert_links(lat, "f64", q.qex_pack_links(lat, "f64", dev(u)), "f32r12h")
    # entries outside [-1, 1] and NaN clamp to +-32767 (NaN to -32767)
    v = u.copy()
    v[0, 0, 0, 0, 0, 0, 0] = 1.5 - 2.5j
    v[0, 0, 0, 0, 1, 0, 1] = complex(np.nan, 0.25)
    hv = host(q.qex_unpack_links(lat, "f32r12h", q.qex_pack_links(lat, "f32r12h", dev(v))))
    assert hv[0, 0, 0, 0, 0, 0, 0] == 1.0 - 1.0j
    assert hv[0, 0, 0, 0, 1, 0, 1] == complex(-1.0, round(0.25 * 32767) / 32767)
    words = host(h).view(np.uint32)
    assert np.array_equal(host(via).view(np.uint32), words)  # raw bits (words are not floats)
    assert (words & 0xFFFF).min() >= 1 and (words >> 16).min() >= 1  # offset binary: q + 32768, q >= -32767


def test_scaled16_links_roundtrip(q):
    """16-bit links with a per-link step (any links, here non-unitary Gaussian
    ones): d = max |re|, |im| over the link / 32767 rounded up to FP32, q =
    round(v * (1/d)); unpack gives q * d; pack and convert agree."""
    dims = (6, 4, 4, 10)
    w = fg.random_links(dims, "gauss3", fg.rng_streams(11)["long_links"])
    w[0, 0, 0, 0, 2] = 0  # a zero link stays zero
    lat = q.Lattice(dims)
    h = q.qex_pack_links(lat, "f32s16", dev(w))
    assert h.numel() * 4 == q.qex_links_bytes(lat, "f32s16") == int(np.prod(dims)) * 4 * 40
    back = host(q.qex_unpack_links(lat, "f32s16", h))
    s = np.maximum(np.abs(w.real), np.abs(w.imag)).max(axis=(-2, -1), keepdims=True)
    d = (s / 32767).astype(np.float32)
    d = np.where(d.astype(np.float64) < s / 32767, np.nextafter(d, np.float32(np.inf)), d).astype(np.float64)
    inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    quant = (np.round(w.real * inv) + 1j * np.round(w.imag * inv)) * d
    assert np.array_equal(back, quant)
    assert not back[0, 0, 0, 0, 2].any()
    err = back - w
    assert (np.abs(err.real) <= d / 2 * (1 + 1e-12)).all() and (np.abs(err.imag) <= d / 2 * (1 + 1e-12)).all()
    via = q.qex_convert_links(lat, "f64", q.qex_pack_links(lat, "f64", dev(w)), "f32s16")
    assert np.array_equal(host(via).view(np.uint32), host(h).view(np.uint32))


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("prec", PRECS)
def test_dslash_parity(q, oracle_mod, dims, naik, prec):
    S = Setup(q, dims, naik, seed=21)
    for ap in (True, False):
        if not ap:
            S = Setup(q, dims, naik, seed=21, antiperiodic=False)
        for out_p in (0, 1):
            inp = S.half(prec, 1 - out_p, S.psi)
            got = S.full(prec, out_p, q.qex_dslash(S.lat, prec, S.fat[prec], S.lng[prec], C3, out_p, inp))
            ref = oracle_mod.dslash_parity(dims, S.u, S.psi, out_p, S.w, C3, ap)
            mask = fg.even_mask(dims) if out_p == 0 else ~fg.even_mask(dims)
            assert_close(got[mask], ref[mask], TOL[prec], (prec, dims, naik, ap, out_p))


def test_dslash_exp_links_and_unit_links(q, oracle_mod):
    dims = (8, 6, 4, 10)
    for fat in ("exp", "unit"):
        S = Setup(q, dims, True, seed=4, fat=fat)
        inp = S.half("f64", 1, S.psi)
        got = S.full("f64", 0, q.qex_dslash(S.lat, "f64", S.fat["f64"], S.lng["f64"], C3, 0, inp))
        ref = oracle_mod.dslash_parity(dims, S.u, S.psi, 0, S.w, C3, True)
        ev = fg.even_mask(dims)
        assert_close(got[ev], ref[ev], 1e-13, fat)


@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("prec", PRECS)
def test_normal_op_parity(q, oracle_mod, naik, prec):
    dims = (8, 4, 6, 10)
    S = Setup(q, dims, naik, seed=22)
    m = 0.07
    x = S.psi.copy()
    ev = fg.even_mask(dims)
    x[~ev] = 0
    got = S.full(prec, 0, q.qex_normal_op(S.lat, prec, S.fat[prec], S.lng[prec], C3, m, S.half(prec, 0, x)))
    ref = oracle_mod.normal_op(dims, S.u, x, m, S.w, C3)
    assert_close(got[ev], ref[ev], TOL[prec], (prec, naik))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_norm2_and_dot(q, prec):
    dims = (8, 8, 6, 10)
    lat = q.Lattice(dims)
    s = fg.rng_streams(8)
    a, b = fg.gaussian_field(s["source"], dims), fg.gaussian_field(s["chi"], dims)
    ev = fg.even_mask(dims)
    ha, hb = q.qex_pack_field(lat, prec, 0, dev(a)), q.qex_pack_field(lat, prec, 0, dev(b))
    cast = np.complex128 if prec == "f64" else np.complex64
    ae, be = a[ev].astype(cast).astype(np.complex128), b[ev].astype(cast).astype(np.complex128)
    n1 = host(q.qex_norm2(lat, prec, ha))[0]
    assert n1 == pytest.approx(np.vdot(ae, ae).real, rel=1e-13 if prec == "f64" else 1e-6)
    d = host(q.qex_dot(lat, prec, ha, hb))
    ref = np.vdot(ae, be)
    assert abs(complex(d[0], d[1]) - ref) <= (1e-12 if prec == "f64" else 1e-5) * np.sqrt(n1 * np.vdot(be, be).real)
    # fixed-order reductions: bitwise reproducible
    assert host(q.qex_norm2(lat, prec, ha))[0] == n1
    assert np.array_equal(host(q.qex_dot(lat, prec, ha, hb)), d)


def _cg(q, S, inner, m, b_full, tol=1e-10, maxiter=20000, delta=0.1, x0=None):
    import torch

    b = S.half("f64", 0, b_full)
    x = S.half("f64", 0, x0) if x0 is not None else torch.zeros_like(b)
    inner_fat = S.fat[inner if inner != "f64" else "f32"]
    inner_lng = S.lng[q.qex_long_links_prec(inner) if inner != "f64" else "f32"]
    st, stats = q.qex_cg(S.lat, inner, S.fat["f64"], S.lng["f64"], inner_fat, inner_lng, C3, m, b, x,
                         tol=tol, maxiter=maxiter, delta=delta, check=False)
    return st, stats, S.full("f64", 0, x)


@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("inner", PRECS)
def test_cg_parity(q, oracle_mod, naik, inner):
    dims = (8, 8, 4, 8)
    m = 0.1
    S = Setup(q, dims, naik, seed=23)
    b = S.psi.copy()
    b[~fg.even_mask(dims)] = 0
    st, stats, x = _cg(q, S, inner, m, b)
    assert st == 0 and stats["converged"], stats
    tr = oracle_mod.true_residual(dims, S.u, b, x, m, S.w, C3)
    assert tr <= 1.05e-10 and stats["true_rel_resid"] == pytest.approx(tr, rel=1e-3, abs=1e-13)
    xr, ok, it, _ = oracle_mod.cg(dims, S.u, b, m, S.w, C3, tol=1e-13, maxiter=50000)
    assert ok
    ev = fg.even_mask(dims)
    assert_close(x[ev], xr[ev], 1e-7, ("x against the oracle's 1e-13 solve", inner, naik))
    if inner != "f64":
        assert stats["reliable_updates"] >= 1


@pytest.mark.parametrize("inner", ["f64", "f32r12"])
def test_cg_graph_and_host_loop_agree_bitwise(q, oracle_mod, inner, monkeypatch):
    """The single-graph solve (conditional while/if nodes) and the host-driven
    batched loop run the same kernels in the same order: identical bits."""
    dims = (8, 4, 6, 8)
    m = 0.05
    S = Setup(q, dims, False, seed=25)
    b = S.psi.copy()
    b[~fg.even_mask(dims)] = 0
    monkeypatch.setenv("QEX_CG_MODE", "host")
    st_h, stats_h, x_h = _cg(q, S, inner, m, b, delta=0.05)
    monkeypatch.setenv("QEX_CG_MODE", "graph")
    st_g, stats_g, x_g = _cg(q, S, inner, m, b, delta=0.05)
    assert st_h == st_g == 0
    assert stats_h["iters"] == stats_g["iters"] and stats_h["reliable_updates"] == stats_g["reliable_updates"]
    assert np.array_equal(x_h, x_g)
    assert oracle_mod.true_residual(dims, S.u, b, x_g, m) <= 1.05e-10
    # maxiter reached inside the graph loop
    st, stats, _ = _cg(q, S, inner, m, b, maxiter=7)
    assert st == 5 and stats["iters"] == 7


def test_cg_workload_4x4_fp64_matches_oracle_iterations(q, oracle_mod):
    """4^4, Haar links, m = 0.1: FP64 CG reaches 1e-10 with the oracle's
    iteration count up to rounding-driven differences."""
    wl = fg.workload("cfg4x4")
    dims = wl["dims"]
    u, _, b = fg.make_inputs(dims, "haar", False, wl["seed"])
    S = Setup(q, dims, False, seed=wl["seed"])  # same streams: S.u is u
    assert np.array_equal(S.u, u)
    st, stats, x = _cg(q, S, "f64", wl["mass"], b)
    assert st == 0
    tr = oracle_mod.true_residual(dims, u, b, x, wl["mass"])
    assert tr <= 1.05e-10
    _, ok, it, _ = oracle_mod.cg(dims, u, b, wl["mass"], tol=1e-10)
    assert abs(stats["iters"] - it) <= max(5, it // 10)


def test_cg_edge_cases(q, oracle_mod):
    import torch

    dims = (4, 4, 4, 8)
    S = Setup(q, dims, True, seed=24)
    zero = np.zeros_like(S.psi)
    st, stats, x = _cg(q, S, "f32", 0.1, zero, x0=S.psi)
    assert st == 0 and stats["converged"] and not x.any()
    b = S.psi.copy()
    b[~fg.even_mask(dims)] = 0
    st, stats, x = _cg(q, S, "f64", 0.1, b, maxiter=2)
    assert st == 5 and stats["iters"] == 2 and not stats["converged"]
    st, stats, x = _cg(q, S, "f32", 0.1, b, maxiter=0)
    assert st == 5
    bad = b.copy()
    bad[0, 0, 0, 0, 1] = np.nan
    st, stats, x = _cg(q, S, "f64", 0.1, bad)
    assert st == 7
    # warm start from the converged solution: at most one iteration
    st, stats, x = _cg(q, S, "f64", 0.1, b, tol=1e-10)
    assert st == 0
    st2, stats2, x2 = _cg(q, S, "f32", 0.1, b, tol=1e-9, x0=x)
    assert st2 == 0 and stats2["iters"] <= 1
    # bitwise reproducible solve
    _, _, xa = _cg(q, S, "f32", 0.1, b)
    _, _, xb = _cg(q, S, "f32", 0.1, b)
    assert np.array_equal(xa, xb)
    torch.cuda.synchronize()


@pytest.mark.parametrize("inner", ["f64", "f32r12h"])
def test_cg_initial_guess_zero_and_one_site(q, oracle_mod, inner):
    """The first residual skips its Dslash passes only for an all-zero guess:
    a guess that is zero except for one tiny element (1e-300, whose square
    underflows) still gets b - A x, and both solves meet the oracle's true
    residual."""
    dims = (6, 4, 4, 10)
    m = 0.1
    S = Setup(q, dims, False, seed=26)
    b = S.psi.copy()
    b[~fg.even_mask(dims)] = 0
    st0, stats0, x0 = _cg(q, S, inner, m, b)
    assert st0 == 0 and oracle_mod.true_residual(dims, S.u, b, x0, m) <= 1.05e-10
    for val in (1e-300, 3.0):
        guess = np.zeros_like(b)
        guess[0, 0, 0, 0, 1] = val  # an even site (x + y + z + t = 0)
        st, stats, x = _cg(q, S, inner, m, b, x0=guess)
        tr = oracle_mod.true_residual(dims, S.u, b, x, m)
        assert st == 0 and tr <= 1.05e-10, (val, tr)
        assert stats["true_rel_resid"] == pytest.approx(tr, rel=1e-3, abs=1e-13)


def test_device_argument_errors(q):
    import torch

    dims = (4, 4, 2, 4)
    lat = q.Lattice(dims)
    f = q.zeros_field(lat, "f64")
    links = q.empty_links(lat, "f64")
    lng = q.empty_links(lat, "f64")
    with pytest.raises(q.QexError) as e:
        q.qex_dslash(lat, "f64", links, lng, C3, 0, f)  # Naik on extent 2
    assert e.value.status == 2
    raw = torch.zeros(f.numel() + 2, dtype=torch.float64, device="cuda")
    mis = raw[1:1 + f.numel()]
    with pytest.raises(q.QexError) as e:
        q.qex_dslash(lat, "f64", links, None, 0.0, 0, mis, q.empty_field(lat, "f64"))
    assert e.value.status == 3
    with pytest.raises(q.QexError) as e:
        q.qex_dslash(lat, "f64", links, None, 0.0, 0, f, f)
    assert e.value.status == 1
    with pytest.raises(q.QexError) as e:
        q.qex_dslash(lat, "f64", links, None, 0.0, 2, f)
    assert e.value.status == 1


@pytest.mark.slow
def test_full_size_32_every_format_and_bench_solve(q, oracle_mod):
    """The 32^4 workload (links exp(i 0.3 H), m = 0.01) against the oracle,
    element by element over the whole lattice:
    * D_oe in all five formats, in the launch shape the autotuner picks in
      this process; for the 16-bit formats also with the grid pinned to two
      resident waves of 128-thread blocks (the shape the benchmark's solve has
      run with), which must give the same bits;
    * the normal operator in FP64 and both 16-bit formats;
    * the benchmark's solve (16-bit two-row inner links, delta = 0.01): the
      oracle recomputes its true residual (<= 1.05e-10), and its solution
      agrees with the oracle's solve to 1e-13 within 1e-7 (the difference
      measured at 16^4 is 3e-10)."""
    import torch

    wl = fg.workload("cfg32")
    dims, mass = wl["dims"], wl["mass"]
    u, _, b = fg.make_inputs(dims, wl["fat"], False, wl["seed"], wl["a"])
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    fats = {"f64": fat64}
    for p in ("f32", "f32r12", "f32r12h", "f32s16"):
        fats[p] = q.qex_convert_links(lat, "f64", fat64, p)
    ev = fg.even_mask(dims)
    b_d = dev(b)
    ref = oracle_mod.dslash_parity(dims, u, b, 1, None, 0.0, True)
    for prec in PRECS:
        inp = q.qex_pack_field(lat, prec, 0, b_d)
        out = q.qex_dslash(lat, prec, fats[prec], None, 0.0, 1, inp)
        assert_close(host(q.qex_unpack_field(lat, prec, 1, out))[~ev], ref[~ev], TOL[prec], (prec, "tuned"))
        if prec in ("f32r12h", "f32s16"):
            tuned = q.qex_tune_info(lat, prec)
            q.qex_tune_set(lat, prec, False, dslash_block=128, reduce_block=tuned["reduce_block"],
                           reduce_blocks_per_sm=tuned["reduce_blocks_per_sm"], dslash_waves=2)
            capped = q.qex_dslash(lat, prec, fats[prec], None, 0.0, 1, inp)
            assert torch.equal(capped, out), prec
            q.qex_tune_set(lat, prec, False, dslash_block=tuned["dslash_block"], reduce_block=tuned["reduce_block"],
                           reduce_blocks_per_sm=tuned["reduce_blocks_per_sm"], dslash_waves=tuned["dslash_waves"])
        del out, inp
    ref_a = oracle_mod.normal_op(dims, u, b, mass)
    for prec in ("f64", "f32r12h", "f32s16"):
        inp = q.qex_pack_field(lat, prec, 0, b_d)
        got = host(q.qex_unpack_field(lat, prec, 0, q.qex_normal_op(lat, prec, fats[prec], None, 0.0, mass, inp)))
        assert_close(got[ev], ref_a[ev], TOL[prec], (prec, "normal operator"))
    bh = q.qex_pack_field(lat, "f64", 0, b_d)
    x = torch.zeros_like(bh)
    st, stats = q.qex_cg(lat, "f32r12h", fat64, None, fats["f32r12h"], None, 0.0, mass, bh, x, tol=1e-10,
                         maxiter=100000, delta=0.01)
    xf = host(q.qex_unpack_field(lat, "f64", 0, x))
    tr = oracle_mod.true_residual(dims, u, b, xf, mass)
    assert st == 0 and tr <= 1.05e-10, (stats, tr)
    assert stats["true_rel_resid"] == pytest.approx(tr, rel=1e-3)
    xr, ok, _, _ = oracle_mod.cg(dims, u, b, mass, tol=1e-13, maxiter=20000)
    assert ok
    assert_close(xf[ev], xr[ev], 1e-7, "bench solve against the oracle's 1e-13 solve")


@pytest.mark.slow
def test_full_size_64_naik_sampled_sites(q, oracle_mod):
    """The 64^4 workload with the Naik term (Haar fat links, Gaussian/sqrt(3)
    long links, c3 = -1/24) in the launch configuration the sweep times:
    both parities and four formats (FP64, FP32, two-row FP32 fat with FP32
    long links, 16-bit two-row fat with 16-bit scaled long links) on 4096
    sampled output sites
    against the oracle's per-site sum, anti-hermiticity
    <chi, D_eo psi> = -<D_oe chi, psi> over the whole lattice in FP64, and the
    workload's mixed-precision solve (m = 0.005, about 34,000 iterations and
    100 s on a GB300) to a true residual of 1e-10 that the oracle
    recomputes."""
    import torch

    wl = fg.workload("cfg64naik")
    dims = wl["dims"]
    u, w, b = fg.make_inputs_sliced(dims, wl["fat"], True, wl["seed"])
    psi = fg.gaussian_field(fg.rng_streams(wl["seed"] + 100)["source"], dims)
    lat = q.Lattice(dims)
    fat64 = q.qex_pack_links(lat, "f64", dev(u))
    lng64 = q.qex_pack_links(lat, "f64", dev(w))
    torch.cuda.empty_cache()
    links = {"f64": (fat64, lng64),
             "f32": (q.qex_convert_links(lat, "f64", fat64, "f32"), q.qex_convert_links(lat, "f64", lng64, "f32"))}
    links["f32r12"] = (q.qex_convert_links(lat, "f64", fat64, "f32r12"), links["f32"][1])
    links["f32r12h"] = (q.qex_convert_links(lat, "f64", fat64, "f32r12h"),
                        q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec("f32r12h")))
    rng = np.random.default_rng(17)
    ev = fg.even_mask(dims).reshape(-1)
    psi_d = dev(psi)
    for out_p in (0, 1):
        cand = np.flatnonzero(ev if out_p == 0 else ~ev)
        sites = np.sort(rng.choice(cand, 4096, replace=False))
        ref = oracle_mod.dslash_sites(dims, u, psi, sites, w, C3, True)
        for prec, (fat, lng) in links.items():
            inp = q.qex_pack_field(lat, prec, 1 - out_p, psi_d)
            out = q.qex_dslash(lat, prec, fat, lng, C3, out_p, inp)
            full = q.qex_unpack_field(lat, prec, out_p, out).reshape(-1, 3)
            got = full[torch.from_numpy(sites).cuda()].cpu().numpy()
            assert_close(got, ref, TOL[prec], (out_p, prec))
            del out, full
    chi_e = q.qex_pack_field(lat, "f64", 0, dev(b))
    psi_o = q.qex_pack_field(lat, "f64", 1, psi_d)
    d_eo_psi = q.qex_dslash(lat, "f64", fat64, lng64, C3, 0, psi_o)
    d_oe_chi = q.qex_dslash(lat, "f64", fat64, lng64, C3, 1, chi_e)
    lhs = host(q.qex_dot(lat, "f64", chi_e, d_eo_psi))
    rhs = host(q.qex_dot(lat, "f64", d_oe_chi, psi_o))
    assert abs(complex(*lhs) + complex(*rhs)) <= 1e-12 * abs(complex(*lhs))
    del d_eo_psi, d_oe_chi, psi_o, links
    torch.cuda.empty_cache()
    # the workload's solve: mixed-precision CG (two-row FP32 fat and FP32 long links inside, FP64
    # reliable updates, delta = 0.01) from x = 0 to a true residual of 1e-10, m = 0.005; the oracle
    # recomputes the true residual of the returned x
    fat_i = q.qex_convert_links(lat, "f64", fat64, "f32r12")
    lng_i = q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec("f32r12"))
    x = torch.zeros_like(chi_e)
    st, stats = q.qex_cg(lat, "f32r12", fat64, lng64, fat_i, lng_i, C3, wl["mass"], chi_e, x, tol=1e-10,
                         maxiter=100000, delta=0.01, check=False)
    assert st == 0 and stats["converged"], stats
    xf = host(q.qex_unpack_field(lat, "f64", 0, x))
    tr = oracle_mod.true_residual(dims, u, b, xf, wl["mass"], w, C3)
    assert tr <= 1.05e-10, (stats, tr)
    assert stats["true_rel_resid"] == pytest.approx(tr, rel=1e-3)
