"""qex_normal_op_static, the normal operator for callers that cannot
allocate device memory (for example code under an allocator that forbids
allocations outside its own pool, or paths that cannot afford cudaMalloc's
device-wide synchronisation).  It keeps the D_oe intermediate in a fixed
device array compiled into the library instead of a caller-provided buffer.

The tests call it through the C ABI (ctypes) and check
* its output against the CPU oracle's (m^2 - D_eo D_oe) x, norm-wise and
  element by element, in FP64, FP32 and the 16-bit two-row format, with and
  without the Naik term;
* that it gives the same bits as qex_normal_op, which takes a
  caller-allocated intermediate, on two calls in a row with different inputs
  and masses (the array keeps the previous call's contents, which must not
  leak into the next result);
* the path such a caller meets: a fresh lattice that nothing has tuned (the
  call never runs the autotuner, which allocates);
* that a call allocates nothing: after a warm-up call, neither torch's
  allocated bytes nor the device's free memory (cudaMemGetInfo) change;
* that a lattice whose intermediate does not fit the array is rejected
  before any launch.
This file is collected last so that a run stopping at the first failure has
run every other test first.
"""

import ctypes
import gc

import numpy as np
import pytest

import fieldgen as fg

pytestmark = pytest.mark.gpu

# oracle tolerances (norm-wise; element-wise against the largest |entry| at 5x)
TOL = {"f64": 1e-13, "f32": 1e-5, "f32r12h": 1e-4}
ELEM = 5.0
C3 = -1.0 / 24.0


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02750_gb300 import build

    build.build()
    import paper_1612_02750_gb300 as mod

    lib = mod.load()
    fn = lib.qex_normal_op_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return mod


def _call_static(q, lat, prec, fat, lng, c3, mass, inp, out):
    import torch

    vp = ctypes.c_void_p
    return q.load().qex_normal_op_static(lat.handle, q._prec(prec), vp(fat.data_ptr()),
                                         None if lng is None else vp(lng.data_ptr()), c3, mass,
                                         vp(inp.data_ptr()), vp(out.data_ptr()),
                                         vp(torch.cuda.current_stream().cuda_stream))


def _links(q, lat, prec, u, w):
    import torch

    fat64 = q.qex_pack_links(lat, "f64", torch.from_numpy(u).cuda())
    fat = fat64 if prec == "f64" else q.qex_convert_links(lat, "f64", fat64, prec)
    lng = None
    if w is not None:
        lng64 = q.qex_pack_links(lat, "f64", torch.from_numpy(w).cuda())
        lng = lng64 if prec == "f64" else q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec(prec))
    return fat, lng


def _inputs(dims, naik, seed):
    s = fg.rng_streams(seed)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    ev = fg.even_mask(dims)
    xs = []
    for key in ("source", "chi"):
        x = fg.gaussian_field(s[key], dims)
        x[~ev] = 0
        xs.append(x)
    return u, w, xs


def _check_oracle(got, ref, tol, what):
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    emax = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= tol and emax <= ELEM * tol, (what, err, emax)


@pytest.mark.parametrize("prec", ["f64", "f32", "f32r12h"])
@pytest.mark.parametrize("naik", [False, True])
def test_static_first_call_on_untuned_lattice_matches_oracle(q, oracle_mod, prec, naik):
    """A fresh lattice: two static calls in a row (different inputs and
    masses) in the compiled default launch shape, each against the oracle;
    the lattice stays untuned; then qex_normal_op (which tunes the lattice)
    gives the same bits as the static calls."""
    import torch

    dims = (10, 6, 4, 8)  # Vh = 960: three 256-site blocks and a ragged tail
    u, w, xs = _inputs(dims, naik, 61)
    c3 = C3 if naik else 0.0
    lat = q.Lattice(dims)
    assert q.qex_tune_info(lat, prec, naik)["source"] == "default"
    fat, lng = _links(q, lat, prec, u, w)
    ev = fg.even_mask(dims)
    results = []
    for x, mass in zip(xs, (0.1, 0.03)):
        inp = q.qex_pack_field(lat, prec, 0, torch.from_numpy(x).cuda())
        out = q.empty_field(lat, prec).fill_(float("nan"))
        assert _call_static(q, lat, prec, fat, lng, c3, mass, inp, out) == 0, q.qex_last_error()
        got = q.qex_unpack_field(lat, prec, 0, out).cpu().numpy()
        ref = oracle_mod.normal_op(dims, u, x, mass, w, c3)
        _check_oracle(got[ev], ref[ev], TOL[prec], (prec, naik, mass))
        results.append((inp, out, mass))
    assert q.qex_tune_info(lat, prec, naik)["source"] == "default"
    for inp, out, mass in results:
        ref = q.qex_normal_op(lat, prec, fat, lng, c3, mass, inp)
        assert torch.equal(out, ref)


@pytest.mark.parametrize("prec", ["f64", "f32", "f32r12h"])
@pytest.mark.parametrize("naik", [False, True])
def test_static_normal_op_matches_allocating_variant(q, oracle_mod, prec, naik):
    """Two calls in a row on a lattice qex_normal_op has already tuned: the
    static result equals qex_normal_op's bit for bit (within any tolerance)
    and meets the oracle."""
    import torch

    dims = (8, 6, 4, 10)
    u, w, xs = _inputs(dims, naik, 31)
    c3 = C3 if naik else 0.0
    lat = q.Lattice(dims)
    fat, lng = _links(q, lat, prec, u, w)
    ev = fg.even_mask(dims)
    for call, (x, mass) in enumerate(zip(xs, (0.1, 0.03))):
        inp = q.qex_pack_field(lat, prec, 0, torch.from_numpy(x).cuda())
        ref = q.qex_normal_op(lat, prec, fat, lng, c3, mass, inp)
        out = q.empty_field(lat, prec).fill_(float("nan"))
        assert _call_static(q, lat, prec, fat, lng, c3, mass, inp, out) == 0, q.qex_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert torch.equal(out, ref), f"call {call}"
        got = q.qex_unpack_field(lat, prec, 0, out).cpu().numpy()
        _check_oracle(got[ev], oracle_mod.normal_op(dims, u, x, mass, w, c3)[ev], TOL[prec], call)


@pytest.mark.parametrize("prec", ["f64", "f32r12h"])
def test_static_normal_op_allocates_nothing(q, prec):
    """After one warm-up call (which loads the kernels), further calls change
    neither torch's allocated bytes nor the device's free memory."""
    import torch

    dims = (8, 8, 8, 8)
    u, w, xs = _inputs(dims, True, 71)
    lat = q.Lattice(dims)
    fat, lng = _links(q, lat, prec, u, w)
    inp = q.qex_pack_field(lat, prec, 0, torch.from_numpy(xs[0]).cuda())
    out = q.empty_field(lat, prec)
    assert _call_static(q, lat, prec, fat, lng, C3, 0.1, inp, out) == 0, q.qex_last_error()
    torch.cuda.synchronize()
    # no Python garbage collection in between: it could free an earlier test's tensor and move
    # torch's count for a reason that has nothing to do with the calls
    gc.collect()
    gc.disable()
    try:
        alloc0 = torch.cuda.memory_allocated()
        free0, _ = torch.cuda.mem_get_info()
        for mass in (0.2, 0.05):
            assert _call_static(q, lat, prec, fat, lng, C3, mass, inp, out) == 0, q.qex_last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        alloc1 = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert alloc1 == alloc0
    assert free1 == free0


def test_static_normal_op_rejects_oversized_lattice(q):
    import torch

    small = q.Lattice((4, 4, 4, 4))
    fat = q.empty_links(small, "f64")
    f = q.zeros_field(small, "f64")
    big = q.Lattice((48, 48, 48, 48))  # FP64 intermediate 127 MB > 32 MiB
    assert big.half_volume * 48 > 32 << 20
    st = _call_static(q, big, "f64", fat, None, 0.0, 0.1, f, q.empty_field(small, "f64"))
    assert st == 2 and "static scratch" in q.qex_last_error()
    torch.cuda.synchronize()
