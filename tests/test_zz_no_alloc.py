"""qex_normal_op_static, the normal operator for callers that cannot
allocate device memory (for example code under an allocator that forbids
allocations outside its own pool, or paths that cannot afford cudaMalloc's
device-wide synchronisation).  It keeps the D_oe intermediate in a fixed
device array compiled into the library instead of a caller-provided buffer.

The test calls it through the C ABI (ctypes) and checks its output against
qex_normal_op, which takes a caller-allocated intermediate, within the FP64 /
FP32 parity tolerances, on two calls in a row with different inputs (the
array keeps the previous call's contents, which must not leak into the next
result).  It also checks that a lattice whose intermediate does not fit the
array is rejected before any launch.  This file is collected last so that a
run stopping at the first failure has run every other test first.
"""

import ctypes

import numpy as np
import pytest

import fieldgen as fg

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6}
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

    p = q.F64 if prec == "f64" else q.F32
    vp = ctypes.c_void_p
    st = q.load().qex_normal_op_static(lat.handle, p, vp(fat.data_ptr()),
                                       None if lng is None else vp(lng.data_ptr()), c3, mass,
                                       vp(inp.data_ptr()), vp(out.data_ptr()),
                                       vp(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("naik", [False, True])
def test_static_normal_op_matches_allocating_variant(q, prec, naik):
    import torch

    dims = (8, 6, 4, 10)
    s = fg.rng_streams(31)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    lat = q.Lattice(dims)
    fat = q.qex_pack_links(lat, prec, torch.from_numpy(u).cuda())
    lng = q.qex_pack_links(lat, prec, torch.from_numpy(w).cuda()) if naik else None
    for call, (seed_field, mass) in enumerate(((s["source"], 0.1), (s["chi"], 0.03))):
        x = fg.gaussian_field(seed_field, dims)
        inp = q.qex_pack_field(lat, prec, 0, torch.from_numpy(x).cuda())
        ref = q.qex_normal_op(lat, prec, fat, lng, C3, mass, inp)
        out = q.empty_field(lat, prec).fill_(float("nan"))
        assert _call_static(q, lat, prec, fat, lng, C3, mass, inp, out) == 0, q.qex_last_error()
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) <= TOL[prec] * np.linalg.norm(b), f"call {call}"


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
