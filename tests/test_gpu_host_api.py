"""qex_cg_host: the whole path from page-locked host buffers (copy in, pack,
convert, solve, unpack, copy out) against the same solve through the device
entry points and against the oracle."""

import numpy as np
import pytest

import fieldgen as fg
from test_gpu_parity import C3, Setup, _cg

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("inner", ["f64", "f32r12h", "f32s16"])
@pytest.mark.parametrize("dims", [(8, 4, 6, 8), (6, 4, 4, 10)])
def test_cg_host_matches_device_solve(q, oracle_mod, inner, naik, dims):
    """Same kernels on the same bits: the host-buffer solve (links copied and
    packed in t-slabs: 8 slabs of one slice, or 8 slabs of one or two slices
    for Lt = 10) returns the device solve's iterate exactly, with zeros on the
    odd sites, and meets the oracle's true residual."""
    import torch

    m = 0.1
    S = Setup(q, dims, naik, seed=41)
    b = S.psi.copy()
    ev = fg.even_mask(dims)
    b[~ev] = 0
    st_d, stats_d, x_d = _cg(q, S, inner, m, b)
    assert st_d == 0 and stats_d["converged"]

    lat = q.Lattice(dims)
    host_fat = torch.from_numpy(S.u).pin_memory()
    host_lng = torch.from_numpy(S.w).pin_memory() if naik else None
    host_b = torch.from_numpy(b).pin_memory()
    host_x = torch.full_like(host_b, complex(np.nan, np.nan)).pin_memory()  # every site is written
    x_h, st_h, stats_h = q.qex_cg_host(lat, inner, host_fat, host_lng, C3, m, host_b, host_x, tol=1e-10)
    x_h = x_h.numpy()
    assert st_h == 0 and stats_h["converged"]
    assert stats_h["iters"] == stats_d["iters"] and stats_h["reliable_updates"] == stats_d["reliable_updates"]
    assert np.array_equal(x_h[ev], x_d[ev])
    assert not np.any(x_h[~ev])
    assert oracle_mod.true_residual(dims, S.u, b, x_h, m, S.w, C3) <= 1.05e-10


def test_cg_host_rejects_device_tensors(q):
    import torch

    lat = q.Lattice((4, 4, 4, 4))
    u = torch.zeros((4, 4, 4, 4, 4, 3, 3), dtype=torch.complex128)
    b = torch.zeros((4, 4, 4, 4, 3), dtype=torch.complex128)
    with pytest.raises(ValueError):
        q.qex_cg_host(lat, "f64", u.cuda(), None, 0.0, 0.1, b)
    with pytest.raises(ValueError):
        q.qex_cg_host(lat, "f64", u, None, 0.0, 0.1, b.to(torch.complex64))
