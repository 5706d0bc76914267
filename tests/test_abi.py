"""C-ABI checks that need no GPU: the library loads, exports every entry point
the header declares, and its host-side index arithmetic (the same inline code
the kernels run) reproduces the oracle's even-odd and neighbour tables
bit-exactly.  Argument errors are reported as status codes."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names |= set(re.findall(r"\b(qex_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1612_02750_gb300 import build

    build.build()
    import paper_1612_02750_gb300 as q

    return q.load()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("qex_dslash", "qex_cg", "qex_pack_links", "qex_lattice_create", "qex_norm2"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_declared_symbols():
    import paper_1612_02750_gb300 as q

    assert set(q.exported_symbols()) <= _declared()


def _lattice(lib, dims, ap=1):
    h = ctypes.c_void_p()
    st = lib.qex_lattice_create((ctypes.c_int * 4)(*dims), ap, ctypes.byref(h))
    return st, h


def test_volume_and_version_host_calls(lib):
    """qex_volume / qex_half_volume of a lattice (-1 for NULL), the same
    through the binding, and a non-empty version string; none touches the
    device."""
    import paper_1612_02750_gb300 as q

    for dims in [(4, 4, 4, 4), (6, 4, 2, 8), (64, 64, 64, 64)]:
        st, h = _lattice(lib, dims)
        assert st == 0
        try:
            V = int(np.prod(dims))
            assert lib.qex_volume(h) == V and lib.qex_half_volume(h) == V // 2
        finally:
            lib.qex_lattice_destroy(h)
        lat = q.Lattice(dims)
        assert (lat.volume, lat.half_volume) == (int(np.prod(dims)), int(np.prod(dims)) // 2)
    assert lib.qex_volume(None) == -1 and lib.qex_half_volume(None) == -1
    v = q.qex_version()
    assert v and v.isprintable()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (2, 6, 4, 10), (8, 4, 6, 4)])
def test_host_index_math_matches_oracle(lib, oracle_mod, dims):
    st, h = _lattice(lib, dims)
    assert st == 0
    try:
        eo = oracle_mod.eo_table(dims)
        V = int(np.prod(dims))
        vh = V // 2
        t, z, y, x = np.indices((dims[3], dims[2], dims[1], dims[0]))
        coords = np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)
        for s in range(0, V, max(1, V // 97)):
            assert lib.qex_eo_index(h, (ctypes.c_int * 4)(*coords[s])) == eo[s]
        out = np.empty(vh, dtype=np.int32)
        for p in (0, 1):
            for mu in range(4):
                hops = (1, -1, 3, -3) if dims[mu] >= 4 else (1, -1)
                for hop in hops:
                    assert lib.qex_neighbor_table(h, p, mu, hop, out.ctypes.data) == 0
                    assert np.array_equal(out, oracle_mod.neighbor_table(dims, p, mu, hop)), (p, mu, hop)
    finally:
        lib.qex_lattice_destroy(h)


def test_fast_division_edge_extents(lib, oracle_mod):
    """Extents that are not powers of two, including large ones, through the
    multiply-high division in the site decoder."""
    for dims in [(14, 6, 10, 2), (2, 2, 2, 2), (30, 2, 18, 2), (2, 26, 2, 6)]:
        st, h = _lattice(lib, dims)
        assert st == 0
        vh = int(np.prod(dims)) // 2
        out = np.empty(vh, dtype=np.int32)
        for p in (0, 1):
            for mu in range(4):
                assert lib.qex_neighbor_table(h, p, mu, 1, out.ctypes.data) == 0
                assert np.array_equal(out, oracle_mod.neighbor_table(dims, p, mu, 1))
        lib.qex_lattice_destroy(h)


def test_argument_errors(lib):
    assert _lattice(lib, (4, 4, 4, 5))[0] == 2       # odd extent
    assert _lattice(lib, (4, 4, 0, 4))[0] == 2       # zero extent
    assert _lattice(lib, (2048, 2048, 2048, 2))[0] == 2  # V >= 2^31
    assert lib.qex_lattice_create(None, 1, None) == 1
    st, h = _lattice(lib, (4, 4, 2, 4))
    out = np.empty(64, dtype=np.int32)
    assert lib.qex_neighbor_table(h, 2, 0, 1, out.ctypes.data) == 1     # bad parity
    assert lib.qex_neighbor_table(h, 0, 4, 1, out.ctypes.data) == 1     # bad direction
    assert lib.qex_neighbor_table(h, 0, 0, 2, out.ctypes.data) == 1     # bad hop
    assert lib.qex_neighbor_table(h, 0, 2, 3, out.ctypes.data) == 2     # 3-hop on extent 2
    assert lib.qex_neighbor_table(h, 0, 0, 1, None) == 1
    assert b"NULL" in lib.qex_last_error()
    assert lib.qex_dslash(None, 0, None, None, 0.0, 0, None, None, None) == 1
    assert lib.qex_cg(h, 0, None, None, None, None, 0.0, 0.1, None, None, 1e-10, 10, 0.1, None, None) == 1
    assert lib.qex_eo_index(h, (ctypes.c_int * 4)(0, 0, 2, 0)) == -1
    assert lib.qex_links_bytes(h, 0) == 4 * 128 * 18 * 8
    assert lib.qex_field_bytes(h, 1) == 64 * 6 * 4
    assert lib.qex_links_bytes(h, 2) == 4 * 128 * 12 * 4
    assert lib.qex_field_bytes(h, 2) == 64 * 6 * 4
    assert lib.qex_links_bytes(h, 3) == 4 * 128 * 12 * 2
    assert lib.qex_links_bytes(h, 4) == 4 * 128 * 40  # 18 16-bit reals + an FP32 step per link
    assert lib.qex_field_bytes(h, 4) == 64 * 6 * 4
    assert lib.qex_pack_links(h, 5, None, None, None) == 1  # unknown precision
    # one-pass pack: NULL buffers, an F64 or unknown second format (all refused before any launch)
    bufs = [np.zeros(64, dtype=np.float64) for _ in range(3)]
    ptrs = [b.ctypes.data for b in bufs]
    assert lib.qex_pack_links_pair(h, None, ptrs[1], 3, ptrs[2], None) == 1
    assert lib.qex_pack_links_pair(h, ptrs[0], ptrs[1], 0, ptrs[2], None) == 1
    assert b"FP32" in lib.qex_last_error()
    assert lib.qex_pack_links_pair(h, ptrs[0], ptrs[1], 7, ptrs[2], None) == 1
    # true residual: NULL inputs, then a NULL result or an unknown arithmetic (refused before any launch)
    rel = ctypes.c_double()
    assert lib.qex_true_residual(h, None, None, 0.0, 0.1, ptrs[0], ptrs[1], 0, ctypes.byref(rel), None) == 1
    assert lib.qex_true_residual(h, ptrs[2], None, 0.0, 0.1, ptrs[0], ptrs[1], 0, None, None) == 1
    assert lib.qex_true_residual(h, ptrs[2], None, 0.0, 0.1, ptrs[0], ptrs[1], 2, ctypes.byref(rel), None) == 1
    assert b"arith" in lib.qex_last_error()
    # long-link format per operator precision: two-row storage never applies to long links
    assert [lib.qex_long_links_prec(p) for p in range(6)] == [0, 1, 1, 4, 4, -1]
    lib.qex_lattice_destroy(h)
