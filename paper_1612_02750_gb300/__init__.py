"""GB300 even-odd staggered Dirac operator and CG solvers (libqex_gpu).

Thin Python binding of the C ABI declared in ``include/qex_gpu.h``: every
function here has the name of the C entry point it calls and only marshals
arguments (torch tensors -> device pointers, the current torch CUDA stream ->
``cudaStream_t``, status codes -> exceptions).  All arithmetic runs in the
library's CUDA kernels; there is no CPU fallback -- importing works without a
GPU, but any call that needs the library raises if ``libqex_gpu.so`` is not
built or no CUDA device is present.

Tensors: canonical links are complex128 ``[Lt, Lz, Ly, Lx, 4, 3, 3]`` and
canonical fields complex128 ``[Lt, Lz, Ly, Lx, 3]`` (``fieldgen`` layout);
internal link sets and half fields are flat float64 (F64) or float32 (F32)
tensors of ``qex_links_bytes`` / ``qex_field_bytes`` bytes.
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

F64 = 0
F32 = 1
F32_R12 = 2  # FP32 fields; FP32 SU(3) fat links stored as two rows
F32_R12H = 3  # FP32 fields; SU(3) fat links as two rows of 16-bit fixed point
F32_S16 = 4  # FP32 fields; links (any kind) as 16-bit fixed point with a per-link step
_PREC = {"f64": F64, "f32": F32, "f32r12": F32_R12, "f32r12h": F32_R12H, "f32s16": F32_S16, F64: F64, F32: F32,
         F32_R12: F32_R12, F32_R12H: F32_R12H, F32_S16: F32_S16, torch.float64: F64, torch.float32: F32}
_NAMES = {F64: "f64", F32: "f32", F32_R12: "f32r12", F32_R12H: "f32r12h", F32_S16: "f32s16"}
_DTYPE = {F64: torch.float64, F32: torch.float32, F32_R12: torch.float32, F32_R12H: torch.float32,
          F32_S16: torch.float32}
_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_ALIGN", 4: "ERR_CUDA",
           5: "ERR_NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_NAN"}

_lib = None


class QexError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class CgItem(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_void_p), ("fat64", ctypes.c_void_p), ("lng64", ctypes.c_void_p),
                ("fat32", ctypes.c_void_p), ("lng32", ctypes.c_void_p), ("c_naik", ctypes.c_double),
                ("mass", ctypes.c_double), ("b64", ctypes.c_void_p), ("x64", ctypes.c_void_p)]


class CgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("ff_updates", ctypes.c_int), ("true_rel_resid", ctypes.c_double), ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libqex_gpu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libqex_gpu.so is not built ({_build.LIB}); run paper_1612_02750_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    vp, i, d, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "qex_lattice_create": (i, [ip, i, ctypes.POINTER(vp)]),
        "qex_lattice_destroy": (i, [vp]),
        "qex_volume": (i64, [vp]),
        "qex_half_volume": (i64, [vp]),
        "qex_eo_index": (i64, [vp, ip]),
        "qex_neighbor_table": (i, [vp, i, i, i, vp]),
        "qex_neighbor_table_device": (i, [vp, i, i, i, vp, vp]),
        "qex_links_bytes": (sz, [vp, i]),
        "qex_field_bytes": (sz, [vp, i]),
        "qex_pack_links": (i, [vp, i, vp, vp, vp]),
        "qex_pack_links_pair": (i, [vp, vp, vp, i, vp, vp]),
        "qex_unpack_links": (i, [vp, i, vp, vp, vp]),
        "qex_pack_field": (i, [vp, i, i, vp, vp, vp]),
        "qex_unpack_field": (i, [vp, i, i, vp, vp, vp]),
        "qex_convert_links": (i, [vp, i, vp, i, vp, vp]),
        "qex_convert_field": (i, [vp, i, vp, i, vp, vp]),
        "qex_dslash": (i, [vp, i, vp, vp, d, i, vp, vp, vp]),
        "qex_normal_op": (i, [vp, i, vp, vp, d, d, vp, vp, vp, vp]),
        "qex_norm2": (i, [vp, i, vp, vp, vp]),
        "qex_dot": (i, [vp, i, vp, vp, vp, vp]),
        "qex_cg": (i, [vp, i, vp, vp, vp, vp, d, d, vp, vp, d, i, d, vp, ctypes.POINTER(CgStats)]),
        "qex_cg_host": (i, [vp, i, vp, vp, d, d, vp, vp, d, i, d, vp, ctypes.POINTER(CgStats)]),
        "qex_cg_profile": (i, [vp, i, vp, vp, vp, vp, d, d, vp, vp, i, vp, ctypes.POINTER(d), ip]),
        "qex_force": (i, [vp, vp, vp, d, vp, vp, i, vp, vp, vp]),
        "qex_dslash_mrhs": (i, [vp, i, vp, vp, d, i, i, vp, vp, vp]),
        "qex_cg_mrhs": (i, [vp, i, vp, vp, vp, vp, d, d, i, vp, vp, d, i, d, vp, ctypes.POINTER(CgStats)]),
        "qex_cg_batch": (i, [i, ctypes.POINTER(CgItem), i, d, i, d, vp, ctypes.POINTER(CgStats)]),
        "qex_cg_batch_tune_info": (i, [vp, ip]),
        "qex_cg_batch_tune_set": (i, [vp, i, i]),
        "qex_long_links_prec": (i, [i]),
        "qex_tune": (i, [vp, i, vp, vp, vp]),
        "qex_tune_info": (i, [vp, i, i, ip]),
        "qex_tune_set": (i, [vp, i, i, ip]),
        "qex_fma_rates": (i, [ctypes.POINTER(d), ctypes.POINTER(d), vp]),
        "qex_true_residual": (i, [vp, vp, vp, d, d, vp, vp, i, ctypes.POINTER(d), vp]),
        "qex_launch_count": (ctypes.c_uint64, []),
        "qex_last_error": (ctypes.c_char_p, []),
        "qex_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding wraps."""
    return ["qex_lattice_create", "qex_lattice_destroy", "qex_volume", "qex_half_volume", "qex_eo_index",
            "qex_neighbor_table", "qex_neighbor_table_device", "qex_links_bytes", "qex_field_bytes",
            "qex_pack_links", "qex_pack_links_pair", "qex_unpack_links", "qex_pack_field", "qex_unpack_field",
            "qex_convert_links", "qex_convert_field", "qex_dslash", "qex_normal_op", "qex_norm2", "qex_dot", "qex_cg",
            "qex_cg_host", "qex_cg_profile", "qex_force", "qex_dslash_mrhs", "qex_cg_mrhs", "qex_cg_batch",
            "qex_cg_batch_tune_info", "qex_cg_batch_tune_set", "qex_long_links_prec", "qex_tune", "qex_tune_info",
            "qex_tune_set", "qex_fma_rates", "qex_true_residual", "qex_launch_count", "qex_last_error",
            "qex_version"]


def _check(status: int):
    if status != 0:
        raise QexError(status, load().qex_last_error().decode())


def _prec(p) -> int:
    try:
        return _PREC[p]
    except KeyError:
        raise ValueError(f"unknown precision {p!r}") from None


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Lattice:
    """Owning handle of a ``qex_lattice`` (extents ``dims = (Lx, Ly, Lz, Lt)``)."""

    def __init__(self, dims, antiperiodic: bool = True):
        lib = load()
        self.dims = tuple(int(v) for v in dims)
        self.antiperiodic = bool(antiperiodic)
        h = ctypes.c_void_p()
        _check(lib.qex_lattice_create((ctypes.c_int * 4)(*self.dims), int(antiperiodic), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def volume(self) -> int:
        return int(load().qex_volume(self._h))

    @property
    def half_volume(self) -> int:
        return int(load().qex_half_volume(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().qex_lattice_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ----------------------------------------------------------------- geometry

def qex_lattice_create(dims, antiperiodic: bool = True) -> Lattice:
    return Lattice(dims, antiperiodic)


def qex_lattice_destroy(lat: Lattice) -> None:
    lat.close()


def qex_eo_index(lat: Lattice, coord) -> int:
    return int(load().qex_eo_index(lat.handle, (ctypes.c_int * 4)(*coord)))


def qex_neighbor_table(lat: Lattice, parity: int, mu: int, hop: int):
    import numpy as np

    out = np.empty(lat.half_volume, dtype=np.int32)
    _check(load().qex_neighbor_table(lat.handle, parity, mu, hop, out.ctypes.data))
    return out


def qex_neighbor_table_device(lat: Lattice, parity: int, mu: int, hop: int, out=None, stream=None):
    if out is None:
        out = torch.empty(lat.half_volume, dtype=torch.int32, device="cuda")
    _check(load().qex_neighbor_table_device(lat.handle, parity, mu, hop, _ptr(out), _stream(stream)))
    return out


def qex_links_bytes(lat: Lattice, prec) -> int:
    return int(load().qex_links_bytes(lat.handle, _prec(prec)))


def qex_field_bytes(lat: Lattice, prec) -> int:
    return int(load().qex_field_bytes(lat.handle, _prec(prec)))


def empty_links(lat: Lattice, prec, device="cuda"):
    p = _prec(prec)
    return torch.empty(qex_links_bytes(lat, p) // _DTYPE[p].itemsize, dtype=_DTYPE[p], device=device)


def empty_field(lat: Lattice, prec, device="cuda"):
    p = _prec(prec)
    return torch.empty(qex_field_bytes(lat, p) // _DTYPE[p].itemsize, dtype=_DTYPE[p], device=device)


def zeros_field(lat: Lattice, prec, device="cuda"):
    return empty_field(lat, prec, device).zero_()


# ------------------------------------------------------------------- layout

def qex_pack_links(lat: Lattice, prec, lex_links, out=None, stream=None):
    if lex_links.dtype != torch.complex128:
        raise TypeError("canonical links must be complex128")
    out = empty_links(lat, prec) if out is None else out
    _check(load().qex_pack_links(lat.handle, _prec(prec), _ptr(lex_links), _ptr(out), _stream(stream)))
    return out


def qex_pack_links_pair(lat: Lattice, lex_links, second, out64=None, out2=None, stream=None):
    """Canonical links -> (internal F64 set, internal set of precision
    ``second``) in one pass; returns both."""
    if lex_links.dtype != torch.complex128:
        raise TypeError("canonical links must be complex128")
    out64 = empty_links(lat, "f64") if out64 is None else out64
    out2 = empty_links(lat, second) if out2 is None else out2
    _check(load().qex_pack_links_pair(lat.handle, _ptr(lex_links), _ptr(out64), _prec(second), _ptr(out2),
                                      _stream(stream)))
    return out64, out2


def qex_unpack_links(lat: Lattice, prec, internal, out=None, stream=None):
    if out is None:
        lx, ly, lz, lt = lat.dims
        out = torch.empty((lt, lz, ly, lx, 4, 3, 3), dtype=torch.complex128, device="cuda")
    _check(load().qex_unpack_links(lat.handle, _prec(prec), _ptr(internal), _ptr(out), _stream(stream)))
    return out


def qex_pack_field(lat: Lattice, prec, parity: int, lex_field, out=None, stream=None):
    if lex_field.dtype != torch.complex128:
        raise TypeError("canonical fields must be complex128")
    out = empty_field(lat, prec) if out is None else out
    _check(load().qex_pack_field(lat.handle, _prec(prec), parity, _ptr(lex_field), _ptr(out), _stream(stream)))
    return out


def qex_unpack_field(lat: Lattice, prec, parity: int, half, out=None, stream=None):
    if out is None:
        lx, ly, lz, lt = lat.dims
        out = torch.zeros((lt, lz, ly, lx, 3), dtype=torch.complex128, device="cuda")
    _check(load().qex_unpack_field(lat.handle, _prec(prec), parity, _ptr(half), _ptr(out), _stream(stream)))
    return out


def qex_convert_links(lat: Lattice, src_prec, internal, dst_prec, out=None, stream=None):
    out = empty_links(lat, dst_prec) if out is None else out
    _check(load().qex_convert_links(lat.handle, _prec(src_prec), _ptr(internal), _prec(dst_prec), _ptr(out),
                                    _stream(stream)))
    return out


def qex_convert_field(lat: Lattice, src_prec, half, dst_prec, out=None, stream=None):
    out = empty_field(lat, dst_prec) if out is None else out
    _check(load().qex_convert_field(lat.handle, _prec(src_prec), _ptr(half), _prec(dst_prec), _ptr(out),
                                    _stream(stream)))
    return out


# ----------------------------------------------------------------- operator

def qex_dslash(lat: Lattice, prec, fat, lng, c_naik: float, out_parity: int, inp, out=None, stream=None):
    out = empty_field(lat, prec) if out is None else out
    _check(load().qex_dslash(lat.handle, _prec(prec), _ptr(fat), _ptr(lng), float(c_naik), int(out_parity),
                             _ptr(inp), _ptr(out), _stream(stream)))
    return out


def empty_fields(lat: Lattice, prec, nrhs: int, device="cuda"):
    """nrhs half fields back to back (the multi-RHS layout)."""
    p = _prec(prec)
    n = qex_field_bytes(lat, p) // _DTYPE[p].itemsize
    return torch.empty(nrhs * n, dtype=_DTYPE[p], device=device)


def qex_dslash_mrhs(lat: Lattice, prec, fat, lng, c_naik: float, out_parity: int, nrhs: int, inp, out=None,
                    stream=None):
    out = empty_fields(lat, prec, nrhs) if out is None else out
    _check(load().qex_dslash_mrhs(lat.handle, _prec(prec), _ptr(fat), _ptr(lng), float(c_naik), int(out_parity),
                                  int(nrhs), _ptr(inp), _ptr(out), _stream(stream)))
    return out


def qex_normal_op(lat: Lattice, prec, fat, lng, c_naik: float, mass: float, inp, out=None, tmp_odd=None,
                  stream=None):
    out = empty_field(lat, prec) if out is None else out
    tmp_odd = empty_field(lat, prec) if tmp_odd is None else tmp_odd
    _check(load().qex_normal_op(lat.handle, _prec(prec), _ptr(fat), _ptr(lng), float(c_naik), float(mass),
                                _ptr(inp), _ptr(out), _ptr(tmp_odd), _stream(stream)))
    return out


def qex_normal_op_static(lat: Lattice, prec, fat, lng, c_naik: float, mass: float, inp, out=None, stream=None):
    """(m^2 - D_eo D_oe) inp with the intermediate in the library's static
    device scratch (no allocation inside the call; ``out`` is allocated here
    only when not given)."""
    fn = load().qex_normal_op_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    out = empty_field(lat, prec) if out is None else out
    _check(fn(lat.handle, _prec(prec), _ptr(fat), _ptr(lng), float(c_naik), float(mass), _ptr(inp), _ptr(out),
              _stream(stream)))
    return out


def qex_norm2(lat: Lattice, prec, f, out=None, stream=None):
    out = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
    _check(load().qex_norm2(lat.handle, _prec(prec), _ptr(f), _ptr(out), _stream(stream)))
    return out


def qex_dot(lat: Lattice, prec, a, b, out=None, stream=None):
    out = torch.empty(2, dtype=torch.float64, device="cuda") if out is None else out
    _check(load().qex_dot(lat.handle, _prec(prec), _ptr(a), _ptr(b), _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------ solvers

def qex_cg(lat: Lattice, inner, fat64, lng64, fat32, lng32, c_naik: float, mass: float, b64, x64,
           tol: float = 1e-10, maxiter: int = 100000, delta: float = 0.1, stream=None, check: bool = True):
    """Solve (m^2 - D_eo D_oe) x = b; x64 is the initial guess, overwritten.
    Returns (status, stats dict); raises on error when ``check``."""
    stats = CgStats()
    st = load().qex_cg(lat.handle, _prec(inner), _ptr(fat64), _ptr(lng64), _ptr(fat32), _ptr(lng32),
                       float(c_naik), float(mass), _ptr(b64), _ptr(x64), float(tol), int(maxiter), float(delta),
                       _stream(stream), ctypes.byref(stats))
    if check:
        _check(st)
    return st, stats.as_dict()


def qex_cg_profile(lat: Lattice, inner, fat64, lng64, fat32, lng32, c_naik: float, mass: float, b64, x64,
                   iters: int = 50, stream=None):
    """Average device time (ms) of each kernel of the CG iteration inside a
    solve: a list of 3 (mixed) or 4 (FP64) numbers in launch order."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int(0)
    _check(load().qex_cg_profile(lat.handle, _prec(inner), _ptr(fat64), _ptr(lng64), _ptr(fat32), _ptr(lng32),
                                 float(c_naik), float(mass), _ptr(b64), _ptr(x64), int(iters), _stream(stream), ms,
                                 ctypes.byref(n)))
    return [ms[k] for k in range(n.value)]


def qex_true_residual(lat: Lattice, fat64, lng64, c_naik: float, mass: float, b64, x64, arith: str = "f64",
                      stream=None) -> float:
    """||b - A x|| / ||b|| on the device, in FP64 (arith "f64") or in the
    float-float arithmetic of the intermediate reliable updates ("ff")."""
    if arith not in ("f64", "ff"):
        raise ValueError("arith must be 'f64' or 'ff'")
    out = ctypes.c_double()
    _check(load().qex_true_residual(lat.handle, _ptr(fat64), _ptr(lng64), float(c_naik), float(mass), _ptr(b64),
                                    _ptr(x64), 0 if arith == "f64" else 1, ctypes.byref(out), _stream(stream)))
    return out.value


# -------------------------------------------------------------------- force

def qex_force(lat: Lattice, fat64, lng64, c_naik: float, x_even, y_odd, kind: int = 0, out_fat=None, out_lng=None,
              stream=None):
    """Per-link force (kind 0: F = 2 TA(U G)) or gradient (kind 1: 2 G^+) of
    S = phi^+ A^{-1} phi from X = A^{-1} phi and Y = D_oe X; internal F64
    link sets.  Returns (out_fat, out_lng or None)."""
    out_fat = empty_links(lat, "f64") if out_fat is None else out_fat
    if lng64 is not None and out_lng is None:
        out_lng = empty_links(lat, "f64")
    _check(load().qex_force(lat.handle, _ptr(fat64), _ptr(lng64), float(c_naik), _ptr(x_even), _ptr(y_odd),
                            int(kind), _ptr(out_fat), _ptr(out_lng) if lng64 is not None else None,
                            _stream(stream)))
    return out_fat, (out_lng if lng64 is not None else None)


class StaggeredAction(torch.autograd.Function):
    """S = Re phi^+ (m^2 - D_eo D_oe)^{-1} phi as a differentiable function of
    the canonical complex128 links U (and long links W).

    forward(U, W, phi, lat, mass, c_naik, inner, tol, delta): phi is a
    canonical complex128 field whose even sites are the pseudofermion (held
    fixed); inner = "f64" or a mixed precision ("f32", "f32r12", "f32r12h",
    "f32s16"; the two-row formats need SU(3) fat links).  The inner copies
    are converted from the FP64 links: the fat links to ``inner``, the long
    links to ``qex_long_links_prec(inner)``.  The solve is qex_cg; the
    backward pass is qex_dslash (Y = D_oe X) and qex_force (kind 1),
    unpacked to canonical links: grad_U = 2 G^+ times the incoming gradient
    (torch's convention for a real loss of complex inputs)."""

    @staticmethod
    def forward(ctx, U, W, phi, lat, mass, c_naik=0.0, inner="f64", tol=1e-12, delta=0.01):
        p = _prec(inner)  # raises ValueError for an unknown format
        if p not in _NAMES:
            raise ValueError(f"unknown inner precision {inner!r}")
        fat64 = qex_pack_links(lat, "f64", U.detach().contiguous())
        lng64 = qex_pack_links(lat, "f64", W.detach().contiguous()) if W is not None else None
        fat32 = lng32 = None
        if p != F64:
            fat32 = qex_convert_links(lat, "f64", fat64, p)
            if lng64 is not None:
                lng32 = qex_convert_links(lat, "f64", lng64, qex_long_links_prec(p))
        b = qex_pack_field(lat, "f64", 0, phi.detach().contiguous())
        x = torch.zeros_like(b)
        qex_cg(lat, p, fat64, lng64, fat32, lng32, c_naik, mass, b, x, tol=tol, delta=delta)
        s = qex_dot(lat, "f64", b, x)[0]
        ctx.lat, ctx.c_naik = lat, c_naik
        ctx.has_w = W is not None
        ctx.save_for_backward(fat64, lng64 if lng64 is not None else fat64, x)
        return s.clone()

    @staticmethod
    def backward(ctx, grad_out):
        fat64, lng64, x = ctx.saved_tensors
        lat = ctx.lat
        lng64 = lng64 if ctx.has_w else None
        y = qex_dslash(lat, "f64", fat64, lng64, ctx.c_naik, 1, x)
        gf, gl = qex_force(lat, fat64, lng64, ctx.c_naik, x, y, kind=1)
        gU = qex_unpack_links(lat, "f64", gf) * grad_out
        gW = qex_unpack_links(lat, "f64", gl) * grad_out if gl is not None else None
        return gU, gW, None, None, None, None, None, None, None


def _host_ptr(t, dtype):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"host tensor must be contiguous {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def qex_cg_host(lat: Lattice, inner, host_fat, host_lng, c_naik: float, mass: float, host_b, host_x=None,
                tol: float = 1e-10, maxiter: int = 100000, delta: float = 0.1, stream=None, check: bool = True):
    """End-to-end solve from host tensors (canonical complex128 links and
    fields; pinned memory for asynchronous copies).  Returns (host_x, status,
    stats dict)."""
    if host_x is None:
        host_x = torch.empty_like(host_b)
    stats = CgStats()
    st = load().qex_cg_host(lat.handle, _prec(inner), _host_ptr(host_fat, torch.complex128),
                            None if host_lng is None else _host_ptr(host_lng, torch.complex128), float(c_naik),
                            float(mass), _host_ptr(host_b, torch.complex128), _host_ptr(host_x, torch.complex128),
                            float(tol), int(maxiter), float(delta), _stream(stream), ctypes.byref(stats))
    if check:
        _check(st)
    return host_x, st, stats.as_dict()


def qex_long_links_prec(prec) -> str:
    """Name of the long-link format an operator of precision ``prec`` reads."""
    return _NAMES[int(load().qex_long_links_prec(_prec(prec)))]


def qex_tune(lat: Lattice, prec, fat, lng=None, stream=None):
    """Time the launch shapes for (lat, prec, Naik iff lng) and keep the best."""
    _check(load().qex_tune(lat.handle, _prec(prec), _ptr(fat), _ptr(lng), _stream(stream)))


def qex_tune_info(lat: Lattice, prec, naik: bool = False) -> dict:
    """Launch shapes in use for (lat, prec, naik)."""
    out = (ctypes.c_int * 6)()
    _check(load().qex_tune_info(lat.handle, _prec(prec), 1 if naik else 0, out))
    src = {0: "default", 1: "measured", 2: "cache", 3: "disabled", 4: "set"}
    return {"dslash_block": out[0], "reduce_block": out[1], "reduce_blocks_per_sm": out[2],
            "blas_blocks_per_sm": out[3], "source": src.get(out[4], str(out[4])), "dslash_waves": out[5]}


def qex_tune_set(lat: Lattice, prec, naik: bool = False, dslash_block: int = 256, reduce_block: int = 256,
                 reduce_blocks_per_sm: int = 4, blas_blocks_per_sm: int = 0, dslash_waves: int = 0) -> None:
    """Pin the launch shapes for (lat, prec, naik) (see qex_tune_info for the
    fields)."""
    arr = (ctypes.c_int * 5)(dslash_block, reduce_block, reduce_blocks_per_sm, blas_blocks_per_sm, dslash_waves)
    _check(load().qex_tune_set(lat.handle, _prec(prec), 1 if naik else 0, arr))


def qex_fma_rates(stream=None) -> dict:
    """Measured FP64 and FP32 FMA rates of the current GPU (GFLOP/s)."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    _check(load().qex_fma_rates(ctypes.byref(f64), ctypes.byref(f32), _stream(stream)))
    return {"fp64_gflops": f64.value, "fp32_gflops": f32.value}


def qex_launch_count() -> int:
    return int(load().qex_launch_count())


def qex_cg_mrhs(lat: Lattice, inner, fat64, lng64, fat32, lng32, c_naik: float, mass: float, nrhs: int, b64, x64,
                tol: float = 1e-10, maxiter: int = 100000, delta: float = 0.1, stream=None, check: bool = True):
    """Multi-RHS solve; b64/x64 hold nrhs F64 even half fields back to back.
    Returns (status, list of per-RHS stats dicts)."""
    stats = (CgStats * int(nrhs))()
    st = load().qex_cg_mrhs(lat.handle, _prec(inner), _ptr(fat64), _ptr(lng64), _ptr(fat32), _ptr(lng32),
                            float(c_naik), float(mass), int(nrhs), _ptr(b64), _ptr(x64), float(tol), int(maxiter),
                            float(delta), _stream(stream), stats)
    if check:
        _check(st)
    return st, [stats[k].as_dict() for k in range(int(nrhs))]


def qex_cg_batch(items, inner, tol: float = 1e-10, maxiter: int = 100000, delta: float = 0.1, stream=None,
                 check: bool = True):
    """Batched solve over independent lattices.  ``items`` is a list of dicts
    with keys lat, fat64, lng64, fat32, lng32, c_naik, mass, b64, x64 (x64 is
    overwritten).  Returns (status, list of per-item stats dicts)."""
    n = len(items)
    arr = (CgItem * n)()
    for k, it in enumerate(items):
        arr[k].lat = it["lat"].handle
        arr[k].fat64 = _ptr(it["fat64"])
        arr[k].lng64 = _ptr(it.get("lng64"))
        arr[k].fat32 = _ptr(it.get("fat32"))
        arr[k].lng32 = _ptr(it.get("lng32"))
        arr[k].c_naik = float(it.get("c_naik", 0.0))
        arr[k].mass = float(it["mass"])
        arr[k].b64 = _ptr(it["b64"])
        arr[k].x64 = _ptr(it["x64"])
    stats = (CgStats * n)()
    st = load().qex_cg_batch(n, arr, _prec(inner), float(tol), int(maxiter), float(delta), _stream(stream), stats)
    if check:
        _check(st)
    return st, [stats[k].as_dict() for k in range(n)]


def qex_cg_batch_tune_info(lead: Lattice) -> dict:
    """Launch shape of the last batch led by ``lead`` (see the C header)."""
    out = (ctypes.c_int * 3)()
    _check(load().qex_cg_batch_tune_info(lead.handle, out))
    src = {0: "none", 1: "measured", 2: "cache", 3: "disabled", 4: "set"}
    return {"blocks_per_sm": out[0], "groups_per_item": out[1], "source": src.get(out[2], str(out[2]))}


def qex_cg_batch_tune_set(lead: Lattice, blocks_per_sm: int, groups_per_item: int) -> None:
    """Pin the batch launch shape for batches led by ``lead`` ((0, 0) unpins)."""
    _check(load().qex_cg_batch_tune_set(lead.handle, int(blocks_per_sm), int(groups_per_item)))


def qex_last_error() -> str:
    return load().qex_last_error().decode()


def qex_version() -> str:
    return load().qex_version().decode()
