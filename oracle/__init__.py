"""Plain FP64 CPU oracle for the staggered Dirac operator, CG and the force.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the product path never imports it.
It shares no code with the CUDA path.

The arithmetic lives in ``qex_oracle.c`` (plain C, lexicographic loops,
complex double), compiled by :func:`build` with gcc into ``_build/``.  This
module only marshals numpy arrays in the canonical layouts of ``fieldgen``:
links ``[Lt, Lz, Ly, Lx, 4, 3, 3]``, fields ``[Lt, Lz, Ly, Lx, 3]``, complex128,
``dims = (Lx, Ly, Lz, Lt)``.  The few numpy-level helpers here (dense matrix
of the normal operator, free-field eigenvalues) are written out from their
definitions.  Every function names what it follows; parity-unpinned functions
are marked as such.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the C oracle with gcc (OpenMP site loops, no FMA contraction).
    ``src``/``out`` compile another copy of the source with the same flags
    (the pin tests build deliberately broken copies this way)."""
    src = src or os.path.join(_HERE, "qex_oracle.c")
    so = out or _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fcx-limited-range", src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, so)
    return so


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i4 = ctypes.POINTER(ctypes.c_int)
        vp = ctypes.c_void_p
        d = ctypes.c_double
        lib.oracle_volume.restype = ctypes.c_int64
        lib.oracle_volume.argtypes = [i4]
        lib.oracle_eo_table.argtypes = [i4, vp]
        lib.oracle_neighbor_table.argtypes = [i4, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.oracle_dslash.argtypes = [i4, ctypes.c_int, vp, vp, d, vp, vp]
        lib.oracle_dslash_parity.argtypes = [i4, ctypes.c_int, vp, vp, d, ctypes.c_int, vp, vp]
        lib.oracle_dslash_sites.argtypes = [i4, ctypes.c_int, vp, vp, d, vp, vp, ctypes.c_int64, vp]
        lib.oracle_normal_op.argtypes = [i4, ctypes.c_int, vp, vp, d, d, vp, vp]
        lib.oracle_true_residual.restype = d
        lib.oracle_true_residual.argtypes = [i4, ctypes.c_int, vp, vp, d, d, vp, vp]
        lib.oracle_cg.restype = ctypes.c_int
        lib.oracle_cg.argtypes = [i4, ctypes.c_int, vp, vp, d, d, vp, vp, d, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        lib.oracle_force.argtypes = [i4, ctypes.c_int, vp, vp, d, vp, vp, ctypes.c_int, vp, vp]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _dims(dims):
    lx, ly, lz, lt = (int(v) for v in dims)
    for v in (lx, ly, lz, lt):
        if v < 2 or v % 2:
            raise ValueError("lattice extents must be even and >= 2")
    return (ctypes.c_int * 4)(lx, ly, lz, lt)


def _shape(dims):
    return (int(dims[3]), int(dims[2]), int(dims[1]), int(dims[0]))


def _cfield(a, dims):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != _shape(dims) + (3,):
        raise ValueError(f"field shape {a.shape} != {_shape(dims) + (3,)}")
    return a


def _clinks(u, dims):
    if u is None:
        return None
    u = np.ascontiguousarray(u, dtype=np.complex128)
    if u.shape != _shape(dims) + (4, 3, 3):
        raise ValueError(f"link shape {u.shape} != {_shape(dims) + (4, 3, 3)}")
    return u


def _ptr(a):
    return None if a is None else a.ctypes.data


def threads() -> int:
    """OpenMP threads the oracle's site loops use (OMP_NUM_THREADS)."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's later site loops (timing only)."""
    _load().oracle_set_threads(int(n))


def eo_table(dims) -> np.ndarray:
    """eo[lex] = parity * V/2 + rank of the site within its parity (lex order)."""
    L = _dims(dims)
    V = int(np.prod(dims))
    out = np.empty(V, dtype=np.int32)
    _load().oracle_eo_table(L, out.ctypes.data)
    return out


def neighbor_table(dims, parity: int, mu: int, hop: int) -> np.ndarray:
    """Rank (within its parity) of x + hop mu_hat for every site x of ``parity``."""
    L = _dims(dims)
    vh = int(np.prod(dims)) // 2
    out = np.empty(vh, dtype=np.int32)
    _load().oracle_neighbor_table(L, int(parity), int(mu), int(hop), out.ctypes.data)
    return out


def dslash(dims, u, psi, w=None, c3: float = 0.0, antiperiodic: bool = True) -> np.ndarray:
    """Full-lattice staggered operator D psi (one-hop plus optional Naik term)."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    psi = _cfield(psi, dims)
    out = np.empty_like(psi)
    _load().oracle_dslash(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3), _ptr(psi), _ptr(out))
    return out


def dslash_sites(dims, u, psi, sites, w=None, c3: float = 0.0, antiperiodic: bool = True) -> np.ndarray:
    """(D psi) at the sites of lexicographic index ``sites`` (shape [n, 3]);
    the same per-site sum as :func:`dslash`, for sampled checks of large
    lattices."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    psi = _cfield(psi, dims)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((sites.size, 3), dtype=np.complex128)
    _load().oracle_dslash_sites(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3), _ptr(psi), sites.ctypes.data,
                                int(sites.size), out.ctypes.data)
    return out


def dslash_parity(dims, u, psi, out_parity: int, w=None, c3: float = 0.0,
                  antiperiodic: bool = True) -> np.ndarray:
    """D_{p,1-p}: input restricted to parity 1-p, output at parity p (zero elsewhere)."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    psi = _cfield(psi, dims)
    out = np.empty_like(psi)
    _load().oracle_dslash_parity(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3),
                                 int(out_parity), _ptr(psi), _ptr(out))
    return out


def normal_op(dims, u, x, mass: float, w=None, c3: float = 0.0,
              antiperiodic: bool = True) -> np.ndarray:
    """A x = (m^2 - D_eo D_oe) x on even sites (odd sites of the result are zero)."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    x = _cfield(x, dims)
    out = np.empty_like(x)
    _load().oracle_normal_op(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3), float(mass),
                             _ptr(x), _ptr(out))
    return out


def true_residual(dims, u, b, x, mass: float, w=None, c3: float = 0.0,
                  antiperiodic: bool = True) -> float:
    """||b - A x|| / ||b|| over even sites, in FP64."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    b = _cfield(b, dims)
    x = _cfield(x, dims)
    return float(_load().oracle_true_residual(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3),
                                              float(mass), _ptr(b), _ptr(x)))


def cg(dims, u, b, mass: float, w=None, c3: float = 0.0, tol: float = 1e-10, maxiter: int = 10000,
       x0=None, antiperiodic: bool = True):
    """Textbook CG on A x = b (even sites).  Returns (x, converged, iters, true_rel)."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    b = _cfield(b, dims)
    x = np.zeros_like(b) if x0 is None else _cfield(x0, dims).copy()
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    rc = _load().oracle_cg(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3), float(mass), _ptr(b),
                           _ptr(x), float(tol), int(maxiter), ctypes.byref(it), ctypes.byref(tr))
    return x, rc == 0, int(it.value), float(tr.value)


def force(dims, u, x_even, y_odd, w=None, c3: float = 0.0, kind: int = 0, antiperiodic: bool = True):
    """Per-link force of S = phi^+ A^{-1} phi from X = A^{-1} phi (even sites)
    and Y = D_oe X (odd sites): kind 0 gives F = 2 TA(U G), kind 1 gives 2 G^+
    (the gradient of the real S with respect to the complex link entries).
    Returns (F_fat, F_long or None) in the links layout."""
    L = _dims(dims)
    u = _clinks(u, dims)
    w = _clinks(w, dims)
    x = _cfield(x_even, dims)
    y = _cfield(y_odd, dims)
    ff = np.empty_like(u)
    fl = np.empty_like(w) if w is not None else None
    _load().oracle_force(L, int(antiperiodic), _ptr(u), _ptr(w), float(c3), _ptr(x), _ptr(y), int(kind), _ptr(ff),
                         _ptr(fl))
    return ff, fl


def pseudofermion(dims, u, chi, mass: float, w=None, c3: float = 0.0, antiperiodic: bool = True):
    """phi = (M^+ chi) on even sites, M = m + D: phi_e = m chi_e - D_eo chi_o."""
    ev = even_sites(dims)
    dch = dslash_parity(dims, u, chi, 0, w, c3, antiperiodic)
    phi = mass * chi - dch
    phi[~ev] = 0
    return phi


def action(dims, u, phi, mass: float, w=None, c3: float = 0.0, tol: float = 1e-13, antiperiodic: bool = True):
    """S = Re phi^+ A^{-1} phi by the oracle's CG; returns (S, X)."""
    x, ok, _, _ = cg(dims, u, phi, mass, w, c3, tol=tol, maxiter=200000, antiperiodic=antiperiodic)
    if not ok:
        raise RuntimeError("oracle CG did not converge")
    return float(np.vdot(phi, x).real), x


# ----------------------------------------------------------------- numpy helpers

def even_sites(dims) -> np.ndarray:
    """Boolean [Lt, Lz, Ly, Lx] mask of even sites (x+y+z+t even)."""
    t, z, y, x = np.indices(_shape(dims))
    return ((x + y + z + t) & 1) == 0


def dense_normal_op(dims, u, mass: float, w=None, c3: float = 0.0,
                    antiperiodic: bool = True) -> np.ndarray:
    """Dense matrix of A on the even-site subspace, built column by column by
    applying :func:`normal_op` to unit vectors (tiny lattices only)."""
    ev = even_sites(dims)
    idx = np.flatnonzero(ev.reshape(-1))
    n = idx.size * 3
    cols = []
    for k in range(n):
        e = np.zeros(_shape(dims) + (3,), dtype=np.complex128)
        e.reshape(-1, 3)[idx[k // 3], k % 3] = 1.0
        cols.append(normal_op(dims, u, e, mass, w, c3, antiperiodic).reshape(-1, 3)[idx].reshape(-1))
    return np.stack(cols, axis=1)


def free_eigenvalue(dims, n, mass: float, c3: float = 0.0, antiperiodic: bool = True) -> float:
    """Eigenvalue of A on unit links for the plane wave of integer momentum
    ``n = (nx, ny, nz, nt)`` restricted to even sites:
    m^2 + sum_mu (2 sin p_mu + 2 c3 sin 3 p_mu)^2, p_mu = 2 pi n_mu / L_mu, with
    n_t shifted by 1/2 for antiperiodic time (closed form; see tests)."""
    lam = mass * mass
    for mu in range(4):
        shift = 0.5 if (mu == 3 and antiperiodic) else 0.0
        p = 2 * np.pi * (n[mu] + shift) / dims[mu]
        lam += (2 * np.sin(p) + 2 * c3 * np.sin(3 * p)) ** 2
    return float(lam)


def plane_wave(dims, n, colour, antiperiodic: bool = True) -> np.ndarray:
    """e^{i p.x} e_colour on every site, momenta as in :func:`free_eigenvalue`."""
    t, z, y, x = np.indices(_shape(dims))
    coords = (x, y, z, t)
    phase = np.zeros(_shape(dims))
    for mu in range(4):
        shift = 0.5 if (mu == 3 and antiperiodic) else 0.0
        phase = phase + 2 * np.pi * (n[mu] + shift) / dims[mu] * coords[mu]
    out = np.zeros(_shape(dims) + (3,), dtype=np.complex128)
    out[..., colour] = np.exp(1j * phase)
    return out
