"""Seeded synthetic inputs for the staggered-fermion workloads.

This module only draws random numbers and builds the random input matrices
and vectors (gauge links, long links, sources, gauge transformations, su(3)
directions).  It holds none of the Dirac operator's arithmetic.  The CPU
oracle's tests and the CUDA path's tests and benchmark both take their inputs
from here, so that both sides see identical inputs for a given seed.

Canonical (external) layouts, numpy complex128, C order, x fastest:

* links  ``[Lt, Lz, Ly, Lx, 4, 3, 3]``: ``U[t, z, y, x, mu, a, b] = U_mu(x)_ab``,
  ``mu = 0:x, 1:y, 2:z, 3:t``; the link joins x to x + mu_hat.
* fields ``[Lt, Lz, Ly, Lx, 3]``: colour vector at each site.

Lattice extents are passed as ``dims = (Lx, Ly, Lz, Lt)``.

Random streams: ``numpy.random.Generator(PCG64)`` children of
``SeedSequence(seed)``, one named child per input kind (see ``STREAMS``), each
filled in lexicographic site order.
"""

from __future__ import annotations

import numpy as np

STREAMS = ("links", "long_links", "source", "chi", "directions", "gauge")


def rng_streams(seed: int) -> dict:
    """One independent generator per input kind, spawned from ``seed``."""
    children = np.random.SeedSequence(seed).spawn(len(STREAMS))
    return {name: np.random.Generator(np.random.PCG64(c)) for name, c in zip(STREAMS, children)}


def lattice_shape(dims) -> tuple:
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def complex_gaussian(rng, shape, scale: float = 1.0) -> np.ndarray:
    """Independent N(0,1) real and imaginary parts, times ``scale``."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    out = np.empty(shape, dtype=np.complex128)
    out.real = re * scale
    out.imag = im * scale
    return out


def _unimodular(q: np.ndarray) -> np.ndarray:
    """Divide a stack of unitary 3x3 matrices by the principal cube root of det."""
    det = np.linalg.det(q)
    theta = np.angle(det)
    return q * np.exp(-1j * theta / 3.0)[..., None, None]


def haar_su3(rng, shape) -> np.ndarray:
    """Haar-random SU(3) matrices, stacked over ``shape``.

    A 3x3 complex Gaussian matrix is orthonormalised column by column
    (modified Gram-Schmidt, with a second projection pass so that rounding
    does not spoil orthogonality for ill-conditioned draws).  That equals the
    QR factor Q with R's diagonal made real positive, i.e. Mezzadri's
    phase-fixed QR, which is Haar on U(3); the determinant phase is then
    removed with the principal cube root.
    """
    z = complex_gaussian(rng, tuple(shape) + (3, 3), 1.0 / np.sqrt(2.0))
    cols = [z[..., :, k].copy() for k in range(3)]
    for k in range(3):
        for _ in range(2):
            for j in range(k):
                proj = np.sum(np.conj(cols[j]) * cols[k], axis=-1)
                cols[k] -= proj[..., None] * cols[j]
        nrm = np.sqrt(np.sum(np.abs(cols[k]) ** 2, axis=-1))
        cols[k] /= nrm[..., None]
    q = np.stack(cols, axis=-1)
    return _unimodular(q)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def su3_algebra(rng, shape) -> np.ndarray:
    """Hermitian traceless H = sum_a h_a lambda_a / 2 with h_a ~ N(0,1)."""
    h = rng.standard_normal(tuple(shape) + (8,))
    return np.einsum("...a,aij->...ij", h, gell_mann() / 2.0)


def exp_i_su3(rng, shape, a: float) -> np.ndarray:
    """SU(3) matrices exp(i a H), H from ``su3_algebra``, via Hermitian eigh."""
    h = su3_algebra(rng, shape)
    w, v = np.linalg.eigh(h)
    return _unimodular(np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * a * w), np.conj(v)))


def unit_links(dims) -> np.ndarray:
    u = np.zeros(lattice_shape(dims) + (4, 3, 3), dtype=np.complex128)
    u[..., :, :, :] = np.eye(3)
    return u


def gaussian_field(rng, dims) -> np.ndarray:
    """Colour-vector field with N(0,1) real and imaginary parts at every site."""
    return complex_gaussian(rng, lattice_shape(dims) + (3,))


def even_mask(dims) -> np.ndarray:
    """Boolean [Lt, Lz, Ly, Lx] mask of sites with even x+y+z+t."""
    t, z, y, x = np.indices(lattice_shape(dims))
    return ((x + y + z + t) & 1) == 0


def random_links(dims, kind: str, rng, a: float = 0.3) -> np.ndarray:
    """Link field of one of the workload kinds.

    ``haar``: Haar SU(3); ``exp``: exp(i a H); ``gauss3``: complex Gaussian
    entries / sqrt(3) (non-unitary long links); ``unit``: identity links.
    """
    return _draw_links(lattice_shape(dims) + (4,), kind, rng, a)


def _draw_links(shape, kind: str, rng, a: float) -> np.ndarray:
    if kind == "unit":
        out = np.zeros(tuple(shape) + (3, 3), dtype=np.complex128)
        out[...] = np.eye(3)
        return out
    if kind == "haar":
        return haar_su3(rng, shape)
    if kind == "exp":
        return exp_i_su3(rng, shape, a)
    if kind == "gauss3":
        return complex_gaussian(rng, tuple(shape) + (3, 3), 1.0 / np.sqrt(3.0))
    raise ValueError(f"unknown link kind {kind!r}")


def gauge_transform(rng, dims) -> np.ndarray:
    """Haar SU(3) matrix g(x) at every site, shape [Lt, Lz, Ly, Lx, 3, 3]."""
    return haar_su3(rng, lattice_shape(dims))


def workload(name: str) -> dict:
    """Synthetic inputs of the named workload (lattice, links, source, mass).

    ``cfg4x4``: 4^4, Haar links, m = 0.1, one Gaussian source on even sites,
    seed 1.  ``cfg32``: 32^4, links exp(i 0.3 H), m = 0.01, seed 2.
    ``cfg64naik``: 64^4 with Naik, Haar fat links, Gaussian/sqrt(3) long links,
    c_naik = -1/24, m = 0.005, seed 3.  ``cfg16force``: 16^4, exp(i 0.5 H),
    m = 0.05, seed 5.
    """
    table = {
        "cfg4x4": dict(dims=(4, 4, 4, 4), fat="haar", a=0.0, naik=False, mass=0.1, seed=1),
        "cfg32": dict(dims=(32, 32, 32, 32), fat="exp", a=0.3, naik=False, mass=0.01, seed=2),
        "cfg64naik": dict(dims=(64, 64, 64, 64), fat="haar", a=0.0, naik=True, mass=0.005, seed=3),
        "cfg16force": dict(dims=(16, 16, 16, 16), fat="exp", a=0.5, naik=False, mass=0.05, seed=5),
    }
    return dict(table[name])


def make_inputs(dims, fat: str = "haar", naik: bool = False, seed: int = 1, a: float = 0.3):
    """Links, optional long links and an even-site Gaussian source.

    Returns ``(fat_links, long_links_or_None, source)``; the source is zero on
    odd sites.
    """
    s = rng_streams(seed)
    u = random_links(dims, fat, s["links"], a)
    w = random_links(dims, "gauss3", s["long_links"]) if naik else None
    b = gaussian_field(s["source"], dims)
    b[~even_mask(dims)] = 0
    return u, w, b


def make_inputs_sliced(dims, fat: str = "haar", naik: bool = False, seed: int = 1, a: float = 0.3):
    """As :func:`make_inputs`, but every input is drawn one t-slice at a time
    (bounded temporary host memory for large lattices such as 64^4).  The
    values differ from :func:`make_inputs`' for the same seed."""
    s = rng_streams(seed)
    shp = lattice_shape(dims)
    u = np.empty(shp + (4, 3, 3), dtype=np.complex128)
    w = np.empty(shp + (4, 3, 3), dtype=np.complex128) if naik else None
    sl = (1,) + shp[1:] + (4,)
    for t in range(shp[0]):
        u[t] = _draw_links(sl, fat, s["links"], a)[0]
        if naik:
            w[t] = _draw_links(sl, "gauss3", s["long_links"], a)[0]
    b = np.empty(shp + (3,), dtype=np.complex128)
    for t in range(shp[0]):
        b[t] = complex_gaussian(s["source"], (1,) + shp[1:] + (3,))[0]
    b[~even_mask(dims)] = 0
    return u, w, b
