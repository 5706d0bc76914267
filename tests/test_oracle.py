"""Pins of the CPU oracle against facts the mathematics fixes (no GPU).

The paper (Sec. 4) names the staggered Dirac operator with the Naik term and
the CG solver but prints no formula and no worked example, so the oracle is
pinned by properties that hold for the operator whatever the links are, by
closed forms on unit links, by hand-derived point-source values and by dense
linear algebra on tiny lattices.  Each test says which plausible mistake it
catches.
"""

import os

import numpy as np
import pytest

import fieldgen as fg

C3 = -1.0 / 24.0
SHAPES = [(4, 4, 4, 4), (6, 4, 2, 8), (4, 6, 4, 4)]


def _site_coords(dims):
    """Coordinates (x, y, z, t) of every site, lexicographic order, x fastest."""
    t, z, y, x = np.indices(fg.lattice_shape(dims))
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


# --------------------------------------------------------------------- geometry

@pytest.mark.parametrize("dims", SHAPES + [(2, 2, 2, 2), (8, 4, 6, 2)])
def test_eo_table_is_parity_ordered_bijection(oracle_mod, dims):
    """Even sites come first, each parity keeps lexicographic order, and the
    map is a permutation of [0, V) (catches an off-by-one in the rank)."""
    eo = oracle_mod.eo_table(dims)
    V = int(np.prod(dims))
    assert sorted(eo.tolist()) == list(range(V))
    par = _site_coords(dims).sum(axis=1) % 2
    assert np.all(eo[par == 0] < V // 2) and np.all(eo[par == 1] >= V // 2)
    for p in (0, 1):
        assert np.all(np.diff(eo[par == p]) == 1)


@pytest.mark.parametrize("dims", SHAPES)
def test_neighbor_tables_invariants(oracle_mod, dims):
    """Forward then backward hop is the identity, tables are permutations,
    a 3-hop is three 1-hops, hops along different axes commute, and L_mu hops
    come back to the start (catches wrong strides and wrong wrap-around)."""
    vh = int(np.prod(dims)) // 2
    ident = np.arange(vh)
    nb = {(p, mu, h): oracle_mod.neighbor_table(dims, p, mu, h)
          for p in (0, 1) for mu in range(4) for h in (1, -1, 3, -3)}
    for p in (0, 1):
        for mu in range(4):
            f = nb[(p, mu, 1)]
            assert sorted(f.tolist()) == ident.tolist()
            assert np.array_equal(nb[(1 - p, mu, -1)][f], ident)
            three = nb[(p, mu, 1)]
            three = nb[(1 - p, mu, 1)][three]
            three = nb[(p, mu, 1)][three]
            assert np.array_equal(three, nb[(p, mu, 3)])
            cur, q = ident.copy(), p
            for _ in range(dims[mu]):
                cur, q = nb[(q, mu, 1)][cur], 1 - q
            assert q == p and np.array_equal(cur, ident)
            for nu in range(mu + 1, 4):
                a = nb[(1 - p, nu, 1)][nb[(p, mu, 1)]]
                b = nb[(1 - p, mu, 1)][nb[(p, nu, 1)]]
                assert np.array_equal(a, b)


def test_neighbor_table_hand_example(oracle_mod):
    """On 4^4 the origin is even rank 0; its +x neighbour (1,0,0,0) is odd
    rank 0, its -x neighbour (3,0,0,0) is odd rank 1, its +y neighbour
    (0,1,0,0) has lex 4 and is odd rank 2, its +t neighbour (0,0,0,1) has lex
    64 and odd rank 32."""
    d = (4, 4, 4, 4)
    assert oracle_mod.neighbor_table(d, 0, 0, 1)[0] == 0
    assert oracle_mod.neighbor_table(d, 0, 0, -1)[0] == 1
    assert oracle_mod.neighbor_table(d, 0, 1, 1)[0] == 2
    assert oracle_mod.neighbor_table(d, 0, 3, 1)[0] == 32


# --------------------------------------------------------------------- operator

def _rand_links(rng, dims):
    """Non-unitary links: the properties below hold for any links."""
    return fg.complex_gaussian(rng, fg.lattice_shape(dims) + (4, 3, 3))


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_antihermitian(oracle_mod, dims, naik, antiperiodic):
    """<chi, D psi> = -<D chi, psi> for arbitrary (even non-unitary) links:
    catches a wrong sign of the backward hop, a missing conjugate or a
    transposed instead of adjoint link, and a sign placed on one hop
    direction only."""
    s = fg.rng_streams(11)
    u = _rand_links(s["links"], dims)
    w = _rand_links(s["long_links"], dims) if naik else None
    psi = fg.gaussian_field(s["source"], dims)
    chi = fg.gaussian_field(s["chi"], dims)
    lhs = np.vdot(chi, oracle_mod.dslash(dims, u, psi, w, C3, antiperiodic))
    rhs = -np.vdot(oracle_mod.dslash(dims, u, chi, w, C3, antiperiodic), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_dslash_at_sampled_sites_equals_full_lattice(oracle_mod):
    """The sampled-site evaluation is the full-lattice sum restricted to the
    listed sites (bit-identical)."""
    dims = (8, 4, 6, 8)
    s = fg.rng_streams(14)
    u = _rand_links(s["links"], dims)
    w = _rand_links(s["long_links"], dims)
    psi = fg.gaussian_field(s["source"], dims)
    full = oracle_mod.dslash(dims, u, psi, w, C3, True).reshape(-1, 3)
    sites = np.array([0, 1, 7, 100, 767, 1535, 900], dtype=np.int64)
    assert np.array_equal(oracle_mod.dslash_sites(dims, u, psi, sites, w, C3, True), full[sites])


@pytest.mark.parametrize("naik", [False, True])
def test_gauge_covariance(oracle_mod, naik):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^+, W_mu(x) -> g(x) W_mu(x) g(x+3mu)^+,
    psi -> g psi gives D psi -> g D psi: catches a link read at the wrong site
    (U(x) instead of U(x-mu)) or a hop of the wrong length."""
    dims = (8, 4, 6, 8)
    s = fg.rng_streams(12)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    psi = fg.gaussian_field(s["source"], dims)
    g = fg.gauge_transform(s["gauge"], dims)  # [t, z, y, x, 3, 3]
    axes = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> array axis of [t, z, y, x]

    def transform(links, k):
        out = np.empty_like(links)
        for mu in range(4):
            gs = np.roll(g, -k, axis=axes[mu])  # g(x + k mu)
            out[..., mu, :, :] = g @ links[..., mu, :, :] @ np.conj(np.swapaxes(gs, -1, -2))
        return out

    u2 = transform(u, 1)
    w2 = transform(w, 3) if naik else None
    psi2 = np.einsum("...ab,...b->...a", g, psi)
    for ap in (False, True):
        d1 = oracle_mod.dslash(dims, u, psi, w, C3, ap)
        d2 = oracle_mod.dslash(dims, u2, psi2, w2, C3, ap)
        expect = np.einsum("...ab,...b->...a", g, d1)
        assert np.linalg.norm(d2 - expect) <= 1e-13 * np.linalg.norm(expect)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_point_source_golden():
    """Hand-derived D psi for a point source on unit links (8^4, antiperiodic
    time, colour 2 at (1,0,0,0)): {"one": {(x,y,z,t): v}, "three": {...}}."""
    out = {"one": {}, "three": {}}
    with open(os.path.join(GOLDEN, "point_source_unit_links_8x8x8x8.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            x, y, z, t = (int(v) for v in line[:4])
            out[line[4]][(x, y, z, t)] = int(line[5])
    return out


POINT = read_point_source_golden()
POINT_ONE_HOP, POINT_THREE_HOP = POINT["one"], POINT["three"]


@pytest.mark.parametrize("naik", [False, True])
def test_point_source_hand_values(oracle_mod, naik):
    """Fixes the conventions the invariants leave open: the eta ordering
    (x, y, z, t with eta_mu from the coordinates before mu), the sign of the
    forward term and the link that carries the antiperiodic sign."""
    assert len(POINT_ONE_HOP) == 8 and len(POINT_THREE_HOP) == 8  # one entry per hop direction
    dims = (8, 8, 8, 8)
    u = fg.unit_links(dims)
    psi = np.zeros(fg.lattice_shape(dims) + (3,), dtype=np.complex128)
    psi[0, 0, 0, 1, 2] = 1.0
    out = oracle_mod.dslash(dims, u, psi, u if naik else None, C3, True)
    expect = np.zeros_like(out)
    for (x, y, z, t), v in POINT_ONE_HOP.items():
        expect[t, z, y, x, 2] += v
    if naik:
        for (x, y, z, t), v in POINT_THREE_HOP.items():
            expect[t, z, y, x, 2] += C3 * v
    assert np.array_equal(out, expect)


FREE_CASES = [
    ((4, 4, 4, 4), (1, 0, 3, 2)),
    ((8, 4, 6, 8), (3, 1, 5, 0)),
    ((8, 8, 8, 8), (1, 2, 3, 7)),
]


@pytest.mark.parametrize("dims,n", FREE_CASES)
@pytest.mark.parametrize("c3", [0.0, C3])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_free_field_spectrum(oracle_mod, dims, n, c3, antiperiodic):
    """Unit links: the even-site restriction of e^{ip.x} e_c is an eigenvector
    of A = m^2 - D_eo D_oe with eigenvalue m^2 + sum_mu (2 sin p + 2 c3 sin 3p)^2
    (the eta phases anticommute, so D^2 = sum_mu (nabla_mu + c3 nabla3_mu)^2);
    antiperiodic time shifts p_t by pi/Lt.  Catches a dropped or mis-scaled
    Naik term, a missing boundary sign, broken anticommutation of the phases
    and a wrong sign in the normal operator."""
    m = 0.1
    u = fg.unit_links(dims)
    w = u if c3 else None
    for colour in range(3):
        pw = oracle_mod.plane_wave(dims, n, colour, antiperiodic)
        pw[~oracle_mod.even_sites(dims)] = 0
        lam = oracle_mod.free_eigenvalue(dims, n, m, c3, antiperiodic)
        a = oracle_mod.normal_op(dims, u, pw, m, w, c3, antiperiodic)
        assert np.abs(a - lam * pw).max() <= 1e-13 * lam


def test_free_field_full_spectrum_dense(oracle_mod):
    """On a 4x2x2x4 lattice with unit links the dense A has exactly the
    multiset of closed-form eigenvalues: each momentum p and its partner p+pi
    (all components) give the same even-site vector, so every value of
    lambda(p) over the full Brillouin zone appears 3/2 times per pair."""
    dims = (4, 2, 2, 4)
    m = 0.3
    u = fg.unit_links(dims)
    a = oracle_mod.dense_normal_op(dims, u, m, u, C3, True)
    ev = np.sort(np.linalg.eigvalsh(a))
    lams = []
    for nx in range(4):
        for ny in range(2):
            for nz in range(2):
                for nt in range(4):
                    lams.append(oracle_mod.free_eigenvalue(dims, (nx, ny, nz, nt), m, C3, True))
    # momenta p and p + (pi,pi,pi,pi) give the same even-site vector: keep half, 3 colours
    expect = np.sort(np.repeat(np.array(lams), 3))[::2]
    assert np.allclose(ev, expect, rtol=0, atol=1e-12)


# ------------------------------------------------------------------- CG / dense

@pytest.mark.parametrize("naik", [False, True])
def test_dense_normal_operator_and_cg(oracle_mod, naik):
    """A built column by column is Hermitian with eigenvalues >= m^2, and CG
    matches numpy's dense solve (catches a wrong alpha/beta or an update on
    the wrong vector)."""
    dims = (2, 2, 2, 2) if not naik else (4, 4, 2, 2)
    m = 0.2
    s = fg.rng_streams(13)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    a = oracle_mod.dense_normal_op(dims, u, m, w, C3)
    assert np.abs(a - a.conj().T).max() <= 1e-13 * np.abs(a).max()
    assert np.linalg.eigvalsh(a).min() >= m * m * (1 - 1e-12)
    b = fg.gaussian_field(s["source"], dims)
    ev = oracle_mod.even_sites(dims)
    b[~ev] = 0
    x, ok, it, tr = oracle_mod.cg(dims, u, b, m, w, C3, tol=1e-13, maxiter=5000)
    assert ok and tr <= 1e-13
    xd = np.linalg.solve(a, b[ev].reshape(-1))
    assert np.linalg.norm(x[ev].reshape(-1) - xd) <= 1e-11 * np.linalg.norm(xd)
    assert np.all(x[~ev] == 0)


def test_cg_plane_wave_exact(oracle_mod):
    """A plane-wave source on unit links is solved by x = b / lambda."""
    dims = (8, 4, 6, 8)
    m = 0.05
    n = (3, 1, 2, 5)
    u = fg.unit_links(dims)
    b = oracle_mod.plane_wave(dims, n, 1)
    b[~oracle_mod.even_sites(dims)] = 0
    lam = oracle_mod.free_eigenvalue(dims, n, m, C3)
    x, ok, it, tr = oracle_mod.cg(dims, u, b, m, u, C3, tol=1e-12)
    assert ok and it <= 2
    assert np.abs(x - b / lam).max() <= 1e-13 / lam


def test_cg_true_residual_and_workload_cfg4(oracle_mod):
    """4^4 Haar links, m = 0.1, one Gaussian even-site source: CG reaches a
    true relative residual of 1e-10, recomputed independently."""
    wl = fg.workload("cfg4x4")
    u, _, b = fg.make_inputs(wl["dims"], wl["fat"], False, wl["seed"])
    x, ok, it, tr = oracle_mod.cg(wl["dims"], u, b, wl["mass"], tol=1e-10)
    assert ok and tr <= 1e-10
    r = b - oracle_mod.normal_op(wl["dims"], u, x, wl["mass"])
    r[~oracle_mod.even_sites(wl["dims"])] = 0
    assert np.linalg.norm(r) / np.linalg.norm(b) == pytest.approx(tr, rel=1e-6)


def test_cg_zero_source_and_maxiter(oracle_mod):
    dims = (4, 4, 4, 4)
    u = fg.unit_links(dims)
    b = np.zeros(fg.lattice_shape(dims) + (3,), dtype=np.complex128)
    x, ok, it, tr = oracle_mod.cg(dims, u, b, 0.1)
    assert ok and it == 0 and not x.any()
    s = fg.rng_streams(3)
    u = fg.random_links(dims, "haar", s["links"])
    b = fg.gaussian_field(s["source"], dims)
    x, ok, it, tr = oracle_mod.cg(dims, u, b, 0.1, maxiter=3)
    assert not ok and it == 3


# ------------------------------------------------------------------- generators

def test_generators_unitary():
    s = fg.rng_streams(5)
    for u in (fg.haar_su3(s["links"], (5000,)), fg.exp_i_su3(s["links"], (5000,), 0.5)):
        uu = np.einsum("...ji,...jk->...ik", u.conj(), u)
        assert np.abs(uu - np.eye(3)).max() < 1e-14
        assert np.abs(np.linalg.det(u) - 1).max() < 1e-14


def test_haar_moments():
    """E|tr U|^2 = 1 and E tr U = 0 for Haar SU(3) (second moment of the
    character); the standard error at 40000 draws is 0.005."""
    u = fg.haar_su3(fg.rng_streams(6)["links"], (40000,))
    tr = np.trace(u, axis1=-2, axis2=-1)
    assert abs(np.mean(np.abs(tr) ** 2) - 1) < 0.03
    assert abs(np.mean(tr)) < 0.03


def test_exp_links_near_identity():
    """exp(i a H) -> 1 as a -> 0: ||U - 1|| scales linearly with a."""
    s = fg.rng_streams(7)
    d1 = np.abs(fg.exp_i_su3(fg.rng_streams(7)["links"], (1000,), 1e-3) - np.eye(3)).mean()
    d2 = np.abs(fg.exp_i_su3(s["links"], (1000,), 2e-3) - np.eye(3)).mean()
    assert d2 / d1 == pytest.approx(2.0, rel=1e-2)
