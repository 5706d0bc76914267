"""Pins of the oracle's fermion force (no GPU).

S = phi^+ A^{-1} phi with A = m^2 - D_eo D_oe and phi = (M^+ chi)_e held
fixed.  The force formula is checked against central finite differences of
the action itself (computed with the oracle's CG and normal operator, both
pinned by test_oracle.py), which a dropped term, a wrong sign, a swapped X/Y
or a missing adjoint would fail, and by its algebraic properties.
"""

import numpy as np
import pytest

import fieldgen as fg

C3 = -1.0 / 24.0


def _expi(omega, eps):
    """exp(i eps omega) for Hermitian omega (stacked), by eigendecomposition."""
    w, v = np.linalg.eigh(omega)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * w), np.conj(v))


def _setup(oracle_mod, dims, naik, seed, m):
    s = fg.rng_streams(seed)
    u = fg.random_links(dims, "exp", s["links"], 0.5)
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    chi = fg.gaussian_field(s["chi"], dims)
    phi = oracle_mod.pseudofermion(dims, u, chi, m, w, C3 if naik else 0.0)
    return s, u, w, phi


def _force(oracle_mod, dims, u, w, phi, m, kind):
    c3 = C3 if w is not None else 0.0
    _, x = oracle_mod.action(dims, u, phi, m, w, c3)
    y = oracle_mod.dslash_parity(dims, u, x, 1, w, c3)
    return oracle_mod.force(dims, u, x, y, w, c3, kind)


@pytest.mark.parametrize("naik", [False, True])
def test_force_matches_finite_differences_su3(oracle_mod, naik):
    """dS/de along U -> exp(i e w) U (w random Hermitian traceless on every
    link) equals sum i tr(w F) to 1e-6 relative (central difference, e = 1e-5,
    solves to 1e-13); the same for the long links with F_long."""
    dims = (4, 4, 4, 6)
    m = 0.2
    s, u, w, phi = _setup(oracle_mod, dims, naik, 41, m)
    ff, fl = _force(oracle_mod, dims, u, w, phi, m, 0)
    c3 = C3 if naik else 0.0
    eps = 1e-5
    targets = [("fat", ff)] + ([("long", fl)] if naik else [])
    for which, F in targets:
        for k in range(3):
            om = fg.su3_algebra(s["directions"], fg.lattice_shape(dims) + (4,))
            pred = float(np.real(np.sum(1j * np.einsum("...ij,...ji->...", om, F))))
            sp = []
            for e in (eps, -eps):
                if which == "fat":
                    sp.append(oracle_mod.action(dims, _expi(om, e) @ u, phi, m, w, c3)[0])
                else:
                    sp.append(oracle_mod.action(dims, u, phi, m, _expi(om, e) @ w, c3)[0])
            fd = (sp[0] - sp[1]) / (2 * eps)
            assert fd == pytest.approx(pred, rel=1e-6), (which, k)


def test_gradient_form_matches_finite_differences(oracle_mod):
    """The gradient form 2 G^+ gives dS = Re sum conj(grad) dU for an arbitrary
    complex (non-unitary) perturbation dU."""
    dims = (4, 4, 2, 4)
    m = 0.3
    s, u, w, phi = _setup(oracle_mod, dims, True, 42, m)
    gf, gl = _force(oracle_mod, dims, u, w, phi, m, 1)
    eps = 1e-6
    du = fg.complex_gaussian(s["directions"], u.shape)
    dw = fg.complex_gaussian(s["directions"], w.shape)
    pred = float(np.real(np.vdot(gf, du) + np.vdot(gl, dw)))
    sp = [oracle_mod.action(dims, u + e * du, phi, m, w + e * dw, C3)[0] for e in (eps, -eps)]
    assert (sp[0] - sp[1]) / (2 * eps) == pytest.approx(pred, rel=1e-6)


def test_force_is_traceless_antihermitian_and_relates_to_gradient(oracle_mod):
    dims = (4, 4, 4, 4)
    m = 0.2
    s, u, w, phi = _setup(oracle_mod, dims, True, 43, m)
    ff, fl = _force(oracle_mod, dims, u, w, phi, m, 0)
    gf, gl = _force(oracle_mod, dims, u, w, phi, m, 1)
    for F in (ff, fl):
        assert np.abs(F + np.conj(np.swapaxes(F, -1, -2))).max() < 1e-13 * np.abs(F).max()
        assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13 * np.abs(F).max()
    # F = 2 TA(U G) with G = (grad / 2)^+
    for links, F, grad in ((u, ff, gf), (w, fl, gl)):
        mm = links @ np.conj(np.swapaxes(grad, -1, -2)) / 2
        ta = (mm - np.conj(np.swapaxes(mm, -1, -2))) / 2
        tr = np.trace(mm - np.conj(np.swapaxes(mm, -1, -2)), axis1=-2, axis2=-1) / 6
        ta = ta - tr[..., None, None] * np.eye(3)
        assert np.abs(2 * ta - F).max() < 1e-13 * np.abs(F).max()


def test_force_gauge_covariance(oracle_mod):
    """U_mu(x) -> g(x) U g(x+mu)^+ and phi -> g phi give F_mu(x) -> g(x) F g(x)^+."""
    dims = (4, 4, 4, 6)
    m = 0.25
    s, u, w, phi = _setup(oracle_mod, dims, False, 44, m)
    g = fg.gauge_transform(s["gauge"], dims)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    u2 = np.empty_like(u)
    for mu in range(4):
        gs = np.roll(g, -1, axis=axes[mu])
        u2[..., mu, :, :] = g @ u[..., mu, :, :] @ np.conj(np.swapaxes(gs, -1, -2))
    phi2 = np.einsum("...ab,...b->...a", g, phi)
    f1, _ = _force(oracle_mod, dims, u, None, phi, m, 0)
    f2, _ = _force(oracle_mod, dims, u2, None, phi2, m, 0)
    gd = np.conj(np.swapaxes(g, -1, -2))
    expect = np.einsum("...ab,...mbc,...cd->...mad", g, f1, gd)
    assert np.abs(f2 - expect).max() < 1e-11 * np.abs(f1).max()


def _dense_full_operator(oracle_mod, dims, u, w, c3, mass, antiperiodic=True):
    """Dense M = m + D on the whole lattice (both parities, 3 colours per
    site), one column per unit vector, each column m e_k + D e_k from the
    oracle's full-lattice operator."""
    shape = fg.lattice_shape(dims) + (3,)
    n = int(np.prod(shape))
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        e = e.reshape(shape)
        cols.append((mass * e + oracle_mod.dslash(dims, u, e, w, c3, antiperiodic)).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims,naik", [((2, 2, 2, 2), False), ((4, 2, 2, 4), True)])
def test_pseudofermion_is_mdagger_chi_on_even_sites(oracle_mod, dims, naik):
    """phi = (M^+ chi) restricted to the even sites, with M = m + D the full
    staggered matrix: M^+ is the conjugate transpose of the dense matrix built
    column by column (no use of D's anti-hermiticity), applied to a random
    full-lattice chi; odd sites of phi are zero.  A sign error in front of the
    hopping term or m^2 in place of m fails here."""
    m = 0.37
    s = fg.rng_streams(44)
    u = fg.random_links(dims, "haar", s["links"])
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    c3 = C3 if naik else 0.0
    chi = fg.gaussian_field(s["chi"], dims)
    M = _dense_full_operator(oracle_mod, dims, u, w, c3, m)
    want = (np.conj(M).T @ chi.reshape(-1)).reshape(chi.shape)
    ev = fg.even_mask(dims)
    got = oracle_mod.pseudofermion(dims, u, chi, m, w, c3)
    assert not got[~ev].any()
    assert np.abs(got[ev] - want[ev]).max() <= 1e-13 * np.abs(want[ev]).max()
