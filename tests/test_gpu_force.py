"""GPU fermion force (qex_force, StaggeredAction) against the oracle and
against finite differences of the action.

S = phi^+ A^{-1} phi, A = m^2 - D_eo D_oe, phi = (M^+ chi)_e held fixed.
"""

import numpy as np
import pytest

import fieldgen as fg
from parity import assert_close

pytestmark = pytest.mark.gpu

C3 = -1.0 / 24.0


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


def _inputs(oracle_mod, dims, naik, seed, m, a=0.5):
    s = fg.rng_streams(seed)
    u = fg.random_links(dims, "exp", s["links"], a)
    w = fg.random_links(dims, "gauss3", s["long_links"]) if naik else None
    chi = fg.gaussian_field(s["chi"], dims)
    phi = oracle_mod.pseudofermion(dims, u, chi, m, w, C3 if naik else 0.0)
    return s, u, w, phi


@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("kind", [0, 1])
def test_force_kernel_matches_oracle(q, oracle_mod, naik, kind):
    """Same X and Y on both sides: the per-link force (kind 0) and gradient
    (kind 1) agree to 1e-13, fat and long links, on a ragged lattice."""
    dims = (6, 4, 4, 10)
    m = 0.2
    s, u, w, phi = _inputs(oracle_mod, dims, naik, 51, m)
    c3 = C3 if naik else 0.0
    _, x = oracle_mod.action(dims, u, phi, m, w, c3)
    y = oracle_mod.dslash_parity(dims, u, x, 1, w, c3)
    ref_f, ref_l = oracle_mod.force(dims, u, x, y, w, c3, kind)
    lat = q.Lattice(dims)
    fat = q.qex_pack_links(lat, "f64", dev(u))
    lng = q.qex_pack_links(lat, "f64", dev(w)) if naik else None
    xe = q.qex_pack_field(lat, "f64", 0, dev(x))
    yo = q.qex_pack_field(lat, "f64", 1, dev(y))
    gf, gl = q.qex_force(lat, fat, lng, c3, xe, yo, kind)
    assert_close(q.qex_unpack_links(lat, "f64", gf).cpu().numpy(), ref_f, 1e-13, ("fat", naik, kind))
    if naik:
        assert_close(q.qex_unpack_links(lat, "f64", gl).cpu().numpy(), ref_l, 1e-13, ("long", kind))


@pytest.mark.parametrize("inner,bound", [("f64", 1e-9), ("f32r12", 1e-7)])
def test_force_chain_matches_oracle(q, oracle_mod, inner, bound):
    """GPU solve (FP64 to 1e-12, or mixed precision to 1e-10), GPU D_oe and
    GPU force against the oracle chain solved to 1e-13: the difference is the
    solver tolerance carried through (stated bound per precision)."""
    import torch

    dims = (8, 8, 4, 8)
    m = 0.1
    s, u, w, phi = _inputs(oracle_mod, dims, True, 52, m)
    _, x = oracle_mod.action(dims, u, phi, m, w, C3)
    y = oracle_mod.dslash_parity(dims, u, x, 1, w, C3)
    ref_f, ref_l = oracle_mod.force(dims, u, x, y, w, C3, 0)
    lat = q.Lattice(dims)
    fat = q.qex_pack_links(lat, "f64", dev(u))
    lng = q.qex_pack_links(lat, "f64", dev(w))
    b = q.qex_pack_field(lat, "f64", 0, dev(phi))
    xg = torch.zeros_like(b)
    tol = 1e-12 if inner == "f64" else 1e-10
    f32 = q.qex_convert_links(lat, "f64", fat, inner) if inner != "f64" else None
    l32 = q.qex_convert_links(lat, "f64", lng, "f32") if inner != "f64" else None
    q.qex_cg(lat, inner, fat, lng, f32, l32, C3, m, b, xg, tol=tol)
    yg = q.qex_dslash(lat, "f64", fat, lng, C3, 1, xg)
    gf, gl = q.qex_force(lat, fat, lng, C3, xg, yg, 0)
    assert_close(q.qex_unpack_links(lat, "f64", gf).cpu().numpy(), ref_f, bound, ("fat", inner))
    assert_close(q.qex_unpack_links(lat, "f64", gl).cpu().numpy(), ref_l, bound, ("long", inner))


def _action_quadratic(q, lat, fat, lng, c3, m, b, tol=1e-13):
    """S estimated as 2 Re phi^+ X - X^+ A X: its error is -e^+ A e for the
    solver error e, second order in the residual (finite differences need
    S to ~1e-13 relative)."""
    import torch

    x = torch.zeros_like(b)
    q.qex_cg(lat, "f64", fat, lng, None, None, c3, m, b, x, tol=tol, maxiter=100000)
    ax = q.qex_normal_op(lat, "f64", fat, lng, c3, m, x)
    return 2 * q.qex_dot(lat, "f64", b, x)[0].item() - q.qex_dot(lat, "f64", x, ax)[0].item()


@pytest.mark.slow
def test_force_finite_differences_cfg16(q):
    """The 16^4 force workload (links exp(i 0.5 H), m = 0.05, phi = M^+ chi
    with chi Gaussian, formed on the GPU): sum i tr(w F) equals the central
    difference of S along U -> exp(+-i e w) U, e = 1e-5, for 32 random su(3)
    directions w on every link, to 1e-6 relative."""
    import torch

    wl = fg.workload("cfg16force")
    dims, m = wl["dims"], wl["mass"]
    s = fg.rng_streams(wl["seed"])
    u = fg.random_links(dims, "exp", s["links"], wl["a"])
    chi = fg.gaussian_field(s["chi"], dims)
    lat = q.Lattice(dims)
    U = dev(u)
    fat = q.qex_pack_links(lat, "f64", U)
    # phi_e = m chi_e - D_eo chi_o on the GPU, held fixed
    ce = q.qex_pack_field(lat, "f64", 0, dev(chi))
    co = q.qex_pack_field(lat, "f64", 1, dev(chi))
    b = m * ce - q.qex_dslash(lat, "f64", fat, None, 0.0, 0, co)
    x = torch.zeros_like(b)
    q.qex_cg(lat, "f64", fat, None, None, None, 0.0, m, b, x, tol=1e-13, maxiter=100000)
    y = q.qex_dslash(lat, "f64", fat, None, 0.0, 1, x)
    F = q.qex_unpack_links(lat, "f64", q.qex_force(lat, fat, None, 0.0, x, y, 0)[0])
    lam = torch.from_numpy(fg.gell_mann() / 2).cuda()
    eps = 1e-5
    errs = []
    for k in range(32):
        h = torch.from_numpy(s["directions"].standard_normal(fg.lattice_shape(dims) + (4, 8))).cuda()
        om = torch.einsum("...a,aij->...ij", h.to(torch.complex128), lam)
        pred = torch.real(torch.sum(1j * torch.einsum("...ij,...ji->...", om, F))).item()
        sp = []
        for e in (eps, -eps):
            ue = torch.linalg.matrix_exp(1j * e * om) @ U
            sp.append(_action_quadratic(q, lat, q.qex_pack_links(lat, "f64", ue.contiguous()), None, 0.0, m, b))
        fd = (sp[0] - sp[1]) / (2 * eps)
        errs.append(abs(fd - pred) / abs(pred))
    assert max(errs) <= 1e-6, max(errs)


def test_autograd_gradient(q, oracle_mod):
    """StaggeredAction: the value equals the oracle's action, U.grad and
    W.grad equal the oracle's 2 G^+, and a directional finite difference of
    the autograd value along a random complex direction matches
    Re <grad, dU> (FP64 solve), with a mixed-precision solve agreeing to the
    stated bound."""
    import torch

    dims = (4, 4, 4, 8)
    m = 0.15
    s, u, w, phi = _inputs(oracle_mod, dims, True, 53, m)
    S_ref, x = oracle_mod.action(dims, u, phi, m, w, C3)
    y = oracle_mod.dslash_parity(dims, u, x, 1, w, C3)
    gref_f, gref_l = oracle_mod.force(dims, u, x, y, w, C3, 1)
    lat = q.Lattice(dims)
    U = dev(u).requires_grad_(True)
    W = dev(w).requires_grad_(True)
    P = dev(phi)
    S = q.StaggeredAction.apply(U, W, P, lat, m, C3, "f64", 1e-13)
    assert S.item() == pytest.approx(S_ref, rel=1e-11)
    S.backward()
    assert_close(U.grad.cpu().numpy(), gref_f, 1e-10, "U.grad")
    assert_close(W.grad.cpu().numpy(), gref_l, 1e-10, "W.grad")
    du = dev(fg.complex_gaussian(s["directions"], u.shape))
    eps = 1e-6
    with torch.no_grad():
        sp = [q.StaggeredAction.apply(U + e * du, W, P, lat, m, C3, "f64", 1e-13).item() for e in (eps, -eps)]
    pred = torch.real(torch.vdot(U.grad.reshape(-1), du.reshape(-1))).item()
    assert (sp[0] - sp[1]) / (2 * eps) == pytest.approx(pred, rel=1e-6)
    # mixed-precision solve: gradient within the bound its 1e-10 solve allows
    U2 = dev(u).requires_grad_(True)
    S2 = q.StaggeredAction.apply(U2, W.detach(), P, lat, m, C3, "f32r12", 1e-10)
    S2.backward()
    assert S2.item() == pytest.approx(S_ref, rel=1e-9)
    assert_close(U2.grad.cpu().numpy(), gref_f, 1e-7, "U.grad, mixed")


@pytest.mark.parametrize("inner", ["f32", "f32r12", "f32r12h", "f32s16"])
def test_autograd_every_mixed_format_with_naik(q, oracle_mod, inner):
    """StaggeredAction with the Naik term and each mixed inner format: the
    long links go to the solver in qex_long_links_prec(inner) (16-bit with a
    per-link step for the 16-bit formats, FP32 otherwise), and the action and
    both gradients meet the oracle within what a 1e-10 solve allows; an
    unknown format is rejected before anything runs."""
    dims = (4, 4, 4, 8)
    m = 0.15
    s, u, w, phi = _inputs(oracle_mod, dims, True, 54, m)
    S_ref, x = oracle_mod.action(dims, u, phi, m, w, C3)
    y = oracle_mod.dslash_parity(dims, u, x, 1, w, C3)
    gref_f, gref_l = oracle_mod.force(dims, u, x, y, w, C3, 1)
    lat = q.Lattice(dims)
    U = dev(u).requires_grad_(True)
    W = dev(w).requires_grad_(True)
    S = q.StaggeredAction.apply(U, W, dev(phi), lat, m, C3, inner, 1e-10)
    S.backward()
    assert S.item() == pytest.approx(S_ref, rel=1e-9)
    assert_close(U.grad.cpu().numpy(), gref_f, 1e-7, ("U.grad", inner))
    assert_close(W.grad.cpu().numpy(), gref_l, 1e-7, ("W.grad", inner))
    with pytest.raises(ValueError):
        q.StaggeredAction.apply(U, W, dev(phi), lat, m, C3, "bf16", 1e-10)
