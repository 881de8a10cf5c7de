"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form ray
paths of Eq. 1, invariants, published generator outputs, exact reproduction
properties of the interpolants, symmetry, the small-angle BOS deflection, complex-step
derivatives and finite differences.  A plausible slip in the oracle (a dropped RKN
term, a wrong sign, a transposed stencil, T/T0 for T0/T) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2509_14442_gb300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))


def unit_grid(n=(8, 8, 8), extent=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0)):
    return S.Grid(n=n, origin=origin, extent=extent)


# ----------------------------------------------------------------- generator, filter

def test_splitmix64_published_outputs(orc):
    with open(os.path.join(HERE, "golden", "splitmix64.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for seed, k, out in rows:
        assert orc.splitmix64_output(int(seed), int(k)) == int(out, 0)


def test_tent_inverse_is_inverse_of_triangular_cdf(orc):
    # CDF of the unit triangular density on [-1, 1]
    def cdf(t):
        return 0.5 * (1 + t) ** 2 if t < 0 else 1 - 0.5 * (1 - t) ** 2

    for xi in np.linspace(0.0, 1.0 - 2 ** -24, 257):
        t = orc.tent_inverse(xi)
        assert -1.0 <= t <= 1.0
        assert abs(cdf(t) - xi) < 1e-12
    assert orc.tent_inverse(0.0) == -1.0
    assert orc.tent_inverse(0.5) == 0.0


def test_tent_samples_have_triangular_moments(orc):
    xi = (np.arange(1 << 14) + 0.5) / (1 << 14)
    t = np.array([orc.tent_inverse(x) for x in xi])
    assert abs(t.mean()) < 1e-6
    assert abs((t ** 2).mean() - 1.0 / 6.0) < 1e-6        # variance of the unit tent


# ----------------------------------------------------------------- eta(T), Sec. 2.1

def test_eta_of_T_physical_values(orc):
    g = unit_grid((2, 2, 2))
    T = np.array([293.0, 586.0, 146.5, 310.0, 293.0, 293.0, 293.0, 293.0]).reshape(2, 2, 2)
    de = orc.deta_from_T(g, T).ravel()
    # at ambient, eta - 1 = rho0 G = 2.712e-4: the refractivity of room-temperature air
    assert de[0] == pytest.approx(1.2 * 2.26e-4, rel=1e-15)
    assert 2.6e-4 < de[0] < 2.9e-4
    # ideal gas at constant pressure: density (and eta - 1) scale as 1/T
    assert de[1] == pytest.approx(de[0] / 2, rel=1e-15)
    assert de[2] == pytest.approx(de[0] * 2, rel=1e-15)
    assert de[3] < de[0]                                     # hot air refracts less


def test_gradient_stencil_exact_for_linear_and_quadratic(orc):
    g = unit_grid((7, 6, 5), extent=(0.7, 1.2, 0.5), origin=(-0.3, 0.1, 2.0))
    h = g.spacing()
    x = [g.centers(a) for a in range(3)]
    X, Y, Z = np.meshgrid(x[0], x[1], x[2], indexing="ij")
    X, Y, Z = (np.transpose(a, (2, 1, 0)) for a in (X, Y, Z))     # (nz, ny, nx)
    lin = 1e-4 + 3e-5 * X - 2e-5 * Y + 7e-6 * Z
    gr = orc.grad_from_deta(g, lin)
    np.testing.assert_allclose(gr[..., 0], 3e-5, rtol=1e-9, atol=0)
    np.testing.assert_allclose(gr[..., 1], -2e-5, rtol=1e-9, atol=0)
    np.testing.assert_allclose(gr[..., 2], 7e-6, rtol=1e-9, atol=0)
    # central differences are exact for quadratics at interior nodes
    quad = 1e-4 + 2e-5 * X ** 2 - 3e-5 * Y * Y + 1e-5 * Z ** 2
    gq = orc.grad_from_deta(g, quad)
    np.testing.assert_allclose(gq[:, :, 1:-1, 0], (4e-5 * X)[:, :, 1:-1], rtol=1e-8, atol=1e-18)
    np.testing.assert_allclose(gq[:, 1:-1, :, 1], (-6e-5 * Y)[:, 1:-1, :], rtol=1e-8, atol=1e-18)
    np.testing.assert_allclose(gq[1:-1, :, :, 2], (2e-5 * Z)[1:-1, :, :], rtol=1e-8, atol=1e-18)
    # one-sided at the faces: exact derivative at the half-cell point next to the face
    np.testing.assert_allclose(gq[:, :, 0, 0], (4e-5 * (X[:, :, 0] + 0.5 * h[0])), rtol=1e-8)
    np.testing.assert_allclose(gq[:, :, -1, 0], (4e-5 * (X[:, :, -1] - 0.5 * h[0])), rtol=1e-8)


# ----------------------------------------------------------------- trilinear field

def _node_field(orc, g, fn):
    x = [g.centers(a) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    de = fn(X, Y, Z)
    return orc.NodeField(de, np.zeros(de.shape + (3,))), de


def test_trilinear_reproduces_nodes_and_multilinear_functions(orc):
    g = unit_grid((4, 3, 5), extent=(1.0, 0.9, 1.5))
    f = lambda X, Y, Z: 2e-4 + 1e-5 * X * Y * Z - 3e-5 * X * Z + 4e-6 * Y   # multilinear
    fld, de = _node_field(orc, g, f)
    x = [g.centers(a) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    eta, _ = orc.field_eval(g, fld, np.stack([X, Y, Z], -1).reshape(-1, 3))
    np.testing.assert_allclose(eta - 1.0, de.ravel(), rtol=0, atol=1e-15)
    rng = np.random.default_rng(1)
    # anywhere inside the box (incl. the half cells beyond the outer centres, where the
    # edge cells extrapolate linearly) a multilinear function is reproduced exactly
    p = rng.random((500, 3)) * np.array(g.extent) + np.array(g.origin)
    eta, _ = orc.field_eval(g, fld, p)
    np.testing.assert_allclose(eta - 1.0, f(p[:, 0], p[:, 1], p[:, 2]), rtol=0, atol=1e-15)


def test_trilinear_is_continuous_across_cell_faces(orc):
    g = unit_grid((5, 5, 5))
    rng = np.random.default_rng(3)
    de = 2.7e-4 + 1e-5 * rng.random((5, 5, 5))
    fld = orc.NodeField(de, orc.grad_from_deta(g, de))
    h = g.spacing()[0]
    face = 0.5 * h + 2 * h                                   # between centres 2 and 3
    for eps in (1e-9, 1e-12):
        a = np.array([[face - eps, 0.41, 0.57]])
        b = np.array([[face + eps, 0.41, 0.57]])
        ea, ga = orc.field_eval(g, fld, a)
        eb, gb = orc.field_eval(g, fld, b)
        assert abs(ea[0] - eb[0]) < 1e-5 * eps / h + 1e-18
        np.testing.assert_allclose(ga, gb, rtol=0, atol=1e-3 * eps / h + 1e-18)


# ----------------------------------------------------------------- Eq. 1 closed forms

@pytest.mark.parametrize("integrator", [0, 1])
def test_uniform_field_gives_straight_rays(orc, integrator):
    g = unit_grid()
    fld = orc.AnalyticField(2, [1.0002712, 0.0, 0.0, 0.0])
    d = np.array([0.2, 0.9, -0.1])
    d /= np.linalg.norm(d)
    r, v, ls = orc.trace_segment(g, fld, [0.1, 0.0, 0.5], d, 1.3, 100, integrator)
    np.testing.assert_allclose(r, np.array([0.1, 0.0, 0.5]) + 1.3 * d, rtol=0, atol=1e-14)
    np.testing.assert_allclose(v, 1.0002712 * d, rtol=0, atol=1e-15)
    assert ls == pytest.approx(1.3, rel=1e-13)


@pytest.mark.parametrize("integrator", [0, 1])
def test_parabolic_path_when_eta_squared_is_linear(orc, integrator):
    # eta^2 = a + b.x  =>  D = eta grad eta = b/2 is constant and r(t) = r0 + v0 t + b t^2 / 4
    a, b = 1.0, np.array([0.02, -0.01, 0.03])
    fld = orc.AnalyticField(1, [a, *b])
    g = unit_grid()
    r0 = np.array([0.3, 0.0, 0.4])
    d = np.array([0.05, 1.0, 0.02])
    d /= np.linalg.norm(d)
    ell, N = 2.0, 37
    r, v, _ = orc.trace_segment(g, fld, r0, d, ell, N, integrator)
    eta0 = math.sqrt(a + b @ r0)
    v0 = eta0 * d
    t = ell / eta0                                            # N dt with dt = ell / (N eta0)
    np.testing.assert_allclose(r, r0 + v0 * t + 0.25 * b * t * t, rtol=0, atol=1e-14)
    np.testing.assert_allclose(v, v0 + 0.5 * b * t, rtol=0, atol=1e-14)


def _linear_eta_closed_form(eta0_fn, gvec, r0, v0, t):
    # u = eta(r(t)) obeys u'' = |g|^2 u, and r'' = g u
    k = np.linalg.norm(gvec)
    u0 = eta0_fn(r0)
    up0 = gvec @ v0
    u = u0 * np.cosh(k * t) + up0 / k * np.sinh(k * t)
    du = u0 * k * np.sinh(k * t) + up0 * np.cosh(k * t)
    r = r0 + v0 * t + gvec / k ** 2 * (u - u0 - up0 * t)
    v = v0 + gvec / k ** 2 * (du - up0)
    return r, v


@pytest.mark.parametrize("integrator", [0, 1])
def test_cosh_path_when_eta_is_linear(orc, integrator):
    gvec = np.array([0.05, 0.2, -0.1])
    e0 = 1.0003
    fld = orc.AnalyticField(2, [e0, *gvec])
    g = unit_grid()
    r0 = np.array([0.2, 0.0, 0.6])
    d = np.array([0.1, 1.0, 0.05])
    d /= np.linalg.norm(d)
    ell, N = 1.2, 96
    r, v, _ = orc.trace_segment(g, fld, r0, d, ell, N, integrator)
    eta0 = e0 + gvec @ r0
    t = ell / eta0
    rc, vc = _linear_eta_closed_form(lambda x: e0 + gvec @ x, gvec, r0, eta0 * d, t)
    dev = np.linalg.norm(rc - (r0 + eta0 * d * t))            # bending, ~1e-2 m
    assert dev > 1e-3
    np.testing.assert_allclose(r, rc, rtol=0, atol=1e-9 * dev)
    np.testing.assert_allclose(v, vc, rtol=0, atol=1e-9)


def test_linear_eta_grid_matches_closed_form_through_the_box(orc):
    # deta sampled at the cell centres from a linear function: the difference stencil and
    # the trilinear interpolant (linear beyond the outer centres) are exact, so the
    # whole grid path equals the analytic linear-eta ray
    g = S.Grid(n=(6, 9, 7), origin=(-0.2, 0.0, 0.1), extent=(0.6, 0.9, 0.7))
    gvec = np.array([0.03, 0.12, -0.05])
    d0 = 2.7e-4
    x = [g.centers(a) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    de = d0 + gvec[0] * X + gvec[1] * Y + gvec[2] * Z
    fld = orc.NodeField(de, orc.grad_from_deta(g, de))
    r0 = np.array([0.05, 0.0, 0.45])
    d = np.array([0.05, 1.0, 0.03])
    d /= np.linalg.norm(d)
    ell, N = 0.85, 120
    for integ in (0, 1):
        r, v, _ = orc.trace_segment(g, fld, r0, d, ell, N, integ)
        eta0 = 1 + d0 + gvec @ r0
        rc, vc = _linear_eta_closed_form(lambda p: 1 + d0 + gvec @ p, gvec, r0, eta0 * d, ell / eta0)
        np.testing.assert_allclose(r, rc, rtol=0, atol=1e-12)
        np.testing.assert_allclose(v, vc, rtol=0, atol=1e-12)


def test_invariant_speed_equals_eta_along_the_ray(orc):
    g = unit_grid()
    fld = orc.AnalyticField(3, [2.7e-4, 3e-3, 0.55, 0.5, 0.45, 0.12])
    d = np.array([0.02, 1.0, -0.01])
    d /= np.linalg.norm(d)
    for integ in (0, 1):
        r, v, _, tape = orc.trace_segment(g, fld, [0.5, 0.0, 0.5], d, 1.0, 200, integ, tape=True)
        eta, _ = orc.field_eval(g, fld, tape[:, :3])
        speed2 = (tape[:, 3:] ** 2).sum(1)
        # truncation only: ~1e-11 here, where a second-order slip would give ~1e-6
        assert np.abs(speed2 - eta ** 2).max() < 1e-10
        # and the ray did bend
        assert np.linalg.norm(r - (np.array([0.5, 0, 0.5]) + d * np.linalg.norm(r - [0.5, 0, 0.5]))) > 1e-5


@pytest.mark.parametrize("integrator", [0, 1])
def test_fourth_order_convergence(orc, integrator):
    # strong Gaussian lens so the truncation error is far above rounding
    g = unit_grid()
    fld = orc.AnalyticField(3, [0.0, 0.05, 0.58, 0.5, 0.44, 0.1])
    r0 = np.array([0.5, 0.0, 0.5])
    d = np.array([0.0, 1.0, 0.0])
    ref, _, _ = orc.trace_segment(g, fld, r0, d, 1.0, 16384, integrator)
    errs = []
    for N in (32, 64, 128, 256):
        r, _, _ = orc.trace_segment(g, fld, r0, d, 1.0, N, integrator)
        errs.append(np.linalg.norm(r - ref))
    for e1, e2 in zip(errs, errs[1:]):
        assert 14.0 < e1 / e2 < 19.0                          # 2^4 = 16


# ----------------------------------------------------------------- camera, box, wall

def test_ray_setup_geometry_of_the_room(orc):
    sc = S.room((64, 64, 48), 40, 30, 1, 5)
    cam = sc.camera
    right = np.cross(cam.fwd, cam.up)
    h = min(sc.grid.spacing())
    for pix in (0, 39, 40 * 15 + 20, 40 * 30 - 1, 617):
        st = orc.ray_setup(sc, pix, 0)
        d = st["d"]
        assert abs(np.linalg.norm(d) - 1) < 1e-15
        px, py = pix % cam.width, pix // cam.width
        # projecting the direction back through the pinhole gives the pixel centre
        x = cam.cx + cam.fx * (d @ right) / (d @ cam.fwd)
        y = cam.cy - cam.fy * (d @ cam.up) / (d @ cam.fwd)
        assert x == pytest.approx(px + 0.5, abs=1e-9) and y == pytest.approx(py + 0.5, abs=1e-9)
        # enters through the front face y = 0, leaves at the back wall y = 4
        assert st["t_in"] == pytest.approx(29.0 / d[1], rel=1e-14)
        assert st["ell"] == pytest.approx(4.0 / d[1], rel=1e-14)
        assert st["tw"] == pytest.approx(33.0 / d[1], rel=1e-14)
        assert st["N"] == math.ceil(st["ell"] / (0.5 * h))
        assert st["wall"] and st["traced"]


def test_jittered_samples_stay_within_the_tent_support(orc):
    sc = S.room((16, 16, 12), 8, 6, 16, 7)
    for pix in range(0, 48, 5):
        xs = np.array([orc.ray_setup(sc, pix, s)["xy"] for s in range(16)])
        px, py = pix % 8, pix // 8
        assert np.all(np.abs(xs[:, 0] - (px + 0.5)) <= 1) and np.all(np.abs(xs[:, 1] - (py + 0.5)) <= 1)
        assert len(np.unique(xs[:, 0])) == 16


def test_luminance_texture_and_projector(orc):
    g = unit_grid()
    wall = S.back_wall(g)
    rng = np.random.default_rng(0)
    tex = rng.random((8, 10)).astype(np.float32)
    light = S.Light(0, tex)
    # texel centres return the texel value; far outside the texture is dark
    pts = []
    want = []
    for j in range(8):
        for i in range(10):
            pts.append([(i + 0.5) / 10, 1.0, (j + 0.5) / 8])
            want.append(tex[j, i])
    np.testing.assert_allclose(orc.luminance(light, wall, pts), want, rtol=0, atol=1e-7)
    assert orc.luminance(light, wall, [[1.5, 1.0, 0.5], [-0.2, 1.0, 0.5]]).max() == 0.0
    # a pattern linear in projector pixels is reproduced exactly inside its support
    sc = S.room((16, 16, 12), 8, 8, 1, 3, pattern_size=64)
    proj = sc.light.proj
    yy, xx = np.mgrid[0:64, 0:64]
    pat = (0.25 + 0.003 * xx + 0.002 * yy).astype(np.float64)
    lp = S.Light(1, pat.astype(np.float32), proj)
    q = np.array([[0.8, 4.0, 1.2], [1.85, 4.0, 1.5], [2.3, 4.0, 0.9]])
    Lv = orc.luminance(lp, sc.wall, q)
    z = q[:, 1] - proj.pos[1]
    px = proj.cx + proj.fx * (q[:, 0] - proj.pos[0]) / z
    py = proj.cy - proj.fy * (q[:, 2] - proj.pos[2]) / z
    np.testing.assert_allclose(Lv, 0.25 + 0.003 * (px - 0.5) + 0.002 * (py - 0.5), rtol=0, atol=2e-7)


# ----------------------------------------------------------------- Eq. 2, whole pipeline

def test_uniform_medium_image_is_cosine_over_distance(orc):
    import dataclasses
    sc = S.room((16, 16, 12), 12, 10, 4, 11)
    cam = dataclasses.replace(sc.camera, fx=2 * sc.camera.fx, fy=2 * sc.camera.fy)   # all jitter on the wall
    sc = sc.replace(T=np.full_like(sc.T, S.T_AMBIENT), camera=cam,
                    light=S.Light(0, np.ones((64, 64), np.float32)))
    out = orc.render(sc, nsteps=True)
    assert out["nsteps"].min() > 0
    ref = np.zeros((10, 12))
    for pix in range(120):
        acc = 0.0
        for s in range(4):
            st = orc.ray_setup(sc, pix, s)
            acc += st["d"][1] / st["tw"]                     # <n, d> / |wall - pinhole|
        ref.flat[pix] = acc / 4
    np.testing.assert_allclose(out["I"], ref, rtol=1e-12, atol=0)
    assert np.abs(out["disp"]).max() < 1e-12


def test_symmetric_blob_gives_point_symmetric_displacement(orc):
    sc = S.blob_cube()
    g = sc.grid
    T = S.blob_field(g, (0.5, 0.5, 0.5), 0.15, 8.0)
    T = 0.5 * (T + T[:, :, ::-1])                            # exact mirror symmetry in x
    T = 0.5 * (T + T[::-1, :, :])                            # and in z
    sc = sc.replace(T=T.astype(np.float64))
    out = orc.render(sc)
    disp = out["disp"]
    assert np.abs(disp).max() > 1e-6
    flipped = disp[::-1, ::-1]
    np.testing.assert_allclose(disp, -flipped, rtol=0, atol=1e-13)
    # rays are pushed away from the hot (low-eta) core: outward in both wall axes
    H, W = disp.shape[:2]
    assert disp[H // 2, W // 2 + 8, 0] > 0 and disp[H // 2 - 8, W // 2, 1] > 0


def test_small_angle_deflection_matches_linearised_bos(orc):
    # first order in the deflection: disp = int_0^Lw (Lw - s) grad_perp(eta)/eta ds along the
    # straight ray (here the principal ray along +y), Lw = distance from entry to wall
    g = unit_grid()
    p = [2.7e-4, -2e-5, 0.6, 0.5, 0.45, 0.15]
    fld = orc.AnalyticField(3, p)
    cam = S.Camera(pos=(0.5, -1.5, 0.5), fwd=(0.0, 1.0, 0.0), up=(0.0, 0.0, 1.0), fx=50.0, fy=50.0,
                   cx=1.5, cy=1.5, width=3, height=3, spp=1)
    sc = S.Scene("lin", g, np.zeros((8, 8, 8)), cam, S.back_wall(g), S.Light(0, np.ones((2, 2), np.float32)),
                 S.Integrator(fixed_steps=400))
    out = orc.render(sc, field=fld, pix=[4])
    s = np.linspace(0.0, 1.0, 20001)
    pts = np.stack([np.full_like(s, 0.5), s, np.full_like(s, 0.5)], 1)
    eta, gr = orc.field_eval(g, fld, pts)
    w = (1.0 - s)[:, None] * gr / eta[:, None]
    lin = np.trapezoid(w, s, axis=0)
    np.testing.assert_allclose(out["disp"][0], [lin[0], lin[2]], rtol=2e-3)
    assert np.abs(lin).max() > 1e-6


# ----------------------------------------------------------------- gradient, Sec. 2.4

def _grad_scene(n=6, w=10, h=8, spp=2):
    g = S.Grid(n=(n, n, n), origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 1.0))
    T = S.blob_field(g, (0.45, 0.55, 0.52), 0.2, 30.0).astype(np.float64)
    cam = S.Camera(pos=(0.5, -1.5, 0.5), fwd=(0.0, 1.0, 0.0), up=(0.0, 0.0, 1.0), fx=w / 0.9, fy=w / 0.9,
                   cx=w / 2, cy=h / 2, width=w, height=h, spp=spp, seed=99)
    light = S.Light(0, S.smooth_pattern(24, 24, 4))
    return S.Scene("grad", g, T, cam, S.back_wall(g), light, S.Integrator(fixed_steps=40))


def test_complex_step_matches_central_differences(orc):
    sc = _grad_scene()
    rng = np.random.default_rng(5)
    dT = rng.standard_normal(sc.T.shape)
    dI, _ = orc.render_cs(sc, dT)
    eps = 1e-3
    Ip = orc.render(sc.replace(T=sc.T + eps * dT))["I"]
    Im = orc.render(sc.replace(T=sc.T - eps * dT))["I"]
    fd = (Ip - Im) / (2 * eps)
    assert np.abs(dI).max() > 1e-8
    np.testing.assert_allclose(dI, fd, rtol=0, atol=1e-6 * np.abs(dI).max())


def test_adjoint_gradient_matches_complex_step(orc):
    sc = _grad_scene()
    rng = np.random.default_rng(6)
    w = rng.standard_normal((sc.camera.height, sc.camera.width))
    gT = orc.grad(sc, w)
    for trial in range(3):
        dT = rng.standard_normal(sc.T.shape)
        dI, _ = orc.render_cs(sc, dT)
        lhs = float((gT * dT).sum())
        rhs = float((w * dI).sum())
        assert abs(lhs - rhs) <= 1e-9 * max(abs(rhs), 1e-30) + 1e-18, (lhs, rhs)


def test_adjoint_gradient_matches_complex_step_with_projector(orc):
    sc = S.room((12, 12, 9), 14, 12, 2, 21, pattern_size=32)
    sc = sc.replace(light=S.Light(1, S.smooth_pattern(32, 32, 8), sc.light.proj), T=sc.T.astype(np.float64))
    rng = np.random.default_rng(7)
    w = rng.standard_normal((12, 14))
    gT = orc.grad(sc, w)
    dT = rng.standard_normal(sc.T.shape)
    dI, _ = orc.render_cs(sc, dT)
    lhs, rhs = float((gT * dT).sum()), float((w * dI).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)


def test_loss_gradient_single_voxel_central_difference(orc):
    sc = _grad_scene(spp=1)
    target = orc.render(sc.replace(T=sc.T + 0.5 * np.sin(np.arange(sc.T.size)).reshape(sc.T.shape)))["I"]
    I = orc.render(sc)["I"]
    gT = orc.grad(sc, -2.0 * (target - I))
    k = np.unravel_index(np.argmax(np.abs(gT)), gT.shape)
    eps = 1e-2

    def loss(T):
        return float(((target - orc.render(sc.replace(T=T))["I"]) ** 2).sum())

    Tp, Tm = sc.T.copy(), sc.T.copy()
    Tp[k] += eps
    Tm[k] -= eps
    fd = (loss(Tp) - loss(Tm)) / (2 * eps)
    assert gT[k] == pytest.approx(fd, rel=1e-5)


def test_adjoint_at_a_uniform_medium_matches_central_differences(orc):
    # In a uniform medium whose box ends at the back wall, rays end on the wall
    # (x_w = r_N) and |x_w - r_N| has a kink there; the adjoint takes its zero
    # subgradient, which is what a central difference (symmetric in +/- eps) sees.
    sc = S.room((12, 12, 9), 24, 18, 1, 23, pattern_size=32)
    sc = sc.replace(T=np.full(sc.T.shape, S.T_AMBIENT))
    rng = np.random.default_rng(8)
    w = rng.standard_normal((18, 24))
    gT = orc.grad(sc, w)
    assert np.isfinite(gT).all() and np.abs(gT).max() > 0
    dT = rng.standard_normal(sc.T.shape)
    eps = 1e-3
    Ip = orc.render(sc.replace(T=sc.T + eps * dT))["I"]
    Im = orc.render(sc.replace(T=sc.T - eps * dT))["I"]
    rhs = float((w * (Ip - Im)).sum()) / (2 * eps)
    lhs = float((gT * dT).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)


# ----------------------------------------------------------------- quasi-linear tracing, Sec. 2.2

def test_quasi_linear_closed_form_when_eta_is_linear(orc):
    # on the straight line eta(r_in + t v0) = eta0 + (g.v0) t, so
    #   v(t) = v0 + g (eta0 t + (g.v0) t^2 / 2),  r(t) = r0 + v0 t + g (eta0 t^2 / 2 + (g.v0) t^3 / 6)
    # which Sharma's weights integrate exactly (the sampled right-hand side is linear in t)
    gvec = np.array([0.05, 0.2, -0.1])
    e0 = 1.0003
    fld = orc.AnalyticField(2, [e0, *gvec])
    g = unit_grid()
    r0 = np.array([0.2, 0.0, 0.6])
    d = np.array([0.1, 1.0, 0.05])
    d /= np.linalg.norm(d)
    ell, N = 1.2, 50
    r, v, _ = orc.trace_segment(g, fld, r0, d, ell, N, 2)
    eta0 = e0 + gvec @ r0
    v0 = eta0 * d
    t = ell / eta0
    gv = gvec @ v0
    np.testing.assert_allclose(v, v0 + gvec * (eta0 * t + gv * t * t / 2), rtol=0, atol=1e-13)
    np.testing.assert_allclose(r, r0 + v0 * t + gvec * (eta0 * t * t / 2 + gv * t ** 3 / 6), rtol=0, atol=1e-13)
    # and differs from the fully coupled ray at second order in the bending
    rn, _, _ = orc.trace_segment(g, fld, r0, d, ell, N, 0)
    bend = np.linalg.norm(rn - (r0 + v0 * t))
    assert 0 < np.linalg.norm(r - rn) < 0.2 * bend


def test_quasi_linear_is_close_to_nonlinear_in_weak_fields(orc):
    # the paper's premise (Sec. 2.2): for small index changes the quasi-linear path deviates
    # little from the true one -- here the displacement differs at second order
    sc = S.blob_cube()
    on = orc.render(sc)
    oq = orc.render(sc.replace(integ=S.Integrator(fixed_steps=128, integrator=2)))
    dmax = np.abs(on["disp"]).max()
    assert np.abs(oq["disp"] - on["disp"]).max() < 1e-2 * dmax
    assert np.abs(oq["disp"] - on["disp"]).max() > 0


def test_quasi_linear_adjoint_matches_complex_step(orc):
    sc = _grad_scene()
    sc = sc.replace(integ=S.Integrator(fixed_steps=40, integrator=2))
    rng = np.random.default_rng(12)
    w = rng.standard_normal((sc.camera.height, sc.camera.width))
    gT = orc.grad(sc, w)
    for _ in range(2):
        dT = rng.standard_normal(sc.T.shape)
        dI, _ = orc.render_cs(sc, dT)
        lhs, rhs = float((gT * dT).sum()), float((w * dI).sum())
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs), (lhs, rhs)


# ------------------------------------------------- refracted projector connection, Sec. 2.3

def _refracted_room(n=(16, 16, 12), w=20, h=16, seed=31, iters=1, boost=4.0, pattern=None):
    """Room scene lit by the projector with its rays traced through the flow; the plume's
    excess temperature is scaled by `boost` so the projector rays bend visibly."""
    sc = S.room(n, w, h, 1, seed, pattern_size=64)
    T = S.T_AMBIENT + boost * (sc.T.astype(np.float64) - S.T_AMBIENT)
    pat = S.smooth_pattern(64, 64, seed) if pattern is None else pattern
    return sc.replace(T=T, light=S.Light(2, pat, sc.light.proj, connect_iters=iters))


def _wall_points(sc, orc, k=12, seed=0):
    """Wall points the camera's flow rays actually hit."""
    hit = orc.render(sc)["hit"].reshape(-1, 2)
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(hit), size=k, replace=False)
    w = sc.wall
    o, eu, ev = (np.asarray(v, dtype=np.float64) for v in (w.origin, w.eu, w.ev))
    return o[None] + hit[idx, 0:1] * eu[None] + hit[idx, 1:2] * ev[None]


def test_refracted_connection_is_straight_in_a_uniform_medium(orc):
    sc = _refracted_room()
    sc = sc.replace(T=np.full(sc.T.shape, S.T_AMBIENT))
    x = _wall_points(sc, orc)
    a, y = orc.connect(sc, x, iters=3)
    np.testing.assert_allclose(a, x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(y, x, rtol=0, atol=1e-12)
    I2 = orc.render(sc)["I"]
    I1 = orc.render(sc.replace(light=S.Light(1, sc.light.pattern, sc.light.proj)))["I"]
    np.testing.assert_allclose(I2, I1, rtol=1e-12, atol=0)


def test_refracted_connection_matches_a_brute_force_search(orc):
    # the connected aim a* is the wall point whose projector ray lands on x; find it by a
    # two-level grid search over aims in the wall plane, independent of the aiming rule
    sc = _refracted_room(boost=8.0)
    x = _wall_points(sc, orc, k=3, seed=1)
    a6, y6 = orc.connect(sc, x, iters=6)
    a1, _ = orc.connect(sc, x, iters=1)
    w = sc.wall
    eu, ev = np.asarray(w.eu, dtype=np.float64), np.asarray(w.ev, dtype=np.float64)
    for j in range(len(x)):
        delta = np.linalg.norm(a1[j] - x[j])
        assert delta > 1e-6                                  # the projector rays do bend
        assert np.linalg.norm(y6[j] - x[j]) < 1e-12          # the aiming rule converges
        assert np.linalg.norm(a1[j] - a6[j]) < 1e-2 * delta  # one round is nearly there
        centre, span = x[j].copy(), 2.0 * delta
        for _ in range(2):
            g = np.linspace(-span, span, 41)
            aims = (centre[None, None] + g[:, None, None] * eu[None, None] + g[None, :, None] * ev[None, None])
            aims = aims.reshape(-1, 3)
            _, y = orc.connect(sc, aims, iters=0)            # y(a) for each candidate aim
            best = np.argmin(np.linalg.norm(y - x[j][None], axis=1))
            centre, span = aims[best], 2.0 * (g[1] - g[0])
        assert np.linalg.norm(centre - a6[j]) <= 2.0 * span


@pytest.mark.parametrize("iters", [1, 2])
def test_refracted_adjoint_matches_complex_step(orc, iters):
    sc = _refracted_room(n=(12, 12, 9), w=14, h=12, seed=37, iters=iters)
    rng = np.random.default_rng(40 + iters)
    w = rng.standard_normal((12, 14))
    gT = orc.grad(sc, w)
    for trial in range(2):
        dT = rng.standard_normal(sc.T.shape)
        dI, _ = orc.render_cs(sc, dT)
        lhs, rhs = float((gT * dT).sum()), float((w * dI).sum())
        assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)


def test_refracted_gradient_differs_from_the_straight_connection(orc):
    # the projector rays' own sensitivity to T is a visible part of dL/dT
    sc = _refracted_room(n=(12, 12, 9), w=14, h=12, seed=43)
    w = np.random.default_rng(3).standard_normal((12, 14))
    g2 = orc.grad(sc, w)
    g1 = orc.grad(sc.replace(light=S.Light(1, sc.light.pattern, sc.light.proj)), w)
    assert np.linalg.norm(g2 - g1) > 1e-3 * np.linalg.norm(g1)


# ----------------------------------------------------------------- one ray, brute force

def _py_trace_pixel(sc, px, py):
    """One pixel (1 spp: its centre) of a constant-luminance wall, traced by a plain Python
    FP64 loop written from the definitions: eta - 1 = rho0 G T0 / T per cell (Sec. 2.1),
    central / one-sided differences for grad eta, trilinear interpolation with the base
    cell clamped and the fraction not (A4, A5), the pinhole ray, its box segment and
    N = ceil(l / (0.5 min h)) (A13), v0 = eta_in d and dt = ds / eta_in (A3), Sharma's RKN
    steps of Eq. 1 (A2), the straight continuation to the wall, the path length from the
    pinhole with the signed continuation (A7) and the weight <n, v> / (|v| len) of Eq. 2."""
    g, cam, wall = sc.grid, sc.camera, sc.wall
    nx, ny, nz = g.n
    h = np.array(g.spacing())
    o = np.array(g.origin)
    T = sc.T.astype(np.float64)
    de = g.rho0 * g.G * g.T0 / T                              # (nz, ny, nx)
    eta = 1.0 + de
    grad = np.zeros(T.shape + (3,))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                idx = [i, j, k]
                for a, n in enumerate((nx, ny, nz)):
                    lo, hi = list(idx), list(idx)
                    if idx[a] == 0:
                        hi[a] += 1
                        den = h[a]
                    elif idx[a] == n - 1:
                        lo[a] -= 1
                        den = h[a]
                    else:
                        lo[a] -= 1
                        hi[a] += 1
                        den = 2.0 * h[a]
                    grad[k, j, i, a] = (eta[hi[2], hi[1], hi[0]] - eta[lo[2], lo[1], lo[0]]) / den

    def interp(x):
        base, frac = [], []
        for a, n in enumerate((nx, ny, nz)):
            u = (x[a] - o[a]) / h[a] - 0.5
            i0 = min(max(int(math.floor(u)), 0), n - 2)
            base.append(i0)
            frac.append(u - i0)
        val = np.zeros(4)
        for c in range(8):
            bits = [(c >> a) & 1 for a in range(3)]
            w = 1.0
            for a in range(3):
                w *= frac[a] if bits[a] else 1.0 - frac[a]
            i, j, k = (base[a] + bits[a] for a in range(3))
            val += w * np.array([de[k, j, i], *grad[k, j, i]])
        return val

    def D(x):
        v = interp(x)
        return (1.0 + v[0]) * v[1:]

    pos, fwd, up = np.array(cam.pos), np.array(cam.fwd), np.array(cam.up)
    right = np.cross(fwd, up)
    d = ((px + 0.5 - cam.cx) / cam.fx) * right - ((py + 0.5 - cam.cy) / cam.fy) * up + fwd
    d /= np.linalg.norm(d)
    with np.errstate(divide="ignore"):                        # axis-parallel rays: slabs at +-inf
        t0 = (o - pos) / d
        t1 = (o + np.array(g.extent) - pos) / d
    t_in, t_out = np.max(np.minimum(t0, t1)), np.min(np.maximum(t0, t1))
    nw, wo = np.array(wall.normal), np.array(wall.origin)
    t_w = np.dot(wo - pos, nw) / np.dot(d, nw)
    ell = min(t_out, t_w) - t_in
    N = int(math.ceil(ell / (0.5 * h.min())))
    r = pos + t_in * d
    eta_in = 1.0 + interp(r)[0]
    v = eta_in * d
    dt = (ell / N) / eta_in
    length = t_in
    for _ in range(N):
        A = dt * D(r)
        B = dt * D(r + 0.5 * dt * v + 0.125 * dt * A)
        C = dt * D(r + dt * v + 0.5 * dt * B)
        r_next = r + dt * (v + (A + 2.0 * B) / 6.0)
        v = v + (A + 4.0 * B + C) / 6.0
        length += np.linalg.norm(r_next - r)
        r = r_next
    t_star = np.dot(wo - r, nw) / np.dot(v, nw)
    x_w = r + t_star * v
    length += t_star * np.linalg.norm(v)
    c = np.dot(nw, v) / np.linalg.norm(v)
    x_ref = pos + t_w * d
    eu, ev = np.array(wall.eu), np.array(wall.ev)
    hit = np.array([np.dot(x_w - wo, eu), np.dot(x_w - wo, ev)])
    hit_ref = np.array([np.dot(x_ref - wo, eu), np.dot(x_ref - wo, ev)])
    return dict(I=c / length, hit=hit, disp=hit - hit_ref, N=N)


def test_one_ray_on_a_tiny_grid_matches_an_independent_python_trace(orc):
    # a 3 x 4 x 3 grid with a refractivity 100x that of air, so that rays bend visibly,
    # and a wall of constant luminance 1; pixels at the centre, edges and corners
    grid = S.Grid(n=(3, 4, 3), origin=(0.0, 0.0, 0.0), extent=(1.0, 1.2, 0.9), G=2.26e-2)
    T = (280.0 + 60.0 * np.random.default_rng(5).random((3, 4, 3))).astype(np.float32)
    cam = S.Camera(pos=(0.5, -1.5, 0.45), fwd=(0.0, 1.0, 0.0), up=(0.0, 0.0, 1.0),
                   fx=20.0, fy=20.0, cx=2.5, cy=2.5, width=5, height=5)   # all hits well inside the wall
    sc = S.Scene("tiny", grid, T, cam, S.back_wall(grid), S.Light(0, np.ones((8, 8), np.float32)),
                 S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=0))
    pix = [0, 4, 7, 12, 17, 20, 24]
    got = orc.render(sc, pix=pix, nsteps=True)
    for q, p in enumerate(pix):
        want = _py_trace_pixel(sc, p % 5, p // 5)
        assert got["nsteps"][q, 0] == want["N"]
        assert abs(got["I"][q] - want["I"]) <= 1e-12 * abs(want["I"])
        assert np.abs(got["hit"][q] - want["hit"]).max() <= 1e-12
        assert np.abs(got["disp"][q] - want["disp"]).max() <= 1e-12
    # the field bends the rays well beyond rounding, so the comparison is not vacuous
    assert np.abs(got["disp"]).max() > 1e-4
