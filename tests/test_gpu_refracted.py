"""Refracted projector connection (light mode 2, Sec. 2.3) on the CUDA path: forward
parity with the FP64 oracle, the connection's own effect on the image against the
oracle's, and dL/dT through the projector rays."""
import numpy as np
import pytest

from helpers import DISP_REL_TOL, I_ABS_TOL, errors, gpu_render
from paper_2509_14442_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GRAD_REL_L2 = 1e-4   # as for the camera-only adjoint


@pytest.fixture(scope="module")
def bos():
    from paper_2509_14442_gb300 import bos as B
    B.lib()
    return B


def refracted(sc, iters=1, boost=4.0):
    """The room scene lit through a refracted projector connection, with the plume's excess
    temperature scaled so the projector rays bend visibly at these small grids."""
    T = (S.T_AMBIENT + boost * (sc.T.astype(np.float64) - S.T_AMBIENT)).astype(np.float32)
    return sc.replace(T=T, light=S.Light(2, sc.light.pattern, sc.light.proj, connect_iters=iters))


def straight_connection(sc):
    return sc.replace(light=S.Light(1, sc.light.pattern, sc.light.proj))


@pytest.mark.parametrize("spp,iters", [(1, 1), (4, 1), (1, 3)])
def test_refracted_forward_matches_oracle(bos, orc, spp, iters):
    sc = refracted(S.room((48, 48, 36), 83, 61, spp, 4100 + spp), iters)
    g = gpu_render(sc, bos.BOS_PREC_FP32_COMP)
    o = orc.render(sc)
    e = errors(g, o)
    assert e["I_abs"] <= I_ABS_TOL, e
    assert e["disp_rel"] <= DISP_REL_TOL, e
    # the connection's own effect on the image (refracted minus straight), GPU vs oracle
    g1 = gpu_render(straight_connection(sc), bos.BOS_PREC_FP32_COMP)
    o1 = orc.render(straight_connection(sc))
    dg, do = g["I"] - g1["I"], o["I"] - o1["I"]
    assert np.abs(do).max() > 1e-4                        # well above the float32 intensity error
    assert np.abs(dg - do).max() <= 0.02 * np.abs(do).max()
    # the projector rays are traced and counted
    assert g["steps"] > g1["steps"]


def test_refracted_bf16_store_matches_oracle_on_the_bf16_field(bos, orc):
    from helpers import bf16_round

    sc = refracted(S.room((40, 40, 30), 64, 48, 1, 4150))
    g = gpu_render(sc, bos.BOS_PREC_BF16_COMP)
    de = orc.deta_from_T(sc.grid, sc.T)
    field_q = orc.NodeField(bf16_round(de), bf16_round(orc.grad_from_deta(sc.grid, de)))
    o = orc.render(sc, field=field_q)
    e = errors(g, o)
    assert e["I_abs"] <= I_ABS_TOL and e["disp_rel"] <= DISP_REL_TOL, e


def gpu_grad(bos, scene, w):
    ctx = bos.Context(0)
    ctx.set_scene(scene, bos.BOS_PREC_FP32_COMP)
    ctx.render(disp=False, save_for_backward=True)
    dT = ctx.backward(torch.as_tensor(np.ascontiguousarray(w, dtype=np.float32), device="cuda"))
    torch.cuda.synchronize()
    ctx.status()
    out = dT.cpu().numpy().astype(np.float64)
    ctx.close()
    return out


@pytest.mark.parametrize("spp", [1, 3])
def test_camera_rays_are_identical_with_and_without_the_cell_cache(bos, spp):
    """The Sharma tracer on the paired float32 store reuses each ray's last cell; the kernels
    of the refracted connection trace their camera rays without that cache.  The camera
    rays' wall hits and displacements do not depend on the light, so the two renders of one
    scene must agree bit for bit: the cache changes where the records come from, not the
    arithmetic."""
    sc = refracted(S.room((64, 64, 48), 96, 72, spp, 4150 + spp))
    a = gpu_render(straight_connection(sc), bos.BOS_PREC_FP32_COMP, hit=True)   # cached tracer
    b = gpu_render(sc, bos.BOS_PREC_FP32_COMP, hit=True)                        # uncached tracer
    assert np.abs(a["disp"]).max() > 0
    assert np.array_equal(a["disp"], b["disp"])
    assert np.array_equal(a["hit"], b["hit"])


@pytest.mark.parametrize("spp", [1, 2])
def test_refracted_gradient_matches_oracle(bos, orc, spp):
    sc = refracted(S.room((40, 40, 30), 70, 52, spp, 4200 + spp))
    w = np.random.default_rng(spp).standard_normal((52, 70))
    gg = gpu_grad(bos, sc, w)
    go = orc.grad(sc, w)
    rel = float(np.linalg.norm(gg - go) / np.linalg.norm(go))
    assert rel <= GRAD_REL_L2, rel
    # and the projector rays' part of it is a visible share of the gradient
    g1 = orc.grad(straight_connection(sc), w)
    assert np.linalg.norm(go - g1) > 0.1 * np.linalg.norm(go)


def test_refracted_backward_limits_are_reported(bos):
    sc = refracted(S.room((24, 24, 18), 32, 24, 1, 4300), iters=2)
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    with pytest.raises(bos.BosError) as e:
        ctx.render(save_for_backward=True)
    assert e.value.status == bos.BOS_ERR_UNIMPLEMENTED
    ctx.render()                                           # the forward alone is fine
    torch.cuda.synchronize()
    ctx.status()
    ctx.close()
    ctx = bos.Context(0)
    ctx.set_scene(refracted(S.room((24, 24, 18), 32, 24, 1, 4300)), bos.BOS_PREC_FP64)
    with pytest.raises(bos.BosError) as e:
        ctx.render()
    assert e.value.status == bos.BOS_ERR_UNIMPLEMENTED
    ctx.close()


# ------------------------------------------------- full size (the benchmarked launch)

@pytest.mark.slow
def test_refracted_full_size_sampled(bos, orc):
    sc = refracted(S.room_adjoint(), boost=1.0)      # 256x256x192, 2048^2, 1 spp, unscaled plume
    g = gpu_render(sc, bos.BOS_PREC_FP32_COMP)
    pix = np.random.default_rng(5).choice(sc.pixels, 400, replace=False)
    e = errors(g, orc.render(sc, pix=pix), pix)
    assert e["I_abs"] <= I_ABS_TOL and e["disp_rel"] <= DISP_REL_TOL, e


def _box_hits(origin, d, center, margin):
    lo, hi = np.asarray(center) - margin, np.asarray(center) + margin
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - origin) / d
        t1 = (hi - origin) / d
    tmin = np.nanmax(np.minimum(t0, t1), axis=-1)
    tmax = np.nanmin(np.maximum(t0, t1), axis=-1)
    return (tmin <= tmax).reshape(-1)


def _pixels_near_either_ray(scene, center, margin):
    """Pixels whose straight camera ray, or the projector ray aimed at that ray's wall hit,
    passes within `margin` (a box) of `center`: the only pixels a voxel there can change."""
    c, w, P = scene.camera, scene.wall, np.asarray(scene.light.proj.pos, dtype=np.float64)
    px, py = np.meshgrid(np.arange(c.width) + 0.5, np.arange(c.height) + 0.5, indexing="xy")
    fwd, up = np.array(c.fwd), np.array(c.up)
    right = np.cross(fwd, up)
    d = ((px - c.cx) / c.fx)[..., None] * right - ((py - c.cy) / c.fy)[..., None] * up + fwd
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    pos, n = np.array(c.pos), np.array(w.normal)
    tw = ((np.array(w.origin) - pos) @ n) / (d @ n)
    xw = pos + tw[..., None] * d
    dp = xw - P
    dp /= np.linalg.norm(dp, axis=-1, keepdims=True)
    hit = _box_hits(pos, d, center, margin) | _box_hits(P, dp, center, margin)
    return np.flatnonzero(hit)


@pytest.mark.slow
def test_refracted_adjoint_full_size_against_oracle_finite_differences(bos, orc):
    # the benchmarked refracted launch: dL/dT at 16 seeded plume voxels against central
    # differences of the oracle over the pixels the voxel can reach through the camera ray or
    # the projector ray (helpers.fd_check: A16's bar, kinks skipped)
    from helpers import fd_check

    sc = refracted(S.room_adjoint(), boost=1.0)
    rng = np.random.default_rng(65)
    w = rng.standard_normal((sc.camera.height, sc.camera.width))
    fd_check(orc, sc, gpu_grad(bos, sc, w), w, 16, rng, _pixels_near_either_ray)

