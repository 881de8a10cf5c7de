"""Pixel-subset renders and their gradient (the paper's reconstruction draws random
minibatches of BOS pixels, Sec. 3.2): a subset render equals the whole-image render at
those pixels, and its gradient equals the oracle's for the seed placed on those pixels."""
import numpy as np
import pytest

from paper_2509_14442_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GRAD_REL_L2 = 1e-4


@pytest.fixture(scope="module")
def bos():
    from paper_2509_14442_gb300 import bos as B
    B.lib()
    return B


@pytest.mark.parametrize("spp", [1, 4, 3])
def test_subset_render_equals_whole_image(bos, spp):
    sc = S.room((48, 48, 36), 83, 61, spp, 3500 + spp)
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    I, D, _ = ctx.render(disp=True)
    rng = np.random.default_rng(spp)
    pix = rng.integers(0, sc.pixels, 777).astype(np.int32)
    pix[:5] = pix[5]                                    # repeats are allowed
    pt = torch.as_tensor(pix, device="cuda")
    Ip, Dp = ctx.render_pixels(pt, disp=True)
    torch.cuda.synchronize()
    ctx.status()
    assert torch.equal(Ip, I.reshape(-1)[pt.long()])
    assert torch.equal(Dp, D.reshape(-1, 2)[pt.long()])
    ctx.close()


@pytest.mark.parametrize("integrator", [0, 2])
def test_subset_gradient_matches_oracle(bos, orc, integrator):
    sc = S.room((40, 40, 30), 70, 52, 1, 3600)
    sc = sc.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=integrator))
    rng = np.random.default_rng(9)
    pix = np.unique(rng.integers(0, sc.pixels, 900)).astype(np.int32)
    w = rng.standard_normal(len(pix))
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    ctx.render_pixels(torch.as_tensor(pix, device="cuda"), save_for_backward=True)
    g = ctx.backward(torch.as_tensor(w.astype(np.float32), device="cuda"))
    torch.cuda.synchronize()
    ctx.status()
    ctx.close()
    wfull = np.zeros(sc.pixels)
    wfull[pix] = w
    go = orc.grad(sc, wfull.reshape(sc.camera.height, sc.camera.width))
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - go) <= GRAD_REL_L2 * np.linalg.norm(go)


def test_out_of_range_pixels_are_skipped_and_flagged(bos):
    sc = S.room((32, 32, 24), 40, 30, 1, 3700)
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    I, _, _ = ctx.render(disp=False)
    pix = torch.tensor([5, -1, 17, 40 * 30, 1199], dtype=torch.int32, device="cuda")
    Ip, _ = ctx.render_pixels(pix)
    torch.cuda.synchronize()
    with pytest.raises(bos.BosError) as e:
        ctx.status()
    assert e.value.status == bos.BOS_ERR_DEVICE_CHECK
    good = torch.tensor([0, 2, 4], device="cuda")
    assert torch.equal(Ip[good], I.reshape(-1)[pix[good].long()])
    ctx.close()


def test_empty_and_single_pixel_minibatches(bos):
    # an empty list is refused on the host (nothing launched, the context stays usable);
    # a one-pixel list is a warp tile with 31 idle lanes
    sc = S.room((32, 32, 24), 40, 30, 1, 3800)
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    I, D, _ = ctx.render(disp=True)
    with pytest.raises(bos.BosError) as e:
        ctx.render_pixels(torch.empty((0,), dtype=torch.int32, device="cuda"))
    assert e.value.status == bos.BOS_ERR_INVALID_ARG
    for p in (0, 611, 40 * 30 - 1):
        pix = torch.tensor([p], dtype=torch.int32, device="cuda")
        Ip, Dp = ctx.render_pixels(pix, disp=True)
        torch.cuda.synchronize()
        ctx.status()
        assert torch.equal(Ip, I.reshape(-1)[pix.long()])
        assert torch.equal(Dp, D.reshape(-1, 2)[pix.long()])
    ctx.close()
