"""bos_render_noalloc, the forward render for callers that must not allocate device
memory (a latency-critical loop where cudaMalloc/cudaFree would synchronise the device,
or a process whose device memory belongs to another allocator): through the C ABI its
images equal those of the allocating path (bos_set_grid + bos_set_geometry + bos_render)
for every precision, light mode and integrator, on two calls in a row whose scratch
contents differ; its device status reads back clean; grids too big for its fixed scratch
are refused.

This file is collected last so that a run stopping at the first failure has run every
other test before it."""
import pytest

from paper_2509_14442_gb300 import scenes as S
from helpers import DISP_REL_TOL, I_ABS_TOL

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def bos():
    from paper_2509_14442_gb300 import bos as B
    B.lib()
    return B


def allocating(bos, sc, T, pattern, prec):
    ctx = bos.Context(0)
    ctx.set_grid(sc.grid, T, prec)
    ctx.set_geometry(sc.camera, sc.wall, sc.light, sc.integ, pattern=pattern)
    I, D, _ = ctx.render(disp=True)
    torch.cuda.synchronize()
    ctx.status()
    out = I.clone(), D.clone()
    ctx.close()
    return out


def no_alloc(bos, sc, T, pattern, prec, disp=True):
    H, W = sc.camera.height, sc.camera.width
    I = torch.full((H, W), -1.0, device="cuda")
    D = torch.full((H, W, 2), -1.0, device="cuda") if disp else None
    bos.bos_render_noalloc(bos.grid_desc(sc.grid, prec), T.data_ptr(), bos.camera_desc(sc.camera),
                           bos.wall_desc(sc.wall), bos.light_desc(sc.light), pattern.data_ptr(),
                           bos.integ_desc(sc.integ), I.data_ptr(), D.data_ptr() if disp else None,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    bos.bos_noalloc_status()
    return I, D


def quasi(sc):
    return sc.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=2, ckpt_every=16))


def refracted(sc):
    return sc.replace(light=S.Light(2, sc.light.pattern, sc.light.proj, connect_iters=1))


def cases(bos):
    """(scene, precision, with displacement) -- every store type, both light kinds,
    all three integrators, and one call without the displacement output."""
    room = S.room((64, 64, 48), 96, 80, 2, 5101)
    big = S.room((128, 128, 96), 64, 48, 1, 5102)
    return [(room, bos.BOS_PREC_FP32_COMP, True), (S.blob_cube(), bos.BOS_PREC_FP32_COMP, True),
            (big, bos.BOS_PREC_FP32_COMP, False), (room, bos.BOS_PREC_BF16_COMP, True),
            (room, bos.BOS_PREC_FP64, True), (room, bos.BOS_PREC_FP32, True),
            (quasi(room), bos.BOS_PREC_FP32_COMP, True), (refracted(room), bos.BOS_PREC_FP32_COMP, True),
            (S.blob_cube().replace(integ=S.Integrator(fixed_steps=128, max_step_vox=0.5, integrator=1,
                                                       ckpt_every=16)), bos.BOS_PREC_FP32_COMP, True)]


def test_no_alloc_render_matches_the_allocating_render_twice_in_a_row(bos):
    inputs = [(sc, torch.as_tensor(sc.T, device="cuda"), torch.as_tensor(sc.light.pattern, device="cuda"), prec, disp)
              for sc, prec, disp in cases(bos)]
    refs = [allocating(bos, sc, T, pat, prec) for sc, T, pat, prec, _ in inputs]
    for _ in range(2):                     # every case rendered twice, each time after another one
        for (sc, T, pat, prec, disp), (I0, D0) in zip(inputs, refs):
            I, D = no_alloc(bos, sc, T, pat, prec, disp)
            assert float((I - I0).abs().max()) <= I_ABS_TOL
            if disp:
                dmax = float(D0.abs().max())
                assert dmax > 0 and float((D - D0).abs().max()) <= DISP_REL_TOL * dmax
            # same kernels on the same inputs: in fact identical
            assert torch.equal(I, I0) and (not disp or torch.equal(D, D0))


def test_no_alloc_refuses_grids_beyond_its_scratch(bos):
    sc = S.room((256, 256, 192), 32, 32, 1, 5103, field=False)      # a 717 MB field store
    T = torch.full((192, 256, 256), 293.0, device="cuda")
    pat = torch.as_tensor(sc.light.pattern, device="cuda")
    with pytest.raises(bos.BosError) as e:
        no_alloc(bos, sc, T, pat, bos.BOS_PREC_FP32_COMP)
    assert e.value.status == bos.BOS_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
