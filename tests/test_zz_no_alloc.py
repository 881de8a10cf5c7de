"""bos_render_noalloc, the forward render for callers that must not allocate device
memory (a latency-critical loop where cudaMalloc/cudaFree would synchronise the device,
or a process whose device memory belongs to another allocator): through the C ABI its
images equal those of the allocating path (bos_set_grid + bos_render), on two calls in a
row whose scratch contents differ, and grids too big for its fixed scratch are refused.

This file is collected last so that a run stopping at the first failure has run every
other test before it."""
import numpy as np
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


def allocating(bos, sc, T, pattern):
    ctx = bos.Context(0)
    ctx.set_grid(sc.grid, T, bos.BOS_PREC_FP32_COMP)
    ctx.set_geometry(sc.camera, sc.wall, sc.light, sc.integ, pattern=pattern)
    I, D, _ = ctx.render(disp=True)
    torch.cuda.synchronize()
    ctx.status()
    out = I.clone(), D.clone()
    ctx.close()
    return out


def no_alloc(bos, sc, T, pattern):
    H, W = sc.camera.height, sc.camera.width
    I = torch.full((H, W), -1.0, device="cuda")
    D = torch.full((H, W, 2), -1.0, device="cuda")
    bos.bos_render_noalloc(bos.grid_desc(sc.grid, bos.BOS_PREC_FP32_COMP), T.data_ptr(), bos.camera_desc(sc.camera),
                           bos.wall_desc(sc.wall), bos.light_desc(sc.light), pattern.data_ptr(),
                           bos.integ_desc(sc.integ), I.data_ptr(), D.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return I, D


def test_no_alloc_render_matches_the_allocating_render_twice_in_a_row(bos):
    scenes = [S.room((64, 64, 48), 96, 80, 2, 5101), S.blob_cube(), S.room((128, 128, 96), 64, 48, 1, 5102)]
    inputs = [(sc, torch.as_tensor(sc.T, device="cuda"), torch.as_tensor(sc.light.pattern, device="cuda"))
              for sc in scenes]
    refs = [allocating(bos, *x) for x in inputs]
    for _ in range(2):                     # every scene rendered twice, each time after another one
        for (sc, T, pat), (I0, D0) in zip(inputs, refs):
            I, D = no_alloc(bos, sc, T, pat)
            assert float((I - I0).abs().max()) <= I_ABS_TOL
            dmax = float(D0.abs().max())
            assert dmax > 0 and float((D - D0).abs().max()) <= DISP_REL_TOL * dmax
            # same kernels on the same inputs: in fact identical
            assert torch.equal(I, I0) and torch.equal(D, D0)


def test_no_alloc_refuses_grids_beyond_its_scratch(bos):
    sc = S.room((256, 256, 192), 32, 32, 1, 5103, field=False)      # a 358 MB field store
    T = torch.full((192, 256, 256), 293.0, device="cuda")
    pat = torch.as_tensor(sc.light.pattern, device="cuda")
    with pytest.raises(bos.BosError) as e:
        no_alloc(bos, sc, T, pat)
    assert e.value.status == bos.BOS_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
