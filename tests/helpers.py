"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import dataclasses

import numpy as np

# Tolerances stated by the problem: ray end positions (displacements) within 1e-6 of
# the largest displacement, intensities within 1e-4 absolute.
DISP_REL_TOL = 1e-6
I_ABS_TOL = 1e-4


def bf16_round(x):
    """float64 -> bfloat16 (round to nearest even), returned as float64 values."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0), e - 8)


def bf16_bits(x):
    v = bf16_round(x).astype(np.float32)
    return (v.view(np.uint32) >> 16).astype(np.uint16)


def gpu_render(scene, prec, hit=False, reference=False, ctx=None):
    import torch

    from paper_2509_14442_gb300 import bos

    own = ctx is None
    if own:
        ctx = bos.Context(0)
        ctx.set_scene(scene, prec)
    if reference:
        I, D, X = ctx.render_reference(disp=True, hit=hit)
    else:
        I, D, X = ctx.render(disp=True, hit=hit)
    torch.cuda.synchronize()
    ctx.status()
    out = dict(I=I.cpu().numpy().astype(np.float64), disp=D.cpu().numpy().astype(np.float64))
    if hit:
        out["hit"] = X.cpu().numpy()
    out["steps"] = ctx.last_ray_steps()
    if own:
        ctx.close()
    return out


def errors(gpu, orc, pix=None):
    gI, gD = gpu["I"], gpu["disp"]
    if pix is not None:
        gI = gI.reshape(-1)[pix]
        gD = gD.reshape(-1, 2)[pix]
    oI, oD = orc["I"], orc["disp"]
    dmax = float(np.abs(oD).max())
    return dict(I_abs=float(np.abs(gI - oI).max()),
                disp_rel=float(np.abs(gD - oD).max()) / max(dmax, 1e-300),
                disp_max=dmax)


def with_camera(scene, **kw):
    return scene.replace(camera=dataclasses.replace(scene.camera, **kw))
