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


# Finite-difference check of a full-size adjoint (the survey's A16 reading): dL/dT_v by
# central differences of the oracle, L(T) = sum_j w_j I_j(T), at voxels of the plume that
# some camera (or projector) ray reaches.  Each difference sums over the pixels whose rays
# pass within 3 cells of the voxel (the only ones its value reaches).  A voxel is a kink
# (a ray's stage point crosses a cell face within the step, where the trilinear field's
# derivative jumps) when its difference at h and at h/2 disagree by more than 1e-5; kinks
# are skipped, as A16 allows.  Bar: |adjoint - FD| <= 1e-4 |FD| + 1e-6 max|FD| (the second
# term is the float32 accumulation floor of voxels whose gradient is a near-cancelling sum).
FD_REL_TOL = 1e-4
FD_FLOOR = 1e-6
FD_KINK = 1e-5


def fd_check(orc, scene, g_gpu, w, nvox, rng, near):
    """Returns (adjoint, fd, kept) at nvox sampled plume voxels; asserts the A16 bar."""
    hg = np.array(scene.grid.spacing())
    origin = np.array(scene.grid.origin)
    hot = np.argwhere(scene.T > 300.0)
    rng.shuffle(hot)
    vox, pixs = [], []
    for k, j, i in hot:                       # plume voxels that some ray reaches
        c = origin + (np.array([i, j, k]) + 0.5) * hg
        pix = near(scene, c, 3.0 * hg + 1e-3)
        if len(pix):
            vox.append((k, j, i))
            pixs.append(pix)
        if len(vox) == nvox:
            break
    assert len(vox) == nvox
    T64 = scene.T.astype(np.float64)

    def fd_at(k, j, i, pix, h):
        vals = []
        for sgn in (1.0, -1.0):
            T = T64.copy()
            T[k, j, i] += sgn * h
            I = orc.render(scene.replace(T=T), pix=pix)["I"]
            vals.append(float((w.reshape(-1)[pix] * I).sum()))
        return (vals[0] - vals[1]) / (2 * h)

    fd, fd2, gp = [], [], []
    for (k, j, i), pix in zip(vox, pixs):
        fd.append(fd_at(k, j, i, pix, 1e-2))
        fd2.append(fd_at(k, j, i, pix, 5e-3))
        gp.append(g_gpu[k, j, i])
    fd, fd2, gp = np.array(fd), np.array(fd2), np.array(gp)
    scale = np.abs(fd).max()
    assert scale > 0
    kept = np.abs(fd - fd2) <= FD_KINK * np.maximum(np.abs(fd), 1e-3 * scale)
    assert kept.sum() >= 0.75 * nvox, kept.sum()
    bad = kept & (np.abs(gp - fd) > FD_REL_TOL * np.abs(fd) + FD_FLOOR * scale)
    assert bad.sum() == 0, (np.flatnonzero(bad), gp[bad], fd[bad])
    return gp, fd, kept
