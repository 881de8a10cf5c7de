"""The seeded input generators follow the stated recipe: the scene geometry of the paper's
room (Sec. 3.1-3.2), the hot-blob cube, the plume field (inlet temperature, plume radius,
noise amplitude), the random-dot texture and the binary speckle, and a seed fixes every
array bit for bit."""
import math

import numpy as np

from paper_2509_14442_gb300 import scenes as S


def test_room_geometry_is_the_papers_frame():
    g = S.room_grid((64, 64, 48))
    assert g.origin == (-1.2, 0.0, 0.0) and g.extent == (4.0, 4.0, 3.0)   # inlet wall at x = -1.2 m
    sc = S.room((64, 64, 48), 100, 100, 2, 7, field=False)
    assert sc.camera.pos == (0.85, -29.0, 1.5) and sc.light.proj.pos == (1.85, -29.0, 1.5)
    assert sc.camera.fwd == (0.0, 1.0, 0.0) and sc.light.proj.fwd == (0.0, 1.0, 0.0)
    assert sc.wall.origin[1] == 4.0 and sc.wall.normal == (0.0, 1.0, 0.0)     # back wall y = 4 m
    # the camera frames +-1.45 m of the wall around its axis: the edge pixel's ray reaches
    # 1.45 m off axis at the wall distance (33 m)
    c = sc.camera
    half = (0.5 * c.height) / c.fy * (4.0 - c.pos[1])
    assert math.isclose(half, 1.45, rel_tol=1e-12)
    assert sc.integ.max_step_vox == 0.5 and sc.integ.ckpt_every == 16


def test_blob_cube_recipe():
    sc = S.blob_cube()
    assert sc.grid.n == (32, 32, 32) and sc.grid.extent == (1.0, 1.0, 1.0)
    T = sc.T.astype(np.float64)
    assert T.min() >= 293.0 and 300.0 < T.max() <= 301.0                    # +8 K peak at the blob
    k, j, i = np.unravel_index(np.argmax(T), T.shape)
    centre = (np.array([i, j, k]) + 0.5) / 32
    assert np.all(centre > 0.33) and np.all(centre < 0.67)                   # seeded in [0.35, 0.65]^3
    # sigma 0.15 m: 0.15 m from the peak cell along x the excess has fallen to exp(-1/2)
    x = (np.arange(32) + 0.5) / 32
    prof = T[k, j, :] - 293.0
    c = x[i]
    assert abs(np.interp(c + 0.15, x, prof) / prof[i] - math.exp(-0.5)) < 0.05
    assert sc.camera.width == sc.camera.height == 64 and sc.integ.fixed_steps == 128
    tex = sc.light.pattern
    assert tex.shape == (64, 64) and set(np.unique(tex)) <= {0.0, 1.0}
    lit = int(tex.sum())
    assert 20 <= lit <= 44                                   # 1 % fill: 10 dots of 2x2 texels


def test_plume_field_recipe():
    g = S.room_grid((48, 48, 36))
    T = S.plume_field(g, 11).astype(np.float64)
    assert T.shape == (36, 48, 48) and T.dtype == np.float64
    # peak below the 310 K inlet (plus the 0.3 K noise); the plume is at least several kelvin hot
    assert 300.0 < T.max() <= 310.3
    # the noise alone stays within +-0.3 K: far from the plume the field is ambient +- 0.3
    prm = S.plume_params(11)
    assert abs(prm["p0"][0] - (-1.2)) < 1e-12 and 1.5 <= prm["lam"] <= 3.0
    assert T.min() >= 293.0 - 0.3 - 1e-6
    # with the inlet at ambient only the noise is left: four octaves, amplitudes summing to 0.3 K
    noise = S.plume_field(g, 11, t_inlet=293.0).astype(np.float64) - 293.0
    assert 0.2 < np.abs(noise).max() <= 0.3 + 1e-4
    # a seed fixes the field bit for bit; another seed moves the plume
    assert np.array_equal(S.plume_field(g, 11), S.plume_field(g, 11))
    assert not np.array_equal(S.plume_field(g, 11), S.plume_field(g, 12))


def test_speckle_and_dots_are_seeded_binary_patterns():
    sp = S.speckle(512, 512, 9)
    assert sp.shape == (512, 512) and set(np.unique(sp)) == {0.0, 1.0}
    assert abs(sp.mean() - 0.5) < 0.01                                      # p = 1/2
    assert np.array_equal(sp, S.speckle(512, 512, 9)) and not np.array_equal(sp, S.speckle(512, 512, 10))
    tex = S.dot_texture(64, 64, 0.01, 2, 3)
    assert np.array_equal(tex, S.dot_texture(64, 64, 0.01, 2, 3))
