"""Parity of the CUDA forward path (steps a1-a5) with the FP64 oracle."""
import numpy as np
import pytest

from paper_2509_14442_gb300 import scenes as S
from helpers import DISP_REL_TOL, I_ABS_TOL, bf16_bits, bf16_round, errors, gpu_render, with_camera

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def bos():
    from paper_2509_14442_gb300 import bos as B
    B.lib()
    return B


# ------------------------------------------------------------------ a1: store, bit-exact

@pytest.mark.parametrize("n", [(32, 32, 32), (13, 21, 9), (2, 2, 2), (128, 128, 96)])
@pytest.mark.parametrize("prec", ["fp32_comp", "bf16_comp", "fp64"])
def test_store_is_bit_exact(bos, orc, n, prec):
    g = S.Grid(n=n, origin=(-0.3, 0.2, 0.1), extent=(1.1, 0.7, 0.9))
    T = S.plume_field(S.room_grid(n), 31) if n[0] >= 64 else (
        293.0 + 20.0 * np.random.default_rng(1).random((n[2], n[1], n[0]))).astype(np.float32)
    ctx = bos.Context(0)
    ctx.set_grid(g, torch.as_tensor(T, device="cuda"), bos.PRECISIONS[prec])
    got = ctx.export_nodes().cpu().numpy()
    ctx.close()
    de = orc.deta_from_T(g, T.astype(np.float64))
    gr = orc.grad_from_deta(g, de)
    want = np.concatenate([de[..., None], gr], -1)
    if prec == "fp64":
        assert np.array_equal(got, want)
    elif prec == "fp32_comp":
        assert np.array_equal(got.view(np.uint32), want.astype(np.float32).view(np.uint32))
    else:
        assert np.array_equal(got.view(np.uint16), bf16_bits(want))


# ------------------------------------------------------------------ a2: integer decisions

@pytest.mark.parametrize("scene", ["blob", "paper", "room_small_jitter", "spp3"])
def test_step_counts_bit_exact(bos, orc, scene):
    sc = {"blob": lambda: S.blob_cube(),
          "paper": lambda: S.paper_sensor(),
          "room_small_jitter": lambda: S.room((40, 36, 30), 37, 29, 4, 77),
          "spp3": lambda: S.room((24, 24, 18), 21, 13, 3, 78)}[scene]()
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    n = ctx.ray_steps().cpu().numpy()
    ctx.close()
    o = orc.render(sc, nsteps=True)["nsteps"].reshape(-1)
    assert np.array_equal(n, o)
    assert (n > 0).mean() > 0.5          # most rays are traced (wide views miss at the corners)


# ------------------------------------------------------------------ a2-a5: images

def _check(gpu, orc_out, disp_tol=DISP_REL_TOL, i_tol=I_ABS_TOL):
    e = errors(gpu, orc_out)
    assert e["disp_max"] > 0
    assert e["I_abs"] <= i_tol, e
    assert e["disp_rel"] <= disp_tol, e
    return e


@pytest.mark.parametrize("integrator", [0, 1])
@pytest.mark.parametrize("prec", ["fp32_comp", "fp64"])
def test_blob_cube_parity(bos, orc, prec, integrator):
    sc = S.blob_cube(integrator=integrator)
    o = orc.render(sc, nsteps=True)
    g = gpu_render(sc, bos.PRECISIONS[prec], hit=True)
    # Both FP64 integrations carry up to ~N * 10 * 2^-53 * |r| = 3e-13 m of rounding on this
    # 1 m path (N = 128), i.e. ~6e-8 of the blob's largest displacement (4.6e-6 m).
    e = _check(g, o, disp_tol=2e-7 if prec == "fp64" else DISP_REL_TOL)
    assert g["steps"] == int(o["nsteps"].sum())
    hit_err = float(np.abs(g["hit"] - o["hit"]).max())
    assert hit_err <= DISP_REL_TOL * e["disp_max"]


def test_paper_sensor_parity(bos, orc):
    sc = S.paper_sensor()          # 64^3 room grid, 100 x 100 sensor, 2 samples per pixel
    o = orc.render(sc)
    _check(gpu_render(sc, bos.BOS_PREC_FP32_COMP), o)


@pytest.mark.parametrize("shape", [(128, 128, 96), (61, 47, 35)])
def test_room_parity_ragged(bos, orc, shape):
    # 203 x 141 pixels: ragged against the 4 x 2 pixel tiles of 4 samples
    sc = S.room(shape, 203, 141, 4, 2600 + shape[0])
    o = orc.render(sc)
    _check(gpu_render(sc, bos.BOS_PREC_FP32_COMP), o)


def test_bf16_store_parity_against_dequantised_field(bos, orc):
    sc = S.room((64, 64, 48), 96, 80, 2, 2711)
    de = orc.deta_from_T(sc.grid, sc.T.astype(np.float64))
    gr = orc.grad_from_deta(sc.grid, de)
    field_q = orc.NodeField(bf16_round(de), bf16_round(gr))
    o = orc.render(sc, field=field_q)
    _check(gpu_render(sc, bos.BOS_PREC_BF16_COMP), o)


def test_plain_fp32_is_worse_than_compensated(bos, orc):
    sc = S.room((64, 64, 48), 64, 48, 1, 2712)
    o = orc.render(sc)
    e32 = errors(gpu_render(sc, bos.BOS_PREC_FP32), o)
    ec = errors(gpu_render(sc, bos.BOS_PREC_FP32_COMP), o)
    assert ec["disp_rel"] <= DISP_REL_TOL
    assert e32["disp_rel"] > 10 * ec["disp_rel"]
    assert e32["I_abs"] < 1e-2


def test_reference_image(bos, orc):
    sc = S.room((32, 32, 24), 50, 40, 4, 2713)
    o = orc.render(sc, straight=True)
    g = gpu_render(sc, bos.BOS_PREC_FP32_COMP, reference=True)
    assert float(np.abs(g["I"] - o["I"]).max()) <= 1e-5      # float32 luminance lookup; bound 1e-4
    assert float(np.abs(g["disp"]).max()) <= 1e-12


@pytest.mark.parametrize("spp", [1, 3, 32])
def test_sample_counts(bos, orc, spp):
    sc = S.room((32, 32, 24), 19, 11, spp, 2714 + spp)
    o = orc.render(sc)
    _check(gpu_render(sc, bos.BOS_PREC_FP32_COMP), o)


def test_single_pixel_and_rays_missing_the_box(bos, orc):
    sc = S.blob_cube(n=16, width=1, height=1, steps=16)
    _check(gpu_render(sc, bos.BOS_PREC_FP32_COMP), orc.render(sc), disp_tol=1.0)   # disp may be ~0
    # a wide camera: border rays pass beside the cube and go straight to the wall plane
    wide = with_camera(S.blob_cube(n=16, width=48, height=40, steps=32), fx=12.0, fy=12.0, cx=24.0, cy=20.0)
    o = orc.render(wide, nsteps=True)
    assert (o["nsteps"] == 0).any() and (o["nsteps"] > 0).any()
    _check(gpu_render(wide, bos.BOS_PREC_FP32_COMP), o)


def test_wide_view_with_tied_slab_faces(bos, orc):
    """A 65 x 65 image centred on the cube's x-z centre line with a wide view: on both image
    diagonals |d_x| = |d_z| exactly, so a ray leaves through an x face and a z face at the
    same distance (a tie the slab test breaks in axis order); the centre row and column have
    d_z = 0 or d_x = 0; border rays miss the cube.  Step counts are bit-exact and images
    within the usual tolerances: the slab test breaks ties like the oracle's plain float64
    evaluation, and the straight reference render (which skips the slab test) agrees too."""
    base = S.blob_cube(n=24, width=65, height=65, steps=32)
    sc = with_camera(base, fx=40.0, fy=40.0, cx=32.5, cy=32.5).replace(
        integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=0, ckpt_every=16))
    o = orc.render(sc, nsteps=True)
    n_orc = o["nsteps"].reshape(65, 65)
    diag = np.array([n_orc[i, i] for i in range(65)])
    assert (diag > 0).sum() >= 20 and (n_orc == 0).any()
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
    n = ctx.ray_steps().cpu().numpy()
    ctx.close()
    assert np.array_equal(n, o["nsteps"].reshape(-1))
    _check(gpu_render(sc, bos.BOS_PREC_FP32_COMP), o)
    o_ref = orc.render(sc, straight=True)
    g_ref = gpu_render(sc, bos.BOS_PREC_FP32_COMP, reference=True)
    assert float(np.abs(g_ref["I"] - o_ref["I"]).max()) <= 1e-5


# ------------------------------------------------------------------ full sizes, sampled pixels

@pytest.mark.slow
def test_room_forward_full_size_sampled(bos, orc):
    sc = S.room_forward()            # 128x128x96, 1024^2, 4 spp: the benchmarked launch
    g = gpu_render(sc, bos.BOS_PREC_FP32_COMP)
    pix = np.random.default_rng(0).choice(sc.pixels, 1500, replace=False)
    o = orc.render(sc, pix=pix)
    e = errors(g, o, pix)
    assert e["I_abs"] <= I_ABS_TOL and e["disp_rel"] <= DISP_REL_TOL, e
    assert np.isfinite(g["I"]).all() and g["I"].max() > 0


@pytest.mark.slow
def test_room_adjoint_scene_full_size_sampled(bos, orc):
    sc = S.room_adjoint()            # 256x256x192, 2048^2, 1 spp
    g = gpu_render(sc, bos.BOS_PREC_FP32_COMP)
    pix = np.random.default_rng(1).choice(sc.pixels, 600, replace=False)
    o = orc.render(sc, pix=pix, nsteps=True)
    e = errors(g, o, pix)
    assert e["I_abs"] <= I_ABS_TOL and e["disp_rel"] <= DISP_REL_TOL, e


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["bf16_comp", "fp64"])
def test_precision_variants_full_size_sampled(bos, orc, prec):
    # the precision configuration: the 256x256x192 scene with the BF16 store (held to the
    # bar against the oracle on the dequantised field, which isolates the integrator) and
    # with the plain float64 tracer
    sc = S.room_adjoint()
    g = gpu_render(sc, bos.PRECISIONS[prec])
    pix = np.random.default_rng(11).choice(sc.pixels, 400, replace=False)
    field = None
    if prec == "bf16_comp":
        de = orc.deta_from_T(sc.grid, sc.T.astype(np.float64))
        field = orc.NodeField(bf16_round(de), bf16_round(orc.grad_from_deta(sc.grid, de)))
    e = errors(g, orc.render(sc, field=field, pix=pix), pix)
    assert e["I_abs"] <= I_ABS_TOL and e["disp_rel"] <= (2e-7 if prec == "fp64" else DISP_REL_TOL), e


# ------------------------------------------------------------------ quasi-linear tracing (Sec. 2.2)

@pytest.mark.parametrize("prec", ["fp32_comp", "fp64", "bf16_comp"])
def test_quasi_linear_parity(bos, orc, prec):
    sc = S.room((96, 96, 72), 121, 97, 2, 2800)
    sc = sc.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=2))
    if prec == "bf16_comp":
        de = orc.deta_from_T(sc.grid, sc.T.astype(np.float64))
        o = orc.render(sc, field=orc.NodeField(bf16_round(de), bf16_round(orc.grad_from_deta(sc.grid, de))))
    else:
        o = orc.render(sc)
    _check(gpu_render(sc, bos.PRECISIONS[prec]), o, disp_tol=2e-7 if prec == "fp64" else DISP_REL_TOL)


@pytest.mark.slow
def test_quasi_linear_full_size_sampled(bos, orc):
    sc = S.room_adjoint()
    sc = sc.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=2))
    g = gpu_render(sc, bos.BOS_PREC_FP32_COMP)
    pix = np.random.default_rng(3).choice(sc.pixels, 600, replace=False)
    e = errors(g, orc.render(sc, pix=pix), pix)
    assert e["I_abs"] <= I_ABS_TOL and e["disp_rel"] <= DISP_REL_TOL, e


# ------------------------------------------------------------------ measurement probes

def test_fma_probe_rates_are_physical(bos):
    """The arithmetic-roofline probe: its flop count matches its launch shape, and the
    rates sit within a factor of the GPU's FMA unit counts (no folded-away work)."""
    sink = torch.zeros(1, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rates = {}
    for kind, reps in ((0, 2000), (1, 2000), (2, 50)):
        bos.bos_probe_fma(kind, reps, sink.data_ptr(), sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        flops = bos.bos_probe_fma(kind, reps, sink.data_ptr(), sp)
        e1.record()
        e1.synchronize()
        assert flops == 2 * (2 if kind == 1 else 1) * sms * 4 * 256 * reps * 16 * 8
        rates[kind] = flops / (e0.elapsed_time(e1) * 1e-3)
    fp32_units = sms * 128 * 2 * 2.2e9          # above any boost clock of this part
    assert 0.3 * fp32_units < rates[0] <= 1.05 * fp32_units
    assert 0.3 * fp32_units < rates[1] <= 2.1 * fp32_units
    assert 0.0 < rates[2] < rates[0]
    assert sink.item() == 0.0


def test_l1_probe_is_faster_than_l2_and_counts_its_bytes(bos):
    """The L1 gather-roofline probe: its byte count matches its launch shape, and reading a
    64 KiB L1-resident buffer is faster than streaming a 24 MiB buffer from L2."""
    sp = torch.cuda.current_stream().cuda_stream
    sink = torch.zeros(1, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        return out, e0.elapsed_time(e1) * 1e-3

    small = torch.ones(16384, device="cuda")
    nread, t1 = timed(lambda: bos.bos_probe_read_l1(small.data_ptr(), 65536, 100, sink.data_ptr(), sp))
    assert nread == sms * 4 * 100 * 65536
    big = torch.ones(6 * 2 ** 20, device="cuda")
    _, t2 = timed(lambda: bos.bos_probe_read(big.data_ptr(), 24 * 2 ** 20, 20, sink.data_ptr(), sp))
    l1, l2 = nread / t1, 24 * 2 ** 20 * 20 / t2
    assert l1 > l2
    assert l1 < 4 * 128 * sms * 2.2e9            # far above any per-SM load path of this part
    with pytest.raises(bos.BosError):
        bos.bos_probe_read_l1(small.data_ptr(), 65536 + 32, 1, sink.data_ptr(), sp)
    assert sink.item() == 0.0
