"""Reconstruction pieces (Sec. 2.4, Sec. 3.2): pixel minibatch sampler, minibatch L_BOS,
AdaBelief update, and a short voxel reconstruction whose image loss must fall."""
import numpy as np
import pytest

from paper_2509_14442_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def bos():
    from paper_2509_14442_gb300 import bos as B
    B.lib()
    return B


def sp():
    return torch.cuda.current_stream().cuda_stream


def test_pixel_sampler_matches_splitmix64(bos, orc):
    n, npx, seed, draw = 1000, 123457, 77, 3
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    bos.bos_sample_pixels(pix.data_ptr(), n, npx, seed, draw, sp())
    got = pix.cpu().numpy()
    want = [(orc.splitmix64_output(seed, draw * n + k + 1) * npx) >> 64 for k in range(n)]
    assert np.array_equal(got, np.array(want))
    assert got.min() >= 0 and got.max() < npx
    # the same draw with its number read from device memory (1 + 2), and a counter bump
    ctr = torch.tensor([1], dtype=torch.int64, device="cuda")
    bos.bos_counter_add(ctr.data_ptr(), 1, sp())
    pix2 = torch.empty_like(pix)
    bos.bos_sample_pixels(pix2.data_ptr(), n, npx, seed, 1, sp(), draw_dev=ctr.data_ptr())
    torch.cuda.synchronize()
    assert ctr.item() == 2
    assert torch.equal(pix2, pix)


def test_minibatch_loss_and_adabelief_match_torch(bos):
    rng = np.random.default_rng(0)
    target = torch.as_tensor(rng.random((50, 60)).astype(np.float32), device="cuda")
    pix = torch.as_tensor(rng.integers(0, 3000, 400).astype(np.int32), device="cuda")
    I = torch.as_tensor(rng.random(400).astype(np.float32), device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(400, device="cuda")
    bos.bos_loss_l2_pixels(I.data_ptr(), target.data_ptr(), pix.data_ptr(), 400, loss.data_ptr(), g.data_ptr(), sp())
    t = target.reshape(-1)[pix.long()]
    assert abs(loss.item() - ((t.double() - I.double()) ** 2).sum().item()) < 1e-12 * loss.item()
    assert torch.equal(g, -2.0 * (t - I))
    bos.bos_loss_l2_pixels(I.data_ptr(), target.data_ptr(), pix.data_ptr(), 400, loss.data_ptr(), g.data_ptr(), sp(),
                           scale=0.25)
    assert abs(loss.item() - 0.25 * ((t.double() - I.double()) ** 2).sum().item()) < 1e-12 * loss.item()
    assert torch.equal(g, -0.5 * (t - I))
    with pytest.raises(bos.BosError):
        bos.bos_loss_l2_pixels(I.data_ptr(), target.data_ptr(), pix.data_ptr(), 400, loss.data_ptr(), g.data_ptr(),
                               sp(), scale=0.0)
    # AdaBelief against a plain torch transcription of its update rule, three steps
    theta = torch.as_tensor(rng.random(1000).astype(np.float32), device="cuda")
    m = torch.zeros_like(theta)
    s = torch.zeros_like(theta)
    th_ref, m_ref, s_ref = theta.clone().double(), m.clone().double(), s.clone().double()
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-12
    ctr = torch.tensor([1], dtype=torch.int64, device="cuda")
    for step in range(1, 4):
        grad = torch.as_tensor(rng.standard_normal(1000).astype(np.float32), device="cuda")
        if step < 3:
            bos.bos_adabelief_step(theta.data_ptr(), grad.data_ptr(), m.data_ptr(), s.data_ptr(), 1000, lr, b1, b2,
                                   eps, step, sp())
        else:   # step number 1 + *ctr = 3, read on the device
            ctr += 1
            bos.bos_adabelief_step(theta.data_ptr(), grad.data_ptr(), m.data_ptr(), s.data_ptr(), 1000, lr, b1, b2,
                                   eps, 1, sp(), step_dev=ctr.data_ptr())
        gd = grad.double()
        m_ref = b1 * m_ref + (1 - b1) * gd
        s_ref = b2 * s_ref + (1 - b2) * (gd - m_ref) ** 2 + eps
        th_ref = th_ref - lr * (m_ref / (1 - b1 ** step)) / (torch.sqrt(s_ref / (1 - b2 ** step)) + eps)
    torch.cuda.synchronize()
    assert torch.allclose(theta.double(), th_ref, rtol=0, atol=1e-5)


def test_reconstruction_lowers_the_image_loss(bos):
    from paper_2509_14442_gb300.recon import Reconstructor

    sc = S.room((24, 24, 18), 96, 96, 1, 3900, pattern_size=64)
    truth = torch.as_tensor(sc.T, device="cuda")
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP, T=truth)
    target, _, _ = ctx.render(disp=False)
    ctx.close()
    T0 = torch.full_like(truth, S.T_AMBIENT)
    # image-loss gradients here are ~1e-11 per voxel: scale them to order one
    rec = Reconstructor(sc, target, T0, batch=4096, lr=0.2, loss_scale=1e11, seed=5)

    def full_loss(T):
        c = bos.Context(0)
        c.set_scene(sc, bos.BOS_PREC_FP32_COMP, T=T.contiguous())
        I, _, _ = c.render(disp=False)
        torch.cuda.synchronize()
        c.close()
        return float(((I - target) ** 2).sum())

    l0 = full_loss(T0)
    for _ in range(100):
        rec.step()
    torch.cuda.synchronize()
    l1 = full_loss(rec.T)
    rec.close()
    assert l0 > 0 and l1 < 0.05 * l0, (l0, l1)


def _adabelief_np(theta, g, m, s, t, lr, b1, b2, eps):
    """AdaBelief (Zhuang et al., NeurIPS 2020) in float64, the update bos_adabelief_step makes."""
    m[:] = b1 * m + (1.0 - b1) * g
    s[:] = b2 * s + (1.0 - b2) * (g - m) ** 2 + eps
    theta -= lr * (m / (1.0 - b1 ** t)) / (np.sqrt(s / (1.0 - b2 ** t)) + eps)


@pytest.mark.parametrize("integrator", [0, 2])
def test_reconstruction_iterations_match_the_oracle_loop(bos, orc, integrator):
    """k iterations of the minibatch reconstruction (Sec. 2.4 Eq. 3 with lambda_2 = lambda_3
    = 0, Sec. 3.2) on the GPU and on the oracle from the same inputs: the same target image
    (rendered by the oracle), the same pixel minibatches (splitmix64 draws, computed on each
    side from the generator's definition), the oracle's discrete-adjoint gradient of the
    scaled minibatch L_BOS and a float64 AdaBelief.  The field after k iterations agrees
    element by element.

    The target is the oracle's render of the true field with 10 % seeded multiplicative
    noise: the residuals target - I are then ~1e-3, a thousand times the float32 render's
    intensity rounding (~1e-6), whereas the noise-free residual of this small scene
    (~3e-6) is at that rounding and would make dL/dI differ at O(1) between the two sides.

    Tolerance: eps is set so that sqrt(eps / (1 - beta2)) is ~1 % of the largest gradient;
    below that AdaBelief's step is linear in the gradient, so the float32 gradient's error
    (~1e-4 of the largest gradient here) moves T by ~1e-2 lr per iteration at most; in the
    saturated regime the step depends only on the gradient's sign history.  The bound is
    2e-3 lr per iteration, summed over the k iterations."""
    from paper_2509_14442_gb300.recon import Reconstructor

    sc = S.room((12, 12, 9), 32, 32, 1, 3970, pattern_size=32)
    sc = sc.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=integrator, ckpt_every=16))
    truth = sc.T.astype(np.float64)
    I_true = orc.render(sc)["I"]                              # (H, W) float64
    target = I_true * (1.0 + 0.1 * np.random.default_rng(3971).standard_normal(I_true.shape))
    T0 = np.full(truth.shape, S.T_AMBIENT)
    H, W = sc.camera.height, sc.camera.width
    k, batch, lr, b1, b2, seed = 5, 256, 0.2, 0.9, 0.999, 11
    scale = 1e8

    def draw(d):
        return np.array([(orc.splitmix64_output(seed, d * batch + j + 1) * (H * W)) >> 64 for j in range(batch)],
                        dtype=np.int64)

    # the gradient scale of this scene fixes eps: the first iteration's largest gradient
    def oracle_grad(T, pix):
        s_T = sc.replace(T=T)
        I = orc.render(s_T, pix=pix)["I"]
        w = np.zeros(H * W)
        np.add.at(w, pix, -2.0 * scale * (target.reshape(-1)[pix] - I))
        return orc.grad(s_T, w.reshape(H, W)), I

    g0, _ = oracle_grad(T0, draw(0))
    eps = (0.01 * float(np.abs(g0).max())) ** 2 * (1.0 - b2)
    T = T0.copy()
    m, s = np.zeros_like(T), np.zeros_like(T)
    for it in range(k):
        g, _ = oracle_grad(T, draw(it))
        _adabelief_np(T, g, m, s, it + 1, lr, b1, b2, eps)

    rec = Reconstructor(sc, torch.as_tensor(target.astype(np.float32)), torch.as_tensor(T0.astype(np.float32)),
                        batch=batch, lr=lr, beta1=b1, beta2=b2, eps=eps, loss_scale=scale, seed=seed)
    for _ in range(k):
        rec.step()
    torch.cuda.synchronize()
    rec.ctx.status()
    Tg = rec.T.cpu().numpy().astype(np.float64)
    rec.close()
    moved = np.abs(T - T0)
    assert moved.max() > 0.5 * lr                               # the loop did move the field
    err = np.abs(Tg - T)
    assert err.max() <= 2e-3 * lr * k, (err.max(), moved.max())
    assert np.linalg.norm(Tg - T) <= 1e-3 * np.linalg.norm(T - T0)


def test_graph_replayed_iterations_match_eager_ones(bos):
    from paper_2509_14442_gb300.recon import Reconstructor

    sc = S.room((24, 24, 18), 96, 96, 1, 3950, pattern_size=64)
    truth = torch.as_tensor(sc.T, device="cuda")
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP, T=truth)
    target, _, _ = ctx.render(disp=False)
    ctx.close()
    T0 = torch.full_like(truth, S.T_AMBIENT)
    eager = Reconstructor(sc, target, T0, batch=2048, lr=0.2, loss_scale=1e11, seed=9)
    graph = Reconstructor(sc, target, T0, batch=2048, lr=0.2, loss_scale=1e11, seed=9)
    for _ in range(6):
        eager.step()
    graph.run(6)
    torch.cuda.synchronize()
    assert graph.it == eager.it == 6
    assert int(graph.it_dev.item()) == int(eager.it_dev.item()) == 6
    d_e, d_g = eager.T - T0, graph.T - T0
    assert float(d_e.abs().max()) > 0.1                     # the field moved
    # same draws and updates; only the float atomics' summation order differs
    assert float((d_g - d_e).norm() / d_e.norm()) < 1e-3
    eager.close()
    graph.close()


def _morton2(x, y):
    def spread(v):
        v = v & 0xFFFF
        v = (v | (v << 8)) & 0x00FF00FF
        v = (v | (v << 4)) & 0x0F0F0F0F
        v = (v | (v << 2)) & 0x33333333
        v = (v | (v << 1)) & 0x55555555
        return v
    return spread(x) | (spread(y) << 1)


@pytest.mark.parametrize("n", [1, 777, 5000, 16384])
def test_sort_pixels_is_a_z_order_permutation(bos, n):
    w, h = 100, 100
    rng = np.random.default_rng(n)
    pix = rng.integers(0, w * h, n).astype(np.int32)
    t = torch.as_tensor(pix, device="cuda")
    bos.bos_sort_pixels(t.data_ptr(), n, w, h, sp())
    got = t.cpu().numpy()
    assert np.array_equal(np.sort(got), np.sort(pix))          # same entries, repeats kept
    keys = np.array([_morton2(int(p) % w, int(p) // w) for p in got])
    assert np.all(np.diff(keys) >= 0)
    with pytest.raises(bos.BosError):
        bos.bos_sort_pixels(t.data_ptr(), 16385, w, h, sp())
