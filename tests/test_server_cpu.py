"""Scheduler of the request server, run with the fake executor (no GPU, no CUDA calls):
admission by memory in arrival order, slot and memory bounds at every instant, bounded
waits, and draining on destroy."""
import numpy as np
import pytest

from paper_2509_14442_gb300 import scenes as S

MiB = 1 << 20


@pytest.fixture(scope="module")
def bos():
    from paper_2509_14442_gb300 import bos as B
    B.lib()
    return B


def request(bos, n=(64, 64, 64), img=(256, 256), adjoint=False, prec=None):
    g = S.room_grid(n)
    cam = S.Camera(pos=S.CAMERA_POS, fwd=(0.0, 1.0, 0.0), up=(0.0, 0.0, 1.0), fx=1000.0, fy=1000.0,
                   cx=img[0] / 2, cy=img[1] / 2, width=img[0], height=img[1], spp=1)
    light = S.Light(1, np.zeros((8, 8), np.float32), cam)
    fake = 0x1000   # the fake executor never dereferences device pointers
    return bos.make_request(g, bos.BOS_PREC_FP32_COMP if prec is None else prec, fake, cam, S.back_wall(g), light,
                            fake, S.Integrator(), fake, None, fake if adjoint else None,
                            fake if adjoint else None, fake if adjoint else None)


def test_footprint_counts_every_buffer(bos):
    # 64^3 cells: 8 bricks per axis, Morton slots 0..511, 729 elements each; a float32
    # element is an x pair of (deta, grad eta) records: 32 bytes
    fwd = bos.bos_request_footprint(request(bos, (64, 64, 64)))
    assert fwd == 512 * 729 * 32
    adj = bos.bos_request_footprint(request(bos, (64, 64, 64), adjoint=True))
    # + checkpoints (rays x ceil(N_max / 16) x 48 B), path excess, node accumulators, dL/dI
    rays = 256 * 256
    n_max = int(np.ceil(np.sqrt(4 ** 2 + 4 ** 2 + 3 ** 2) / (0.5 * 3.0 / 64))) + 2
    ck = -(-n_max // 16) * 48 * rays
    seg = 2 * 1024 * 2 * 16 * 6 * 32 * 4      # two segments of step states per warp of the Sharma adjoint (K = 16)
    expect = fwd + ck + rays * 4 + 64 ** 3 * 16 + seg + rays * 4
    assert adj == expect
    # quasi-linear tracing keeps only the final state per ray
    q = request(bos, (64, 64, 64), adjoint=True)
    q.integ.integrator = 2
    assert bos.bos_request_footprint(q) == fwd + 48 * rays + rays * 4 + 64 ** 3 * 16 + rays * 4
    # the refracted projector connection adds the projector rays' checkpoints and a
    # 32-byte connection record per ray (adjoint only)
    r2 = request(bos, (64, 64, 64), adjoint=True)
    r2.light.mode, r2.light.connect_iters = 2, 1
    assert bos.bos_request_footprint(r2) == expect + ck + 32 * rays
    f2 = request(bos, (64, 64, 64))
    f2.light.mode, f2.light.connect_iters = 2, 1
    assert bos.bos_request_footprint(f2) == fwd
    # bigger grids and images need more
    assert bos.bos_request_footprint(request(bos, (128, 128, 96))) > fwd
    assert bos.bos_request_footprint(request(bos, img=(512, 512), adjoint=True)) > adj


def test_oversized_and_malformed_requests_are_refused(bos):
    srv = bos.Server(0, 64 * MiB, 2, fake=True)
    big = request(bos, (256, 256, 192))                      # ~360 MB store
    with pytest.raises(bos.BosError) as e:
        srv.submit(big)
    assert e.value.status == bos.BOS_ERR_ADMISSION
    bad = request(bos)
    bad.T_dev = None
    with pytest.raises(bos.BosError) as e:
        srv.submit(bad)
    assert e.value.status == bos.BOS_ERR_INVALID_ARG
    srv.close()


def test_admission_respects_slots_memory_and_arrival_order(bos):
    limit = 40 * MiB
    srv = bos.Server(0, limit, 3, fake=True)
    sizes = [(64, 64, 64), (32, 32, 32), (64, 64, 64), (48, 48, 48), (64, 64, 64), (32, 32, 32)] * 4
    tickets = [srv.submit(request(bos, n)) for n in sizes]
    for t in tickets:
        assert srv.wait(t, 30.0) == bos.BOS_OK
    info = [srv.info(t) for t in tickets]
    srv.close()
    # arrival order is admission order
    admits = [i["admit_ns"] for i in info]
    assert admits == sorted(admits)
    # at every admission instant: running requests <= slots, their footprints <= the arena
    for i in info:
        t = i["admit_ns"]
        live = [j for j in info if j["admit_ns"] <= t < j["done_ns"]]
        assert len(live) <= 3
        assert sum(-(-j["footprint_bytes"] // 256) * 256 for j in live) <= limit
    assert all(i["done"] and i["status"] == bos.BOS_OK for i in info)
    # requests were admitted while others were still running (continuous, not one batch)
    overlapped = sum(1 for a in info for b in info if a is not b and b["admit_ns"] < a["done_ns"] and
                     a["admit_ns"] < b["admit_ns"])
    assert overlapped > 0


def test_wait_is_bounded(bos):
    srv = bos.Server(0, 2048 * MiB, 1, fake=True)
    slow = [srv.submit(request(bos, (256, 256, 192))) for _ in range(3)]   # ~6 ms each in the fake executor
    assert srv.wait(slow[-1], 1e-4) == bos.BOS_ERR_TIMEOUT
    assert srv.wait(slow[-1], 30.0) == bos.BOS_OK
    srv.close()


def test_destroy_drains_queued_and_running_requests(bos):
    srv = bos.Server(0, 100 * MiB, 2, fake=True)
    tickets = [srv.submit(request(bos, (64, 64, 64))) for _ in range(8)]
    srv.close(timeout_s=30.0)           # returns only once every request has run
    assert srv.h is None
