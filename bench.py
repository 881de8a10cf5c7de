"""Benchmark of the BOS forward model (and its adjoint) on one GB300, one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload room_adj|room_fwd]
                    [--prec fp32_comp|bf16_comp|fp32|fp64] [--impl ours|reference]

A step is one pass of the whole hot path over one frame of synthetic input:
  room_adj  (default) 256x256x192 plume grid, 2048^2 camera, 1 ray/pixel:
            build the field store from T, render I_flow saving checkpoints every 16 steps,
            L_BOS against a seeded target image, backward to dL/dT.
  room_fwd  128x128x96 plume grid, 1024^2 camera, 4 jittered rays/pixel: build the
            field store, render I_flow with the displacement field, render I_ref.
Metric: ray-steps per second, one ray-step = one integrator step of one ray (sum of the
per-ray step counts N of the flow render), whole job (all ranks).

The default line (room_adj, one GPU) also carries the metric's other parts as sub-records,
each from its own timed region in the same run: `fwd` (the room_fwd forward rate and its
roofline), `precision` (render time and error against the FP64 oracle's sample of the
CPU-baseline leg for every store/integrator precision) and `serving` (p50/p99 latency of
the request loop at 0.7x its saturated throughput, and that throughput).  --no-extras
leaves them out (profiler captures).

Under torchrun every rank renders its own frame (independent seeds): weak scaling, no
collective on the data path (the barrier only brackets the timing).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload on
the host cores (the only GPU-free arm; it needs no GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_14442_gb300 import scenes as S  # noqa: E402

def quasi(scene):
    return scene.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=2,
                                            ckpt_every=scene.integ.ckpt_every))


def refracted(scene):
    """The same scene with the projector's rays traced through the flow (one aiming round)."""
    L = scene.light
    return scene.replace(light=S.Light(2, L.pattern, L.proj, connect_iters=1))


WORKLOADS = {
    "room_adj": dict(desc="room 256x256x192 plume, 2048^2 camera, 1 spp, forward + adjoint (K=16)",
                     make=lambda seed: S.room_adjoint(seed), adjoint=True),
    "room_fwd": dict(desc="room 128x128x96 plume, 1024^2 camera, 4 jittered spp, forward + I_ref",
                     make=lambda seed: S.room_forward(seed), adjoint=False),
    # the paper's quasi-linear tracer (Sec. 2.2) on the same scenes
    "room_adj_quasi": dict(desc="room 256x256x192 plume, 2048^2 camera, 1 spp, quasi-linear forward + adjoint",
                           make=lambda seed: quasi(S.room_adjoint(seed)), adjoint=True, fwd_bytes=256, adj_bytes=512),
    "room_fwd_quasi": dict(desc="room 128x128x96 plume, 1024^2 camera, 4 jittered spp, quasi-linear forward + I_ref",
                           make=lambda seed: quasi(S.room_forward(seed)), adjoint=False, fwd_bytes=256),
    # the projector's own rays traced through the flow too (refracted connection, light mode 2):
    # every camera sample also traces the projector ray aimed at its wall hit; ray-steps
    # count both rays
    "room_fwd_refr": dict(desc="room 128x128x96 plume, 1024^2 camera, 4 jittered spp, refracted projector "
                               "connection, forward + I_ref",
                          make=lambda seed: refracted(S.room_forward(seed)), adjoint=False),
    "room_adj_refr": dict(desc="room 256x256x192 plume, 2048^2 camera, 1 spp, refracted projector connection, "
                               "forward + adjoint (K=16)",
                          make=lambda seed: refracted(S.room_adjoint(seed)), adjoint=True),
    # small case of the same kernels for profiler captures (not a benchmark line)
    "room_fwd_small": dict(desc="room 128x128x96 plume, 256^2 camera, 4 jittered spp, forward + I_ref",
                           make=lambda seed: S.room((128, 128, 96), 256, 256, 4, seed), adjoint=False),
    "room_adj_small": dict(desc="room 256x256x192 plume, 512^2 camera, 1 spp, forward + adjoint (K=16)",
                           make=lambda seed: S.room((256, 256, 192), 512, 512, 1, seed), adjoint=True),
    "room_adj_quasi_small": dict(desc="room 256x256x192 plume, 512^2 camera, 1 spp, quasi-linear forward + adjoint",
                                 make=lambda seed: quasi(S.room((256, 256, 192), 512, 512, 1, seed)), adjoint=True,
                                 fwd_bytes=256, adj_bytes=512),
}
# Algorithmic bytes of one Sharma ray-step of the forward tracer: 3 field evaluations x 8
# trilinear corners x one (deta, grad eta) record (16 B in float32).
BYTES_PER_STEP = {"fp32_comp": 384, "fp32": 384, "bf16_comp": 192, "fp64": 768}
# Adjoint, per ray-step: the segment recompute gathers 384 B, the reverse step gathers the
# same 3 x 8 records again, and scatters 3 x 8 corner sensitivities of 16 B.  (Quasi-linear
# tracing samples 2 new points per step: 256 B forward; its one-sweep adjoint gathers and
# scatters those 2 points: 512 B.)
ADJ_BYTES_PER_STEP = {"fp32_comp": 3 * 384, "bf16_comp": 2 * 192 + 384}
# Bytes the gathers load through L1 per ray-step (the scatter of the adjoint goes to shared
# memory and atomics instead): forward 3 x 8 corners x 16 B; adjoint recompute + reverse.
L1_BYTES_PER_STEP = {"fp32_comp": 384, "fp32": 384, "bf16_comp": 192, "fp64": 768}
ADJ_L1_BYTES_PER_STEP = {"fp32_comp": 2 * 384, "bf16_comp": 2 * 192}
L2_BYTES = 129 * 2 ** 20
# Algorithmic floating-point operations of one ray-step (an FMA counts 2), counted from the
# method's formulas, not from the kernels (which add the compensation of the fixed-point
# straight line, bounds tests and index arithmetic):
#   field evaluation D(r) = (1 + deta) grad eta at a point: 3 fractions (sub, mul) = 6,
#     trilinear interpolation of the 4 channels, 7 lerps x 3 flops each = 84, D = 4:  94
#   Sharma RKN step (Sec. 2.2, Eq. 1): 3 evaluations 282, A, B, C = dt D 9, the two inner
#     stage points 24, the position update 18, the velocity update 15, the path-length
#     increment |dr| 8:  356
#   quasi-linear step: 2 new line samples (point on the line 6 + 94 each) 200, the same
#     updates and path length 41:  241
#   adjoint of an RKN step: the segment recompute 356, 3 value-and-fraction-derivative
#     evaluations 3 x (6 + 4 x 36) = 450, the adjoint of D per stage 3 x 36 = 108, the
#     transpose of the step's linear combinations 66, the path-length adjoint 11, and the
#     corner scatter per stage (3 complements, 8 weights x 2, 8 x 4 FMAs) 3 x 83 = 249:  1240
#   one-sweep quasi-linear adjoint: per line sample the point, fractions and value 96, the
#     adjoint of D 9 and the corner scatter 83 (2 samples: 376), the velocity adjoint 24:  400
FLOPS_PER_STEP = {"rkn": 356, "quasi": 241}
ADJ_FLOPS_PER_STEP = {"rkn": 1240, "quasi": 400}
# The arithmetic peak: 152 SMs x 128 float32 FMA lanes x 2 flops x the SM clock (derived
# from the unit counts; the in-run probe measures it as well).  Float64: GB300's nominal
# 1.25 TFLOP/s at 2070 MHz.
FP32_LANES_PER_SM = 128
FP64_NOMINAL_FLOPS = 1.25e12

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the timed kernels,
# captured by ncu on the small case of the same kernels (room_adj_small: the 256^2x192 field,
# a 512^2 camera; one kernel, one launch).  The timed launch's figure is that capture with
# its per-ray algorithmic bytes (checkpoints, path records, image) replaced by those of the
# timed launch (`algorithmic_hbm`): the per-grid part (the field store, the accumulators)
# is the same at both sizes.  Reported only while the kernel sources still hash to the
# captured ones.
TRAFFIC_SOURCES = ("bos_forward.cu", "bos_adjoint.cu", "bos_comp.cuh", "bos_device.cuh", "bos_full.cuh")
TRAFFIC_CAPTURE = {"workload": "room_adj_small", "sha256": "7fac1ee6e2e1104ea8741aca7bf56e4f7191c9d44ffaa67a74c5589f51ee5e94",
                   "render_kernel": 409746176 + 430900736, "adjoint_kernel": 952656896 + 245624320,
                   # per-ray algorithmic bytes of the captured launches (512^2 rays, 8,650,752 checkpoints)
                   "rays": {"render_kernel": 417333248, "adjoint_kernel": 417333248}}


def kernel_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2509_14442_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def algorithmic_hbm(scene, ckpt_slots: int, store_bytes: int) -> dict:
    """Algorithmic DRAM bytes of one launch of the render (with checkpoints) and of the
    adjoint, split into the part that grows with the rays ("rays": ckpt_slots = sum over
    rays of ceil(N/K) checkpoints of 48 B, 4 B of path-length record per ray, the render's
    4 B image or the adjoint's 4 B of dL/dI per pixel) and the part fixed by the grid
    ("grid": the field store read once; for the adjoint also its float4 node accumulators,
    read and written by the atomics, 32 B per cell).  "total" = their sum."""
    rays = ckpt_slots * 48 + scene.rays * 4 + scene.pixels * 4
    grid = {"render_kernel": store_bytes, "adjoint_kernel": store_bytes + scene.grid.cells * 32}
    return {k: {"rays": rays, "grid": g, "total": rays + g} for k, g in grid.items()}


def kernel_traffic(name: str, alg: dict):
    c = TRAFFIC_CAPTURE
    if c["sha256"] is None or c.get(name) is None or c["rays"].get(name) is None or \
            kernel_sources_sha256() != c["sha256"]:
        return None
    return {"bytes": c[name] - c["rays"][name] + alg[name]["rays"], "captured_bytes": c[name],
            "captured_on": c["workload"],
            "scaling": "captured DRAM bytes - per-ray algorithmic bytes of the captured launch "
                       "+ per-ray algorithmic bytes of this launch (the per-grid part is the same grid)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default="room_adj",
                   choices=sorted(WORKLOADS) + ["serving", "precision", "recon", "oracle"])
    p.add_argument("--prec", default="fp32_comp", choices=sorted(BYTES_PER_STEP))
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="leave out the fwd / precision / serving sub-records")
    p.add_argument("--requests", type=int, default=256, help="serving: number of requests")
    p.add_argument("--sample-pixels", type=int, default=4000, help="precision: oracle-checked pixels")
    p.add_argument("--slots", type=int, default=6, help="serving: concurrent requests")
    p.add_argument("--mem-limit-gb", type=int, default=120, help="serving: admission limit (GiB)")
    return p.parse_args()


# ------------------------------------------------------------------ oracle (CPU) arm

def oracle_rate(scene, adjoint: bool, seconds: float, seed: int = 0, threads: int = 0) -> dict:
    """Time the FP64 oracle on a pixel sample sized for ~`seconds` on all host cores (or on
    `threads` of them).  Returns rate (ray-steps/s), threads, a description of the sample,
    the measured seconds, the sample's pixel indices and the oracle's render of them."""
    from oracle import oracle as O

    O.build()
    threads = threads or os.cpu_count() or 1
    field = O.field_from_T(scene.grid, scene.T)
    rng = np.random.default_rng(seed)
    npix = scene.pixels

    def run(pix, with_adjoint):
        t0 = time.perf_counter()
        out = O.render(scene, field=field, pix=pix, threads=threads, nsteps=True)
        steps = int(out["nsteps"].sum())
        if with_adjoint:
            w = np.zeros((scene.camera.height, scene.camera.width))
            w.reshape(-1)[pix] = 1.0
            O.grad(scene, w, threads=threads)
        return steps, time.perf_counter() - t0, out

    # size the sample from the forward render's per-pixel time (the oracle's gradient
    # re-traces every ray with a tape and then reverses it: about three renders' work, plus
    # a fixed per-call cost), so that the sample takes about `seconds`
    m0 = min(npix, 4000)
    per_pix = run(np.sort(rng.choice(npix, m0, replace=False)), False)[1] / m0
    m = int(min(npix, max(m0, seconds / (per_pix * (4.0 if adjoint else 1.0)))))
    pix = np.sort(rng.choice(npix, m, replace=False))
    steps, t, out = run(pix, adjoint)
    kind = "forward + adjoint" if adjoint else "forward"
    return {"rate": steps / t, "threads": threads, "seconds": t, "pix": pix, "out": out,
            "desc": f"{m} of {npix} pixels ({kind}), {steps} ray-steps in {t:.1f} s"}


def oracle_arm(args):
    """The FP64 oracle's own rates on this machine's host cores, per configuration (no GPU
    work): the 32^3 blob cube's whole image (all cores and one thread), pixel samples of the
    128^2x96 forward and of the 256^2x192 forward and forward + adjoint scenes (one thread
    too for the forward), and the gradient of the 32^3 crop (whole image)."""
    import platform

    from oracle import oracle as O

    O.build()
    threads = os.cpu_count() or 1
    out = {}
    sc = S.blob_cube()
    field = O.field_from_T(sc.grid, sc.T)
    for nthr, tag in ((threads, "all_cores"), (1, "one_thread")):
        t0 = time.perf_counter()
        r = O.render(sc, field=field, threads=nthr, nsteps=True)
        t = time.perf_counter() - t0
        steps = int(r["nsteps"].sum())
        out[f"blob_cube_32_forward_{tag}"] = {"ray_steps_per_s": steps / t, "threads": nthr,
                                              "sample": f"all {sc.pixels} pixels, {steps} ray-steps in {t:.2f} s"}
    cases = (("room_128x128x96_forward", S.room_forward, False, 10.0, 0),
             ("room_256x256x192_forward", S.room_adjoint, False, 10.0, 0),
             ("room_256x256x192_forward_one_thread", S.room_adjoint, False, 5.0, 1),
             ("room_256x256x192_forward_adjoint", S.room_adjoint, True, 15.0, 0))
    for name, make, adj, secs, nthr in cases:
        r = oracle_rate(make(), adj, secs, threads=nthr)
        out[name] = {"ray_steps_per_s": r["rate"], "threads": r["threads"], "sample": r["desc"]}
    big = S.room_adjoint()
    k, j, i = np.unravel_index(np.argmax(big.T), big.T.shape)
    lo = [int(np.clip(c - 16, 0, n - 32)) for c, n in zip((i, j, k), big.grid.n)]
    crop = S.crop(big, lo, 32, 256, 256, 1)
    w = np.random.default_rng(13).standard_normal((crop.camera.height, crop.camera.width))
    steps = int(O.render(crop, threads=threads, nsteps=True)["nsteps"].sum())
    t0 = time.perf_counter()
    O.grad(crop, w, threads=threads)
    t = time.perf_counter() - t0
    out["crop_32_gradient"] = {"ray_steps_per_s": steps / t, "threads": threads,
                               "sample": f"all {crop.pixels} pixels, {steps} ray-steps, gradient in {t:.2f} s"}
    print(json.dumps({
        "metric": "FP64 oracle ray-steps/s per configuration (host cores)",
        "value": out["room_256x256x192_forward_adjoint"]["ray_steps_per_s"], "unit": "ray-steps/s",
        "higher_is_better": True, "dtype": "f64", "data": "synthetic (seeded plume fields and speckle patterns)",
        "config": {"workload": "oracle", "cores": threads, "machine": platform.machine()},
        "oracle": out}))


def reference_arm(args):
    """The FP64 oracle on the host cores, as it stands: each step is one bounded pixel
    sample of the same workload (a short sizing pass, then the timed sample); value = the
    mean of the timed samples' ray-steps/s, ms_per_step = their mean measured time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the ray-tracing workloads, "
                                                              f"not '{args.workload}'"}))
        return
    wl = WORKLOADS[args.workload]
    scene = wl["make"](S.BASE_SEED + 2 if wl["adjoint"] else S.BASE_SEED + 1)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    rates, secs = [], []
    r = None
    for i in range(args.warmup + args.steps):
        r = oracle_rate(scene, wl["adjoint"], per_step, seed=i)
        if i >= args.warmup:
            rates.append(r["rate"])
            secs.append(r["seconds"])
    v = statistics.mean(rates)
    unit = "ray-steps/s"
    print(json.dumps({
        "impl": "reference", "metric": metric_name(args), "value": v, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, wl, scene),
        "cpu_baseline": {"value": v, "unit": unit, "cores": r["threads"], "kind": "oracle",
                         "sample": f"per step: {r['desc']} (last step)"},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm

def metric_name(args):
    wl = WORKLOADS[args.workload]
    return "ray-steps/s (forward + adjoint)" if wl["adjoint"] else "ray-steps/s (forward)"


def config_of(args, wl, scene):
    c = {"workload": args.workload, "description": wl["desc"], "prec": args.prec,
         "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{args.gpus}"}
    if scene is not None:
        c.update(grid=list(scene.grid.n), image=[scene.camera.width, scene.camera.height],
                 spp=scene.camera.spp, ckpt_every=scene.integ.ckpt_every)
    return c


class Clocks:
    """nvidia-smi samples (every 100 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(prefix="bos_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            return self._summary()
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)

    def _summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def l2_read_peak(torch, dev, bos):
    """L2 read bandwidth: 16-byte L1-bypassing loads over a 24 MiB buffer (fits one L2
    partition), best of 10 launches of 50 passes."""
    nbytes = 24 * 2 ** 20
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    sp = torch.cuda.current_stream().cuda_stream
    reps = 50
    bos.bos_probe_read(buf.data_ptr(), nbytes, reps, sink.data_ptr(), sp)
    best = 1e30
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bos.bos_probe_read(buf.data_ptr(), nbytes, reps, sink.data_ptr(), sp)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return nbytes * reps / (best * 1e-3) / 1e9


def l1_read_peak(torch, dev, bos):
    """L1 read bandwidth of 256-bit loads (GB/s): a 64 KiB buffer every block re-reads, best
    of 10 launches of 200 passes."""
    nbytes = 64 * 2 ** 10
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    sp = torch.cuda.current_stream().cuda_stream
    reps = 200
    bos.bos_probe_read_l1(buf.data_ptr(), nbytes, reps, sink.data_ptr(), sp)
    best, nread = 1e30, 0.0
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        nread = bos.bos_probe_read_l1(buf.data_ptr(), nbytes, reps, sink.data_ptr(), sp)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return nread / (best * 1e-3) / 1e9


def fma_peaks(torch, dev, bos):
    """FMA throughput of this GPU (TFLOP/s): float32, packed float32 pairs and float64, each
    the best of 5 launches of the probe (about 2-4 ms each)."""
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    sp = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, kind, reps in (("fp32", 0, 4000), ("fp32x2", 1, 4000), ("fp64", 2, 100)):
        bos.bos_probe_fma(kind, reps, sink.data_ptr(), sp)
        best = 1e30
        flops = 0.0
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            flops = bos.bos_probe_fma(kind, reps, sink.data_ptr(), sp)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = flops / (best * 1e-3) / 1e12
    return out


def aggregate(my_ms: float, units_per_rank: int, dist=None, device=None):
    """Whole-job rate of a weak-scaling run: every rank processed `units_per_rank` units in
    `my_ms` of device time; the job took the slowest rank's time.  Returns (job_ms, units/s)."""
    job_ms = my_ms
    world = 1
    if dist is not None and dist.is_initialized():
        import torch

        world = dist.get_world_size()
        t = torch.tensor([my_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        job_ms = float(t.item())
    return job_ms, units_per_rank * world / (job_ms * 1e-3)


def frame_bench(args, wl_name: str, ctxs: dict, rank: int = 0, world: int = 1, dist=None, e2e: bool = False):
    """Time `args.steps` steps (after `args.warmup`) of workload `wl_name`: each step builds
    the field store from T, renders I_flow (with checkpoints for the adjoint workloads),
    then either L_BOS + backward, or I_ref.  L2 is flushed between timed steps.  With e2e,
    the same steps again with T (and the target) copied from pinned host memory and the
    result copied back, inside the timed region."""
    torch, bos, dev = ctxs["torch"], ctxs["bos"], ctxs["dev"]
    wl = WORKLOADS[wl_name]
    prec = bos.PRECISIONS[args.prec]
    scene = wl["make"]((S.BASE_SEED + 2 if wl["adjoint"] else S.BASE_SEED + 1) + 1000 * rank)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    T_host = torch.from_numpy(np.ascontiguousarray(scene.T)).pin_memory()
    T = T_host.to(dev)
    ctx = bos.Context(dev.index)
    ctx.set_scene(scene, prec, T=T)
    store_bytes = bos.bos_device_bytes(ctx.h) - 256
    H, W = scene.camera.height, scene.camera.width
    I = torch.empty((H, W), dtype=torch.float32, device=dev)
    Iref = torch.empty_like(I)
    disp = torch.empty((H, W, 2), dtype=torch.float32, device=dev)
    target = target_host = None
    if wl["adjoint"]:
        # target image: a render of the same plume family drawn with the next seed
        Tt = torch.from_numpy(S.with_target_seed(scene, scene.camera.seed % 100000 + 1)).to(dev)
        ctx.set_grid(scene.grid, Tt, prec)
        target = torch.empty_like(I)
        ctx.render(disp=False, out=(target, None, None))
        ctx.set_grid(scene.grid, T, prec)
        target_host = target.cpu().pin_memory()
        del Tt
    loss = torch.empty((1,), dtype=torch.float64, device=dev)
    dLdI = torch.empty_like(I)
    dLdT = torch.empty_like(T)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)   # 256 MiB > L2
    ev_r = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    launches = {"n": 0}

    def step(T_in, ev=None):
        L = bos.lib()
        bos.check(L.bos_set_grid(ctx.h, bos.C.byref(bos.grid_desc(scene.grid, prec)), T_in.data_ptr(), sp),
                  "set_grid")
        if ev is not None:
            ev[0].record(stream)
        if wl["adjoint"]:
            bos.check(L.bos_render(ctx.h, I.data_ptr(), None, None, 1, sp), "render")
        else:
            bos.check(L.bos_render(ctx.h, I.data_ptr(), disp.data_ptr(), None, 0, sp), "render")
        if ev is not None:
            ev[1].record(stream)
        if wl["adjoint"]:
            bos.check(L.bos_loss_l2(I.data_ptr(), target.data_ptr(), I.numel(), loss.data_ptr(), dLdI.data_ptr(),
                                    sp), "loss")
            if ev is not None:
                ev[2].record(stream)
            bos.check(L.bos_backward(ctx.h, dLdI.data_ptr(), dLdT.data_ptr(), sp), "backward")
            if ev is not None:
                ev[3].record(stream)
            launches["n"] = 5          # build_store, render, loss_l2, adjoint, gradient
        else:
            bos.check(L.bos_render_reference(ctx.h, Iref.data_ptr(), None, None, sp), "render_ref")
            launches["n"] = 3          # build_store, render, render (reference)

    for _ in range(args.warmup):
        step(T)
    torch.cuda.synchronize()
    ctx.status()
    steps_per_frame = ctx.last_ray_steps()
    nsteps = ctx.ray_steps().to(torch.int64)
    K = scene.integ.ckpt_every
    ckpt_slots = int(((nsteps + K - 1) // K).sum().item()) if wl["adjoint"] else 0
    del nsteps

    # ---- timed region: device time of K steps, L2 flushed between steps
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    step_ms, render_ms, back_ms = [], [], []
    with clocks:
        for _ in range(args.steps):
            flush.fill_(0.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(T, ev_r)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            render_ms.append(ev_r[0].elapsed_time(ev_r[1]))
            if wl["adjoint"]:
                back_ms.append(ev_r[2].elapsed_time(ev_r[3]))
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ctx.status()
    res = dict(scene=scene, wl=wl, steps_per_frame=steps_per_frame, step_ms=step_ms, render_ms=render_ms,
               back_ms=back_ms, clocks=clocks.summary(), launches_per_step=launches["n"], store_bytes=store_bytes,
               ckpt_slots=ckpt_slots)

    if e2e:
        # ---- end to end through the C ABI with host buffers: H2D inputs, D2H result
        e2e_ms = []
        h2d = T_host.numel() * 4 + (target_host.numel() * 4 if target is not None else 0)
        out_host = torch.empty_like(dLdT if wl["adjoint"] else I, device="cpu").pin_memory()
        loss_host = torch.empty((1,), dtype=torch.float64).pin_memory()
        d2h = out_host.numel() * 4 + (8 if wl["adjoint"] else 0)
        T_dev2 = torch.empty_like(T)
        for i in range(args.warmup + args.steps):
            flush.fill_(0.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T_dev2.copy_(T_host, non_blocking=True)
            if target is not None:
                target.copy_(target_host, non_blocking=True)
            step(T_dev2)
            if wl["adjoint"]:
                out_host.copy_(dLdT, non_blocking=True)
                loss_host.copy_(loss, non_blocking=True)
            else:
                out_host.copy_(I, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
        res.update(e2e_ms=e2e_ms, h2d=h2d, d2h=d2h)
    ctx.close()
    del flush
    torch.cuda.empty_cache()
    return res


def measure_peaks(ctxs) -> dict:
    torch, bos, dev = ctxs["torch"], ctxs["bos"], ctxs["dev"]
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    return {"file": peaks, "l2": l2_read_peak(torch, dev, bos), "l1": l1_read_peak(torch, dev, bos),
            "fma": fma_peaks(torch, dev, bos), "sms": torch.cuda.get_device_properties(dev).multi_processor_count}


def alu_peak_of(prec: str, P: dict):
    clock_mhz = float(P["file"].get("sm_max_mhz") or 2070.0)
    probe = P["fma"]
    if prec == "fp64":
        derived = FP64_NOMINAL_FLOPS * clock_mhz / 2070.0 / 1e12
        measured = probe["fp64"]
        src = (f"float64: GB300 nominal 1.25 TFLOP/s at 2070 MHz, scaled to {clock_mhz:.0f} MHz; "
               f"in-run probe {measured:.2f} TFLOP/s; the larger is the peak")
    else:
        derived = P["sms"] * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
        measured = max(probe["fp32"], probe["fp32x2"])
        src = (f"float32 FMA: {P['sms']} SMs x {FP32_LANES_PER_SM} lanes x 2 flops x {clock_mhz:.0f} MHz "
               f"= {derived:.1f} TFLOP/s (derived); in-run probe {measured:.1f} TFLOP/s; the larger is the peak")
    return max(derived, measured), src


def kernel_entries(res, prec: str, P: dict) -> dict:
    """Roofline figures of the render and (adjoint workloads) the backward of one frame
    benchmark: arithmetic (algorithmic flops per ray-step), L1 and L2 gathered bytes."""
    wl, scene, spf = res["wl"], res["scene"], res["steps_per_frame"]
    alu_peak, _ = alu_peak_of(prec, P)
    integ = {0: "rkn", 2: "quasi"}.get(scene.integ.integrator)
    fwd_b = wl.get("fwd_bytes", BYTES_PER_STEP[prec])
    adj_b = wl.get("adj_bytes", ADJ_BYTES_PER_STEP.get(prec, 0))
    fwd_l1 = wl.get("fwd_bytes", L1_BYTES_PER_STEP[prec])
    adj_l1 = wl.get("fwd_bytes", ADJ_L1_BYTES_PER_STEP.get(prec, 0))
    alg = algorithmic_hbm(scene, res["ckpt_slots"], res["store_bytes"]) if wl["adjoint"] else None

    def entry(ms, flops_per_step, bytes_per_step, l1_bytes_per_step, name):
        tflops = flops_per_step * spf / (ms * 1e-3) / 1e12 if flops_per_step else None
        gbs = bytes_per_step * spf / (ms * 1e-3) / 1e9
        l1_gbs = l1_bytes_per_step * spf / (ms * 1e-3) / 1e9
        return {"ms": ms, "flops_per_ray_step": flops_per_step, "achieved_tflops": tflops,
                "frac": tflops / alu_peak if tflops is not None else None,
                "bytes_per_ray_step": bytes_per_step, "achieved_gbs": gbs, "l2_frac": gbs / P["l2"],
                "l1_bytes_per_ray_step": l1_bytes_per_step, "l1_achieved_gbs": l1_gbs, "l1_frac": l1_gbs / P["l1"],
                "algorithmic_hbm_bytes": alg[name]["total"] if alg else None,
                "traffic": kernel_traffic(name, alg) if alg else None}

    k = {"render_kernel": entry(statistics.mean(res["render_ms"]), FLOPS_PER_STEP.get(integ), fwd_b, fwd_l1,
                                "render_kernel")}
    if prec == "fp32_comp" and integ == "rkn" and scene.light.mode != 2:
        k["render_kernel"]["l1_note"] = ("algorithmic gathered bytes: the tracer keeps each ray's last cell in "
                                         "registers, so most stages load nothing through L1")
    if wl["adjoint"]:
        k["adjoint_kernel"] = entry(statistics.mean(res["back_ms"]), ADJ_FLOPS_PER_STEP.get(integ), adj_b, adj_l1,
                                    "adjoint_kernel")
        k["adjoint_kernel"]["timed"] = "bos_backward: accumulator clear + adjoint_kernel + gradient_kernel"
    return k


def fwd_record(args, ctxs, P) -> dict:
    """The metric's forward half: room_fwd (128^2x96 plume, 1024^2 camera, 4 jittered spp)."""
    res = frame_bench(args, "room_fwd", ctxs)
    k = kernel_entries(res, args.prec, P)["render_kernel"]
    spf = res["steps_per_frame"]
    return {"workload": "room_fwd", "description": WORKLOADS["room_fwd"]["desc"],
            "ray_steps_per_s": spf * len(res["step_ms"]) / (sum(res["step_ms"]) * 1e-3),
            "ms_per_step": statistics.mean(res["step_ms"]), "render_ms": k["ms"],
            "render_ray_steps_per_s": spf / (k["ms"] * 1e-3), "ray_steps_per_frame": spf,
            "step": "field build + I_flow (with displacement) + I_ref", "steps": args.steps,
            "l1_frac": k["l1_frac"], "l2_frac": k["l2_frac"], "alu_frac": k["frac"], "render_kernel": k,
            "clocks": res["clocks"]}


def cpu_leg(scene, adjoint: bool, seconds: float, precision_pixels: int):
    """The CPU baseline: the FP64 oracle as it stands on a bounded pixel sample of the
    workload on all host cores.  With precision_pixels > 0, its renders of that many of the
    sample's pixels (and the oracle's render of them on the BF16-rounded field) are kept for
    the precision table's error columns."""
    from oracle import oracle as O

    r = oracle_rate(scene, adjoint, seconds)
    cpu = {"value": r["rate"], "unit": "ray-steps/s", "cores": r["threads"], "kind": "oracle", "sample": r["desc"]}
    if precision_pixels <= 0:
        return cpu, None
    sel = np.linspace(0, len(r["pix"]) - 1, min(precision_pixels, len(r["pix"]))).astype(np.int64)
    pix = r["pix"][sel]
    true = {"I": r["out"]["I"].reshape(-1)[sel], "disp": r["out"]["disp"].reshape(-1, 2)[sel]}
    de = O.deta_from_T(scene.grid, scene.T.astype(np.float64))
    gr = O.grad_from_deta(scene.grid, de)
    o = O.render(scene, field=O.NodeField(bf16_round(de), bf16_round(gr)), pix=pix, threads=r["threads"])
    return cpu, {"pix": pix, "true": true, "bf16": {"I": o["I"].reshape(-1), "disp": o["disp"].reshape(-1, 2)}}


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2509_14442_gb300 import bos

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctxs = {"torch": torch, "bos": bos, "dev": dev}
    wl = WORKLOADS[args.workload]

    res = frame_bench(args, args.workload, ctxs, rank, world, dist if world > 1 else None, e2e=True)
    scene, spf = res["scene"], res["steps_per_frame"]
    total_ms, value = aggregate(sum(res["step_ms"]), spf * args.steps, dist if world > 1 else None, dev)
    e2e_value = spf * args.steps / (sum(res["e2e_ms"]) * 1e-3) * world

    # ---- roofline of the timed kernels (peaks measured in the same run)
    P = measure_peaks(ctxs)
    alu_peak, alu_src = alu_peak_of(args.prec, P)
    kernels = kernel_entries(res, args.prec, P)
    dominant = "adjoint_kernel" if wl["adjoint"] else "render_kernel"
    dk = kernels[dominant]
    traffic = dk["traffic"]["bytes"] if dk["traffic"] else None
    roofline = {"bound": "alu", "kernel": dominant, "achieved": dk["achieved_tflops"], "peak": alu_peak,
                "unit": "TFLOP/s", "frac": dk["frac"], "traffic": traffic, "peak_source": alu_src,
                "flops_per_ray_step": dk["flops_per_ray_step"],
                "fma_probe_tflops": P["fma"],
                "note": ("algorithmic flops per ray-step counted from the method's formulas; the gathers are "
                         "served on chip and DRAM carries only the store, checkpoints and outputs, so the "
                         "arithmetic roof is the one that applies"),
                "kernels": kernels,
                "l2": {"achieved": dk["achieved_gbs"], "peak": P["l2"], "unit": "GB/s", "frac": dk["l2_frac"],
                       "bytes_per_ray_step": dk["bytes_per_ray_step"],
                       "peak_source": "in-run L2 read probe (bos_probe_read, 24 MiB x 50 passes, best of 10)",
                       "note": ("gather roofline R = L2 read bandwidth / algorithmic gathered bytes per ray-step; "
                                "the gathers hit L1, so a kernel can exceed R")},
                "l1": {"achieved": dk["l1_achieved_gbs"], "peak": P["l1"], "unit": "GB/s", "frac": dk["l1_frac"],
                       "bytes_per_ray_step": dk["l1_bytes_per_ray_step"],
                       "peak_source": "in-run L1 read probe (bos_probe_read_l1, 256-bit loads, 64 KiB x 200 passes "
                                      "per block, best of 10)",
                       "note": "the gathers' algorithmic bytes per ray-step over the L1 read bandwidth"},
                "hbm_peak_gbs": P["file"].get("hbm_gbs")}
    if P["file"].get("hbm_gbs"):
        # the same kernel against the HBM roofline: DRAM bytes per launch (measured on the
        # small case and scaled, else the algorithmic bytes) over the kernel's time
        hb = traffic if traffic is not None else dk["algorithmic_hbm_bytes"]
        if hb is not None:
            hbm_gbs = hb / (dk["ms"] * 1e-3) / 1e9
            roofline["hbm"] = {"achieved": hbm_gbs, "peak": P["file"]["hbm_gbs"], "unit": "GB/s",
                               "frac": hbm_gbs / P["file"]["hbm_gbs"],
                               "bytes": "traffic (scaled ncu capture)" if traffic is not None else "algorithmic",
                               "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}

    extras = world == 1 and not args.no_extras and args.workload == "room_adj"
    out = {}
    if extras:
        out["fwd"] = fwd_record(args, ctxs, P)
    cpu, orc = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, orc = cpu_leg(scene, wl["adjoint"], args.cpu_seconds, args.sample_pixels if extras else 0)
    if extras:
        out["precision"] = precision_record(args, ctxs, P, scene, orc)
        out["serving"] = serving_record(args, ctxs, rates=(0.7,))
    if rank == 0:
        line = {
            "metric": metric_name(args), "value": value, "unit": "ray-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded plume fields and speckle patterns)",
            "config": config_of(args, wl, scene),
            "ray_steps_per_frame": spf,
            "clocks": res["clocks"],
            "e2e": {"value": e2e_value, "unit": "ray-steps/s", "h2d_bytes_per_step": res["h2d"],
                    "d2h_bytes_per_step": res["d2h"]},
            "gpu_launches": res["launches_per_step"] * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
        }
        line.update(out)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ serving

SERVE_GRIDS = [(64, 64, 64), (128, 128, 96), (256, 256, 192)]
SERVE_IMAGES = [256, 1024, 2048]


def serving_record(args, ctxs, rates=(0.7, 1.0)) -> dict:
    """256 requests (forward or forward + adjoint; grid and image drawn per request; plume
    seed per request) through the continuous-batching server under a 120 GiB admission
    limit: first all at once (saturated throughput), then with Poisson arrivals at the
    given fractions of that rate; latency = completion - submission."""
    torch, bos, dev = ctxs["torch"], ctxs["bos"], ctxs["dev"]
    rng = np.random.default_rng(S.BASE_SEED + 5)
    n = args.requests
    pattern_np = S.speckle(512, 512, S.BASE_SEED + 5000)
    pattern = torch.as_tensor(pattern_np, device=dev)
    classes = {}
    reqs = []
    for i in range(n):
        u = rng.random(3)
        adj = bool(u[0] < 0.5)
        g = SERVE_GRIDS[int(u[1] * 3)]
        im = SERVE_IMAGES[int(u[2] * 3)]
        sc = classes[(g, im)][0] if (g, im) in classes else S.room(g, im, im, 1, S.BASE_SEED + 100 + i, field=False)
        T = S.plume_field(S.room_grid(g), S.BASE_SEED + 100 + i, device=dev).contiguous()
        r = dict(adj=adj, grid=g, image=im, T=T, I=torch.empty((im, im), device=dev))
        if adj:
            r.update(target=torch.full((im, im), 0.02, device=dev), loss=torch.empty(1, dtype=torch.float64, device=dev),
                     dLdT=torch.empty_like(T))
        else:
            r["disp"] = torch.empty((im, im, 2), device=dev)
        if (g, im) not in classes:
            ctx = bos.Context(dev.index)
            ctx.set_grid(sc.grid, T, bos.BOS_PREC_FP32_COMP)
            ctx.set_geometry(sc.camera, sc.wall, sc.light, sc.integ, pattern=pattern)
            steps = int(ctx.ray_steps().sum().item())
            ctx.close()
            classes[(g, im)] = (sc, steps)
        r["scene"], r["steps"] = classes[(g, im)]
        reqs.append(r)
    torch.cuda.synchronize()

    def req_of(r):
        sc = r["scene"]
        p = lambda k: r[k].data_ptr() if k in r else None
        return bos.make_request(sc.grid, bos.BOS_PREC_FP32_COMP, r["T"].data_ptr(), sc.camera, sc.wall, sc.light,
                                pattern.data_ptr(), sc.integ, p("I"), p("disp"), p("target"), p("loss"), p("dLdT"))

    def run(rate):
        srv = bos.Server(dev.index, args.mem_limit_gb << 30, args.slots)
        t0 = time.perf_counter()
        gaps = np.random.default_rng(7).exponential(1.0 / rate, n) if rate else np.zeros(n)
        due = t0 + np.cumsum(gaps) - gaps[0]
        tickets = []
        for r, d in zip(reqs, due):
            while True:
                w = d - time.perf_counter()
                if w <= 0:
                    break
                time.sleep(min(w, 0.002))
            tickets.append(srv.submit(req_of(r)))
        for t in tickets:
            st = srv.wait(t, 600.0)
            if st != bos.BOS_OK:
                raise RuntimeError(f"request {t} failed with status {st}")
        infos = [srv.info(t) for t in tickets]
        stats = srv.stats()
        srv.close()
        lat = np.array([(i["done_ns"] - i["submit_ns"]) * 1e-6 for i in infos])
        span = (max(i["done_ns"] for i in infos) - min(i["submit_ns"] for i in infos)) * 1e-9
        steps = sum(r["steps"] for r in reqs)
        live = [sum(1 for j in infos if j["admit_ns"] <= i["admit_ns"] < j["done_ns"]) for i in infos]
        return dict(req_per_s=n / span, ray_steps_per_s=steps / span, p50_ms=float(np.percentile(lat, 50)),
                    p99_ms=float(np.percentile(lat, 99)), mean_concurrency=float(np.mean(live)),
                    peak_arena_gb=stats["peak_used_bytes"] / 2 ** 30, makespan_s=span)

    run(0)                                   # warm-up (module load, first launches)
    sat = run(0)
    out = {"requests": n, "slots": args.slots, "admission_limit_gb": args.mem_limit_gb,
           "mix": "fwd | fwd+adjoint x grids {64^3,128^2x96,256^2x192} x images {256^2,1024^2,2048^2}, 1 spp",
           "saturated": sat}
    for f in rates:
        out[f"at_{f}x"] = run(f * sat["req_per_s"])
    if 0.7 in rates:
        out["latency_ms_at_0.7x"] = {"p50": out["at_0.7x"]["p50_ms"], "p99": out["at_0.7x"]["p99_ms"]}
    del reqs
    torch.cuda.empty_cache()
    return out


def serving_arm(args):
    import torch

    from paper_2509_14442_gb300 import bos

    ctxs = {"torch": torch, "bos": bos, "dev": torch.device("cuda", 0)}
    r = serving_record(args, ctxs, rates=(0.7, 1.0))
    print(json.dumps({
        "metric": "serving p99 latency (ms), Poisson arrivals at 0.7x saturated throughput",
        "value": r["at_0.7x"]["p99_ms"], "unit": "ms", "n_gpus": 1, "steps": r["requests"],
        "warmup": r["requests"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded plume fields and speckle patterns)",
        "config": {"workload": "serving", "requests": r["requests"], "slots": r["slots"],
                   "admission_limit_gb": r["admission_limit_gb"], "mix": r["mix"]},
        "latency_ms": r["latency_ms_at_0.7x"], "at_0.7x": r["at_0.7x"], "at_1.0x": r["at_1.0x"],
        "saturated": r["saturated"]}))


# ------------------------------------------------------------------ reconstruction loop

RECON_ITERS_PER_STEP = 100


def recon_arm(args):
    """Voxel reconstruction on the paper's measurement set-up (Sec. 3.1-3.2): 64^3 grid over
    the room, 100 x 100 sensor with 2 samples per pixel, 5000-pixel minibatches, AdaBelief,
    and the paper's quasi-linear tracer (Sec. 2.2).
    One iteration = minibatch draw, field build, subset render, minibatch L_BOS, backward and
    the AdaBelief update, all on the device.  A timed step is RECON_ITERS_PER_STEP iterations."""
    import torch

    from paper_2509_14442_gb300 import bos
    from paper_2509_14442_gb300.recon import Reconstructor

    dev = torch.device("cuda", 0)
    sc = quasi(S.paper_sensor())
    truth = torch.as_tensor(sc.T, device=dev)
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP, T=truth)
    target, _, _ = ctx.render(disp=False)
    ctx.close()

    def full_loss(T):
        c = bos.Context(0)
        c.set_scene(sc, bos.BOS_PREC_FP32_COMP, T=T.contiguous())
        I, _, _ = c.render(disp=False)
        torch.cuda.synchronize()
        c.close()
        return float(((I - target) ** 2).sum())

    T0 = torch.full_like(truth, S.T_AMBIENT)
    loss0 = full_loss(T0)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def timed(rec, graph: bool, clk=None):
        """ms per RECON_ITERS_PER_STEP iterations, launched call by call or as graph replays."""
        def chunk():
            if graph:
                rec.run(RECON_ITERS_PER_STEP)
            else:
                for _ in range(RECON_ITERS_PER_STEP):
                    rec.step()
        for _ in range(args.warmup):
            chunk()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        for k in range(args.steps):
            flush.fill_(0.0)
            ev[2 * k].record(stream)
            chunk()
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]))

    eager = Reconstructor(sc, target, T0, batch=5000, lr=0.2, loss_scale=1e11, seed=1)
    ms_eager = timed(eager, False)
    eager.close()
    rec = Reconstructor(sc, target, T0, batch=5000, lr=0.2, loss_scale=1e11, seed=1)
    with Clocks(0) as clk:
        ms = timed(rec, True)
    # ray-steps of one iteration's minibatch render (every one is also reversed)
    counts = []
    for _ in range(4):
        rec.step()
        torch.cuda.synchronize()
        counts.append(rec.ctx.last_ray_steps())
    rs_per_iter = float(np.mean(counts))
    loss1 = full_loss(rec.T)
    iters_done = rec.it
    rec.close()
    it_per_s = RECON_ITERS_PER_STEP * 1e3 / ms
    print(json.dumps({
        "metric": "reconstruction iterations/s", "value": it_per_s, "unit": "iterations/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded plume field, its own render as the measurement)",
        "config": {"workload": "recon", "grid": [64, 64, 64], "image": [100, 100], "spp": 2, "batch": 5000,
                   "tracer": "quasi-linear (Sec. 2.2)", "minibatch_order": "Z-order sorted (bos_sort_pixels)",
                   "iterations_per_step": RECON_ITERS_PER_STEP, "optimizer": "AdaBelief lr 0.2, loss scale 1e11",
                   "launch": "one CUDA graph replay per iteration",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "ray_steps_per_s": rs_per_iter * it_per_s, "ray_steps_per_iteration": rs_per_iter,
        "eager_iterations_per_s": RECON_ITERS_PER_STEP * 1e3 / ms_eager,
        "loss_full_image": {"start": loss0, "after": loss1, "iterations": iters_done},
        "clocks": clk.summary(),
    }))


# ------------------------------------------------------------------ precision variants

def bf16_round(x):
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def precision_record(args, ctxs, P, scene, orc) -> dict:
    """The 256^2x192 / 2048^2 scene rendered by every precision: render time, its share of
    the arithmetic peak and, given the oracle's renders of a pixel sample (`orc`, from the
    CPU-baseline leg; None leaves the error columns out), displacement and intensity errors
    against the FP64 oracle (for BF16 also against the oracle on the BF16-rounded field)."""
    torch, bos, dev = ctxs["torch"], ctxs["bos"], ctxs["dev"]
    T = torch.as_tensor(scene.T, device=dev)
    fp32_peak, _ = alu_peak_of("fp32_comp", P)
    fp64_peak, _ = alu_peak_of("fp64", P)
    dmax = float(np.abs(orc["true"]["disp"]).max()) if orc else None

    def err(I, D, ref):
        pix = orc["pix"]
        return {"disp_rel": float(np.abs(D.reshape(-1, 2)[pix] - ref["disp"]).max()) / dmax,
                "I_abs": float(np.abs(I.reshape(-1)[pix] - ref["I"]).max())}

    out = {}
    for name in ("fp64", "fp32", "fp32_comp", "bf16_comp"):
        ctx = bos.Context(dev.index)
        ctx.set_scene(scene, bos.PRECISIONS[name], T=T)
        reps = 1 if name == "fp64" else 5
        ms = []
        for i in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            I, D, _ = ctx.render(disp=True)
            e1.record()
            e1.synchronize()
            if i:
                ms.append(e0.elapsed_time(e1))
        ctx.status()
        steps = ctx.last_ray_steps()
        rate = steps / (statistics.mean(ms) * 1e-3)
        tflops = rate * FLOPS_PER_STEP["rkn"] / 1e12
        peak = fp64_peak if name == "fp64" else fp32_peak
        r = {"render_ms": statistics.mean(ms), "ray_steps_per_s": rate,
             "alu": {"achieved_tflops": tflops, "peak_tflops": peak, "frac": tflops / peak,
                     "dtype": "f64" if name == "fp64" else "f32"}}
        if orc is not None:
            Ih, Dh = I.cpu().numpy().astype(np.float64), D.cpu().numpy().astype(np.float64)
            r["vs_fp64_oracle"] = err(Ih, Dh, orc["true"])
            if name == "bf16_comp":
                r["vs_oracle_on_bf16_field"] = err(Ih, Dh, orc["bf16"])
        out[name] = r
        ctx.close()
    del T
    torch.cuda.empty_cache()
    return {"grid": list(scene.grid.n), "image": [scene.camera.width, scene.camera.height], "spp": scene.camera.spp,
            "sample_pixels": int(len(orc["pix"])) if orc else 0, "max_displacement_m": dmax,
            "errors": "against the FP64 oracle's render of the CPU-baseline leg's pixel sample" if orc else None,
            "precisions": out}


def precision_arm(args):
    import torch

    from paper_2509_14442_gb300 import bos

    ctxs = {"torch": torch, "bos": bos, "dev": torch.device("cuda", 0)}
    scene = S.room_adjoint(S.BASE_SEED + 2)
    P = measure_peaks(ctxs)
    cpu, orc = cpu_leg(scene, False, args.cpu_seconds, args.sample_pixels)
    r = precision_record(args, ctxs, P, scene, orc)
    print(json.dumps({
        "metric": "ray-steps/s and errors per precision (forward render)",
        "value": r["precisions"]["fp32_comp"]["ray_steps_per_s"], "unit": "ray-steps/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded plume fields and speckle patterns)",
        "config": {"workload": "precision", "grid": r["grid"], "image": r["image"], "spp": r["spp"],
                   "sample_pixels": r["sample_pixels"], "max_displacement_m": r["max_displacement_m"]},
        "fma_probe_tflops": P["fma"], "precisions": r["precisions"], "cpu_baseline": cpu}))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "serving":
        serving_arm(args)
    elif args.workload == "precision":
        precision_arm(args)
    elif args.workload == "recon":
        recon_arm(args)
    elif args.workload == "oracle":
        oracle_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
