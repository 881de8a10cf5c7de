"""Host-side pieces of the benchmark that need no GPU: the reference arm's refusal of
workloads it does not time, its silence on ranks other than 0, the DRAM-traffic guard
and the per-ray-step tables behind the rooflines."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _bench(*args, env=None):
    e = dict(os.environ, **(env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=300, env=e, cwd=ROOT)


def test_reference_arm_refuses_workloads_it_does_not_time():
    r = _bench("--impl", "reference", "--workload", "serving")
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_reference_arm_is_silent_on_other_ranks():
    r = _bench("--impl", "reference", env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_traffic_is_reported_only_for_the_captured_sources():
    """The DRAM traffic of a timed launch is the small-case capture with its per-ray
    algorithmic bytes replaced by the timed launch's, and only while the kernel sources
    hash to the captured ones."""
    import bench

    from paper_2509_14442_gb300 import scenes

    sc = scenes.room((16, 16, 12), 64, 32, 1, 7, field=False)
    alg = bench.algorithmic_hbm(sc, ckpt_slots=1000, store_bytes=4096)
    rays = 1000 * 48 + sc.rays * 4 + sc.pixels * 4
    assert alg["render_kernel"] == {"rays": rays, "grid": 4096, "total": rays + 4096}
    assert alg["adjoint_kernel"]["grid"] == 4096 + sc.grid.cells * 32
    # the committed capture: the small case's per-ray bytes follow from its own counts
    small = scenes.room((256, 256, 192), 512, 512, 1, 7, field=False)
    cap = bench.TRAFFIC_CAPTURE
    assert cap["rays"]["adjoint_kernel"] == 8650752 * 48 + small.rays * 4 + small.pixels * 4
    saved = {k: (dict(v) if isinstance(v, dict) else v) for k, v in cap.items()}
    try:
        cap.update(sha256=bench.kernel_sources_sha256(), adjoint_kernel=3.0e6,
                   rays={"render_kernel": 1.0, "adjoint_kernel": 1.0e6})
        t = bench.kernel_traffic("adjoint_kernel", alg)
        assert t["bytes"] == 3.0e6 - 1.0e6 + rays
        cap["sha256"] = "0" * 64                                          # sources changed since the capture
        assert bench.kernel_traffic("adjoint_kernel", alg) is None
    finally:
        cap.clear()
        cap.update(saved)


def test_reference_arm_reports_the_gpu_arms_config_and_its_measured_time(monkeypatch, capsys):
    """The reference arm names the same workload keys as the GPU arm (grid, image, spp,
    ckpt_every) and reports the measured time of its samples as ms_per_step."""
    import argparse

    import bench

    def fake_rate(scene, adjoint, seconds, seed=0, threads=0):
        return {"rate": 1.0e6, "threads": 3, "seconds": 0.25, "pix": None, "out": None, "desc": "fake sample"}

    monkeypatch.setattr(bench, "oracle_rate", fake_rate)
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(workload="room_fwd_small", steps=2, warmup=1, gpus=1, prec="fp32_comp")
    bench.reference_arm(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    wl = bench.WORKLOADS["room_fwd_small"]
    want = bench.config_of(args, wl, wl["make"](bench.S.BASE_SEED + 1))
    assert line["config"] == want
    for k in ("grid", "image", "spp", "ckpt_every", "workload"):
        assert k in line["config"]
    assert line["ms_per_step"] == 250.0
    assert line["cpu_baseline"]["cores"] == 3 and line["e2e"]["h2d_bytes_per_step"] == 0


def test_per_ray_step_tables_follow_their_counts():
    import bench

    ev = 6 + 7 * 3 * 4 + 4                                   # fractions, 4-channel trilinear, D
    assert ev == 94
    assert bench.FLOPS_PER_STEP["rkn"] == 3 * ev + 9 + 24 + 18 + 15 + 8
    assert bench.FLOPS_PER_STEP["quasi"] == 2 * (6 + ev) + 41
    assert bench.ADJ_FLOPS_PER_STEP["rkn"] == bench.FLOPS_PER_STEP["rkn"] + 3 * (6 + 4 * 36) + 3 * 36 + 66 + 11 + 3 * 83
    assert bench.ADJ_FLOPS_PER_STEP["quasi"] == 2 * (96 + 9 + 83) + 24
    assert bench.BYTES_PER_STEP["fp32_comp"] == 3 * 8 * 16                # 3 evaluations x 8 corners x float4
    assert bench.ADJ_BYTES_PER_STEP["fp32_comp"] == 3 * bench.BYTES_PER_STEP["fp32_comp"]
    assert bench.L1_BYTES_PER_STEP["fp32_comp"] == 3 * 8 * 16
    assert bench.ADJ_L1_BYTES_PER_STEP["fp32_comp"] == 2 * bench.L1_BYTES_PER_STEP["fp32_comp"]


def test_profile_commands_name_existing_workloads():
    # every command recorded under profiles/ runs committed files: bench.py with a workload
    # that bench.py still defines
    import re

    import bench

    names = set(bench.WORKLOADS) | {"serving", "precision", "recon", "oracle"}
    found = 0
    pdir = os.path.join(ROOT, "profiles")
    for fn in sorted(os.listdir(pdir)):
        with open(os.path.join(pdir, fn)) as f:
            text = f.read()
        for w in re.findall(r"bench\.py --workload ([A-Za-z0-9_]+)", text):
            assert w in names, (fn, w)
            found += 1
        assert "bench.py" in text, fn
    assert found > 0
