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
    import bench

    sha = bench.kernel_sources_sha256()
    assert bench.kernel_traffic("room_fwd", "render_kernel") is None          # another workload
    if bench.KERNEL_TRAFFIC["sha256"] == sha:
        assert bench.kernel_traffic("room_adj", "adjoint_kernel") == bench.KERNEL_TRAFFIC["adjoint_kernel"]
    saved = bench.KERNEL_TRAFFIC["sha256"]
    try:
        bench.KERNEL_TRAFFIC["sha256"] = "0" * 64                         # sources changed since the capture
        assert bench.kernel_traffic("room_adj", "adjoint_kernel") is None
    finally:
        bench.KERNEL_TRAFFIC["sha256"] = saved


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
