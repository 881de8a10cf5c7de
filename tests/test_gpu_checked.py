"""The checked build (libbos_checked.so, BOS_CHECKED=1) on the GPU: the paths of the
library run through it with every field-store gather, node-accumulator atomic and
checkpoint access bounds-checked, report no out-of-range index, and give the same images
(and, up to the float32 atomics' order, the same gradients) as the ordinary build; an
understated store bound makes the checks fire without any access leaving the store."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Each case: name, scene maker (from the scenes module), precision name, adjoint
CASES = [
    ("rkn_fp32comp", "S.room((40, 40, 30), 61, 47, 2, 5201)", "fp32_comp", True),
    ("quasi_fp32comp", "quasi(S.room((40, 40, 30), 64, 48, 1, 5202))", "fp32_comp", True),
    ("rkn_bf16", "S.room((32, 32, 24), 48, 40, 1, 5203)", "bf16_comp", True),
    ("rkn_fp64", "S.room((24, 24, 18), 32, 24, 1, 5204)", "fp64", True),
    ("plain_fp32", "S.room((32, 32, 24), 48, 40, 3, 5205)", "fp32", False),
    ("refracted", "refr(S.room((40, 40, 30), 64, 48, 1, 5206))", "fp32_comp", True),
    ("blob_rk4", "S.blob_cube().replace(integ=S.Integrator(fixed_steps=128, integrator=1))", "fp32_comp", False),
]

SCRIPT = r'''
import json, sys, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2509_14442_gb300 import bos, scenes as S
quasi = lambda sc: sc.replace(integ=S.Integrator(fixed_steps=0, max_step_vox=0.5, integrator=2))
refr = lambda sc: sc.replace(light=S.Light(2, sc.light.pattern, sc.light.proj, connect_iters=1))
out = {"checked": int(bos.lib().bos_checked_build())}
for name, make, prec, adj in CASES:
    sc = eval(make)
    ctx = bos.Context(0)
    ctx.set_scene(sc, bos.PRECISIONS[prec])
    I, D, _ = ctx.render(disp=True, save_for_backward=adj)
    r = {"I": I.cpu().numpy().tolist(), "disp": D.cpu().numpy().tolist()}
    if adj:
        w = np.random.default_rng(7).standard_normal((sc.camera.height, sc.camera.width)).astype(np.float32)
        r["g"] = ctx.backward(torch.as_tensor(w, device="cuda")).cpu().numpy().tolist()
    torch.cuda.synchronize()
    ctx.status()
    ctx.close()
    out[name] = r
# an understated store bound: gathers beyond the first brick are reported (and read element 0)
sc = S.room((40, 40, 30), 32, 24, 1, 5207)
ctx = bos.Context(0)
ctx.set_scene(sc, bos.BOS_PREC_FP32_COMP)
st = bos.lib().bos_debug_store_bound(ctx.h, 729)
if st != bos.BOS_OK:
    out["fired"] = [st, bos.lib().bos_last_error().decode()]
else:
    ctx.render(disp=True)
    torch.cuda.synchronize()
    try:
        ctx.status()
        out["fired"] = None
    except bos.BosError as e:
        out["fired"] = [e.status, str(e)]
ctx.close()
json.dump(out, open(sys.argv[1], "w"))
'''


def run(tmp_path, checked: bool):
    path = tmp_path / ("checked.json" if checked else "plain.json")
    src = "ROOT = %r\nCASES = %r\n" % (ROOT, CASES) + SCRIPT
    env = dict(os.environ, BOS_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, "-c", src, str(path)], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.load(open(path))


def test_checked_build_finds_nothing_and_matches_the_ordinary_build(tmp_path):
    c = run(tmp_path, True)
    p = run(tmp_path, False)
    assert c["checked"] == 1 and p["checked"] == 0
    for name, _, _, adj in CASES:
        assert np.array_equal(np.array(c[name]["I"]), np.array(p[name]["I"])), name
        assert np.array_equal(np.array(c[name]["disp"]), np.array(p[name]["disp"])), name
        if adj:
            gc, gp = np.array(c[name]["g"]), np.array(p[name]["g"])
            assert np.linalg.norm(gc - gp) <= 1e-5 * np.linalg.norm(gp), name
    # the checks fire on an understated bound; the ordinary build has no checks to fire
    from paper_2509_14442_gb300 import bos
    assert c["fired"] is not None and c["fired"][0] == bos.BOS_ERR_DEVICE_CHECK
    assert "outside its buffer" in c["fired"][1]
    assert p["fired"] is not None and p["fired"][0] == bos.BOS_ERR_UNIMPLEMENTED
