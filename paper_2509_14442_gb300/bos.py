"""Thin ctypes binding of the BOS C ABI (include/bos.h) with the same names.

Argument marshalling only: every step of the forward model and of its adjoint runs
in the CUDA library (libbos.so, built in-tree for sm_103a).  PyTorch provides device
memory and streams.  There is no CPU fallback: if the library cannot be loaded the
import of `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import _build

BOS_OK = 0
BOS_ERR_INVALID_ARG = 1
BOS_ERR_NOT_READY = 2
BOS_ERR_OOM = 3
BOS_ERR_ADMISSION = 4
BOS_ERR_CUDA = 5
BOS_ERR_TIMEOUT = 6
BOS_ERR_DEVICE_CHECK = 7
BOS_ERR_UNIMPLEMENTED = 8

BOS_PREC_FP64 = 0
BOS_PREC_FP32 = 1
BOS_PREC_FP32_COMP = 2
BOS_PREC_BF16_COMP = 3

PRECISIONS = {"fp64": BOS_PREC_FP64, "fp32": BOS_PREC_FP32, "fp32_comp": BOS_PREC_FP32_COMP,
              "bf16_comp": BOS_PREC_BF16_COMP}


class BosError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class bos_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("origin", C.c_double * 3),
                ("extent", C.c_double * 3), ("T0", C.c_double), ("rho0", C.c_double), ("G", C.c_double),
                ("prec", C.c_int)]


class bos_camera_desc(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("fwd", C.c_double * 3), ("up", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int),
                ("height", C.c_int), ("spp", C.c_int), ("seed", C.c_uint64)]


class bos_wall_desc(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("eu", C.c_double * 3), ("ev", C.c_double * 3),
                ("normal", C.c_double * 3), ("size_u", C.c_double), ("size_v", C.c_double)]


class bos_light_desc(C.Structure):
    _fields_ = [("mode", C.c_int), ("proj", bos_camera_desc), ("tw", C.c_int), ("th", C.c_int),
                ("connect_iters", C.c_int)]


class bos_integrator_desc(C.Structure):
    _fields_ = [("fixed_steps", C.c_int), ("max_step_vox", C.c_double), ("integrator", C.c_int),
                ("ckpt_every", C.c_int)]


class bos_request(C.Structure):
    _fields_ = [("grid", bos_grid_desc), ("T_dev", C.c_void_p), ("cam", bos_camera_desc), ("wall", bos_wall_desc),
                ("light", bos_light_desc), ("pattern_dev", C.c_void_p), ("integ", bos_integrator_desc),
                ("I_dev", C.c_void_p), ("disp_dev", C.c_void_p), ("target_dev", C.c_void_p),
                ("loss_dev", C.c_void_p), ("dLdT_dev", C.c_void_p)]


class bos_ticket_info(C.Structure):
    _fields_ = [("submit_ns", C.c_uint64), ("admit_ns", C.c_uint64), ("done_ns", C.c_uint64),
                ("footprint_bytes", C.c_uint64), ("status", C.c_int), ("done", C.c_int), ("slot", C.c_int)]


BOS_SERVER_FAKE_EXECUTOR = 1

# every exported symbol of include/bos.h: name -> (restype, argtypes)
_v, _i, _u64, _i64, _d = C.c_void_p, C.c_int, C.c_uint64, C.c_int64, C.c_double
_P = C.POINTER
SIGNATURES = {
    "bos_create": (_i, [_P(_v), _i, _u64]),
    "bos_destroy": (_i, [_v]),
    "bos_set_grid": (_i, [_v, _P(bos_grid_desc), _v, _v]),
    "bos_set_geometry": (_i, [_v, _P(bos_camera_desc), _P(bos_wall_desc), _P(bos_light_desc), _v,
                              _P(bos_integrator_desc)]),
    "bos_render": (_i, [_v, _v, _v, _v, _i, _v]),
    "bos_render_reference": (_i, [_v, _v, _v, _v, _v]),
    "bos_render_pixels": (_i, [_v, _v, _i64, _v, _v, _i, _v]),
    "bos_ray_steps": (_i, [_v, _v, _v]),
    "bos_last_ray_steps": (_i, [_v, _P(_u64)]),
    "bos_loss_l2": (_i, [_v, _v, _i64, _v, _v, _v]),
    "bos_backward": (_i, [_v, _v, _v, _v]),
    "bos_backward_f64": (_i, [_v, _v, _v, _v]),
    "bos_loss_l2_pixels": (_i, [_v, _v, _v, _i64, C.c_float, _v, _v, _v]),
    "bos_sample_pixels": (_i, [_v, _i64, _i64, _u64, _u64, _v, _v]),
    "bos_adabelief_step": (_i, [_v, _v, _v, _v, _i64, C.c_float, C.c_float, C.c_float, C.c_float, _i64, _v, _v]),
    "bos_counter_add": (_i, [_v, _u64, _v]),
    "bos_sort_pixels": (_i, [_v, _i64, _i, _i, _v]),
    "bos_export_nodes": (_i, [_v, _v, _v]),
    "bos_probe_read": (_i, [_v, _u64, _i, _v, _v]),
    "bos_probe_fma": (_i, [_i, _i, _v, _P(_d), _v]),
    "bos_probe_read_l1": (_i, [_v, _u64, _i, _v, _P(_d), _v]),
    "bos_render_noalloc": (_i, [_P(bos_grid_desc), _v, _P(bos_camera_desc), _P(bos_wall_desc), _P(bos_light_desc),
                                _v, _P(bos_integrator_desc), _v, _v, _v]),
    "bos_noalloc_status": (_i, []),
    "bos_checked_build": (_i, []),
    "bos_debug_store_bound": (_i, [_v, C.c_uint32]),
    "bos_status": (_i, [_v]),
    "bos_error_string": (C.c_char_p, [_i]),
    "bos_last_error": (C.c_char_p, []),
    "bos_device_bytes": (_u64, [_v]),
    "bos_request_footprint": (_i, [_P(bos_request), _P(_u64)]),
    "bos_server_create": (_i, [_P(_v), _i, _u64, _i, _i]),
    "bos_submit": (_i, [_v, _P(bos_request), _P(_u64)]),
    "bos_wait": (_i, [_v, _u64, _u64]),
    "bos_ticket": (_i, [_v, _u64, _P(bos_ticket_info)]),
    "bos_server_stats": (_i, [_v, _P(_u64), _P(_u64), _P(_i), _P(_i)]),
    "bos_server_batches": (_i, [_v, _P(_u64), _P(_u64), _P(_u64), _P(_i)]),
    "bos_server_destroy": (_i, [_v, _u64]),
}

_lib = None


def checked() -> bool:
    """True when this process uses the checked build (environment BOS_CHECKED=1)."""
    return os.environ.get("BOS_CHECKED", "0") == "1"


def lib_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def lib(build: bool = True):
    """Load libbos.so, or libbos_checked.so with BOS_CHECKED=1 in the environment (building
    it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build(checked=checked()) if build else lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"BOS CUDA library not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != BOS_OK:
        L = lib()
        msg = L.bos_last_error().decode() or L.bos_error_string(status).decode()
        raise BosError(status, where, msg)


# ------------------------------------------------------------------ descriptors

def _v3(x):
    return (C.c_double * 3)(*[float(a) for a in x])


def grid_desc(g, prec: int) -> bos_grid_desc:
    return bos_grid_desc(g.n[0], g.n[1], g.n[2], _v3(g.origin), _v3(g.extent), g.T0, g.rho0, g.G, prec)


def camera_desc(c) -> bos_camera_desc:
    return bos_camera_desc(_v3(c.pos), _v3(c.fwd), _v3(c.up), c.fx, c.fy, c.cx, c.cy, c.width, c.height, c.spp,
                           int(c.seed) & 0xFFFFFFFFFFFFFFFF)


def wall_desc(w) -> bos_wall_desc:
    return bos_wall_desc(_v3(w.origin), _v3(w.eu), _v3(w.ev), _v3(w.normal), w.size_u, w.size_v)


def light_desc(L) -> bos_light_desc:
    th, tw = L.pattern.shape
    proj = camera_desc(L.proj) if L.proj is not None else bos_camera_desc()
    return bos_light_desc(L.mode, proj, tw, th, int(getattr(L, "connect_iters", 1)))


def integ_desc(it) -> bos_integrator_desc:
    return bos_integrator_desc(it.fixed_steps, it.max_step_vox, it.integrator, it.ckpt_every)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ------------------------------------------------------------------ raw calls (same names)

def bos_create(device: int = 0, mem_limit_bytes: int = 0) -> int:
    h = C.c_void_p()
    check(lib().bos_create(C.byref(h), device, mem_limit_bytes), "bos_create")
    return h.value


def bos_destroy(ctx: int) -> None:
    check(lib().bos_destroy(ctx), "bos_destroy")


def bos_set_grid(ctx: int, desc: bos_grid_desc, T_dev: int, stream: int) -> None:
    check(lib().bos_set_grid(ctx, C.byref(desc), T_dev, stream), "bos_set_grid")


def bos_set_geometry(ctx, cam, wall, light, pattern_dev, integ) -> None:
    check(lib().bos_set_geometry(ctx, C.byref(cam), C.byref(wall), C.byref(light), pattern_dev, C.byref(integ)),
          "bos_set_geometry")


def bos_render(ctx, I_dev, disp_dev, hit_dev, save_for_backward: int, stream) -> None:
    check(lib().bos_render(ctx, I_dev, disp_dev, hit_dev, int(save_for_backward), stream), "bos_render")


def bos_render_pixels(ctx, pix_dev, npix: int, I_dev, disp_dev, save_for_backward: int, stream) -> None:
    check(lib().bos_render_pixels(ctx, pix_dev, npix, I_dev, disp_dev, int(save_for_backward), stream),
          "bos_render_pixels")


def bos_render_reference(ctx, I_dev, disp_dev, hit_dev, stream) -> None:
    check(lib().bos_render_reference(ctx, I_dev, disp_dev, hit_dev, stream), "bos_render_reference")


def bos_ray_steps(ctx, nsteps_dev, stream) -> None:
    check(lib().bos_ray_steps(ctx, nsteps_dev, stream), "bos_ray_steps")


def bos_last_ray_steps(ctx) -> int:
    v = C.c_uint64()
    check(lib().bos_last_ray_steps(ctx, C.byref(v)), "bos_last_ray_steps")
    return v.value


def bos_loss_l2(I_dev, target_dev, n: int, loss_dev, dLdI_dev, stream) -> None:
    check(lib().bos_loss_l2(I_dev, target_dev, n, loss_dev, dLdI_dev, stream), "bos_loss_l2")


def bos_loss_l2_pixels(I_dev, target_dev, pix_dev, npix: int, loss_dev, dLdI_dev, stream, scale: float = 1.0) -> None:
    check(lib().bos_loss_l2_pixels(I_dev, target_dev, pix_dev, npix, scale, loss_dev, dLdI_dev, stream),
          "bos_loss_l2_pixels")


def bos_sample_pixels(pix_dev, npix: int, n_pixels: int, seed: int, draw: int, stream, draw_dev=None) -> None:
    check(lib().bos_sample_pixels(pix_dev, npix, n_pixels, seed, draw, draw_dev, stream), "bos_sample_pixels")


def bos_adabelief_step(theta_dev, grad_dev, m_dev, s_dev, n: int, lr: float, beta1: float, beta2: float, eps: float,
                       step: int, stream, step_dev=None) -> None:
    check(lib().bos_adabelief_step(theta_dev, grad_dev, m_dev, s_dev, n, lr, beta1, beta2, eps, step, step_dev,
                                   stream), "bos_adabelief_step")


def bos_sort_pixels(pix_dev, npix: int, width: int, height: int, stream) -> None:
    check(lib().bos_sort_pixels(pix_dev, npix, width, height, stream), "bos_sort_pixels")


def bos_counter_add(counter_dev, inc: int, stream) -> None:
    check(lib().bos_counter_add(counter_dev, inc, stream), "bos_counter_add")


def bos_backward(ctx, dLdI_dev, dLdT_dev, stream) -> None:
    check(lib().bos_backward(ctx, dLdI_dev, dLdT_dev, stream), "bos_backward")


def bos_backward_f64(ctx, dLdI_dev, dLdT_dev, stream) -> None:
    check(lib().bos_backward_f64(ctx, dLdI_dev, dLdT_dev, stream), "bos_backward_f64")


def bos_export_nodes(ctx, out_dev, stream) -> None:
    check(lib().bos_export_nodes(ctx, out_dev, stream), "bos_export_nodes")


def bos_probe_read(buf_dev, nbytes: int, repeats: int, sink_dev, stream) -> None:
    check(lib().bos_probe_read(buf_dev, nbytes, repeats, sink_dev, stream), "bos_probe_read")


def bos_probe_fma(kind: int, repeats: int, sink_dev, stream) -> float:
    """Launch the FMA-throughput probe; returns the launch's flop count."""
    flops = C.c_double(0.0)
    check(lib().bos_probe_fma(kind, repeats, sink_dev, C.byref(flops), stream), "bos_probe_fma")
    return flops.value


def bos_probe_read_l1(buf_dev, nbytes: int, repeats: int, sink_dev, stream) -> float:
    """Launch the L1 read-bandwidth probe; returns the bytes the launch reads."""
    nread = C.c_double(0.0)
    check(lib().bos_probe_read_l1(buf_dev, nbytes, repeats, sink_dev, C.byref(nread), stream), "bos_probe_read_l1")
    return nread.value


def bos_render_noalloc(grid: bos_grid_desc, T_dev, cam: bos_camera_desc, wall: bos_wall_desc,
                       light: bos_light_desc, pattern_dev, integ: bos_integrator_desc, I_dev, disp_dev, stream) -> None:
    check(lib().bos_render_noalloc(C.byref(grid), T_dev, C.byref(cam), C.byref(wall), C.byref(light), pattern_dev,
                                   C.byref(integ), I_dev, disp_dev, stream), "bos_render_noalloc")


def bos_noalloc_status() -> None:
    """Raise if the most recent bos_render_noalloc on the current device flagged an error."""
    check(lib().bos_noalloc_status(), "bos_noalloc_status")


def bos_status(ctx) -> None:
    check(lib().bos_status(ctx), "bos_status")


def bos_device_bytes(ctx) -> int:
    return int(lib().bos_device_bytes(ctx))


# ------------------------------------------------------------------ tensor-level context

class Context:
    """A BOS context bound to torch tensors.  Holds the T and pattern tensors it was
    given for as long as the library may read them."""

    def __init__(self, device: int = 0, mem_limit_bytes: int = 0):
        import torch

        self.device = device
        self.torch_device = torch.device("cuda", device)
        self.h = bos_create(device, mem_limit_bytes)
        self.T = None
        self.pattern = None
        self.scene = None
        self.prec = None

    def close(self):
        if self.h:
            import torch

            torch.cuda.synchronize(self.torch_device)
            bos_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_grid(self, grid, T, prec: int = BOS_PREC_FP32_COMP, stream=None):
        import torch

        assert T.is_cuda and T.dtype == torch.float32 and T.is_contiguous()
        assert tuple(T.shape) == (grid.n[2], grid.n[1], grid.n[0])
        bos_set_grid(self.h, grid_desc(grid, prec), T.data_ptr(), _stream(stream))
        self.T = T
        self.grid = grid
        self.prec = prec

    def set_geometry(self, camera, wall, light, integ, pattern=None):
        import torch

        pat = pattern if pattern is not None else torch.as_tensor(np.ascontiguousarray(light.pattern),
                                                                  device=self.torch_device)
        assert pat.is_cuda and pat.dtype == torch.float32 and pat.is_contiguous()
        bos_set_geometry(self.h, camera_desc(camera), wall_desc(wall), light_desc(light), pat.data_ptr(),
                         integ_desc(integ))
        self.pattern = pat
        self.camera = camera

    def set_scene(self, scene, prec: int = BOS_PREC_FP32_COMP, T=None, stream=None):
        import torch

        if T is None:
            T = torch.as_tensor(np.ascontiguousarray(scene.T, dtype=np.float32), device=self.torch_device)
        self.set_grid(scene.grid, T, prec, stream)
        self.set_geometry(scene.camera, scene.wall, scene.light, scene.integ)
        self.scene = scene

    def _outputs(self, disp: bool, hit: bool):
        import torch

        H, W = self.camera.height, self.camera.width
        I = torch.empty((H, W), dtype=torch.float32, device=self.torch_device)
        D = torch.empty((H, W, 2), dtype=torch.float32, device=self.torch_device) if disp else None
        X = torch.empty((H, W, 2), dtype=torch.float64, device=self.torch_device) if hit else None
        return I, D, X

    def render(self, disp: bool = True, hit: bool = False, save_for_backward: bool = False, stream=None, out=None):
        I, D, X = out if out is not None else self._outputs(disp, hit)
        bos_render(self.h, _ptr(I), _ptr(D), _ptr(X), int(save_for_backward), _stream(stream))
        return I, D, X

    def render_pixels(self, pix, disp: bool = False, save_for_backward: bool = False, stream=None):
        """Render the pixels of the int32 device tensor `pix` (flat indices); returns (I, disp)."""
        import torch

        assert pix.is_cuda and pix.dtype == torch.int32 and pix.is_contiguous()
        n = pix.numel()
        I = torch.empty((n,), dtype=torch.float32, device=self.torch_device)
        D = torch.empty((n, 2), dtype=torch.float32, device=self.torch_device) if disp else None
        bos_render_pixels(self.h, pix.data_ptr(), n, I.data_ptr(), _ptr(D), int(save_for_backward), _stream(stream))
        self._pix = pix
        return I, D

    def render_reference(self, disp: bool = False, hit: bool = False, stream=None):
        I, D, X = self._outputs(disp, hit)
        bos_render_reference(self.h, _ptr(I), _ptr(D), _ptr(X), _stream(stream))
        return I, D, X

    def ray_steps(self, stream=None):
        import torch

        c = self.camera
        n = torch.empty((c.height * c.width * c.spp,), dtype=torch.int32, device=self.torch_device)
        bos_ray_steps(self.h, n.data_ptr(), _stream(stream))
        return n

    def last_ray_steps(self) -> int:
        return bos_last_ray_steps(self.h)

    def export_nodes(self, stream=None):
        import torch

        g = self.grid
        shape = (g.n[2], g.n[1], g.n[0], 4)
        dt = {BOS_PREC_FP64: torch.float64, BOS_PREC_BF16_COMP: torch.int16}.get(self.prec, torch.float32)
        out = torch.empty(shape, dtype=dt, device=self.torch_device)
        bos_export_nodes(self.h, out.data_ptr(), _stream(stream))
        return out

    def backward(self, dLdI, stream=None):
        import torch

        assert dLdI.is_cuda and dLdI.dtype == torch.float32 and dLdI.is_contiguous()
        dT = torch.empty_like(self.T)
        bos_backward(self.h, dLdI.data_ptr(), dT.data_ptr(), _stream(stream))
        return dT

    def backward_f64(self, dLdI, stream=None):
        """dL/dT in float64 from a float64 dL/dI (FP64 renders)."""
        import torch

        assert dLdI.is_cuda and dLdI.dtype == torch.float64 and dLdI.is_contiguous()
        dT = torch.empty(self.T.shape, dtype=torch.float64, device=self.torch_device)
        bos_backward_f64(self.h, dLdI.data_ptr(), dT.data_ptr(), _stream(stream))
        return dT

    def status(self):
        bos_status(self.h)


def loss_l2(I, target, stream=None):
    """L_BOS = sum (target - I)^2 and dL/dI = -2 (target - I), both on the device."""
    import torch

    loss = torch.empty((1,), dtype=torch.float64, device=I.device)
    g = torch.empty_like(I)
    bos_loss_l2(I.data_ptr(), target.data_ptr(), I.numel(), loss.data_ptr(), g.data_ptr(), _stream(stream))
    return loss, g


# ------------------------------------------------------------------ request server

def make_request(grid, prec, T_dev, camera, wall, light, pattern_dev, integ, I_dev, disp_dev=None,
                 target_dev=None, loss_dev=None, dLdT_dev=None) -> bos_request:
    """A bos_request from scene descriptors and device pointers (ints or None)."""
    return bos_request(grid_desc(grid, prec), T_dev, camera_desc(camera), wall_desc(wall), light_desc(light),
                       pattern_dev, integ_desc(integ), I_dev, disp_dev, target_dev, loss_dev, dLdT_dev)


def bos_request_footprint(req: bos_request) -> int:
    v = C.c_uint64()
    check(lib().bos_request_footprint(C.byref(req), C.byref(v)), "bos_request_footprint")
    return v.value


class Server:
    """Continuous-batching request server (include/bos.h, request server section)."""

    def __init__(self, device: int = 0, mem_limit_bytes: int = 120 << 30, slots: int = 4, fake: bool = False):
        h = C.c_void_p()
        flags = BOS_SERVER_FAKE_EXECUTOR if fake else 0
        check(lib().bos_server_create(C.byref(h), device, mem_limit_bytes, slots, flags), "bos_server_create")
        self.h = h.value
        self.keep = {}          # ticket -> objects the request points into

    def submit(self, req: bos_request, keep=None) -> int:
        t = C.c_uint64()
        check(lib().bos_submit(self.h, C.byref(req), C.byref(t)), "bos_submit")
        if keep is not None:
            self.keep[t.value] = keep
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        """Status of the request (BOS_ERR_TIMEOUT if not done within the timeout)."""
        return int(lib().bos_wait(self.h, ticket, int(timeout_s * 1e9)))

    def info(self, ticket: int) -> dict:
        i = bos_ticket_info()
        check(lib().bos_ticket(self.h, ticket, C.byref(i)), "bos_ticket")
        return {f: getattr(i, f) for f, _ in bos_ticket_info._fields_}

    def stats(self) -> dict:
        a, p = C.c_uint64(), C.c_uint64()
        q, r = C.c_int(), C.c_int()
        check(lib().bos_server_stats(self.h, C.byref(a), C.byref(p), C.byref(q), C.byref(r)), "bos_server_stats")
        return dict(arena_bytes=a.value, peak_used_bytes=p.value, queued=q.value, running=r.value)

    def batches(self) -> dict:
        """Batched launches so far: launches, tiles, request shares, most requests per launch."""
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        m = C.c_int()
        check(lib().bos_server_batches(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(m)), "bos_server_batches")
        return dict(launches=a.value, tiles=b.value, job_shares=c.value, max_jobs=m.value)

    def close(self, timeout_s: float = 600.0) -> None:
        if self.h:
            check(lib().bos_server_destroy(self.h, int(timeout_s * 1e9)), "bos_server_destroy")
            self.h = None
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
