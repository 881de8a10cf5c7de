"""ctypes front end of the FP64 CPU oracle (``bos_oracle.cpp``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares nothing with the CUDA library
except the seeded scene descriptions it is handed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bos_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc.so")


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("origin", C.c_double * 3), ("extent", C.c_double * 3),
                ("T0", C.c_double), ("rho0", C.c_double), ("G", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("fwd", C.c_double * 3), ("up", C.c_double * 3),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int), ("height", C.c_int), ("spp", C.c_int), ("seed", C.c_uint64)]


class Wall(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("eu", C.c_double * 3), ("ev", C.c_double * 3),
                ("normal", C.c_double * 3), ("size_u", C.c_double), ("size_v", C.c_double)]


class Light(C.Structure):
    _fields_ = [("mode", C.c_int), ("proj", Camera), ("tw", C.c_int), ("th", C.c_int),
                ("pattern", C.POINTER(C.c_float)), ("connect_iters", C.c_int)]


class Integ(C.Structure):
    _fields_ = [("fixed_steps", C.c_int), ("max_step_vox", C.c_double), ("integrator", C.c_int)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("deta", C.POINTER(C.c_double)), ("grad", C.POINTER(C.c_double)),
                ("p", C.c_double * 8)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        d, i, l, v = C.c_double, C.c_int, C.c_long, C.c_void_p
        P = C.POINTER
        _lib.orc_splitmix64_output.restype = C.c_uint64
        _lib.orc_splitmix64_output.argtypes = [C.c_uint64, C.c_uint64]
        _lib.orc_tent_inverse.restype = d
        _lib.orc_tent_inverse.argtypes = [d]
        for name in ("orc_deta_from_T", "orc_grad_from_deta"):
            getattr(_lib, name).argtypes = [P(Grid), v, v]
        _lib.orc_field_eval.argtypes = [P(Grid), P(Field), l, v, v, v]
        _lib.orc_trace_segment.argtypes = [P(Grid), P(Field), v, v, d, l, i, v, v, v, v]
        _lib.orc_ray_setup.argtypes = [P(Grid), P(Camera), P(Wall), P(Integ), l, i, v, v, v, v, v, v, v]
        _lib.orc_luminance.argtypes = [P(Light), P(Wall), l, v, v]
        _lib.orc_connect.argtypes = [P(Grid), P(Field), P(Wall), P(Light), P(Integ), l, v, i, v, v]
        _lib.orc_render.argtypes = [P(Grid), P(Field), P(Camera), P(Wall), P(Light), P(Integ), l, v, i, i,
                                    v, v, v, v]
        _lib.orc_render_cs.argtypes = [P(Grid), v, v, d, P(Camera), P(Wall), P(Light), P(Integ), l, v, i, v, v]
        _lib.orc_grad.argtypes = [P(Grid), v, P(Camera), P(Wall), P(Light), P(Integ), v, i, v, v, v]
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ descriptors

def grid_desc(g) -> Grid:
    return Grid((C.c_int * 3)(*g.n), (C.c_double * 3)(*g.origin), (C.c_double * 3)(*g.extent),
                g.T0, g.rho0, g.G)


def camera_desc(c) -> Camera:
    return Camera((C.c_double * 3)(*c.pos), (C.c_double * 3)(*c.fwd), (C.c_double * 3)(*c.up),
                  c.fx, c.fy, c.cx, c.cy, c.width, c.height, c.spp, c.seed)


def wall_desc(w) -> Wall:
    return Wall((C.c_double * 3)(*w.origin), (C.c_double * 3)(*w.eu), (C.c_double * 3)(*w.ev),
                (C.c_double * 3)(*w.normal), w.size_u, w.size_v)


class _LightHolder:
    def __init__(self, light):
        self.pattern = np.ascontiguousarray(light.pattern, dtype=np.float32)
        th, tw = self.pattern.shape
        proj = camera_desc(light.proj) if light.proj is not None else Camera()
        self.desc = Light(light.mode, proj, tw, th, self.pattern.ctypes.data_as(C.POINTER(C.c_float)),
                          int(getattr(light, "connect_iters", 1)))


def integ_desc(it) -> Integ:
    return Integ(it.fixed_steps, it.max_step_vox, it.integrator)


class NodeField:
    """Grid field given by FP64 node arrays deta (nz, ny, nx) and grad (nz, ny, nx, 3)."""

    def __init__(self, deta, grad):
        self.deta = _f64(deta)
        self.grad = _f64(grad)
        self.desc = Field(0, self.deta.ctypes.data_as(C.POINTER(C.c_double)),
                          self.grad.ctypes.data_as(C.POINTER(C.c_double)), (C.c_double * 8)())


class AnalyticField:
    """kind 1: eta^2 = p0 + p1 x + p2 y + p3 z; kind 2: eta = p0 + p1 x + p2 y + p3 z;
    kind 3: eta = 1 + p0 + p1 exp(-|x - (p2, p3, p4)|^2 / (2 p5^2))."""

    def __init__(self, kind: int, params):
        p = list(params) + [0.0] * (8 - len(params))
        self.desc = Field(kind, None, None, (C.c_double * 8)(*p))


# ------------------------------------------------------------------ field build

def deta_from_T(grid, T) -> np.ndarray:
    T = _f64(T)
    out = np.empty_like(T)
    lib().orc_deta_from_T(C.byref(grid_desc(grid)), _ptr(T), _ptr(out))
    return out


def grad_from_deta(grid, deta) -> np.ndarray:
    deta = _f64(deta)
    out = np.empty(deta.shape + (3,), dtype=np.float64)
    lib().orc_grad_from_deta(C.byref(grid_desc(grid)), _ptr(deta), _ptr(out))
    return out


def field_from_T(grid, T) -> NodeField:
    de = deta_from_T(grid, T)
    return NodeField(de, grad_from_deta(grid, de))


def field_eval(grid, field, x):
    x = _f64(x).reshape(-1, 3)
    eta = np.empty(x.shape[0])
    g = np.empty((x.shape[0], 3))
    lib().orc_field_eval(C.byref(grid_desc(grid)), C.byref(field.desc), x.shape[0], _ptr(x), _ptr(eta), _ptr(g))
    return eta, g


# ------------------------------------------------------------------ rays

def trace_segment(grid, field, r_in, d, ell, N, integrator=0, tape=False):
    r_in, d = _f64(r_in), _f64(d)
    r = np.empty(3)
    v = np.empty(3)
    ls = np.empty(1)
    tp = np.empty((N + 1, 6)) if tape else None
    lib().orc_trace_segment(C.byref(grid_desc(grid)), C.byref(field.desc), _ptr(r_in), _ptr(d), float(ell),
                            int(N), int(integrator), _ptr(r), _ptr(v), _ptr(ls), _ptr(tp))
    return (r, v, ls[0], tp) if tape else (r, v, ls[0])


def ray_setup(scene, pix: int, s: int):
    xy = np.empty(2)
    d = np.empty(3)
    t_in, ell, tw = np.empty(1), np.empty(1), np.empty(1)
    N = np.empty(1, dtype=np.int64)
    flags = np.empty(1, dtype=np.int32)
    lib().orc_ray_setup(C.byref(grid_desc(scene.grid)), C.byref(camera_desc(scene.camera)),
                        C.byref(wall_desc(scene.wall)), C.byref(integ_desc(scene.integ)), int(pix), int(s),
                        _ptr(xy), _ptr(d), _ptr(t_in), _ptr(ell), _ptr(tw), _ptr(N), _ptr(flags))
    return dict(xy=xy, d=d, t_in=t_in[0], ell=ell[0], tw=tw[0], N=int(N[0]), wall=bool(flags[0] & 1),
                traced=bool(flags[0] & 2))


def splitmix64_output(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64_output(seed, k))


def tent_inverse(xi: float) -> float:
    return float(lib().orc_tent_inverse(xi))


def luminance(light, wall, x) -> np.ndarray:
    x = _f64(x).reshape(-1, 3)
    out = np.empty(x.shape[0])
    lh = _LightHolder(light)
    lib().orc_luminance(C.byref(lh.desc), C.byref(wall_desc(wall)), x.shape[0], _ptr(x), _ptr(out))
    return out


def connect(scene, x, iters: int = -1, field=None):
    """Refracted projector connection of wall points x (n, 3): returns (a, y), the aim after
    `iters` rounds (default: the light's connect_iters) and the wall hit of the projector
    ray aimed at it."""
    if field is None:
        field = field_from_T(scene.grid, scene.T)
    x = _f64(x).reshape(-1, 3)
    a = np.empty_like(x)
    y = np.empty_like(x)
    lh = _LightHolder(scene.light)
    lib().orc_connect(C.byref(grid_desc(scene.grid)), C.byref(field.desc), C.byref(wall_desc(scene.wall)),
                      C.byref(lh.desc), C.byref(integ_desc(scene.integ)), x.shape[0], _ptr(x), int(iters),
                      _ptr(a), _ptr(y))
    return a, y


# ------------------------------------------------------------------ render

def render(scene, field=None, pix=None, straight: bool = False, threads: int = 0, nsteps: bool = False):
    """Render pixels of `scene` (all, or the flat indices `pix`).  `field` defaults to the
    field built from scene.T in FP64.  Returns dict(I, disp, hit[, nsteps]); I has shape
    (npix,) or (H, W) when rendering all pixels."""
    if field is None:
        field = field_from_T(scene.grid, scene.T)
    cam = scene.camera
    full = pix is None
    npix = cam.width * cam.height if full else len(pix)
    pix_a = None if full else np.ascontiguousarray(pix, dtype=np.int64)
    I = np.empty(npix)
    disp = np.empty((npix, 2))
    hit = np.empty((npix, 2))
    ns = np.empty(npix * cam.spp, dtype=np.int64) if nsteps else None
    lh = _LightHolder(scene.light)
    lib().orc_render(C.byref(grid_desc(scene.grid)), C.byref(field.desc), C.byref(camera_desc(cam)),
                     C.byref(wall_desc(scene.wall)), C.byref(lh.desc), C.byref(integ_desc(scene.integ)),
                     npix, _ptr(pix_a), int(straight), int(threads), _ptr(I), _ptr(disp), _ptr(hit), _ptr(ns))
    out = dict(I=I, disp=disp, hit=hit)
    if nsteps:
        out["nsteps"] = ns.reshape(npix, cam.spp)
    if full:
        H, W = cam.height, cam.width
        out = {k: v.reshape((H, W) + v.shape[1:]) for k, v in out.items()}
    return out


def render_cs(scene, dT, h: float = 1e-20, pix=None, threads: int = 0):
    """Complex-step directional derivative of (I, disp) along dT (same shape as scene.T)."""
    cam = scene.camera
    full = pix is None
    npix = cam.width * cam.height if full else len(pix)
    pix_a = None if full else np.ascontiguousarray(pix, dtype=np.int64)
    T = _f64(scene.T)
    dT = _f64(dT)
    dI = np.empty(npix)
    dd = np.empty((npix, 2))
    lh = _LightHolder(scene.light)
    lib().orc_render_cs(C.byref(grid_desc(scene.grid)), _ptr(T), _ptr(dT), float(h), C.byref(camera_desc(cam)),
                        C.byref(wall_desc(scene.wall)), C.byref(lh.desc), C.byref(integ_desc(scene.integ)),
                        npix, _ptr(pix_a), int(threads), _ptr(dI), _ptr(dd))
    if full:
        return dI.reshape(cam.height, cam.width), dd.reshape(cam.height, cam.width, 2)
    return dI, dd


def grad(scene, dLdI, threads: int = 0, nodes: bool = False):
    """dL/dT for the seed dL/dI (H, W), by the discrete adjoint (Sharma RKN)."""
    T = _f64(scene.T)
    w = _f64(dLdI)
    out = np.empty_like(T)
    nde = np.empty_like(T) if nodes else None
    ng = np.empty(T.shape + (3,)) if nodes else None
    lh = _LightHolder(scene.light)
    lib().orc_grad(C.byref(grid_desc(scene.grid)), _ptr(T), C.byref(camera_desc(scene.camera)),
                   C.byref(wall_desc(scene.wall)), C.byref(lh.desc), C.byref(integ_desc(scene.integ)),
                   _ptr(w), int(threads), _ptr(out), _ptr(nde), _ptr(ng))
    return (out, nde, ng) if nodes else out
