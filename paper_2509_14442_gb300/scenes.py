"""Seeded synthetic inputs for the BOS forward model.

This module only *makes inputs*: temperature fields, wall textures, projector
patterns and the camera / wall / projector geometry.  It holds none of the
method's arithmetic (no refractive index, no ray tracing, no rendering), so it
can feed both the CUDA path and the FP64 oracle.

The paper's own inputs (an OpenFOAM RANS temperature field and a wavelet-noise
projector pattern, Sec. 3.1) are not available; these generators stand in for
them with the paper's scene shape: a room whose side wall at x = -1.2 m holds an
inlet pointing +x (Sec. 3.2), a camera at (0.85, -29, 1.5) m and a projector at
(1.85, -29, 1.5) m, both looking +y with a long focal length (Sec. 3.1).

All randomness comes from ``numpy.random.default_rng(seed).random`` so that a
seed fixes every array bit for bit.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

# Physical constants of every scene: ambient temperature (K), ambient air
# density (kg/m^3) and Gladstone-Dale coefficient (m^3/kg).
T_AMBIENT = 293.0
RHO0 = 1.2
GLADSTONE_DALE = 2.26e-4

# Room of Sec. 3: inlet wall at x = -1.2 m, back wall at y = 4 m.
ROOM_ORIGIN = (-1.2, 0.0, 0.0)
ROOM_EXTENT = (4.0, 4.0, 3.0)
CAMERA_POS = (0.85, -29.0, 1.5)
PROJECTOR_POS = (1.85, -29.0, 1.5)
# Half of the wall height / width the camera and projector frame at the back wall.
CAMERA_HALF_VIEW = 1.45
PROJECTOR_HALF_VIEW = 3.1

BASE_SEED = 2509


@dataclass
class Grid:
    n: Tuple[int, int, int]              # (nx, ny, nz) cells
    origin: Tuple[float, float, float]   # box corner (m)
    extent: Tuple[float, float, float]   # box size (m)
    T0: float = T_AMBIENT
    rho0: float = RHO0
    G: float = GLADSTONE_DALE

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def spacing(self) -> Tuple[float, float, float]:
        return tuple(self.extent[a] / self.n[a] for a in range(3))

    def centers(self, axis: int) -> np.ndarray:
        h = self.extent[axis] / self.n[axis]
        return self.origin[axis] + (np.arange(self.n[axis], dtype=np.float64) + 0.5) * h


@dataclass
class Camera:
    pos: Tuple[float, float, float]
    fwd: Tuple[float, float, float]
    up: Tuple[float, float, float]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    spp: int = 1
    seed: int = 0


@dataclass
class Wall:
    origin: Tuple[float, float, float]
    eu: Tuple[float, float, float]
    ev: Tuple[float, float, float]
    normal: Tuple[float, float, float]
    size_u: float
    size_v: float


@dataclass
class Light:
    mode: int                       # 0: texture on the wall, 1: pinhole projector (straight
                                    # connection), 2: projector rays traced through the flow
    pattern: np.ndarray             # (th, tw) float32
    proj: Optional[Camera] = None   # projector pinhole (modes 1, 2)
    connect_iters: int = 1          # mode 2: projector rays traced per wall point


@dataclass
class Integrator:
    fixed_steps: int = 0            # > 0: this many steps per ray; 0: adaptive
    max_step_vox: float = 0.5       # adaptive step bound in units of the smallest cell size
    integrator: int = 0             # 0: Sharma RKN, 1: classic RK4, 2: quasi-linear (Sharma weights)
    ckpt_every: int = 16            # adjoint checkpoint interval (steps)


@dataclass
class Scene:
    name: str
    grid: Grid
    T: np.ndarray                   # (nz, ny, nx) float32, kelvin
    camera: Camera
    wall: Wall
    light: Light
    integ: Integrator = field(default_factory=Integrator)

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)

    @property
    def pixels(self) -> int:
        return self.camera.width * self.camera.height

    @property
    def rays(self) -> int:
        return self.pixels * self.camera.spp


# --------------------------------------------------------------------------
# fields
# --------------------------------------------------------------------------

def _cell_centers(grid: Grid):
    xc, yc, zc = (grid.centers(a) for a in range(3))
    return xc, yc, zc


def blob_field(grid: Grid, center, sigma: float, amplitude: float,
               ambient: float = T_AMBIENT) -> np.ndarray:
    """Ambient temperature plus one Gaussian hot blob, (nz, ny, nx) float32."""
    xc, yc, zc = _cell_centers(grid)
    d2 = ((xc[None, None, :] - center[0]) ** 2 + (yc[None, :, None] - center[1]) ** 2
          + (zc[:, None, None] - center[2]) ** 2)
    T = ambient + amplitude * np.exp(-d2 / (2.0 * sigma * sigma))
    return T.astype(np.float32)


def _bezier(p0, p1, p2, m: int) -> np.ndarray:
    t = np.linspace(0.0, 1.0, m)[:, None]
    return (1 - t) ** 2 * p0 + 2 * (1 - t) * t * p1 + t ** 2 * p2


def plume_params(seed: int) -> dict:
    """Seeded centreline and decay length of the inlet plume."""
    u = np.random.default_rng(seed).random(24)
    x0 = ROOM_ORIGIN[0]
    p0 = np.array([x0, 1.0 + 2.0 * u[0], 0.3 + 0.7 * u[1]])
    p1 = p0 + np.array([1.0 + 0.8 * u[2], -0.3 + 0.6 * u[3], 0.1 * u[4]])
    p2 = p1 + np.array([0.3 + 0.5 * u[5], -0.3 + 0.6 * u[6], 1.2 + 0.7 * u[7]])
    p2[2] = min(p2[2], 2.9)
    lam = 1.5 + 1.5 * u[8]
    octaves = []
    for o in range(4):
        cz = 2.0 * u[9 + 3 * o] - 1.0                 # uniform direction on the sphere
        az = 2.0 * math.pi * u[10 + 3 * o]
        sz = math.sqrt(max(0.0, 1.0 - cz * cz))
        phase = 2.0 * math.pi * u[11 + 3 * o]
        octaves.append(((sz * math.cos(az), sz * math.sin(az), cz), phase))
    return dict(p0=p0, p1=p1, p2=p2, lam=lam, octaves=octaves)


def plume_field(grid: Grid, seed: int, t_inlet: float = 310.0, radius: float = 0.2,
                noise_amp: float = 0.3, ambient: float = T_AMBIENT, device=None):
    """Buoyant plume from the side-wall inlet plus multi-octave sinusoidal noise.

    T = ambient + (t_inlet - ambient) * exp(-d^2 / (2 radius^2)) * exp(-s / lam) + noise,
    with d the distance to a seeded curved centreline (a quadratic Bezier that
    leaves the inlet along +x and bends upward), s the arc length of the closest
    centreline point and noise = sum_o a_o sin(2 pi 2^o (u_o . x) / 1 m + phi_o),
    sum_o a_o = noise_amp.  Returns (nz, ny, nx) float32: a numpy array, or with `device`
    a torch tensor computed on that device.
    """
    prm = plume_params(seed)
    m = 96
    pts = _bezier(prm["p0"], prm["p1"], prm["p2"], m)            # (m, 3)
    seg = pts[1:] - pts[:-1]
    seg_len = np.sqrt((seg ** 2).sum(1))
    s_at = np.concatenate([[0.0], np.cumsum(seg_len)])          # arc length at points
    import torch  # CPU, float64: only to spread the distance search over the host cores

    xc, yc, zc = _cell_centers(grid)
    nx, ny, nz = grid.n
    amp = t_inlet - ambient
    amps = [noise_amp * 2.0 ** (-o) / 1.875 for o in range(4)]
    dev = torch.device("cpu") if device is None else torch.device(device)
    tp = torch.from_numpy(pts).to(dev)
    tseg = torch.from_numpy(seg).to(dev)
    tlen = torch.from_numpy(seg_len).to(dev)
    ts_at = torch.from_numpy(s_at).to(dev)
    pp = (tp ** 2).sum(1)
    X = torch.from_numpy(xc).to(dev)
    Y = torch.from_numpy(yc).to(dev)
    out = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    slabs = max(1, (1 << 20) // (nx * ny))
    for k0 in range(0, nz, slabs):
        k1 = min(nz, k0 + slabs)
        Z = torch.from_numpy(zc[k0:k1]).to(dev)
        P = torch.stack(torch.meshgrid(X, Y, Z, indexing="xy"), -1)        # (ny, nx, nk, 3)
        P = P.permute(2, 0, 1, 3).reshape(-1, 3)                          # z, y, x order
        d2 = (P ** 2).sum(1, keepdim=True) - 2.0 * (P @ tp.T) + pp[None, :]
        i = torch.argmin(d2, dim=1)
        best = torch.full((P.shape[0],), float("inf"), dtype=torch.float64, device=dev)
        best_s = torch.zeros(P.shape[0], dtype=torch.float64, device=dev)
        for off in (-1, 0):                                      # the two segments at point i
            j = torch.clamp(i + off, 0, m - 2)
            a = tp[j]
            ab = tseg[j]
            t = ((P - a) * ab).sum(1) / (tlen[j] ** 2)
            t = torch.clamp(t, 0.0, 1.0)
            dd = ((P - a - t[:, None] * ab) ** 2).sum(1)
            take = dd < best
            best = torch.where(take, dd, best)
            best_s = torch.where(take, ts_at[j] + t * tlen[j], best_s)
        val = amp * torch.exp(-best / (2.0 * radius * radius)) * torch.exp(-best_s / prm["lam"])
        for o, (uvec, phi) in enumerate(prm["octaves"]):
            proj = P @ torch.tensor(uvec, dtype=torch.float64, device=dev)
            val = val + amps[o] * torch.sin(2.0 * math.pi * (2.0 ** o) * proj + phi)
        out[k0:k1] = (ambient + val).reshape(k1 - k0, ny, nx).to(torch.float32)
    return out if device is not None else out.numpy()


def linear_field_T(grid: Grid, grad_deta, deta0: float) -> np.ndarray:
    """Temperature whose eta - 1 = rho0 G T0 / T equals deta0 + grad_deta . (x - origin)
    at the cell centres, computed in float64 (returned as float64, (nz, ny, nx))."""
    xc, yc, zc = _cell_centers(grid)
    o = grid.origin
    de = (deta0 + grad_deta[0] * (xc[None, None, :] - o[0]) + grad_deta[1] * (yc[None, :, None] - o[1])
          + grad_deta[2] * (zc[:, None, None] - o[2]))
    return grid.rho0 * grid.G * grid.T0 / de


# --------------------------------------------------------------------------
# patterns
# --------------------------------------------------------------------------

def dot_texture(tw: int, th: int, fill: float, dot: int, seed: int) -> np.ndarray:
    """Random-dot wall texture: `fill` of the texels lit, in dot x dot blocks (value 1 on 0)."""
    ndots = int(round(fill * tw * th / (dot * dot)))
    u = np.random.default_rng(seed).random((ndots, 2))
    tex = np.zeros((th, tw), dtype=np.float32)
    for a, b in u:
        i = int(a * (tw - dot + 1))
        j = int(b * (th - dot + 1))
        tex[j:j + dot, i:i + dot] = 1.0
    return tex


def speckle(w: int, h: int, seed: int, p: float = 0.5) -> np.ndarray:
    """Binary speckle: each pixel lit with probability p."""
    return (np.random.default_rng(seed).random((h, w)) < p).astype(np.float32)


def smooth_pattern(w: int, h: int, seed: int) -> np.ndarray:
    """Smooth random pattern in [0, 1] (sum of a few sinusoids); for gradient tests."""
    u = np.random.default_rng(seed).random(12)
    x = (np.arange(w) + 0.5) / w
    y = (np.arange(h) + 0.5) / h
    X, Y = np.meshgrid(x, y, indexing="xy")
    v = np.zeros_like(X)
    for q in range(4):
        fx, fy, ph = 2 + 6 * u[3 * q], 2 + 6 * u[3 * q + 1], 6.28 * u[3 * q + 2]
        v += np.sin(2 * math.pi * (fx * X + 0.7 * fy * Y) + ph)
    return (0.5 + 0.125 * v).astype(np.float32)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def _pinhole(pos, width, height, half_view, distance, spp=1, seed=0) -> Camera:
    f = (0.5 * height) * distance / half_view
    return Camera(pos=tuple(float(c) for c in pos), fwd=(0.0, 1.0, 0.0), up=(0.0, 0.0, 1.0),
                  fx=f, fy=f, cx=0.5 * width, cy=0.5 * height, width=width, height=height,
                  spp=spp, seed=seed)


def back_wall(grid: Grid) -> Wall:
    o = grid.origin
    return Wall(origin=(o[0], o[1] + grid.extent[1], o[2]), eu=(1.0, 0.0, 0.0),
                ev=(0.0, 0.0, 1.0), normal=(0.0, 1.0, 0.0),
                size_u=grid.extent[0], size_v=grid.extent[2])


def room_grid(n) -> Grid:
    return Grid(n=tuple(int(v) for v in n), origin=ROOM_ORIGIN, extent=ROOM_EXTENT)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def blob_cube(seed: int = BASE_SEED + 0, n: int = 32, width: int = 64, height: int = 64,
              steps: int = 128, integrator: int = 0) -> Scene:
    """32^3 grid over a 1 m cube, ambient plus one +8 K Gaussian blob (sigma 0.15 m) at a
    seeded centre, a 64x64 pinhole camera 2 m from the cube centre looking +y at the back
    face, which carries a 1 %-fill random-dot texture of 2-texel dots; 1 ray per pixel,
    a fixed number of steps."""
    grid = Grid(n=(n, n, n), origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 1.0))
    u = np.random.default_rng(seed).random(3)
    center = 0.35 + 0.3 * u
    T = blob_field(grid, center, 0.15, 8.0)
    cam = _pinhole((0.5, -1.5, 0.5), width, height, 0.5, 2.5)
    wall = back_wall(grid)
    tex = dot_texture(64, 64, 0.01, 2, seed + 1000)
    return Scene("blob_cube", grid, T, cam, wall, Light(0, tex),
                 Integrator(fixed_steps=steps, integrator=integrator))


def room(n=(128, 128, 96), width: int = 1024, height: int = 1024, spp: int = 4,
         seed: int = BASE_SEED + 1, pattern_size: int = 512, integrator: int = 0,
         ckpt_every: int = 16, name: str = "room", field: bool = True) -> Scene:
    """Room-scale scene: plume field on an n-cell grid over the 4x4x3 m room, a projector
    casting a binary speckle on the back wall, a pinhole camera with `spp` tent-jittered
    rays per pixel and adaptive steps of at most half the smallest cell.  field=False
    leaves T empty (geometry only)."""
    grid = room_grid(n)
    T = plume_field(grid, seed) if field else None
    dist = ROOM_ORIGIN[1] + ROOM_EXTENT[1] - CAMERA_POS[1]
    cam = _pinhole(CAMERA_POS, width, height, CAMERA_HALF_VIEW, dist, spp=spp, seed=seed * 7919 + 17)
    proj = _pinhole(PROJECTOR_POS, pattern_size, pattern_size, PROJECTOR_HALF_VIEW,
                    ROOM_ORIGIN[1] + ROOM_EXTENT[1] - PROJECTOR_POS[1])
    pat = speckle(pattern_size, pattern_size, seed + 5000)
    return Scene(name, grid, T, cam, back_wall(grid), Light(1, pat, proj),
                 Integrator(fixed_steps=0, max_step_vox=0.5, integrator=integrator,
                            ckpt_every=ckpt_every))


def room_forward(seed: int = BASE_SEED + 1) -> Scene:
    """128x128x96 room, 1024^2 camera, 4 jittered rays per pixel."""
    return room((128, 128, 96), 1024, 1024, 4, seed, name="room_128x128x96_1024sq_4spp")


def room_adjoint(seed: int = BASE_SEED + 2) -> Scene:
    """256x256x192 room, 2048^2 camera, 1 ray per pixel, checkpoint every 16 steps."""
    return room((256, 256, 192), 2048, 2048, 1, seed, name="room_256x256x192_2048sq_1spp")


def paper_sensor(seed: int = BASE_SEED + 9) -> Scene:
    """The paper's own measurement render (Sec. 3.1-3.2): a 64^3 grid over the room and a
    100x100 sensor with 2 samples per pixel."""
    return room((64, 64, 64), 100, 100, 2, seed, name="paper_64cube_100sq_2spp")


def crop(scene: Scene, lo, size: int = 32, width: int = 256, height: int = 256,
         spp: int = 1) -> Scene:
    """A size^3 sub-box of `scene`'s field (cells lo .. lo+size) at the same spacing, as a
    standalone scene with its own camera (looking +y from the scene camera's distance)
    framing the crop's back face, and the same projector."""
    g = scene.grid
    h = g.spacing()
    i0, j0, k0 = lo
    T = np.ascontiguousarray(scene.T[k0:k0 + size, j0:j0 + size, i0:i0 + size])
    origin = tuple(g.origin[a] + lo[a] * h[a] for a in range(3))
    extent = tuple(size * h[a] for a in range(3))
    cg = Grid(n=(size, size, size), origin=origin, extent=extent, T0=g.T0, rho0=g.rho0, G=g.G)
    wall = back_wall(cg)
    cpos = (origin[0] + 0.5 * extent[0], scene.camera.pos[1], origin[2] + 0.5 * extent[2])
    dist = origin[1] + extent[1] - cpos[1]
    half = 0.45 * min(extent[0], extent[2])
    cam = _pinhole(cpos, width, height, half, dist, spp=spp, seed=scene.camera.seed + 1)
    return Scene(scene.name + "_crop", cg, T, cam, wall, scene.light, scene.integ)


def with_target_seed(scene: Scene, seed: int) -> np.ndarray:
    """Temperature field of the same plume family drawn with another seed (the target of the
    image loss is a render of this field)."""
    return plume_field(scene.grid, seed)
