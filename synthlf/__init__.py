"""Seeded synthetic inputs for HMLFC: two-plane light fields and novel views.

This module is shared by the oracle-side tests and by the product benchmark,
and it holds none of the codec's arithmetic.  It produces

* RGB8 light fields ``uint8[nu][nv][H][W][3]`` (``lf[i, j, y, x, c]``: camera
  ``(i, j)`` on the (u,v) plane, pixel ``(x, y)`` on the (s,t) plane), built
  from fronto-parallel textured planes at fixed per-camera-step disparities;
* view descriptions: an output size plus two 3x3 homographies (stored as
  float32) mapping an output pixel centre ``(px + 0.5, py + 0.5, 1)`` to the
  (u,v) and (s,t) coordinates of its ray (two-plane parameterisation, Sec. 2.1);
* configuration records that name the workloads (sizes, levels, blocks).

The Stanford light-field archive used by the paper's experiments (Sec. 5) is
not available; these seeded scenes stand in for it with the same grid and
image shapes.  Every array is produced with elementwise IEEE float64 or
integer arithmetic from numpy's PCG64 stream, so the same seed gives the same
bytes on x86 and Arm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "View", "LFConfig", "CONFIGS", "make_scene", "render_lf", "make_lf",
    "lf_geometry", "pinhole_view", "grid_view", "circle_path", "random_views",
    "batched_workload", "views_to_array", "VIEW_DTYPE",
]


# --------------------------------------------------------------------------
# textures
# --------------------------------------------------------------------------

def _value_noise(rng: np.random.Generator, h: int, w: int, cell: int) -> np.ndarray:
    """Random lattice values upsampled bilinearly to ``h x w`` (float64, 3 ch)."""
    gh, gw = h // cell + 2, w // cell + 2
    g = rng.random((gh, gw, 3))
    y = np.arange(h)
    x = np.arange(w)
    y0, fy = y // cell, (y % cell) / cell
    x0, fx = x // cell, (x % cell) / cell
    a = g[y0][:, x0]
    b = g[y0][:, x0 + 1]
    c = g[y0 + 1][:, x0]
    d = g[y0 + 1][:, x0 + 1]
    fx = fx[None, :, None]
    fy = fy[:, None, None]
    top = a * (1.0 - fx) + b * fx
    bot = c * (1.0 - fx) + d * fx
    return top * (1.0 - fy) + bot * fy


def _normalise(t: np.ndarray) -> np.ndarray:
    lo = t.min()
    hi = t.max()
    if hi <= lo:
        return np.full_like(t, 127.0)
    return (t - lo) * (255.0 / (hi - lo))


def _texture(rng: np.random.Generator, kind: str, h: int, w: int) -> np.ndarray:
    """A float64 RGB texture in [0, 255].

    ``noise_gradient``: half uniform per-pixel noise, half a linear colour ramp.
    ``pink``: octaves of value noise with amplitude proportional to the cell
    size, i.e. an approximately 1/f amplitude spectrum.
    """
    if kind == "noise_gradient":
        noise = rng.random((h, w, 3)) * 255.0
        ang = rng.random() * 2.0 * math.pi
        c0 = rng.random(3) * 255.0
        c1 = rng.random(3) * 255.0
        yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
        r = (xx * math.cos(ang) + yy * math.sin(ang))
        r = _normalise(r[..., None]) / 255.0
        ramp = c0[None, None, :] * (1.0 - r) + c1[None, None, :] * r
        return 0.5 * noise + 0.5 * ramp
    if kind == "pink":
        acc = np.zeros((h, w, 3))
        cell = 1
        while cell <= max(h, w) // 2:
            acc = acc + float(cell) * _value_noise(rng, h, w, cell)
            cell *= 2
        return _normalise(acc)
    raise ValueError(f"unknown texture kind {kind!r}")


# --------------------------------------------------------------------------
# scene and light field
# --------------------------------------------------------------------------

@dataclass
class Plane:
    disparity: float          # pixels of shift per camera step (multiple of 1/16)
    rect: tuple               # (x0, y0, x1, y1) coverage in centre-view pixels
    tex: np.ndarray           # float64 [Ht][Wt][3], origin at (-margin, -margin)


@dataclass
class Scene:
    nu: int
    nv: int
    width: int
    height: int
    margin: int
    planes: list = field(default_factory=list)   # far to near (painter order)


def make_scene(seed: int, nu: int, nv: int, width: int, height: int,
               n_planes: int, disp_max: float, kind: str) -> Scene:
    """Fronto-parallel textured planes; plane 0 is a full-frame background.

    Disparities are drawn from U[0, disp_max] and rounded to 1/16 px; the
    planes are ordered by disparity so that a larger disparity is nearer.
    """
    rng = np.random.default_rng(seed)
    cu, cv = (nu - 1) / 2.0, (nv - 1) / 2.0
    margin = int(math.ceil(disp_max * max(cu, cv))) + 4
    th, tw = height + 2 * margin, width + 2 * margin
    disps = sorted(round(float(rng.random()) * disp_max * 16.0) / 16.0 for _ in range(n_planes))
    planes = []
    for k, d in enumerate(disps):
        if k == 0:
            rect = (-1e9, -1e9, 1e9, 1e9)
        else:
            rw = (0.2 + 0.4 * rng.random()) * width
            rh = (0.2 + 0.4 * rng.random()) * height
            x0 = rng.random() * (width - rw)
            y0 = rng.random() * (height - rh)
            rect = (x0, y0, x0 + rw, y0 + rh)
        planes.append(Plane(d, rect, _texture(rng, kind, th, tw)))
    return Scene(nu, nv, width, height, margin, planes)


def _render_view(scene: Scene, i: int, j: int) -> np.ndarray:
    h, w, m = scene.height, scene.width, scene.margin
    cu, cv = (scene.nu - 1) / 2.0, (scene.nv - 1) / 2.0
    out = None
    xs = np.arange(w, dtype=np.float64)
    ys = np.arange(h, dtype=np.float64)
    for p in scene.planes:
        sx = p.disparity * (i - cu)
        sy = p.disparity * (j - cv)
        ix = math.floor(sx)
        iy = math.floor(sy)
        fx = sx - ix
        fy = sy - iy
        t = p.tex
        a = t[m + iy:m + iy + h, m + ix:m + ix + w]
        b = t[m + iy:m + iy + h, m + ix + 1:m + ix + 1 + w]
        c = t[m + iy + 1:m + iy + 1 + h, m + ix:m + ix + w]
        d = t[m + iy + 1:m + iy + 1 + h, m + ix + 1:m + ix + 1 + w]
        val = (a * (1.0 - fx) + b * fx) * (1.0 - fy) + (c * (1.0 - fx) + d * fx) * fy
        if out is None:
            out = val
            continue
        x0, y0, x1, y1 = p.rect
        tx = xs + sx
        ty = ys + sy
        cov = ((ty >= y0) & (ty < y1))[:, None] & ((tx >= x0) & (tx < x1))[None, :]
        out = np.where(cov[..., None], val, out)
    return np.clip(np.floor(out + 0.5), 0, 255).astype(np.uint8)


def render_lf(scene: Scene, threads: int = 0) -> np.ndarray:
    """All camera views of the scene as ``uint8[nu][nv][H][W][3]``; views are
    rendered on host threads (numpy releases the GIL), the bytes do not depend
    on the thread count."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    lf = np.empty((scene.nu, scene.nv, scene.height, scene.width, 3), np.uint8)

    def one(ij):
        lf[ij[0], ij[1]] = _render_view(scene, ij[0], ij[1])

    cams = [(i, j) for i in range(scene.nu) for j in range(scene.nv)]
    n = threads or min(16, os.cpu_count() or 1)
    if n <= 1 or len(cams) < 4:
        for ij in cams:
            one(ij)
    else:
        with ThreadPoolExecutor(n) as ex:
            list(ex.map(one, cams))
    return lf


def make_lf(seed: int, nu: int, nv: int, width: int, height: int,
            n_planes: int, disp_max: float, kind: str) -> np.ndarray:
    return render_lf(make_scene(seed, nu, nv, width, height, n_planes, disp_max, kind))


# --------------------------------------------------------------------------
# views: output size + two homographies
# --------------------------------------------------------------------------

@dataclass
class View:
    lf: int
    width: int
    height: int
    H_uv: np.ndarray          # float32[9], row-major
    H_st: np.ndarray          # float32[9], row-major


VIEW_DTYPE = np.dtype([("lf", "<i4"), ("width", "<i4"), ("height", "<i4"),
                       ("H_uv", "<f4", (9,)), ("H_st", "<f4", (9,)),
                       ("_pad", "<i4"), ("out_offset", "<i8")], align=False)
assert VIEW_DTYPE.itemsize == 96


def views_to_array(views, out_offsets=None) -> np.ndarray:
    """Pack views into the 96-byte C record used by both implementations."""
    arr = np.zeros(len(views), VIEW_DTYPE)
    off = 0
    for k, v in enumerate(views):
        arr[k]["lf"] = v.lf
        arr[k]["width"] = v.width
        arr[k]["height"] = v.height
        arr[k]["H_uv"] = v.H_uv
        arr[k]["H_st"] = v.H_st
        if out_offsets is None:
            arr[k]["out_offset"] = off
            off += v.width * v.height * 3
        else:
            arr[k]["out_offset"] = out_offsets[k]
    return arr


def lf_geometry(nu: int, nv: int, width: int, height: int) -> dict:
    """Physical layout of the two planes.

    Cameras sit at integer (u, v) = (i, j) on the plane z = 0 (unit spacing).
    The (s,t) plane is at z = zf; pixel (x, y) of every camera image is the
    point (cu + (x - (W-1)/2) * sigma, cv + (y - (H-1)/2) * sigma, zf).
    """
    n = max(nu, nv)
    ext = float(max(n - 1, 1))
    zf = 2.0 * ext
    sigma = 2.0 * ext / max(width, height)
    return dict(cu=(nu - 1) / 2.0, cv=(nv - 1) / 2.0, zf=zf, sigma=sigma,
                nu=nu, nv=nv, width=width, height=height)


def _norm(v):
    return v / np.linalg.norm(v)


def pinhole_view(geo: dict, eye, target, out_w: int, out_h: int,
                 half_fov: float, lf: int = 0) -> View:
    """A pinhole camera at ``eye`` looking at ``target`` (world coordinates).

    The homographies are products of K^-1, the camera rotation, the central
    projection onto the plane z = z0 and the plane's affine (u,v) or (s,t)
    coordinate map.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = _norm(target - eye)
    xc = _norm(np.cross(np.array([0.0, 1.0, 0.0]), f))
    yc = np.cross(f, xc)
    R = np.stack([xc, yc, f], axis=1)
    fpx = (max(out_w, out_h) / 2.0) / math.tan(half_fov)
    Kinv = np.array([[1.0 / fpx, 0.0, -(out_w / 2.0) / fpx],
                     [0.0, 1.0 / fpx, -(out_h / 2.0) / fpx],
                     [0.0, 0.0, 1.0]])
    ex, ey, ez = eye

    def onto(z0):
        return np.array([[z0 - ez, 0.0, ex], [0.0, z0 - ez, ey], [0.0, 0.0, 1.0]])

    s = 1.0 / geo["sigma"]
    A_st = np.array([[s, 0.0, -geo["cu"] * s + (geo["width"] - 1) / 2.0],
                     [0.0, s, -geo["cv"] * s + (geo["height"] - 1) / 2.0],
                     [0.0, 0.0, 1.0]])
    H_uv = onto(0.0) @ R @ Kinv
    H_st = A_st @ onto(geo["zf"]) @ R @ Kinv

    def pack(H):
        if abs(H[2, 2]) > 1e-12:
            H = H / H[2, 2]
        return H.reshape(9).astype(np.float32)

    return View(lf, out_w, out_h, pack(H_uv), pack(H_st))


def grid_view(u0: float, v0: float, s_off: float, t_off: float,
              out_w: int, out_h: int, lf: int = 0) -> View:
    """A camera placed on the (u,v) plane: constant (u, v) for every pixel and
    (s, t) = (px + s_off, py + t_off) at pixel centres."""
    H_uv = np.array([0, 0, u0, 0, 0, v0, 0, 0, 1], np.float32)
    H_st = np.array([1, 0, s_off - 0.5, 0, 1, t_off - 0.5, 0, 0, 1], np.float32)
    return View(lf, out_w, out_h, H_uv, H_st)


def circle_path(geo: dict, n_poses: int, out_w: int, out_h: int,
                radius_frac: float = 0.3, dist_frac: float = 0.25, lf: int = 0) -> list:
    """A camera circling in front of the (u,v) plane, looking at the (s,t)
    centre; radius = radius_frac * grid extent, distance = dist_frac * zf."""
    n = max(geo["nu"], geo["nv"])
    r = radius_frac * (n - 1)
    ez = -dist_frac * geo["zf"]
    target = (geo["cu"], geo["cv"], geo["zf"])
    half_extent = 0.5 * geo["sigma"] * max(geo["width"], geo["height"])
    half_fov = math.atan(half_extent / (geo["zf"] - ez))
    views = []
    for k in range(n_poses):
        th = 2.0 * math.pi * k / n_poses
        eye = (geo["cu"] + r * math.cos(th), geo["cv"] + r * math.sin(th), ez)
        views.append(pinhole_view(geo, eye, target, out_w, out_h, half_fov, lf))
    return views


def random_views(seed: int, geo: dict, n_views: int, sizes, lf: int = 0,
                 radius_frac: float = 0.35) -> list:
    """Random pinhole views in front of the (u,v) plane (uniform positions in
    a disc, random distance and aim jitter); ``sizes`` is a list of (w, h)."""
    rng = np.random.default_rng(seed)
    n = max(geo["nu"], geo["nv"])
    half_extent = 0.5 * geo["sigma"] * max(geo["width"], geo["height"])
    views = []
    for _ in range(n_views):
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        rr = radius_frac * (n - 1) * math.sqrt(rng.random())
        th = 2.0 * math.pi * rng.random()
        ez = -(0.15 + 0.2 * rng.random()) * geo["zf"]
        eye = (geo["cu"] + rr * math.cos(th), geo["cv"] + rr * math.sin(th), ez)
        jit = (rng.random(2) - 0.5) * 0.1 * (n - 1)
        target = (geo["cu"] + jit[0], geo["cv"] + jit[1], geo["zf"])
        half_fov = math.atan(half_extent / (geo["zf"] - ez)) * (0.8 + 0.4 * rng.random())
        views.append(pinhole_view(geo, eye, target, w, h, half_fov, lf))
    return views


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class LFConfig:
    name: str
    nu: int
    nv: int
    width: int
    height: int
    n_planes: int
    disp_max: float
    texture: str
    levels: int
    block: int
    search: int
    qstep: int
    seed: int


CONFIGS = {
    # 4x4 grid of 64x64 views, 3 planes, 0-6 px disparity, 2 levels, 8x8
    # blocks, quarter-pel MC with a +-4 px integer search, quantiser step 4.
    "tiny": LFConfig("tiny", 4, 4, 64, 64, 3, 6.0, "noise_gradient", 2, 8, 4, 4, 1),
    # 17x17 grid of 512x512 views, 6 planes, 0-12 px disparity, 1/f
    # textures, 4 levels, 16x16 blocks, quantiser step 4 (sweep {2, 4, 8}).
    "paper": LFConfig("paper", 17, 17, 512, 512, 6, 12.0, "pink", 4, 16, 4, 4, 2),
    # 9x9 grid of 256x256 views, 3 levels (differentiable form).
    "diff": LFConfig("diff", 9, 9, 256, 256, 5, 8.0, "pink", 3, 16, 4, 4, 3),
    # 32x32 grid of 1024x1024 views, 10 planes, 5 levels (serving form).
    "serve": LFConfig("serve", 32, 32, 1024, 1024, 10, 6.0, "pink", 5, 16, 4, 4, 5),
}

# The eight light fields of the batched form: (n, size, levels).
BATCHED_LFS = [(5, 256), (9, 384), (13, 512), (17, 512), (7, 768), (11, 640), (15, 320), (17, 1024)]


def batched_views(seed: int, cfgs, n_views: int = 256, sizes=(256, 384, 512, 640, 768, 1024)) -> list:
    """n_views random pinhole views spread over the light fields of `cfgs`,
    square outputs of mixed resolution drawn from `sizes`."""
    rng = np.random.default_rng(seed)
    views = []
    for k in range(n_views):
        lf = int(rng.integers(0, len(cfgs)))
        c = cfgs[lf]
        geo = lf_geometry(c.nu, c.nv, c.width, c.height)
        s = int(sizes[int(rng.integers(0, len(sizes)))])
        views += random_views(int(rng.integers(0, 2 ** 31)), geo, 1, [(s, s)], lf=lf)
    return views


@dataclass
class StereoRequest:
    rid: int
    arrival: float            # seconds after the start of the stream
    left: View
    right: View


def stereo_requests(seed: int, geo: dict, n: int, rate: float,
                    sizes=((512, 512), (1024, 1024), (1440, 1600)), ipd_frac: float = 0.02) -> list:
    """A Poisson stream (rate per second) of stereo view pairs along a seeded
    head-pose random walk in front of the (u,v) plane: the head moves by a
    small random step per request and looks at a jittered point of the (s,t)
    plane; the two eyes sit ipd_frac * grid extent apart along u."""
    rng = np.random.default_rng(seed)
    n_ext = max(geo["nu"], geo["nv"]) - 1
    half_extent = 0.5 * geo["sigma"] * max(geo["width"], geo["height"])
    head = np.array([geo["cu"], geo["cv"], -0.25 * geo["zf"]])
    t = 0.0
    out = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate))
        head = head + np.array([rng.normal(0, 0.02 * n_ext), rng.normal(0, 0.02 * n_ext), rng.normal(0, 0.01 * geo["zf"])])
        head[0] = min(max(head[0], geo["cu"] - 0.35 * n_ext), geo["cu"] + 0.35 * n_ext)
        head[1] = min(max(head[1], geo["cv"] - 0.35 * n_ext), geo["cv"] + 0.35 * n_ext)
        head[2] = min(max(head[2], -0.4 * geo["zf"]), -0.1 * geo["zf"])
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        target = (geo["cu"] + rng.normal(0, 0.03 * n_ext), geo["cv"] + rng.normal(0, 0.03 * n_ext), geo["zf"])
        half_fov = math.atan(half_extent / (geo["zf"] - head[2]))
        d = 0.5 * ipd_frac * n_ext
        left = pinhole_view(geo, head - np.array([d, 0, 0]), target, w, h, half_fov)
        right = pinhole_view(geo, head + np.array([d, 0, 0]), target, w, h, half_fov)
        out.append(StereoRequest(k, t, left, right))
    return out


def batched_workload(seed: int = 4):
    """LFConfig list for the eight uneven light fields of the batched form;
    levels = clamp(ceil(log2 n), 3, 5)."""
    out = []
    for k, (n, s) in enumerate(BATCHED_LFS):
        lv = min(max(int(math.ceil(math.log2(n))), 3), 5)
        out.append(LFConfig(f"batch{k}", n, n, s, s, 4, 8.0, "pink", lv, 16, 4, 4, seed * 100 + k))
    return out
