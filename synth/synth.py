"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds no renderer or oracle arithmetic.  It produces:

* SPIM-like multi-channel uint16 volumes (stand-ins for the paper's data sets
  D1-D3 of Table 1, which are not available): a host generator (C, threads)
  and a bit-identical device generator (CUDA) over the same counter-based
  definition in ``synth_common.h``;
* per-channel 256-entry RGBA transfer-function tables built from four random
  knots;
* camera sets (static, orbit, random mixed-resolution batches).

Workload recipes (the five workloads the build is measured on) live in
``WORKLOADS``; each names its volume, brick size, homogeneity threshold,
cameras and transfer-function seeds.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
HOST_LIB = os.path.join(_HERE, "libsynth_host.so")
DEV_LIB = os.path.join(_HERE, "libsynth_dev.so")

KIND_BLOBS = 0
KIND_SPIM = 1

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


class SplitMix64:
    """SplitMix64 stream (Steele, Lea and Flood, 2014); uniform doubles with 53 bits."""

    def __init__(self, seed: int, tag: int = 0):
        self.state = _mix64(seed ^ ((tag * 0xD1B54A32D192ED03) & _M64))

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _M64
        return _mix64(self.state)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        return a + (b - a) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))


_host = None
_dev = None


def host_lib():
    global _host
    if _host is None:
        if not os.path.exists(HOST_LIB):
            raise RuntimeError(f"{HOST_LIB} is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(HOST_LIB)
        lib.sy_spec_create.restype = ctypes.c_void_p
        lib.sy_spec_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_int64, ctypes.c_uint64]
        lib.sy_spec_destroy.argtypes = [ctypes.c_void_p]
        lib.sy_spec_view.restype = ctypes.c_void_p
        lib.sy_spec_view.argtypes = [ctypes.c_void_p]
        lib.sy_spec_arrays.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 6
        lib.sy_host_voxels.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        lib.sy_host_generate_box.restype = ctypes.c_int
        lib.sy_host_generate_box.argtypes = [ctypes.c_void_p] + [ctypes.c_int64] * 6 + [ctypes.c_void_p, ctypes.c_int]
        _host = lib
    return _host


def dev_lib():
    global _dev
    if _dev is None:
        if not os.path.exists(DEV_LIB):
            raise RuntimeError(f"{DEV_LIB} is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(DEV_LIB)
        lib.sy_dev_create.restype = ctypes.c_void_p
        lib.sy_dev_create.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        lib.sy_dev_destroy.argtypes = [ctypes.c_void_p]
        lib.sy_dev_generate_box.restype = ctypes.c_int
        lib.sy_dev_generate_box.argtypes = [ctypes.c_void_p] + [ctypes.c_int64] * 6 + [ctypes.c_void_p, ctypes.c_void_p]
        _dev = lib
    return _dev


class VolumeSpec:
    """A seeded synthetic volume: dims (X, Y, Z), C channels, uint16 values."""

    def __init__(self, kind: int, dims, channels: int, count: int, seed: int = 1):
        self.kind, self.dims, self.C, self.count, self.seed = kind, tuple(int(d) for d in dims), channels, count, seed
        X, Y, Z = self.dims
        self._h = host_lib().sy_spec_create(kind, X, Y, Z, channels, count, seed)
        if not self._h:
            raise ValueError("invalid synthetic volume specification")
        self._dev = None

    def close(self):
        if self._dev:
            dev_lib().sy_dev_destroy(self._dev)
            self._dev = None
        if self._h:
            host_lib().sy_spec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h

    @property
    def voxel_fn(self) -> int:
        """Address of ``sy_host_voxel(handle, x, y, z, out[C])`` (for C callers)."""
        return ctypes.cast(host_lib().sy_host_voxel, ctypes.c_void_p).value

    def box(self, x0, x1, y0, y1, z0, z1, threads: int = 0) -> np.ndarray:
        out = np.empty((z1 - z0, y1 - y0, x1 - x0, self.C), dtype=np.uint16)
        rc = host_lib().sy_host_generate_box(self._h, x0, x1, y0, y1, z0, z1, out.ctypes.data, threads)
        if rc != 0:
            raise ValueError("box outside the volume")
        return out

    def slices(self, z0: int, z1: int, threads: int = 0) -> np.ndarray:
        X, Y, _ = self.dims
        return self.box(0, X, 0, Y, z0, z1, threads)

    def volume(self, threads: int = 0) -> np.ndarray:
        X, Y, Z = self.dims
        return self.box(0, X, 0, Y, 0, Z, threads)

    def voxels(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, 3))
        out = np.empty((c.shape[0], self.C), dtype=np.uint16)
        host_lib().sy_host_voxels(self._h, c.shape[0], c.ctypes.data, out.ctypes.data)
        return out

    def _device(self):
        if self._dev is None:
            lib = host_lib()
            nuc, nn, cs, nc, ci, ni = (ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_int64(),
                                       ctypes.c_void_p(), ctypes.c_int64())
            lib.sy_spec_arrays(self._h, ctypes.byref(nuc), ctypes.byref(nn), ctypes.byref(cs), ctypes.byref(nc),
                               ctypes.byref(ci), ctypes.byref(ni))
            self._dev = dev_lib().sy_dev_create(lib.sy_spec_view(self._h), nn.value, nc.value, ni.value)
            if not self._dev:
                raise RuntimeError("device generator: allocation failed")
        return self._dev

    def generate_device(self, out_ptr: int, z0: int, z1: int, stream_ptr: int = 0, box=None):
        """Writes slices [z0, z1) as [z][y][x][C] uint16 to device memory ``out_ptr`` (stream-ordered)."""
        X, Y, _ = self.dims
        x0, x1, y0, y1 = box if box is not None else (0, X, 0, Y)
        rc = dev_lib().sy_dev_generate_box(self._device(), x0, x1, y0, y1, z0, z1, ctypes.c_void_p(out_ptr),
                                           ctypes.c_void_p(stream_ptr))
        if rc != 0:
            raise RuntimeError(f"device generator failed ({rc})")


# ---------------------------------------------------------------------------------------------
# Transfer functions
# ---------------------------------------------------------------------------------------------

def make_tf_channel(seed: int) -> np.ndarray:
    """256x4 float32 RGBA table from 4 random knots (x ~ U(0,1) sorted, rgb ~ U[0,1], alpha ~ U[0,0.1]),
    plus end knots (0, rgb of the first knot, alpha 0) and (1, the last knot's values); piecewise
    linear between knots, evaluated at i/255.  Alpha is opacity per unit length (one voxel)."""
    rng = SplitMix64(seed, tag=0x7F)
    knots = []
    for _ in range(4):
        x = rng.uniform()
        r, g, b = rng.uniform(), rng.uniform(), rng.uniform()
        a = rng.uniform(0.0, 0.1)
        knots.append((x, r, g, b, a))
    knots.sort(key=lambda k: k[0])
    first, last = knots[0], knots[-1]
    pts = [(0.0, first[1], first[2], first[3], 0.0)] + knots + [(1.0, last[1], last[2], last[3], last[4])]
    xs = np.array([p[0] for p in pts])
    vals = np.array([p[1:] for p in pts])
    grid = np.arange(256) / 255.0
    out = np.empty((256, 4))
    for k in range(4):
        out[:, k] = np.interp(grid, xs, vals[:, k])
    return out.astype(np.float32)


def make_tf(seeds) -> np.ndarray:
    """[C][256][4] float32 tables, one seed per channel."""
    return np.stack([make_tf_channel(s) for s in seeds]).astype(np.float32)


# ---------------------------------------------------------------------------------------------
# Cameras (plain dicts; the binding converts them to the C struct)
# ---------------------------------------------------------------------------------------------

def camera(eye, target, up, width, height, fov_y_deg=45.0, lod_error_px=1.0, step_voxels=0.5, ert_alpha=0.99,
           clip=()):
    return {"eye": tuple(float(v) for v in eye), "target": tuple(float(v) for v in target),
            "up": tuple(float(v) for v in up), "fov_y_deg": float(fov_y_deg), "width": int(width),
            "height": int(height), "lod_error_px": float(lod_error_px), "step_voxels": float(step_voxels),
            "ert_alpha": float(ert_alpha), "clip": [tuple(float(v) for v in p) for p in clip]}


def orbit_camera(dims, distance, azimuth_deg, elevation_deg, width, height, **kw):
    """Eye on a sphere around the volume centre, rotating about +z; up = +z."""
    c = [d / 2.0 for d in dims]
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    eye = (c[0] + distance * math.cos(el) * math.cos(az), c[1] + distance * math.cos(el) * math.sin(az),
           c[2] + distance * math.sin(el))
    return camera(eye, c, (0.0, 0.0, 1.0), width, height, **kw)


def centre_plane(dims, normal, offset=0.0):
    """Half-space n.p + d >= 0 whose boundary passes through centre + offset*n (n normalised)."""
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    c = np.asarray(dims, dtype=np.float64) / 2.0
    d = -float(n @ c) - offset
    return (float(n[0]), float(n[1]), float(n[2]), d)


def batch_cameras(dims, seed=4):
    """64 cameras: 16 each at 256x256, 640x480, 1280x720, 1920x1080; azimuth ~ U(0,360),
    elevation ~ U(-60,60), distance ~ U(1.5,3) x extent; one clip plane each through the centre
    with a random unit normal and an offset ~ U(-8,8)."""
    rng = SplitMix64(seed, tag=0xCA)
    ext = max(dims)
    cams = []
    for (w, h) in [(256, 256), (640, 480), (1280, 720), (1920, 1080)]:
        for _ in range(16):
            az, el, dist = rng.uniform(0, 360), rng.uniform(-60, 60), rng.uniform(1.5, 3.0) * ext
            zc = rng.uniform(-1.0, 1.0)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            rr = math.sqrt(max(0.0, 1.0 - zc * zc))
            n = (rr * math.cos(ph), rr * math.sin(ph), zc)
            off = rng.uniform(-8.0, 8.0)
            cams.append(orbit_camera(dims, dist, az, el, w, h, clip=[centre_plane(dims, n, off)]))
    return cams


# ---------------------------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    kind: int
    dims: tuple
    channels: int
    count: int
    brick: int
    tau: int
    background: int = 0
    seed: int = 1
    tf_seeds: tuple = (11, 12, 13)
    scales: tuple = (1.0, 1.0, 1.0)
    cameras: list = field(default_factory=list)

    def spec(self) -> VolumeSpec:
        return VolumeSpec(self.kind, self.dims, self.channels, self.count, self.seed)

    def tf(self) -> np.ndarray:
        return make_tf(self.tf_seeds[: self.channels])


def tiny(tau=0):
    """64^3 x 3 blobs, bricks 16^3, 128x128 camera from -z at twice the extent."""
    dims = (64, 64, 64)
    cam = camera((32.0, 32.0, 32.0 - 128.0), (32.0, 32.0, 32.0), (0.0, 1.0, 0.0), 128, 128)
    return Workload("tiny-64^3x3", KIND_BLOBS, dims, 3, 20, 16, tau, cameras=[cam])


def streamed(tau=3277, frame=0, dims=(1024, 1024, 512), nuclei=20000):
    """1024x1024x512 x 3 SPIM-like, bricks 32^3, 1920x1080, oblique clip plane through the centre,
    orbit at 2x the largest extent, elevation 20 deg, azimuth 5.625 deg per frame."""
    d = max(dims)
    clip = [centre_plane(dims, (1.0, 0.5, 0.25))]
    cam = orbit_camera(dims, 2.0 * d, 5.625 * frame, 20.0, 1920, 1080, clip=clip)
    return Workload(f"streamed-{dims[0]}x{dims[1]}x{dims[2]}x3", KIND_SPIM, dims, 3, nuclei, 32, tau, cameras=[cam])


def large(tau=3277, frames=(0,), dims=(2048, 2048, 1024), nuclei=160000):
    """2048x2048x1024 x 3 SPIM-like (24 GiB), bricks 32^3, 60-frame orbit at 2x the extent, 6 deg steps."""
    d = max(dims)
    cams = [orbit_camera(dims, 2.0 * d, 6.0 * f, 20.0, 1920, 1080) for f in frames]
    return Workload(f"large-{dims[0]}x{dims[1]}x{dims[2]}x3", KIND_SPIM, dims, 3, nuclei, 32, tau, cameras=cams)


def batched(tau=0):
    """The tiny volume seen by 64 mixed-resolution cameras, one clip plane each."""
    w = tiny(tau)
    w.name = "batched-64cams-tiny"
    w.cameras = batch_cameras(w.dims)
    return w


def differentiable(tau=3277, dims=(512, 512, 512), nuclei=10000, width=512, height=512):
    """512^3 x 3 SPIM-like, 512x512 render at 2x the extent; target TF seeds 2xx, scales (0.8,1,1.25)."""
    d = max(dims)
    cam = orbit_camera(dims, 2.0 * d, 30.0, 20.0, width, height)
    return Workload(f"differentiable-{dims[0]}^3x3", KIND_SPIM, dims, 3, nuclei, 32, tau, cameras=[cam])


TARGET_TF_SEEDS = (201, 202, 203)
TARGET_SCALES = (0.8, 1.0, 1.25)
