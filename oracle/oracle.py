"""ctypes binding of the FP64 CPU oracle (liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``; never by the product package.  It shares no code with the CUDA
path.  See ``oracle.h`` for what each call computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(_HERE, "liboracle.so")

MAXL, MAXC, MAXCAND = 16, 4, 4
MAXFLAG = 3
GEOMETRY = {"fp32": 0, "fp64": 1}


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fov_y_deg", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("lod_error_px", ctypes.c_float), ("step_voxels", ctypes.c_float), ("ert_alpha", ctypes.c_float),
                ("n_clip", ctypes.c_int), ("clip", (ctypes.c_float * 4) * 3)]


class Pixel(ctypes.Structure):
    _fields_ = [("n_cand", ctypes.c_int), ("rgba", (ctypes.c_double * 4) * MAXCAND), ("samples", ctypes.c_int64)]


class Node(ctypes.Structure):
    _fields_ = [("touched", ctypes.c_int), ("has_children", ctypes.c_int), ("has_brick", ctypes.c_int),
                ("brick_homog", ctypes.c_int), ("subtree_homog", ctypes.c_int), ("avg", ctypes.c_uint16 * MAXC),
                ("bmin", ctypes.c_uint16 * MAXC), ("bmax", ctypes.c_uint16 * MAXC),
                ("smin", ctypes.c_uint16 * MAXC), ("smax", ctypes.c_uint16 * MAXC), ("count", ctypes.c_int64)]


class Geom(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int64 * 3), ("C", ctypes.c_int), ("M", ctypes.c_int), ("N", ctypes.c_int),
                ("ldim", (ctypes.c_int64 * 3) * MAXL), ("nb", (ctypes.c_int64 * 3) * MAXL),
                ("bg", ctypes.c_uint16), ("tau", ctypes.c_uint16)]


_lib = None

GEN_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                          ctypes.POINTER(ctypes.c_uint16))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.or_geom_init.argtypes = [ctypes.POINTER(Geom), i64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16,
                                   ctypes.c_uint16]
        L.or_dense_create.restype = ctypes.c_void_p
        L.or_dense_create.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, ctypes.c_uint16]
        L.or_dense_insert.argtypes = [ctypes.c_void_p, i64p, i64p, ctypes.c_void_p]
        L.or_dense_build.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_dense_level.restype = ctypes.c_void_p
        L.or_dense_level.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_lazy_create.restype = ctypes.c_void_p
        L.or_lazy_create.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, ctypes.c_uint16,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
        L.or_stream_create.restype = ctypes.c_void_p
        L.or_stream_create.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, ctypes.c_uint16,
                                       ctypes.c_void_p, ctypes.c_void_p]
        L.or_stream_feed.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        L.or_stream_finish.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_volume_destroy.argtypes = [ctypes.c_void_p]
        L.or_volume_geom.restype = ctypes.POINTER(Geom)
        L.or_volume_geom.argtypes = [ctypes.c_void_p]
        L.or_value.restype = ctypes.c_uint16
        L.or_value.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int]
        L.or_node_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.POINTER(Node)]
        L.or_render.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int]
        L.or_render_grad.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.or_render_xf.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]
        L.or_render_grad_xf.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.or_render_geo.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.or_render_check.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                      ctypes.c_int]
        L.or_render_grad_edges.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        L.or_render_cache.argtypes = [ctypes.c_void_p, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int]
        L.or_node_count.restype = ctypes.c_int64
        L.or_node_count.argtypes = [ctypes.POINTER(Geom)]
        L.or_node_index.restype = ctypes.c_int64
        L.or_node_index.argtypes = [ctypes.POINTER(Geom), ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int64]
        L.or_ray.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Camera), ctypes.c_int, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                             ctypes.POINTER(ctypes.c_float)]
        L.or_lod_thresholds.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Camera), ctypes.POINTER(ctypes.c_float)]
        _lib = L
    return _lib


def _i64(v):
    return (ctypes.c_int64 * 3)(*[int(x) for x in v])


def camera_struct(cam: dict) -> Camera:
    c = Camera()
    for k in ("eye", "target", "up"):
        getattr(c, k)[:] = [float(x) for x in cam[k]]
    c.fov_y_deg, c.width, c.height = cam["fov_y_deg"], cam["width"], cam["height"]
    c.lod_error_px, c.step_voxels, c.ert_alpha = cam["lod_error_px"], cam["step_voxels"], cam["ert_alpha"]
    clip = cam.get("clip", [])
    c.n_clip = len(clip)
    for i, p in enumerate(clip):
        c.clip[i][:] = [float(x) for x in p]
    return c


class Volume:
    """Oracle volume state (dense flat arrays, or lazy from a generator callback)."""

    def __init__(self, handle, keep=()):
        self._h = handle
        self._keep = keep

    def close(self):
        if self._h:
            lib().or_volume_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def geom(self) -> Geom:
        return lib().or_volume_geom(self._h).contents

    @property
    def N(self) -> int:
        return self.geom.N

    def level_dims(self, L):
        g = self.geom
        return tuple(g.ldim[L][a] for a in range(3))

    def value(self, L, x, y, z, c) -> int:
        return lib().or_value(self._h, L, x, y, z, c)

    def node(self, L, i, j, k) -> Node:
        n = Node()
        if lib().or_node_info(self._h, L, i, j, k, ctypes.byref(n)) != 0:
            raise IndexError("node outside the real node grid")
        return n


class DenseVolume(Volume):
    def __init__(self, dims, channels, brick, background=0, tau=0):
        h = lib().or_dense_create(_i64(dims), channels, brick, background, tau)
        if not h:
            raise ValueError("invalid volume geometry")
        super().__init__(h)
        self.C = channels

    def insert(self, origin, block: np.ndarray):
        b = np.ascontiguousarray(block, dtype=np.uint16)
        ext = (b.shape[2], b.shape[1], b.shape[0])
        if lib().or_dense_insert(self._h, _i64(origin), _i64(ext), b.ctypes.data) != 0:
            raise ValueError("block outside the volume")

    def build(self, threads=0):
        lib().or_dense_build(self._h, threads)

    def level(self, L) -> np.ndarray:
        g = self.geom
        X, Y, Z = (g.ldim[L][a] for a in range(3))
        ptr = lib().or_dense_level(self._h, L)
        arr = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint16)), shape=(Z * Y * X * g.C,))
        return arr.reshape(Z, Y, X, g.C).copy()


class StreamVolume(Volume):
    """A fully inserted volume whose level 0 is fed once, in z order, as slabs [nz][Y][X][C] and read
    back through ``gen_fn`` (for volumes too large to hold level 0 in host memory); levels >= 1 and
    the node records are complete after ``finish()``."""

    def __init__(self, dims, channels, brick, gen_fn_addr: int, user: int, background=0, tau=0, owner=None):
        """owner: the object that keeps ``user`` valid (e.g. the generator spec); held as long as this volume."""
        h = lib().or_stream_create(_i64(dims), channels, brick, background, tau, ctypes.c_void_p(gen_fn_addr),
                                   ctypes.c_void_p(user))
        if not h:
            raise ValueError("invalid volume geometry")
        super().__init__(h, keep=(owner,))
        self.C = channels
        self.next_z = 0

    def feed(self, z0, slab: np.ndarray, threads=0):
        b = np.ascontiguousarray(slab)
        if b.dtype == np.int16:
            b = b.view(np.uint16)
        if lib().or_stream_feed(self._h, z0, b.shape[0], b.ctypes.data, threads) != 0:
            raise ValueError("slabs must arrive in z order and lie inside the volume")
        self.next_z = z0 + b.shape[0]

    def finish(self, threads=0):
        if lib().or_stream_finish(self._h, threads) != 0:
            raise ValueError("volume not completely fed")

    def level(self, L) -> np.ndarray:
        if L < 1:
            raise ValueError("level 0 of a streamed volume is not stored")
        return DenseVolume.level(self, L)


class LazyVolume(Volume):
    """Level 0 from ``gen_fn(user, x, y, z, out[C])`` for z in [z_lo, z_hi), background elsewhere."""

    def __init__(self, dims, channels, brick, gen_fn_addr: int, user: int, z_lo=0, z_hi=None, background=0, tau=0,
                 owner=None):
        """owner: the object that keeps ``user`` valid (e.g. the generator spec); held as long as this volume."""
        z_hi = dims[2] if z_hi is None else z_hi
        h = lib().or_lazy_create(_i64(dims), channels, brick, background, tau, ctypes.c_void_p(gen_fn_addr),
                                 ctypes.c_void_p(user), z_lo, z_hi)
        if not h:
            raise ValueError("invalid volume geometry")
        super().__init__(h, keep=(owner,))
        self.C = channels


def admissible_error(gpu_rgba: np.ndarray, n_cand: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """Per-pixel max-abs error of gpu_rgba [n][4] to the nearest admissible oracle state (the
    FP64 result, or one of the stopping states near the early-termination threshold)."""
    g = np.asarray(gpu_rgba, dtype=np.float64).reshape(-1, 1, 4)
    c = cand.reshape(g.shape[0], MAXCAND, 4)
    e = np.abs(c - g).max(axis=-1)
    valid = np.arange(MAXCAND)[None, :] < n_cand.reshape(-1, 1)
    return np.where(valid, e, np.inf).min(axis=-1)


def image_pixels(width, height):
    py, px = np.meshgrid(np.arange(height, dtype=np.int32), np.arange(width, dtype=np.int32), indexing="ij")
    return px.ravel().copy(), py.ravel().copy()


def render(vol: Volume, cam: dict, tf: np.ndarray, scale, pixels=None, mode=0, threads=0, xf=None, geometry="fp64"):
    """Returns (n_cand [n], cand [n][MAXCAND][4], samples [n]); pixels = (px, py) arrays or None (all).
    xf: optional per-channel affine sample transforms [C][3][4].  geometry: "fp64" (the definition,
    natural branch of every decision) or "fp32" (single-precision decisions in a fixed order)."""
    if pixels is None:
        px, py = image_pixels(cam["width"], cam["height"])
    else:
        px = np.ascontiguousarray(pixels[0], dtype=np.int32)
        py = np.ascontiguousarray(pixels[1], dtype=np.int32)
    n = px.shape[0]
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    out = (Pixel * max(n, 1))()
    cs = camera_struct(cam)
    xfa = None if xf is None else np.ascontiguousarray(xf, dtype=np.float32).reshape(-1, 3, 4)
    rc = lib().or_render_geo(vol.handle, ctypes.byref(cs), tf.ctypes.data, sc.ctypes.data,
                             None if xfa is None else xfa.ctypes.data, mode, GEOMETRY[geometry], n, px.ctypes.data,
                             py.ctypes.data, ctypes.addressof(out), threads)
    if rc != 0:
        raise ValueError("oracle render: invalid arguments")
    arr = np.ctypeslib.as_array(ctypes.cast(out, ctypes.POINTER(ctypes.c_uint8)),
                                shape=(max(n, 1) * ctypes.sizeof(Pixel),))
    dt = np.dtype([("n_cand", np.int32), ("pad", np.int32), ("rgba", np.float64, (MAXCAND, 4)),
                   ("samples", np.int64)])
    assert dt.itemsize == ctypes.sizeof(Pixel)
    rec = arr.view(dt)[:n]
    return rec["n_cand"].copy(), rec["rgba"].copy(), rec["samples"].copy()


CHECK_DTYPE = np.dtype([("err", np.float64), ("rgba", np.float64, (4,)), ("samples", np.int64), ("flagged", np.int32),
                        ("variants", np.int32), ("unresolved", np.int32), ("pad", np.int32)])


def check(vol: Volume, cam: dict, tf, scale, rgba, pixels=None, mode=0, threads=0, xf=None, geometry="fp64",
          stop_err=0.0):
    """Parity check of rendered pixels against every admissible oracle result (knife-edge decision
    variants x early-termination band; see or_render_check).  rgba: [n][4] (or an image [H][W][4]
    with pixels=None).  Returns a record array with fields err (smallest max-abs difference), rgba
    (natural result), samples, flagged, variants, unresolved."""
    if pixels is None:
        px, py = image_pixels(cam["width"], cam["height"])
    else:
        px = np.ascontiguousarray(pixels[0], dtype=np.int32)
        py = np.ascontiguousarray(pixels[1], dtype=np.int32)
    n = px.shape[0]
    target = np.ascontiguousarray(np.asarray(rgba, dtype=np.float32).reshape(n, 4))
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    out = np.zeros(max(n, 1), dtype=CHECK_DTYPE)
    cs = camera_struct(cam)
    xfa = None if xf is None else np.ascontiguousarray(xf, dtype=np.float32).reshape(-1, 3, 4)
    rc = lib().or_render_check(vol.handle, ctypes.byref(cs), tf.ctypes.data, sc.ctypes.data,
                               None if xfa is None else xfa.ctypes.data, mode, GEOMETRY[geometry], n, px.ctypes.data,
                               py.ctypes.data, target.ctypes.data, float(stop_err), out.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle render_check: invalid arguments")
    return out[:n]


def set_edge_margins(dir_ulps=8.0, safety=1.5):
    """Knife-edge margins of the double-precision geometry (see or_set_edge_margins)."""
    lib().or_set_edge_margins.argtypes = [ctypes.c_double, ctypes.c_double]
    lib().or_set_edge_margins(float(dir_ulps), float(safety))


def render_image(vol, cam, tf, scale, mode=0, threads=0, xf=None):
    """Natural-decision image [H][W][4] (float64) plus the candidate arrays."""
    nc, cand, samples = render(vol, cam, tf, scale, None, mode, threads, xf)
    H, W = cam["height"], cam["width"]
    return cand[:, 0, :].reshape(H, W, 4), nc.reshape(H, W), cand.reshape(H, W, MAXCAND, 4), samples.reshape(H, W)


def render_grad(vol, cam, tf, scale, pixels, dl, threads=0, xf=None, ert_margin=None):
    """d(sum dl * I)/d(tf, scale) over the listed pixels; dl [n][4].  With ert_margin, also returns
    a per-pixel bool array marking the rays whose opacity comes within ert_margin of the
    early-termination threshold after some sample (up to the stopping one)."""
    px = np.ascontiguousarray(pixels[0], dtype=np.int32)
    py = np.ascontiguousarray(pixels[1], dtype=np.int32)
    n = px.shape[0]
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    dl = np.ascontiguousarray(dl, dtype=np.float64).reshape(n, 4)
    C = tf.shape[0]
    dtf = np.zeros((C, 256, 4), dtype=np.float64)
    dsc = np.zeros(C, dtype=np.float64)
    cs = camera_struct(cam)
    xfa = None if xf is None else np.ascontiguousarray(xf, dtype=np.float32).reshape(-1, 3, 4)
    edge = np.zeros(max(n, 1), np.uint8)
    rc = lib().or_render_grad_edges(vol.handle, ctypes.byref(cs), tf.ctypes.data, sc.ctypes.data,
                                    None if xfa is None else xfa.ctypes.data, n, px.ctypes.data, py.ctypes.data,
                                    dl.ctypes.data, dtf.ctypes.data, dsc.ctypes.data,
                                    edge.ctypes.data if ert_margin is not None else None,
                                    float(ert_margin or 0.0), threads)
    if rc != 0:
        raise ValueError("oracle render_grad: invalid arguments")
    if ert_margin is not None:
        return dtf, dsc, edge[:n].astype(bool)
    return dtf, dsc


def render_footprint(vol: Volume, cam: dict, tf: np.ndarray, scale, threads=0):
    """Distinct voxels per level read by trilinear corners and distinct node entries read on the
    descents of a whole DVR frame (single-precision decisions, samples up to the natural stop)."""
    L = lib()
    L.or_render_footprint.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    cs = camera_struct(cam)
    vox = np.zeros(vol.N + 1, dtype=np.int64)
    nodes = np.zeros(1, dtype=np.int64)
    if L.or_render_footprint(vol.handle, ctypes.byref(cs), tf.ctypes.data, sc.ctypes.data, vox.ctypes.data,
                             nodes.ctypes.data, threads) != 0:
        raise ValueError("oracle render_footprint: invalid arguments")
    return [int(x) for x in vox], int(nodes[0])


def ray(vol_or_geom, cam, px, py):
    g = vol_or_geom.geom if isinstance(vol_or_geom, Volume) else vol_or_geom
    d = (ctypes.c_float * 3)()
    t0, t1 = ctypes.c_float(), ctypes.c_float()
    cs = camera_struct(cam)
    hit = lib().or_ray(ctypes.byref(g), ctypes.byref(cs), px, py, d, ctypes.byref(t0), ctypes.byref(t1))
    return bool(hit), np.array(d[:], dtype=np.float32), t0.value, t1.value


def lod_thresholds(vol_or_geom, cam):
    g = vol_or_geom.geom if isinstance(vol_or_geom, Volume) else vol_or_geom
    tl = (ctypes.c_float * MAXL)()
    cs = camera_struct(cam)
    lib().or_lod_thresholds(ctypes.byref(g), ctypes.byref(cs), tl)
    return np.array(tl[: g.N + 1], dtype=np.float32)


def geom(dims, channels, brick, background=0, tau=0) -> Geom:
    g = Geom()
    if lib().or_geom_init(ctypes.byref(g), _i64(dims), channels, brick, background, tau) != 0:
        raise ValueError("invalid geometry")
    return g


def sample_trilinear(vol: Volume, L, p, c=0) -> float:
    lib().or_sample_trilinear.restype = ctypes.c_double
    lib().or_sample_trilinear.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    pp = (ctypes.c_float * 3)(*[float(x) for x in p])
    return lib().or_sample_trilinear(vol.handle, L, pp, c)


def tf_eval(tf_channel: np.ndarray, s: float, I: float) -> np.ndarray:
    lib().or_tf_eval.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    t = np.ascontiguousarray(tf_channel, dtype=np.float32)
    out = (ctypes.c_double * 4)()
    lib().or_tf_eval(t.ctypes.data, float(s), float(I), out)
    return np.array(out[:])


def node_count(vol_or_geom) -> int:
    g = vol_or_geom.geom if isinstance(vol_or_geom, Volume) else vol_or_geom
    return int(lib().or_node_count(ctypes.byref(g)))


def node_index(vol_or_geom, L, i, j, k) -> int:
    g = vol_or_geom.geom if isinstance(vol_or_geom, Volume) else vol_or_geom
    return int(lib().or_node_index(ctypes.byref(g), L, i, j, k))


def render_cache(vol: Volume, cam: dict, tf, scale, resident, pixels=None, mode=0, threads=0):
    """Full-frame render with a partial brick cache.  resident: uint8 per node (node_index order).
    Returns (n_cand, cand, samples, used, requested)."""
    if pixels is None:
        px, py = image_pixels(cam["width"], cam["height"])
    else:
        px = np.ascontiguousarray(pixels[0], dtype=np.int32)
        py = np.ascontiguousarray(pixels[1], dtype=np.int32)
    n = px.shape[0]
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    res = np.ascontiguousarray(resident, dtype=np.uint8)
    nn = node_count(vol)
    assert res.shape == (nn,)
    used = np.zeros(nn, np.uint8)
    req = np.zeros(nn, np.uint8)
    out = (Pixel * max(n, 1))()
    cs = camera_struct(cam)
    rc = lib().or_render_cache(vol.handle, ctypes.byref(cs), tf.ctypes.data, sc.ctypes.data, mode, n,
                               px.ctypes.data, py.ctypes.data, res.ctypes.data, used.ctypes.data, req.ctypes.data,
                               ctypes.addressof(out), threads)
    if rc != 0:
        raise ValueError("oracle render_cache: invalid arguments")
    arr = np.ctypeslib.as_array(ctypes.cast(out, ctypes.POINTER(ctypes.c_uint8)),
                                shape=(max(n, 1) * ctypes.sizeof(Pixel),))
    dt = np.dtype([("n_cand", np.int32), ("pad", np.int32), ("rgba", np.float64, (MAXCAND, 4)),
                   ("samples", np.int64)])
    rec = arr.view(dt)[:n]
    return rec["n_cand"].copy(), rec["rgba"].copy(), rec["samples"].copy(), used, req
