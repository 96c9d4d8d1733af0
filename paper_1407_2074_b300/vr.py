"""ctypes binding of libvr (include/vr.h).  Argument marshalling only: every step of the path runs
in the library's CUDA kernels; without the built library or a CUDA device the calls raise.

Cameras are dicts with the fields of ``vr_camera`` (see ``synth.synth.camera``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("VR_LIBRARY", os.path.join(_HERE, "libvr.so"))

VR_OK, VR_ERR_INVALID_ARG, VR_ERR_OUT_OF_MEMORY, VR_ERR_CUDA, VR_ERR_STATE, VR_ERR_TIMEOUT, VR_ERR_DEVICE_ASSERT = range(7)
VR_FP32, VR_FP16_INTERP = 0, 1
VR_MODE_DVR, VR_MODE_MIP = 0, 1
VR_RENDER_FP16 = 0x10
VR_HOST_BLOCK, VR_DEVICE_BLOCK, VR_HOST_ASYNC = 0, 1, 2  # vr_insert_block on_device
F_CHILDREN, F_BRICK, F_TOUCHED = 1, 2, 4


class VRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libvr status {status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("background", ctypes.c_uint16), ("homog_threshold", ctypes.c_uint16),
                ("pool_capacity_bytes", ctypes.c_size_t), ("precision", ctypes.c_int),
                ("cache_capacity_bytes", ctypes.c_size_t), ("store_on_host", ctypes.c_int)]


class CacheReport(ctypes.Structure):
    _fields_ = [("requested", ctypes.c_int64), ("uploaded", ctypes.c_int64), ("evicted", ctypes.c_int64),
                ("resident", ctypes.c_int64), ("capacity", ctypes.c_int64)]


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fov_y_deg", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("lod_error_px", ctypes.c_float), ("step_voxels", ctypes.c_float), ("ert_alpha", ctypes.c_float),
                ("n_clip", ctypes.c_int), ("clip", (ctypes.c_float * 4) * 3)]


class Stats(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("channels", ctypes.c_int), ("brick_size", ctypes.c_int),
                ("levels", ctypes.c_int), ("nodes", ctypes.c_int64), ("slots_capacity", ctypes.c_int64),
                ("slots_used", ctypes.c_int64), ("pool_bytes", ctypes.c_int64), ("node_table_bytes", ctypes.c_int64),
                ("last_render_samples", ctypes.c_int64), ("last_render_rays", ctypes.c_int64),
                ("last_render_continued", ctypes.c_int64)]


_AllocFn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FreeFn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _AllocFn), ("free", _FreeFn), ("user", ctypes.c_void_p)]


def torch_allocator(device_index: int) -> Allocator:
    """vr_allocator callbacks on PyTorch's caching allocator: the library's device memory (brick
    pool, node tables, render buffers) is then torch's, counted by torch.cuda.memory_allocated and
    released to torch when the context is destroyed.  alloc returns NULL when torch cannot
    allocate (the library reports VR_ERR_OUT_OF_MEMORY)."""
    import torch

    def alloc(nbytes, user, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device_index, stream if stream else None)
        except Exception:
            return None

    def free(ptr, user, stream):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    return Allocator(_AllocFn(alloc), _FreeFn(free), None)


_live = None  # contexts to destroy before the interpreter (and torch) shuts down


def _close_all():
    for r in list(_live or ()):
        try:
            r.close()
        except Exception:
            pass


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        L.vr_create.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.vr_destroy.argtypes = [vp]
        L.vr_insert_block.argtypes = [vp, i64p, i64p, vp, ctypes.c_int, vp]
        L.vr_insert_slice.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int, vp]
        L.vr_set_transfer_functions.argtypes = [vp, vp, vp, vp]
        L.vr_set_clip_planes.argtypes = [vp, ctypes.c_int, vp]
        L.vr_set_channel_transforms.argtypes = [vp, vp]
        L.vr_render.argtypes = [vp, ctypes.POINTER(Camera), ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, vp]
        L.vr_render_backward.argtypes = [vp, ctypes.POINTER(Camera), ctypes.c_int, ctypes.POINTER(vp), vp, vp, vp]
        L.vr_render_backward_with_images.argtypes = [vp, ctypes.POINTER(Camera), ctypes.c_int, ctypes.POINTER(vp),
                                                     ctypes.POINTER(vp), vp, vp, vp]
        L.vr_read_level.argtypes = [vp, ctypes.c_int, vp, vp]
        L.vr_render_footprint.argtypes = [vp, ctypes.POINTER(Camera), ctypes.c_int, ctypes.POINTER(vp),
                                          ctypes.POINTER(vp), vp, vp]
        L.vr_read_voxels.argtypes = [vp, ctypes.c_int, ctypes.c_int64, vp, vp, vp]
        L.vr_read_node.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint16), vp]
        L.vr_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.vr_debug_raise_error.argtypes = [vp, ctypes.c_int]
        L.vr_last_error.restype = ctypes.c_char_p
        L.vr_last_error.argtypes = [vp]
        L.vr_set_tile_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.vr_cache_update.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(CacheReport)]
        L.vr_cache_load.argtypes = [vp, ctypes.c_int64, vp, vp]
        L.vr_cache_read.argtypes = [vp, vp, vp, vp, vp]
        L.vr_refine_begin.argtypes = [vp, ctypes.POINTER(Camera), vp, ctypes.POINTER(vp)]
        L.vr_refine_pass.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.vr_refine_end.argtypes = [vp]
        L.vr_set_launch_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.vr_set_tile_order.argtypes = [vp, ctypes.c_int]
        L.vr_set_insert_staging.argtypes = [vp, ctypes.c_int]
        L.vr_set_ray_continuation.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.vr_set_gradient_precision.argtypes = [vp, ctypes.c_int]
        L.vr_set_mip_segment_length.argtypes = [vp, ctypes.c_int]
        L.vr_plan_create.argtypes = [vp, ctypes.POINTER(Camera), ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int,
                                     ctypes.POINTER(vp)]
        L.vr_plan_launch.argtypes = [vp, vp]
        L.vr_plan_samples.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.vr_plan_destroy.argtypes = [vp]
        for f in ("vr_create", "vr_destroy", "vr_insert_block", "vr_insert_slice", "vr_set_transfer_functions",
                  "vr_set_clip_planes", "vr_set_channel_transforms", "vr_render", "vr_render_backward", "vr_render_backward_with_images", "vr_read_level", "vr_read_voxels", "vr_read_node", "vr_render_footprint",
                  "vr_stats", "vr_set_tile_shape", "vr_set_launch_shape", "vr_set_tile_order", "vr_set_insert_staging", "vr_set_ray_continuation", "vr_set_mip_segment_length",
                  "vr_set_gradient_precision", "vr_plan_create",
                  "vr_plan_launch",
                  "vr_cache_update", "vr_cache_load", "vr_cache_read", "vr_refine_begin", "vr_refine_pass",
                  "vr_refine_end",
                  "vr_plan_samples", "vr_plan_destroy"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def camera_struct(cam: dict) -> Camera:
    c = Camera()
    for k in ("eye", "target", "up"):
        getattr(c, k)[:] = [float(x) for x in cam[k]]
    c.fov_y_deg, c.width, c.height = cam["fov_y_deg"], cam["width"], cam["height"]
    c.lod_error_px, c.step_voxels, c.ert_alpha = cam["lod_error_px"], cam["step_voxels"], cam["ert_alpha"]
    clip = cam.get("clip", [])
    if clip is None:
        c.n_clip = -1
    else:
        c.n_clip = len(clip)
        for i, p in enumerate(clip):
            c.clip[i][:] = [float(x) for x in p]
    return c


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return int(stream)


class Renderer:
    """One volume context (vr_ctx) on the current CUDA device."""

    def __init__(self, dims, channels, brick, background=0, tau=0, pool_capacity_bytes=0, precision="fp32",
                 device=None, cache_capacity_bytes=0, store_on_host=False, allocator="torch"):
        """allocator: "torch" (default) -- the library's device memory comes from PyTorch's caching
        allocator through vr_allocator; None -- the library allocates with cudaMalloc itself."""
        global _live
        import atexit
        import weakref

        import torch

        self._ctx = None
        if device is not None:
            torch.cuda.set_device(torch.device(device))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.dims, self.C, self.M = tuple(int(d) for d in dims), int(channels), int(brick)
        self.precision = precision
        opt = Options(background, tau, pool_capacity_bytes, VR_FP16_INTERP if precision == "fp16" else VR_FP32,
                      cache_capacity_bytes, 1 if store_on_host else 0)
        # the callbacks live as long as the context
        self._alloc = torch_allocator(self.device.index) if allocator == "torch" else None
        if allocator not in ("torch", None):
            raise ValueError('allocator must be "torch" or None')
        h = ctypes.c_void_p()
        rc = lib().vr_create((ctypes.c_int64 * 3)(*self.dims), self.C, self.M, ctypes.byref(opt),
                             ctypes.byref(self._alloc) if self._alloc is not None else None, ctypes.byref(h))
        if rc != VR_OK:
            raise VRError(rc, lib().vr_last_error(None).decode())
        self._ctx = h.value
        self._plans = weakref.WeakSet()  # destroyed before the context (a plan refers to it)
        if _live is None:
            _live = weakref.WeakSet()
            atexit.register(_close_all)
        _live.add(self)
        st = self.stats()
        self.levels = st.levels

    def _check(self, rc):
        if rc != VR_OK:
            raise VRError(rc, lib().vr_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            for p in list(getattr(self, "_plans", ())):
                p.close()
            lib().vr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._ctx

    # ---- construction ----
    def insert_block(self, origin, block, stream=None, overlap=False):
        """block: [ez][ey][ex][C] uint16, a CUDA tensor (device) or a numpy array / CPU tensor (host).
        overlap=True (host blocks): the upload runs on the library's upload stream beside the work
        already queued on `stream` (VR_HOST_ASYNC); keep the block unchanged until `stream` has
        passed this insert."""
        import torch

        ext = None
        if isinstance(block, torch.Tensor) and block.is_cuda:
            assert block.dtype == torch.uint16 or block.dtype == torch.int16
            b = block.contiguous()
            ext = (b.shape[2], b.shape[1], b.shape[0])
            ptr, on_dev, keep = b.data_ptr(), 1, b
        else:
            b = np.ascontiguousarray(block.numpy() if isinstance(block, torch.Tensor) else block)
            if b.dtype == np.int16:
                b = b.view(np.uint16)  # same bytes; keeps pinned host memory pinned
            b = np.ascontiguousarray(b, dtype=np.uint16)
            ext = (b.shape[2], b.shape[1], b.shape[0])
            ptr, on_dev, keep = b.ctypes.data, (VR_HOST_ASYNC if overlap else 0), b
        self._check(lib().vr_insert_block(self._ctx, (ctypes.c_int64 * 3)(*origin), (ctypes.c_int64 * 3)(*ext),
                                          ctypes.c_void_p(ptr), on_dev, ctypes.c_void_p(_stream_ptr(stream))))
        return keep

    def insert_slice(self, z, slice_, stream=None):
        """slice_: [Y][X][C] uint16 (device tensor or host array)."""
        import torch

        if isinstance(slice_, torch.Tensor) and slice_.is_cuda:
            s = slice_.contiguous()
            ptr, on_dev = s.data_ptr(), 1
        else:
            s = np.ascontiguousarray(slice_.numpy() if isinstance(slice_, torch.Tensor) else slice_)
            if s.dtype == np.int16:
                s = s.view(np.uint16)
            s = np.ascontiguousarray(s, dtype=np.uint16)
            ptr, on_dev = s.ctypes.data, 0
        self._check(lib().vr_insert_slice(self._ctx, int(z), ctypes.c_void_p(ptr), on_dev,
                                          ctypes.c_void_p(_stream_ptr(stream))))
        return s

    # ---- render parameters ----
    def set_transfer_functions(self, tf, scale, stream=None):
        import torch

        tf = torch.as_tensor(tf, dtype=torch.float32, device=self.device).contiguous()
        sc = torch.as_tensor(scale, dtype=torch.float32, device=self.device).contiguous()
        assert tf.shape == (self.C, 256, 4) and sc.shape == (self.C,)
        self._check(lib().vr_set_transfer_functions(self._ctx, ctypes.c_void_p(tf.data_ptr()),
                                                    ctypes.c_void_p(sc.data_ptr()),
                                                    ctypes.c_void_p(_stream_ptr(stream))))
        self._tf_keep = (tf, sc)

    def set_clip_planes(self, planes):
        p = np.ascontiguousarray(np.asarray(planes, dtype=np.float32).reshape(-1, 4))
        self._check(lib().vr_set_clip_planes(self._ctx, p.shape[0], p.ctypes.data if p.shape[0] else None))

    def set_channel_transforms(self, xf):
        """xf: [C][3][4] per-channel affine sample transforms, or None for identity."""
        if xf is None:
            self._check(lib().vr_set_channel_transforms(self._ctx, None))
            return
        m = np.ascontiguousarray(np.asarray(xf, dtype=np.float32).reshape(self.C, 3, 4))
        self._check(lib().vr_set_channel_transforms(self._ctx, m.ctypes.data))

    def set_tile_shape(self, tw, th):
        self._check(lib().vr_set_tile_shape(self._ctx, tw, th))

    def set_launch_shape(self, tw, th, threads=768, ctas_per_sm=1):
        self._check(lib().vr_set_launch_shape(self._ctx, tw, th, threads, ctas_per_sm))

    def set_mip_segment_length(self, samples):
        """MIP: samples per ray segment (0: rays marched whole; default 1024)."""
        self._check(lib().vr_set_mip_segment_length(self._ctx, samples))

    def set_gradient_precision(self, fp64):
        """render_backward accumulation: False (single precision) or True (FP64 gradient-check mode)."""
        self._check(lib().vr_set_gradient_precision(self._ctx, 1 if fp64 else 0))

    def set_tile_order(self, mode):
        """0: raster tile queue; 1 (default): costliest tiles of the previous render of the same grid first."""
        self._check(lib().vr_set_tile_order(self._ctx, mode))

    def set_insert_staging(self, mode):
        """1 (default): level 0 of an insert stages the block's rows in shared memory by TMA copies
        when the block is 16-byte aligned; 0: per-thread loads.  Same tree either way."""
        self._check(lib().vr_set_insert_staging(self._ctx, mode))

    def set_ray_continuation(self, lanes_per_ray=16, min_samples_left=32):
        """Once the tile queue runs dry, finish rays with more than ``min_samples_left`` samples to go
        in a second launch with ``lanes_per_ray`` lanes each (0 = off); see vr_set_ray_continuation."""
        self._check(lib().vr_set_ray_continuation(self._ctx, int(lanes_per_ray), int(min_samples_left)))

    def plan(self, cams, images=None, mode=VR_MODE_DVR):
        """A graph-captured single launch over all ``cams``; returns a RenderPlan."""
        return RenderPlan(self, cams, images, mode)

    # ---- render ----
    def render(self, cams, images=None, mode=VR_MODE_DVR, stream=None):
        import torch

        n = len(cams)
        cs = (Camera * n)(*[camera_struct(c) for c in cams])
        if images is None:
            images = [torch.empty((c["height"], c["width"], 4), dtype=torch.float32, device=self.device) for c in cams]
        ptrs = (ctypes.c_void_p * n)(*[im.data_ptr() for im in images])
        self._check(lib().vr_render(self._ctx, cs, n, ptrs, mode, ctypes.c_void_p(_stream_ptr(stream))))
        return images

    def footprint(self, cams, stream=None):
        """Algorithmic footprint of a DVR render of ``cams``: (distinct voxels per level, distinct
        node entries visited)."""
        import torch

        n = len(cams)
        cs = (Camera * n)(*[camera_struct(c) for c in cams])
        images = [torch.empty((c["height"], c["width"], 4), dtype=torch.float32, device=self.device) for c in cams]
        ptrs = (ctypes.c_void_p * n)(*[im.data_ptr() for im in images])
        X, Y, Z = self.dims
        marks = []
        for L in range(self.levels):
            marks.append(torch.zeros(((X * Y * Z + 31) // 32,), dtype=torch.int32, device=self.device))
            X, Y, Z = (X + 1) // 2, (Y + 1) // 2, (Z + 1) // 2
        nodes = torch.zeros(((self.stats().nodes + 31) // 32,), dtype=torch.int32, device=self.device)
        mptr = (ctypes.c_void_p * len(marks))(*[m.data_ptr() for m in marks])
        self._check(lib().vr_render_footprint(self._ctx, cs, n, ptrs, mptr, ctypes.c_void_p(nodes.data_ptr()),
                                              ctypes.c_void_p(_stream_ptr(stream))))

        def popcount(t):
            tot = 0
            for ch in torch.split(t, 1 << 24):
                x = ch.to(torch.int64) & 0xFFFFFFFF
                x = x - ((x >> 1) & 0x55555555)
                x = (x & 0x33333333) + ((x >> 2) & 0x33333333)
                x = (x + (x >> 4)) & 0x0F0F0F0F
                x = ((x * 0x01010101) & 0xFFFFFFFF) >> 24
                tot += int(x.sum().item())
            return tot

        return [popcount(m) for m in marks], popcount(nodes)

    def render_backward(self, cams, grads, dtf=None, dscale=None, stream=None, images=None):
        """dL/d(tf, scale) for dL/dimage ``grads``.  ``images``: the FP32 DVR images render() gave
        for the same cameras and state -- each ray is then marched once instead of twice
        (vr_render_backward_with_images)."""
        import torch

        n = len(cams)
        cs = (Camera * n)(*[camera_struct(c) for c in cams])
        gs = [g.contiguous().float() for g in grads]
        ptrs = (ctypes.c_void_p * n)(*[g.data_ptr() for g in gs])
        if dtf is None:
            dtf = torch.empty((self.C, 256, 4), dtype=torch.float32, device=self.device)
        if dscale is None:
            dscale = torch.empty((self.C,), dtype=torch.float32, device=self.device)
        if images is None:
            self._check(lib().vr_render_backward(self._ctx, cs, n, ptrs, ctypes.c_void_p(dtf.data_ptr()),
                                                 ctypes.c_void_p(dscale.data_ptr()),
                                                 ctypes.c_void_p(_stream_ptr(stream))))
        else:
            ims = [im.contiguous() for im in images]
            iptrs = (ctypes.c_void_p * n)(*[im.data_ptr() for im in ims])
            self._check(lib().vr_render_backward_with_images(self._ctx, cs, n, iptrs, ptrs,
                                                             ctypes.c_void_p(dtf.data_ptr()),
                                                             ctypes.c_void_p(dscale.data_ptr()),
                                                             ctypes.c_void_p(_stream_ptr(stream))))
        return dtf, dscale

    # ---- inspection ----
    def read_level(self, L, stream=None) -> np.ndarray:
        st = self.stats()
        X, Y, Z = self.dims
        for _ in range(L):
            X, Y, Z = (X + 1) // 2, (Y + 1) // 2, (Z + 1) // 2
        out = np.empty((Z, Y, X, self.C), dtype=np.uint16)
        self._check(lib().vr_read_level(self._ctx, L, out.ctypes.data, ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def read_voxels(self, L, xyz, stream=None) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(xyz, dtype=np.int64).reshape(-1, 3))
        out = np.empty((c.shape[0], self.C), dtype=np.uint16)
        self._check(lib().vr_read_voxels(self._ctx, L, c.shape[0], c.ctypes.data, out.ctypes.data,
                                         ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def read_node(self, L, i, j, k, stream=None):
        fl = ctypes.c_uint32()
        avg = (ctypes.c_uint16 * 4)()
        self._check(lib().vr_read_node(self._ctx, L, i, j, k, ctypes.byref(fl), avg,
                                       ctypes.c_void_p(_stream_ptr(stream))))
        return int(fl.value), list(avg[: self.C])

    # ---- out-of-core rendering ----
    def cache_update(self, max_uploads=1 << 30, refinement=False, stream=None) -> dict:
        rep = CacheReport()
        self._check(lib().vr_cache_update(self._ctx, int(min(max_uploads, 2 ** 31 - 1)), 1 if refinement else 0,
                                          ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(rep)))
        return {k: getattr(rep, k) for k, _ in CacheReport._fields_}

    def cache_load(self, nodes, stream=None):
        a = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64).reshape(-1))
        self._check(lib().vr_cache_load(self._ctx, a.shape[0], a.ctypes.data, ctypes.c_void_p(_stream_ptr(stream))))

    def cache_read(self, stream=None):
        n = self.stats().nodes
        res, used, req = (np.zeros(n, np.uint8) for _ in range(3))
        self._check(lib().vr_cache_read(self._ctx, res.ctypes.data, used.ctypes.data, req.ctypes.data,
                                        ctypes.c_void_p(_stream_ptr(stream))))
        return res, used, req

    def refine(self, cam, image=None):
        """Refinement session of one view; call .pass_() and cache_update(refinement=True) until done."""
        return RefineSession(self, cam, image)

    def debug_raise_error(self, code=1):
        """Test hook: sets the device error word as a failed kernel check would (vr_debug_raise_error)."""
        self._check(lib().vr_debug_raise_error(self._ctx, code))

    def stats(self) -> Stats:
        s = Stats()
        self._check(lib().vr_stats(self._ctx, ctypes.byref(s)))
        return s


class RefineSession:
    """vr_refine: refinement ray casting of one view (resumable rays over passes)."""

    def __init__(self, renderer, cam, image=None):
        import torch

        self.r = renderer
        self.cam = cam
        self.image = image if image is not None else torch.zeros((cam["height"], cam["width"], 4),
                                                                 dtype=torch.float32, device=renderer.device)
        cs = camera_struct(cam)
        h = ctypes.c_void_p()
        renderer._check(lib().vr_refine_begin(renderer.handle, ctypes.byref(cs), ctypes.c_void_p(self.image.data_ptr()),
                                              ctypes.byref(h)))
        self._p = h.value

    def pass_(self, stream=None):
        """One pass; returns (rays still pending, samples composited in the pass)."""
        pend, samp = ctypes.c_int64(), ctypes.c_int64()
        self.r._check(lib().vr_refine_pass(self._p, ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(pend),
                                           ctypes.byref(samp)))
        return pend.value, samp.value

    def close(self):
        if self._p:
            lib().vr_refine_end(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderPlan:
    """vr_render_plan: one persistent launch over a fixed camera batch, replayed as a CUDA graph."""

    def __init__(self, renderer, cams, images=None, mode=VR_MODE_DVR):
        import torch

        self.r = renderer
        n = len(cams)
        self.cams = cams
        self.images = images if images is not None else [
            torch.empty((c["height"], c["width"], 4), dtype=torch.float32, device=renderer.device) for c in cams]
        cs = (Camera * n)(*[camera_struct(c) for c in cams])
        ptrs = (ctypes.c_void_p * n)(*[im.data_ptr() for im in self.images])
        h = ctypes.c_void_p()
        self._p = None
        renderer._check(lib().vr_plan_create(renderer.handle, cs, n, ptrs, mode, ctypes.byref(h)))
        self._p = h.value
        renderer._plans.add(self)

    def launch(self, stream=None):
        self.r._check(lib().vr_plan_launch(self._p, ctypes.c_void_p(_stream_ptr(stream))))
        return self.images

    def samples(self):
        s, r = ctypes.c_int64(), ctypes.c_int64()
        self.r._check(lib().vr_plan_samples(self._p, ctypes.byref(s), ctypes.byref(r)))
        return s.value, r.value

    def close(self):
        if self._p:
            lib().vr_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _torch_fn():
    import torch

    class RenderFn(torch.autograd.Function):
        """images = RenderFn.apply(tf [C,256,4], scale [C], renderer, cams); backward through the
        hand-written adjoint (vr_render_backward), recomputing each ray's march."""

        @staticmethod
        def forward(ctx, tf, scale, renderer, cams):
            renderer.set_transfer_functions(tf.detach(), scale.detach())
            imgs = renderer.render(cams, mode=VR_MODE_DVR)
            ctx.renderer, ctx.cams = renderer, cams
            # FP32 images: the backward reads each ray's final colour and transmittance from them
            ctx.fp32 = renderer.precision != "fp16"
            ctx.save_for_backward(tf, scale, *imgs)
            return tuple(imgs)

        @staticmethod
        def backward(ctx, *grads):
            tf, scale, *imgs = ctx.saved_tensors
            r = ctx.renderer
            gs = [g if g is not None else torch.zeros((c["height"], c["width"], 4), device=r.device)
                  for g, c in zip(grads, ctx.cams)]
            r.set_transfer_functions(tf.detach(), scale.detach())
            dtf, dsc = r.render_backward(ctx.cams, gs, images=imgs if ctx.fp32 else None)
            return dtf, dsc, None, None

    return RenderFn


class _Lazy:
    def __init__(self):
        self._fn = None

    def apply(self, *a):
        if self._fn is None:
            self._fn = _torch_fn()
        return self._fn.apply(*a)


RenderFn = _Lazy()


def render(renderer: Renderer, cams, tf, scale):
    """Differentiable render of ``cams`` with tables ``tf`` and scales ``scale`` (torch tensors)."""
    return list(RenderFn.apply(tf, scale, renderer, cams))
