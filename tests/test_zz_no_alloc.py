"""vr_render_noalloc: the render entry point for callers that cannot let the library allocate
during a call (memory budgeted up front, or no device-wide synchronisation from cudaMalloc /
cudaFree allowed).  Called through the C ABI, it must give the same images as vr_render, on two
calls in a row (its fixed scratch array keeps the previous call's contents and must be reset).
Both entry points run the same kernel and a pixel does not depend on the order in which tiles are
taken, so the images must be identical bit for bit, in FP32 and with FP16 interpolation.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from synth import synth as S

pytestmark = pytest.mark.gpu


def test_noalloc_render_matches_vr_render_twice():
    import torch
    import paper_1407_2074_b300 as vr
    from paper_1407_2074_b300 import vr as V

    L = V.lib()
    L.vr_render_noalloc.restype = ctypes.c_int
    L.vr_render_noalloc.argtypes = [ctypes.c_void_p, ctypes.POINTER(V.Camera), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    w = S.tiny()
    vol = w.spec().volume()
    r = vr.Renderer(w.dims, 3, 16)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(64):
        r.insert_slice(z, dev[z])
    r.set_transfer_functions(torch.from_numpy(w.tf()), torch.ones(3))
    stream = torch.cuda.current_stream().cuda_stream
    # 16 mixed-size views, then one view; DVR, DVR with FP16 interpolation, MIP
    for cams in (S.batch_cameras(w.dims)[::4], w.cameras):
        n = len(cams)
        cs = (V.Camera * n)(*[V.camera_struct(c) for c in cams])
        for mode, fp16 in ((V.VR_MODE_DVR, False), (V.VR_MODE_DVR, True), (V.VR_MODE_MIP, False)):
            word = mode | (V.VR_RENDER_FP16 if fp16 else 0)
            ref = r.render(cams, mode=word)
            for _ in range(2):
                out = [torch.full((c["height"], c["width"], 4), -1.0, device="cuda") for c in cams]
                ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in out])
                assert L.vr_render_noalloc(r.handle, cs, n, ptrs, word, ctypes.c_void_p(stream)) == V.VR_OK
                torch.cuda.synchronize()
                for a, b in zip(out, ref):
                    assert torch.equal(a, b)
    too_many = [w.cameras[0]] * 65
    cs = (V.Camera * 65)(*[V.camera_struct(c) for c in too_many])
    out = torch.empty((128, 128, 4), device="cuda")
    ptrs = (ctypes.c_void_p * 65)(*([out.data_ptr()] * 65))
    assert L.vr_render_noalloc(r.handle, cs, 65, ptrs, V.VR_MODE_DVR, ctypes.c_void_p(stream)) == V.VR_ERR_INVALID_ARG
    r.close()
