"""Render parity: every GPU pixel is within RGBA max-abs 2e-3 of an admissible oracle result: the
double-precision render with either branch of each knife-edge decision (level floor, child at a
split plane) and any stopping state in the early-termination band."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import RGBA_TOL, oracle_dense, parity

pytestmark = pytest.mark.gpu


def _build(vol, M, bg=0, tau=0, z_hi=None, precision="fp32"):
    import torch
    import paper_1407_2074_b300 as vr

    Z, Y, X, C = vol.shape
    r = vr.Renderer((X, Y, Z), C, M, background=bg, tau=tau, precision=precision)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(Z if z_hi is None else z_hi):
        r.insert_slice(z, dev[z])
    return r


def _render(r, cams, tf, scale, mode=0):
    import torch

    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor(scale, dtype=torch.float32))
    imgs = r.render(cams, mode=mode)
    torch.cuda.synchronize()
    return [im.cpu().numpy() for im in imgs]


def _check_full(img, ov, cam, tf, scale, mode=0, tol=RGBA_TOL, xf=None):
    return parity(ov, cam, tf, scale, img.reshape(-1, 4), None, mode, xf=xf, tol=tol)["err"]


def _check_pixels(img, ov, cam, tf, scale, px, py, mode=0, tol=RGBA_TOL):
    return parity(ov, cam, tf, scale, img[py, px], (px, py), mode, tol=tol)["err"]


@pytest.fixture(scope="module")
def tiny():
    w = S.tiny()
    vol = w.spec().volume()
    return w, vol, oracle_dense(vol, 16)


def test_tiny_full_image(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    img = _render(r, w.cameras, tf, sc)[0]
    err = _check_full(img, ov, w.cameras[0], tf, sc)
    assert err.mean() < 1e-5
    st = r.stats()
    _, _, samples = O.render(ov, w.cameras[0], tf, sc, None, 0, geometry="fp32")
    assert st.last_render_samples == int(samples.sum())


def test_tiny_opaque_tf_clip_planes_and_scales(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    tf = w.tf()
    tf[..., 3] = np.minimum(1.0, tf[..., 3] * 12.0)  # most rays terminate early
    sc = [1.7, 0.6, 2.5]
    cam = dict(w.cameras[0])
    cam["clip"] = [S.centre_plane(w.dims, (1.0, 0.5, 0.25), 3.0), (0.0, 1.0, 0.0, -10.0)]
    img = _render(r, [cam], tf, sc)[0]
    _check_full(img, ov, cam, tf, sc)


def test_tiny_mip(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    img = _render(r, w.cameras, tf, sc, mode=1)[0]
    _check_full(img, ov, w.cameras[0], tf, sc, mode=1)


@pytest.mark.parametrize("tau,eps", [(0, 0.6), (3277, 1.5)])
def test_mip_streamed_matches_oracle(tau, eps):
    """MIP (samples of a brick node taken in pairs) on a SPIM-like volume rendered while it
    streams in and again when complete: the image and the sample count equal the oracle's
    sample-by-sample maximum."""
    import torch

    dims = (160, 128, 96)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 150, seed=21)
    vol = spec.volume()
    r = _build(vol, 16, tau=tau, z_hi=48)
    cam = S.orbit_camera(dims, 1.7 * 160, 25.0, 15.0, 200, 150, lod_error_px=eps)
    tf, sc = S.make_tf([11, 12, 13]), [1.0, 1.0, 1.0]
    _render(r, [cam], tf, sc, mode=1)  # render, then stream the rest of the volume in
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(48, 96):
        r.insert_slice(z, dev[z])
    ov = oracle_dense(vol, 16, tau=tau)
    img = _render(r, [cam], tf, sc, mode=1)[0]
    _check_full(img, ov, cam, tf, sc, mode=1)
    _, _, samples = O.render(ov, cam, tf, sc, None, 1, geometry="fp32")
    assert r.stats().last_render_samples == int(samples.sum())


def test_context_clip_planes_apply_to_cameras_without_their_own(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    plane = (0.0, 0.0, -1.0, 40.0)
    r.set_clip_planes([plane])
    cam = dict(w.cameras[0])
    cam["clip"] = None  # n_clip = -1: the context's planes
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    img = _render(r, [cam], tf, sc)[0]
    ref_cam = dict(w.cameras[0])
    ref_cam["clip"] = [plane]
    _check_full(img, ov, ref_cam, tf, sc)


@pytest.mark.parametrize("eye,target", [((20.0, 30.0, 25.0), (40.0, 35.0, 60.0)),   # inside the volume
                                        ((32.0, 32.0, -96.0), (32.0, 32.0, 32.0)),   # axis-aligned centre rays
                                        ((200.0, 200.0, 200.0), (400.0, 400.0, 400.0))])  # looking away
def test_tiny_camera_placements(tiny, eye, target):
    w, vol, ov = tiny
    r = _build(vol, 16)
    cam = S.camera(eye, target, (0.0, 1.0, 0.0), 64, 63, fov_y_deg=70.0)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    img = _render(r, [cam], tf, sc)[0]
    _check_full(img, ov, cam, tf, sc)


@pytest.mark.parametrize("C,M,dims,tau", [(1, 6, (45, 38, 29), 300), (2, 4, (33, 40, 21), 0), (4, 8, (48, 32, 40), 900)])
def test_channels_and_brick_sizes(C, M, dims, tau):
    spec = S.VolumeSpec(S.KIND_SPIM, dims, C, 40, seed=6)
    vol = spec.volume()
    ov = oracle_dense(vol, M, bg=30, tau=tau)
    r = _build(vol, M, bg=30, tau=tau)
    d = max(dims)
    cam = S.orbit_camera(dims, 1.6 * d, 37.0, 25.0, 96, 80, lod_error_px=0.35)
    tf = S.make_tf([21 + c for c in range(C)])
    tf[..., 3] *= 4.0
    sc = [1.0 + 0.3 * c for c in range(C)]
    img = _render(r, [cam], tf, sc)[0]
    _check_full(img, ov, cam, tf, sc)


def test_medium_spim_homogeneity_partial_insert_and_lod():
    # A reduced streamed workload: SPIM-like volume, tau = 3277, half of the slices inserted,
    # oblique clip plane, LOD thresholds inside the volume (levels 0..2 sampled).
    dims = (192, 160, 96)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 160, seed=2)
    vol = spec.volume()
    ov = oracle_dense(vol, 16, tau=3277, z_hi=60)
    r = _build(vol, 16, tau=3277, z_hi=60)
    cam = S.orbit_camera(dims, 2.0 * 192, 20.0, 20.0, 480, 270, lod_error_px=2.5,
                         clip=[S.centre_plane(dims, (1.0, 0.5, 0.25))])
    tl = O.lod_thresholds(ov, cam)
    assert 0 < tl[1] < 2.0 * 192 + 200
    tf, sc = S.make_tf([11, 12, 13]), [1.0, 1.0, 1.0]
    tf[..., 3] *= 3.0
    img = _render(r, [cam], tf, sc)[0]
    _check_full(img, ov, cam, tf, sc)


def test_batched_cameras_one_launch(tiny):
    """The batched workload: 64 views of uneven resolution (53.9 M rays) in one launch, FP32 and FP16
    interpolation, every pixel of every view against the oracle."""
    from paper_1407_2074_b300 import vr as V

    w, vol, ov = tiny
    r = _build(vol, 16)
    cams = S.batch_cameras(w.dims)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    imgs = _render(r, cams, tf, sc)
    imgs16 = _render(r, cams, tf, sc, mode=V.VR_MODE_DVR | V.VR_RENDER_FP16)
    e32 = e16 = 0.0
    for cam, a32, a16 in zip(cams, imgs, imgs16):
        e32 = max(e32, float(_check_full(a32, ov, cam, tf, sc).max()))
        e16 = max(e16, float(_check_full(a16, ov, cam, tf, sc).max()))
    print(f"batched, 64 views: FP32 max {e32:.2e}, FP16 max {e16:.2e}")
    alone = _render(r, [cams[7]], tf, sc)[0]
    assert np.array_equal(alone, imgs[7])  # a ray does not depend on the other views of the launch


def test_render_is_deterministic(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    a = _render(r, w.cameras, tf, sc)[0]
    b = _render(r, w.cameras, tf, sc)[0]
    assert np.array_equal(a, b)


def test_tile_shapes_give_identical_images(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    ref = _render(r, w.cameras, tf, sc)[0]
    for tw, th in ((32, 1), (16, 2), (4, 8)):
        r.set_tile_shape(tw, th)
        assert np.array_equal(_render(r, w.cameras, tf, sc)[0], ref)


def test_tile_order_buffers_grow_and_shrink_with_the_grid(tiny):
    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    small = dict(w.cameras[0], width=40, height=24)
    large = dict(w.cameras[0], width=333, height=197)  # ragged tiles
    r.set_tile_order(0)
    ref_s, ref_l = _render(r, [small], tf, sc)[0], _render(r, [large], tf, sc)[0]
    r.set_tile_order(1)
    for cam, ref in ((small, ref_s), (small, ref_s), (large, ref_l), (large, ref_l), (small, ref_s),
                     (large, ref_l), (large, ref_l), (small, ref_s), (small, ref_s)):
        assert np.array_equal(_render(r, [cam], tf, sc)[0], ref)
    r.close()


def test_tile_order_from_previous_costs_changes_no_pixel(tiny):
    from paper_1407_2074_b300 import vr as V

    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    cams = S.batch_cameras(w.dims)[:9]
    r.set_tile_order(0)
    ref = _render(r, cams, tf, sc)
    counts = (r.stats().last_render_samples, r.stats().last_render_rays)
    ref1 = _render(r, w.cameras, tf, sc)[0]
    r.set_tile_order(1)
    for _ in range(3):  # raster order and costs first, then queued by the costs of the call before
        for a, b in zip(_render(r, cams, tf, sc), ref):
            assert np.array_equal(a, b)
        assert (r.stats().last_render_samples, r.stats().last_render_rays) == counts
    for _ in range(2):  # another grid starts over in raster order
        assert np.array_equal(_render(r, w.cameras, tf, sc)[0], ref1)
    fp16 = V.VR_MODE_DVR | V.VR_RENDER_FP16
    r.set_tile_order(0)
    ref16 = _render(r, cams, tf, sc, mode=fp16)
    r.set_tile_order(1)
    for _ in range(2):
        for a, b in zip(_render(r, cams, tf, sc, mode=fp16), ref16):
            assert np.array_equal(a, b)
    with pytest.raises(V.VRError):
        r.set_tile_order(2)
    r.close()


def _full_size_render(w, frames, tau, n_px, seed):
    import torch
    import paper_1407_2074_b300 as vr

    spec = w.spec()
    X, Y, Z = w.dims
    r = vr.Renderer(w.dims, 3, w.brick, tau=tau)
    buf = torch.empty((8, Y, X, 3), dtype=torch.int16, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for z0 in range(0, Z, 8):
        spec.generate_device(buf.data_ptr(), z0, min(Z, z0 + 8), st)
        r.insert_block((0, 0, z0), buf[: min(Z, z0 + 8) - z0])
    del buf
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    imgs = _render(r, w.cameras, tf, sc)
    lazy = O.LazyVolume(w.dims, 3, w.brick, spec.voxel_fn, spec.handle, 0, Z, tau=0, owner=spec)
    rng = np.random.default_rng(seed)
    for cam, img in zip(w.cameras, imgs):
        hit = np.argwhere(img[..., 3] > 0.05)
        pick = hit[rng.choice(len(hit), size=min(n_px, len(hit)), replace=False)]
        _check_pixels(img, lazy, cam, tf, sc, pick[:, 1].astype(np.int32), pick[:, 0].astype(np.int32))
    r.close()


def test_streamed_full_size_sampled_pixels():
    """1024x1024x512 at 1920x1080 with the oblique clip plane (tau = 0: the lazy oracle needs no
    node scans), sampled pixels against the lazy oracle."""
    _full_size_render(S.streamed(tau=0), None, 0, 48, 1)


def test_large_full_size_sampled_pixels():
    """The 24 GiB 2048x2048x1024 volume at 1920x1080 (orbit frame 0), sampled pixels."""
    _full_size_render(S.large(tau=0), None, 0, 24, 2)


def _stream_oracle(w, tau, slab=16):
    """The oracle state of the whole workload volume, fed in z order from the synthetic generator
    (its device form, checked against the host form on one slab here and in the generator tests)."""
    import torch

    spec = w.spec()
    X, Y, Z = w.dims
    st = O.StreamVolume(w.dims, 3, w.brick, spec.voxel_fn, spec.handle, tau=tau, owner=spec)
    buf = torch.empty((slab, Y, X, 3), dtype=torch.int16, device="cuda")
    host = torch.empty((slab, Y, X, 3), dtype=torch.int16, pin_memory=True)
    s = torch.cuda.current_stream().cuda_stream
    for z0 in range(0, Z, slab):
        z1 = min(Z, z0 + slab)
        spec.generate_device(buf.data_ptr(), z0, z1, s)
        host[: z1 - z0].copy_(buf[: z1 - z0])
        torch.cuda.synchronize()
        if z0 == slab * (Z // (2 * slab)):
            assert np.array_equal(host[: z1 - z0].numpy().view(np.uint16), spec.slices(z0, z1))
        st.feed(z0, host[: z1 - z0].numpy())
    st.finish()
    return st


@pytest.mark.parametrize("name", ["streamed", "large"])
def test_full_size_tau_3277_frames_fp32_and_fp16(name):
    """The benchmarked configuration: full-size volume with tau = 3277 (homogeneous subtrees pruned,
    closed-form runs), 1920x1080 orbit frames 0, 15, 30, 45, the default launch shape; every pixel
    of frame 0 and sampled pixels of the other frames, FP32 and FP16 interpolation, within the
    parity tolerance of the oracle's admissible results."""
    import torch
    import paper_1407_2074_b300 as vr
    from paper_1407_2074_b300 import vr as V

    frames = (0, 15, 30, 45)
    if name == "streamed":
        w = S.streamed(tau=3277)
        w.cameras = [S.streamed(tau=3277, frame=f).cameras[0] for f in frames]
    else:
        w = S.large(tau=3277, frames=frames)
    spec = w.spec()
    X, Y, Z = w.dims
    r = vr.Renderer(w.dims, 3, w.brick, tau=w.tau)
    buf = torch.empty((8, Y, X, 3), dtype=torch.int16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for z0 in range(0, Z, 8):
        spec.generate_device(buf.data_ptr(), z0, min(Z, z0 + 8), s)
        r.insert_block((0, 0, z0), buf[: min(Z, z0 + 8) - z0])
    del buf
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    r.set_transfer_functions(torch.from_numpy(tf).cuda(), torch.ones(3, device="cuda"))
    H, W = w.cameras[0]["height"], w.cameras[0]["width"]
    img32 = torch.empty((H, W, 4), device="cuda")
    img16 = torch.empty((H, W, 4), device="cuda")
    st = _stream_oracle(w, 3277)
    rng = np.random.default_rng(7)
    for f, cam in zip(frames, w.cameras):
        r.render([cam], [img32])
        r.render([cam], [img16], mode=V.VR_MODE_DVR | V.VR_RENDER_FP16)
        torch.cuda.synchronize()
        a32, a16 = img32.cpu().numpy(), img16.cpu().numpy()
        if f == 0:  # the whole frame
            e32 = parity(st, cam, tf, sc, a32.reshape(-1, 4))["err"]
            e16 = parity(st, cam, tf, sc, a16.reshape(-1, 4))["err"]
            print(f"{name} frame 0, {e32.size} pixels: FP32 max {e32.max():.2e}; FP16 max {e16.max():.2e}")
            continue
        hit = np.argwhere(a32[..., 3] > 0.05)
        pick = np.concatenate([hit[rng.choice(len(hit), size=min(40, len(hit)), replace=False)],
                               np.stack([rng.integers(0, H, 8), rng.integers(0, W, 8)], 1)])
        px, py = pick[:, 1].astype(np.int32), pick[:, 0].astype(np.int32)
        e32 = parity(st, cam, tf, sc, a32[py, px], (px, py))["err"]
        e16 = parity(st, cam, tf, sc, a16[py, px], (px, py))["err"]
        print(f"{name} frame {f}: FP32 max {e32.max():.2e}; FP16 max {e16.max():.2e} mean {e16.mean():.2e}")
    r.close()


def test_homogeneous_runs_with_early_termination():
    # tau = 3277 makes the background outside the tissue one homogeneous subtree: long runs of
    # equal samples composited in closed form.  Constant alpha 0.03 per voxel makes most rays
    # terminate inside such runs; the oracle composites sample by sample.
    dims = (160, 128, 96)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 120, seed=12)
    vol = spec.volume()
    ov = oracle_dense(vol, 16, tau=3277)
    r = _build(vol, 16, tau=3277)
    tf = S.make_tf([31, 32, 33])
    tf[..., 3] = 0.03
    sc = [1.0, 1.0, 1.0]
    for eps, ert in ((1.0, 0.99), (0.3, 0.7), (4.0, 2.0)):
        cam = S.orbit_camera(dims, 1.7 * 160, 50.0, 30.0, 200, 150, lod_error_px=eps, ert_alpha=ert)
        img = _render(r, [cam], tf, sc)[0]
        _check_full(img, ov, cam, tf, sc)


def _fp16_errors(img, ov, cam, tf, sc):
    return _check_full(img, ov, cam, tf, sc)


def test_fp16_interpolation_error_against_the_oracle(tiny):
    import paper_1407_2074_b300 as vr
    from paper_1407_2074_b300 import vr as V

    w, vol, ov = tiny
    r = _build(vol, 16)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    img = _render(r, w.cameras, tf, sc, mode=V.VR_MODE_DVR | V.VR_RENDER_FP16)[0]
    err = _fp16_errors(img, ov, w.cameras[0], tf, sc)
    print(f"FP16 tiny: max {err.max():.2e} mean {err.mean():.2e}")
    r16 = _build(vol, 16, precision="fp16")  # the context-wide setting gives the same image
    assert np.array_equal(_render(r16, w.cameras, tf, sc)[0], img)


def test_fp16_medium_spim_error():
    from paper_1407_2074_b300 import vr as V

    dims = (192, 160, 96)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 160, seed=2)
    vol = spec.volume()
    ov = oracle_dense(vol, 16, tau=3277)
    r = _build(vol, 16, tau=3277)
    cam = S.orbit_camera(dims, 2.0 * 192, 20.0, 20.0, 320, 180, lod_error_px=2.5)
    tf, sc = S.make_tf([11, 12, 13]), [1.0, 1.0, 1.0]
    tf[..., 3] *= 3.0
    img32 = _render(r, [cam], tf, sc)[0]
    img16 = _render(r, [cam], tf, sc, mode=V.VR_MODE_DVR | V.VR_RENDER_FP16)[0]
    e32 = _fp16_errors(img32, ov, cam, tf, sc)
    e16 = _fp16_errors(img16, ov, cam, tf, sc)
    print(f"medium SPIM: FP32 max {e32.max():.2e}; FP16 max {e16.max():.2e} mean {e16.mean():.2e}")


def test_graph_plan_matches_render_and_sees_updates(tiny, tmp_path, monkeypatch):
    import torch
    from paper_1407_2074_b300 import autotune
    from paper_1407_2074_b300 import vr as V

    w, vol, ov = tiny
    r = _build(vol, 16)
    cams = S.batch_cameras(w.dims)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    ref = _render(r, cams, tf, sc)
    plan = r.plan(cams)
    for _ in range(3):  # from the second replay on, tiles are queued by the previous replay's costs
        plan.launch()
        torch.cuda.synchronize()
        for a, b in zip(plan.images, ref):
            assert np.array_equal(a.cpu().numpy(), b)
    s_plan, rays = plan.samples()
    r.render(cams)
    assert s_plan == r.stats().last_render_samples and rays > 0
    tf2 = tf.copy()
    tf2[..., 3] *= 0.5
    r.set_transfer_functions(torch.from_numpy(tf2), torch.ones(3))
    plan.launch()
    again = _render(r, cams, tf2, sc)
    torch.cuda.synchronize()
    for a, b in zip(plan.images, again):
        assert np.array_equal(a.cpu().numpy(), b)
    plan.close()
    monkeypatch.setenv("VR_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    shape, timings = autotune.autotune(r, cams, "tiny-64cams", reps=2,
                                       candidates=[(8, 4, 256, 8), (16, 2, 128, 16), (32, 1, 64, 32)])
    assert len(timings) == 3 and (tmp_path / "tune.json").exists()
    tuned = _render(r, cams, tf2, sc)
    for a, b in zip(tuned, again):
        assert np.array_equal(a, b)
    shape2, _ = autotune.autotune(r, cams, "tiny-64cams")  # cached
    assert shape2 == shape
    p16 = r.plan(cams[:4], mode=V.VR_MODE_DVR | V.VR_RENDER_FP16)
    p16.launch()
    torch.cuda.synchronize()
    p16.close()


def _random_xf(C, seed, shift=2.5, scale=0.03, rot=0.04, centre=(32.0, 32.0, 32.0)):
    # small per-channel affine transforms about the volume centre: translation, scaling, rotation
    rng = np.random.default_rng(seed)
    out = np.zeros((C, 3, 4), np.float32)
    c = np.asarray(centre, np.float64)
    for ch in range(C):
        ang = rng.uniform(-rot, rot, size=3)
        cx, cy, cz = np.cos(ang)
        sx, sy, sz = np.sin(ang)
        Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
        Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
        Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
        A = Rz @ Ry @ Rx @ np.diag(1.0 + rng.uniform(-scale, scale, size=3))
        t = c - A @ c + rng.uniform(-shift, shift, size=3)
        out[ch, :, :3] = A
        out[ch, :, 3] = t
    return out


@pytest.mark.parametrize("tau,M", [(0, 16), (2000, 16), (600, 6)])
def test_channel_transforms_against_oracle(tiny, tau, M):
    w, vol, _ = tiny
    ov = oracle_dense(vol, M, tau=tau)
    r = _build(vol, M, tau=tau)
    xf = _random_xf(3, seed=tau + M)
    r.set_channel_transforms(xf)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    tf[..., 3] *= 3.0
    cam = dict(w.cameras[0])
    cam["lod_error_px"] = 0.6
    import torch

    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor(sc))
    img = r.render([cam])[0].cpu().numpy()
    _check_full(img, ov, cam, tf, sc, xf=xf)
    # MIP with transforms
    mip = r.render([cam], mode=1)[0].cpu().numpy()
    _check_full(mip, ov, cam, tf, sc, mode=1, xf=xf)
    # back to identity: the plain path again
    r.set_channel_transforms(None)
    plain = r.render([cam])[0].cpu().numpy()
    _check_full(plain, ov, cam, tf, sc)


def test_channel_transforms_adjoint():
    import torch
    import paper_1407_2074_b300 as vr

    w = S.tiny()
    vol = w.spec().volume()
    ov = oracle_dense(vol, 16)
    r = _build(vol, 16)
    xf = _random_xf(3, seed=5)
    r.set_channel_transforms(xf)
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = 40
    cam["ert_alpha"] = 2.0
    tf, sc = w.tf(), np.array([1.0, 0.9, 1.2], np.float32)
    r.set_transfer_functions(torch.from_numpy(tf), torch.from_numpy(sc))
    dl = np.random.default_rng(3).normal(size=(40, 40, 4)).astype(np.float32)
    dtf, dsc = r.render_backward([cam], [torch.from_numpy(dl).cuda()])
    px, py = O.image_pixels(40, 40)
    rtf, rsc = O.render_grad(ov, cam, tf, sc, (px, py), dl.reshape(-1, 4).astype(np.float64), xf=xf)
    assert np.linalg.norm(dtf.cpu().numpy() - rtf) <= 1e-3 * np.linalg.norm(rtf)
    assert np.linalg.norm(dsc.cpu().numpy() - rsc) <= 1e-3 * np.linalg.norm(rsc)


def test_cost_ordered_queue_changes_no_pixel_with_channel_transforms(tiny):
    """The per-channel-transform pass in the cost-ordered queue: three renders give the
    raster-order images and sample and ray counts bit for bit."""
    w, vol, ov = tiny
    r = _build(vol, 16)
    r.set_channel_transforms(_random_xf(3, seed=7))
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    cams = S.batch_cameras(w.dims)[:5]
    r.set_tile_order(0)
    ref = _render(r, cams, tf, sc)
    counts = (r.stats().last_render_samples, r.stats().last_render_rays)
    r.set_tile_order(1)
    for _ in range(3):
        for a, b in zip(_render(r, cams, tf, sc), ref):
            assert np.array_equal(a, b)
        assert (r.stats().last_render_samples, r.stats().last_render_rays) == counts
    r.close()
