"""Pins of the oracle's render (Algorithm 1 and Sec. "Basic Ray-Casting") against closed forms,
hand-computed values and invariants.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cam1(eye=(32.0, 32.0, -96.0), target=(32.0, 32.0, 32.0), up=(0.0, 1.0, 0.0), W=1, H=1, eps=1.0, ert=2.0,
         step=0.5, clip=()):
    return S.camera(eye, target, up, W, H, fov_y_deg=45.0, lod_error_px=eps, step_voxels=step, ert_alpha=ert,
                    clip=clip)


def const_tf(rgb, alpha, C=1):
    t = np.zeros((C, 256, 4), dtype=np.float32)
    t[..., 0], t[..., 1], t[..., 2], t[..., 3] = rgb[0], rgb[1], rgb[2], alpha
    return t


def dense(block, M=16, bg=0, tau=0):
    Z, Y, X, C = block.shape
    v = O.DenseVolume((X, Y, Z), C, M, bg, tau)
    v.insert((0, 0, 0), block)
    v.build(threads=2)
    return v


def px1(vol, cam, tf, scale=None, mode=0):
    C = tf.shape[0]
    nc, cand, samples = O.render(vol, cam, tf, scale if scale is not None else [1.0] * C, ([0], [0]), mode, 1)
    return cand[0, 0], int(samples[0]), int(nc[0])


SIG = 0.05
RGB = (0.2, 0.5, 0.9)


@pytest.fixture(scope="module")
def const_vol():
    return dense(np.full((64, 64, 64, 1), 30000, dtype=np.uint16))


@pytest.mark.parametrize("eye_z,length", [(-96.0, 64.0), (np.float32(10.3), 64.0 - float(np.float32(10.3)))])
def test_constant_slab_opacity(const_vol, eye_z, length):
    # emission-absorption of a constant medium: A = 1 - exp(-sigma L) for any thickness L (the
    # partial last segment makes the sum of segment lengths equal to L), C = rgb * A.
    tf = const_tf(RGB, 1.0 - math.exp(-SIG))
    rgba, _, _ = px1(const_vol, cam1(eye=(32.0, 32.0, float(eye_z))), tf)
    A = 1.0 - math.exp(-SIG * length)
    assert abs(rgba[3] - A) < 1e-6
    assert np.allclose(rgba[:3], np.array(RGB) * A, atol=1e-6)


@pytest.mark.parametrize("plane,length", [((0.0, 0.0, -1.0, 40.0), 40.0), ((0.0, 0.0, 1.0, -25.5), 38.5)])
def test_clip_plane_opacity(const_vol, plane, length):
    # Only the part of the ray inside the half-space n.p + d >= 0 is integrated.
    tf = const_tf(RGB, 1.0 - math.exp(-SIG))
    rgba, _, _ = px1(const_vol, cam1(clip=[plane]), tf)
    assert abs(rgba[3] - (1.0 - math.exp(-SIG * length))) < 1e-6


def test_fully_clipped_or_missed_ray_is_empty(const_vol):
    tf = const_tf(RGB, 0.5)
    rgba, samples, _ = px1(const_vol, cam1(clip=[(0.0, 0.0, 1.0, -100.0)]), tf)
    assert samples == 0 and not rgba.any()
    rgba, samples, _ = px1(const_vol, cam1(eye=(100.0, 32.0, -96.0), target=(100.0, 32.0, 32.0)), tf)
    assert samples == 0 and not rgba.any()


def test_identical_channels_equal_one_denser_channel():
    # C identical channels composited inside the sample loop act as one channel with
    # alpha' = 1 - (1 - alpha)^C: A = 1 - exp(-C sigma L), C_rgb = rgb * A.
    v = dense(np.full((64, 64, 64, 3), 30000, dtype=np.uint16))
    tf = const_tf(RGB, 1.0 - math.exp(-SIG), C=3)
    rgba, _, _ = px1(v, cam1(), tf)
    A = 1.0 - math.exp(-3 * SIG * 64.0)
    assert abs(rgba[3] - A) < 1e-6 and np.allclose(rgba[:3], np.array(RGB) * A, atol=1e-6)


def test_channel_order_inside_each_sample():
    # Two channels, red then green, composited per sample in channel order (accumulation-level
    # intermixing, Alg. 1): over n equal samples with q = (1-a0)(1-a1),
    # red = a0 (1 - q^n)/(1 - q), green = (1 - a0) a1 (1 - q^n)/(1 - q), A = 1 - q^n.
    v = dense(np.full((64, 64, 64, 2), 30000, dtype=np.uint16))
    al0, al1 = 0.06, 0.03
    tf = np.zeros((2, 256, 4), dtype=np.float32)
    tf[0, :, 0], tf[0, :, 3] = 1.0, al0
    tf[1, :, 1], tf[1, :, 3] = 1.0, al1
    rgba, samples, _ = px1(v, cam1(), tf)
    n = 128
    assert samples == n
    a0, a1 = 1 - (1 - float(np.float32(al0))) ** 0.5, 1 - (1 - float(np.float32(al1))) ** 0.5
    q = (1 - a0) * (1 - a1)
    geo = (1 - q ** n) / (1 - q)
    assert abs(rgba[0] - a0 * geo) < 1e-9 and abs(rgba[1] - (1 - a0) * a1 * geo) < 1e-9
    assert abs(rgba[3] - (1 - q ** n)) < 1e-9 and rgba[2] == 0.0


def test_early_ray_termination_index(const_vol):
    # alpha 0.1 per voxel at step 0.5: A_n = 1 - 0.9^(n/2) first reaches 0.99 at n = 88.
    tf = const_tf((1.0, 1.0, 1.0), 0.1)
    rgba, samples, _ = px1(const_vol, cam1(ert=0.99), tf)
    a32 = float(np.float32(0.1))
    assert samples == 88 and abs(rgba[3] - (1 - (1 - a32) ** 44)) < 1e-9
    # opaque limit: alpha clamps to 1 - 1e-6, one sample saturates A = 1 - 1e-3 >= 0.99
    rgba, samples, _ = px1(const_vol, cam1(ert=0.99), const_tf((1.0, 1.0, 1.0), 1.0))
    assert samples == 1 and abs(rgba[3] - (1 - 1e-3)) < 1e-9


def test_ert_band_lists_admissible_stops(const_vol):
    # alpha chosen so that A crosses 0.99 inside the +-2e-4 band: more than one admissible state.
    n = 40
    a = 1 - 0.01 ** (1.0 / n)  # A_n = 0.99 exactly at sample n
    alpha = 1 - (1 - a) ** 2
    rgba, samples, nc = px1(const_vol, cam1(ert=0.99), const_tf((1.0, 1.0, 1.0), alpha))
    assert nc >= 2
    nc_, cand, _ = O.render(const_vol, cam1(ert=0.99), const_tf((1.0, 1.0, 1.0), alpha), [1.0], ([0], [0]), 0, 1)
    As = sorted(cand[0, : nc_[0], 3])
    assert As[0] >= 0.99 - 2e-4 - 1e-6 and As[-1] <= 0.99 + 2e-4 + 0.05


def test_homogeneous_root_renders_its_average():
    # V0[z] = 1000 + z (range 63).  Level 1 = 1000 + 2j + 1 (round half up), level 2 = 1000 + 4i + 2,
    # so the root brick's AVG is 1032.  With tau = 64 the whole tree is one homogeneous subtree
    # and every sample reads the AVG (Alg. 1 lines 7-8): with an identity colour ramp, constant
    # alpha 0.05 and x = I / 2048, C_red = (1032/2048) * A, A = 1 - 0.95^64.
    blk = np.zeros((64, 64, 64, 1), dtype=np.uint16)
    blk[..., 0] = (1000 + np.arange(64))[:, None, None]
    tf = np.zeros((1, 256, 4), dtype=np.float32)
    tf[0, :, 0] = np.arange(256) / 255.0
    tf[0, :, 3] = 0.05
    scale = [65535.0 / 2048.0]
    vh = dense(blk, tau=64)
    assert vh.node(2, 0, 0, 0).avg[0] == 1032 and not vh.node(2, 0, 0, 0).has_children
    cam = cam1(eps=1e-3)
    rgba, _, _ = px1(vh, cam, tf, scale)
    a32 = float(np.float32(0.05))
    A = 1 - (1 - a32) ** 64
    x = float(np.float32(65535.0 / 2048.0)) * 1032 / 65535.0
    assert abs(rgba[3] - A) < 1e-9 and abs(rgba[0] - x * A) < 1e-6
    v0 = dense(blk, tau=0)  # without pruning the ramp is sampled and the colour differs
    rgba0, _, _ = px1(v0, cam, tf, scale)
    assert abs(rgba0[0] - rgba[0]) > 1e-3


def test_untouched_nodes_render_background():
    # Only slices z < 32 inserted (value 20000, background 0).  Level-0 nodes above z = 32 are
    # untouched and hold only the background (Sec. "Incremental Construction"), so along +z
    # the samples z = 0 .. 31.5 (64 of them) see alpha 0.08 and the rest alpha 0.
    X = 64
    v = O.DenseVolume((X, X, X), 1, 16, 0, 0)
    v.insert((0, 0, 0), np.full((32, X, X, 1), 20000, dtype=np.uint16))
    v.build(threads=2)
    tf = np.zeros((1, 256, 4), dtype=np.float32)
    tf[0, :, :3] = 1.0
    tf[0, 1:, 3] = 0.08
    rgba, _, _ = px1(v, cam1(eps=1e-3), tf)
    a32 = float(np.float32(0.08))
    assert abs(rgba[3] - (1 - (1 - a32) ** 32)) < 1e-9


def test_far_camera_samples_the_coarsest_level():
    # Checkerboard 1000/3000 at level 0 averages to 2000 on every coarser level.  A one-pixel
    # camera has a pixel footprint >> 1 voxel, so every sample uses level N: C_red = x A with
    # x = 2000/4096.  A near camera (eps tiny) samples level 0 off the voxel lattice and differs.
    zz, yy, xx = np.meshgrid(np.arange(64), np.arange(64), np.arange(64), indexing="ij")
    blk = np.where((xx + yy + zz) % 2 == 0, 1000, 3000).astype(np.uint16)[..., None]
    v = dense(blk)
    tf = np.zeros((1, 256, 4), dtype=np.float32)
    tf[0, :, 0] = np.arange(256) / 255.0
    tf[0, :, 3] = 0.05
    scale = [65535.0 / 4096.0]
    eye = (32.25, 32.25, -96.0)
    far, _, _ = px1(v, cam1(eye=eye, target=(32.25, 32.25, 32.0), eps=1.0), tf, scale)
    a32 = float(np.float32(0.05))
    A = 1 - (1 - a32) ** 64
    x = float(np.float32(65535.0 / 4096.0)) * 2000 / 65535.0
    assert abs(far[0] - x * A) < 1e-6
    near, _, _ = px1(v, cam1(eye=eye, target=(32.25, 32.25, 32.0), eps=1e-3), tf, scale)
    assert abs(near[0] - far[0]) > 1e-3


def test_lod_thresholds_match_projected_pixel_footprint():
    # The level L is used from the distance where a level-L voxel (2^L level-0 voxels) projects to
    # eps pixels (Sec. "Basic Ray-Casting", optimal LOD).  Footprint measured from the angle between
    # two vertically adjacent pixel rays at the image centre.
    g = O.geom((2048, 2048, 1024), 3, 32)
    for eps in (1.0, 2.0):
        cam = S.camera((1024.0, 1024.0, -4000.0), (1024.0, 1024.0, 512.0), (0.0, 1.0, 0.0), 1920, 1080,
                       lod_error_px=eps)
        tl = O.lod_thresholds(g, cam)
        _, d1, _, _ = O.ray(g, cam, 960, 539)
        _, d2, _, _ = O.ray(g, cam, 960, 540)
        ang = 2.0 * math.asin(float(np.linalg.norm(d1.astype(np.float64) - d2.astype(np.float64))) / 2.0)
        for L in range(1, g.N + 1):
            footprint = tl[L] * ang
            assert abs(2 ** L / (eps * footprint) - 1.0) < 2e-3


def test_camera_conventions():
    # pinhole: pixel (0,0) is top-left; x to the right (f x up), y up, square pixels.
    W, H = 64, 48
    cam = S.camera((0.0, 0.0, -100.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), W, H, fov_y_deg=60.0)
    g = O.geom((10, 10, 10), 1, 2)
    _, d, _, _ = O.ray(g, cam, 0, 0)
    f, r, u = np.array([0, 0, 1.0]), np.array([-1.0, 0, 0]), np.array([0, 1.0, 0])
    th = math.tan(math.radians(30.0))
    assert abs(d @ u / (d @ f) - (1 - 1 / H) * th) < 1e-6
    assert abs(d @ r / (d @ f) - (1 / W - 1) * th * W / H) < 1e-6
    _, dm, _, _ = O.ray(g, cam, W - 1, H - 1)
    assert np.allclose(dm @ r, -(d @ r), atol=1e-6) and np.allclose(dm @ u, -(d @ u), atol=1e-6)


def test_trilinear_hand_computed():
    vals = {}
    for line in open(os.path.join(GOLDEN, "trilinear_cell.txt")):
        if line.strip() and line[0] != "#":
            k, *rest = line.split()
            vals[k] = [float(x) for x in rest]
    blk = np.zeros((2, 2, 2, 1), dtype=np.uint16)
    blk[0, 1, 1, 0], blk[1, 1, 1, 0] = 100, 1000
    v = dense(blk, M=2)
    for pk, vk in (("p", "value"), ("p2", "value2"), ("p3", "value3")):
        assert abs(O.sample_trilinear(v, 0, vals[pk], 0) - vals[vk][0]) < 1e-9


def test_trilinear_reproduces_linear_fields():
    # trilinear interpolation is exact on a*x + b*y + c*z + d (at any level, inside the centres)
    zz, yy, xx = np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij")
    blk = (100 + 3 * xx + 5 * yy + 7 * zz).astype(np.uint16)[..., None]
    v = dense(blk, M=8)
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = rng.uniform(0.5, 31.5, size=3).astype(np.float32)
        q = p.astype(np.float64)
        ex = 100 + 3 * (q[0] - 0.5) + 5 * (q[1] - 0.5) + 7 * (q[2] - 0.5)
        assert abs(O.sample_trilinear(v, 0, p, 0) - ex) < 1e-6


def test_transfer_function_lookup():
    ramp = np.zeros((256, 4), dtype=np.float32)
    ramp[:] = (np.arange(256) / 255.0)[:, None]
    for I in (0.0, 1.0, 12345.6, 40000.0, 65535.0):
        assert np.allclose(O.tf_eval(ramp, 1.0, I), I / 65535.0, atol=1e-7)
    assert np.allclose(O.tf_eval(ramp, 2.0, 40000.0), 1.0)  # clamp at x = 1
    hat = np.zeros((256, 4), dtype=np.float32)
    hat[100] = 1.0
    assert np.allclose(O.tf_eval(hat, 1.0, 100.5 / 255 * 65535), 0.5)
    assert np.allclose(O.tf_eval(hat, 1.0, 99.25 / 255 * 65535), 0.25)
    const = np.full((256, 4), 0.3, dtype=np.float32)
    assert np.allclose(O.tf_eval(const, 1.0, 777.0), float(np.float32(0.3)))


def test_mip_is_the_maximum_then_one_lookup():
    # MIP (Sec. "Integration into Voreen", Table 1): the maximum sampled intensity along the
    # ray, one transfer-function lookup.  On V0[z] = 1000 + 100 z the maximum is the last sample
    # (z = 63.5 at level 0, value 7300): C_red = alpha * x, A = alpha for one channel.
    blk = np.zeros((64, 64, 64, 1), dtype=np.uint16)
    blk[..., 0] = (1000 + 100 * np.arange(64))[:, None, None]
    v = dense(blk)
    tf = np.zeros((1, 256, 4), dtype=np.float32)
    tf[0, :, 0] = np.arange(256) / 255.0
    tf[0, :, 3] = 0.05
    rgba, _, _ = px1(v, cam1(eps=1e-3), tf, [1.0], mode=1)
    a32 = float(np.float32(0.05))
    assert abs(rgba[3] - a32) < 1e-9 and abs(rgba[0] - a32 * 7300 / 65535.0) < 1e-7


def _identity_xf(C):
    m = np.zeros((C, 3, 4), dtype=np.float32)
    m[:, 0, 0] = m[:, 1, 1] = m[:, 2, 2] = 1.0
    return m


def test_channel_transform_identity_changes_nothing():
    w = S.tiny()
    vol = w.spec().volume()
    v = dense(vol)
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = 32
    a = O.render(v, cam, w.tf(), [1, 1, 1], None, 0, 2)[1]
    b = O.render(v, cam, w.tf(), [1, 1, 1], None, 0, 2, xf=_identity_xf(3))[1]
    assert np.array_equal(a, b)


def test_channel_translation_equals_shifted_data():
    # Sec. "Correction of Chromatic Aberration": channel 1 sampled at p + (3, 0, 0) sees the same
    # values as an unshifted render of data whose channel 1 is V'[x] = V[min(x + 3, X - 1)]
    # at level 0 without pruning (zero margins keep the clamped edges equal).
    w = S.tiny()
    vol = w.spec().volume()
    X = vol.shape[2]
    vol[:, :, :8] = 0  # zero margins: clamp-to-edge then reads equal values on both sides
    vol[:, :, X - 8:] = 0
    shifted = vol.copy()
    shifted[..., 1] = vol[:, :, np.minimum(np.arange(X) + 3, X - 1), 1]
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = 40
    cam["lod_error_px"] = 1e-3
    xf = _identity_xf(3)
    xf[1, 0, 3] = 3.0
    a = O.render_image(dense(vol), cam, w.tf(), [1, 1, 1], xf=xf)[0]
    b = O.render_image(dense(shifted), cam, w.tf(), [1, 1, 1])[0]
    assert np.abs(a - b).max() < 1e-6
    c = O.render_image(dense(vol), cam, w.tf(), [1, 1, 1])[0]
    assert np.abs(a - c).max() > 1e-3  # the transform does something


def test_full_frame_cache_semantics():
    # Sec. "Full-Frame Ray-Casting".  (1) every brick present: the plain render, nothing requested;
    # (2) only the root present: a level-0 sample falls back to its grandparent (the root, N = 2),
    # i.e. the image of a camera whose level choice is the root everywhere; every missing brick on
    # the paths is requested; (3) nothing present: a constant volume still renders its closed form
    # through the AVG values.  The cache render takes single-precision (mirrored) decisions, so the
    # plain renders it is compared with do too.
    w = S.tiny()
    vol = w.spec().volume()
    v = dense(vol)
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = 32
    cam["lod_error_px"] = 1e-3  # level 0 everywhere
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    nn = O.node_count(v)
    root = O.node_index(v, v.N, 0, 0, 0)
    allres = np.ones(nn, np.uint8)
    nc, cand, _, used, req = O.render_cache(v, cam, tf, sc, allres)
    ref = O.render(v, cam, tf, sc, None, 0, geometry="fp32")[1]
    assert np.array_equal(cand, ref) and req.sum() == 0 and used.sum() > 0 and used[root] == 0
    onlyroot = np.zeros(nn, np.uint8)
    onlyroot[root] = 1
    _, cand2, _, used2, req2 = O.render_cache(v, cam, tf, sc, onlyroot)
    far = dict(cam)
    far["lod_error_px"] = 1e6  # level N everywhere
    ref2 = O.render(v, far, tf, sc, None, 0, geometry="fp32")[1]
    assert np.abs(cand2[:, 0] - ref2[:, 0]).max() < 1e-12
    assert used2[root] == 1 and used2.sum() == 1
    lvl1 = [O.node_index(v, 1, i, j, k) for i in range(2) for j in range(2) for k in range(2)]
    assert req2[lvl1].sum() > 0 and req2[:64].sum() > 0 and req2[root] == 0
    const = dense(np.full((64, 64, 64, 1), 30000, dtype=np.uint16))
    tf1 = const_tf(RGB, 1.0 - math.exp(-SIG))
    c1 = cam1()
    _, cc, _, _, rq = O.render_cache(const, c1, tf1, [1.0], np.zeros(O.node_count(const), np.uint8), ([0], [0]))
    assert abs(cc[0, 0, 3] - (1.0 - math.exp(-SIG * 64.0))) < 1e-6 and rq.sum() > 0


# ---- double-precision geometry and its knife-edge decisions (A16 reading) ----

def test_fp64_geometry_equals_fp32_geometry_away_from_knife_edges():
    """The two geometry modes compute the same rays up to rounding: wherever the double-precision
    march met no knife-edge decision, its result equals the single-precision one to within what a
    sample-position difference of ~1e-4 voxel can change; and knife edges are rare."""
    w = S.tiny()
    v = dense(w.spec().volume(), M=16)
    for cam in (S.orbit_camera(w.dims, 128.0, 40.0, 25.0, 96, 80, lod_error_px=3.0),
                S.orbit_camera(w.dims, 100.0, 200.0, -30.0, 96, 80, lod_error_px=0.3,
                               clip=[S.centre_plane(w.dims, (1.0, 0.5, 0.25))])):
        _, c32, _ = O.render(v, cam, w.tf(), [1.0, 1.0, 1.0], None, 0, geometry="fp32")
        chk = O.check(v, cam, w.tf(), [1.0, 1.0, 1.0], c32[:, 0, :].astype(np.float32))
        calm = chk["flagged"] == 0
        assert calm.mean() > 0.95
        assert np.abs(chk["rgba"][calm] - c32[calm, 0, :]).max() < 2e-5
        assert chk["err"].max() < 2e-3  # the single-precision march is one of the admissible results


def _lod_edge_camera(eps):
    # one pixel looking down +z through the tiny volume from z = -96: sample k at t = 96 + k/2; the
    # level-1 threshold t_1 = H / (eps tan(22.5 deg)) equals t = 108 (sample 24) when eps = eps0
    return S.camera((20.3, 40.1, -96.0), (20.3, 40.1, 32.0), (0.0, 1.0, 0.0), 1, 1, fov_y_deg=45.0,
                    lod_error_px=eps, step_voxels=0.5, ert_alpha=2.0)


def test_knife_edge_at_a_level_threshold_admits_both_levels():
    """A sample exactly at t_L: both the finer and the coarser level are correct.  The two results
    are those of cameras whose threshold sits just before / just after that sample (every other
    sample is 0.5 away from t_L), they differ, and the check admits each of them exactly."""
    w = S.tiny()
    v = dense(w.spec().volume(), M=16)
    tf = w.tf()
    eps0 = 1.0 / (108.0 * math.tan(math.radians(22.5)))
    lo = O.render(v, _lod_edge_camera(eps0 * (1 + 1e-3)), tf, [1, 1, 1], ([0], [0]))[1][0, 0]  # sample 24: level 1
    hi = O.render(v, _lod_edge_camera(eps0 * (1 - 1e-3)), tf, [1, 1, 1], ([0], [0]))[1][0, 0]  # sample 24: level 0
    assert np.abs(lo - hi).max() > 4e-4
    cam = _lod_edge_camera(eps0)
    for target in (lo, hi):
        r = O.check(v, cam, tf, [1, 1, 1], target.astype(np.float32)[None], ([0], [0]))
        assert r["flagged"][0] == 1 and r["variants"][0] == 2 and r["unresolved"][0] == 0
        assert r["err"][0] < 1e-6
    # a threshold half a step away from every sample is no knife edge
    r = O.check(v, _lod_edge_camera(1.0 / (108.25 * math.tan(math.radians(22.5)))), tf, [1, 1, 1],
                hi.astype(np.float32)[None], ([0], [0]))
    assert r["flagged"][0] == 0 and r["variants"][0] == 1


def _split_volume():
    # x < 32 constant (a homogeneous level-1 subtree with AVG 5000 and no brick), x >= 32 the blobs
    blob = S.tiny().spec().volume()
    vol = blob.copy()
    vol[:, :, :32, :] = 5000
    return dense(vol, M=16, tau=50)


def test_knife_edge_at_a_split_plane_admits_both_children():
    """A sample on the split plane x = 32 between a brick-less node (AVG) and a brick node: either
    child is correct.  The ray direction is (0.6, 0, 0.8); it crosses x = 32 at its third sample.
    Shifting the eye by -+1e-3 voxel puts that sample on one side or the other."""
    v = _split_volume()
    tf = S.tiny().tf()
    tf[..., 3] = np.minimum(1.0, tf[..., 3] * 8.0)

    def cam(dx):
        e = (1.4 + dx, 20.25, -40.0)
        return S.camera(e, (e[0] + 60.0, e[1], e[2] + 80.0), (0.0, 1.0, 0.0), 1, 1, lod_error_px=1e-3,
                        step_voxels=0.5, ert_alpha=2.0)

    left = O.render(v, cam(-1e-3), tf, [1, 1, 1], ([0], [0]))[1][0, 0]
    right = O.render(v, cam(+1e-3), tf, [1, 1, 1], ([0], [0]))[1][0, 0]
    assert np.abs(left - right).max() > 1e-3
    for target in (left, right):
        r = O.check(v, cam(0.0), tf, [1, 1, 1], target.astype(np.float32)[None], ([0], [0]))
        assert r["flagged"][0] == 1 and r["variants"][0] == 2
        assert r["err"][0] < 1e-4  # the shifted cameras move every other sample by 1e-3 voxel


def test_ray_along_a_split_plane_is_unresolved():
    """A ray inside the split plane x = 32 meets a knife edge at every sample of that stretch: more
    than the enumerated decisions, so the ray is reported unresolved."""
    v = _split_volume()
    tf = S.tiny().tf()
    cam = S.camera((32.0, 20.25, -40.0), (32.0, 20.25, 32.0), (0.0, 1.0, 0.0), 1, 1, lod_error_px=1e-3,
                   step_voxels=0.5, ert_alpha=2.0)
    nat = O.render(v, cam, tf, [1, 1, 1], ([0], [0]))[1][0, 0]
    r = O.check(v, cam, tf, [1, 1, 1], nat.astype(np.float32)[None], ([0], [0]))
    assert r["unresolved"][0] == 1 and r["flagged"][0] > O.MAXFLAG and r["variants"][0] == 2 ** O.MAXFLAG
