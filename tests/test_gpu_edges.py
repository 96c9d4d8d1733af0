"""Degenerate and boundary cases of the method against the oracle: single-voxel and single-slice
volumes, a tree of one node, the largest brick, nothing inserted, clip planes that remove every
ray, ragged and one-pixel images, extreme sampling steps and termination thresholds."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import oracle_dense, parity

pytestmark = pytest.mark.gpu


def _renderer(vol, M, bg=0, tau=0, insert=True):
    import torch
    import paper_1407_2074_b300 as vr

    Z, Y, X, C = vol.shape
    r = vr.Renderer((X, Y, Z), C, M, background=bg, tau=tau)
    if insert:
        r.insert_block((0, 0, 0), torch.from_numpy(vol.view(np.int16)).cuda())
    return r


def _render_check(r, ov, cam, tf, sc, mode=0):
    import torch

    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor(sc, dtype=torch.float32))
    img = r.render([cam], mode=mode)[0]
    torch.cuda.synchronize()
    img = img.cpu().numpy()
    parity(ov, cam, tf, sc, img.reshape(-1, 4), None, mode)
    _, _, samples = O.render(ov, cam, tf, sc, None, mode, geometry="fp32")  # decision for decision
    return img, samples


def _spim(dims, C=3, seed=9):
    return S.VolumeSpec(S.KIND_SPIM, dims, C, max(2, dims[0] * dims[1] * dims[2] // 400), seed=seed).volume()


def _levels_equal(r, ov):
    for L in range(ov.N + 1):
        assert np.array_equal(r.read_level(L), ov.level(L)), L


@pytest.mark.parametrize("dims,M", [((1, 1, 1), 4), ((1, 5, 3), 4), ((7, 1, 1), 4), ((2, 2, 2), 4),
                                    ((5, 3, 130), 8), ((130, 70, 40), 128)])
def test_degenerate_extents_and_the_largest_brick(dims, M):
    vol = _spim(dims)
    ov = oracle_dense(vol, M, bg=11, tau=500)
    r = _renderer(vol, M, bg=11, tau=500)
    _levels_equal(r, ov)
    X, Y, Z = dims
    if Z > 10 * max(X, Y):  # a long thin column: look down its axis
        cam = S.camera((X / 2 + 1.3, Y / 2 + 0.7, -15.0), (X / 2, Y / 2, Z / 2), (0.0, 1.0, 0.0), 40, 29,
                       lod_error_px=0.5)
    else:
        cam = S.orbit_camera(dims, 3.0 * max(dims) + 4.0, 33.0, 21.0, 40, 29, lod_error_px=0.5)
    tf = S.make_tf([11, 12, 13])
    tf[..., 3] = np.clip(tf[..., 3] * 8.0, 0.0, 1.0)
    _, samples = _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0])
    assert samples.sum() > 0
    r.close()


def test_nothing_inserted_renders_the_background_root():
    dims = (40, 30, 20)
    vol = np.full((20, 30, 40, 3), 900, np.uint16)
    ov = oracle_dense(vol, 8, bg=900, tau=0, z_hi=0)
    r = _renderer(vol, 8, bg=900, insert=False)
    _levels_equal(r, ov)
    cam = S.orbit_camera(dims, 100.0, 10.0, 10.0, 32, 32)
    tf = S.make_tf([11, 12, 13])
    img, samples = _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0])
    assert samples.sum() > 0 and img[..., 3].max() > 0.0
    r.close()


def test_clip_planes_that_remove_every_ray():
    dims = (32, 32, 32)
    vol = _spim(dims)
    ov = oracle_dense(vol, 8)
    r = _renderer(vol, 8)
    cam = S.orbit_camera(dims, 80.0, 0.0, 0.0, 24, 24)
    cam["clip"] = [(1.0, 0.0, 0.0, -40.0)]  # keeps x >= 40 only: outside the volume
    tf = S.make_tf([11, 12, 13])
    img, samples = _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0])
    assert samples.sum() == 0 and not img.any()
    assert r.stats().last_render_rays == 0
    cam["clip"] = [(1.0, 0.0, 0.0, -16.0), (-1.0, 0.0, 0.0, 15.0)]  # empty slab 16 <= x <= 15
    img, samples = _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0])
    assert samples.sum() == 0 and not img.any()
    r.close()


@pytest.mark.parametrize("w,h", [(1, 1), (33, 7), (1, 200), (200, 1)])
def test_ragged_and_one_pixel_images(w, h):
    dims = (24, 20, 16)
    vol = _spim(dims)
    ov = oracle_dense(vol, 8, tau=300)
    r = _renderer(vol, 8, tau=300)
    cam = S.camera((12.0, 10.0, -30.0), (12.0, 10.0, 8.0), (0.0, 1.0, 0.0), w, h, fov_y_deg=60.0)
    tf = S.make_tf([11, 12, 13])
    tf[..., 3] = np.clip(tf[..., 3] * 6.0, 0.0, 1.0)
    _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0])
    r.close()


@pytest.mark.parametrize("step,ert", [(4.0, 0.99), (0.05, 0.99), (0.5, 2.0), (0.5, 0.0), (1.0, 0.5)])
def test_sampling_steps_and_termination_thresholds(step, ert):
    dims = (40, 36, 30)
    vol = _spim(dims, seed=4)
    ov = oracle_dense(vol, 8, tau=2000)
    r = _renderer(vol, 8, tau=2000)
    cam = S.orbit_camera(dims, 90.0, 50.0, 30.0, 48, 40, lod_error_px=0.8)
    cam["step_voxels"] = step
    cam["ert_alpha"] = ert
    tf = S.make_tf([11, 12, 13])
    tf[..., 3] = np.clip(tf[..., 3] * 5.0, 0.0, 1.0)
    img, samples = _render_check(r, ov, cam, tf, [1.0, 1.3, 0.7])
    if ert <= 0.0:
        assert samples.max() <= 1  # every ray stops after its first sample
    r.close()


def test_everything_homogeneous_and_mip():
    from paper_1407_2074_b300 import vr as V

    dims = (36, 28, 20)
    vol = _spim(dims, seed=5)
    ov = oracle_dense(vol, 8, tau=65535)  # every brick and subtree homogeneous: the root's AVG
    r = _renderer(vol, 8, tau=65535)
    assert r.read_node(ov.N, 0, 0, 0)[0] & V.F_CHILDREN == 0
    cam = S.orbit_camera(dims, 70.0, 20.0, 15.0, 32, 30)
    tf = S.make_tf([11, 12, 13])
    _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0])
    _render_check(r, ov, cam, tf, [1.0, 1.0, 1.0], mode=V.VR_MODE_MIP)
    r.close()
