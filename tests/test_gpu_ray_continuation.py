"""Ray continuation: once the tile queue of a DVR render has run dry, lanes whose rays still have
far to go record their state and a second launch finishes each such ray with a group of 1 to 32
lanes.  Every lane of a group composites the group's shaded samples in order, and runs of equal
samples through brick-less nodes start at the same samples as in the one-lane march, so images and
sample counts must equal the render without continuation bit for bit: for every group width, FP32
and FP16 interpolation, with and without early termination, with a clip plane, and on a volume with
brick-less runs (tau = 3277) as well as one without (tau = 0)."""
import numpy as np
import pytest

from synth import synth as S
from tests.helpers import oracle_dense, parity

pytestmark = pytest.mark.gpu


def _renderer(vol, M, tau):
    import torch
    import paper_1407_2074_b300 as vr

    Z, Y, X, C = vol.shape
    r = vr.Renderer((X, Y, Z), C, M, tau=tau)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(Z):
        r.insert_slice(z, dev[z])
    return r


def _frame(r, cams, mode=0):
    import torch

    imgs = r.render(cams, mode=mode)
    torch.cuda.synchronize()
    st = r.stats()
    return [im.cpu().numpy() for im in imgs], (st.last_render_samples, st.last_render_rays), st.last_render_continued


@pytest.fixture(scope="module")
def spim():
    """A SPIM-like volume: with tau = 3277 brick-less background and tissue bricks."""
    dims = (96, 80, 64)
    return dims, S.VolumeSpec(S.KIND_SPIM, dims, 3, 60, seed=17).volume()


def _cameras(dims):
    X, Y, Z = dims
    c = np.array([X / 2, Y / 2, Z / 2], np.float32)
    base = dict(target=c.tolist(), up=[0.0, 1.0, 0.0], fov_y_deg=45.0, width=72, height=56, lod_error_px=1.0,
                step_voxels=0.5, ert_alpha=0.99, clip=[])
    cams = []
    for i, (az, el, ert) in enumerate(((20.0, 15.0, 0.99), (140.0, -30.0, 2.0), (250.0, 40.0, 0.99))):
        a, e = np.radians(az), np.radians(el)
        eye = c + 1.6 * max(dims) * np.array([np.cos(e) * np.sin(a), np.sin(e), np.cos(e) * np.cos(a)], np.float32)
        cam = dict(base, eye=eye.tolist(), ert_alpha=ert)
        if i == 2:  # an oblique clip plane through the centre
            n = np.array([1.0, 0.5, 0.25]) / np.linalg.norm([1.0, 0.5, 0.25])
            cam["clip"] = [[*n.tolist(), float(-n @ c)]]
        cams.append(cam)
    return cams


@pytest.mark.parametrize("tau", [3277, 0])
@pytest.mark.parametrize("fp16", [False, True])
def test_continued_rays_equal_one_lane(spim, tau, fp16):
    import torch
    from paper_1407_2074_b300 import vr as V

    dims, vol = spim
    r = _renderer(vol, 16, tau)
    r.set_transfer_functions(torch.from_numpy(S.tiny().tf()), torch.tensor([1.0, 1.2, 0.9]))
    cams = _cameras(dims)
    mode = V.VR_MODE_DVR | (V.VR_RENDER_FP16 if fp16 else 0)
    r.set_ray_continuation(0, 0)
    ref, counts, cont = _frame(r, cams, mode)
    assert cont == 0
    for lanes in (1, 2, 4, 8, 16, 32):
        r.set_ray_continuation(lanes, 0)  # every ray still marching when the queue runs dry
        for f in range(2):  # raster order, then the cost order of the frame before
            imgs, cnt, cont = _frame(r, cams, mode)
            for a, b in zip(imgs, ref):
                assert np.array_equal(a, b), f"{lanes} lanes per ray, frame {f}"
            assert cnt == counts
            assert 0 < cont < counts[1], (lanes, f, cont)
    r.close()


def test_continued_frame_against_the_oracle(spim):
    """A continued frame on its own against the oracle's admissible results."""
    import torch

    dims, vol = spim
    r = _renderer(vol, 16, 3277)
    tf, sc = S.tiny().tf(), [1.0, 1.2, 0.9]
    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor(sc))
    r.set_ray_continuation(8, 16)
    cams = _cameras(dims)
    imgs, _, cont = _frame(r, cams)
    assert cont > 0
    ov = oracle_dense(vol, 16, tau=3277)
    for cam, img in zip(cams, imgs):
        parity(ov, cam, tf, sc, img.reshape(-1, 4))
    r.close()


def test_ray_continuation_arguments():
    import paper_1407_2074_b300 as vr
    from paper_1407_2074_b300 import vr as V

    r = vr.Renderer((16, 16, 16), 3, 8)
    for lanes, left in ((3, 0), (64, 0), (-1, 0), (8, -1)):
        with pytest.raises(V.VRError):
            r.set_ray_continuation(lanes, left)
    r.set_ray_continuation(0, 0)
    r.set_ray_continuation(32, 1 << 20)
    r.close()
