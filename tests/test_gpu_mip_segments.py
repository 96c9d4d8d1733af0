"""MIP ray segments (vr_set_mip_segment_length): the samples of a ray split into segments marched
as separate work items, merged by the per-channel maximum.  A maximum does not round, so the image
and the sample counts must equal the whole-ray MIP bit for bit, for any segment length, across
batches and render plans; and the image must match the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import oracle_dense, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spim():
    dims = (48, 40, 36)
    vol = S.VolumeSpec(S.KIND_SPIM, dims, 3, 150, seed=3).volume()
    return dims, vol, oracle_dense(vol, 8, tau=500)


def _renderer(vol, M=8, tau=500):
    import torch
    import paper_1407_2074_b300 as vr

    Z, Y, X, C = vol.shape
    r = vr.Renderer((X, Y, Z), C, M, tau=tau)
    r.insert_block((0, 0, 0), torch.from_numpy(vol.view(np.int16)).cuda())
    return r


def _render(r, cams, mode):
    import torch

    tf = S.make_tf([11, 12, 13])
    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor([1.0, 1.2, 0.8]))
    imgs = r.render(cams, mode=mode)
    torch.cuda.synchronize()
    st = r.stats()
    return [im.cpu().numpy() for im in imgs], (st.last_render_samples, st.last_render_rays), tf


def _cam(dims, az, el, w=56, h=44):
    return S.orbit_camera(dims, 2.2 * max(dims), az, el, w, h, lod_error_px=0.6)


@pytest.mark.parametrize("kseg", [4, 13, 64])
def test_mip_segments_equal_whole_rays_and_match_the_oracle(spim, kseg):
    from paper_1407_2074_b300 import vr as V

    dims, vol, ov = spim
    r = _renderer(vol)
    cam = _cam(dims, 37.0, 24.0)
    r.set_mip_segment_length(0)
    (whole,), c0, tf = _render(r, [cam], V.VR_MODE_MIP)
    r.set_mip_segment_length(kseg)
    for _ in range(2):
        (seg,), c1, _ = _render(r, [cam], V.VR_MODE_MIP)
        assert c1 == c0
        assert np.array_equal(seg, whole)
    parity(ov, cam, tf, [1.0, 1.2, 0.8], seg.reshape(-1, 4), None, V.VR_MODE_MIP)
    _, _, samples = O.render(ov, cam, tf, [1.0, 1.2, 0.8], None, V.VR_MODE_MIP, geometry="fp32")
    assert c1[0] == int(samples.sum())
    r.close()


def test_mip_segments_in_batches_and_plans(spim):
    import torch
    from paper_1407_2074_b300 import vr as V

    dims, vol, ov = spim
    r = _renderer(vol)
    cams = [_cam(dims, 15.0 * i, 10.0 * (i % 5) - 20.0, w=24 + 8 * i, h=40 - 4 * (i % 3)) for i in range(7)]
    r.set_mip_segment_length(0)
    whole, c0, _ = _render(r, cams, V.VR_MODE_MIP)
    r.set_mip_segment_length(8)
    imgs, c1, _ = _render(r, cams, V.VR_MODE_MIP)
    assert c1 == c0 and all(np.array_equal(a, b) for a, b in zip(imgs, whole))
    plan = r.plan(cams, mode=V.VR_MODE_MIP)
    plan.launch()
    torch.cuda.synchronize()
    for a, b in zip(plan.images, whole):
        assert np.array_equal(a.cpu().numpy(), b)
    assert plan.samples() == c0
    plan.close()
    for bad in (-1, 1, 3, (1 << 24) + 1):
        with pytest.raises(V.VRError):
            r.set_mip_segment_length(bad)
    r.close()
