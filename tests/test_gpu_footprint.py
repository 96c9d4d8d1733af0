"""The roofline numerator: the algorithmic footprint the library measures on the GPU
(vr_render_footprint: distinct voxels per level read by trilinear corners, distinct node entries
read on descents) against the oracle's count of the same frame (or_render_footprint, pinned on
hand-counted rays).  Without early termination the two take the same single-precision decisions and
must agree exactly; with it, rays whose opacity crosses the threshold within rounding may stop a
sample apart."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import oracle_dense

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


def _compare(r, ov, cam, tf, sc, exact):
    import torch

    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor(sc, dtype=torch.float32))
    gvox, gnodes = r.footprint([cam])
    ovox, onodes = O.render_footprint(ov, cam, tf, sc)
    if exact:
        assert list(gvox) == list(ovox) and gnodes == onodes, (gvox, ovox, gnodes, onodes)
    else:
        for a, b in zip(gvox, ovox):
            assert abs(a - b) <= 1e-3 * max(b, 1), (gvox, ovox)
        assert abs(gnodes - onodes) <= max(2, 1e-3 * onodes), (gnodes, onodes)
    return ovox, onodes


@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_footprint_tiny(ert):
    w = S.tiny()
    vol = w.spec().volume()
    r = _renderer(vol, 16, 0)
    ov = oracle_dense(vol, 16)
    cam = dict(w.cameras[0], width=96, height=80, ert_alpha=ert)
    _compare(r, ov, cam, w.tf(), [1.0, 1.0, 1.0], exact=ert > 1.0)
    r.close()


@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_footprint_spim_with_runs_lod_and_clip(ert):
    """tau = 3277 (brick-less runs), a camera far enough that two levels are sampled (t_1 = 109,
    t_2 = 217 voxels for 90 rows at a 2-pixel error), and an oblique clip plane."""
    dims = (96, 80, 64)
    vol = S.VolumeSpec(S.KIND_SPIM, dims, 3, 60, seed=17).volume()
    r = _renderer(vol, 16, 3277)
    ov = oracle_dense(vol, 16, tau=3277)
    c = np.array([48.0, 40.0, 32.0])
    n = np.array([1.0, 0.5, 0.25]) / np.linalg.norm([1.0, 0.5, 0.25])
    cam = dict(eye=[48.0 + 60.0, 40.0 + 50.0, 32.0 - 170.0], target=c.tolist(), up=[0.0, 1.0, 0.0], fov_y_deg=45.0,
               width=120, height=90, lod_error_px=2.0, step_voxels=0.5, ert_alpha=ert,
               clip=[[*n.tolist(), float(-n @ c) + 5.0]])
    vox, _ = _compare(r, ov, cam, S.tiny().tf(), [1.0, 1.2, 0.9], exact=ert > 1.0)
    assert sum(v > 0 for v in vox) >= 2  # more than one level read
    r.close()
