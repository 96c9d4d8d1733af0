"""Out-of-core rendering: full-frame ray casting over a partial render cache (Sec. "Full-Frame
Ray-Casting"), refinement ray casting (Sec. "Refinement Ray-Casting"), the brick upload policy and
insert invalidation (Sec. "Data Transfer"), against the oracle's residency-aware render."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import RGBA_TOL, admissible_error, oracle_dense, parity

pytestmark = pytest.mark.gpu

SLOT16 = 18 ** 3 * 4 * 2  # bytes of one 16^3 brick slot with border, 3(+1) channels


def _build(vol, M, tau=0, cache_slots=0, store_on_host=False, z_hi=None):
    import torch
    import paper_1407_2074_b300 as vr

    Z, Y, X, C = vol.shape
    slot = (M + 2) ** 3 * (4 if C >= 3 else C) * 2
    r = vr.Renderer((X, Y, Z), C, M, tau=tau, cache_capacity_bytes=cache_slots * slot, store_on_host=store_on_host)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(Z if z_hi is None else z_hi):
        r.insert_slice(z, dev[z])
    return r


def _set_tf(r, tf, sc):
    import torch

    r.set_transfer_functions(torch.from_numpy(tf), torch.tensor(sc, dtype=torch.float32))


def _render(r, cam, mode=0):
    import torch

    img = r.render([cam], mode=mode)[0]
    torch.cuda.synchronize()
    return img.cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    w = S.tiny()
    vol = w.spec().volume()
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = 64
    cam["lod_error_px"] = 0.5
    return w, vol, cam


@pytest.mark.parametrize("tau", [0, 2000])
def test_full_frame_matches_oracle_for_the_same_residency(tiny, tau):
    w, vol, cam = tiny
    ov = oracle_dense(vol, 16, tau=tau)
    r = _build(vol, 16, tau=tau, cache_slots=30)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    _set_tf(r, tf, sc)
    for step in range(4):
        res, _, _ = r.cache_read()
        img = _render(r, cam)
        _, used, req = r.cache_read()
        nc, cand, _, oused, oreq = O.render_cache(ov, cam, tf, sc, res)
        assert admissible_error(img.reshape(-1, 4), nc, cand).max() <= RGBA_TOL, step
        assert np.array_equal(used, oused) and np.array_equal(req, oreq), step
        rep = r.cache_update(max_uploads=9)
        assert rep["resident"] <= 30 and rep["uploaded"] <= 9
    # MIP over the cache as well
    res, _, _ = r.cache_read()
    mip = _render(r, cam, mode=1)
    nc, cand, _, _, _ = O.render_cache(ov, cam, tf, sc, res, mode=1)
    assert admissible_error(mip.reshape(-1, 4), nc, cand).max() <= RGBA_TOL


def test_root_only_equals_coarsest_level_and_load_hook(tiny):
    w, vol, cam = tiny
    ov = oracle_dense(vol, 16)
    r = _build(vol, 16, cache_slots=8)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    _set_tf(r, tf, sc)
    root = O.node_index(ov, ov.N, 0, 0, 0)
    r.cache_load([root])
    res, _, _ = r.cache_read()
    assert res.sum() == 1 and res[root] == 1
    img = _render(r, cam)
    nc, cand, _, _, _ = O.render_cache(ov, cam, tf, sc, res)
    assert admissible_error(img.reshape(-1, 4), nc, cand).max() <= RGBA_TOL


def test_full_frame_converges_to_the_full_quality_render(tiny):
    w, vol, cam = tiny
    ov = oracle_dense(vol, 16)
    r = _build(vol, 16, cache_slots=73)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    _set_tf(r, tf, sc)
    for _ in range(12):
        img = _render(r, cam)
        rep = r.cache_update()
        if rep["requested"] == 0:
            break
    assert rep["requested"] == 0
    parity(ov, cam, tf, sc, img.reshape(-1, 4))


@pytest.mark.parametrize("store_on_host", [False, True])
def test_refinement_with_a_small_cache(tiny, store_on_host):
    w, vol, cam = tiny
    ov = oracle_dense(vol, 16)
    r = _build(vol, 16, cache_slots=6, store_on_host=store_on_host)
    for L in range(ov.N + 1):  # construction into a host-resident store is unchanged
        assert np.array_equal(r.read_level(L), ov.level(L))
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    _set_tf(r, tf, sc)
    ses = r.refine(cam)
    passes, total = 0, 0
    while True:
        pending, samples = ses.pass_()
        passes += 1
        total += samples
        if pending == 0:
            break
        r.cache_update(refinement=True)
        assert passes < 500
    import torch

    torch.cuda.synchronize()
    img = ses.image.cpu().numpy()
    ses.close()
    assert passes > 2
    osamples = parity(ov, cam, tf, sc, img.reshape(-1, 4))["samples"]
    assert abs(total - int(osamples.sum())) <= 0.001 * osamples.sum()


def test_insert_drops_stale_cached_bricks(tiny):
    w, vol, cam = tiny
    r = _build(vol, 16, cache_slots=73)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    _set_tf(r, tf, sc)
    ov = oracle_dense(vol, 16)
    r.cache_load(np.arange(O.node_count(ov)))
    res, _, _ = r.cache_read()
    assert res.sum() == 73
    new = vol.copy()
    new[20] = 65535 - vol[20]  # rewrite slice 20
    r.insert_slice(20, new[20])
    res2, _, _ = r.cache_read()
    # bricks whose slot covers z = 20: level-0 z-brick 1 (interior), level 1 brick 0, the root
    assert res2.sum() < 73
    for (L, k) in ((0, 1), (1, 0), (2, 0)):
        g = ov.geom
        for j in range(g.nb[L][1]):
            for i in range(g.nb[L][0]):
                assert res2[O.node_index(ov, L, i, j, k)] == 0
    img = _render(r, cam)
    ov2 = oracle_dense(new, 16)
    nc, cand, _, _, _ = O.render_cache(ov2, cam, tf, sc, res2)
    assert admissible_error(img.reshape(-1, 4), nc, cand).max() <= RGBA_TOL


def test_medium_spim_out_of_core():
    dims = (160, 128, 96)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 120, seed=8)
    vol = spec.volume()
    ov = oracle_dense(vol, 16, tau=3277)
    r = _build(vol, 16, tau=3277, cache_slots=40)
    cam = S.orbit_camera(dims, 1.8 * 160, 40.0, 25.0, 160, 120, lod_error_px=1.5)
    tf, sc = S.make_tf([11, 12, 13]), [1.0, 1.0, 1.0]
    tf[..., 3] *= 3.0
    _set_tf(r, tf, sc)
    for _ in range(3):
        res, _, _ = r.cache_read()
        img = _render(r, cam)
        _, used, req = r.cache_read()
        nc, cand, _, oused, oreq = O.render_cache(ov, cam, tf, sc, res)
        assert admissible_error(img.reshape(-1, 4), nc, cand).max() <= RGBA_TOL
        assert np.array_equal(used, oused) and np.array_equal(req, oreq)
        r.cache_update(max_uploads=16)
    ses = r.refine(cam)
    for _ in range(400):
        pending, _ = ses.pass_()
        if pending == 0:
            break
        r.cache_update(refinement=True)
    assert pending == 0
    import torch

    torch.cuda.synchronize()
    parity(ov, cam, tf, sc, ses.image.cpu().numpy().reshape(-1, 4))
    ses.close()


def test_cost_ordered_queue_changes_no_pixel_of_a_cache_pass(tiny):
    """The render-cache pass takes its tiles from the cost-ordered queue as well: three renders in
    that order give the raster-order images, sample and ray counts and used/requested flags bit for
    bit, and a render of another tile grid in between does not disturb the order of this one."""
    w, vol, cam = tiny
    r = _build(vol, 16, cache_slots=30)
    tf, sc = w.tf(), [1.0, 1.0, 1.0]
    _set_tf(r, tf, sc)
    r.cache_update(max_uploads=12)
    cams = [cam, dict(cam, width=57, height=33)]  # a ragged second view
    r.set_tile_order(0)
    import torch

    def run(cs):
        imgs = r.render(cs)
        torch.cuda.synchronize()
        st = r.stats()
        _, used, req = r.cache_read()
        return [im.cpu().numpy() for im in imgs], (st.last_render_samples, st.last_render_rays), used, req

    ref, counts, used0, req0 = run(cams)
    other = dict(cam, width=40, height=24)
    r.set_tile_order(1)
    for i in range(3):
        imgs, cnt, used, req = run(cams)
        for a, b in zip(imgs, ref):
            assert np.array_equal(a, b), i
        assert cnt == counts, i
        if i < 2:  # the flags accumulate until the next cache update: compare before `other` adds its own
            assert np.array_equal(used, used0) and np.array_equal(req, req0), i
        if i == 1:
            run([other])  # another grid between two passes of the same grid
    r.close()
