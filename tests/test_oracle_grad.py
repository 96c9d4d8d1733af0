"""Pins of the oracle's adjoint: it must be the derivative of the oracle's forward render.
Central finite differences of the forward (h = 1e-3, as the differentiable workload specifies)
against the FP64 reverse sweep.  The adjoint is the derivative at the forward's own decisions,
so the forward here takes the single-precision geometry the adjoint marches with.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S


@pytest.fixture(scope="module")
def scene():
    w = S.tiny()
    vol = w.spec().volume()
    v = O.DenseVolume(w.dims, 3, w.brick, 0, 0)
    v.insert((0, 0, 0), vol)
    v.build(threads=2)
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = 24
    cam["ert_alpha"] = 2.0  # no early termination: the loss is smooth in the tables
    rng = np.random.default_rng(7)
    px = rng.integers(4, 20, size=24).astype(np.int32)
    py = rng.integers(4, 20, size=24).astype(np.int32)
    dl = rng.normal(size=(24, 4))
    return v, cam, w.tf(), np.array([1.0, 0.9, 1.1], dtype=np.float32), (px, py), dl


def _loss(v, cam, tf, sc, pix, dl, xf=None):
    _, cand, _ = O.render(v, cam, tf, sc, pix, 0, 2, xf=xf, geometry="fp32")
    return float((cand[:, 0, :] * dl).sum())


def test_tf_gradient_matches_central_differences(scene):
    v, cam, tf, sc, pix, dl = scene
    dtf, _ = O.render_grad(v, cam, tf, sc, pix, dl, threads=2)
    # entries whose +-h step would leave [0, 1] sit on the clamp of the opacity (a kink); skip them
    ok = ((tf >= 2e-3) & (tf <= 1 - 2e-3)).ravel()
    order = [f for f in np.argsort(-np.abs(dtf).ravel()) if ok[f]]
    flat = order[:12]
    for f in flat:
        c, i, k = np.unravel_index(f, dtf.shape)
        tp, tm = tf.copy(), tf.copy()
        tp[c, i, k] += np.float32(1e-3)
        tm[c, i, k] -= np.float32(1e-3)
        h2 = float(tp[c, i, k]) - float(tm[c, i, k])
        fd = (_loss(v, cam, tp, sc, pix, dl) - _loss(v, cam, tm, sc, pix, dl)) / h2
        assert abs(fd - dtf[c, i, k]) <= 1e-4 * max(1.0, abs(dtf[c, i, k])), (c, i, k, fd, dtf[c, i, k])


def test_scale_gradient_matches_central_differences_on_smooth_tables(scene):
    # With tables that are linear in x on every entry (ramps) the render is smooth in the scale.
    v, cam, _, sc, pix, dl = scene
    tf = np.zeros((3, 256, 4), dtype=np.float32)
    g = np.arange(256) / 255.0
    tf[0] = np.stack([g, 0.5 * g, 0.2 + 0 * g, 0.08 * g], -1)
    tf[1] = np.stack([0.3 + 0 * g, g, 0.5 * g, 0.05 * g], -1)
    tf[2] = np.stack([0.5 * g, 0.2 + 0 * g, g, 0.06 * g], -1)
    _, dsc = O.render_grad(v, cam, tf, sc, pix, dl, threads=2)
    for c in range(3):
        sp, sm = sc.copy(), sc.copy()
        sp[c] += np.float32(1e-3)
        sm[c] -= np.float32(1e-3)
        h2 = float(sp[c]) - float(sm[c])
        fd = (_loss(v, cam, tf, sp, pix, dl) - _loss(v, cam, tf, sm, pix, dl)) / h2
        assert abs(fd - dsc[c]) <= 1e-4 * max(1.0, abs(dsc[c])), (c, fd, dsc[c])


def test_colour_gradient_is_exact_when_opacity_is_fixed(scene):
    # With the alpha column fixed, every pixel colour is linear in the rgb table entries, so one
    # finite difference with any step is exact: I(T + e) - I(T) = e * dI/dT.
    v, cam, tf, sc, pix, dl = scene
    dtf, _ = O.render_grad(v, cam, tf, sc, pix, dl, threads=2)
    base = _loss(v, cam, tf, sc, pix, dl)
    c, i = 1, int(np.argmax(np.abs(dtf[1, :, 0])))
    tp = tf.copy()
    tp[c, i, 0] += np.float32(0.25)
    step = float(tp[c, i, 0]) - float(tf[c, i, 0])
    assert abs((_loss(v, cam, tp, sc, pix, dl) - base) - step * dtf[c, i, 0]) < 1e-10


def _xf():
    """Non-identity per-channel affine transforms about the volume centre (rotation, anisotropic
    scale, shift), channel 0 included."""
    c = np.array([32.0, 32.0, 32.0])
    out = np.zeros((3, 3, 4), dtype=np.float32)
    for ch, (ang, s, sh) in enumerate((((0.03, -0.02, 0.05), (1.01, 0.99, 1.0), (0.7, -0.4, 0.3)),
                                       ((-0.04, 0.02, 0.01), (0.98, 1.02, 1.01), (-0.5, 0.6, -0.9)),
                                       ((0.02, 0.05, -0.03), (1.0, 1.03, 0.97), (0.2, 0.9, 1.4)))):
        cx, cy, cz = np.cos(ang)
        sx, sy, sz = np.sin(ang)
        R = (np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]]) @ np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
             @ np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]]) @ np.diag(s))
        out[ch, :, :3] = R
        out[ch, :, 3] = c - R @ c + np.array(sh)
    return out


def test_gradient_with_channel_transforms_matches_central_differences(scene):
    """or_render_grad_xf (Sec. "Correction of Chromatic Aberration": each channel samples at its
    own transformed point) against central differences of the transformed forward: table entries
    and, on ramp tables, the scales."""
    v, cam, tf, sc, pix, dl = scene
    xf = _xf()
    dtf, _ = O.render_grad(v, cam, tf, sc, pix, dl, threads=2, xf=xf)
    plain, _ = O.render_grad(v, cam, tf, sc, pix, dl, threads=2)
    assert np.abs(dtf - plain).max() > 1e-3 * np.abs(plain).max()  # the transforms do change the gradient
    ok = ((tf >= 2e-3) & (tf <= 1 - 2e-3)).ravel()
    for f in [f for f in np.argsort(-np.abs(dtf).ravel()) if ok[f]][:10]:
        c, i, k = np.unravel_index(f, dtf.shape)
        tp, tm = tf.copy(), tf.copy()
        tp[c, i, k] += np.float32(1e-3)
        tm[c, i, k] -= np.float32(1e-3)
        h2 = float(tp[c, i, k]) - float(tm[c, i, k])
        fd = (_loss(v, cam, tp, sc, pix, dl, xf) - _loss(v, cam, tm, sc, pix, dl, xf)) / h2
        assert abs(fd - dtf[c, i, k]) <= 1e-4 * max(1.0, abs(dtf[c, i, k])), (c, i, k, fd, dtf[c, i, k])
    ramp = np.zeros((3, 256, 4), dtype=np.float32)
    g = np.arange(256) / 255.0
    ramp[0] = np.stack([g, 0.5 * g, 0.2 + 0 * g, 0.08 * g], -1)
    ramp[1] = np.stack([0.3 + 0 * g, g, 0.5 * g, 0.05 * g], -1)
    ramp[2] = np.stack([0.5 * g, 0.2 + 0 * g, g, 0.06 * g], -1)
    _, dsc = O.render_grad(v, cam, ramp, sc, pix, dl, threads=2, xf=xf)
    for c in range(3):
        sp, sm = sc.copy(), sc.copy()
        sp[c] += np.float32(1e-3)
        sm[c] -= np.float32(1e-3)
        h2 = float(sp[c]) - float(sm[c])
        fd = (_loss(v, cam, ramp, sp, pix, dl, xf) - _loss(v, cam, ramp, sm, pix, dl, xf)) / h2
        assert abs(fd - dsc[c]) <= 1e-4 * max(1.0, abs(dsc[c])), (c, fd, dsc[c])


def test_ert_knife_edges_are_marked():
    """A constant medium gives A_k = 1 - q^k after sample k (closed form): a threshold equal to A_10
    makes the ray an early-termination knife edge, one halfway between A_10 and A_11 does not."""
    import math

    v = O.DenseVolume((8, 8, 64), 1, 16, 0, 0)
    v.insert((0, 0, 0), np.full((64, 8, 8, 1), 30000, dtype=np.uint16))
    v.build(threads=1)
    sig = 0.05
    tf = np.zeros((1, 256, 4), dtype=np.float32)
    tf[..., :3] = 0.5
    tf[..., 3] = 1.0 - math.exp(-sig)
    q = (1.0 - float(tf[0, 0, 3])) ** 0.5  # per sample of length 0.5
    cam = S.camera((4.0, 4.0, -20.0), (4.0, 4.0, 32.0), (0.0, 1.0, 0.0), 1, 1, fov_y_deg=45.0,
                   lod_error_px=1.0, step_voxels=0.5, ert_alpha=float(1.0 - q ** 10))
    dl = np.ones((1, 4))
    _, _, edge = O.render_grad(v, cam, tf, [1.0], ([0], [0]), dl, threads=1, ert_margin=1e-5)
    assert edge[0]
    cam["ert_alpha"] = float(1.0 - q ** 10.5)
    _, _, edge = O.render_grad(v, cam, tf, [1.0], ([0], [0]), dl, threads=1, ert_margin=1e-5)
    assert not edge[0]
