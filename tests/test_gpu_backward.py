"""Adjoint parity: the hand-written backward (per-ray recompute, forward-order reverse sweep)
against the oracle's exact FP64 gradient and against central finite differences of the GPU
forward.  Gradient tolerance: relative 1e-3, norm-wise, and element by element wherever
|g| > 1e-6 max|g| in the FP64 gradient-check mode (vr_set_gradient_precision); the single-precision
mode is held to 1e-3 relative plus 1e-5 max|g| per element (its sums cancel in FP32)."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import oracle_dense

pytestmark = pytest.mark.gpu


def _setup(tau=0, ert=2.0, size=40):
    import torch
    import paper_1407_2074_b300 as vr

    w = S.tiny(tau)
    vol = w.spec().volume()
    r = vr.Renderer(w.dims, 3, 16, tau=tau)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(64):
        r.insert_slice(z, dev[z])
    cam = dict(w.cameras[0])
    cam["width"] = cam["height"] = size
    cam["ert_alpha"] = ert
    return w, vol, r, cam


# Rays whose opacity passes this close to the threshold may stop a sample apart: the stop is decided
# by the single-precision forward, whose opacity differs from the double one by up to ~1e-4 on the
# near-opaque tables below (1 - alpha of a few 1e-4 loses most of its bits in single precision).
# The same band as the early-termination band of the image check.
ERT_MARGIN = 2e-4


def _grad_close(got, ref, rel=1e-3, fp64=True):
    """Norm-wise, and per element: with fp64 (the FP64 gradient-check mode) relative error <= rel
    wherever |g| > 1e-6 max|g| and smaller entries within 1e-6 max|g|; otherwise (single-precision
    sums) within rel |g| + 1e-5 max|g|."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    scale = np.abs(ref).max()
    assert np.linalg.norm(got - ref) <= rel * np.linalg.norm(ref)
    d = np.abs(got - ref)
    if not fp64:
        assert (d <= rel * np.abs(ref) + 1e-5 * scale).all()
        return
    big = np.abs(ref) > 1e-6 * scale
    worst = np.argmax(np.where(big, d / np.maximum(np.abs(ref), 1e-300), 0.0))
    assert (d[big] <= rel * np.abs(ref[big])).all(), \
        f"max rel {d.flat[worst] / abs(ref.flat[worst]):.3e} at {worst}: |g| / max|g| = {abs(ref.flat[worst]) / scale:.2e}"
    assert (d[~big] <= 1e-6 * scale).all()


def _backward_both(r, cam, tf, sc, dl, rtf, rsc):
    """The GPU adjoint in single precision and in the FP64 gradient-check mode, against the oracle."""
    import torch

    r.set_transfer_functions(torch.from_numpy(tf), torch.from_numpy(sc))
    for fp64 in (False, True):
        r.set_gradient_precision(fp64)
        dtf, dsc = r.render_backward([cam], [torch.from_numpy(dl).cuda()])
        torch.cuda.synchronize()
        _grad_close(dtf.cpu().numpy(), rtf, fp64=fp64)
        _grad_close(dsc.cpu().numpy(), rsc, fp64=fp64)
    r.set_gradient_precision(False)


def _oracle_grad_ert(ov, cam, tf, sc, dl):
    """The oracle gradient of every pixel, with dL/dimage zeroed on the rays the oracle marks as
    early-termination knife edges; returns (dl used, dtf, dscale, number of rays excluded)."""
    px, py = O.image_pixels(cam["width"], cam["height"])
    flat = dl.reshape(-1, 4).astype(np.float64)
    _, _, edge = O.render_grad(ov, cam, tf, sc, (px, py), flat, ert_margin=ERT_MARGIN)
    dl2 = dl.copy().reshape(-1, 4)
    dl2[edge] = 0.0
    rtf, rsc = O.render_grad(ov, cam, tf, sc, (px, py), dl2.astype(np.float64))
    return dl2.reshape(dl.shape), rtf, rsc, int(edge.sum())


def test_backward_matches_oracle_gradient():
    import torch

    w, vol, r, cam = _setup()
    ov = oracle_dense(vol, 16)
    tf = w.tf()
    sc = np.array([1.0, 0.8, 1.3], np.float32)
    rng = np.random.default_rng(0)
    dl = rng.normal(size=(cam["height"], cam["width"], 4)).astype(np.float32)
    px, py = O.image_pixels(cam["width"], cam["height"])
    rtf, rsc = O.render_grad(ov, cam, tf, sc, (px, py), dl.reshape(-1, 4).astype(np.float64))
    _backward_both(r, cam, tf, sc, dl, rtf, rsc)


def test_backward_with_early_termination():
    """ERT on (most rays stop): per element against the oracle, the rays whose opacity passes within
    ERT_MARGIN of the threshold (a stop one sample apart is correct there) excluded on both sides."""
    import torch

    w, vol, r, cam = _setup(ert=0.99)
    ov = oracle_dense(vol, 16)
    tf = w.tf()
    tf[..., 3] = np.minimum(1.0, tf[..., 3] * 10.0)
    sc = np.array([1.0, 1.0, 1.0], np.float32)
    dl = np.random.default_rng(1).normal(size=(cam["height"], cam["width"], 4)).astype(np.float32)
    dl, rtf, rsc, excluded = _oracle_grad_ert(ov, cam, tf, sc, dl)
    print(f"ERT knife-edge rays excluded: {excluded} of {dl.shape[0] * dl.shape[1]}")
    _backward_both(r, cam, tf, sc, dl, rtf, rsc)


@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_backward_through_homogeneous_runs(ert):
    """A SPIM-like volume with tau = 3277: the background outside the tissue is brick-less, and
    the sweep takes its runs of equal samples in closed form; the gradient still equals the
    oracle's sample-by-sample FP64 one."""
    import torch
    import paper_1407_2074_b300 as vr

    dims = (96, 80, 64)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 60, seed=17)
    vol = spec.volume()
    r = vr.Renderer(dims, 3, 16, tau=3277)
    r.insert_block((0, 0, 0), torch.from_numpy(vol.view(np.int16)).cuda())
    ov = oracle_dense(vol, 16, tau=3277)
    g = ov.geom
    brickless = sum(not ov.node(L, i, j, k).has_brick for L in range(g.N + 1) for k in range(g.nb[L][2])
                    for j in range(g.nb[L][1]) for i in range(g.nb[L][0]) if ov.node(L, i, j, k).touched)
    assert brickless > 10
    cam = S.orbit_camera(dims, 2.0 * 96, 30.0, 20.0, 40, 36, lod_error_px=0.7)
    cam["ert_alpha"] = ert
    tf = S.make_tf([11, 12, 13])
    tf[..., 3] = np.minimum(1.0, tf[..., 3] * (8.0 if ert < 1.0 else 2.0))
    sc = np.array([1.0, 0.9, 1.2], np.float32)
    dl = np.random.default_rng(3).normal(size=(cam["height"], cam["width"], 4)).astype(np.float32)
    dl, rtf, rsc, _ = _oracle_grad_ert(ov, cam, tf, sc, dl)
    _backward_both(r, cam, tf, sc, dl, rtf, rsc)


def test_autograd_function_and_finite_differences():
    import torch
    import paper_1407_2074_b300 as vr

    w, vol, r, cam = _setup(size=24)
    g = np.arange(256) / 255.0
    tf_np = np.zeros((3, 256, 4), np.float32)
    tf_np[0] = np.stack([g, 0.5 * g, 0.2 + 0 * g, 0.08 * g], -1)
    tf_np[1] = np.stack([0.3 + 0 * g, g, 0.5 * g, 0.05 * g], -1)
    tf_np[2] = np.stack([0.5 * g, 0.2 + 0 * g, g, 0.06 * g], -1)
    tf = torch.from_numpy(tf_np).cuda().requires_grad_(True)
    sc = torch.tensor([1.0, 0.9, 1.2], device="cuda", requires_grad=True)
    target = torch.rand((24, 24, 4), device="cuda")
    loss = ((vr.render(r, [cam], tf, sc)[0] - target) ** 2).mean()
    loss.backward()

    def L(tfv, scv):
        with torch.no_grad():
            return ((vr.render(r, [cam], tfv, scv)[0].double() - target.double()) ** 2).mean().item()

    for c in range(3):
        h = 1e-3
        sp, sm = sc.detach().clone(), sc.detach().clone()
        sp[c] += h
        sm[c] -= h
        fd = (L(tf.detach(), sp) - L(tf.detach(), sm)) / (float(sp[c]) - float(sm[c]))
        assert abs(fd - sc.grad[c].item()) <= 2e-3 * abs(fd) + 1e-5
    # entries within 2e-3 of 0 or 1 sit on the opacity clamp (a kink for a +-1e-3 step): skip them
    ok = ((tf.detach() >= 2e-3) & (tf.detach() <= 1 - 2e-3)).flatten()
    big = torch.topk(torch.where(ok, tf.grad.abs().flatten(), torch.zeros_like(tf.grad.flatten())), 6).indices
    for f in big.tolist():
        c, i, q = np.unravel_index(f, (3, 256, 4))
        tp, tm = tf.detach().clone(), tf.detach().clone()
        tp[c, i, q] += 1e-3
        tm[c, i, q] -= 1e-3
        fd = (L(tp, sc.detach()) - L(tm, sc.detach())) / (float(tp[c, i, q]) - float(tm[c, i, q]))
        assert abs(fd - tf.grad[c, i, q].item()) <= 2e-3 * abs(fd) + 1e-5


def test_differentiable_full_size_sampled_gradient():
    """512^3 x 3 SPIM-like volume (tau = 3277), 512x512: dL/dimage nonzero on sampled pixels;
    gradient against the oracle's FP64 gradient of the same pixels."""
    import torch
    import paper_1407_2074_b300 as vr

    w = S.differentiable()
    spec = w.spec()
    vol = spec.volume()
    X, Y, Z = w.dims
    r = vr.Renderer(w.dims, 3, 32, tau=w.tau)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z0 in range(0, Z, 16):
        r.insert_block((0, 0, z0), dev[z0:z0 + 16])
    del dev
    ov = oracle_dense(vol, 32, tau=w.tau)
    cam = w.cameras[0]
    tf = w.tf()
    sc = np.array([1.0, 1.0, 1.0], np.float32)
    r.set_transfer_functions(torch.from_numpy(tf), torch.from_numpy(sc))
    rng = np.random.default_rng(9)
    n = 400
    flat = rng.choice(512 * 512, size=n, replace=False)
    px, py = (flat % 512).astype(np.int32), (flat // 512).astype(np.int32)
    dl = np.zeros((512, 512, 4), np.float32)
    dl[py, px] = rng.normal(size=(n, 4))
    dtf, dsc = r.render_backward([cam], [torch.from_numpy(dl).cuda()])
    rtf, rsc = O.render_grad(ov, cam, tf, sc, (px, py), dl[py, px].astype(np.float64))
    g = dtf.cpu().numpy()
    assert np.linalg.norm(g - rtf) <= 1e-3 * np.linalg.norm(rtf)
    assert np.linalg.norm(dsc.cpu().numpy() - rsc) <= 1e-3 * np.linalg.norm(rsc)


def test_backward_from_forward_images():
    """vr_render_backward_with_images: each ray's final colour and transmittance read from the
    forward's image instead of a second march.  Equal to the re-marching adjoint up to the rounding
    of 1 - alpha, and within the gradient tolerance of the oracle; also through the autograd
    function (which passes its forward images)."""
    import torch
    import paper_1407_2074_b300 as vr

    w, vol, r, cam = _setup(ert=0.99)
    ov = oracle_dense(vol, 16)
    tf = w.tf()
    tf[..., 3] = np.minimum(1.0, tf[..., 3] * 4.0)
    sc = np.array([1.0, 0.9, 1.1], np.float32)
    dl = np.random.default_rng(4).normal(size=(cam["height"], cam["width"], 4)).astype(np.float32)
    dl, rtf, rsc, _ = _oracle_grad_ert(ov, cam, tf, sc, dl)
    r.set_transfer_functions(torch.from_numpy(tf), torch.from_numpy(sc))
    fwd = r.render([cam])
    g = [torch.from_numpy(dl).cuda()]
    a_tf, a_sc = r.render_backward([cam], g)
    b_tf, b_sc = r.render_backward([cam], g, images=fwd)
    torch.cuda.synchronize()
    a_tf, b_tf = a_tf.cpu().numpy().astype(np.float64), b_tf.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a_tf - b_tf) <= 1e-5 * np.linalg.norm(a_tf)
    assert np.abs(a_sc.cpu().numpy() - b_sc.cpu().numpy()).max() <= 1e-5 * np.abs(a_sc.cpu().numpy()).max()
    _grad_close(b_tf, rtf, fp64=False)
    _grad_close(b_sc.cpu().numpy(), rsc, fp64=False)
    # the autograd path: d(sum dl * image) through RenderFn
    tf_t = torch.from_numpy(tf).cuda().requires_grad_(True)
    sc_t = torch.from_numpy(sc).cuda().requires_grad_(True)
    img = vr.render(r, [cam], tf_t, sc_t)[0]
    (img * g[0]).sum().backward()
    torch.cuda.synchronize()
    # (the sums use atomics: equal up to their order)
    assert np.linalg.norm(tf_t.grad.cpu().numpy() - b_tf) <= 1e-6 * np.linalg.norm(b_tf)
    # the FP64 check mode ignores the images (recomputes the double forward)
    r.set_gradient_precision(True)
    c_tf, _ = r.render_backward([cam], g, images=fwd)
    torch.cuda.synchronize()
    _grad_close(c_tf.cpu().numpy(), rtf, fp64=True)
    r.set_gradient_precision(False)
    r.close()


def test_backward_from_images_several_views_in_one_launch():
    """The per-lane ray queue of the backward from forward images (rays handed out one per lane
    over the tiles of all views, a warp regrouping when lanes fall idle): one launch over three
    views of different, ragged sizes gives the sum of the three single-view gradients (the
    adjoint is linear in dL/dimage), up to the order of the floating-point atomics."""
    import torch

    w, vol, r, _ = _setup(ert=0.99)
    tf = w.tf()
    tf[..., 3] = np.minimum(1.0, tf[..., 3] * 4.0)
    sc = np.array([1.0, 0.9, 1.1], np.float32)
    r.set_transfer_functions(torch.from_numpy(tf), torch.from_numpy(sc))
    cams = []
    for i, (wd, ht) in enumerate(((40, 40), (37, 23), (64, 48))):
        cam = dict(w.cameras[i % len(w.cameras)])
        cam["width"], cam["height"] = wd, ht
        cam["ert_alpha"] = 0.99
        cams.append(cam)
    rng = np.random.default_rng(9)
    gs = [torch.from_numpy(rng.normal(size=(c["height"], c["width"], 4)).astype(np.float32)).cuda() for c in cams]
    fwd = r.render(cams)
    all_tf, all_sc = r.render_backward(cams, gs, images=fwd)
    all_tf, all_sc = all_tf.cpu().numpy().astype(np.float64), all_sc.cpu().numpy().astype(np.float64)
    sum_tf, sum_sc = np.zeros_like(all_tf), np.zeros_like(all_sc)
    for cam, g, im in zip(cams, gs, fwd):
        one = r.render([cam])[0]
        assert torch.equal(one, im)  # a ray does not depend on the other views of the launch
        t, s = r.render_backward([cam], [g], images=[one])
        sum_tf += t.cpu().numpy()
        sum_sc += s.cpu().numpy()
    assert np.abs(all_tf).max() > 0.0
    assert np.linalg.norm(all_tf - sum_tf) <= 1e-5 * np.linalg.norm(sum_tf)
    assert np.abs(all_sc - sum_sc).max() <= 1e-5 * np.abs(sum_sc).max()
    r.close()
