"""Shared helpers of the GPU parity tests."""
import numpy as np

from oracle import oracle as O

RGBA_TOL = 2e-3  # max-abs RGBA, every pixel, against some admissible oracle result
UNRESOLVED_FRAC = 1e-4  # rays with more knife-edge decisions than the oracle enumerates, at most


admissible_error = O.admissible_error  # per-pixel error to the nearest candidate of an oracle render


def parity(vol, cam, tf, scale, rgba, pixels=None, mode=0, xf=None, tol=RGBA_TOL):
    """GPU pixels against the oracle's admissible results (double-precision geometry, every
    combination of branches of the ray's first knife-edge decisions, any stop in the
    early-termination band).  Gate: every resolved pixel within tol; an unresolved ray (more
    knife-edge decisions than enumerated) may miss it, but such misses number at most
    UNRESOLVED_FRAC of the pixels; on a whole image the unresolved rays themselves number at most
    UNRESOLVED_FRAC of its pixels.  Returns the oracle's per-pixel record (err, natural rgba,
    samples, flagged, variants, unresolved)."""
    n = len(pixels[0]) if pixels is not None else cam["width"] * cam["height"]
    r = O.check(vol, cam, tf, scale, np.asarray(rgba, dtype=np.float32).reshape(n, 4), pixels, mode, xf=xf,
                stop_err=tol)
    unres = r["unresolved"] != 0
    over = r["err"] > tol
    worst = int(np.argmax(np.where(unres, 0.0, r["err"]))) if n else 0
    assert not (over & ~unres).any(), \
        f"{(over & ~unres).sum()} pixels over {tol:g}; max err {r['err'][worst]:.3e} at index {worst}"
    assert over.sum() <= UNRESOLVED_FRAC * n, f"{over.sum()} unresolved rays over {tol:g} of {n}"
    if pixels is None:
        assert unres.sum() <= max(1.0, UNRESOLVED_FRAC * n), f"{unres.sum()} unresolved rays of {n}"
    return r


def oracle_dense(volume: np.ndarray, brick, bg=0, tau=0, z_hi=None):
    Z, Y, X, C = volume.shape
    v = O.DenseVolume((X, Y, Z), C, brick, bg, tau)
    zz = Z if z_hi is None else z_hi
    if zz > 0:
        v.insert((0, 0, 0), volume[:zz])
    v.build()
    return v


def cam_rgba(img_t, px, py):
    img = img_t.detach().cpu().numpy()
    return img[py, px]
