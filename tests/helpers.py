"""Shared helpers of the GPU parity tests."""
import numpy as np

from oracle import oracle as O

RGBA_TOL = 2e-3  # max-abs RGBA, every pixel, against some admissible oracle result


admissible_error = O.admissible_error  # per-pixel error to the nearest admissible oracle state


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
