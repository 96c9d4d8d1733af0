"""Shared helpers of the GPU parity tests."""
import numpy as np

from oracle import oracle as O

RGBA_TOL = 2e-3  # max-abs RGBA, every pixel, against some admissible oracle result


def admissible_error(gpu_rgba: np.ndarray, n_cand: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """Per-pixel max-abs error of gpu_rgba [n][4] to the nearest admissible oracle state."""
    g = np.asarray(gpu_rgba, dtype=np.float64).reshape(-1, 1, 4)
    c = cand.reshape(g.shape[0], O.MAXCAND, 4)
    e = np.abs(c - g).max(axis=-1)
    valid = np.arange(O.MAXCAND)[None, :] < n_cand.reshape(-1, 1)
    return np.where(valid, e, np.inf).min(axis=-1)


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
