"""The oracle's algorithmic footprint of a frame (the numerator of the HBM roofline): distinct
voxels read by trilinear corners and distinct node entries read on descents, pinned on rays whose
cells and descent paths can be counted by hand."""
import numpy as np

from oracle import oracle as O
from tests.helpers import oracle_dense


def _volume(dims=(40, 24, 24), M=8, seed=3):
    X, Y, Z = dims
    vol = np.random.default_rng(seed).integers(0, 65535, size=(Z, Y, X, 3), dtype=np.uint16)
    return oracle_dense(vol, M)


def _axis_ray_camera(lod_error_px, ert=2.0):
    """One pixel whose ray runs along +x at y = z = 10.3 through the whole 40-voxel extent."""
    return dict(eye=[-10.0, 10.3, 10.3], target=[30.0, 10.3, 10.3], up=[0.0, 1.0, 0.0], fov_y_deg=45.0, width=1,
                height=1, lod_error_px=lod_error_px, step_voxels=0.5, ert_alpha=ert, clip=[])


def test_axis_ray_at_level_0():
    """Level 0 everywhere: the cells of x = 0 .. 39.5 cover voxels x = 0 .. 39 (clamped at both
    ends) and y, z in {9, 10} (u = 10.3 - 0.5 = 9.8), so 40 x 2 x 2 voxels.  The descent paths
    visit the level-0 bricks x = 0 .. 4 (M = 8), the level-1 nodes 0 .. 2, the level-2 nodes 0, 1
    and the root: 5 + 3 + 2 + 1 nodes."""
    ov = _volume()
    assert ov.N == 3
    tf = np.zeros((3, 256, 4), np.float32)
    vox, nodes = O.render_footprint(ov, _axis_ray_camera(0.01), tf, [1.0, 1.0, 1.0])
    assert vox == [160, 0, 0, 0]
    assert nodes == 11


def test_far_camera_reads_the_root_only():
    """A pixel error so large that every sample's level is the top one: only the root's node
    entry, and level-3 voxels (extent 5 x 3 x 3) of the cells along the ray: x = 0 .. 4,
    y, z: u = 10.3 / 8 - 0.5 = 0.79 -> {0, 1}."""
    ov = _volume()
    tf = np.zeros((3, 256, 4), np.float32)
    vox, nodes = O.render_footprint(ov, _axis_ray_camera(1e6), tf, [1.0, 1.0, 1.0])
    assert vox == [0, 0, 0, 5 * 2 * 2]
    assert nodes == 1


def test_early_termination_shortens_the_footprint():
    """An opaque table stops the ray at its first sample (A = 1 - 1e-6 per channel): one cell at
    x = 0 (voxels x = 0, y, z in {9, 10}: 4) and the path of that sample (4 nodes)."""
    ov = _volume()
    tf = np.ones((3, 256, 4), np.float32)
    vox, nodes = O.render_footprint(ov, _axis_ray_camera(0.01, ert=0.99), tf, [1.0, 1.0, 1.0])
    assert vox == [4, 0, 0, 0]
    assert nodes == 4
