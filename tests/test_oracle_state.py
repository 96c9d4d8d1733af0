"""Pins of the oracle's volume state (downsampling, node records, homogeneity) against values the
paper and arithmetic fix: hand-computed golden cases, closed forms and invariants.  CPU only."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(dims, C, M, block=None, bg=0, tau=0):
    v = O.DenseVolume(dims, C, M, bg, tau)
    if block is not None:
        v.insert((0, 0, 0), block)
    v.build(threads=2)
    return v


def test_geometry_levels_and_virtual_extension():
    # Eq. 1 and Sec. "Handling Volumes of Arbitrary Dimensions": the volume is virtually
    # extended to M*2^N; the paper's example 3865 x 1966 x 2893 with M = 32 becomes 4096^3.
    g = O.geom((3865, 1966, 2893), 1, 32)
    assert g.N == 7 and 32 * 2 ** g.N == 4096
    assert [g.ldim[1][a] for a in range(3)] == [1933, 983, 1447]
    assert [g.nb[0][a] for a in range(3)] == [121, 62, 91]
    assert [g.nb[g.N][a] for a in range(3)] == [1, 1, 1]
    # the streamed workload 1024x1024x512 with M = 32: 6 levels, virtual 1024^3
    g2 = O.geom((1024, 1024, 512), 3, 32)
    assert g2.N == 5 and [g2.nb[0][a] for a in range(3)] == [32, 32, 16]


def test_brick_pool_overhead_closed_form():
    # Sec. "CPU Data Structure": each level holds 1/8 of the previous one, so the pool tends to
    # 8/7 of the data; with a one-voxel border the 32^3 brick grows by 34^3/32^3 (Sec.
    # "Filtering across Brick Boundaries": about 20%).
    g = O.geom((4096, 4096, 4096), 1, 32)
    vox = sum(g.ldim[L][0] * g.ldim[L][1] * g.ldim[L][2] for L in range(g.N + 1))
    assert abs(vox / 4096 ** 3 - 8 / 7) < 1e-4
    assert abs(34 ** 3 / 32 ** 3 - 1.199) < 1e-3


def test_round_half_up_on_a_ramp():
    # V0[x] = x; each level-1 voxel averages 2x and 2x+1 (four copies each): mean 2x + 0.5, which
    # rounds UP to 2x + 1; level 2 averages 4i+1 and 4i+3: exactly 4i + 2.
    X, Y, Z = 8, 4, 4
    blk = np.zeros((Z, Y, X, 1), dtype=np.uint16)
    blk[..., 0] = np.arange(X)[None, None, :]
    v = _dense((X, Y, Z), 1, 2, blk)
    l1 = v.level(1)[..., 0]
    assert (l1 == (2 * np.arange(4) + 1)[None, None, :]).all()
    l2 = v.level(2)[..., 0]
    assert (l2 == (4 * np.arange(2) + 2)[None, None, :]).all()


def test_hand_computed_odd_extent_3x3x3():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "downsample_3x3x3.txt")) if l.strip() and l[0] != "#"]
    blk = np.zeros((3, 3, 3, 1), dtype=np.uint16)
    for z in range(3):
        for y in range(3):
            for x in range(3):
                blk[z, y, x, 0] = 1 + x + 3 * y + 9 * z
    v = _dense((3, 3, 3), 1, 2, blk)
    assert v.N == 1
    l1 = v.level(1)
    for r in rows:
        x, y, z, k, S_, V1 = map(int, r)
        assert l1[z, y, x, 0] == V1, (x, y, z)


def test_constant_volume_is_constant_at_every_level():
    blk = np.full((20, 23, 17, 3), 777, dtype=np.uint16)
    blk[..., 1] = 5
    v = _dense((17, 23, 20), 3, 4, blk, tau=1)
    for L in range(v.N + 1):
        lv = v.level(L)
        assert (lv[..., 0] == 777).all() and (lv[..., 1] == 5).all()
    root = v.node(v.N, 0, 0, 0)
    assert root.touched and root.subtree_homog and not root.has_children and not root.has_brick
    assert list(root.avg[:2]) == [777, 5]


def test_level_values_lie_between_children_min_and_max():
    spec = S.VolumeSpec(S.KIND_BLOBS, (24, 20, 18), 2, 6, seed=5)
    vol = spec.volume()
    v = _dense((24, 20, 18), 2, 4, vol)
    for L in range(1, v.N + 1):
        P, Q = v.level(L - 1).astype(np.int64), v.level(L).astype(np.int64)
        Zq, Yq, Xq, _ = Q.shape
        for z in range(Zq):
            for y in range(Yq):
                for x in range(Xq):
                    ch = P[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * x:2 * x + 2].reshape(-1, 2)
                    assert (ch.min(0) <= Q[z, y, x]).all() and (Q[z, y, x] <= ch.max(0)).all()


def test_insertion_order_independence():
    # The state is a function of the current values only: any insertion order, any block shape,
    # and overwrites give bit-identical levels and node records (the paper allows blocks at
    # arbitrary positions and overwriting, Sec. "Incremental Construction").
    dims = (40, 36, 28)
    spec = S.VolumeSpec(S.KIND_BLOBS, dims, 3, 8, seed=9)
    vol = spec.volume()
    ref = _dense(dims, 3, 8, vol, bg=50, tau=900)
    rng = np.random.default_rng(0)
    other = O.DenseVolume(dims, 3, 8, 50, 900)
    junk = rng.integers(0, 65535, size=vol.shape, dtype=np.uint16)
    other.insert((0, 0, 0), junk)  # garbage first, then overwritten slice by slice in random order
    for z in rng.permutation(dims[2]):
        other.insert((0, 0, int(z)), vol[z:z + 1])
    other.build(threads=2)
    for L in range(ref.N + 1):
        assert (ref.level(L) == other.level(L)).all()
        g = ref.geom
        for k in range(g.nb[L][2]):
            for j in range(g.nb[L][1]):
                for i in range(g.nb[L][0]):
                    a, b = ref.node(L, i, j, k), other.node(L, i, j, k)
                    for f in ("touched", "has_children", "has_brick"):
                        assert getattr(a, f) == getattr(b, f)
                    assert list(a.avg) == list(b.avg)


def test_figure3_analogue_flags_and_avg():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "fig3_analogue.txt")) if l.strip() and l[0] != "#"]
    blocks = [(int(l[1]), int(l[2]), [int(x) for x in l[3:]]) for l in lines if l[0] == "block"]
    nodes = [tuple(int(x) for x in l[1:]) for l in lines if l[0] == "node"]
    v = O.DenseVolume((16, 1, 1), 1, 4, 3, 1)
    assert v.N == 2
    for bi in sorted({b[0] for b in blocks}):
        for name, x0, vals in blocks:
            if name == bi:
                v.insert((x0, 0, 0), np.array(vals, dtype=np.uint16).reshape(1, 1, -1, 1))
        v.build(threads=1)
        for after, L, idx, touched, has_brick, has_children, avg in nodes:
            if after == bi:
                n = v.node(L, idx, 0, 0)
                assert (n.touched, n.has_brick, n.has_children, n.avg[0]) == (touched, has_brick, has_children, avg), \
                    (after, L, idx)
        if bi == 3:
            assert list(v.level(0)[0, 0, :, 0]) == [1, 5, 2, 4, 3, 3, 3, 3, 3, 3, 2, 2, 3, 3, 3, 3]
            assert list(v.level(1)[0, 0, :, 0]) == [3, 3, 3, 3, 3, 2, 3, 3]


def test_out_of_volume_voxels_do_not_enter_stats():
    # A partial brick (real extent 5 of M = 4 -> second brick holds one real voxel column):
    # the AVG/min/max of that brick use only the in-volume voxels.
    blk = np.zeros((1, 1, 5, 1), dtype=np.uint16)
    blk[0, 0, :, 0] = [10, 10, 10, 10, 7]
    v = _dense((5, 1, 1), 1, 4, blk, bg=999, tau=1)
    n1 = v.node(0, 1, 0, 0)
    assert n1.count == 1 and n1.avg[0] == 7 and n1.bmin[0] == 7 and n1.bmax[0] == 7
    assert n1.brick_homog and not n1.has_brick
    # level 1 voxel 2 averages the single in-volume child (x = 4) only
    assert v.level(1)[0, 0, 2, 0] == 7


def test_channels_all_homogeneous_for_deletion():
    # Sec. "Handling Multi-Channel Data": a brick is deleted only if every channel is homogeneous.
    blk = np.zeros((4, 4, 4, 2), dtype=np.uint16)
    blk[..., 0] = 100
    blk[..., 1] = 100
    blk[0, 0, 0, 1] = 200
    v = _dense((4, 4, 4), 2, 4, blk, tau=50)
    n = v.node(0, 0, 0, 0)
    assert not n.brick_homog and n.has_brick
    blk[0, 0, 0, 1] = 120
    v2 = _dense((4, 4, 4), 2, 4, blk, tau=50)
    assert v2.node(0, 0, 0, 0).brick_homog and not v2.node(0, 0, 0, 0).has_brick


def test_lazy_volume_matches_dense_volume():
    dims = (48, 40, 36)
    spec = S.VolumeSpec(S.KIND_SPIM, dims, 3, 40, seed=3)
    vol = spec.volume()
    for tau in (0, 400):
        dense = O.DenseVolume(dims, 3, 8, 100, tau)
        dense.insert((0, 0, 10), vol[10:30])
        dense.build(threads=2)
        lazy = O.LazyVolume(dims, 3, 8, spec.voxel_fn, spec.handle, 10, 30, background=100, tau=tau, owner=spec)
        rng = np.random.default_rng(tau)
        for L in range(dense.N + 1):
            X, Y, Z = dense.level_dims(L)
            lv = dense.level(L)
            for _ in range(60):
                x, y, z = int(rng.integers(X)), int(rng.integers(Y)), int(rng.integers(Z))
                for c in range(3):
                    assert lazy.value(L, x, y, z, c) == lv[z, y, x, c]
            g = dense.geom
            for k in range(g.nb[L][2]):
                for j in range(g.nb[L][1]):
                    for i in range(g.nb[L][0]):
                        a, b = dense.node(L, i, j, k), lazy.node(L, i, j, k)
                        assert (a.touched, a.has_children, a.has_brick) == (b.touched, b.has_children, b.has_brick)
                        if not a.has_brick:
                            assert list(a.avg[:3]) == list(b.avg[:3])


@pytest.mark.parametrize("dims,C,M,tau,cuts", [((48, 40, 37), 3, 8, 400, (5, 6, 1, 7, 18)),
                                               ((33, 21, 19), 1, 4, 0, (2, 2, 2, 2, 2, 2, 2, 2, 3)),
                                               ((40, 24, 30), 2, 6, 900, (30,)),
                                               ((64, 64, 64), 3, 16, 3277, (8,) * 8)])
def test_streamed_volume_matches_dense_volume(dims, C, M, tau, cuts):
    """The streamed construction (level 0 fed once in z order, levels >= 1 and node records from
    one pass) is the dense oracle's state: every level >= 1 and every node record are equal, level
    0 reads back the generator, and a render gives the same numbers."""
    spec = S.VolumeSpec(S.KIND_SPIM, dims, C, 30, seed=5)
    vol = spec.volume()
    dense = O.DenseVolume(dims, C, M, 0, tau)
    dense.insert((0, 0, 0), vol)
    dense.build(threads=2)
    st = O.StreamVolume(dims, C, M, spec.voxel_fn, spec.handle, tau=tau, owner=spec)
    z = 0
    for n in cuts:  # uneven slabs, odd and even starts
        st.feed(z, vol[z:z + n], threads=2)
        z += n
    assert z == dims[2]
    with pytest.raises(ValueError):
        st.feed(0, vol[:1])  # out of order
    st.finish(threads=2)
    for L in range(1, dense.N + 1):
        assert np.array_equal(st.level(L), dense.level(L)), L
    g = dense.geom
    fields = ("touched", "has_children", "has_brick", "brick_homog", "subtree_homog", "count")
    for L in range(dense.N + 1):
        for k in range(g.nb[L][2]):
            for j in range(g.nb[L][1]):
                for i in range(g.nb[L][0]):
                    a, b = dense.node(L, i, j, k), st.node(L, i, j, k)
                    assert all(getattr(a, f) == getattr(b, f) for f in fields), (L, i, j, k)
                    for arr in ("avg", "bmin", "bmax", "smin", "smax"):
                        assert list(getattr(a, arr)[:C]) == list(getattr(b, arr)[:C]), (L, i, j, k, arr)
    rng = np.random.default_rng(1)
    for _ in range(40):
        x, y, zz = (int(rng.integers(d)) for d in dims)
        assert [st.value(0, x, y, zz, c) for c in range(C)] == list(vol[zz, y, x])
    if C == 3:
        cam = S.orbit_camera(dims, 2.0 * max(dims), 30.0, 20.0, 24, 20, lod_error_px=0.7)
        tf = S.make_tf([11, 12, 13])
        nc_a, ca, sa = O.render(dense, cam, tf, [1.0, 1.0, 1.0])
        nc_b, cb, sb = O.render(st, cam, tf, [1.0, 1.0, 1.0])
        assert np.array_equal(nc_a, nc_b) and np.array_equal(ca, cb) and np.array_equal(sa, sb)
