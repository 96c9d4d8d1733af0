"""Construction parity: every level of the device brick pool is bit-identical to the oracle's
iterated round-half-up downsampling, and every node record (touched, children, brick, AVG) equals
the oracle's, after slice streams, random orders, overwriting blocks and partial inserts."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import synth as S
from tests.helpers import oracle_dense

pytestmark = pytest.mark.gpu


def _renderer(dims, C, M, bg=0, tau=0, **kw):
    import paper_1407_2074_b300 as vr

    return vr.Renderer(dims, C, M, background=bg, tau=tau, **kw)


def _compare_state(r, ov, check_nodes=True):
    from paper_1407_2074_b300 import vr as V

    g = ov.geom
    for L in range(ov.N + 1):
        got, ref = r.read_level(L), ov.level(L)
        assert got.shape == ref.shape
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"level {L}: {len(bad)} voxels differ, first {bad[:3].tolist()}"
    if not check_nodes:
        return
    for L in range(ov.N + 1):
        for k in range(g.nb[L][2]):
            for j in range(g.nb[L][1]):
                for i in range(g.nb[L][0]):
                    fl, avg = r.read_node(L, i, j, k)
                    n = ov.node(L, i, j, k)
                    exp = (V.F_TOUCHED if n.touched else 0) | (V.F_CHILDREN if n.has_children else 0) | \
                          (V.F_BRICK if n.has_brick else 0)
                    assert fl == exp, (L, i, j, k, fl, exp)
                    assert avg == list(n.avg[: r.C]), (L, i, j, k, avg, list(n.avg[: r.C]))


@pytest.mark.parametrize("tau", [0, 2000, 65535])
def test_tiny_slice_stream_levels_and_nodes(tau):
    import torch

    w = S.tiny()
    vol = w.spec().volume()
    r = _renderer(w.dims, 3, 16, tau=tau)
    dev = torch.from_numpy(vol.view(np.int16)).cuda()
    for z in range(64):
        r.insert_slice(z, dev[z])
    _compare_state(r, oracle_dense(vol, 16, tau=tau))


def test_partial_stream_untouched_regions_stay_background():
    w = S.tiny()
    vol = w.spec().volume()
    r = _renderer(w.dims, 3, 16, bg=77, tau=500)
    for z in range(37):
        r.insert_slice(z, vol[z])  # host pointers
    _compare_state(r, oracle_dense(vol, 16, bg=77, tau=500, z_hi=37))


@pytest.mark.parametrize("C,M,dims", [(2, 6, (37, 29, 23)), (1, 4, (19, 33, 8)), (4, 8, (40, 24, 17))])
def test_random_order_blocks_and_overwrites(C, M, dims):
    spec = S.VolumeSpec(S.KIND_SPIM, dims, C, 30, seed=4)
    vol = spec.volume()
    rng = np.random.default_rng(C * 100 + M)
    r = _renderer(dims, C, M, bg=123, tau=600)
    X, Y, Z = dims
    junk = rng.integers(0, 65535, size=vol.shape, dtype=np.uint16)
    # garbage blocks first, then the real data in random slices and random blocks
    for _ in range(6):
        o = [int(rng.integers(0, d)) for d in dims]
        e = [int(rng.integers(1, d - oo + 1)) for d, oo in zip(dims, o)]
        r.insert_block(o, junk[o[2]:o[2] + e[2], o[1]:o[1] + e[1], o[0]:o[0] + e[0]])
    for z in rng.permutation(Z):
        r.insert_slice(int(z), vol[z])
    for _ in range(4):
        o = [int(rng.integers(0, d)) for d in dims]
        e = [int(rng.integers(1, d - oo + 1)) for d, oo in zip(dims, o)]
        r.insert_block(o, vol[o[2]:o[2] + e[2], o[1]:o[1] + e[1], o[0]:o[0] + e[0]])
    _compare_state(r, oracle_dense(vol, M, bg=123, tau=600))


@pytest.mark.parametrize("C,M,dims", [(3, 32, (96, 72, 80)), (3, 64, (136, 72, 70)), (4, 16, (40, 24, 17)),
                                      (1, 8, (48, 20, 9)), (2, 8, (36, 20, 12))])
def test_staged_level0_matches_per_thread_loads(C, M, dims):
    """Level 0 through rows staged in shared memory by bulk tensor copies and through per-thread
    loads build the same tree, equal to the oracle's: a whole-volume block (up to M + 2 planes per
    slot: several staged chunks; M = 64 holds two planes per chunk), sub-boxes whose rows are or are
    not 16-byte aligned (the latter take the per-thread loads), a device block at a base address
    off the 16-byte grid, then 8-slice slabs over the whole volume."""
    import torch

    spec = S.VolumeSpec(S.KIND_SPIM, dims, C, 40, seed=9)
    vol = spec.volume()
    X, Y, Z = dims
    rng = np.random.default_rng(C * 1000 + M)
    junk = rng.integers(0, 65535, size=vol.shape, dtype=np.uint16)
    boxes = []
    for q in range(8):
        o = [int(rng.integers(0, d)) for d in dims]
        e = [int(rng.integers(1, d - oo + 1)) for d, oo in zip(dims, o)]
        if q % 2 == 0:  # a row pitch that is a multiple of 16 bytes where the box allows one
            step = 8 // np.gcd(8, C)
            if e[0] >= step:
                e[0] -= e[0] % step
        boxes.append((o, e))
    rs = []
    for staged in (1, 0):
        r = _renderer(dims, C, M, bg=321, tau=900)
        r.set_insert_staging(staged)
        r.insert_block((0, 0, 0), torch.from_numpy(junk.view(np.int16)).cuda())
        for o, e in boxes:
            r.insert_block(o, vol[o[2]:o[2] + e[2], o[1]:o[1] + e[1], o[0]:o[0] + e[0]])
        # a device block whose base is 2 bytes past a 16-byte boundary
        ez = min(5, Z)
        flat = torch.empty(ez * Y * X * C + 1, dtype=torch.int16, device="cuda")
        blk = flat[1:].view(ez, Y, X, C)
        blk.copy_(torch.from_numpy(junk[:ez].view(np.int16)))
        r.insert_block((0, 0, 0), blk)
        for z0 in range(0, Z, 8):
            r.insert_block((0, 0, z0), torch.from_numpy(vol[z0:z0 + 8].view(np.int16)).cuda())
        torch.cuda.synchronize()
        rs.append(r)
    for L in range(rs[0].levels):
        a, b = rs[0].read_level(L), rs[1].read_level(L)
        assert np.array_equal(a, b), f"level {L}: staged and per-thread loads differ"
    _compare_state(rs[0], oracle_dense(vol, M, bg=321, tau=900))


def test_overlapped_host_uploads_interleaved_with_renders():
    """VR_HOST_ASYNC: pinned host blocks of changing sizes uploaded on the library's upload
    stream while renders are queued between the inserts; the state equals the oracle's."""
    import ctypes

    import torch
    from paper_1407_2074_b300 import vr as V

    w = S.tiny()
    vol = w.spec().volume()
    r = _renderer(w.dims, 3, 16, tau=2000)
    r.set_transfer_functions(torch.from_numpy(w.tf()).cuda(), torch.ones(3, device="cuda"))
    cam = dict(w.cameras[0])
    img = torch.empty((cam["height"], cam["width"], 4), device="cuda")
    keep = []
    z = 0
    for n in (1, 4, 2, 8, 3, 16, 5, 25):  # staging buffers grow and alternate
        h = torch.empty((n, 64, 64, 3), dtype=torch.int16, pin_memory=True)
        h.numpy()[:] = vol[z:z + n].view(np.int16)
        keep.append((h, r.insert_block((0, 0, z), h.numpy(), overlap=True)))
        r.render([cam], [img])
        z += n
    assert z == 64
    torch.cuda.synchronize()
    _compare_state(r, oracle_dense(vol, 16, tau=2000))
    blk = np.zeros((1, 2, 2, 3), np.uint16)
    st = r._ctx
    with pytest.raises(V.VRError):
        r._check(V.lib().vr_insert_block(st, (ctypes.c_int64 * 3)(0, 0, 0), (ctypes.c_int64 * 3)(2, 2, 1),
                                         ctypes.c_void_p(blk.ctypes.data), 3, None))


def test_pool_exhaustion_status():
    from paper_1407_2074_b300 import vr as V

    w = S.tiny()
    vol = w.spec().volume()
    slot = 18 ** 3 * 4 * 2
    r = _renderer(w.dims, 3, 16, pool_capacity_bytes=25 * slot)
    r.insert_slice(0, vol[0])  # 16 + 4 + 1 = 21 slots
    before = r.read_level(0).copy()
    with pytest.raises(V.VRError) as ei:
        r.insert_slice(20, vol[20])  # needs 16 more leaf slots
    assert ei.value.status == V.VR_ERR_OUT_OF_MEMORY
    assert np.array_equal(r.read_level(0), before)
    assert r.stats().slots_used == 21
    r.insert_slice(1, vol[1])  # the context is still usable


def test_invalid_slice_index():
    from paper_1407_2074_b300 import vr as V

    r = _renderer((16, 16, 16), 3, 8)
    with pytest.raises(V.VRError) as ei:
        r.insert_slice(16, np.zeros((16, 16, 3), np.uint16))
    assert ei.value.status == V.VR_ERR_INVALID_ARG
    with pytest.raises(V.VRError):
        r.insert_block((10, 0, 0), np.zeros((1, 1, 7, 3), np.uint16))


def test_streamed_full_size_sampled_bricks():
    """The 1024x1024x512 streamed workload at full size: every slice inserted from the device
    generator; sampled voxels of every level bit-exact against the lazy oracle."""
    import torch

    w = S.streamed()
    spec = w.spec()
    X, Y, Z = w.dims
    r = _renderer(w.dims, 3, 32, tau=w.tau)
    buf = torch.empty((8, Y, X, 3), dtype=torch.int16, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for z0 in range(0, Z, 8):
        spec.generate_device(buf.data_ptr(), z0, z0 + 8, st)
        r.insert_block((0, 0, z0), buf)
    torch.cuda.synchronize()
    lazy = O.LazyVolume(w.dims, 3, 32, spec.voxel_fn, spec.handle, 0, Z, tau=0, owner=spec)
    rng = np.random.default_rng(11)
    for L in range(lazy.N + 1):
        dims_L = lazy.level_dims(L)
        n = 300 if L < 2 else 120
        xyz = np.stack([rng.integers(0, d, size=n) for d in dims_L], -1)
        got = r.read_voxels(L, xyz)
        ref = np.array([[lazy.value(L, int(x), int(y), int(z), c) for c in range(3)] for x, y, z in xyz])
        assert np.array_equal(got, ref), f"level {L}"
