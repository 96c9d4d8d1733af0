"""Device memory through PyTorch: by default a Renderer hands the library PyTorch's caching
allocator (vr_allocator), so the brick pool, node tables and render buffers are torch's memory,
returned to torch when the context is destroyed.  With allocator=None the library allocates
itself and torch's count does not move."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_pool_and_tables_come_from_torch():
    import torch
    import paper_1407_2074_b300 as vr

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    r = vr.Renderer((96, 80, 64), 3, 16, tau=0)
    st = r.stats()
    held = torch.cuda.memory_allocated() - before
    assert held >= st.pool_bytes + st.node_table_bytes
    # a render allocates its camera and tile-order buffers through torch as well, and works
    vol = np.random.default_rng(0).integers(0, 65535, size=(64, 80, 96, 3), dtype=np.uint16)
    r.insert_block((0, 0, 0), vol)
    from synth import synth as S

    w = S.tiny()
    r.set_transfer_functions(torch.from_numpy(w.tf()), torch.ones(3))
    cam = dict(w.cameras[0], width=64, height=48)
    img = r.render([cam])[0]
    torch.cuda.synchronize()
    assert torch.isfinite(img).all() and img[..., 3].max() > 0
    in_use = torch.cuda.memory_allocated()
    assert in_use - before > held
    r.close()
    torch.cuda.synchronize()
    # everything the context held went back to torch (the image and tables the test made remain)
    assert in_use - torch.cuda.memory_allocated() >= held
    del img
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() - before < 64 * 1024


def test_library_allocator_leaves_torch_alone():
    import torch
    import paper_1407_2074_b300 as vr

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    r = vr.Renderer((64, 64, 64), 3, 16, allocator=None)
    assert torch.cuda.memory_allocated() == before
    r.close()
    with pytest.raises(ValueError):
        vr.Renderer((64, 64, 64), 3, 16, allocator="cuda")
