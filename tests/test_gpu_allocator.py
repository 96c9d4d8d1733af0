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


def test_process_exit_with_live_renderer_and_plan(tmp_path):
    """A script that leaves a Renderer and a render plan alive until the interpreter exits ends
    cleanly: the contexts still open are destroyed at exit (their memory goes back to torch while
    torch is still up), each after its plans."""
    import subprocess
    import sys

    root = __import__("os").path.dirname(__import__("os").path.dirname(__file__))
    script = tmp_path / "live.py"
    script.write_text(
        "import sys\n"
        f"sys.path.insert(0, {root!r})\n"
        "import numpy as np, torch\n"
        "import paper_1407_2074_b300 as vr\n"
        "from synth import synth as S\n"
        "w = S.tiny()\n"
        "r = vr.Renderer(w.dims, 3, 16)\n"
        "r.insert_block((0, 0, 0), w.spec().volume())\n"
        "r.set_transfer_functions(torch.from_numpy(w.tf()), torch.ones(3))\n"
        "cam = dict(w.cameras[0], width=32, height=32)\n"
        "p = r.plan([cam])\n"
        "p.launch()\n"
        "torch.cuda.synchronize()\n"
        "print('ok')\n")
    res = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    assert res.stdout.strip().endswith("ok")
