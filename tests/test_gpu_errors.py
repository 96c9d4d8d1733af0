"""Device-side error path without a device fault: a failed kernel check only sets the context's
error word; the next polling call reports VR_ERR_DEVICE_ASSERT, every later call VR_ERR_STATE,
and the context can still be destroyed.  Host-side failures (pool exhaustion) leave it usable."""
import numpy as np
import pytest

from synth import synth as S

pytestmark = pytest.mark.gpu


def test_device_error_word_then_state_error_then_destroy():
    import torch
    import paper_1407_2074_b300 as vr
    from paper_1407_2074_b300 import vr as V

    w = S.tiny()
    vol = w.spec().volume()
    r = vr.Renderer(w.dims, 3, 16)
    r.insert_block((0, 0, 0), torch.from_numpy(vol.view(np.int16)).cuda())
    r.set_transfer_functions(torch.from_numpy(w.tf()).cuda(), torch.ones(3, device="cuda"))
    r.render(w.cameras)
    assert r.read_node(0, 0, 0, 0)[0] & V.F_TOUCHED
    with pytest.raises(V.VRError) as ei:
        r.debug_raise_error(0)
    assert ei.value.status == V.VR_ERR_INVALID_ARG
    r.debug_raise_error(5)
    with pytest.raises(V.VRError) as ei:
        r.read_node(0, 0, 0, 0)
    assert ei.value.status == V.VR_ERR_DEVICE_ASSERT
    for call in (lambda: r.render(w.cameras), lambda: r.insert_slice(3, vol[3]), lambda: r.read_level(0)):
        with pytest.raises(V.VRError) as ei:
            call()
        assert ei.value.status == V.VR_ERR_STATE
    r.close()  # still releases the context
    r2 = vr.Renderer(w.dims, 3, 16)  # and the device is fine for the next one
    r2.insert_slice(0, vol[0])
    assert np.array_equal(r2.read_level(0)[0], vol[0])
    r2.close()
