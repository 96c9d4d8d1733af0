"""The device input generator is bit-identical to the host generator (same counter-based
definition, IEEE-rounded single operations only)."""
import numpy as np
import pytest

from synth import synth as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,dims,count", [(S.KIND_BLOBS, (64, 64, 64), 20), (S.KIND_SPIM, (200, 150, 90), 300)])
def test_device_generator_matches_host(kind, dims, count):
    import torch

    spec = S.VolumeSpec(kind, dims, 3, count, seed=1)
    X, Y, Z = dims
    host = spec.box(0, X, 0, Y, 0, Z)
    dev = torch.empty((Z, Y, X, 3), dtype=torch.uint16, device="cuda")
    spec.generate_device(dev.data_ptr(), 0, Z, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)


def test_device_generator_full_size_samples():
    import torch

    w = S.large()
    spec = w.spec()
    X, Y, Z = w.dims
    rng = np.random.default_rng(3)
    for z in rng.integers(0, Z, size=3):
        dev = torch.empty((1, Y, X, 3), dtype=torch.uint16, device="cuda")
        spec.generate_device(dev.data_ptr(), int(z), int(z) + 1, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        d = dev.cpu().numpy()[0]
        ys, xs = rng.integers(0, Y, size=200), rng.integers(0, X, size=200)
        host = spec.voxels(np.stack([xs, ys, np.full(200, z)], -1))
        assert np.array_equal(d[ys, xs], host)
