"""The overlapped host pipeline (serve.CloudPipeline) returns, for every cloud of a
sequence, exactly the plain call's rows, in order, whatever the depth (including a
three-point and an empty cloud)."""
import numpy as np
import pytest
import torch

from paper_2102_11084_gb300 import serve, synth, vg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth", [2, 3])
def test_pipeline_equals_plain_calls(depth):
    clouds = [synth.rgbd_frame(640, 480, seed=70 + k) for k in range(3)]
    clouds += [synth.random_cloud(50_000, seed=5, extent=3.0), synth.rgbd_frame(320, 240, seed=9)]
    clouds += [synth.random_cloud(3, seed=6, extent=1.0), np.zeros((0, 3), np.float32)]
    pinned = [torch.from_numpy(c).pin_memory() for c in clouds]
    pipe = serve.CloudPipeline(max(c.shape[0] for c in clouds), 0.05, depth=depth)
    got = [(k.copy(), c.copy(), n.copy()) for k, c, n in pipe.run(pinned)]
    assert len(got) == len(clouds)
    for (k, c, n), x in zip(got, clouds):
        ref = vg.downsample(torch.from_numpy(x).cuda(), 0.05)
        assert np.array_equal(k, ref.keys.cpu().numpy().view(np.uint64))
        assert np.array_equal(n, ref.counts.cpu().numpy().view(np.uint32))
        assert np.array_equal(c, ref.centroids.cpu().numpy())
