"""Error containment: once the key kernel has set the device error word (a point whose
voxel index leaves [0, 2^21)), every later step of the call returns at once -- the
grouping (both layouts, every method), the reduction, the minimum-count filter, the
pyramid merge and the thinning loop -- and the call reports the error.  A later clean
call on the same process then gives the oracle's rows again.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import assert_decimation_equal

pytestmark = pytest.mark.gpu

FAR = np.float32(1.0e7)  # ~2e8 leaves from the minimum: beyond the 21-bit index range


def with_outlier(xyz):
    bad = np.array(xyz, np.float32, copy=True)
    i = len(bad) // 2
    bad[i] = (FAR, 0.0, 0.0)
    return bad


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.fixture(scope="module")
def clouds():
    # 307,200 points takes the global radix sort under "auto"; 4.5M the bucket grouping
    return {"rgbd": synth.rgbd_frame(640, 480, seed=11),
            "map": synth.fused_map(4_500_000, seed=11)}


@pytest.mark.parametrize("cloud", ["rgbd", "map"])
@pytest.mark.parametrize("method", ["auto", "sort", "sort_lsd", "hash", "frame"])
@pytest.mark.parametrize("extra", [{}, {"point_to_voxel": True}, {"min_count": 2}])
def test_range_error_stops_later_steps(clouds, cloud, method, extra):
    xyz = clouds[cloud]
    with pytest.raises(vg.VGError) as e:
        vg.downsample(cuda(with_outlier(xyz)), 0.02, method=method, **extra)
    assert e.value.status == vg.Status.RANGE
    # the next call on a clean cloud is unaffected
    if cloud == "rgbd":
        res = vg.downsample(cuda(xyz), 0.02, method=method, point_to_voxel=True)
        assert_decimation_equal(res, oracle.downsample(xyz, 0.02))


@pytest.mark.parametrize("cloud", ["rgbd", "map"])
def test_range_error_stops_the_pyramid(clouds, cloud):
    with pytest.raises(vg.VGError) as e:
        vg.pyramid(cuda(with_outlier(clouds[cloud])), 0.02, 4, point_to_voxel=True)
    assert e.value.status == vg.Status.RANGE


def test_range_error_stops_the_frames_call(clouds):
    xyz = clouds["rgbd"]
    frames = [cuda(xyz), cuda(with_outlier(xyz)), cuda(xyz)]
    with pytest.raises(vg.VGError) as e:
        vg.downsample_frames(frames, [0.02, 0.02, 0.02], point_to_voxel=True)
    assert e.value.status == vg.Status.RANGE


def test_range_error_stops_the_thinning_loop(clouds):
    xyz = with_outlier(clouds["rgbd"])
    prio = torch.arange(len(xyz), dtype=torch.int32, device="cuda")
    with pytest.raises(vg.VGError) as e:
        vg.thin(cuda(xyz), 0.05, 20, prio)
    assert e.value.status == vg.Status.RANGE
