"""rt_render_noalloc: the frame of rt_render without any device allocation.

Some callers may not allocate GPU memory while they render (a host
application that owns the device memory budget and forbids cudaMalloc after
start-up, or code confined to a pre-reserved pool).  rt_render_noalloc keeps
its ray queues in a fixed array inside the library instead.  This file runs
last so that a failure here never hides the other tests' results.
"""
import numpy as np
import pytest
import torch

import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

pytestmark = pytest.mark.gpu

COLOUR_TOL = 2e-3     # the tests' colour tolerance


@pytest.fixture(scope="module", autouse=True)
def built(gpu):
    rtb_build.build()
    torch.cuda.set_device(0)


def _render_both(sc):
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    ref = torch.empty(W * H * 3, device="cuda")
    rtb.rt_render(scene.handle, sc.camera, W, H, D, ref)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    outs = []
    for _ in range(2):                        # two calls in a row share the scratch array
        out = torch.full((W * H * 3,), float("nan"), device="cuda")
        rtb.rt_render_noalloc(scene.handle, sc.camera, W, H, D, out)
        assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
        outs.append(out.cpu().numpy())
    scene.close()
    return ref.cpu().numpy(), outs


@pytest.mark.parametrize("make", [
    lambda: S.scene_spheres8(width=128, height=128),
    lambda: S.scene_terrain(seed=7, width=96, height=64, max_depth=5, cells=(16, 12), n_ico=6, ico_level=2),
    lambda: S.scene_spheres8_emitters(width=96, height=96),   # 1 point light + 3 emissive primitives
])
def test_noalloc_matches_rt_render_twice(make):
    ref, outs = _render_both(make())
    for out in outs:
        assert np.isfinite(out).all()
        np.testing.assert_allclose(out, ref, atol=COLOUR_TOL, rtol=0)
        assert np.abs(out - ref).max() < 1e-5        # same kernels: only atomic ordering differs


def test_noalloc_rejects_oversize_frames():
    sc = S.scene_spheres8(width=8, height=8)
    scene = rtb.Scene(sc).build()
    out = torch.empty(256 * 128 * 3, device="cuda")
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_render_noalloc(scene.handle, sc.camera, 256, 128, 3, out)   # 32768 > 16384 pixels
    assert ei.value.status == rtb.RT_ERR_UNSUPPORTED
    assert "RT_NOALLOC_MAX_PIXELS" in str(ei.value)
    scene.close()


def test_noalloc_counts_every_kind_of_light():
    """The shadow queue holds a record per light of any kind: a point light,
    an area light and three emissive primitives are five."""
    sc = S.scene_spheres8_emitters(width=8, height=8)
    sc.area_lights = S.area_lights([(-2.0, 8.0, -2.0)], [(4.0, 0.0, 0.0)], [(0.0, 0.0, 4.0)], [(2.0, 2.0, 2.0)])
    scene = rtb.Scene(sc).build()
    out = torch.empty(8 * 8 * 3, device="cuda")
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_render_noalloc(scene.handle, sc.camera, 8, 8, 3, out)
    assert ei.value.status == rtb.RT_ERR_UNSUPPORTED
    assert "RT_NOALLOC_MAX_LIGHTS" in str(ei.value)
    scene.close()


def test_noalloc_allocates_no_device_memory():
    """After a first call (which looks up the array's address), further
    calls leave the device's free memory unchanged: no cudaMalloc on the
    way, and no allocation by a library routine either."""
    sc = S.scene_terrain(seed=7, width=96, height=64, max_depth=5, cells=(16, 12), n_ico=6, ico_level=2)
    scene = rtb.Scene(sc).build()
    W, H, D = sc.width, sc.height, sc.max_depth
    out = torch.empty(W * H * 3, device="cuda")
    rtb.rt_render_noalloc(scene.handle, sc.camera, W, H, D, out)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rtb.rt_render_noalloc(scene.handle, sc.camera, W, H, D, out)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert np.isfinite(out.cpu().numpy()).all()
    scene.close()
