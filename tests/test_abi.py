"""The C ABI library: it loads, exports every declared symbol, and rejects
bad arguments on the host before touching the GPU (CPU only)."""
import math
import os
import re

import numpy as np
import pytest

import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    rtb_build.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rtb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 16
    L = rtb.lib()
    for n in names:
        assert hasattr(L, n), n


def test_abi_version_and_defaults():
    assert rtb.rt_abi_version() == 1
    o = rtb.rt_render_options_default()
    assert o.use_bvh == 1 and o.flags == 0 and o.queue_capacity == 0
    assert list(o.background) == pytest.approx([0.1, 0.1, 0.1])
    assert o.eps_scale == pytest.approx(1e-4)
    assert o.ray_counts is None


def test_struct_sizes_match_header_layout():
    assert S.SPHERE_DTYPE.itemsize == 20 and S.TRIANGLE_DTYPE.itemsize == 40
    assert S.MATERIAL_DTYPE.itemsize == 44 and S.LIGHT_DTYPE.itemsize == 24
    import ctypes
    assert ctypes.sizeof(rtb.rt_camera) == S.CAMERA_DTYPE.itemsize == 40
    assert ctypes.sizeof(rtb.rt_render_options) == 48   # ... traversal_cap, then the ray_counts pointer
    assert ctypes.sizeof(rtb.rt_tune) == 16
    assert ctypes.sizeof(rtb.rt_pass) == 24


def _base():
    sc = S.scene_spheres8()
    return sc.spheres.copy(), sc.triangles.copy(), sc.materials.copy(), sc.lights.copy()


@pytest.mark.parametrize("what", ["nan_center", "inf_vertex", "zero_radius", "neg_radius", "bad_sphere_mat",
                                  "bad_tri_mat", "no_materials", "bad_kind"])
def test_scene_create_rejects_bad_input_on_host(what):
    sph, tri, mats, li = _base()
    if what == "nan_center":
        sph["center"][0, 1] = np.nan
    elif what == "inf_vertex":
        tri["v1"][1, 2] = np.inf
    elif what == "zero_radius":
        sph["radius"][3] = 0.0
    elif what == "neg_radius":
        sph["radius"][3] = -1.0
    elif what == "bad_sphere_mat":
        sph["material"][2] = len(mats)
    elif what == "bad_tri_mat":
        tri["material"][0] = 99
    elif what == "no_materials":
        mats = mats[:0]
    elif what == "bad_kind":
        mats["kind"][1] = 7
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_scene_create(sph, tri, mats, li)
    assert ei.value.status == rtb.RT_ERR_INVALID_ARG
    assert rtb.rt_last_error()


def test_null_handles_rejected():
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_bvh_build(None, 0)
    assert ei.value.status == rtb.RT_ERR_INVALID_ARG
    assert rtb.lib().rt_scene_sync(None, None) == rtb.RT_ERR_INVALID_ARG
    assert rtb.lib().rt_scene_destroy(None) == rtb.RT_OK


def test_camera_validation_on_host():
    import ctypes
    cam = rtb.make_camera(S.camera((0, 0, 5), (0, 0, 5)))        # eye == look_at
    st = rtb.lib().rt_camera_rays(ctypes.byref(cam), 4, 4, 1, 1, None)
    assert st == rtb.RT_ERR_INVALID_ARG
    cam = rtb.make_camera(S.camera((0, 0, 5), (0, 0, 0), up=(0, 0, 1)))   # up parallel to view
    assert rtb.lib().rt_camera_rays(ctypes.byref(cam), 4, 4, 1, 1, None) == rtb.RT_ERR_INVALID_ARG
    cam = rtb.make_camera(S.camera((0, 0, 5), (0, 0, 0), vfov_deg=math.nan))
    assert rtb.lib().rt_camera_rays(ctypes.byref(cam), 4, 4, 1, 1, None) == rtb.RT_ERR_INVALID_ARG
