"""Progressive passes on the GPU: area lights and emissive primitives
sampled once per pass and pixel jitter (Alg. 1, Sec. IV.A, Eq. 7-8),
against the oracle's passes (same Philox4x32-10 samples) and against
closed forms."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

from gpu_helpers import BUDGET, COLOUR_TOL, compare, gpu_render

import test_oracle_pass as P   # the closed-form scenes and Lambert's formula

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(gpu):
    rtb_build.build()
    torch.cuda.set_device(0)


def gpu_passes(sc, passes, strata, seed=3, jitter=False, depth=None, flags=0):
    scene = rtb.Scene(sc).build()
    D = sc.max_depth if depth is None else depth
    acc = torch.full((sc.width * sc.height * 3,), float("nan"), device="cuda")
    opts = rtb.make_options(background=sc.background, flags=flags)
    for k in range(passes):
        rtb.rt_render_pass(scene.handle, sc.camera, sc.width, sc.height, D, rtb.make_pass(k, seed, strata, jitter),
                           acc, opts)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    img = acc.view(-1, 3).double().cpu().numpy()
    scene.close()
    return img


def oracle_passes(sc, passes, strata, seed=3, jitter=False, depth=None):
    orc = O.OracleScene.from_scene(sc)
    D = sc.max_depth if depth is None else depth
    acc, robust = None, None
    for k in range(passes):
        orc.set_pass(seed, k, strata, jitter)
        r = orc.render(sc.camera, sc.width, sc.height, D, mode="bvh")
        acc = r["rgb"] if acc is None else acc + (r["rgb"] - acc) / (k + 1)
        robust = r["robust"] if robust is None else np.minimum(robust, r["robust"])
    return acc, robust


def check_colour(img, ref, robust):
    err = np.abs(img - ref).max(axis=1)
    assert np.isfinite(img).all()
    assert not ((err > COLOUR_TOL) & (robust >= 1)).any(), np.where((err > COLOUR_TOL) & (robust >= 1))[0][:10]
    assert (err > COLOUR_TOL).mean() <= BUDGET


def test_first_pass_with_an_area_light_matches_oracle():
    """rt_render_ex renders pass 0 of seed 0: hits, depths and area-light
    samples as the oracle's pass 0."""
    sc = S.scene_spheres8_area(width=64, height=48, max_depth=3)
    orc = O.OracleScene.from_scene(sc)
    orc.set_pass(0, 0, 1, False)
    ref = orc.render(sc.camera, sc.width, sc.height, sc.max_depth, mode="bvh")
    compare(gpu_render(sc), ref)


@pytest.mark.parametrize("flags", [0, rtb.RT_FLAG_PER_DEPTH_WAVEFRONT])
def test_progressive_passes_match_oracle(flags):
    sc = S.scene_spheres8_area(width=48, height=40, max_depth=3)
    img = gpu_passes(sc, 16, 4, seed=11, jitter=True, flags=flags)
    ref, robust = oracle_passes(sc, 16, 4, seed=11, jitter=True)
    check_colour(img, ref, robust)


def test_area_light_converges_to_lambert_on_gpu():
    sc = P.plane_under_light((1.0, 2.0, -1.5), (2.0, 0.5, 0.0), (0.0, 0.0, 3.0), L=(2.0, 1.0, 0.5))
    c = np.array((1.0, 2.0, -1.5))
    E = P.polygon_irradiance(np.zeros(3), np.array([0.0, 1.0, 0.0]),
                             [c, c + (2.0, 0.5, 0.0), c + (2.0, 0.5, 3.0), c + (0.0, 0.0, 3.0)])
    img = gpu_passes(sc, 1024, 32, depth=0)
    centre = (sc.height // 2) * sc.width + sc.width // 2
    np.testing.assert_allclose(img[centre], 0.5 * np.array([2.0, 1.0, 0.5]) * E, rtol=2e-3)


def test_jitter_converges_to_edge_coverage_on_gpu():
    W = H = 9
    hfov, d = 20.0, 10.0
    px = 2 * np.tan(np.radians(hfov) / 2) / H * d
    xe = (-0.5 + 0.3) * px
    mats = S.material(S.MAT_DIFFUSE, (0.6, 0.6, 0.6), ks=0.0)
    tris = S.triangles_from([(xe - 100, -100, 0), (xe - 100, -100, 0)], [(xe, -100, 0), (xe, 100, 0)],
                            [(xe, 100, 0), (xe - 100, 100, 0)], 0)
    sc = S.Scene("edge", np.zeros(0, S.SPHERE_DTYPE), tris, mats, S.lights([(0.0, 0.0, 1e4)], [(1.0, 1.0, 1.0)]),
                 S.camera((0.0, 0.0, d), (0.0, 0.0, 0.0), vfov_deg=hfov), W, H, 0)
    img = gpu_passes(sc, 1024, 32, jitter=True)
    centre = (H // 2) * W + W // 2
    np.testing.assert_allclose(img[centre], 0.3 * 0.6 + 0.7 * 0.1, atol=3e-3)


def test_terrain_with_area_lights_pass_parity():
    """The bench terrain (small) with two area lights over it, a few
    jittered passes, depth 3."""
    sc = S.scene_terrain(seed=7, width=80, height=48, max_depth=3, cells=(16, 12), n_ico=6, ico_level=2)
    sc.area_lights = S.area_lights([(-20.0, 15.0, -10.0), (5.0, 12.0, 0.0)], [(8.0, 0.0, 0.0), (0.0, 0.0, 6.0)],
                                   [(0.0, 0.0, 8.0), (6.0, -1.0, 0.0)], [(1.5, 1.5, 1.2), (0.4, 0.6, 1.0)])
    img = gpu_passes(sc, 4, 2, seed=5, jitter=True)
    ref, robust = oracle_passes(sc, 4, 2, seed=5, jitter=True)
    check_colour(img, ref, robust)


def test_batch_with_area_lights_matches_single_frames():
    sc = S.scene_spheres8_area(width=40, height=32, max_depth=3)
    scene = rtb.Scene(sc).build()
    out = torch.empty(40 * 32 * 3, device="cuda")
    ref = torch.empty(40 * 32 * 3, device="cuda")
    b = rtb.Batch([scene], [sc.camera], [40], [32], 3, [out], rtb.make_options(background=sc.background))
    b.render()
    rtb.rt_render_ex(scene.handle, sc.camera, 40, 32, 3, ref, rtb.make_options(background=sc.background))
    torch.cuda.synchronize()
    err = (out - ref).abs().view(-1, 3).max(dim=1).values
    assert (err > 1e-5).float().mean().item() <= 1e-3
    b.close()
    scene.close()


def test_emissive_quad_converges_to_lambert_on_gpu():
    c = np.array((1.0, 2.0, -1.5))
    eu, ev = np.array((2.0, 0.5, 0.0)), np.array((0.0, 0.0, 3.0))
    quad = S.triangles_from([c, c], [c + eu, c + eu + ev], [c + eu + ev, c + ev], 1)
    sc = P.floor_with_emitters(tris=quad, L=(2.0, 1.0, 0.5))
    E = P.polygon_irradiance(np.zeros(3), np.array([0.0, 1.0, 0.0]), [c, c + eu, c + eu + ev, c + ev])
    img = gpu_passes(sc, 1024, 32, depth=0)
    centre = (sc.height // 2) * sc.width + sc.width // 2
    np.testing.assert_allclose(img[centre], 0.5 * np.array([2.0, 1.0, 0.5]) * E, rtol=3e-3)


def test_emissive_sphere_converges_to_its_solid_angle_on_gpu():
    r, d = 0.6, 3.0
    sph = S.spheres_from([(0.0, d, 0.0)], [r], [1])
    sc = P.floor_with_emitters(spheres=sph, L=(1.0, 0.5, 0.25))
    sc.camera = S.camera((0.0, 1.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=10.0)
    img = gpu_passes(sc, 1024, 32, depth=0)
    centre = (sc.height // 2) * sc.width + sc.width // 2
    np.testing.assert_allclose(img[centre], 0.5 * np.array([1.0, 0.5, 0.25]) * np.pi * (r / d) ** 2, rtol=5e-3)
    # seen directly, the sphere shows its own emission (Eq. 7); it does not light itself
    sc.camera = S.camera((0.0, 10.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=2.0)
    top = gpu_render(sc, max_depth=0)["rgb"][centre]
    np.testing.assert_allclose(top, (1.0, 0.5, 0.25), atol=1e-6)


def test_first_pass_with_emitters_matches_oracle():
    """Pass 0 of seed 0 with an emissive sphere, an emissive quad and a
    glass sphere: hits, depths and emitter samples as the oracle's."""
    sc = S.scene_spheres8_emitters(width=64, height=48, max_depth=3)
    orc = O.OracleScene.from_scene(sc)
    orc.set_pass(0, 0, 1, False)
    ref = orc.render(sc.camera, sc.width, sc.height, sc.max_depth, mode="bvh")
    # shadow rays that end on a sampled point of an emitter's own surface
    # (an eps short of it) make 5.1 % of this frame's pixels rounding-fragile
    compare(gpu_render(sc), ref, fragile_budget=0.06)


@pytest.mark.parametrize("flags", [0, rtb.RT_FLAG_PER_DEPTH_WAVEFRONT])
def test_emitter_passes_match_oracle(flags):
    sc = S.scene_spheres8_emitters(width=48, height=40, max_depth=3)
    img = gpu_passes(sc, 8, 2, seed=11, jitter=True, flags=flags)
    ref, robust = oracle_passes(sc, 8, 2, seed=11, jitter=True)
    check_colour(img, ref, robust)


def test_emitters_with_area_lights_pass_parity():
    """Area lights take the first sample slots, emitters the next: both kinds
    in one scene."""
    sc = S.scene_spheres8_emitters(width=40, height=32, max_depth=2)
    sc.area_lights = S.area_lights([(-2.0, 8.0, -2.0)], [(4.0, 0.0, 0.0)], [(0.0, 0.0, 4.0)], [(2.0, 2.0, 2.0)])
    img = gpu_passes(sc, 4, 2, seed=2)
    ref, robust = oracle_passes(sc, 4, 2, seed=2)
    check_colour(img, ref, robust)


def test_batch_with_emitters_matches_single_frames():
    sc = S.scene_spheres8_emitters(width=40, height=32, max_depth=3)
    scene = rtb.Scene(sc).build()
    out = torch.empty(40 * 32 * 3, device="cuda")
    ref = torch.empty(40 * 32 * 3, device="cuda")
    b = rtb.Batch([scene], [sc.camera], [40], [32], 3, [out], rtb.make_options(background=sc.background))
    b.render()
    rtb.rt_render_ex(scene.handle, sc.camera, 40, 32, 3, ref, rtb.make_options(background=sc.background))
    torch.cuda.synchronize()
    err = (out - ref).abs().view(-1, 3).max(dim=1).values
    assert (err > 1e-5).float().mean().item() <= 1e-3
    b.close()
    scene.close()


def test_pass_argument_errors():
    sc = S.scene_spheres8_area(width=16, height=16, max_depth=1)
    scene = rtb.Scene(sc).build()
    acc = torch.empty(16 * 16 * 3, device="cuda")
    for bad in [rtb.rt_pass(0, -1, 1, 0, 0), rtb.rt_pass(0, 0, 0, 0, 0), rtb.rt_pass(0, 0, 1, 0, 7)]:
        with pytest.raises(rtb.RtError):
            rtb.rt_render_pass(scene.handle, sc.camera, 16, 16, 1, bad, acc)
    for bad in [S.area_lights([(0, 0, 0)], [(1, 0, 0)], [(2, 0, 0)], [(1, 1, 1)]),            # degenerate
                S.area_lights([(0, 0, 0)], [(1, 0, 0)], [(0, 0, 1)], [(-1, 1, 1)]),           # negative radiance
                S.area_lights([(np.nan, 0, 0)], [(1, 0, 0)], [(0, 0, 1)], [(1, 1, 1)])]:      # not finite
        with pytest.raises(rtb.RtError):
            rtb.rt_scene_set_area_lights(scene.handle, bad)
    rtb.rt_scene_set_area_lights(scene.handle, np.zeros(0, S.AREA_LIGHT_DTYPE))   # none: allowed
    scene.close()
