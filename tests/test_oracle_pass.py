"""Pins of the oracle's progressive passes: area lights sampled once per
pass (Alg. 1, Sec. IV.A) and pixel jitter, converging to closed forms.

The counter-based generator (Philox4x32-10) is pinned by its statistics;
the estimators are pinned by Lambert's closed form for the light a point
receives from a polygon, and by the coverage of a pixel cut by an edge."""
import numpy as np
import pytest

import oracle as O
from paper_1504_03151_b300 import scenes as S


def u24(x):
    return (np.asarray(x, np.uint64) >> 8).astype(np.float64) / 16777216.0


def test_philox_statistics_and_sensitivity():
    key = (0x1234567, 0x89ABCDEF)
    vals = np.array([O.philox4x32((i, 7, 3, 1), key) for i in range(4096)])   # 16,384 words
    u = u24(vals.reshape(-1))
    n = len(u)
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 0.01
    hist = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 120          # 63 degrees of freedom; p ~ 1e-5
    # serial correlation of consecutive counters
    assert abs(np.corrcoef(u[:-4:4], u[4::4])[0, 1]) < 0.05
    # one input bit changes about half of the 128 output bits (counter and key)
    base = O.philox4x32((5, 6, 7, 8), key)
    for ctr, k in [((4, 6, 7, 8), key), ((5, 6, 7, 8 | (1 << 31)), key), ((5, 6, 7, 8), (key[0] ^ 1, key[1]))]:
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, O.philox4x32(ctr, k)))
        assert 40 <= flips <= 88


def polygon_irradiance(x, n, verts):
    """Lambert's formula: the integral over a polygon (vertices in order) of
    cos(theta_x) cos(theta_y) / r^2 dA, seen from point x with normal n, for
    a polygon facing x: (1/2) sum_i beta_i (n . g_i), beta_i the angle the
    edge i subtends at x and g_i the unit normal of the plane through x and
    that edge."""
    tot = 0.0
    m = len(verts)
    for i in range(m):
        a = np.asarray(verts[i], float) - x
        b = np.asarray(verts[(i + 1) % m], float) - x
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        beta = np.arccos(np.clip(a @ b, -1, 1))
        g = np.cross(a, b)
        g /= np.linalg.norm(g)
        tot += beta * (n @ g)
    return abs(tot) / 2


def plane_under_light(corner, eu, ev, L=(1.0, 1.0, 1.0), albedo=(0.5, 0.5, 0.5), W=9, H=9):
    """A large diffuse floor (ks = 0) at y = 0, no point light, one area
    light; the camera looks straight down so that the centre pixel's ray
    hits the floor at the origin."""
    mats = S.material(S.MAT_DIFFUSE, albedo, ks=0.0)
    tris = S.triangles_from([(-50, 0, -50), (-50, 0, -50)], [(-50, 0, 50), (50, 0, 50)],
                            [(50, 0, 50), (50, 0, -50)], 0)
    cam = S.camera((0.0, 20.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=10.0)
    sc = S.Scene("floor_area", np.zeros(0, S.SPHERE_DTYPE), tris, mats, np.zeros(0, S.LIGHT_DTYPE), cam, W, H, 0)
    sc.area_lights = S.area_lights([corner], [eu], [ev], [L])
    return sc


def progressive(orc, sc, passes, strata, seed=3, jitter=False, pixels=None, depth=None):
    acc = None
    for k in range(passes):
        orc.set_pass(seed, k, strata, jitter)
        r = orc.render(sc.camera, sc.width, sc.height, sc.max_depth if depth is None else depth, mode="brute",
                       pixels=pixels)["rgb"]
        acc = r if acc is None else acc + (r - acc) / (k + 1)
    return acc


@pytest.mark.parametrize("corner,eu,ev", [
    ((-2.0, 3.0, -2.0), (4.0, 0.0, 0.0), (0.0, 0.0, 4.0)),          # centred square, facing down
    ((1.0, 2.0, -1.5), (2.0, 0.5, 0.0), (0.0, 0.0, 3.0)),           # off to the side, tilted
])
def test_area_light_converges_to_lambert(corner, eu, ev):
    sc = plane_under_light(corner, eu, ev, L=(2.0, 1.0, 0.5))
    orc = O.OracleScene.from_scene(sc)
    c = np.array(corner, float)
    verts = [c, c + eu, c + np.add(eu, ev), c + ev]
    E = polygon_irradiance(np.zeros(3), np.array([0.0, 1.0, 0.0]), verts)
    centre = np.array([(sc.height // 2) * sc.width + sc.width // 2])
    got = progressive(orc, sc, passes=1024, strata=32, pixels=centre)[0]
    want = 0.5 * np.array([2.0, 1.0, 0.5]) * E
    np.testing.assert_allclose(got, want, rtol=2e-3)


def test_stratified_passes_beat_independent_ones():
    """Over S x S passes every stratum is visited once: the error of the
    stratified mean is far below that of S x S independent samples."""
    sc = plane_under_light((-2.0, 3.0, -2.0), (4.0, 0.0, 0.0), (0.0, 0.0, 4.0))
    orc = O.OracleScene.from_scene(sc)
    E = polygon_irradiance(np.zeros(3), np.array([0.0, 1.0, 0.0]),
                           [(-2, 3, -2), (-2, 3, 2), (2, 3, 2), (2, 3, -2)])
    centre = np.array([(sc.height // 2) * sc.width + sc.width // 2])
    err_s, err_i = [], []
    for seed in range(6):
        err_s.append(abs(progressive(orc, sc, 64, 8, seed=seed, pixels=centre)[0, 0] - 0.5 * E))
        err_i.append(abs(progressive(orc, sc, 64, 1, seed=seed, pixels=centre)[0, 0] - 0.5 * E))
    assert np.mean(err_s) < 0.3 * np.mean(err_i)


def test_blocked_area_light_adds_nothing():
    sc = plane_under_light((-1.0, 4.0, -1.0), (2.0, 0.0, 0.0), (0.0, 0.0, 2.0))
    blocker = S.triangles_from([(-5, 2, -5), (-5, 2, -5)], [(-5, 2, 5), (5, 2, 5)], [(5, 2, 5), (5, 2, -5)], 0)
    sc.triangles = np.concatenate([sc.triangles, blocker])
    orc = O.OracleScene.from_scene(sc)
    centre = np.array([(sc.height // 2) * sc.width + sc.width // 2])
    # the camera ray meets the blocker first; look at the floor from below the blocker instead
    sc.camera = S.camera((0.0, 1.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=10.0)
    got = progressive(orc, sc, 16, 4, pixels=centre)[0]
    np.testing.assert_allclose(got, 0.0, atol=1e-12)


def test_light_facing_away_adds_nothing():
    sc = plane_under_light((-2.0, 3.0, -2.0), (0.0, 0.0, 4.0), (4.0, 0.0, 0.0))   # normal points up
    orc = O.OracleScene.from_scene(sc)
    centre = np.array([(sc.height // 2) * sc.width + sc.width // 2])
    np.testing.assert_allclose(progressive(orc, sc, 16, 4, pixels=centre)[0], 0.0, atol=1e-12)


def test_pixel_jitter_converges_to_edge_coverage():
    """A lit diffuse half-plane whose edge cuts the centre pixel at 30 % of
    its width: the jittered passes converge to 0.3 shade + 0.7 background."""
    W = H = 9
    hfov = 20.0
    # image plane coordinates of the centre pixel: the edge sits at x = -0.5 + 0.3 pixels from its centre
    h = np.tan(np.radians(hfov) / 2)
    d = 10.0
    px = 2 * h / H * d                                   # one pixel at the plane, distance d
    xe = (-0.5 + 0.3) * px                               # the edge: covered part x < xe (30 % of the pixel)
    mats = S.material(S.MAT_DIFFUSE, (0.6, 0.6, 0.6), ks=0.0)
    tris = S.triangles_from([(xe - 100, -100, 0), (xe - 100, -100, 0)], [(xe, -100, 0), (xe, 100, 0)],
                            [(xe, 100, 0), (xe - 100, 100, 0)], 0)
    light = S.lights([(0.0, 0.0, 1e4)], [(1.0, 1.0, 1.0)])
    cam = S.camera((0.0, 0.0, d), (0.0, 0.0, 0.0), vfov_deg=hfov)
    sc = S.Scene("edge", np.zeros(0, S.SPHERE_DTYPE), tris, mats, light, cam, W, H, 0)
    orc = O.OracleScene.from_scene(sc)
    centre = np.array([(H // 2) * W + W // 2])
    got = progressive(orc, sc, 1024, 32, jitter=True, pixels=centre)[0]
    shade = 0.6 * 1.0   # n.l = 1 for the far light straight ahead
    np.testing.assert_allclose(got, 0.3 * shade + 0.7 * 0.1, atol=3e-3)
    # without jitter the pixel centre decides: background only
    orc.set_pass(0, 0, 1, False)
    np.testing.assert_allclose(orc.render(cam, W, H, 0, mode="brute", pixels=centre)["rgb"][0], 0.1, atol=1e-12)


def test_passes_are_deterministic_and_differ():
    sc = S.scene_spheres8_area(width=24, height=20, max_depth=2)
    orc = O.OracleScene.from_scene(sc)
    orc.set_pass(9, 3, 4, True)
    a = orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"]
    b = orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"]
    np.testing.assert_array_equal(a, b)
    orc.set_pass(9, 4, 4, True)
    c = orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"]
    assert np.abs(a - c).max() > 1e-3
    # the BVH and the iterative form agree with brute force under a pass too
    orc.set_pass(9, 3, 4, True)
    for mode in ("bvh", "iterative"):
        np.testing.assert_allclose(orc.render(sc.camera, sc.width, sc.height, 2, mode=mode)["rgb"], a, atol=1e-12)


def test_passes_change_nothing_without_area_lights_and_jitter():
    sc = S.scene_spheres8(width=24, height=20, max_depth=2)
    orc = O.OracleScene.from_scene(sc)
    ref = orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"]
    orc.set_pass(123, 17, 5, False)
    np.testing.assert_array_equal(orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"], ref)


def floor_with_emitters(spheres=None, tris=None, L=(1.0, 1.0, 1.0), albedo=(0.5, 0.5, 0.5), W=9, H=9):
    """The floor scene of plane_under_light with emissive primitives (material
    1, emission L) instead of an area light; the centre pixel sees the floor
    at the origin (the camera is above the emitters' reach)."""
    mats = np.concatenate([S.material(S.MAT_DIFFUSE, albedo, ks=0.0),
                           S.material(S.MAT_DIFFUSE, (0.0, 0.0, 0.0), ks=0.0, emission=L)])
    floor = S.triangles_from([(-50, 0, -50), (-50, 0, -50)], [(-50, 0, 50), (50, 0, 50)],
                             [(50, 0, 50), (50, 0, -50)], 0)
    tri = floor if tris is None else np.concatenate([floor, tris])
    sph = np.zeros(0, S.SPHERE_DTYPE) if spheres is None else spheres
    cam = S.camera((0.0, 20.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=10.0)
    return S.Scene("floor_emit", sph, tri, mats, np.zeros(0, S.LIGHT_DTYPE), cam, W, H, 0)


def test_emissive_quad_converges_to_lambert():
    """Two emissive triangles forming the tilted parallelogram of the area
    light test light the floor as Lambert's formula says (they emit on both
    sides; the camera looks past them at the floor below)."""
    c = np.array((1.0, 2.0, -1.5))
    eu, ev = np.array((2.0, 0.5, 0.0)), np.array((0.0, 0.0, 3.0))
    quad = S.triangles_from([c, c], [c + eu, c + eu + ev], [c + eu + ev, c + ev], 1)
    sc = floor_with_emitters(tris=quad, L=(2.0, 1.0, 0.5))
    orc = O.OracleScene.from_scene(sc)
    E = polygon_irradiance(np.zeros(3), np.array([0.0, 1.0, 0.0]), [c, c + eu, c + eu + ev, c + ev])
    centre = np.array([(sc.height // 2) * sc.width + sc.width // 2])
    got = progressive(orc, sc, passes=1024, strata=32, pixels=centre)[0]
    np.testing.assert_allclose(got, 0.5 * np.array([2.0, 1.0, 0.5]) * E, rtol=3e-3)


def test_emissive_sphere_converges_to_its_solid_angle():
    """A uniformly emitting sphere of radius r at height d straight above
    the point: the cosine-weighted solid angle is pi (r / d)^2."""
    r, d = 0.6, 3.0
    sph = S.spheres_from([(0.0, d, 0.0)], [r], [1])
    sc = floor_with_emitters(spheres=sph, L=(1.0, 0.5, 0.25))
    sc.camera = S.camera((0.0, 1.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=10.0)
    orc = O.OracleScene.from_scene(sc)
    centre = np.array([(sc.height // 2) * sc.width + sc.width // 2])
    got = progressive(orc, sc, passes=1024, strata=32, pixels=centre)[0]
    want = 0.5 * np.array([1.0, 0.5, 0.25]) * np.pi * (r / d) ** 2
    np.testing.assert_allclose(got, want, rtol=5e-3)
    # seen directly, the sphere shows its own emission (Eq. 7)
    sc2 = floor_with_emitters(spheres=sph, L=(1.0, 0.5, 0.25))
    sc2.camera = S.camera((0.0, 10.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=2.0)
    top = O.OracleScene.from_scene(sc2).render(sc2.camera, 9, 9, 0, mode="brute", pixels=centre)["rgb"][0]
    np.testing.assert_allclose(top, (1.0, 0.5, 0.25), atol=1e-12)
