"""Pins of the oracle's Monte-Carlo GI: Eq. 8's hemisphere integral
estimated with one cosine-weighted diffuse bounce per vertex, besides the
light samples of each pass.

Two closed forms pin it:
- A closed emitting box ("furnace"). Every point of its inside sees
  emitters over its whole hemisphere, so the light samples of a vertex
  give pi a L_e. Each diffuse bounce multiplies that by pi a, and a bounce
  that lands on an emitter adds no L_e of its own. That fixes the pixel at
  L_e (1 + pi a + ... + (pi a)^(D+1)).
- A floor under an open sky with a black wall. The bounce escapes to the
  background B unless it meets the wall. The expected pixel is a B
  (pi - E), where E is Lambert's polygon integral of the wall. Only a
  cosine distribution of the bounce directions gives it, so rotated copies
  of the scene also check the tangent basis for normals of either sign
  of z.
"""
import numpy as np
import pytest

import oracle as O
from paper_1504_03151_b300 import scenes as S

from test_oracle_pass import polygon_irradiance


def gi_progressive(sc, passes, strata, depth, seed=3, pixels=None, bounce=True):
    orc = O.OracleScene.from_scene(sc)
    orc.set_diffuse_bounce(bounce)
    acc = None
    for k in range(passes):
        orc.set_pass(seed, k, strata, False)
        r = orc.render(sc.camera, sc.width, sc.height, depth, mode="brute", pixels=pixels)["rgb"]
        acc = r if acc is None else acc + (r - acc) / (k + 1)
    return acc


def box_triangles(lo, hi, mat):
    """The 12 triangles of the axis-aligned box [lo, hi]."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    c = np.array([(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
                  (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)], np.float64)
    quads = [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (3, 2, 6, 7), (0, 3, 7, 4), (1, 2, 6, 5)]
    v0, v1, v2 = [], [], []
    for a, b, cc, d in quads:
        v0 += [c[a], c[a]]
        v1 += [c[b], c[cc]]
        v2 += [c[cc], c[d]]
    return S.triangles_from(v0, v1, v2, mat)


def furnace(albedo, Le, W=9, H=9):
    """The inside of the emitting box [-1, 1]^3 (albedo `albedo`, emission
    Le, no Phong lobe), seen from its centre."""
    mats = S.material(S.MAT_DIFFUSE, (albedo,) * 3, ks=0.0, emission=Le)
    cam = S.camera((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), vfov_deg=60.0)
    return S.Scene("furnace", np.zeros(0, S.SPHERE_DTYPE), box_triangles((-1, -1, -1), (1, 1, 1), 0), mats,
                   np.zeros(0, S.LIGHT_DTYPE), cam, W, H, 0)


def furnace_value(albedo, Le, depth):
    q = np.pi * albedo
    return np.asarray(Le, float) * sum(q ** j for j in range(depth + 2))


WALL = np.array([(-3.0, 0.5, -2.0), (3.0, 0.5, -2.0), (3.0, 4.5, -2.0), (-3.0, 4.5, -2.0)])


def floor_and_wall(albedo=(0.6, 0.4, 0.2), background=(0.3, 0.5, 0.7), W=9, H=9):
    """A diffuse floor at y = 0 (no lights), a black vertical wall beside
    the part the camera sees, and the sky (background) above."""
    mats = np.concatenate([S.material(S.MAT_DIFFUSE, albedo, ks=0.0),
                           S.material(S.MAT_DIFFUSE, (0.0, 0.0, 0.0), ks=0.0)])
    # one triangle: a floor of two would meet at a crease once its rotated
    # vertices are rounded to FP32, and grazing bounces would hit it
    floor = S.triangles_from([(-3e3, 0, -1e3)], [(0, 0, 2e3)], [(3e3, 0, -1e3)], 0)
    w = WALL
    wall = S.triangles_from([w[0], w[0]], [w[1], w[2]], [w[2], w[3]], 1)
    cam = S.camera((0.0, 20.0, 0.0), (0.0, 0.0, 0.0), up=(0.0, 0.0, -1.0), vfov_deg=10.0)
    return S.Scene("floor_wall", np.zeros(0, S.SPHERE_DTYPE), np.concatenate([floor, wall]), mats,
                   np.zeros(0, S.LIGHT_DTYPE), cam, W, H, 0, background=background)


def rotation(axis, deg):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    t = np.radians(deg)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K


def rotated(sc, R):
    """The scene with its geometry and camera turned by R about the origin."""
    tris = sc.triangles.copy()
    for k in ("v0", "v1", "v2"):
        tris[k] = (tris[k].astype(np.float64) @ R.T).astype(np.float32)
    cam = sc.camera.copy()
    for k in ("eye", "look_at", "up"):
        cam[k] = (cam[k].astype(np.float64) @ R.T).astype(np.float32)
    return S.Scene(sc.name + "_rot", sc.spheres, tris, sc.materials, sc.lights, cam, sc.width, sc.height,
                   sc.max_depth, background=sc.background)


def wall_expected(sc, R=np.eye(3)):
    """a B (pi - E_wall) at the floor point each pixel sees (unrotated
    frame: the rotation changes nothing)."""
    a = sc.materials["albedo"][0].astype(np.float64)
    B = np.asarray(sc.background, float)
    out = np.zeros((sc.width * sc.height, 3))
    os_, ds = O.camera_rays(sc.camera, sc.width, sc.height)
    for i, (o, d) in enumerate(zip(os_, ds)):
        o, d = R.T @ o, R.T @ d          # back to the unrotated frame
        p = o - d * (o[1] / d[1])
        E = polygon_irradiance(p, np.array([0.0, 1.0, 0.0]), list(WALL))
        out[i] = a * B * (np.pi - E)
    return out


# A vertex near an edge of the box samples the adjacent face at small r,
# where A cos cos / r^2 has heavy tails, so deeper paths converge slowly.
# Every plausible mistake moves the value far more than these tolerances:
# weight a instead of pi a (-60 % and more), L_e kept on bounce hits (+17 %
# at depth 1), a depth off by one (+-12 % at depth 3).
@pytest.mark.parametrize("depth,passes,rtol", [(0, 64, 4e-3), (1, 64, 5e-3), (3, 256, 1.5e-2)])
def test_furnace_closed_form(depth, passes, rtol):
    a, Le = 0.25, (1.0, 0.5, 2.0)
    sc = furnace(a, Le)
    got = gi_progressive(sc, passes, 8, depth)
    want = furnace_value(a, Le, depth)
    # every pixel has the same expectation: the mean over pixels and passes
    np.testing.assert_allclose(got.mean(axis=0), want, rtol=rtol)
    assert np.median(np.abs(got / want - 1)) < 0.05


def test_furnace_without_the_bounce_is_one_light_sample():
    """GI off: L_e + the emitters sampled once (pi a L_e), at any depth."""
    a, Le = 0.25, (1.0, 0.5, 2.0)
    sc = furnace(a, Le)
    got = gi_progressive(sc, 64, 8, 3, bounce=False)
    np.testing.assert_allclose(got.mean(axis=0), furnace_value(a, Le, 0), rtol=4e-3)


@pytest.mark.parametrize("R", [np.eye(3), rotation((1.0, 0.3, 0.2), 50.0), rotation((1.0, -0.4, 0.1), -70.0)],
                         ids=["upright", "normal_z_pos", "normal_z_neg"])
def test_open_sky_with_a_wall(R):
    base = floor_and_wall()
    n = R @ np.array([0.0, 1.0, 0.0])
    assert abs(n[2]) > 0.3 or np.allclose(R, np.eye(3))
    sc = rotated(base, R)
    want = wall_expected(sc, R)
    assert (want[:, 0] < 0.6 * 0.3 * np.pi * 0.97).all()   # the wall takes a visible share of the sky
    got = gi_progressive(sc, 256, 16, 2)
    np.testing.assert_allclose(got.mean(axis=0), want.mean(axis=0), rtol=4e-3)
    np.testing.assert_allclose(got, want, rtol=0.08)
    # one hit probability per pixel: the channels keep the ratio a B
    ratio = got / (np.array((0.6, 0.4, 0.2)) * np.array((0.3, 0.5, 0.7)))
    np.testing.assert_allclose(ratio[:, 1:], ratio[:, :1].repeat(2, axis=1), rtol=1e-6)   # FP32 albedo


def test_bounce_changes_nothing_where_it_cannot_happen():
    """No bounce at the last depth (depth 0), none off a black surface, and
    none without the switch: the Whitted image is unchanged."""
    sc = S.scene_spheres8_emitters(width=24, height=20, max_depth=2)
    orc = O.OracleScene.from_scene(sc)
    orc.set_pass(5, 3, 2, True)
    ref0 = orc.render(sc.camera, sc.width, sc.height, 0, mode="brute")["rgb"]
    ref2 = orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"]
    orc.set_diffuse_bounce(True)
    np.testing.assert_array_equal(orc.render(sc.camera, sc.width, sc.height, 0, mode="brute")["rgb"], ref0)
    assert not np.array_equal(orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"], ref2)
    orc.set_diffuse_bounce(False)
    np.testing.assert_array_equal(orc.render(sc.camera, sc.width, sc.height, 2, mode="brute")["rgb"], ref2)
    black = furnace(0.0, (1.0, 1.0, 1.0))
    got = gi_progressive(black, 4, 2, 3)
    np.testing.assert_allclose(got, 1.0, atol=1e-12)   # L_e only: no light term, no bounce


def test_gi_forms_agree():
    """Recursion, the iteration over depth and the BVH give one GI pass."""
    sc = S.scene_spheres8_emitters(width=24, height=20, max_depth=3)
    orc = O.OracleScene.from_scene(sc)
    orc.set_diffuse_bounce(True)
    orc.set_pass(9, 2, 2, True)
    a = orc.render(sc.camera, sc.width, sc.height, 3, mode="brute")["rgb"]
    b = orc.render(sc.camera, sc.width, sc.height, 3, mode="iterative")["rgb"]
    c = orc.render(sc.camera, sc.width, sc.height, 3, mode="bvh")["rgb"]
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c, a, rtol=1e-9, atol=1e-12)
