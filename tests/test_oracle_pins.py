"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Every test here runs on the CPU only.  None of them reuses the oracle's own
code path to produce its expected values: they use values worked by hand
(tests/golden), geometric identities, special cases with a closed form, and
the oracle's brute-force definition against its BVH and iterative forms.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1504_03151_b300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Eq. 9-12: the ray-sphere quadratic
# ---------------------------------------------------------------------------
def test_sphere_roots_golden():
    cases = json.load(open(os.path.join(GOLDEN, "sphere_roots.json")))["cases"]
    for c in cases:
        got = O.sphere_roots(c["o"], c["d"], c["c"], c["r"])
        exp = np.array(c["roots"], float)
        if len(exp) == 1:
            assert len(got) == 1, c["what"]
        else:
            assert len(got) == len(exp), c["what"]
        np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12, err_msg=c["what"])


def test_sphere_roots_offset_family():
    # a ray parallel to z at lateral offset h meets the unit sphere where
    # x = h: z = -+ sqrt(1 - h^2), i.e. t = 5 -+ sqrt(1 - h^2)
    for h in np.linspace(0, 0.999, 37):
        got = O.sphere_roots([h, 0, -5], [0, 0, 1], [0, 0, 0], 1.0)
        w = math.sqrt(1 - h * h)
        np.testing.assert_allclose(got, [5 - w, 5 + w], atol=1e-12)


def _scene_one_sphere(c, r, mat_kind=S.MAT_DIFFUSE):
    return O.OracleScene(S.spheres_from([c], [r], [0]), np.zeros(0, S.TRIANGLE_DTYPE),
                         S.material(mat_kind, (0.5, 0.5, 0.5)), S.lights([(0, 10, 0)], [(1, 1, 1)]))


def test_closest_hit_takes_nearest_positive_root():
    sc = _scene_one_sphere((0, 0, 0), 1.0)
    o = np.array([[0, 0, -5], [0, 0, 0.5], [0, 0, 0], [0, 0, 5], [0.6, 0, -5]], np.float32)
    d = np.tile(np.array([[0, 0, 1]], np.float32), (5, 1))
    prim, t, _ = sc.closest_hits(o, d, use_bvh=False)
    np.testing.assert_array_equal(prim, [0, 0, 0, -1, 0])
    np.testing.assert_allclose(t[[0, 1, 2, 4]], [4.0, 0.5, 1.0, 4.2], atol=1e-12)
    assert math.isinf(t[3])


# ---------------------------------------------------------------------------
# triangles (Moller-Trumbore)
# ---------------------------------------------------------------------------
V0, V1, V2 = (0, 0, 0), (1, 0, 0), (0, 1, 0)


def test_triangle_closed_forms():
    hit, t, u, v = O.triangle_hit((0.25, 0.25, -1), (0, 0, 1), V0, V1, V2)
    assert hit and t == pytest.approx(1.0, abs=1e-15)
    assert u == pytest.approx(0.25, abs=1e-15) and v == pytest.approx(0.25, abs=1e-15)
    # p = v0 + u e1 + v e2 for an off-axis ray
    hit, t, u, v = O.triangle_hit((0.1, 0.2, -2), (0.05, 0.1, 1), V0, V1, V2)
    assert hit and t == pytest.approx(2.0, abs=1e-14)
    assert u == pytest.approx(0.2, abs=1e-14) and v == pytest.approx(0.4, abs=1e-14)
    assert not O.triangle_hit((0.6, 0.6, -1), (0, 0, 1), V0, V1, V2)[0]      # u + v > 1
    assert O.triangle_hit((0.5, 0.5, -1), (0, 0, 1), V0, V1, V2)[0]          # edge inclusive
    assert O.triangle_hit((0.0, 0.0, -1), (0, 0, 1), V0, V1, V2)[0]          # vertex inclusive
    assert O.triangle_hit((0.25, 0.25, 1), (0, 0, -1), V0, V1, V2)[0]        # two-sided
    assert not O.triangle_hit((0.25, 0.25, 1), (0, 0, 1), V0, V1, V2)[0]     # behind
    assert not O.triangle_hit((0.25, 0.25, 1), (1, 0, 0), V0, V1, V2)[0]     # parallel


# ---------------------------------------------------------------------------
# camera
# ---------------------------------------------------------------------------
def _angle(a, b):
    return math.acos(max(-1.0, min(1.0, float(np.dot(a, b)))))


def test_camera_centre_and_fov():
    W, H = 101, 61
    cam = S.camera((1, 2, 3), (-2, 0.5, -4), vfov_deg=50.0)
    f = np.array([-3, -1.5, -7.0])
    f /= np.linalg.norm(f)
    _, dc = O.camera_rays(cam, W, H, [(H // 2) * W + W // 2])
    np.testing.assert_allclose(dc[0], f, atol=1e-15)
    # rays through the centres of the top and bottom rows of the middle
    # column subtend 2 atan((1 - 1/H) tan(vfov/2)); left/right columns use
    # the aspect W/H.
    _, d = O.camera_rays(cam, W, H, [W // 2, (H - 1) * W + W // 2, (H // 2) * W, (H // 2) * W + W - 1])
    h = math.tan(math.radians(25.0))
    assert _angle(d[0], d[1]) == pytest.approx(2 * math.atan((1 - 1 / H) * h), abs=1e-12)
    assert _angle(d[2], d[3]) == pytest.approx(2 * math.atan((1 - 1 / W) * h * W / H), abs=1e-12)
    # row 0 is the top: its ray points further along `up` than the centre's
    up = np.array([0, 1.0, 0])
    assert np.dot(d[0], up) > np.dot(dc[0], up) > np.dot(d[1], up)
    # x grows to the right = along f x up
    right = np.cross(f, up)
    assert np.dot(d[3], right) > 0 > np.dot(d[2], right)


# ---------------------------------------------------------------------------
# analytic Lambert image of one lit sphere (Eq. 3 / Eq. 6 with f_r = albedo)
# ---------------------------------------------------------------------------
def test_lambert_sphere_image_closed_form():
    sc = S.single_sphere(width=65, height=65, albedo=(0.7, 0.5, 0.3), light=(0.0, 0.0, 10.0))
    orc = O.OracleScene.from_scene(sc)
    res = orc.render(sc.camera, 65, 65, 0, mode="brute")
    o, d = O.camera_rays(sc.camera, 65, 65)
    # independent hit: closest approach + Pythagoras (not the quadratic)
    tca = -(o * d).sum(1)                         # sphere at the origin
    dist2 = (o * o).sum(1) - tca ** 2
    hit = dist2 <= 1.0
    thc = np.sqrt(np.clip(1.0 - dist2, 0, None))
    p = o + (tca - thc)[:, None] * d
    n = p                                          # unit sphere: n = p
    L = np.array([0, 0, 10.0])
    l = (L - p) / np.linalg.norm(L - p, axis=1, keepdims=True)
    nl = np.clip((n * l).sum(1), 0, None)
    exp = np.where(hit[:, None], np.array([0.7, 0.5, 0.3]) * nl[:, None], 0.1)
    np.testing.assert_allclose(res["rgb"], exp, atol=1e-12)
    # the centre pixel sees the sphere head-on: n.l = 1 exactly
    c = 32 * 65 + 32
    np.testing.assert_allclose(res["rgb"][c], [0.7, 0.5, 0.3], atol=1e-15)
    # the hit disc: angle from the axis below asin(1/5)
    ang = np.arccos(np.clip(-d[:, 2], -1, 1))
    assert np.array_equal(res["prim"] >= 0, ang < math.asin(1 / 5.0))


def test_phong_peak_and_add_once():
    # ground triangle facing +z, light and eye on the axis: at the centre
    # pixel n.l = 1 and the mirrored light direction is the view direction,
    # so the colour is I * (albedo + ks) exactly.
    big = 50.0
    tri = S.triangles_from([(-big, -big, 0)], [(big, -big, 0)], [(0, big, 0)], 0)
    mat = S.material(S.MAT_DIFFUSE, (0.4, 0.6, 0.2), ks=0.3, shininess=32)
    li = S.lights([(0, 0, 7.0)], [(0.9, 0.8, 0.7)])
    cam = S.camera((0, 0, 5.0), (0, 0, 0), up=(0, 1, 0))
    orc = O.OracleScene(np.zeros(0, S.SPHERE_DTYPE), tri, mat, li)
    r = orc.render(cam, 33, 33, 0, mode="brute", pixels=[16 * 33 + 16])
    np.testing.assert_allclose(r["rgb"][0], np.array([0.9, 0.8, 0.7]) * (np.array([0.4, 0.6, 0.2]) + 0.3),
                               atol=1e-14)
    # Alg. 1 (G1 reading): objects that do not block the shadow ray add
    # nothing and do not multiply the light's contribution.
    far = S.spheres_from([(30, 30, 30), (-30, 20, 40), (25, -35, 10)], [1.0, 2.0, 0.5], [0, 0, 0])
    orc2 = O.OracleScene(far, tri, mat, li)
    r2 = orc2.render(cam, 33, 33, 0, mode="brute")
    r1 = orc.render(cam, 33, 33, 0, mode="brute")
    np.testing.assert_array_equal(r1["rgb"], r2["rgb"])
    # a blocker between the surface and the light removes it completely
    blk = S.spheres_from([(0, 0, 6.0)], [0.5], [0])
    orc3 = O.OracleScene(blk, tri, mat, li)
    r3 = orc3.render(cam, 33, 33, 0, mode="brute", pixels=[16 * 33 + 16])
    # the primary ray hits the blocker sphere first at the centre pixel? no:
    # the eye is at z=5 below the blocker (z in [5.5, 6.5]); the ray goes -z.
    assert r3["prim"][0] == 1
    np.testing.assert_allclose(r3["rgb"][0], 0.0, atol=1e-15)


# ---------------------------------------------------------------------------
# Fresnel-Schlick and Snell (dielectrics)
# ---------------------------------------------------------------------------
def test_schlick_normal_incidence_and_snell():
    ok, R, dt = O.refract([0, 0, -1], [0, 0, 1], 1.0, 1.5)
    assert ok and R == pytest.approx(0.04, abs=1e-15)
    np.testing.assert_allclose(dt, [0, 0, -1], atol=1e-15)
    ok, R, _ = O.refract([0, 0, -1], [0, 0, 1], 1.5, 1.0)
    assert ok and R == pytest.approx(0.04, abs=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(200):
        n1, n2 = rng.uniform(1.0, 2.0, 2)
        th = rng.uniform(0, math.pi / 2 * 0.999)
        d = np.array([math.sin(th), 0, -math.cos(th)])
        ok, R, dt = O.refract(d, [0, 0, 1], n1, n2)
        crit = math.asin(min(1.0, n2 / n1)) if n1 > n2 else math.pi
        if th < crit - 1e-9:
            assert ok
            s1 = math.sin(th)
            s2 = math.hypot(dt[0], dt[1])
            assert n1 * s1 == pytest.approx(n2 * s2, abs=1e-12)      # Snell
            assert np.linalg.norm(dt) == pytest.approx(1.0, abs=1e-14)
            assert dt[2] < 0                                          # goes through
            assert 0.0 <= R <= 1.0
        elif th > crit + 1e-9:
            assert not ok and R == 1.0                                # TIR


def test_schlick_oblique_incidence_golden():
    """Fresnel-Schlick at oblique angles on both sides of the interface:
    the cosine on the less dense side (cos theta_i from air, cos theta_t from
    glass or water) and the fifth power, against hand-worked values."""
    g = json.load(open(os.path.join(GOLDEN, "schlick_oblique.json")))
    for c in g["cases"]:
        th = math.radians(c["theta_deg"])
        d = np.array([math.sin(th), 0.0, -math.cos(th)])
        ok, R, dt = O.refract(d, [0, 0, 1], c["n1"], c["n2"])
        assert ok, c["what"]
        assert R == pytest.approx(c["R"], abs=1e-12), c["what"]
        # the refracted ray obeys Snell's law at the same angle
        assert c["n1"] * math.sin(th) == pytest.approx(c["n2"] * math.hypot(dt[0], dt[1]), abs=1e-12)
        # the pins tell the readings apart: the other cosine, or a fourth
        # power, would be off by far more than the tolerance
        r0 = ((c["n1"] - c["n2"]) / (c["n1"] + c["n2"])) ** 2
        ci = math.cos(th)
        ct = math.sqrt(1.0 - (c["n1"] / c["n2"] * math.sin(th)) ** 2)
        other = ct if c["cos_used"] == "incident" else ci
        assert abs(R - (r0 + (1 - r0) * (1 - other) ** 5)) > 1e-5, c["what"]
        used = ci if c["cos_used"] == "incident" else ct
        assert abs(R - (r0 + (1 - r0) * (1 - used) ** 4)) > 1e-5, c["what"]


def test_total_internal_reflection_angle():
    crit = math.degrees(math.asin(1 / 1.5))
    assert crit == pytest.approx(41.8103, abs=1e-4)
    for deg, expect in [(crit - 0.01, True), (crit + 0.01, False)]:
        th = math.radians(deg)
        ok, _, _ = O.refract([math.sin(th), 0, -math.cos(th)], [0, 0, 1], 1.5, 1.0)
        assert ok == expect


def test_index_matched_refraction_is_straight():
    d = np.array([0.3, -0.2, -0.9])
    d /= np.linalg.norm(d)
    ok, R, dt = O.refract(d, [0, 0, 1], 1.0, 1.0)
    assert ok
    np.testing.assert_allclose(dt, d, atol=1e-15)


# ---------------------------------------------------------------------------
# scene-level invariants
# ---------------------------------------------------------------------------
def _mirror_glass_scene(seed):
    rng = np.random.default_rng(seed)
    n = 6
    c = np.stack([rng.uniform(-3, 3, n), rng.uniform(0.5, 3, n), rng.uniform(-3, 3, n)], 1)
    r = rng.uniform(0.3, 1.0, n)
    mats = [S.material(S.MAT_MIRROR, (0.5, 0.5, 0.5), reflectivity=1.0)]
    for i in range(n):
        if i % 2:
            mats.append(S.material(S.MAT_MIRROR, (0.5, 0.5, 0.5), reflectivity=rng.uniform(0.2, 1)))
        else:
            mats.append(S.material(S.MAT_DIELECTRIC, (1, 1, 1), ks=0, ior=rng.uniform(1.2, 1.8)))
    sph = S.spheres_from(c, r, np.arange(1, n + 1))
    g = 10.0
    tris = S.triangles_from([(-g, 0, -g), (-g, 0, -g)], [(-g, 0, g), (g, 0, g)], [(g, 0, g), (g, 0, -g)], 0)
    return sph, tris, np.concatenate(mats)


def test_energy_bound_without_lights():
    # no lights, background B: every path weight is a product of rho <= 1,
    # R and 1-R, so no pixel can exceed B (depth truncation only loses).
    B = (0.3, 0.5, 0.7)
    sph, tris, mats = _mirror_glass_scene(1)
    orc = O.OracleScene(sph, tris, mats, np.zeros(0, S.LIGHT_DTYPE), background=B)
    cam = S.camera((0, 5, 12), (0, 1, 0))
    r = orc.render(cam, 96, 96, 6, mode="brute")
    assert (r["rgb"] <= np.array(B) + 1e-12).all()
    assert (r["rgb"] >= 0).all()
    # with lossless mirrors only (rho = 1 everywhere), deep enough, every
    # pixel whose path tree ends in misses returns exactly B
    mats2 = mats.copy()
    mats2["kind"] = S.MAT_MIRROR
    mats2["reflectivity"] = 1.0
    orc2 = O.OracleScene(sph, tris, mats2, np.zeros(0, S.LIGHT_DTYPE), background=B)
    r2 = orc2.render(cam, 48, 48, 16, mode="brute")
    frac_exact = np.mean(np.all(np.abs(r2["rgb"] - np.array(B)) < 1e-12, axis=1))
    assert frac_exact > 0.98


def test_mirror_plane_equals_mirrored_camera():
    # A rho = 1 mirror plane at y = 0 seen from above equals, pixel (x, y),
    # the scene without the plane seen from the mirrored camera at pixel
    # (W-1-x, y) (a mirror reverses handedness).
    big = 1e3
    plane = S.triangles_from([(-big, 0, -big), (-big, 0, -big)], [(-big, 0, big), (big, 0, big)],
                             [(big, 0, big), (big, 0, -big)], 0)
    sph = S.spheres_from([(0.5, 1.5, -1.0), (-1.2, 0.8, 0.5)], [0.7, 0.5], [1, 2])
    mats = np.concatenate([S.material(S.MAT_MIRROR, (0.5, 0.5, 0.5), reflectivity=1.0),
                           S.material(S.MAT_DIFFUSE, (0.8, 0.3, 0.2)),
                           S.material(S.MAT_DIFFUSE, (0.2, 0.5, 0.9))])
    li = S.lights([(3, 8, 2)], [(1, 1, 1)])
    W = H = 48
    cam = S.camera((0, 4, 6), (0, -2, -3), up=(0, 1, 0))
    camm = S.camera((0, -4, 6), (0, 2, -3), up=(0, -1, 0))
    # a tiny offset scale: the reflected ray then starts (to 1e-8) on the
    # mirror, where the mirrored camera's ray crosses it
    a = O.OracleScene(sph, plane, mats, li, eps_scale=1e-10).render(cam, W, H, 1, mode="brute")
    b = O.OracleScene(sph, np.zeros(0, S.TRIANGLE_DTYPE), mats, li, eps_scale=1e-10).render(
        camm, W, H, 0, mode="brute")
    A = a["rgb"].reshape(H, W, 3)
    Bm = b["rgb"].reshape(H, W, 3)[:, ::-1]
    via_mirror = (a["prim"] >= 2).reshape(H, W)          # primary ray meets the mirror first
    assert via_mirror.mean() > 0.5
    np.testing.assert_allclose(A[via_mirror], Bm[via_mirror], atol=1e-7)
    # the spheres are visible in the reflection
    assert (np.abs(Bm[via_mirror] - 0.1).max(axis=1) > 1e-3).sum() > 40


def test_recursive_equals_iterative():
    # Sec. IV.A: the recursion over depth and its iteration form agree.
    for sc in (S.scene_spheres8(), _small_terrain()):
        orc = O.OracleScene.from_scene(sc)
        a = orc.render(sc.camera, 64, 48, sc.max_depth, mode="brute")
        b = orc.render(sc.camera, 64, 48, sc.max_depth, mode="iterative")
        np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)
        assert a["counts"] == b["counts"]
        np.testing.assert_array_equal(a["prim"], b["prim"])


def _small_terrain():
    return S.scene_terrain(seed=7, width=64, height=48, max_depth=5, cells=(12, 9), n_ico=6, ico_level=1)


def test_depth_semantics():
    sc = S.scene_spheres8()
    orc = O.OracleScene.from_scene(sc)
    r0 = orc.render(sc.camera, 64, 64, 0, mode="brute")
    assert r0["counts"]["secondary"] == 0
    assert r0["counts"]["primary"] == 64 * 64
    r3 = orc.render(sc.camera, 64, 64, 3, mode="brute")
    # depth-0 hits are shaded identically; only mirror pixels change
    mirror = np.isin(r3["prim"], np.where(sc.materials["kind"][sc.spheres["material"]] == S.MAT_MIRROR)[0])
    np.testing.assert_array_equal(r0["rgb"][~mirror], r3["rgb"][~mirror])
    assert r3["counts"]["rays_per_depth"][1] == int(mirror.sum())


def test_per_pixel_ray_counts():
    """The per-pixel counts of the oracle: hand cases and the totals."""
    # one lit sphere seen from its light's side, depth 0: a hit pixel casts
    # one shadow ray (n.l > 0 on the whole visible cap), a miss casts none
    sc = S.single_sphere(width=33, height=33)
    orc = O.OracleScene.from_scene(sc)
    r = orc.render(sc.camera, 33, 33, 0, mode="brute", per_pixel=True)
    px = r["px_counts"]
    hit = r["prim"] >= 0
    assert hit.sum() > 50 and (~hit).sum() > 50
    assert (px[:, 0, 0] == 1).all()
    np.testing.assert_array_equal(px[:, 0, 1], hit.astype(np.uint32))
    # a mirror sphere (rho = 1) over nothing, depth 2: every hit pixel sends
    # one reflection that misses (nothing else is there), and no shadow ray
    mats = S.material(S.MAT_MIRROR, (0.5, 0.5, 0.5), reflectivity=1.0)
    sc2 = S.Scene("mirror", S.spheres_from([(0, 0, 0)], [1.0], [0]), np.zeros(0, S.TRIANGLE_DTYPE), mats,
                  S.lights([(0, 0, 10)], [(1, 1, 1)]), S.camera((0, 0, 5), (0, 0, 0)), 33, 33, 2)
    r2 = O.OracleScene.from_scene(sc2).render(sc2.camera, 33, 33, 2, mode="brute", per_pixel=True)
    hit2 = r2["prim"] >= 0
    np.testing.assert_array_equal(r2["px_counts"][:, 1, 0], hit2.astype(np.uint32))
    assert (r2["px_counts"][:, :, 1] == 0).all()
    assert (r2["px_counts"][:, 2, 0] == 0).all()
    # on the terrain the per-pixel counts add up to the totals, and asking
    # for them changes no other output
    st = _small_terrain()
    orc = O.OracleScene.from_scene(st)
    a = orc.render(st.camera, 64, 48, st.max_depth, mode="bvh")
    b = orc.render(st.camera, 64, 48, st.max_depth, mode="bvh", per_pixel=True)
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    np.testing.assert_array_equal(a["robust"], b["robust"])
    s = b["px_counts"].astype(np.int64).sum(axis=0)
    assert list(s[:, 0]) == b["counts"]["rays_per_depth"]
    assert list(s[:, 1]) == b["counts"]["shadow_per_depth"]


# ---------------------------------------------------------------------------
# the oracle's BVH returns the brute-force answer
# ---------------------------------------------------------------------------
def _random_tiny_scene(rng, n):
    ns = int(rng.integers(0, n + 1))
    nt = n - ns
    c = rng.uniform(-2, 2, (ns, 3))
    sph = S.spheres_from(c, rng.uniform(0.05, 0.8, ns), np.zeros(ns, int))
    base = rng.uniform(-2, 2, (nt, 3))
    tris = S.triangles_from(base, base + rng.normal(0, 0.7, (nt, 3)), base + rng.normal(0, 0.7, (nt, 3)),
                            np.zeros(nt, int))
    mats = S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))
    return O.OracleScene(sph, tris, mats, S.lights([(0, 5, 0)], [(1, 1, 1)]))


def test_bvh_equals_brute_force_on_tiny_scenes():
    rng = np.random.default_rng(123)
    for n in list(range(1, 17)) * 2:
        orc = _random_tiny_scene(rng, n)
        o = rng.uniform(-4, 4, (10000 // 8, 3)).astype(np.float32)
        tgt = rng.uniform(-2, 2, (len(o), 3))
        d = (tgt - o)
        d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
        p1, t1, r1 = orc.closest_hits(o, d, use_bvh=False)
        p2, t2, r2 = orc.closest_hits(o, d, use_bvh=True)
        np.testing.assert_array_equal(p1, p2)
        np.testing.assert_array_equal(t1, t2)
        np.testing.assert_array_equal(r1 < 1, r2 < 1)
        tmax = rng.uniform(0.5, 8, len(o)).astype(np.float32)
        a1, _ = orc.any_hits(o, d, tmax, use_bvh=False)
        a2, _ = orc.any_hits(o, d, tmax, use_bvh=True)
        np.testing.assert_array_equal(a1, a2)
        # any-hit agrees with closest-hit
        np.testing.assert_array_equal(a1, (p1 >= 0) & (t1 < tmax))


def test_bvh_equals_brute_force_on_terrain_sample():
    sc = _small_terrain()
    orc = O.OracleScene.from_scene(sc)
    a = orc.render(sc.camera, 64, 48, sc.max_depth, mode="brute")
    b = orc.render(sc.camera, 64, 48, sc.max_depth, mode="bvh")
    np.testing.assert_array_equal(a["prim"], b["prim"])
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    assert a["counts"] == b["counts"]


def test_scene_rejects_bad_input():
    good_s = S.spheres_from([(0, 0, 0)], [1.0], [0])
    mats = S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))
    li = S.lights([(0, 5, 0)], [(1, 1, 1)])
    notri = np.zeros(0, S.TRIANGLE_DTYPE)
    O.OracleScene(good_s, notri, mats, li)
    for bad in (S.spheres_from([(0, 0, 0)], [0.0], [0]), S.spheres_from([(np.nan, 0, 0)], [1.0], [0]),
                S.spheres_from([(0, 0, 0)], [1.0], [3])):
        with pytest.raises(ValueError):
            O.OracleScene(bad, notri, mats, li)


def _duplicated_scene(red_first):
    """A floor (2 triangles) and a sphere, each present twice at exactly the
    same place: once grey (material 0), once red (material 1).  red_first
    puts the red copies at the lower primitive ids."""
    mats = np.concatenate([S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5), ks=0.0),
                           S.material(S.MAT_DIFFUSE, (0.9, 0.1, 0.1), ks=0.0)])
    first, second = (1, 0) if red_first else (0, 1)
    v0 = [(-5, 0, -5), (-5, 0, -5)]
    v1 = [(-5, 0, 5), (5, 0, 5)]
    v2 = [(5, 0, 5), (5, 0, -5)]
    tris = np.concatenate([S.triangles_from(v0, v1, v2, first), S.triangles_from(v0, v1, v2, second)])
    sph = S.spheres_from([(0.0, 1.0, 0.0), (0.0, 1.0, 0.0)], [0.8, 0.8], [first, second])
    return S.Scene("dup", sph, tris, mats, S.lights([(3.0, 8.0, 4.0)], [(1.0, 1.0, 1.0)]),
                   S.camera((0.0, 4.0, 7.0), (0.0, 0.5, 0.0)), 48, 36, 1)


@pytest.mark.parametrize("red_first", [False, True])
def test_exact_ties_go_to_the_lower_primitive_id(red_first):
    """Duplicated primitives tie exactly: the hit is the lower id, in brute
    force and through the BVH, and the colour is that primitive's."""
    sc = _duplicated_scene(red_first)
    orc = O.OracleScene.from_scene(sc)
    # ids: the spheres 0, 1; the first floor 2, 3; its copy 4, 5
    for mode in ("brute", "bvh"):
        r = orc.render(sc.camera, sc.width, sc.height, 0, mode=mode)
        hit = r["prim"] >= 0
        assert hit.mean() > 0.5
        assert set(np.unique(r["prim"][hit])) <= {0, 2, 3}
        assert (r["prim"][hit] != 1).all() and not np.isin(r["prim"][hit], [4, 5]).any()
        lit = r["rgb"][hit]
        red = lit[:, 0] > 3 * lit[:, 2] + 1e-9
        assert (red == red_first)[lit[:, 0] > 1e-6].all()
