"""Seeded synthetic scenes for the Whitted tracer (inputs only).

This module creates input data and nothing else: it holds no intersection,
shading or traversal arithmetic.  Both the CUDA path and the CPU oracle
consume the arrays it returns, in the binary layout of the C ABI structs
(``rt_sphere``, ``rt_triangle``, ``rt_material``, ``rt_point_light``,
``rt_camera``).

The paper (Sec. V) measures on a third-party sphere scene that is not
available; these generators stand in for it with the workloads the tracer is
benchmarked on:

* ``scene_spheres8`` - 256x256, 8 random spheres on a 20x20 two-triangle
  ground plane, one white light at (0,10,0), depth 3.
* ``scene_terrain`` - 1920x1080, a 256x192-cell fBm value-noise heightfield
  (98,304 triangles) plus 20 level-3 icospheres (1,280 triangles each,
  123,904 triangles in total), 4 point lights, 60/25/15 % diffuse / mirror /
  dielectric icosphere materials, depth 5.
* ``scene_batch`` - uneven scenes of the terrain+icosphere kind, for batched
  launches.

Every random draw comes from ``numpy.random.default_rng(seed)`` (PCG64), so a
(config, seed) pair always gives the same bytes.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np

# ---------------------------------------------------------------------------
# Binary layouts of the C ABI structs (include/rtb.h).  All fields are 4-byte,
# so there is no padding.
# ---------------------------------------------------------------------------
SPHERE_DTYPE = np.dtype([("center", "<f4", 3), ("radius", "<f4"), ("material", "<u4")])
TRIANGLE_DTYPE = np.dtype([("v0", "<f4", 3), ("v1", "<f4", 3), ("v2", "<f4", 3), ("material", "<u4")])
MATERIAL_DTYPE = np.dtype([
    ("kind", "<u4"), ("albedo", "<f4", 3), ("ks", "<f4"), ("shininess", "<f4"),
    ("reflectivity", "<f4"), ("ior", "<f4"), ("emission", "<f4", 3)])
LIGHT_DTYPE = np.dtype([("position", "<f4", 3), ("intensity", "<f4", 3)])
CAMERA_DTYPE = np.dtype([("eye", "<f4", 3), ("look_at", "<f4", 3), ("up", "<f4", 3), ("vfov_deg", "<f4")])
AREA_LIGHT_DTYPE = np.dtype([("corner", "<f4", 3), ("edge_u", "<f4", 3), ("edge_v", "<f4", 3),
                             ("radiance", "<f4", 3)])

assert SPHERE_DTYPE.itemsize == 20
assert TRIANGLE_DTYPE.itemsize == 40
assert MATERIAL_DTYPE.itemsize == 44
assert LIGHT_DTYPE.itemsize == 24
assert CAMERA_DTYPE.itemsize == 40
assert AREA_LIGHT_DTYPE.itemsize == 48

MAT_DIFFUSE, MAT_MIRROR, MAT_DIELECTRIC = 0, 1, 2

BACKGROUND = (0.1, 0.1, 0.1)


@dataclasses.dataclass
class Scene:
    """One renderable job: geometry, materials, lights, camera and frame size."""
    name: str
    spheres: np.ndarray
    triangles: np.ndarray
    materials: np.ndarray
    lights: np.ndarray
    camera: np.ndarray          # shape (1,), CAMERA_DTYPE
    width: int
    height: int
    max_depth: int
    background: tuple = BACKGROUND
    area_lights: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, AREA_LIGHT_DTYPE))

    @property
    def n_prims(self) -> int:
        return len(self.spheres) + len(self.triangles)

    def digest(self) -> str:
        """SHA-256 over every input byte (freezes a generated scene)."""
        h = hashlib.sha256()
        for a in (self.spheres, self.triangles, self.materials, self.lights, self.camera):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(np.array([self.width, self.height, self.max_depth], np.int64).tobytes())
        h.update(np.array(self.background, np.float64).tobytes())
        if len(self.area_lights):
            h.update(np.ascontiguousarray(self.area_lights).tobytes())
        return h.hexdigest()


def material(kind, albedo, ks=0.3, shininess=32.0, reflectivity=0.0, ior=1.0, emission=(0, 0, 0)):
    m = np.zeros(1, MATERIAL_DTYPE)
    m["kind"] = kind
    m["albedo"] = albedo
    m["ks"] = ks
    m["shininess"] = shininess
    m["reflectivity"] = reflectivity
    m["ior"] = ior
    m["emission"] = emission
    return m


def camera(eye, look_at, up=(0.0, 1.0, 0.0), vfov_deg=60.0):
    c = np.zeros(1, CAMERA_DTYPE)
    c["eye"] = eye
    c["look_at"] = look_at
    c["up"] = up
    c["vfov_deg"] = vfov_deg
    return c


def lights(positions, intensities):
    a = np.zeros(len(positions), LIGHT_DTYPE)
    a["position"] = positions
    a["intensity"] = intensities
    return a


def area_lights(corners, edges_u, edges_v, radiances):
    """Parallelogram lights corner + a edge_u + b edge_v (a, b in [0, 1]),
    emitting `radiance` on the side of edge_u x edge_v."""
    a = np.zeros(len(corners), AREA_LIGHT_DTYPE)
    a["corner"] = corners
    a["edge_u"] = edges_u
    a["edge_v"] = edges_v
    a["radiance"] = radiances
    return a


def triangles_from(v0, v1, v2, mat):
    t = np.zeros(len(v0), TRIANGLE_DTYPE)
    t["v0"] = v0
    t["v1"] = v1
    t["v2"] = v2
    t["material"] = mat
    return t


def spheres_from(centers, radii, mats):
    s = np.zeros(len(centers), SPHERE_DTYPE)
    s["center"] = centers
    s["radius"] = radii
    s["material"] = mats
    return s


# ---------------------------------------------------------------------------
# Geometry builders (mesh generation only).
# ---------------------------------------------------------------------------
_PHI = (1.0 + math.sqrt(5.0)) / 2.0
_ICO_V = np.array([
    (-1, _PHI, 0), (1, _PHI, 0), (-1, -_PHI, 0), (1, -_PHI, 0),
    (0, -1, _PHI), (0, 1, _PHI), (0, -1, -_PHI), (0, 1, -_PHI),
    (_PHI, 0, -1), (_PHI, 0, 1), (-_PHI, 0, -1), (-_PHI, 0, 1)], np.float64)
_ICO_F = np.array([
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
    (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
    (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
    (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], np.int64)


def icosphere(level: int):
    """Unit icosphere mesh with 20*4**level outward (CCW) faces.

    Returns (vertices float64 [V,3], faces int64 [F,3]).
    """
    verts = [v / np.linalg.norm(v) for v in _ICO_V]
    faces = [tuple(f) for f in _ICO_F]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces, np.int64)
    # Make every face wind counter-clockwise seen from outside.
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = (n * V[F].mean(axis=1)).sum(axis=1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def _value_noise_lattice(rng, n):
    return rng.uniform(-1.0, 1.0, size=(n, n))


def fbm_heights(rng, xs, zs, octaves=6, lacunarity=2.0, gain=0.5, amplitude=3.0,
                base_freq=1.0 / 16.0):
    """fBm of value noise, smoothstep-interpolated, sampled on the grid xs x zs.

    Returns heights [len(zs), len(xs)], scaled so |h| <= amplitude.
    """
    X, Z = np.meshgrid(xs, zs)
    h = np.zeros_like(X)
    norm = 0.0
    for k in range(octaves):
        f = base_freq * lacunarity ** k
        a = gain ** k
        lat = _value_noise_lattice(rng, 257)
        u = (X - xs[0]) * f
        v = (Z - zs[0]) * f
        i0 = np.floor(u).astype(np.int64)
        j0 = np.floor(v).astype(np.int64)
        fu = u - i0
        fv = v - j0
        su = fu * fu * (3 - 2 * fu)
        sv = fv * fv * (3 - 2 * fv)
        i0 %= 256
        j0 %= 256
        n00 = lat[j0, i0]
        n10 = lat[j0, i0 + 1]
        n01 = lat[j0 + 1, i0]
        n11 = lat[j0 + 1, i0 + 1]
        h += a * ((n00 * (1 - su) + n10 * su) * (1 - sv) + (n01 * (1 - su) + n11 * su) * sv)
        norm += a
    return amplitude * h / norm


def heightfield_triangles(xs, zs, H):
    """Two triangles per grid cell with a fixed diagonal; faces wind so the
    geometric normal points to +y."""
    X, Z = np.meshgrid(xs, zs)
    P = np.stack([X, H, Z], axis=-1)            # [nz, nx, 3]
    p00 = P[:-1, :-1].reshape(-1, 3)
    p10 = P[:-1, 1:].reshape(-1, 3)             # +x
    p01 = P[1:, :-1].reshape(-1, 3)             # +z
    p11 = P[1:, 1:].reshape(-1, 3)
    # (p00, p01, p11) and (p00, p11, p10): e1 x e2 has +y for both.
    v0 = np.concatenate([p00, p00])
    v1 = np.concatenate([p01, p11])
    v2 = np.concatenate([p11, p10])
    # interleave the two halves so a cell's triangles are adjacent in the input
    n = len(p00)
    order = np.stack([np.arange(n), np.arange(n) + n], axis=1).reshape(-1)
    return v0[order], v1[order], v2[order]


def _bilinear_height(xs, zs, H, x, z):
    fx = (x - xs[0]) / (xs[1] - xs[0])
    fz = (z - zs[0]) / (zs[1] - zs[0])
    i = min(max(int(math.floor(fx)), 0), len(xs) - 2)
    j = min(max(int(math.floor(fz)), 0), len(zs) - 2)
    u, v = fx - i, fz - j
    return ((H[j, i] * (1 - u) + H[j, i + 1] * u) * (1 - v)
            + (H[j + 1, i] * (1 - u) + H[j + 1, i + 1] * u) * v)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def scene_spheres8(seed: int = 1, width: int = 256, height: int = 256, max_depth: int = 3) -> Scene:
    """8 random spheres on a 20x20 ground quad, one white light, depth 3."""
    rng = np.random.default_rng(seed)
    centers = np.stack([rng.uniform(-4, 4, 8), rng.uniform(0, 3, 8), rng.uniform(-4, 4, 8)], axis=1)
    radii = rng.uniform(0.3, 1.0, 8)
    refl = np.where(rng.random(8) < 0.5, 0.5, 0.0)
    albedo = rng.uniform(0.2, 0.9, (8, 3))
    mats = [material(MAT_DIFFUSE, (0.8, 0.8, 0.8))]
    for i in range(8):
        kind = MAT_MIRROR if refl[i] > 0 else MAT_DIFFUSE
        mats.append(material(kind, albedo[i], reflectivity=refl[i]))
    sph = spheres_from(centers, radii, np.arange(1, 9))
    g = 10.0
    v0 = np.array([(-g, 0, -g), (-g, 0, -g)], np.float64)
    v1 = np.array([(-g, 0, g), (g, 0, g)], np.float64)
    v2 = np.array([(g, 0, g), (g, 0, -g)], np.float64)
    tris = triangles_from(v0, v1, v2, 0)
    return Scene("spheres8_256", sph, tris, np.concatenate(mats),
                 lights([(0, 10, 0)], [(1, 1, 1)]),
                 camera((0, 5, 12), (0, 1, 0)), width, height, max_depth)


def _terrain_icospheres(rng, cells_x, cells_z, half_x, half_z, n_ico, ico_level,
                        n_lights, ior_range=(1.5, 1.5), amplitude=3.0, radius_range=(0.5, 2.0),
                        base_freq=1.0 / 16.0, light_y=(20.0, 30.0)):
    xs = np.linspace(-half_x, half_x, cells_x + 1)
    zs = np.linspace(-half_z, half_z, cells_z + 1)
    H = fbm_heights(rng, xs, zs, amplitude=amplitude, base_freq=base_freq)
    tv0, tv1, tv2 = heightfield_triangles(xs, zs, H)
    mats = [material(MAT_DIFFUSE, (0.8, 0.8, 0.8))]
    v0s, v1s, v2s, ms = [tv0], [tv1], [tv2], [np.zeros(len(tv0), np.int64)]
    V, F = icosphere(ico_level)
    for i in range(n_ico):
        r = rng.uniform(*radius_range)
        cx = rng.uniform(-half_x + r, half_x - r)
        cz = rng.uniform(-half_z + r, half_z - r)
        cy = _bilinear_height(xs, zs, H, cx, cz) + r + rng.uniform(0.0, 2.0)
        u = rng.random()
        albedo = rng.uniform(0.2, 0.9, 3)
        if u < 0.60:
            m = material(MAT_DIFFUSE, albedo)
        elif u < 0.85:
            m = material(MAT_MIRROR, albedo, reflectivity=0.8)
        else:
            m = material(MAT_DIELECTRIC, (1, 1, 1), ks=0.0, ior=rng.uniform(*ior_range))
        mats.append(m)
        P = V * r + np.array([cx, cy, cz])
        v0s.append(P[F[:, 0]])
        v1s.append(P[F[:, 1]])
        v2s.append(P[F[:, 2]])
        ms.append(np.full(len(F), len(mats) - 1, np.int64))
    tris = triangles_from(np.concatenate(v0s), np.concatenate(v1s), np.concatenate(v2s),
                          np.concatenate(ms))
    lp = np.stack([rng.uniform(-half_x, half_x, n_lights), rng.uniform(*light_y, n_lights),
                   rng.uniform(-half_z, half_z, n_lights)], axis=1)
    li = lights(lp, np.full((n_lights, 3), 1.0 / n_lights))
    return tris, np.concatenate(mats), li


def scene_terrain(seed: int = 2, width: int = 1920, height: int = 1080, max_depth: int = 5,
                  cells=(256, 192), n_ico: int = 20, ico_level: int = 3) -> Scene:
    """fBm terrain (256x192 cells) + 20 icospheres (L3), 4 lights, depth 5."""
    rng = np.random.default_rng(seed)
    tris, mats, li = _terrain_icospheres(rng, cells[0], cells[1], 32.0, 24.0, n_ico, ico_level, 4)
    return Scene(f"terrain{len(tris)}_{width}x{height}", np.zeros(0, SPHERE_DTYPE), tris, mats, li,
                 camera((0, 12, 38), (0, 0, 0)), width, height, max_depth)


def scene_terrain_lit(seed: int = 2, width: int = 1920, height: int = 1080, max_depth: int = 5, **kw) -> Scene:
    """The terrain with sampled lights besides its 4 point lights: two
    parallelogram area lights (8 x 8 at height 18 facing down, radiance 0.6;
    6 x 4 tilted at height 14, radiance 0.4 x (1, 0.8, 0.6)) and a glowing
    sphere of radius 1.5 at (6, 9, -4) (emission (2, 1.6, 1.2), no albedo)."""
    sc = scene_terrain(seed, width, height, max_depth, **kw)
    mats = np.concatenate([sc.materials, material(MAT_DIFFUSE, (0.0, 0.0, 0.0), ks=0.0, emission=(2.0, 1.6, 1.2))])
    sc.materials = mats
    sc.spheres = spheres_from([(6.0, 9.0, -4.0)], [1.5], [len(mats) - 1])
    sc.area_lights = area_lights([(-12.0, 18.0, -8.0), (4.0, 14.0, 2.0)], [(8.0, 0.0, 0.0), (6.0, -1.0, 0.0)],
                                 [(0.0, 0.0, 8.0), (0.0, 0.0, 4.0)], [(0.6, 0.6, 0.6), (0.4, 0.32, 0.24)])
    sc.name = sc.name + "_lit"
    return sc


def scene_batch_member(seed: int, n_tris_target: int, width: int, height: int, max_depth: int = 4) -> Scene:
    """One scene of a batch: ~80 % terrain / ~20 % across 20 icospheres, sized to
    roughly n_tris_target triangles."""
    rng = np.random.default_rng(seed)
    terr = max(int(0.8 * n_tris_target), 8)
    cz = max(int(math.sqrt(terr / 2 * 0.75)), 1)
    cx = max(int(round(terr / 2 / cz)), 1)
    per_ico = max(0.2 * n_tris_target / 20.0, 20)
    level = int(min(max(round(math.log(per_ico / 20.0, 4)), 0), 5))
    tris, mats, li = _terrain_icospheres(rng, cx, cz, 32.0, 24.0, 20, level, 4)
    return Scene(f"batch{seed}_{len(tris)}_{width}x{height}", np.zeros(0, SPHERE_DTYPE), tris,
                 mats, li, camera((0, 12, 38), (0, 0, 0)), width, height, max_depth)


def scene_batch(seed: int = 3, n_scenes: int = 64, max_depth: int = 4):
    """64 scenes with log-uniform triangle counts in [1e3, 2e6] and resolutions
    drawn from {256^2, 512^2, 1024^2, 1280x720}."""
    rng = np.random.default_rng(seed)
    res = [(256, 256), (512, 512), (1024, 1024), (1280, 720)]
    out = []
    for i in range(n_scenes):
        n = int(math.exp(rng.uniform(math.log(1e3), math.log(2e6))))
        w, h = res[int(rng.integers(0, 4))]
        out.append(scene_batch_member(int(rng.integers(0, 2**31)), n, w, h, max_depth))
    return out


def scene_scaleup(seed: int = 5, width: int = 3840, height: int = 2160, max_depth: int = 8, cells: int = 2048,
                  n_ico: int = 500, ico_level: int = 4):
    """The scale-up workload: a 2048x2048-cell fBm terrain (8,388,608
    triangles) over [-256, 256]^2 plus 500 level-4 icospheres (5,120
    triangles each), 10,948,608 triangles; 8 lights; mirrors and dielectrics
    with IOR U[1.3, 1.7]; depth 8.  Its four views (views_scaleup) look at
    the centre from the compass points."""
    rng = np.random.default_rng(seed)
    tris, mats, li = _terrain_icospheres(rng, cells, cells, 256.0, 256.0, n_ico, ico_level, 8,
                                         ior_range=(1.3, 1.7), amplitude=24.0, radius_range=(2.0, 8.0),
                                         base_freq=1.0 / 128.0, light_y=(160.0, 240.0))
    return Scene(f"scaleup{len(tris)}_{width}x{height}", np.zeros(0, SPHERE_DTYPE), tris, mats, li,
                 views_scaleup()[0], width, height, max_depth)


def views_scaleup():
    """Four cameras on a circle of radius 300 at height 90, looking at the centre."""
    return [camera((300.0 * sx, 90.0, 300.0 * sz), (0.0, 0.0, 0.0))
            for sx, sz in ((0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0))]


def scene_spheres8_area(seed: int = 1, width: int = 256, height: int = 256, max_depth: int = 3) -> Scene:
    """spheres8 lit by a 4 x 4 square area light at height 8 facing down
    (radiance 2), besides its point light."""
    sc = scene_spheres8(seed, width, height, max_depth)
    sc.area_lights = area_lights([(-2.0, 8.0, -2.0)], [(4.0, 0.0, 0.0)], [(0.0, 0.0, 4.0)], [(2.0, 2.0, 2.0)])
    sc.name = sc.name + "_area"
    return sc


def scene_spheres8_emitters(seed: int = 1, width: int = 256, height: int = 256, max_depth: int = 3) -> Scene:
    """spheres8 with emissive primitives as lights besides its point light
    (Eq. 7's L_e): sphere 2 glows (emission (2, 1.5, 1)), sphere 5 is glass
    (IOR 1.5), and a tilted 2 x 2 quad of two triangles at height 6 emits
    (1, 1, 2) from both faces."""
    sc = scene_spheres8(seed, width, height, max_depth)
    mats = sc.materials.copy()
    mats["emission"][3] = (2.0, 1.5, 1.0)
    mats[6] = material(MAT_DIELECTRIC, (1.0, 1.0, 1.0), ks=0.0, ior=1.5)[0]
    mats = np.concatenate([mats, material(MAT_DIFFUSE, (0.0, 0.0, 0.0), ks=0.0, emission=(1.0, 1.0, 2.0))])
    c = np.array((-1.0, 6.0, -1.0))
    eu, ev = np.array((2.0, 0.4, 0.0)), np.array((0.0, -0.3, 2.0))
    quad = triangles_from([c, c], [c + eu, c + eu + ev], [c + eu + ev, c + ev], len(mats) - 1)
    sc.materials = mats
    sc.triangles = np.concatenate([sc.triangles, quad])
    sc.name = sc.name + "_emit"
    return sc


def single_sphere(width=65, height=65, albedo=(0.7, 0.5, 0.3), light=(0.0, 0.0, 10.0),
                  eye=(0.0, 0.0, 5.0), radius=1.0, ks=0.0) -> Scene:
    """One unit sphere at the origin, one light, no ground: a closed-form Lambert image."""
    mats = material(MAT_DIFFUSE, albedo, ks=ks)
    sph = spheres_from(np.zeros((1, 3)), [radius], [0])
    return Scene("single_sphere", sph, np.zeros(0, TRIANGLE_DTYPE), mats,
                 lights([light], [(1, 1, 1)]), camera(eye, (0, 0, 0)), width, height, 0)


CONFIGS = {
    "spheres8": scene_spheres8,
    "terrain": scene_terrain,
}
