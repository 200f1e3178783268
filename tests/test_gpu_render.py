"""GPU parity of the CUDA tracer against the FP64 oracle, through the C ABI."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

from gpu_helpers import COLOUR_TOL, check_totals, compare, gpu_render, oracle_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(gpu):
    rtb_build.build()
    torch.cuda.set_device(0)


def small_terrain(w=96, h=64, depth=5, seed=7):
    return S.scene_terrain(seed=seed, width=w, height=h, max_depth=depth, cells=(16, 12), n_ico=6, ico_level=2)


def large_terrain():
    """222,208 triangles: above 2^17, so the build sorts all 30 bits of the
    Morton codes (four passes) instead of their top 24."""
    return S.scene_terrain(seed=3, width=64, height=48, cells=(384, 256))


# ---------------------------------------------------------------------------
# closed forms on the GPU
# ---------------------------------------------------------------------------
def test_lambert_sphere_closed_form():
    sc = S.single_sphere(width=65, height=65)
    g = gpu_render(sc, use_bvh=True)
    o, d = O.camera_rays(sc.camera, 65, 65)
    tca = -(o * d).sum(1)
    dist2 = (o * o).sum(1) - tca ** 2
    hit = dist2 <= 1.0
    p = o + (tca - np.sqrt(np.clip(1 - dist2, 0, None)))[:, None] * d
    l = np.array([0, 0, 10.0]) - p
    l /= np.linalg.norm(l, axis=1, keepdims=True)
    exp = np.where(hit[:, None], np.array([0.7, 0.5, 0.3]) * np.clip((p * l).sum(1), 0, None)[:, None], 0.1)
    edge = np.abs(dist2 - 1.0) < 1e-4          # silhouette pixels: hit/miss decided by rounding
    err = np.abs(g["rgb"] - exp).max(axis=1)
    assert err[~edge].max() < 1e-5
    np.testing.assert_array_equal(g["prim"][~edge] >= 0, hit[~edge])


def test_camera_rays_match_oracle():
    for sc in (S.scene_spheres8(width=37, height=23), S.scene_terrain(width=64, height=36)):
        W, H = sc.width, sc.height
        o = torch.empty(W * H * 3, device="cuda")
        d = torch.empty(W * H * 3, device="cuda")
        rtb.rt_camera_rays(sc.camera, W, H, o, d)
        torch.cuda.synchronize()
        ro, rd = O.camera_rays(sc.camera, W, H)
        np.testing.assert_allclose(o.view(-1, 3).cpu().numpy(), ro, atol=1e-6)
        np.testing.assert_allclose(d.view(-1, 3).cpu().numpy(), rd, atol=1e-6)


# ---------------------------------------------------------------------------
# image parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("use_bvh", [False, True])
def test_spheres8_parity(use_bvh):
    sc = S.scene_spheres8()
    ref = oracle_render(sc, mode="brute", per_pixel=True)
    g = gpu_render(sc, use_bvh=use_bvh, per_pixel=True)
    rep = compare(g, ref)
    assert rep["max_err_robust"] < 1e-4, rep
    check_totals(g, sc.max_depth)
    st = g["stats"]
    c = ref["counts"]
    assert st["primary"] == c["primary"] == 256 * 256
    for k in ("shadow", "secondary"):
        assert abs(st[k] - c[k]) <= rep["count_slack_rays"], (k, st[k], c[k], rep)
    print(rep)


def test_terrain_small_parity_all_modes():
    sc = small_terrain()
    ref = oracle_render(sc, mode="brute", per_pixel=True)
    gb = gpu_render(sc, use_bvh=False, per_pixel=True)
    gv = gpu_render(sc, use_bvh=True, per_pixel=True)
    compare(gb, ref)
    compare(gv, ref)
    check_totals(gv, sc.max_depth)
    # BVH and brute force on the GPU: same FP32 tests, same answer
    np.testing.assert_array_equal(gb["prim"], gv["prim"])
    np.testing.assert_allclose(gb["rgb"], gv["rgb"], atol=1e-5)


@pytest.mark.parametrize("wh", [(1, 1), (7, 3), (37, 23), (8, 4), (129, 65)])
def test_ragged_sizes(wh):
    W, H = wh
    sc = S.scene_spheres8(width=W, height=H)
    ref = oracle_render(sc, mode="brute")
    g = gpu_render(sc)
    compare(g, ref, budget=1.0 if W * H < 1000 else 1e-3)


def test_terrain_1080p_full_frame_parity():
    """The benchmark frame, every pixel: ids, colours and, per pixel and
    depth, the closest-hit and shadow rays, against the oracle."""
    sc = S.scene_terrain()
    g = gpu_render(sc, per_pixel=True)
    ref = oracle_render(sc, mode="bvh", per_pixel=True)
    rep = compare(g, ref)
    check_totals(g, sc.max_depth)
    st = g["stats"]
    c = ref["counts"]
    assert st["primary"] == 1920 * 1080
    # outside the exempted pixels the counts match exactly (compare); the
    # totals differ by at most what the exempted pixels hold
    for k in ("shadow", "secondary"):
        assert abs(st[k] - c[k]) <= rep["count_slack_rays"], (k, st[k], c[k], rep)
    print(rep)
    # the same frame rendered without counting: identical image
    g2 = gpu_render(sc)
    assert np.abs(g2["rgb"] - g["rgb"]).max() <= 1e-5
    np.testing.assert_array_equal(g2["prim"], g["prim"])


def test_depth_zero_and_max_depth():
    sc = S.scene_spheres8(width=64, height=64)
    for D in (0, 1, 16):
        ref = oracle_render(sc, mode="brute", max_depth=D, per_pixel=True)
        g = gpu_render(sc, max_depth=D, per_pixel=True)
        compare(g, ref, budget=2e-3)
        check_totals(g, D)
        if D == 0:
            assert g["stats"]["secondary"] == 0


# ---------------------------------------------------------------------------
# intersection parity on the GPU's own FP32 rays
# ---------------------------------------------------------------------------
def _gpu_closest(scene, o, d, use_bvh=True):
    n = len(o)
    od = torch.from_numpy(np.ascontiguousarray(o, np.float32)).cuda()
    dd = torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda()
    prim = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    rtb.rt_trace_closest(scene.handle, od, dd, n, 0.0, use_bvh, prim, t)
    torch.cuda.synchronize()
    return prim.cpu().numpy(), t.double().cpu().numpy()


def test_intersection_parity_on_gpu_rays():
    for sc in (S.scene_spheres8(), S.scene_terrain(width=480, height=270)):
        W, H = sc.width, sc.height
        o = torch.empty(W * H * 3, device="cuda")
        d = torch.empty(W * H * 3, device="cuda")
        rtb.rt_camera_rays(sc.camera, W, H, o, d)
        o = o.view(-1, 3).cpu().numpy()
        d = d.view(-1, 3).cpu().numpy()
        scene = rtb.Scene(sc).build()
        gp, gt = _gpu_closest(scene, o, d)
        scene.close()
        orc = O.OracleScene.from_scene(sc)
        rp, rt, rb = orc.closest_hits(o, d, use_bvh=True)
        robust = rb >= 1
        assert not ((gp != rp) & robust).any()
        assert (gp != rp).mean() <= 1e-3
        m = (gp == rp) & (rp >= 0) & robust
        assert (np.abs(gt[m] - rt[m]) / rt[m]).max() <= 1e-5


def test_random_rays_bvh_equals_bruteforce_and_oracle():
    sc = small_terrain()
    rng = np.random.default_rng(5)
    n = 20000
    o = np.stack([rng.uniform(-34, 34, n), rng.uniform(-2, 12, n), rng.uniform(-26, 26, n)], 1).astype(np.float32)
    tgt = np.stack([rng.uniform(-32, 32, n), rng.uniform(-3, 5, n), rng.uniform(-24, 24, n)], 1)
    d = tgt - o
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    scene = rtb.Scene(sc).build()
    p1, t1 = _gpu_closest(scene, o, d, True)
    p0, t0 = _gpu_closest(scene, o, d, False)
    np.testing.assert_array_equal(p1, p0)
    orc = O.OracleScene.from_scene(sc)
    rp, rt, rb = orc.closest_hits(o, d, use_bvh=True)
    assert not ((p1 != rp) & (rb >= 1)).any()
    # any hit on (0, tmax)
    tmax = rng.uniform(1, 60, n).astype(np.float32)
    occ = torch.empty(n, dtype=torch.uint8, device="cuda")
    rtb.rt_trace_any(scene.handle, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                     torch.from_numpy(tmax).cuda(), n, 0.0, True, occ)
    torch.cuda.synchronize()
    g_occ = occ.cpu().numpy().astype(bool)
    r_occ, r_rb = orc.any_hits(o, d, tmax, use_bvh=True)
    assert not ((g_occ != r_occ) & (r_rb >= 1)).any()
    assert (g_occ != r_occ).mean() <= 1e-3
    scene.close()


# ---------------------------------------------------------------------------
# BVH structure
# ---------------------------------------------------------------------------
def _walk(nodes, root, n_prims):
    """Visits the traversal layout from the root; returns leaf ranges and depth."""
    seen = np.zeros(n_prims, np.int32)
    max_depth = 0
    stack = [(root, 1)]
    internal = 0
    links = nodes[:, 12:14].view(np.int32)
    while stack:
        node, depth = stack.pop()
        internal += 1
        max_depth = max(max_depth, depth)
        for c in range(2):
            link = int(links[node, c])
            if link < 0:
                v = ~link
                start, cnt = v >> 3, (v & 7) + 1
                seen[start:start + cnt] += 1
            else:
                stack.append((link, depth + 1))
    return seen, max_depth, internal


def _child_box(nodes, node, c):
    n = nodes[node]
    if c == 0:
        return np.array([n[0], n[2], n[8]]), np.array([n[1], n[3], n[9]])
    return np.array([n[4], n[6], n[10]]), np.array([n[5], n[7], n[11]])


@pytest.mark.parametrize("which", ["spheres8", "terrain_small", "terrain", "terrain_large"])
def test_bvh_structure_invariants(which):
    sc = {"spheres8": S.scene_spheres8, "terrain_small": small_terrain, "terrain": S.scene_terrain,
          "terrain_large": large_terrain}[which]()
    n = sc.n_prims
    scene = rtb.Scene(sc).build()
    info = rtb.rt_bvh_get_info(scene.handle)
    nodes, order, morton = rtb.rt_bvh_export(scene.handle, n, 2 * max(n, 2))
    scene.close()
    # the sort: a permutation, codes ascending, equal codes keep index order
    assert np.array_equal(np.sort(order), np.arange(n))
    assert (np.diff(morton.astype(np.int64)) >= 0).all()
    eq = np.diff(morton.astype(np.int64)) == 0
    assert (np.diff(order)[eq] > 0).all()
    # every primitive in exactly one leaf reachable from the root
    root = info["root"]
    seen, depth, internal = _walk(nodes, root, n)
    assert (seen == 1).all()
    assert depth == info["max_depth"] and internal == info["n_nodes"]
    assert depth <= 64
    # every child box holds its primitives (leaf boxes) / child's children
    prim_lo = np.zeros((n, 3))
    prim_hi = np.zeros((n, 3))
    ns = len(sc.spheres)
    if ns:
        c, r = sc.spheres["center"].astype(np.float64), sc.spheres["radius"].astype(np.float64)
        prim_lo[:ns], prim_hi[:ns] = c - r[:, None], c + r[:, None]
    if len(sc.triangles):
        V = np.stack([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]], 1).astype(np.float64)
        prim_lo[ns:], prim_hi[ns:] = V.min(1), V.max(1)
    links = nodes[:, 12:14].view(np.int32)
    stack = [root]
    while stack:
        node = stack.pop()
        for c in range(2):
            lo, hi = _child_box(nodes, node, c)
            link = int(links[node, c])
            if link < 0:
                v = ~link
                ids = order[(v >> 3):(v >> 3) + (v & 7) + 1]
                tol = 1e-6 * (1 + np.abs(prim_lo[ids]).max())
                assert (prim_lo[ids] >= lo - tol).all() and (prim_hi[ids] <= hi + tol).all()
            else:
                for cc in range(2):
                    clo, chi = _child_box(nodes, link, cc)
                    assert (clo >= lo).all() and (chi <= hi).all()
                stack.append(link)
    # refinement never makes the tree worse than the plain LBVH by SAH
    assert info["sah_cost"] <= info["sah_cost_lbvh"] * 1.001 or which == "spheres8"


def test_rebuilds_sort_the_same():
    """The single-launch sort's digit counts are made by the Morton kernel
    and by each pass's scatter, and cleared after use: every rebuild of a
    scene (24-bit keys, and 30-bit keys above 2^17 primitives) sorts the
    same, and an update that changes the geometry sorts its new codes."""
    for sc in (S.scene_terrain(), large_terrain()):
        n = sc.n_prims
        scene = rtb.Scene(sc).build()
        first = rtb.rt_bvh_export(scene.handle, n, 2 * n)
        for _ in range(3):
            rtb.rt_bvh_build(scene.handle)
            _, order, morton = rtb.rt_bvh_export(scene.handle, n, 2 * n)
            assert np.array_equal(order, first[1]) and np.array_equal(morton, first[2])
        tris = sc.triangles.copy()
        for k in ("v0", "v1", "v2"):
            tris[k][:, 1] *= 0.5                     # flatten: new codes
        rtb.rt_scene_update(scene.handle, sc.spheres, tris)
        rtb.rt_bvh_build(scene.handle)
        _, order, morton = rtb.rt_bvh_export(scene.handle, n, 2 * n)
        assert np.array_equal(np.sort(order), np.arange(n))
        assert (np.diff(morton.astype(np.int64)) >= 0).all()
        eq = np.diff(morton.astype(np.int64)) == 0
        assert (np.diff(order)[eq] > 0).all()
        assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
        scene.close()


def _prim_boxes(sc):
    n = sc.n_prims
    lo, hi = np.zeros((n, 3)), np.zeros((n, 3))
    ns = len(sc.spheres)
    if ns:
        c, r = sc.spheres["center"].astype(np.float64), sc.spheres["radius"].astype(np.float64)
        lo[:ns], hi[:ns] = c - r[:, None], c + r[:, None]
    if len(sc.triangles):
        V = np.stack([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]], 1).astype(np.float64)
        lo[ns:], hi[ns:] = V.min(1), V.max(1)
    return lo, hi


def _binary_leaves(nodes, root):
    links = nodes[:, 12:14].view(np.int32)
    leaves, stack = set(), [root]
    while stack:
        node = stack.pop()
        for c in range(2):
            link = int(links[node, c])
            if link < 0:
                leaves.add(link)
            else:
                stack.append(link)
    return leaves


@pytest.mark.parametrize("which", ["single", "spheres8", "terrain_small", "terrain"])
def test_wide_bvh_structure(which):
    """The 4-wide tree the kernels walk, from the binary root: a tree over
    the binary tree's leaves (same leaves, each reached once), 2-4 used
    slots a node (one for a single primitive), unused slots
    empty, every box holding what lies below it."""
    sc = {"single": lambda: S.single_sphere(width=8, height=8), "spheres8": S.scene_spheres8,
          "terrain_small": small_terrain, "terrain": S.scene_terrain}[which]()
    n = sc.n_prims
    scene = rtb.Scene(sc).build()
    info = rtb.rt_bvh_get_info(scene.handle)
    bnodes, order, _ = rtb.rt_bvh_export(scene.handle, n, 2 * max(n, 2))
    wide = rtb.rt_bvh_export_wide(scene.handle)
    scene.close()
    assert len(wide) >= max(info["n_nodes"], 1)
    box_lo = np.stack([wide[:, 0:4], wide[:, 8:12], wide[:, 16:20]], 2).astype(np.float64)    # (node, slot, axis)
    box_hi = np.stack([wide[:, 4:8], wide[:, 12:16], wide[:, 20:24]], 2).astype(np.float64)
    links = wide[:, 24:28].view(np.int32)
    used = wide[:, 28:29].view(np.int32)[:, 0]
    plo, phi = _prim_boxes(sc)
    visited = np.zeros(len(wide), np.int64)
    leaves = []
    stack, depth = [(info["root"], 0)], 0
    while stack:
        node, d = stack.pop()
        visited[node] += 1
        depth = max(depth, d)
        for c in range(int(used[node])):
            link, lo_c, hi_c = int(links[node, c]), box_lo[node, c], box_hi[node, c]
            if link < 0:
                leaves.append(link)
                v = ~link
                ids = order[(v >> 3):(v >> 3) + (v & 7) + 1]
                tol = 1e-6 * (1 + np.abs(plo[ids]).max())
                assert (plo[ids] >= lo_c - tol).all() and (phi[ids] <= hi_c + tol).all()
            else:
                k = int(used[link])
                assert (box_lo[link, :k] >= lo_c).all() and (box_hi[link, :k] <= hi_c).all()
                stack.append((link, d + 1))
    assert visited.max() == 1 and 1 <= visited.sum() <= max(info["n_nodes"], 1)
    r = visited == 1   # the reachable nodes
    assert ((used[r] >= (1 if n == 1 else 2)) & (used[r] <= 4)).all()
    empty = (np.arange(4)[None, :] >= used[:, None]) & r[:, None]
    full = (np.arange(4)[None, :] < used[:, None]) & r[:, None]
    assert (links[empty] == np.iinfo(np.int32).min).all()
    assert np.isposinf(box_lo[empty]).all() and np.isneginf(box_hi[empty]).all()
    assert (links[full] != np.iinfo(np.int32).min).all()
    assert len(leaves) == len(set(leaves))
    assert set(leaves) == _binary_leaves(bnodes, info["root"])
    assert depth <= info["max_depth"]


@pytest.mark.parametrize("which", ["terrain", "terrain_large"])
def test_morton_codes_against_cpu_interleave(which):
    sc = S.scene_terrain() if which == "terrain" else large_terrain()
    n = sc.n_prims
    scene = rtb.Scene(sc).build()
    _, order, morton = rtb.rt_bvh_export(scene.handle, n, 2 * n)
    scene.close()
    V = np.stack([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]], 1).astype(np.float64)
    c = 0.5 * (V.min(1) + V.max(1))
    lo, hi = c.min(0), c.max(0)
    q = np.clip(((c - lo) / (hi - lo) * 1024).astype(np.int64), 0, 1023)

    def spread(v):
        out = np.zeros_like(v)
        for b in range(10):
            out |= ((v >> b) & 1) << (3 * b)
        return out

    code = (spread(q[:, 0]) << 2) | (spread(q[:, 1]) << 1) | spread(q[:, 2])
    # the sort key is the code's top 24 bits for at most 2^17 primitives,
    # all 30 above
    assert (n <= 1 << 17) == (which == "terrain")
    if n <= 1 << 17:
        code &= ~np.int64(63)
    got = morton.astype(np.int64)
    exp = code[order]
    # quantisation may differ by one cell where a centroid sits on a cell edge
    assert (got == exp).mean() > 0.999

    def unspread(v):
        out = np.zeros_like(v)
        for b in range(10):
            out |= ((v >> (3 * b)) & 1) << b
        return out

    for shift in (2, 1, 0):
        assert np.abs(unspread(got >> shift) - unspread(exp >> shift)).max() <= 1


# ---------------------------------------------------------------------------
# host API behaviour
# ---------------------------------------------------------------------------
def test_render_host_matches_device():
    sc = S.scene_spheres8(width=64, height=48)
    g = gpu_render(sc)
    scene = rtb.Scene(sc).build()
    host = np.zeros(64 * 48 * 3, np.float32)
    rtb.rt_render_host(scene.handle, sc.camera, 64, 48, sc.max_depth, host,
                       rtb.make_options(background=sc.background))
    scene.close()
    np.testing.assert_allclose(host.reshape(-1, 3), g["rgb"], atol=1e-6)


def test_scene_update_then_rebuild():
    a = small_terrain(seed=7)
    b = small_terrain(seed=8)
    assert len(a.triangles) == len(b.triangles)
    # only the geometry is replaced: keep a's materials and lights
    b.materials = a.materials.copy()
    b.lights = a.lights.copy()
    scene = rtb.Scene(a).build()
    rtb.rt_scene_update(scene.handle, b.spheres, b.triangles)
    rtb.rt_bvh_build(scene.handle)
    out = torch.empty(b.width * b.height * 3, device="cuda")
    rtb.rt_render_ex(scene.handle, b.camera, b.width, b.height, b.max_depth, out,
                     rtb.make_options(background=b.background))
    torch.cuda.synchronize()
    fresh = gpu_render(b)
    np.testing.assert_allclose(out.view(-1, 3).double().cpu().numpy(), fresh["rgb"], atol=1e-5)
    scene.close()


@pytest.mark.parametrize("flags", [0, rtb.RT_FLAG_PER_DEPTH_WAVEFRONT])
def test_deterministic_frames_are_bit_identical(flags):
    """RT_FLAG_DETERMINISTIC: the pixel sums are 64-bit fixed-point integers,
    so repeated frames agree to the bit (float atomics differ in their last
    bits from run to run), and they agree with the float frame within the
    rounding of the accumulation."""
    sc = S.scene_terrain(seed=7, width=96, height=64, max_depth=5, cells=(16, 12), n_ico=6, ico_level=2)
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    det = rtb.make_options(background=sc.background, flags=flags | rtb.RT_FLAG_DETERMINISTIC)
    imgs = []
    for _ in range(3):
        out = torch.full((W * H * 3,), float("nan"), device="cuda")
        rtb.rt_render_ex(scene.handle, sc.camera, W, H, D, out, det)
        imgs.append(out.cpu().numpy())
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    for img in imgs[1:]:
        assert np.array_equal(img, imgs[0])
    ref = torch.empty(W * H * 3, device="cuda")
    rtb.rt_render_ex(scene.handle, sc.camera, W, H, D, ref, rtb.make_options(background=sc.background, flags=flags))
    np.testing.assert_allclose(imgs[0], ref.cpu().numpy(), atol=1e-5, rtol=0)
    # parity with the oracle holds as for the float frame
    g = oracle_render(sc)
    err = np.abs(imgs[0].reshape(-1, 3).astype(np.float64) - g["rgb"]).max(axis=1)
    assert not ((err > COLOUR_TOL) & (g["robust"] >= 1.0)).any()
    # refused with the radiance cache and by a batch
    nrc = rtb.rt_nrc_create(scene.handle)
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_render_nrc(scene.handle, nrc, sc.camera, W, H, D, ref, train=False, options=det)
    assert ei.value.status == rtb.RT_ERR_UNSUPPORTED
    rtb.rt_nrc_destroy(nrc)
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_batch_create([scene.handle], [sc.camera], [W], [H], D, [ref], det)
    assert ei.value.status == rtb.RT_ERR_UNSUPPORTED
    scene.close()


def test_render_host_async_frames_match_sync():
    """Frames queued back to back through the two device images, each copied
    to its own pinned buffer; a third frame reuses the first image (it waits
    for that image's copy).  Every image equals rt_render_host's."""
    sc = small_terrain(seed=7)
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    opts = rtb.make_options(background=sc.background)
    cams = [sc.camera, S.camera((10.0, 8.0, 20.0), (0.0, 0.0, 0.0)), S.camera((-5.0, 6.0, 15.0), (0.0, 1.0, 0.0))]
    refs = []
    for c in cams:
        ref = np.zeros(W * H * 3, np.float32)
        rtb.rt_render_host(scene.handle, c, W, H, D, ref, opts)
        refs.append(ref)
    outs = [torch.full((W * H * 3,), float("nan")).pin_memory() for _ in range(3)]
    for c, o in zip(cams, outs):
        rtb.rt_render_host_async(scene.handle, c, W, H, D, o, opts)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    for o, ref in zip(outs, refs):
        np.testing.assert_allclose(o.numpy(), ref, atol=1e-5, rtol=0)   # only atomic ordering differs
    scene.close()


def test_step_captured_in_a_cuda_graph():
    """rt_scene_update from a device buffer, rt_bvh_build and rt_render_ex
    are stream-ordered and allocate nothing once a scene has rendered: a
    step captured into a CUDA graph replays the same image, and takes new
    geometry written into the device buffer its copy reads."""
    sc = small_terrain(seed=7)
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    h = scene.handle
    opts = rtb.make_options(background=sc.background)
    tri = torch.from_numpy(sc.triangles.view(np.uint8).reshape(-1).copy()).cuda()
    out = torch.empty(W * H * 3, device="cuda")

    def step():
        rtb.rt_scene_update(h, sc.spheres, tri)
        rtb.rt_bvh_build(h)
        rtb.rt_render_ex(h, sc.camera, W, H, D, out, opts)

    step()
    torch.cuda.synchronize()
    ref = out.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    out.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    assert (out - ref).abs().max().item() < 1e-5          # only atomic ordering differs
    # new geometry in the same buffer: the replayed copy, build and render take it
    tris = sc.triangles.copy()
    for k in ("v0", "v1", "v2"):
        tris[k][:, 1] *= 0.5
    tri.copy_(torch.from_numpy(tris.view(np.uint8).reshape(-1).copy()).cuda())
    g.replay()
    torch.cuda.synchronize()
    got = out.clone()
    step()                                                # the same calls, launched directly
    torch.cuda.synchronize()
    assert (got - out).abs().max().item() < 1e-5
    assert (got - ref).abs().max().item() > 1e-2          # the image did change
    assert rtb.rt_scene_sync(h) == rtb.RT_OK
    scene.close()


def test_frames_with_host_copies_replayed_from_two_graphs():
    """The end-to-end frame loop the benchmark times: graph j repacks from
    upload buffer j, builds, and renders into image j while a side branch
    copies the previous image to pinned host memory and uploads the next
    geometry into buffer 1 - j.  Every host image equals the frame rendered
    directly from the same geometry."""
    from cuda.bindings import runtime as cudart

    def copy_async(dst, src, st):
        n = src.numel() * src.element_size()
        err, = cudart.cudaMemcpyAsync(dst.data_ptr(), src.data_ptr(), n, cudart.cudaMemcpyKind.cudaMemcpyDefault,
                                      st.cuda_stream)
        assert err == cudart.cudaError_t.cudaSuccess

    sc = small_terrain(seed=7)
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    h = scene.handle
    opts = rtb.make_options(background=sc.background)
    geo = []
    for k in range(4):                                   # four frames of different geometry
        t = sc.triangles.copy()
        for v in ("v0", "v1", "v2"):
            t[v][:, 1] *= 1.0 - 0.15 * k
        geo.append(torch.from_numpy(t.view(np.uint8).reshape(-1).copy()).pin_memory())
    host_in = torch.empty_like(geo[0]).pin_memory()      # the pinned input the side branch uploads
    imgs = [torch.empty(W * H * 3, device="cuda") for _ in range(2)]
    stage = [geo[0].cuda() for _ in range(2)]             # valid geometry from the first read on
    host_out = [torch.empty(W * H * 3).pin_memory() for _ in range(2)]
    side = torch.cuda.Stream()

    def frame(j):
        rtb.rt_scene_update(h, sc.spheres, stage[j])
        rtb.rt_bvh_build(h)
        cur = torch.cuda.current_stream()
        side.wait_stream(cur)
        copy_async(host_out[1 - j], imgs[1 - j], side)
        copy_async(stage[1 - j], host_in, side)
        rtb.rt_render_ex(h, sc.camera, W, H, D, imgs[j], opts)
        cur.wait_stream(side)

    host_in.copy_(geo[0])
    for j in (0, 1):
        frame(j)
    torch.cuda.synchronize()
    graphs = [torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()]
    for j in range(2):
        with torch.cuda.graph(graphs[j]):
            frame(j)
    torch.cuda.synchronize()
    copy_async(stage[0], geo[0], torch.cuda.current_stream())
    got = []
    for k in range(4):
        host_in.copy_(geo[(k + 1) % 4])                  # the next frame's geometry, read by this replay
        graphs[k % 2].replay()
        torch.cuda.synchronize()
        if k > 0:
            got.append(host_out[(k - 1) % 2].clone())   # the previous frame's image
    last = 3 % 2
    copy_async(host_out[last], imgs[last], torch.cuda.current_stream())
    torch.cuda.synchronize()
    got.append(host_out[last].clone())
    ref = torch.empty(W * H * 3, device="cuda")
    for k in range(4):
        rtb.rt_scene_update(h, sc.spheres, geo[k].cuda())
        rtb.rt_bvh_build(h)
        rtb.rt_render_ex(h, sc.camera, W, H, D, ref, opts)
        torch.cuda.synchronize()
        assert (got[k] - ref.cpu()).abs().max().item() < 1e-5, k   # only atomic ordering differs
    assert (got[0] - got[3]).abs().max().item() > 1e-2               # the frames differ
    assert rtb.rt_scene_sync(h) == rtb.RT_OK
    scene.close()


def test_scene_update_with_a_bad_material_is_reported():
    """rt_scene_update does not validate; a material index out of range is
    replaced by material 0 on the device and reported by the next sync."""
    a = small_terrain(seed=7)
    scene = rtb.Scene(a).build()
    tris = a.triangles.copy()
    tris["material"][5] = len(a.materials) + 3
    rtb.rt_scene_update(scene.handle, a.spheres, tris)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_ERR_INVALID_ARG
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK          # the flag is cleared once read
    rtb.rt_bvh_build(scene.handle)
    out = torch.empty(a.width * a.height * 3, device="cuda")
    rtb.rt_render_ex(scene.handle, a.camera, a.width, a.height, a.max_depth, out,
                     rtb.make_options(background=a.background))
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    fixed = a.triangles.copy()
    fixed["material"][5] = 0
    b = dataclasses.replace(a, triangles=fixed)
    np.testing.assert_allclose(out.view(-1, 3).double().cpu().numpy(), gpu_render(b)["rgb"], atol=1e-5)
    scene.close()


def test_not_built_is_reported():
    sc = S.scene_spheres8(width=8, height=8)
    scene = rtb.Scene(sc)
    out = torch.empty(8 * 8 * 3, device="cuda")
    with pytest.raises(rtb.RtError) as ei:
        rtb.rt_render(scene.handle, sc.camera, 8, 8, 3, out)
    assert ei.value.status == rtb.RT_ERR_NOT_BUILT
    # brute force needs no BVH
    rtb.rt_render_ex(scene.handle, sc.camera, 8, 8, 3, out, rtb.make_options(use_bvh=False))
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    scene.close()


def test_invalid_render_arguments():
    sc = S.scene_spheres8(width=8, height=8)
    scene = rtb.Scene(sc).build()
    out = torch.empty(8 * 8 * 3, device="cuda")
    for w, h, d in ((0, 8, 3), (8, -1, 3), (8, 8, -1), (8, 8, 17)):
        with pytest.raises(rtb.RtError) as ei:
            rtb.rt_render(scene.handle, sc.camera, w, h, d, out)
        assert ei.value.status == rtb.RT_ERR_INVALID_ARG
    scene.close()


def test_queue_overflow_is_reported_not_hung():
    sc = small_terrain()
    scene = rtb.Scene(sc).build()
    out = torch.empty(sc.width * sc.height * 3, device="cuda")
    rtb.rt_render_ex(scene.handle, sc.camera, sc.width, sc.height, sc.max_depth, out,
                     rtb.make_options(queue_capacity=8))
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_ERR_QUEUE_OVERFLOW
    # the status is cleared once read; a normal render is fine afterwards
    rtb.rt_render(scene.handle, sc.camera, sc.width, sc.height, sc.max_depth, out)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    scene.close()


def test_traversal_limit_is_reported_not_hung():
    sc = small_terrain()
    scene = rtb.Scene(sc).build()
    out = torch.empty(sc.width * sc.height * 3, device="cuda")
    rtb.rt_render_ex(scene.handle, sc.camera, sc.width, sc.height, sc.max_depth, out,
                     rtb.make_options(traversal_cap=1))
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_ERR_TRAVERSAL_LIMIT
    scene.close()


def test_empty_scene_and_single_primitive():
    mats = S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))
    li = S.lights([(0, 10, 0)], [(1, 1, 1)])
    empty = S.Scene("empty", np.zeros(0, S.SPHERE_DTYPE), np.zeros(0, S.TRIANGLE_DTYPE), mats, li,
                    S.camera((0, 0, 5), (0, 0, 0)), 16, 8, 2)
    g = gpu_render(empty)
    np.testing.assert_allclose(g["rgb"], 0.1, atol=0)
    assert (g["prim"] == -1).all() and np.isinf(g["t"]).all()
    one = S.single_sphere(width=33, height=33)
    compare(gpu_render(one), oracle_render(one, mode="brute"))
    tri = S.Scene("tri", np.zeros(0, S.SPHERE_DTYPE),
                  S.triangles_from([(-1, -1, 0)], [(1, -1, 0)], [(0, 1, 0)], 0), mats, li,
                  S.camera((0, 0, 5), (0, 0, 0)), 33, 33, 1)
    # a lone triangle's edges cross 5.6 % of a 33 x 33 image: those pixels are exempt
    compare(gpu_render(tri), oracle_render(tri, mode="brute"), fragile_budget=0.1)


@pytest.mark.parametrize("red_first", [False, True])
def test_exact_ties_go_to_the_lower_primitive_id_on_gpu(red_first):
    """Duplicated primitives (a floor and a sphere, each twice, in two
    colours): the GPU keeps the lower id on the exact tie, as the oracle."""
    import test_oracle_pins as P
    sc = P._duplicated_scene(red_first)
    g = gpu_render(sc)
    hit = g["prim"] >= 0
    assert hit.mean() > 0.5
    assert set(np.unique(g["prim"][hit])) <= {0, 2, 3}
    # every hit is an exact tie, which the rounding model exempts (55 % of
    # the pixels); the tie rule itself is what the assertions above check
    compare(g, oracle_render(sc, mode="brute"), fragile_budget=1.0)


def test_degenerate_triangles_never_hit():
    mats = S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))
    li = S.lights([(0, 10, 0)], [(1, 1, 1)])
    tris = S.triangles_from([(-1, -1, 0), (-5, 0, 0), (0, 0, 0)], [(1, -1, 0), (5, 0, 0), (0, 0, 0)],
                            [(0, 1, 0), (0, 0, 0), (0, 0, 0)], 0)   # a line and a point
    sc = S.Scene("degenerate", np.zeros(0, S.SPHERE_DTYPE), tris, mats, li, S.camera((0, 0, 5), (0, 0, 0)), 33,
                 33, 1)
    g = gpu_render(sc)
    assert set(np.unique(g["prim"])) <= {-1, 0}
    compare(g, oracle_render(sc, mode="brute"), fragile_budget=0.1)   # the lone triangle's edges


@pytest.mark.parametrize("which", ["spheres8", "terrain_small_deep"])
def test_pipeline_modes_agree(which):
    """Depth-first secondary paths (default) and per-depth wavefronts trace
    the same rays with the same FP32 functions: same counts, same image."""
    sc = S.scene_spheres8(width=128, height=96) if which == "spheres8" else small_terrain(depth=8)
    ref = oracle_render(sc, mode="brute")
    g_paths = gpu_render(sc)
    g_wave = gpu_render(sc, flags=rtb.RT_FLAG_PER_DEPTH_WAVEFRONT)
    compare(g_paths, ref)
    compare(g_wave, ref)
    np.testing.assert_array_equal(g_paths["prim"], g_wave["prim"])
    np.testing.assert_allclose(g_paths["rgb"], g_wave["rgb"], atol=1e-5)
    for k in ("primary", "shadow", "secondary", "rays_per_depth", "shadow_per_depth", "hits_per_depth"):
        assert g_paths["stats"][k] == g_wave["stats"][k], k
