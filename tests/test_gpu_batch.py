"""Batched rendering (rt_batch_*): many frames of uneven scenes and sizes in
one persistent launch must give the images that rendering each frame alone
gives, and the oracle's, for every tune."""
import numpy as np
import pytest
import torch

import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

from gpu_helpers import COLOUR_TOL, BUDGET, cached_colour_tol, oracle_render

pytestmark = pytest.mark.gpu

SAME_TOL = 1e-5   # the same hits and terms, summed by float atomics in another order
SAME_BUDGET = 1e-3   # pixels allowed past it: the two kernels' FP32 expressions may contract to
                     # FMAs differently, which can flip a decision on a near-tie (a grazing or
                     # total-internal-reflection ray); at scale about 1 pixel in 4 million does


def assert_same_image(a, b):
    err = np.abs(a - b).max(axis=1)
    assert np.isfinite(a).all() and np.isfinite(b).all()
    assert (err > SAME_TOL).mean() <= SAME_BUDGET, (err > SAME_TOL).sum()


@pytest.fixture(scope="module", autouse=True)
def built(gpu):
    rtb_build.build()
    torch.cuda.set_device(0)


def small_terrain(w=72, h=40, depth=3, seed=7):
    return S.scene_terrain(seed=seed, width=w, height=h, max_depth=depth, cells=(16, 12), n_ico=6, ico_level=2)


def single_frame(scene, cam, w, h, depth, background):
    out = torch.empty(w * h * 3, device="cuda")
    rtb.rt_render_ex(scene.handle, cam, w, h, depth, out, rtb.make_options(background=background))
    torch.cuda.synchronize()
    return out.view(h * w, 3).double().cpu().numpy()


@pytest.fixture(scope="module")
def frames():
    """Four frames: three scenes, one of them twice with another camera and
    size; sizes that do not divide into tiles."""
    a = S.scene_spheres8(width=64, height=48, max_depth=3)
    b = small_terrain()
    c = S.single_sphere(width=33, height=17)
    sa, sb, sc_ = rtb.Scene(a).build(), rtb.Scene(b).build(), rtb.Scene(c).build()
    fr = [(sa, a, a.camera, 64, 48), (sb, b, b.camera, 72, 40), (sc_, c, c.camera, 33, 17),
          (sb, b, S.camera((10.0, 8.0, 20.0), (0.0, 0.0, 0.0)), 40, 72)]
    yield fr
    for s in (sa, sb, sc_):
        s.close()


def make_batch(fr, depth=3, background=(0.1, 0.1, 0.1)):
    outs = [torch.full((w * h * 3,), float("nan"), device="cuda") for _, _, _, w, h in fr]
    b = rtb.Batch([f[0] for f in fr], [f[2] for f in fr], [f[3] for f in fr], [f[4] for f in fr], depth, outs,
                  rtb.make_options(background=background))
    return b, outs


def images(outs, fr):
    torch.cuda.synchronize()
    return [o.view(h * w, 3).double().cpu().numpy() for o, (_, _, _, w, h) in zip(outs, fr)]


def test_batch_matches_single_frames(frames):
    b, outs = make_batch(frames)
    b.render()
    for img, (scene, sc, cam, w, h) in zip(images(outs, frames), frames):
        ref = single_frame(scene, cam, w, h, 3, sc.background)
        assert np.isfinite(img).all()
        assert_same_image(img, ref)
    b.close()


def test_batch_matches_oracle():
    """Colour parity with the FP64 oracle (the batch has no hit outputs)."""
    a = S.scene_spheres8(width=48, height=40, max_depth=3)
    c = S.single_sphere(width=33, height=17)
    sa, sc_ = rtb.Scene(a).build(), rtb.Scene(c).build()
    fr = [(sa, a, a.camera, 48, 40), (sc_, c, c.camera, 33, 17)]
    b, outs = make_batch(fr)
    b.render()
    for img, (_, sc, _, w, h) in zip(images(outs, fr), fr):
        ref = oracle_render(sc, mode="brute", width=w, height=h)
        robust = ref["robust"] >= 1.0
        err = np.abs(img - ref["rgb"]).max(axis=1)
        assert not ((err > COLOUR_TOL) & robust).any()
        assert (err > COLOUR_TOL).mean() <= BUDGET
    b.close()
    sa.close()
    sc_.close()


def test_one_call_render_batch(frames):
    """rt_render_batch (create, render, wait, destroy in one call) makes the
    images of the batch handle, background 0.1 (the default options)."""
    fr = [f for f in frames if tuple(f[1].background) == (0.1, 0.1, 0.1)] or frames[:1]
    outs = [torch.full((w * h * 3,), float("nan"), device="cuda") for _, _, _, w, h in fr]
    rtb.rt_render_batch([f[0].handle for f in fr], [f[2] for f in fr], [f[3] for f in fr], [f[4] for f in fr], 3,
                        outs, rtb.make_tune(8, 4, 128, 0))
    for img, (scene, sc, cam, w, h) in zip(images(outs, fr), fr):
        assert_same_image(img, single_frame(scene, cam, w, h, 3, (0.1, 0.1, 0.1)))


@pytest.mark.parametrize("tune", [(8, 4, 128, 0), (4, 8, 64, 0), (16, 2, 256, 0), (32, 1, 128, 2), (1, 32, 64, 1)])
def test_every_tune_gives_the_same_image(frames, tune):
    b, outs = make_batch(frames)
    b.render(rtb.make_tune(*tune))
    for img, (scene, sc, cam, w, h) in zip(images(outs, frames), frames):
        assert_same_image(img, single_frame(scene, cam, w, h, 3, sc.background))
    b.close()


def test_batch_stats_are_the_frames_sums(frames):
    b, outs = make_batch(frames)
    st = b.render(stats=True)
    prim = sec = shadow = 0
    for scene, sc, cam, w, h in frames:
        s1 = rtb.rt_render_ex(scene.handle, cam, w, h, 3, torch.empty(w * h * 3, device="cuda"),
                              rtb.make_options(background=sc.background), stats=True)
        prim += s1["primary"]
        sec += s1["secondary"]
        shadow += s1["shadow"]
    assert st["primary"] == prim == sum(w * h for *_, w, h in frames)
    assert st["secondary"] == sec
    assert st["shadow"] == shadow
    b.close()


def test_many_tiny_frames():
    """40 frames of random sizes (1x1 up to 50x50) over two scenes: the tile
    list, its search and the image edges."""
    rng = np.random.default_rng(5)
    a = S.scene_spheres8(width=8, height=8, max_depth=2)
    c = S.single_sphere(width=8, height=8)
    sa, sc_ = rtb.Scene(a).build(), rtb.Scene(c).build()
    fr = []
    for i in range(40):
        s, sc = (sa, a) if i % 3 else (sc_, c)
        w, h = int(rng.integers(1, 51)), int(rng.integers(1, 51))
        fr.append((s, sc, sc.camera, w, h))
    b, outs = make_batch(fr, depth=2)
    b.render(rtb.make_tune(16, 2, 64, 0))
    for img, (scene, sc, cam, w, h) in zip(images(outs, fr), fr):
        assert_same_image(img, single_frame(scene, cam, w, h, 2, sc.background))
    b.close()
    sa.close()
    sc_.close()


def test_autotune_graph_replay_and_new_cameras(frames):
    b, outs = make_batch(frames)
    tune, ms = b.autotune()
    assert tune.tile_w * tune.tile_h == 32 and tune.block_threads in (64, 128, 256) and ms > 0
    first = images(outs, frames)
    b.render()   # the graph of the chosen tune, replayed
    for x, y in zip(first, images(outs, frames)):
        assert_same_image(x, y)
    cams = [f[2] for f in frames]
    cams[0] = S.camera((3.0, 4.0, 9.0), (0.0, 1.0, 0.0))
    b.set_cameras(cams)
    b.render()
    scene, sc, _, w, h = frames[0]
    assert_same_image(images(outs, frames)[0], single_frame(scene, cams[0], w, h, 3, sc.background))
    b.close()


def test_depth_zero_batch(frames):
    b, outs = make_batch(frames, depth=0)
    st = b.render(stats=True)
    assert st["secondary"] == 0
    for img, (scene, sc, cam, w, h) in zip(images(outs, frames), frames):
        assert_same_image(img, single_frame(scene, cam, w, h, 0, sc.background))
    b.close()


def test_batch_argument_errors(frames):
    scene, sc, cam, w, h = frames[0]
    out = torch.empty(w * h * 3, device="cuda")
    with pytest.raises(rtb.RtError):
        rtb.rt_batch_create([], [], [], [], 3, [])
    with pytest.raises(rtb.RtError):
        rtb.rt_batch_create([scene.handle], [cam], [0], [h], 3, [out])
    with pytest.raises(rtb.RtError):
        rtb.rt_batch_create([scene.handle], [cam], [w], [h], 17, [out])
    with pytest.raises(rtb.RtError):
        rtb.rt_batch_create([scene.handle], [S.camera((0, 0, 0), (0, 0, 0))], [w], [h], 3, [out])
    b = rtb.Batch([scene], [cam], [w], [h], 3, [out])
    for bad in [(5, 6, 128, 0), (8, 4, 96, 0), (8, 4, 128, -1)]:
        with pytest.raises(rtb.RtError):
            b.render(rtb.make_tune(*bad))
    b.close()
    # a scene without a BVH
    c = S.single_sphere(width=8, height=8)
    raw = rtb.Scene(c)
    o2 = torch.empty(8 * 8 * 3, device="cuda")
    b2 = rtb.Batch([raw], [c.camera], [8], [8], 1, [o2])
    with pytest.raises(rtb.RtError) as ei:
        b2.render()
    assert ei.value.status == rtb.RT_ERR_NOT_BUILT
    b2.close()
    raw.close()


# ---------------------------------------------------------------------------
# the radiance cache inside the persistent launch
# ---------------------------------------------------------------------------
def _cache_frames():
    """One terrain with 20 icospheres (its mirrors and glass give the first
    view some 50 hits at depth 2) seen by three cameras at three sizes, and a
    radiance cache on it trained a few steps on smooth targets so that its
    answers vary over the scene."""
    sc = S.scene_terrain(seed=3, width=72, height=40, max_depth=5, cells=(16, 12), n_ico=20, ico_level=1)
    scene = rtb.Scene(sc).build()
    views = [sc.camera, S.camera((10.0, 8.0, 20.0), (0.0, 0.0, 0.0)), S.camera((-12.0, 6.0, -18.0), (0.0, 1.0, 0.0))]
    sizes = [(72, 40), (40, 72), (33, 17)]
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=21))
    V = np.concatenate([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]]).astype(np.float64)
    rng = np.random.default_rng(8)
    n = 2048
    p = rng.uniform(V.min(0), V.max(0), (n, 3))
    nv = rng.normal(size=(n, 6)).reshape(n, 2, 3)
    nv /= np.linalg.norm(nv, axis=2, keepdims=True)
    pnv = np.concatenate([p, nv.reshape(n, 6)], 1).astype(np.float32)
    tgt = (0.2 + 0.1 * np.cos(pnv[:, :3])).astype(np.float32)
    for _ in range(5):
        rtb.rt_nrc_train_step(nrc, scene.handle, torch.from_numpy(pnv).cuda(), torch.from_numpy(tgt).cuda(), n)
    return sc, scene, views, sizes, nrc


def test_batch_cache_matches_cached_frames():
    """rt_batch_render_nrc without training makes, frame by frame, the image
    rt_render_nrc makes with the same network: the same hits read the cache
    at depth 2 and nothing is traced past it."""
    sc, scene, views, sizes, nrc = _cache_frames()
    outs = [torch.full((w * h * 3,), float("nan"), device="cuda") for w, h in sizes]
    b = rtb.Batch([scene] * 3, views, [w for w, _ in sizes], [h for _, h in sizes], 5, outs,
                  rtb.make_options(background=sc.background))
    st = b.render_nrc(nrc, train=False, stats=True)
    assert sum(st["rays_per_depth"][3:]) == 0 and st["hits_per_depth"][2] > 0
    torch.cuda.synchronize()
    for o, v, (w, h) in zip(outs, views, sizes):
        ref = torch.empty(w * h * 3, device="cuda")
        rtb.rt_render_nrc(scene.handle, nrc, v, w, h, 5, ref, train=False,
                          options=rtb.make_options(background=sc.background))
        torch.cuda.synchronize()
        assert_same_image(o.view(h * w, 3).double().cpu().numpy(), ref.view(h * w, 3).double().cpu().numpy())
    b.close()
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def test_batch_cache_matches_oracle():
    """The batched cached frames against the oracle's cached-frame render
    (the same BF16 network at depth 2)."""
    sc, scene, views, sizes, nrc = _cache_frames()
    import oracle as O
    outs = [torch.empty(w * h * 3, device="cuda") for w, h in sizes]
    b = rtb.Batch([scene] * 3, views, [w for w, _ in sizes], [h for _, h in sizes], 5, outs,
                  rtb.make_options(background=sc.background))
    b.render_nrc(nrc, train=False)
    torch.cuda.synchronize()
    params = rtb.rt_nrc_get_params(nrc)
    V = np.concatenate([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]])
    lo32, hi32 = V.min(0).astype(np.float32), V.max(0).astype(np.float32)
    orc = O.OracleScene.from_scene(sc)
    orc.set_cache(2, params, lo32.astype(np.float64), (np.float32(1.0) / (hi32 - lo32)).astype(np.float64), bf16=True)
    for o, v, (w, h) in zip(outs, views, sizes):
        ref = orc.render(v, w, h, 5, mode="brute")
        img = o.view(h * w, 3).double().cpu().numpy()
        err = np.abs(img - ref["rgb"]).max(axis=1)
        robust = ref["robust"] >= 1.0
        bad = err > cached_colour_tol(ref["rgb"])   # the cache's BF16 answers: the bar of the cached-frame tests
        assert not (bad & robust).any(), np.where(bad & robust)[0][:10]
        assert bad.mean() <= 5e-3
    b.close()
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def test_batch_cache_trains_and_checks_its_scene():
    """With training the launch also traces a subset of the cached hits to
    full depth (rays past depth 2), the network moves and stays finite, and
    the image is the inference-only image of the network it started with.
    A frame of another scene is refused."""
    sc, scene, views, sizes, nrc = _cache_frames()
    outs = [torch.empty(w * h * 3, device="cuda") for w, h in sizes]
    b = rtb.Batch([scene] * 3, views, [w for w, _ in sizes], [h for _, h in sizes], 5, outs,
                  rtb.make_options(background=sc.background))
    b.render_nrc(nrc, train=False)
    torch.cuda.synchronize()
    a = [o.clone() for o in outs]
    p0 = rtb.rt_nrc_get_params(nrc)
    st = b.render_nrc(nrc, train=True, stats=True)
    assert sum(st["rays_per_depth"][3:]) > 0
    torch.cuda.synchronize()
    for x, y in zip(a, outs):
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), atol=1e-5)
    p1 = rtb.rt_nrc_get_params(nrc)
    assert np.isfinite(p1).all() and np.abs(p1 - p0).max() > 0
    for _ in range(8):
        b.render_nrc(nrc, train=True)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    assert np.isfinite(rtb.rt_nrc_get_params(nrc)).all()
    other = rtb.Scene(S.scene_spheres8(width=16, height=16)).build()
    o2 = torch.empty(16 * 16 * 3, device="cuda")
    b2 = rtb.Batch([scene, other], views[:1] + [S.scene_spheres8().camera], [72, 16], [40, 16], 5,
                   [outs[0], o2], rtb.make_options(background=sc.background))
    with pytest.raises(rtb.RtError) as ei:
        b2.render_nrc(nrc)
    assert ei.value.status == rtb.RT_ERR_INVALID_ARG
    b2.close()
    other.close()
    b.close()
    rtb.rt_nrc_destroy(nrc)
    scene.close()
