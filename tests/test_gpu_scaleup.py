"""The two large workloads at full size, in the launch configuration the
benchmark times (a batch, autotuned): the four 4K views of the 10.9 M
triangle scale-up scene (depth 8, 8 lights, IOR U[1.3, 1.7]) and the
64-scene batch (16.6 M triangles, 36.8 Mpixel, depth 4).  Sampled pixels
are checked one by one against the FP64 oracle under the parity rule."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

from gpu_helpers import COLOUR_TOL, cached_colour_tol

pytestmark = pytest.mark.gpu

SAMPLE_BUDGET = 5e-3   # sampled pixels that may differ (all of them fragile); 1-2 of a few hundred


@pytest.fixture(scope="module", autouse=True)
def built(gpu):
    rtb_build.build()
    torch.cuda.set_device(0)


def check_sampled(img, ref, tol=COLOUR_TOL, hard_tol=None):
    """Robust pixels within hard_tol (default tol); pixels beyond tol at
    most SAMPLE_BUDGET."""
    hard_tol = tol if hard_tol is None else hard_tol
    robust = ref["robust"] >= 1.0
    err = np.abs(img - ref["rgb"]).max(axis=1)
    assert np.isfinite(img).all()
    assert not ((err > hard_tol) & robust).any(), (np.where((err > hard_tol) & robust)[0], err.max())
    assert (err > tol).mean() <= SAMPLE_BUDGET, (err > tol).sum()


def test_scaleup_four_views_sampled_parity():
    sc = S.scene_scaleup()
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    info = rtb.rt_bvh_get_info(scene.handle)
    assert info["n_prims"] == 10_948_608
    views = S.views_scaleup()
    outs = [torch.empty(W * H * 3, device="cuda") for _ in views]
    b = rtb.Batch([scene] * 4, views, [W] * 4, [H] * 4, D, outs, rtb.make_options(background=sc.background))
    b.autotune()
    st = b.render(stats=True)
    assert st["primary"] == 4 * W * H and st["secondary"] > 0 and st["shadow"] > 0
    torch.cuda.synchronize()
    imgs = [o.view(H * W, 3).double().cpu().numpy() for o in outs]
    orc = O.OracleScene.from_scene(sc)
    rng = np.random.default_rng(11)
    hit_frac = []
    for v, img in zip(views, imgs):
        px = np.sort(rng.choice(W * H, 400, replace=False))
        ref = orc.render(v, W, H, D, mode="bvh", pixels=px)
        check_sampled(img[px], ref)
        hit_frac.append((ref["prim"] >= 0).mean())
    assert min(hit_frac) > 0.3   # the samples see geometry, not just the background
    b.close()
    scene.close()


def test_scaleup_radiance_cache_in_one_launch_sampled_parity():
    """The four 4K views with the radiance cache at depth 2 of 8, in one
    persistent launch (rt_batch_render_nrc, the benchmark's scale-up cache
    leg), against the oracle's cached-frame mode with the same BF16 network
    on sampled pixels."""
    sc = S.scene_scaleup()
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    views = S.views_scaleup()
    outs = [torch.empty(W * H * 3, device="cuda") for _ in views]
    b = rtb.Batch([scene] * 4, views, [W] * 4, [H] * 4, D, outs, rtb.make_options(background=sc.background))
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=1))
    for _ in range(3):                        # a few online steps: the network is no longer its initial one
        b.render_nrc(nrc, train=True)
    st = b.render_nrc(nrc, train=False, stats=True)
    assert st["primary"] == 4 * W * H and sum(st["rays_per_depth"][3:]) == 0
    torch.cuda.synchronize()
    params = rtb.rt_nrc_get_params(nrc)
    V = np.concatenate([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]])
    lo32, hi32 = V.min(0).astype(np.float32), V.max(0).astype(np.float32)
    orc = O.OracleScene.from_scene(sc)
    orc.set_cache(2, params, lo32.astype(np.float64), (np.float32(1.0) / (hi32 - lo32)).astype(np.float64), bf16=True)
    rng = np.random.default_rng(13)
    for v, o in zip(views, outs):
        img = o.view(H * W, 3).double().cpu().numpy()
        px = np.sort(rng.choice(W * H, 300, replace=False))
        ref = orc.render(v, W, H, D, mode="bvh", pixels=px)
        # The encoding's top frequency, 2^11 pi over the scene's 512-unit box,
        # turns the FP32 error of a hit position some 600 units from the
        # camera (about 1.4e-4) into about 2e-3 of feature, about 1 % of
        # output: the oracle's exact positions cannot reproduce that, so a
        # robust pixel may be off by up to 3 % of its value, and pixels past
        # the network's 1e-2 bar are held to the sample budget.
        rel3 = np.maximum(COLOUR_TOL, 3e-2 * np.abs(ref["rgb"]).max(axis=1))
        check_sampled(img[px], ref, cached_colour_tol(ref["rgb"]), hard_tol=rel3)
    rtb.rt_nrc_destroy(nrc)
    b.close()
    scene.close()


def test_sixty_four_scene_batch_sampled_parity():
    scs = S.scene_batch()
    scenes = [rtb.Scene(x).build() for x in scs]
    outs = [torch.empty(x.width * x.height * 3, device="cuda") for x in scs]
    b = rtb.Batch(scenes, [x.camera for x in scs], [x.width for x in scs], [x.height for x in scs], 4, outs,
                  rtb.make_options(background=scs[0].background))
    b.autotune()
    st = b.render(stats=True)
    assert st["primary"] == sum(x.width * x.height for x in scs)
    torch.cuda.synchronize()
    # the largest and the smallest scene, and four more
    order = np.argsort([x.n_prims for x in scs])
    pick = [int(order[0]), int(order[-1])] + [int(i) for i in order[[10, 25, 40, 55]]]
    rng = np.random.default_rng(12)
    for i in pick:
        x = scs[i]
        img = outs[i].view(x.height * x.width, 3).double().cpu().numpy()
        px = np.sort(rng.choice(x.width * x.height, 300, replace=False))
        ref = O.OracleScene.from_scene(x).render(x.camera, x.width, x.height, 4, mode="bvh", pixels=px)
        check_sampled(img[px], ref)
    b.close()
    for s in scenes:
        s.close()
