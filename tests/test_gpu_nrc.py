"""GPU radiance cache against the FP64 network oracle, through the C ABI.

The GPU computes in BF16 with FP32 accumulation; the oracle runs in FP64 on
the same BF16-rounded weights and features, with its hidden activations
rounded to BF16 as the network stores them.  Bars: outputs within 1e-2
relative, gradients with cosine >= 0.999 and relative norm error <= 1e-2,
Adam exactly as its closed form on the GPU's own gradient.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1504_03151_b300 as rtb
from paper_1504_03151_b300 import build as rtb_build
from paper_1504_03151_b300 import scenes as S

pytestmark = pytest.mark.gpu

LAYERS = [(0, 64, 96), (6144, 64, 64), (10240, 64, 64), (14336, 64, 64), (18432, 3, 64)]


@pytest.fixture(scope="module", autouse=True)
def built(gpu):
    rtb_build.build()
    torch.cuda.set_device(0)


def bf16(x):
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _scene():
    sc = S.scene_terrain(seed=7, width=96, height=64, max_depth=5, cells=(16, 12), n_ico=6, ico_level=2)
    return sc, rtb.Scene(sc).build()


def _bbox(sc):
    V = np.concatenate([sc.triangles["v0"], sc.triangles["v1"], sc.triangles["v2"]]).astype(np.float64)
    return V.min(0), V.max(0)


def _samples(sc, n, rng):
    lo, hi = _bbox(sc)
    p = rng.uniform(lo, hi, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.concatenate([p, nrm, v], 1).astype(np.float32)


def _oracle_inputs(sc, pnv):
    # The kernel forms x_hat = (p - lo) * (1 / extent) in FP32; the sin/cos of
    # 2^11 pi x_hat magnify any difference there, so the oracle encodes the
    # same FP32 x_hat (an identity box) and the rest in FP64.
    lo, hi = _bbox(sc)
    lo32, hi32 = lo.astype(np.float32), hi.astype(np.float32)
    inv32 = np.float32(1.0) / (hi32 - lo32)
    xh = ((pnv[:, :3].astype(np.float32) - lo32) * inv32).astype(np.float32)
    q = np.concatenate([xh.astype(np.float64), pnv[:, 3:].astype(np.float64)], 1)
    return bf16(O.nrc_encode(q, np.zeros(3), np.ones(3)))


def _split(params):
    return bf16(params[:O.N_W]), params[O.N_W:].astype(np.float64)


def test_nrc_inference_matches_oracle():
    sc, scene = _scene()
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=3))
    rng = np.random.default_rng(0)
    n = 1000   # several 128-row tiles and a ragged tail
    pnv = _samples(sc, n, rng)
    out = torch.full((n * 3,), float("nan"), device="cuda")
    rtb.rt_nrc_infer(nrc, scene.handle, torch.from_numpy(pnv).cuda(), n, out)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    g = out.view(n, 3).double().cpu().numpy()
    W, B = _split(rtb.rt_nrc_get_params(nrc))
    ref = O.mlp_forward(_oracle_inputs(sc, pnv), W, B, bf16_acts=True)
    assert np.isfinite(g).all()
    rel = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3)
    # Where an activation sits on a BF16 rounding boundary, FP32 and FP64
    # accumulation may round it to neighbouring values: a few outputs move
    # by one such step; every other output agrees to rounding noise.
    q = np.quantile(rel, [0.5, 0.99, 0.999, 1.0])
    # against the plain FP64 network (activations not rounded): the BF16
    # activations of the network's definition are the only difference
    ref64 = O.mlp_forward(_oracle_inputs(sc, pnv), W, B, bf16_acts=False)
    rel64 = np.abs(g - ref64) / np.maximum(np.abs(ref64), 1e-3)
    q64 = np.quantile(rel64, [0.5, 0.99, 0.999, 1.0])
    print("vs BF16-activation oracle", q, "vs plain FP64 oracle", q64)
    assert q[0] <= 1e-5 and q[1] <= 1e-2 and q[3] <= 1e-2, q
    # The network's BF16 activations put it off the FP64 network by up to
    # about 2 % (0.2 % rounding per activation, through four layers; measured
    # on B300: median 2.5e-3, 99th percentile 1.0e-2, max 1.7e-2).  The GPU
    # may be off the FP64 output by the oracle's own BF16 gap at that output
    # plus the 1e-2 bar, and its median stays within the 1e-2 bar.
    ref16 = O.mlp_forward(_oracle_inputs(sc, pnv), W, B, bf16_acts=True)
    gap = np.abs(ref16 - ref64)
    assert (np.abs(g - ref64) <= gap + 1e-2 * np.maximum(np.abs(ref64), 1e-3)).all()
    assert q64[0] <= 1e-2, q64
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def _cos(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))


def test_nrc_gradients_and_adam_match_oracle():
    sc, scene = _scene()
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=5))
    rng = np.random.default_rng(1)
    n = 700
    pnv = _samples(sc, n, rng)
    target = rng.uniform(0.05, 1.5, (n, 3)).astype(np.float32)
    p0 = rtb.rt_nrc_get_params(nrc)
    rtb.rt_nrc_train_step(nrc, scene.handle, torch.from_numpy(pnv).cuda(), torch.from_numpy(target).cuda(), n)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    g, loss = rtb.rt_nrc_get_grads(nrc)
    W, B = _split(p0)
    ref_loss, dW, dB = O.mlp_loss_grad(_oracle_inputs(sc, pnv), target.astype(np.float64), W, B, bf16_acts=True)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    for off, rows, cols in LAYERS:
        a = g[off:off + rows * cols].astype(np.float64)
        b = dW[off:off + rows * cols]
        assert _cos(a, b) >= 0.999, (off, _cos(a, b))
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-12, (off, np.linalg.norm(a - b), np.linalg.norm(b))
    gb = g[O.N_W:].astype(np.float64)
    assert _cos(gb, dB) >= 0.999
    assert np.linalg.norm(gb - dB) <= 1e-2 * np.linalg.norm(dB)
    # Against the plain FP64 gradient (no BF16 rounding of activations and
    # backward signals).  Rounding each per-sample term to BF16 (2^-9
    # relative) is magnified where the sum over samples cancels, so the
    # network's own BF16 definition sits measurably off the FP64 gradient;
    # the oracle measures that gap on these inputs (bf16 vs plain), and the
    # GPU may be off the FP64 gradient by 1.5 times it plus the 1e-2 bar.
    l64, dW64, dB64 = O.mlp_loss_grad(_oracle_inputs(sc, pnv), target.astype(np.float64), W, B, bf16_acts=False)
    assert loss == pytest.approx(l64, rel=1e-2)
    for off, rows, cols in LAYERS + [(O.N_W, 1, O.N_B)]:
        a = g[off:off + rows * cols].astype(np.float64)
        b64 = (dW64[off:off + rows * cols] if off < O.N_W else dB64)
        bb = (dW[off:off + rows * cols] if off < O.N_W else dB)
        gap_cos = 1.0 - _cos(bb, b64)
        gap_rel = np.linalg.norm(bb - b64) / np.linalg.norm(b64)
        c64 = _cos(a, b64)
        r64 = np.linalg.norm(a - b64) / np.linalg.norm(b64)
        print(f"layer at {off}: GPU vs FP64 cos {c64:.6f} rel {r64:.4f}; BF16 oracle vs FP64 cos {1 - gap_cos:.6f} "
              f"rel {gap_rel:.4f}")
        assert c64 >= 1.0 - (2.0 * gap_cos + 1e-3), (off, c64, gap_cos)
        assert r64 <= 1.5 * gap_rel + 1e-2, (off, r64, gap_rel)
    # Adam's first step from zero moments: w - lr * g / (|g| + eps) on the GPU's own gradient
    p1 = rtb.rt_nrc_get_params(nrc)
    exp = p0.astype(np.float64) - 1e-2 * g / (np.abs(g.astype(np.float64)) + 1e-8)
    np.testing.assert_allclose(p1, exp, rtol=0, atol=2e-6)
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def test_nrc_gradients_many_tiles_per_sm():
    # More tiles than two per SM (the training kernel keeps two in flight on
    # each SM and accumulates every tile of a CTA into one gradient row), a
    # ragged last tile; the same step on two caches of one seed gives the
    # same gradient bit for bit.
    sc, scene = _scene()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 128 * (2 * sms + sms // 2) + 77
    rng = np.random.default_rng(11)
    pnv = _samples(sc, n, rng)
    target = rng.uniform(0.05, 1.5, (n, 3)).astype(np.float32)
    pd, td = torch.from_numpy(pnv).cuda(), torch.from_numpy(target).cuda()
    grads = []
    for _ in range(2):
        nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=5))
        p0 = rtb.rt_nrc_get_params(nrc)
        rtb.rt_nrc_train_step(nrc, scene.handle, pd, td, n)
        assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
        grads.append(rtb.rt_nrc_get_grads(nrc))
        rtb.rt_nrc_destroy(nrc)
    (g, loss), (g2, loss2) = grads
    assert np.array_equal(g, g2) and loss == loss2
    W, B = _split(p0)
    ref_loss, dW, dB = O.mlp_loss_grad(_oracle_inputs(sc, pnv), target.astype(np.float64), W, B, bf16_acts=True)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    for off, rows, cols in LAYERS:
        a = g[off:off + rows * cols].astype(np.float64)
        b = dW[off:off + rows * cols]
        assert _cos(a, b) >= 0.999, (off, _cos(a, b))
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-12, (off, np.linalg.norm(a - b), np.linalg.norm(b))
    gb = g[O.N_W:].astype(np.float64)
    assert _cos(gb, dB) >= 0.999
    assert np.linalg.norm(gb - dB) <= 1e-2 * np.linalg.norm(dB)
    scene.close()


@pytest.mark.parametrize("tiles_per_sm", [0, 1, 3])
@pytest.mark.parametrize("extra", [1, 128, 129])
def test_nrc_gradients_edge_batches(tiles_per_sm, extra):
    # Batches around the kernel's boundaries: a single sample, whole tiles,
    # one past a tile, and CTAs whose two slots hold an odd number of tiles
    # (the second slot idle in the last round).
    sc, scene = _scene()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 128 * sms * tiles_per_sm + extra
    rng = np.random.default_rng(100 + n)
    pnv = _samples(sc, n, rng)
    target = rng.uniform(0.05, 1.5, (n, 3)).astype(np.float32)
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=6))
    p0 = rtb.rt_nrc_get_params(nrc)
    rtb.rt_nrc_train_step(nrc, scene.handle, torch.from_numpy(pnv).cuda(), torch.from_numpy(target).cuda(), n)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    g, loss = rtb.rt_nrc_get_grads(nrc)
    W, B = _split(p0)
    ref_loss, dW, dB = O.mlp_loss_grad(_oracle_inputs(sc, pnv), target.astype(np.float64), W, B, bf16_acts=True)
    assert np.isfinite(g).all()
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    ref = np.concatenate([dW, dB])
    assert _cos(g.astype(np.float64), ref) >= 0.999
    assert np.linalg.norm(g.astype(np.float64) - ref) <= 1e-2 * np.linalg.norm(ref)
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def test_nrc_training_reduces_loss():
    sc, scene = _scene()
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=9))
    rng = np.random.default_rng(2)
    n = 4096
    pnv = _samples(sc, n, rng)
    target = (0.3 + 0.2 * np.sin(pnv[:, :3])).astype(np.float32)   # a smooth function of position
    pd, td = torch.from_numpy(pnv).cuda(), torch.from_numpy(target).cuda()
    losses = []
    for _ in range(60):
        rtb.rt_nrc_train_step(nrc, scene.handle, pd, td, n)
        losses.append(rtb.rt_nrc_get_grads(nrc)[1])
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.2 * losses[0], losses[::10]
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def _gpu_bbox32(sc):
    lo, hi = _bbox(sc)
    lo32, hi32 = lo.astype(np.float32), hi.astype(np.float32)
    return lo32.astype(np.float64), (np.float32(1.0) / (hi32 - lo32)).astype(np.float64)


def _render_nrc(scene, nrc, sc, train, flags=0, ray_counts=None):
    W, H = sc.width, sc.height
    out = torch.full((W * H * 3,), float("nan"), device="cuda")
    st = rtb.rt_render_nrc(scene.handle, nrc, sc.camera, W, H, sc.max_depth, out, train=train,
                           options=rtb.make_options(background=sc.background, flags=flags, ray_counts=ray_counts),
                           stats=True)
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    return out.view(-1, 3).double().cpu().numpy(), st


@pytest.mark.parametrize("flags", [0, rtb.RT_FLAG_PER_DEPTH_WAVEFRONT])
def test_cached_frame_matches_oracle(flags):
    """rt_render_nrc without training: hits at depth 2 read the cache; the
    oracle terminates the same hits with the same (BF16) network.  Both
    pipeline modes (depth-first paths, per-depth wavefronts)."""
    from gpu_helpers import compare
    sc, scene = _scene()
    sc.background = (0.1, 0.1, 0.1)
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=11))
    # a few training steps so that the cache's answers vary over the scene
    rng = np.random.default_rng(4)
    pnv = _samples(sc, 2048, rng)
    tgt = (0.2 + 0.1 * np.cos(pnv[:, :3])).astype(np.float32)
    for _ in range(5):
        rtb.rt_nrc_train_step(nrc, scene.handle, torch.from_numpy(pnv).cuda(), torch.from_numpy(tgt).cuda(), 2048)
    params = rtb.rt_nrc_get_params(nrc)
    D = sc.max_depth
    px = torch.full((sc.width * sc.height * 2 * (D + 1),), -1, device="cuda", dtype=torch.int32)
    img, st = _render_nrc(scene, nrc, sc, train=False, flags=flags | rtb.RT_FLAG_COUNT_WORK, ray_counts=px)
    orc = O.OracleScene.from_scene(sc)
    lo, inv = _gpu_bbox32(sc)
    orc.set_cache(2, params, lo, inv, bf16=True)
    ref = orc.render(sc.camera, sc.width, sc.height, D, mode="brute", per_pixel=True)
    g = {"rgb": img, "prim": ref["prim"], "t": ref["t"],   # primary AOVs are checked elsewhere
         "px": px.view(-1, D + 1, 2).cpu().numpy().astype(np.uint32)}
    from gpu_helpers import cached_colour_tol
    # per-pixel ray counts exact outside the exempted pixels
    rep = compare(g, ref, budget=5e-3, colour_tol=cached_colour_tol(ref["rgb"]))
    c = ref["counts"]
    assert st["primary"] == c["primary"]
    for k in ("shadow", "secondary"):
        assert abs(st[k] - c[k]) <= rep["count_slack_rays"], (k, st[k], c[k], rep)
    assert sum(st["rays_per_depth"][3:]) == 0            # nothing is traced past the cache
    assert (g["px"][:, 3:, :] == 0).all()
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def _relmse(x, r):
    return float(np.mean((x - r) ** 2 / (r ** 2 + 0.01)))


def test_trained_cache_beats_truncation():
    """Online training on the tracer's own depth-2 radiance: after a few
    dozen frames the cached image is closer to the full-depth trace than
    the trace truncated at depth 2 is."""
    sc = S.scene_terrain(seed=2, width=192, height=108, max_depth=5)
    scene = rtb.Scene(sc).build()
    W, H = sc.width, sc.height
    full = torch.empty(W * H * 3, device="cuda")
    rtb.rt_render(scene.handle, sc.camera, W, H, 5, full)
    trunc = torch.empty(W * H * 3, device="cuda")
    rtb.rt_render(scene.handle, sc.camera, W, H, 2, trunc)
    full = full.view(-1, 3).double().cpu().numpy()
    trunc = trunc.view(-1, 3).double().cpu().numpy()
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=1))
    for _ in range(64):
        _render_nrc(scene, nrc, sc, train=True)
    img, st = _render_nrc(scene, nrc, sc, train=False)
    e_cache, e_trunc = _relmse(img, full), _relmse(trunc, full)
    print(f"relMSE cache {e_cache:.3e}, truncated {e_trunc:.3e}")
    assert np.isfinite(img).all()
    assert e_cache < e_trunc
    rtb.rt_nrc_destroy(nrc)
    scene.close()


@pytest.mark.parametrize("flags", [0, rtb.RT_FLAG_PER_DEPTH_WAVEFRONT])
def test_training_frame_image_and_rays(flags):
    """A training frame shows the same cached image as an inference-only
    frame (training rays write targets, not pixels) and traces the
    training rays to full depth."""
    sc, scene = _scene()
    nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=13))
    a, sa = _render_nrc(scene, nrc, sc, train=False, flags=flags)
    b, sb = _render_nrc(scene, nrc, sc, train=True, flags=flags)
    np.testing.assert_allclose(a, b, atol=1e-5)
    assert sum(sa["rays_per_depth"][3:]) == 0
    assert sum(sb["rays_per_depth"][3:]) > 0 or sb["hits_per_depth"][2] == 0
    p1 = rtb.rt_nrc_get_params(nrc)
    assert np.isfinite(p1).all()
    rtb.rt_nrc_destroy(nrc)
    scene.close()


def test_nrc_save_and_load(tmp_path):
    """rt_nrc_save / rt_nrc_load restore parameters, Adam moments and step:
    a loaded cache infers exactly as the saved one and takes the same next
    training step.  Damaged or foreign files are refused and leave the
    cache as it was."""
    sc, scene = _scene()
    rng = np.random.default_rng(4)
    n = 2048
    pnv = _samples(sc, n, rng)
    target = (0.3 + 0.2 * np.sin(pnv[:, :3])).astype(np.float32)
    pd, td = torch.from_numpy(pnv).cuda(), torch.from_numpy(target).cuda()
    a = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=3))
    for _ in range(5):
        rtb.rt_nrc_train_step(a, scene.handle, pd, td, n)
    path = tmp_path / "cache.rtbnrc"
    rtb.rt_nrc_save(a, path)
    b = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=99))   # other weights
    before = rtb.rt_nrc_get_params(b)
    raw = path.read_bytes()
    for bad in (raw[:-4], raw + b"x", b"XXXXXXXX" + raw[8:]):
        (tmp_path / "bad").write_bytes(bad)
        with pytest.raises(rtb.RtError) as ei:
            rtb.rt_nrc_load(b, tmp_path / "bad")
        assert ei.value.status == rtb.RT_ERR_INVALID_ARG
    np.testing.assert_array_equal(rtb.rt_nrc_get_params(b), before)
    with pytest.raises(rtb.RtError):
        rtb.rt_nrc_load(b, tmp_path / "missing")
    rtb.rt_nrc_load(b, path)
    np.testing.assert_array_equal(rtb.rt_nrc_get_params(b), rtb.rt_nrc_get_params(a))
    oa = torch.empty(n * 3, device="cuda")
    ob = torch.empty(n * 3, device="cuda")
    rtb.rt_nrc_infer(a, scene.handle, pd, n, oa)
    rtb.rt_nrc_infer(b, scene.handle, pd, n, ob)
    assert torch.equal(oa, ob)
    # the same next step: the Adam moments and the step count came along
    rtb.rt_nrc_train_step(a, scene.handle, pd, td, n)
    rtb.rt_nrc_train_step(b, scene.handle, pd, td, n)
    np.testing.assert_array_equal(rtb.rt_nrc_get_params(b), rtb.rt_nrc_get_params(a))
    assert rtb.rt_scene_sync(scene.handle) == rtb.RT_OK
    rtb.rt_nrc_destroy(a)
    rtb.rt_nrc_destroy(b)
    scene.close()
