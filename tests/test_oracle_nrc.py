"""Pins of the FP64 radiance-cache network oracle (CPU only).

The gradients are checked against central finite differences of the loss
(not against another copy of the backward pass), Adam against its closed
form after one step, and the encoding against values worked by hand.
"""
import math

import numpy as np
import pytest

import oracle as O


def _params(rng, scale=0.3):
    W = rng.normal(0, scale, O.N_W)
    B = rng.normal(0, 0.1, O.N_B)
    return W, B


def test_encoding_hand_values():
    lo, hi = np.array([-1.0, 0.0, 2.0]), np.array([1.0, 4.0, 6.0])
    p = np.array([0.0, 1.0, 5.0])            # x_hat = (0.5, 0.25, 0.75)
    n = np.array([0.0, 1.0, 0.0])
    v = np.array([0.6, 0.0, 0.8])
    f = O.nrc_encode(np.concatenate([p, n, v])[None], lo, hi)[0]
    np.testing.assert_allclose(f[:3], [0.5, 0.25, 0.75], atol=1e-15)
    np.testing.assert_allclose(f[3:6], n)
    np.testing.assert_allclose(f[6:9], v)
    # k = 0: sin(pi x_hat), cos(pi x_hat)
    np.testing.assert_allclose(f[9:12], [1.0, math.sqrt(0.5), math.sqrt(0.5)], atol=1e-15)
    np.testing.assert_allclose(f[12:15], [0.0, math.sqrt(0.5), -math.sqrt(0.5)], atol=1e-15)
    # k = 1: sin(2 pi x_hat) = (0, 1, -1)
    np.testing.assert_allclose(f[15:18], [0.0, 1.0, -1.0], atol=1e-15)
    # k = 11 at x_hat = 0.5: sin(2048 pi * 0.5) = 0, cos = 1
    np.testing.assert_allclose(f[9 + 66], 0.0, atol=1e-12)
    np.testing.assert_allclose(f[9 + 66 + 3], 1.0, atol=1e-12)
    assert (f[81:] == 0).all() and len(f) == 96


def test_forward_closed_form_small():
    # all weights zero except the output bias: y = exp(b_out) for any input
    W = np.zeros(O.N_W)
    B = np.zeros(O.N_B)
    B[-3:] = [0.0, math.log(2.0), -1.0]
    y = O.mlp_forward(np.random.default_rng(0).normal(size=(5, 96)), W, B)
    np.testing.assert_allclose(y, np.tile([1.0, 2.0, math.exp(-1)], (5, 1)), rtol=1e-15)
    # one path: x0 -> h1[0] -> h2[0] -> h3[0] -> h4[0] -> out, all weights 1
    W = np.zeros(O.N_W)
    offs = np.cumsum([0, 96 * 64, 64 * 64, 64 * 64, 64 * 64])
    for o in offs:
        W[o] = 1.0                              # row 0, column 0 of each layer
    x = np.zeros((2, 96))
    x[0, 0] = 0.7
    x[1, 0] = -0.7                              # ReLU kills the negative path
    y = O.mlp_forward(x, W, np.zeros(O.N_B))
    np.testing.assert_allclose(y[0], [math.exp(0.7), 1.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(y[1], [1.0, 1.0, 1.0], rtol=1e-15)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    W, B = _params(rng, 0.15)
    x = rng.normal(0, 1, (6, 96))
    t = rng.uniform(0.1, 2.0, (6, 3))
    loss, dW, dB = O.mlp_loss_grad(x, t, W, B)
    y0 = O.mlp_forward(x, W, B)
    den = y0 ** 2 + 0.01                    # sg(y)^2 + 0.01, frozen at the current y

    def L(Wp, Bp):
        y = O.mlp_forward(x, Wp, Bp)
        return float(np.mean((y - t) ** 2 / den))

    assert loss == pytest.approx(L(W, B), rel=1e-14)
    h = 1e-5
    idx_w = rng.choice(O.N_W, 60, replace=False)
    for i in idx_w:
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h
        Wm[i] -= h
        fd = (L(Wp, B) - L(Wm, B)) / (2 * h)
        assert dW[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    for i in range(O.N_B):
        Bp, Bm = B.copy(), B.copy()
        Bp[i] += h
        Bm[i] -= h
        fd = (L(W, Bp) - L(W, Bm)) / (2 * h)
        assert dB[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adam_first_step_closed_form():
    # from zero moments, bias correction gives m_hat = g, v_hat = g^2, so the
    # first step is -lr * g / (|g| + eps)
    rng = np.random.default_rng(2)
    w = rng.normal(size=1000)
    g = rng.normal(size=1000)
    m = np.zeros(1000)
    v = np.zeros(1000)
    w0 = w.copy()
    O.adam(w, g, m, v, 1, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8)
    np.testing.assert_allclose(w - w0, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-13)
    np.testing.assert_allclose(v, 0.01 * g * g, rtol=1e-13)


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    W, B = _params(rng, 0.1)
    x = rng.normal(0, 1, (64, 96))
    t = np.exp(0.3 * x[:, :3])              # a smooth positive target
    m = np.zeros(O.N_W + O.N_B)
    v = np.zeros(O.N_W + O.N_B)
    p = np.concatenate([W, B])
    first = None
    for step in range(1, 61):
        loss, dW, dB = O.mlp_loss_grad(x, t, p[:O.N_W], p[O.N_W:])
        first = loss if first is None else first
        O.adam(p, np.concatenate([dW, dB]), m, v, step, lr=1e-2)
    last, _, _ = O.mlp_loss_grad(x, t, p[:O.N_W], p[O.N_W:])
    assert last < 0.2 * first


def test_bf16_activation_rounding_option():
    # one path x0 -> h -> ... -> out with all weights 1: h = x0 rounded to BF16
    W = np.zeros(O.N_W)
    offs = np.cumsum([0, 96 * 64, 64 * 64, 64 * 64, 64 * 64])
    for o in offs:
        W[o] = 1.0
    x = np.zeros((1, 96))
    x[0, 0] = 1.0 + 2.0 ** -10          # not representable in BF16 (8 bits of mantissa): rounds to 1
    y = O.mlp_forward(x, W, np.zeros(O.N_B), bf16_acts=True)
    assert y[0, 0] == pytest.approx(math.exp(1.0), rel=1e-15)
    y = O.mlp_forward(x, W, np.zeros(O.N_B), bf16_acts=False)
    assert y[0, 0] == pytest.approx(math.exp(1.0 + 2.0 ** -10), rel=1e-15)


def test_cached_frame_closed_form():
    # A constant cache (all weights 0, output bias log c) at depth 1: a
    # primary hit on a rho = 1 mirror with no lights is exactly c wherever
    # its reflection meets a surface, and the background where it does not.
    from paper_1504_03151_b300 import scenes as S
    big = 50.0
    plane = S.triangles_from([(-big, 0, -big), (-big, 0, -big)], [(-big, 0, big), (big, 0, big)],
                             [(big, 0, big), (big, 0, -big)], 0)
    sph = S.spheres_from([(0.0, 1.5, -1.0)], [1.0], [1])
    mats = np.concatenate([S.material(S.MAT_MIRROR, (0.5, 0.5, 0.5), reflectivity=1.0),
                           S.material(S.MAT_DIFFUSE, (0.8, 0.3, 0.2))])
    cam = S.camera((0, 4, 6), (0, 0, -2))
    orc = O.OracleScene(sph, plane, mats, np.zeros(0, S.LIGHT_DTYPE), background=(0.1, 0.2, 0.3))
    c = np.array([0.25, 0.5, 2.0])
    params = np.zeros(O.N_W + O.N_B)
    params[O.N_W + O.N_B - 3:] = np.log(c)
    plain = orc.render(cam, 40, 30, 3, mode="brute")
    orc.set_cache(1, params, lo=np.zeros(3), inv_ext=np.ones(3), bf16=False)
    cached = orc.render(cam, 40, 30, 3, mode="brute")
    it = orc.render(cam, 40, 30, 3, mode="iterative")
    np.testing.assert_allclose(cached["rgb"], it["rgb"], atol=1e-14)
    on_mirror = plain["prim"] >= 1
    # the reflected ray's fate: hit -> c, miss -> background
    reflected_hit = on_mirror & (np.abs(plain["rgb"] - np.array([0.1, 0.2, 0.3])).max(1) > 1e-12)
    np.testing.assert_allclose(cached["rgb"][reflected_hit], np.tile(c, (reflected_hit.sum(), 1)), atol=1e-14)
    assert reflected_hit.sum() > 20
    assert cached["counts"]["shadow"] == 0
    orc.clear_cache()
    np.testing.assert_array_equal(orc.render(cam, 40, 30, 3, mode="brute")["rgb"], plain["rgb"])


def test_cached_vertex_adds_its_own_emission():
    # The cache stands for the radiance a hit reflects; the hit's own L_e
    # (Eq. 7) is added as at any other hit.  A constant cache c at depth 1
    # behind a rho = 1 mirror: where the reflection meets the emitting
    # sphere the pixel is exactly c + L_e, elsewhere c or the background.
    from paper_1504_03151_b300 import scenes as S
    big = 50.0
    plane = S.triangles_from([(-big, 0, -big), (-big, 0, -big)], [(-big, 0, big), (big, 0, big)],
                             [(big, 0, big), (big, 0, -big)], 0)
    sph = S.spheres_from([(0.0, 1.5, -1.0)], [1.0], [1])
    Le = np.array([0.3, 0.1, 0.05])
    mats = np.concatenate([S.material(S.MAT_MIRROR, (0.5, 0.5, 0.5), reflectivity=1.0),
                           S.material(S.MAT_DIFFUSE, (0.8, 0.3, 0.2), emission=tuple(Le))])
    cam = S.camera((0, 4, 6), (0, 0, -2))
    orc = O.OracleScene(sph, plane, mats, np.zeros(0, S.LIGHT_DTYPE), background=(0.1, 0.2, 0.3))
    Le = Le.astype(np.float32).astype(np.float64)   # the scene's values are FP32
    c = np.array([0.25, 0.5, 2.0])
    params = np.zeros(O.N_W + O.N_B)
    params[O.N_W + O.N_B - 3:] = np.log(c)
    plain = orc.render(cam, 40, 30, 3, mode="brute")
    orc.set_cache(1, params, lo=np.zeros(3), inv_ext=np.ones(3), bf16=False)
    cached = orc.render(cam, 40, 30, 3, mode="brute")
    it = orc.render(cam, 40, 30, 3, mode="iterative")
    np.testing.assert_allclose(cached["rgb"], it["rgb"], atol=1e-14)
    on_mirror = plain["prim"] >= 1
    # with no lights, a reflection that meets the sphere shows exactly its L_e in the plain frame
    sees_sphere = on_mirror & (np.abs(plain["rgb"] - Le).max(1) < 1e-12)
    assert sees_sphere.sum() > 20
    np.testing.assert_allclose(cached["rgb"][sees_sphere], np.tile(c + Le, (sees_sphere.sum(), 1)), atol=1e-14)
    # the sphere seen directly (depth 0, before the cache) shows its L_e
    direct = plain["prim"] == 0
    np.testing.assert_allclose(cached["rgb"][direct], np.tile(Le, (direct.sum(), 1)), atol=1e-14)
