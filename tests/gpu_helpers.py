"""Shared helpers of the GPU tests: render through the C ABI and compare with
the FP64 oracle under the parity rules.

Parity rules (floating point decides which primitive is hit, so near-ties
may legitimately differ):
  * a pixel whose oracle path tree has a decision within reach of FP32
    rounding (oracle robust < 1) may differ; every other pixel must match:
    primary hit id bit-exact, colour within 2e-3 max-abs;
  * pixels that do differ (id or colour beyond 2e-3) are at most 0.1 %;
  * primary hit distances agree to 1e-5 relative where the ids match.
"""
import numpy as np
import torch

import oracle as O
import paper_1504_03151_b300 as rtb

COLOUR_TOL = 2e-3
T_REL_TOL = 1e-5
BUDGET = 1e-3


def gpu_render(sc, use_bvh=True, flags=0, width=None, height=None, max_depth=None, **opt):
    W = width or sc.width
    H = height or sc.height
    D = sc.max_depth if max_depth is None else max_depth
    scene = rtb.Scene(sc)
    if use_bvh:
        scene.build()
    out = torch.full((H * W * 3,), float("nan"), device="cuda", dtype=torch.float32)
    prim = torch.full((H * W,), -7, device="cuda", dtype=torch.int32)
    t = torch.full((H * W,), float("nan"), device="cuda", dtype=torch.float32)
    options = rtb.make_options(use_bvh=use_bvh, flags=flags, background=sc.background, **opt)
    st = rtb.rt_render_ex(scene.handle, sc.camera, W, H, D, out, options, prim, t, stats=True)
    torch.cuda.synchronize()
    res = {
        "rgb": out.view(H * W, 3).double().cpu().numpy(),
        "prim": prim.cpu().numpy(),
        "t": t.double().cpu().numpy(),
        "stats": st,
    }
    scene.close()
    return res


def oracle_render(sc, mode="bvh", width=None, height=None, max_depth=None, pixels=None):
    W = width or sc.width
    H = height or sc.height
    D = sc.max_depth if max_depth is None else max_depth
    orc = O.OracleScene.from_scene(sc)
    return orc.render(sc.camera, W, H, D, mode=mode, pixels=pixels)


def compare(gpu, ref, pixels=None, budget=BUDGET):
    """Returns a report dict; raises AssertionError on a parity failure."""
    g_rgb, g_prim, g_t = gpu["rgb"], gpu["prim"], gpu["t"]
    if pixels is not None:
        g_rgb, g_prim, g_t = g_rgb[pixels], g_prim[pixels], g_t[pixels]
    robust = ref["robust"] >= 1.0
    err = np.abs(g_rgb - ref["rgb"]).max(axis=1)
    assert np.isfinite(g_rgb).all(), "non-finite GPU colour"
    bad_c = err > COLOUR_TOL
    bad_p = g_prim != ref["prim"]
    both = (ref["prim"] >= 0) & ~bad_p
    rel_t = np.zeros_like(err)
    rel_t[both] = np.abs(g_t[both] - ref["t"][both]) / ref["t"][both]
    rep = {
        "n": int(len(err)),
        "fragile_frac": float(1 - robust.mean()),
        "colour_mismatch_frac": float(bad_c.mean()),
        "prim_mismatch_frac": float(bad_p.mean()),
        "max_err_robust": float(err[robust].max()) if robust.any() else 0.0,
        "max_rel_t_robust": float(rel_t[robust & both].max()) if (robust & both).any() else 0.0,
    }
    assert not (bad_p & robust).any(), f"primary id differs on robust pixels: {np.where(bad_p & robust)[0][:10]} {rep}"
    assert not (bad_c & robust).any(), f"colour differs on robust pixels: {np.where(bad_c & robust)[0][:10]} {rep}"
    assert rep["colour_mismatch_frac"] <= budget, rep
    assert rep["prim_mismatch_frac"] <= budget, rep
    assert rep["max_rel_t_robust"] <= T_REL_TOL, rep
    return rep
