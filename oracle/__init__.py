"""FP64 CPU oracle for the Whitted tracer (ctypes binding of liboracle.so).

TEST INFRASTRUCTURE ONLY.  This is the slow, plain reference the CUDA path
is checked against; only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it.  It imports nothing from the CUDA
package and the CUDA package imports nothing from it.

Inputs are numpy arrays in the byte layout of the C ABI structs (the
seeded generators produce them); every value is promoted to FP64 inside.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int
D = ctypes.c_double

# Multiplier of the FP32 rounding model used to flag decision-fragile rays.
FRAGILE_K = 4.0
EPS_SCALE = 1e-4


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_scene_create.restype = P
        L.orc_scene_create.argtypes = [P, I64, P, I64, P, I64, P, I64, P, D, D]
        L.orc_scene_free.argtypes = [P]
        L.orc_bvh_node_count.restype = I64
        L.orc_bvh_node_count.argtypes = [P]
        L.orc_camera_ray.argtypes = [P, I32, I32, I32, I32, P, P]
        L.orc_render.restype = I32
        L.orc_render.argtypes = [P, P, I32, I32, I32, I32, P, I64, P, P, P, P, P, I32]
        L.orc_render_px.restype = I32
        L.orc_render_px.argtypes = [P, P, I32, I32, I32, I32, P, I64, P, P, P, P, P, P, P, I32]
        L.orc_closest_hits.restype = I32
        L.orc_closest_hits.argtypes = [P, I64, P, P, D, I32, P, P, P, I32]
        L.orc_any_hits.restype = I32
        L.orc_any_hits.argtypes = [P, I64, P, P, D, P, I32, P, P, I32]
        L.orc_sphere_roots.restype = I32
        L.orc_sphere_roots.argtypes = [P, P, P, D, P]
        L.orc_triangle_hit.restype = I32
        L.orc_triangle_hit.argtypes = [P, P, P, P, P, P, P, P]
        L.orc_refract.restype = I32
        L.orc_refract.argtypes = [P, P, D, D, P, P]
        L.orc_nrc_encode.argtypes = [I64, P, P, P, P]
        L.orc_mlp_forward.argtypes = [I64, P, P, P, P]
        L.orc_mlp_loss_grad.restype = D
        L.orc_mlp_loss_grad.argtypes = [I64, P, P, P, P, P, P]
        L.orc_mlp_forward_ex.argtypes = [I64, P, P, P, P, I32]
        L.orc_mlp_loss_grad_ex.restype = D
        L.orc_mlp_loss_grad_ex.argtypes = [I64, P, P, P, P, P, P, I32]
        L.orc_adam.argtypes = [I64, P, P, P, P, I64, D, D, D, D]
        L.orc_set_cache.argtypes = [P, I32, P, P, I32, P, P]
        L.orc_round_bf16.restype = D
        L.orc_round_bf16.argtypes = [D]
        L.orc_set_area_lights.restype = I32
        L.orc_set_area_lights.argtypes = [P, P, I64]
        L.orc_set_pass.argtypes = [P, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.orc_set_diffuse_bounce.argtypes = [P, ctypes.c_int32]
        L.orc_philox4x32.argtypes = [P, P, P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleScene:
    """The oracle's copy of a scene (FP64) plus its own median-split BVH."""

    def __init__(self, spheres, triangles, materials, lights, background=(0.1, 0.1, 0.1),
                 eps_scale=EPS_SCALE, fragile_k=FRAGILE_K):
        self._keep = [np.ascontiguousarray(a) for a in (spheres, triangles, materials, lights)]
        self.n_spheres = len(spheres)
        self.n_triangles = len(triangles)
        bg = _f64(background)
        L = lib()
        h = L.orc_scene_create(_ptr(self._keep[0]), len(spheres), _ptr(self._keep[1]), len(triangles),
                               _ptr(self._keep[2]), len(materials), _ptr(self._keep[3]), len(lights),
                               _ptr(bg), eps_scale, fragile_k)
        if not h:
            raise ValueError("oracle rejected the scene (non-finite value, radius <= 0 or bad material)")
        self._h = h

    @classmethod
    def from_scene(cls, sc, **kw):
        o = cls(sc.spheres, sc.triangles, sc.materials, sc.lights, sc.background, **kw)
        al = getattr(sc, "area_lights", None)
        if al is not None and len(al):
            o.set_area_lights(al)
        return o

    def set_area_lights(self, lights):
        """Parallelogram lights in the rt_area_light layout (12 floats each)."""
        self._alights = np.ascontiguousarray(lights)
        if lib().orc_set_area_lights(self._h, _ptr(self._alights), len(self._alights)) != 0:
            raise ValueError("oracle rejected the area lights (non-finite or degenerate)")

    def set_pass(self, seed=0, index=0, strata=1, jitter=False):
        """The pass later renders use (see orc_set_pass)."""
        lib().orc_set_pass(self._h, int(seed), int(index), int(strata), int(bool(jitter)))

    def set_diffuse_bounce(self, on=True):
        """Monte-Carlo GI for later renders (see orc_set_diffuse_bounce)."""
        lib().orc_set_diffuse_bounce(self._h, int(bool(on)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_scene_free(h)
            self._h = None

    def set_cache(self, depth, params, lo, inv_ext, bf16=True):
        """Terminates hits at `depth` with the radiance cache (params: the
        18,883 FP32 parameters; weights rounded to BF16 when bf16)."""
        params = np.asarray(params, np.float64)
        W = params[:N_W].copy()
        if bf16:
            W = round_bf16(W)
        B = np.ascontiguousarray(params[N_W:N_W + N_B])
        self._cache = (np.ascontiguousarray(W), B, _f64(lo), _f64(inv_ext))
        lib().orc_set_cache(self._h, int(depth), _ptr(self._cache[0]), _ptr(self._cache[1]), int(bf16),
                            _ptr(self._cache[2]), _ptr(self._cache[3]))

    def clear_cache(self):
        lib().orc_set_cache(self._h, -1, None, None, 0, None, None)

    @property
    def bvh_nodes(self) -> int:
        return lib().orc_bvh_node_count(self._h)

    def render(self, camera, width, height, max_depth, mode="bvh", pixels=None, nthreads=0, per_pixel=False):
        """Renders (all or the listed) pixels.  mode: 'brute', 'bvh' or 'iterative'.

        Returns dict(rgb [n,3] f64, prim [n] i32, t [n] f64, robust [n] f64,
        counts dict).  per_pixel: also robust_struct [n] f64 (margins of the
        decisions that change ray counts) and px_counts [n, max_depth+1, 2]
        u32 (closest-hit rays traced at each depth, shadow rays cast from
        each depth's hits), see orc_render_px."""
        m = {"brute": 0, "bvh": 1, "iterative": 2}[mode]
        cam = np.ascontiguousarray(camera)
        if pixels is not None:
            pixels = np.ascontiguousarray(pixels, dtype=np.int64)
            n = len(pixels)
        else:
            n = width * height
        rgb = np.zeros((n, 3))
        prim = np.zeros(n, np.int32)
        t = np.zeros(n)
        robust = np.zeros(n)
        counts = np.zeros(3 + 3 * (max_depth + 1), np.uint64)
        rs = np.zeros(n) if per_pixel else None
        px = np.zeros((n, max_depth + 1, 2), np.uint32) if per_pixel else None
        rc = lib().orc_render_px(self._h, _ptr(cam), width, height, max_depth, m, _ptr(pixels),
                                 n if pixels is not None else 0, _ptr(rgb), _ptr(prim), _ptr(t),
                                 _ptr(robust), _ptr(counts), _ptr(rs), _ptr(px), nthreads)
        if rc != 0:
            raise ValueError("oracle render rejected its arguments")
        per_depth = counts[3:].reshape(max_depth + 1, 3)
        extra = {"robust_struct": rs, "px_counts": px} if per_pixel else {}
        return {**extra,
            "rgb": rgb, "prim": prim, "t": t, "robust": robust,
            "counts": {"primary": int(counts[0]), "shadow": int(counts[1]),
                       "secondary": int(counts[2]),
                       "rays_per_depth": [int(x) for x in per_depth[:, 0]],
                       "shadow_per_depth": [int(x) for x in per_depth[:, 1]],
                       "hits_per_depth": [int(x) for x in per_depth[:, 2]]},
        }

    def closest_hits(self, o, d, tmin=0.0, use_bvh=True, robust=True, nthreads=0):
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        n = len(o)
        prim = np.zeros(n, np.int32)
        t = np.zeros(n)
        rb = np.zeros(n) if robust else None
        lib().orc_closest_hits(self._h, n, _ptr(o), _ptr(d), tmin, int(use_bvh), _ptr(prim), _ptr(t),
                               _ptr(rb), nthreads)
        return prim, t, rb

    def any_hits(self, o, d, tmax, tmin=0.0, use_bvh=True, robust=True, nthreads=0):
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        tmax = np.ascontiguousarray(tmax, np.float32).reshape(-1)
        n = len(o)
        occ = np.zeros(n, np.uint8)
        rb = np.zeros(n) if robust else None
        lib().orc_any_hits(self._h, n, _ptr(o), _ptr(d), tmin, _ptr(tmax), int(use_bvh), _ptr(occ),
                           _ptr(rb), nthreads)
        return occ.astype(bool), rb


def philox4x32(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key (the oracle's)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32(_ptr(c), _ptr(k), _ptr(out))
    return out


def camera_rays(camera, width, height, pixels=None):
    """FP64 pinhole rays (origin, unit direction) for the listed pixels."""
    cam = np.ascontiguousarray(camera)
    if pixels is None:
        pixels = np.arange(width * height)
    o = np.zeros((len(pixels), 3))
    d = np.zeros((len(pixels), 3))
    oo = np.zeros(3)
    dd = np.zeros(3)
    L = lib()
    for i, p in enumerate(pixels):
        L.orc_camera_ray(_ptr(cam), width, height, int(p % width), int(p // width), _ptr(oo), _ptr(dd))
        o[i] = oo
        d[i] = dd
    return o, d


def sphere_roots(o, d, c, r):
    t = np.zeros(2)
    n = lib().orc_sphere_roots(_ptr(_f64(o)), _ptr(_f64(d)), _ptr(_f64(c)), float(r), _ptr(t))
    return t[:n] if n == 2 else (t[:1] if n == 1 else t[:0])


def triangle_hit(o, d, v0, v1, v2):
    t = np.zeros(1)
    u = np.zeros(1)
    v = np.zeros(1)
    hit = lib().orc_triangle_hit(_ptr(_f64(o)), _ptr(_f64(d)), _ptr(_f64(v0)), _ptr(_f64(v1)),
                                 _ptr(_f64(v2)), _ptr(t), _ptr(u), _ptr(v))
    return bool(hit), float(t[0]), float(u[0]), float(v[0])


def refract(d, n, n1, n2):
    """(ok, R, refracted dir) for unit d, unit n facing the ray."""
    R = np.zeros(1)
    dt = np.zeros(3)
    ok = lib().orc_refract(_ptr(_f64(d)), _ptr(_f64(n)), float(n1), float(n2), _ptr(R), _ptr(dt))
    return bool(ok), float(R[0]), dt


# ---- radiance cache network ------------------------------------------------
def round_bf16(x):
    """Nearest BF16 value (ties to even), through FP32, as float64."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


MLP_DIMS = (96, 64, 64, 64, 64, 3)
N_W = sum(MLP_DIMS[i] * MLP_DIMS[i + 1] for i in range(5))
N_B = sum(MLP_DIMS[1:])


def nrc_encode(pnv, bbox_lo, bbox_hi):
    pnv = _f64(pnv).reshape(-1, 9)
    out = np.zeros((len(pnv), 96))
    lib().orc_nrc_encode(len(pnv), _ptr(pnv), _ptr(_f64(bbox_lo)), _ptr(_f64(bbox_hi)), _ptr(out))
    return out


def mlp_forward(x, W, B, bf16_acts=False):
    """bf16_acts: hidden activations rounded to BF16 after the ReLU."""
    x = _f64(x).reshape(-1, 96)
    y = np.zeros((len(x), 3))
    lib().orc_mlp_forward_ex(len(x), _ptr(x), _ptr(_f64(W)), _ptr(_f64(B)), _ptr(y), int(bf16_acts))
    return y


def mlp_loss_grad(x, target, W, B, bf16_acts=False):
    x = _f64(x).reshape(-1, 96)
    tg = _f64(target).reshape(-1, 3)
    dW = np.zeros(N_W)
    dB = np.zeros(N_B)
    loss = lib().orc_mlp_loss_grad_ex(len(x), _ptr(x), _ptr(tg), _ptr(_f64(W)), _ptr(_f64(B)), _ptr(dW),
                                      _ptr(dB), int(bf16_acts))
    return loss, dW, dB


def adam(w, g, m, v, step, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8):
    """In place on float64 arrays w, m, v."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _f64(g)
    lib().orc_adam(len(w), _ptr(w), _ptr(gg), _ptr(m), _ptr(v), int(step), lr, beta1, beta2, eps)
