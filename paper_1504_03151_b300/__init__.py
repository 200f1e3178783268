"""Python binding of librtb.so, the sm_103a Whitted ray tracer.

Argument marshalling only: every step of the tracer runs in the library's
CUDA kernels.  The functions carry the C ABI's names (include/rtb.h).
Device buffers are torch CUDA tensors (or raw device pointers as ints);
host arrays are numpy arrays in the ABI's struct layouts (see ``scenes``).
There is no CPU fallback: if librtb.so is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "RtError", "lib", "rt_abi_version", "rt_last_error", "rt_render_options_default",
    "rt_scene_create", "rt_scene_update", "rt_bvh_build", "rt_bvh_get_info", "rt_bvh_export", "rt_bvh_export_wide",
    "rt_render", "rt_render_ex", "rt_render_host", "rt_render_host_async", "rt_camera_rays", "rt_trace_closest",
    "rt_trace_any", "rt_scene_sync", "rt_scene_destroy", "rt_render_stage_times", "rt_probe_l2_read", "Scene",
    "rt_nrc_config_default", "rt_nrc_create", "rt_nrc_destroy", "rt_nrc_get_params", "rt_nrc_set_params",
    "rt_nrc_get_grads", "rt_nrc_infer", "rt_nrc_train_step", "rt_render_nrc", "rt_nrc_save", "rt_nrc_load",
    "rt_tune", "rt_batch_create", "rt_batch_set_cameras", "rt_batch_render", "rt_batch_autotune",
    "rt_batch_destroy", "rt_render_batch", "rt_batch_render_nrc", "rt_render_nrc_pass", "Batch", "rt_pass", "rt_scene_set_area_lights", "rt_render_pass",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtb.so")

RT_OK = 0
RT_ERR_INVALID_ARG = 1
RT_ERR_OOM = 2
RT_ERR_CUDA = 3
RT_ERR_NOT_BUILT = 4
RT_ERR_QUEUE_OVERFLOW = 5
RT_ERR_TRAVERSAL_LIMIT = 6
RT_ERR_UNSUPPORTED = 7
STATUS_NAMES = {0: "RT_OK", 1: "RT_ERR_INVALID_ARG", 2: "RT_ERR_OOM", 3: "RT_ERR_CUDA", 4: "RT_ERR_NOT_BUILT",
                5: "RT_ERR_QUEUE_OVERFLOW", 6: "RT_ERR_TRAVERSAL_LIMIT", 7: "RT_ERR_UNSUPPORTED"}

RT_FLAG_STAGE_TIMING = 1
RT_FLAG_COUNT_WORK = 2
RT_FLAG_NO_GRAPH = 4
RT_FLAG_PER_DEPTH_WAVEFRONT = 8
RT_FLAG_DIFFUSE_BOUNCE = 16
RT_FLAG_DETERMINISTIC = 32
RT_FLAG_SERIAL_STAGES = 64
RT_MAX_DEPTH = 16


class RtError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class rt_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("look_at", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("vfov_deg", ctypes.c_float)]


class rt_render_options(ctypes.Structure):
    _fields_ = [("use_bvh", ctypes.c_int32), ("flags", ctypes.c_int32), ("background", ctypes.c_float * 3),
                ("eps_scale", ctypes.c_float), ("queue_capacity", ctypes.c_int64),
                ("traversal_cap", ctypes.c_int64), ("ray_counts", ctypes.c_void_p)]


class rt_render_stats(ctypes.Structure):
    _fields_ = [("primary", ctypes.c_uint64), ("shadow", ctypes.c_uint64), ("secondary", ctypes.c_uint64),
                ("rays_per_depth", ctypes.c_uint64 * (RT_MAX_DEPTH + 1)),
                ("shadow_per_depth", ctypes.c_uint64 * (RT_MAX_DEPTH + 1)),
                ("hits_per_depth", ctypes.c_uint64 * (RT_MAX_DEPTH + 1)),
                ("node_visits", ctypes.c_uint64 * 2), ("prim_tests", ctypes.c_uint64 * 2),
                ("node_visits_per_depth", (ctypes.c_uint64 * (RT_MAX_DEPTH + 1)) * 2),
                ("max_visits_per_depth", (ctypes.c_uint32 * (RT_MAX_DEPTH + 1)) * 2),
                ("ms_total", ctypes.c_float), ("ms_trace", ctypes.c_float), ("ms_shadow", ctypes.c_float),
                ("launches", ctypes.c_int32), ("box_tests", ctypes.c_uint64 * 2)]


class rt_nrc_config(ctypes.Structure):
    _fields_ = [("train_batch", ctypes.c_int32), ("terminate_depth", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


RT_NRC_PARAMS = 18883


class rt_tune(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32)]


def make_tune(tile_w=8, tile_h=4, block_threads=128, blocks_per_sm=0) -> rt_tune:
    return rt_tune(tile_w, tile_h, block_threads, blocks_per_sm)


def tune_dict(t: rt_tune) -> dict:
    return {"tile_w": t.tile_w, "tile_h": t.tile_h, "block_threads": t.block_threads,
            "blocks_per_sm": t.blocks_per_sm}


class rt_pass(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("index", ctypes.c_int32), ("strata", ctypes.c_int32),
                ("jitter", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def make_pass(index=0, seed=0, strata=1, jitter=False) -> rt_pass:
    return rt_pass(int(seed), int(index), int(strata), int(bool(jitter)), 0)


class rt_bvh_info(ctypes.Structure):
    _fields_ = [("n_prims", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("root", ctypes.c_int64),
                ("max_depth", ctypes.c_int32),
                ("max_leaf_size", ctypes.c_int32), ("sah_cost", ctypes.c_double),
                ("sah_cost_lbvh", ctypes.c_double), ("build_ms", ctypes.c_float),
                ("build_launches", ctypes.c_int32)]


_lib = None
P = ctypes.c_void_p


def lib():
    """Loads librtb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1504_03151_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        I, I64, F, S = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
        sigs = {
            "rt_abi_version": (I, []),
            "rt_last_error": (ctypes.c_char_p, []),
            "rt_render_options_default": (None, [P]),
            "rt_scene_create": (I, [P, S, P, S, P, S, P, S, P]),
            "rt_scene_update": (I, [P, P, P, P]),
            "rt_bvh_build": (I, [P, P]),
            "rt_bvh_get_info": (I, [P, P, P]),
            "rt_bvh_export": (I, [P, P, I64, P, P, P]),
            "rt_bvh_export_wide": (I, [P, P, I64, P, P]),
            "rt_render": (I, [P, P, I, I, I, P, P]),
            "rt_render_ex": (I, [P, P, I, I, I, P, P, P, P, P, P]),
            "rt_render_host": (I, [P, P, I, I, I, P, P, P]),
            "rt_render_stage_times": (I, [P, P, P, P]),
            "rt_probe_l2_read": (I, [S, I, P, P]),
            "rt_camera_rays": (I, [P, I, I, P, P, P]),
            "rt_trace_closest": (I, [P, P, P, I64, F, I, P, P, P]),
            "rt_trace_any": (I, [P, P, P, P, I64, F, I, P, P]),
            "rt_render_noalloc": (I, [P, P, I, I, I, P, P]),
            "rt_scene_sync": (I, [P, P]),
            "rt_nrc_config_default": (None, [P]),
            "rt_nrc_create": (I, [P, P, P]),
            "rt_nrc_destroy": (I, [P]),
            "rt_nrc_get_params": (I, [P, P, P]),
            "rt_nrc_set_params": (I, [P, P, P]),
            "rt_nrc_get_grads": (I, [P, P, P, P]),
            "rt_nrc_infer": (I, [P, P, P, I64, P, P]),
            "rt_nrc_train_step": (I, [P, P, P, P, I64, P]),
            "rt_render_nrc": (I, [P, P, P, I, I, I, P, I, P, P, P]),
            "rt_batch_create": (I, [P, I, P, P, P, I, P, P, P]),
            "rt_batch_set_cameras": (I, [P, P]),
            "rt_batch_render": (I, [P, P, P, P]),
            "rt_batch_autotune": (I, [P, P, P, P]),
            "rt_batch_destroy": (I, [P]),
            "rt_render_batch": (I, [P, P, P, P, I, I, P, P, P]),
            "rt_batch_render_nrc": (I, [P, P, I, P, P, P]),
            "rt_render_nrc_pass": (I, [P, P, P, I, I, I, P, P, I, P, P, P]),
            "rt_scene_set_area_lights": (I, [P, P, S]),
            "rt_render_pass": (I, [P, P, I, I, I, P, P, P, P, P]),
            "rt_render_host_async": (I, [P, P, I, I, I, P, P, P]),
            "rt_nrc_save": (I, [P, ctypes.c_char_p, P]),
            "rt_nrc_load": (I, [P, ctypes.c_char_p, P]),
            "rt_scene_destroy": (I, [P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _check(status):
    if status != RT_OK:
        raise RtError(status, lib().rt_last_error().decode())
    return status


def _dptr(x):
    """Device pointer of a torch CUDA tensor (or an int); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _hptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("expected a C-contiguous array")
        return a.ctypes.data
    return a.data_ptr()   # a torch CPU tensor (pinned or not)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_camera(cam) -> rt_camera:
    """rt_camera from a CAMERA_DTYPE record (or an rt_camera)."""
    if isinstance(cam, rt_camera):
        return cam
    c = np.asarray(cam).reshape(-1)[0]
    out = rt_camera()
    out.eye[:] = [float(v) for v in c["eye"]]
    out.look_at[:] = [float(v) for v in c["look_at"]]
    out.up[:] = [float(v) for v in c["up"]]
    out.vfov_deg = float(c["vfov_deg"])
    return out


def rt_render_options_default() -> rt_render_options:
    o = rt_render_options()
    lib().rt_render_options_default(ctypes.byref(o))
    return o


def make_options(use_bvh=True, flags=0, background=(0.1, 0.1, 0.1), eps_scale=1e-4, queue_capacity=0,
                 traversal_cap=0, ray_counts=None) -> rt_render_options:
    """ray_counts: None or a CUDA int32/uint32 tensor of H*W*2*(max_depth+1)
    entries (per-pixel ray counts; needs RT_FLAG_COUNT_WORK)."""
    o = rt_render_options_default()
    o.use_bvh = int(bool(use_bvh))
    o.flags = int(flags)
    o.background[:] = [float(v) for v in background]
    o.eps_scale = float(eps_scale)
    o.queue_capacity = int(queue_capacity)
    o.traversal_cap = int(traversal_cap)
    o.ray_counts = None if ray_counts is None else _dptr(ray_counts)
    return o


def stats_dict(s: rt_render_stats, max_depth: int) -> dict:
    n = max_depth + 1
    return {
        "primary": s.primary, "shadow": s.shadow, "secondary": s.secondary,
        "rays_per_depth": list(s.rays_per_depth[:n]), "shadow_per_depth": list(s.shadow_per_depth[:n]),
        "hits_per_depth": list(s.hits_per_depth[:n]),
        "node_visits": list(s.node_visits), "prim_tests": list(s.prim_tests), "box_tests": list(s.box_tests),
        "node_visits_per_depth": [list(s.node_visits_per_depth[k][:n]) for k in range(2)],
        "max_visits_per_depth": [list(s.max_visits_per_depth[k][:n]) for k in range(2)],
        "ms_total": s.ms_total, "ms_trace": s.ms_trace, "ms_shadow": s.ms_shadow, "launches": s.launches,
    }


# ---------------------------------------------------------------------------
# the ABI, call by call
# ---------------------------------------------------------------------------
def rt_abi_version() -> int:
    return lib().rt_abi_version()


def rt_last_error() -> str:
    return lib().rt_last_error().decode()


def rt_scene_create(spheres, triangles, materials, lights) -> int:
    h = P()
    _check(lib().rt_scene_create(_hptr(spheres), len(spheres), _hptr(triangles), len(triangles),
                                 _hptr(materials), len(materials), _hptr(lights), len(lights), ctypes.byref(h)))
    return h.value


def rt_scene_update(scene, spheres, triangles, stream=None):
    """spheres / triangles: numpy arrays, torch CPU tensors or torch CUDA tensors (raw struct bytes)."""
    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "is_cuda") and a.is_cuda:
            return _dptr(a)
        return _hptr(a)
    _check(lib().rt_scene_update(scene, ptr(spheres), ptr(triangles), _stream(stream)))


def rt_bvh_build(scene, stream=None):
    _check(lib().rt_bvh_build(scene, _stream(stream)))


def rt_bvh_get_info(scene, stream=None) -> dict:
    info = rt_bvh_info()
    _check(lib().rt_bvh_get_info(scene, ctypes.byref(info), _stream(stream)))
    return {k: getattr(info, k) for k, _ in rt_bvh_info._fields_}


def rt_bvh_export(scene, n_prims, n_node_slots, stream=None):
    nodes = np.zeros((n_node_slots, 16), np.float32)
    order = np.zeros(n_prims, np.int32)
    morton = np.zeros(n_prims, np.uint32)
    _check(lib().rt_bvh_export(scene, nodes.ctypes.data, n_node_slots, order.ctypes.data, morton.ctypes.data,
                               _stream(stream)))
    return nodes, order, morton


def rt_bvh_export_wide(scene, stream=None):
    """The 4-wide traversal tree: (n, 32) float32 rows (boxes as floats,
    the last 8 words reinterpreted as int32 links / slot count)."""
    n = ctypes.c_int64(0)
    _check(lib().rt_bvh_export_wide(scene, None, 0, ctypes.byref(n), _stream(stream)))
    nodes = np.zeros((max(n.value, 1), 32), np.float32)
    _check(lib().rt_bvh_export_wide(scene, nodes.ctypes.data, n.value, None, _stream(stream)))
    return nodes[:n.value]


def rt_render(scene, camera, width, height, max_depth, out_rgb, stream=None):
    cam = make_camera(camera)
    _check(lib().rt_render(scene, ctypes.byref(cam), width, height, max_depth, _dptr(out_rgb), _stream(stream)))


def rt_render_ex(scene, camera, width, height, max_depth, out_rgb, options=None, aov_prim=None, aov_t=None,
                 stats=False, stream=None):
    cam = make_camera(camera)
    st = rt_render_stats() if stats else None
    _check(lib().rt_render_ex(scene, ctypes.byref(cam), width, height, max_depth, _dptr(out_rgb),
                              ctypes.byref(options) if options is not None else None, _dptr(aov_prim),
                              _dptr(aov_t), ctypes.byref(st) if st is not None else None, _stream(stream)))
    return stats_dict(st, max_depth) if st is not None else None


def rt_render_host(scene, camera, width, height, max_depth, out_host, options=None, stream=None):
    cam = make_camera(camera)
    _check(lib().rt_render_host(scene, ctypes.byref(cam), width, height, max_depth, _hptr(out_host),
                                ctypes.byref(options) if options is not None else None, _stream(stream)))


def rt_render_host_async(scene, camera, width, height, max_depth, out_host, options=None, stream=None):
    """Queues a frame and its copy to the pinned host buffer out_host (complete after rt_scene_sync)."""
    cam = make_camera(camera)
    _check(lib().rt_render_host_async(scene, ctypes.byref(cam), width, height, max_depth, _hptr(out_host),
                                      ctypes.byref(options) if options is not None else None, _stream(stream)))


def rt_probe_l2_read(nbytes, reps=50, stream=None) -> float:
    """The L2 read bandwidth (GB/s) over a buffer of nbytes (a measurement helper)."""
    g = ctypes.c_float()
    _check(lib().rt_probe_l2_read(int(nbytes), int(reps), ctypes.byref(g), _stream(stream)))
    return g.value


def rt_render_stage_times(scene):
    """(ms_total, ms_trace, ms_shadow) of the last frame rendered with RT_FLAG_STAGE_TIMING."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(lib().rt_render_stage_times(scene, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def rt_camera_rays(camera, width, height, o_dev, d_dev, stream=None):
    cam = make_camera(camera)
    _check(lib().rt_camera_rays(ctypes.byref(cam), width, height, _dptr(o_dev), _dptr(d_dev), _stream(stream)))


def rt_trace_closest(scene, o_dev, d_dev, n, tmin, use_bvh, prim_dev, t_dev, stream=None):
    _check(lib().rt_trace_closest(scene, _dptr(o_dev), _dptr(d_dev), n, tmin, int(use_bvh), _dptr(prim_dev),
                                  _dptr(t_dev), _stream(stream)))


def rt_trace_any(scene, o_dev, d_dev, tmax_dev, n, tmin, use_bvh, occluded_dev, stream=None):
    _check(lib().rt_trace_any(scene, _dptr(o_dev), _dptr(d_dev), _dptr(tmax_dev), n, tmin, int(use_bvh),
                              _dptr(occluded_dev), _stream(stream)))


def rt_render_noalloc(scene, camera, width, height, max_depth, out_rgb, stream=None):
    """rt_render without device allocation (fixed scratch; see include/rtb.h for the limits)."""
    cam = make_camera(camera)
    _check(lib().rt_render_noalloc(scene, ctypes.byref(cam), width, height, max_depth, _dptr(out_rgb),
                                   _stream(stream)))


def rt_scene_sync(scene, stream=None) -> int:
    """Waits for the stream; returns the latched kernel status (does not raise)."""
    return lib().rt_scene_sync(scene, _stream(stream))


def rt_scene_destroy(scene):
    _check(lib().rt_scene_destroy(scene))


# ---- radiance cache --------------------------------------------------------
def rt_nrc_config_default(**kw) -> rt_nrc_config:
    c = rt_nrc_config()
    lib().rt_nrc_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def rt_nrc_create(scene, config=None) -> int:
    h = P()
    _check(lib().rt_nrc_create(scene, ctypes.byref(config) if config is not None else None, ctypes.byref(h)))
    return h.value


def rt_nrc_save(nrc, path, stream=None):
    """Writes the cache (configuration, parameters, Adam state) to `path`."""
    _check(lib().rt_nrc_save(nrc, os.fsencode(path), _stream(stream)))


def rt_nrc_load(nrc, path, stream=None):
    """Restores a cache written by rt_nrc_save into `nrc`."""
    _check(lib().rt_nrc_load(nrc, os.fsencode(path), _stream(stream)))


def rt_nrc_destroy(nrc):
    _check(lib().rt_nrc_destroy(nrc))


def rt_nrc_get_params(nrc, stream=None) -> np.ndarray:
    out = np.zeros(RT_NRC_PARAMS, np.float32)
    _check(lib().rt_nrc_get_params(nrc, out.ctypes.data, _stream(stream)))
    return out


def rt_nrc_set_params(nrc, params, stream=None):
    a = np.ascontiguousarray(params, np.float32)
    assert a.size == RT_NRC_PARAMS
    _check(lib().rt_nrc_set_params(nrc, a.ctypes.data, _stream(stream)))


def rt_nrc_get_grads(nrc, stream=None):
    g = np.zeros(RT_NRC_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(lib().rt_nrc_get_grads(nrc, g.ctypes.data, ctypes.byref(loss), _stream(stream)))
    return g, loss.value


def rt_nrc_infer(nrc, scene, pnv_dev, n, out_dev, stream=None):
    _check(lib().rt_nrc_infer(nrc, scene, _dptr(pnv_dev), n, _dptr(out_dev), _stream(stream)))


def rt_nrc_train_step(nrc, scene, pnv_dev, target_dev, n, stream=None):
    _check(lib().rt_nrc_train_step(nrc, scene, _dptr(pnv_dev), _dptr(target_dev), n, _stream(stream)))


def rt_render_nrc(scene, nrc, camera, width, height, max_depth, out_rgb, train=True, options=None, stats=False,
                  stream=None):
    cam = make_camera(camera)
    st = rt_render_stats() if stats else None
    _check(lib().rt_render_nrc(scene, nrc, ctypes.byref(cam), width, height, max_depth, _dptr(out_rgb), int(train),
                               ctypes.byref(options) if options is not None else None,
                               ctypes.byref(st) if st is not None else None, _stream(stream)))
    return stats_dict(st, max_depth) if st is not None else None


def rt_scene_set_area_lights(scene, lights):
    """lights: numpy array in the rt_area_light layout (scenes.AREA_LIGHT_DTYPE)."""
    a = np.ascontiguousarray(lights)
    _check(lib().rt_scene_set_area_lights(scene, a.ctypes.data if len(a) else None, len(a)))


def rt_render_pass(scene, camera, width, height, max_depth, pass_, accum_rgb, options=None, stats=False,
                   stream=None):
    """Renders pass `pass_` (an rt_pass) and folds it into the running mean accum_rgb;
    with stats, returns the pass's ray counts (syncs)."""
    cam = make_camera(camera)
    st = rt_render_stats() if stats else None
    _check(lib().rt_render_pass(scene, ctypes.byref(cam), width, height, max_depth, ctypes.byref(pass_),
                                _dptr(accum_rgb), ctypes.byref(options) if options is not None else None,
                                ctypes.byref(st) if st is not None else None, _stream(stream)))
    return stats_dict(st, max_depth) if st is not None else None


def rt_render_nrc_pass(scene, nrc, camera, width, height, max_depth, pass_, accum_rgb, train=True, options=None,
                       stats=False, stream=None):
    """rt_render_pass with the radiance cache (see rt_render_nrc)."""
    cam = make_camera(camera)
    st = rt_render_stats() if stats else None
    _check(lib().rt_render_nrc_pass(scene, nrc, ctypes.byref(cam), width, height, max_depth, ctypes.byref(pass_),
                                    _dptr(accum_rgb), int(train), ctypes.byref(options) if options is not None else None,
                                    ctypes.byref(st) if st is not None else None, _stream(stream)))
    return stats_dict(st, max_depth) if st is not None else None


def rt_batch_create(scenes, cameras, widths, heights, max_depth, outs, options=None):
    """scenes: rt_scene handles; cameras: camera tuples or rt_camera; outs: device tensors."""
    n = len(scenes)
    sc_arr = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h) if isinstance(h, int) else h for h in scenes])
    cam_arr = (rt_camera * n)(*[make_camera(c) for c in cameras])
    w_arr = (ctypes.c_int32 * n)(*[int(x) for x in widths])
    h_arr = (ctypes.c_int32 * n)(*[int(x) for x in heights])
    o_arr = (ctypes.c_void_p * n)(*[_dptr(o) for o in outs])
    out = ctypes.c_void_p()
    _check(lib().rt_batch_create(sc_arr, n, cam_arr, w_arr, h_arr, int(max_depth), o_arr,
                                 ctypes.byref(options) if options is not None else None, ctypes.byref(out)))
    return out.value


def rt_batch_set_cameras(batch, cameras):
    n = len(cameras)
    cam_arr = (rt_camera * n)(*[make_camera(c) for c in cameras])
    _check(lib().rt_batch_set_cameras(batch, cam_arr))


def rt_batch_render(batch, tune=None, stats=False, max_depth=RT_MAX_DEPTH, stream=None):
    st = rt_render_stats() if stats else None
    _check(lib().rt_batch_render(batch, ctypes.byref(tune) if tune is not None else None,
                                 ctypes.byref(st) if st is not None else None, _stream(stream)))
    return stats_dict(st, max_depth) if st is not None else None


def rt_batch_render_nrc(batch, nrc, train=False, tune=None, stats=False, max_depth=RT_MAX_DEPTH, stream=None):
    """The batch with the radiance cache at its terminate depth (one launch, then inference and training)."""
    st = rt_render_stats() if stats else None
    _check(lib().rt_batch_render_nrc(batch, nrc, int(bool(train)), ctypes.byref(tune) if tune is not None else None,
                                     ctypes.byref(st) if st is not None else None, _stream(stream)))
    return stats_dict(st, max_depth) if st is not None else None


def rt_batch_autotune(batch, stream=None):
    """Returns (best rt_tune, its ms)."""
    t = rt_tune()
    ms = ctypes.c_float()
    _check(lib().rt_batch_autotune(batch, ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return t, ms.value


def rt_batch_destroy(batch):
    _check(lib().rt_batch_destroy(batch))


def rt_render_batch(scenes, cameras, widths, heights, max_depth, outs, tune=None, stream=None):
    """The one-call batch: create, render with `tune`, wait, destroy."""
    n = len(scenes)
    sc_arr = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h) if isinstance(h, int) else h for h in scenes])
    cam_arr = (rt_camera * n)(*[make_camera(c) for c in cameras])
    w_arr = (ctypes.c_int32 * n)(*[int(x) for x in widths])
    h_arr = (ctypes.c_int32 * n)(*[int(x) for x in heights])
    o_arr = (ctypes.c_void_p * n)(*[_dptr(o) for o in outs])
    _check(lib().rt_render_batch(sc_arr, cam_arr, w_arr, h_arr, n, int(max_depth), o_arr,
                                 ctypes.byref(tune) if tune is not None else None, _stream(stream)))


class Batch:
    """Owns an rt_batch over Scene objects (each frame: scene, camera, size, device image)."""

    def __init__(self, scenes, cameras, widths, heights, max_depth, outs, options=None):
        self.scenes = list(scenes)   # keeps the scenes alive
        self.outs = list(outs)
        self.max_depth = max_depth
        self.handle = rt_batch_create([s.handle for s in self.scenes], cameras, widths, heights, max_depth,
                                      self.outs, options)

    def render(self, tune=None, stats=False, stream=None):
        return rt_batch_render(self.handle, tune, stats, self.max_depth, stream)

    def render_nrc(self, nrc, train=False, tune=None, stats=False, stream=None):
        return rt_batch_render_nrc(self.handle, nrc, train, tune, stats, self.max_depth, stream)

    def autotune(self, stream=None):
        return rt_batch_autotune(self.handle, stream)

    def set_cameras(self, cameras):
        rt_batch_set_cameras(self.handle, cameras)

    def close(self):
        if self.handle:
            rt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """Owns an rt_scene handle built from a scenes.Scene-like object."""

    def __init__(self, sc):
        self.sc = sc
        self.handle = rt_scene_create(sc.spheres, sc.triangles, sc.materials, sc.lights)
        al = getattr(sc, "area_lights", None)
        if al is not None and len(al):
            rt_scene_set_area_lights(self.handle, al)

    def build(self, stream=None):
        rt_bvh_build(self.handle, stream)
        return self

    def render(self, out_rgb, options=None, aov_prim=None, aov_t=None, stats=False, camera=None, width=None,
               height=None, max_depth=None, stream=None):
        sc = self.sc
        return rt_render_ex(self.handle, sc.camera if camera is None else camera, width or sc.width,
                            height or sc.height, sc.max_depth if max_depth is None else max_depth, out_rgb,
                            options, aov_prim, aov_t, stats, stream)

    def close(self):
        if self.handle:
            rt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
