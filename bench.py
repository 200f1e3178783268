"""Benchmark: Mrays/s of the B300 Whitted tracer on the 1080p / 123,904-triangle
terrain scene at depth 5 (4 point lights, 60/25/15 % diffuse / mirror /
dielectric icospheres), synthetic and seeded.

One step = one pass of the whole hot path over the scene, inputs resident
in HBM: SoA repacking of the geometry (device-to-device), the BVH build
(Morton codes, radix sort, LBVH, binned-SAH top levels, SAH leaf
collapsing) and the frame (primary rays, closest hit + shading, shadow
rays, reflection / refraction rays to depth 5).  Rays counted: primary +
shadow + secondary.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation
of this method here) on a bounded sample of the same workload.
Under torchrun (N > 1) every rank renders its own replica of the frame
(replicas only: the path needs no collective); value = all ranks' rays /
the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mrays/s at 1080p 100k-tri depth 5, plain vs radiance cache at relMSE ≤ 0.01"
UNIT = "Mrays/s"
# algorithmic FP32 operations per unit of work (counted from the math)
OPS_BOX = 14      # ordered slab test of one child box: 6 FFMA + 6 min/max + 1 widening FMUL + 1 compare
OPS_TRI = 30      # Moller-Trumbore
# algorithmic bytes per unit of work: a 4-wide node visit reads its 128-B
# node, a primitive test its 48-B record, and a ray reads its 48-B record
# and writes a 16-B hit (the per-ray figures, as if no ray shared a load)
BYTES_NODE = 128
BYTES_RAY_IO = 48 + 16

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one frame's
# launches of each kernel class, from one ncu capture of the bench workload
# (the summaries are in profiles/).  They stand only for the kernel sources
# they were taken on: any change to those files reports null instead.
PROFILED_SOURCES = ["paper_1504_03151_b300/csrc/render.cu", "paper_1504_03151_b300/csrc/trace_device.cuh",
                    "paper_1504_03151_b300/csrc/rtb_internal.cuh"]
PROFILED_SHA = "ccd6cbd2e027b63a"
PROFILED_TRAFFIC = {
    0: (8_801_792 + 128_627_968 + 5_335_552 + 0 + 7_919_360 + 112_625_920,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of the first frame's k_trace<1,0,0>, k_trace<0,0,0> "
        "(depth 1) and k_paths<0,0> (depths 2-5) launches, one capture per kernel (-k, -c 2 / -c 1); "
        "L2 bytes (lts__t_bytes.sum) 619,376,672"),
    1: (179_826_176 + 7_308_032 + 5_791_488 + 0,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of the first frame's two k_shadow<0> launches "
        "(depths 0, 1), -k k_shadow -c 2; L2 bytes (lts__t_bytes.sum) 722,356,544"),
}


def profiled_traffic(cls):
    """(bytes per frame, source) of a kernel class while its sources match the capture, else (None, why)."""
    import hashlib
    h = hashlib.sha256()
    for f in PROFILED_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != PROFILED_SHA:
        return None, "kernel sources changed since the ncu capture"
    return PROFILED_TRAFFIC[cls]


BYTES_TRI = 48


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return p, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region:
    the sampler runs every 10 ms and is running (its first sample is in)
    before the region starts; samples that arrive while the region runs are
    its record.  A region shorter than one interval is represented by the
    first sample after it (then "samples" is 0)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 10

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.lock = threading.Lock()
        self.window = (0, 0)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0:
                time.sleep(0.005)
        except (FileNotFoundError, OSError):
            self.proc = None
        with self.lock:
            self.window = (len(self.lines), len(self.lines))
        return self

    def _read(self):
        for line in self.proc.stdout:
            with self.lock:
                self.lines.append(line.strip())

    def __exit__(self, *a):
        with self.lock:
            self.window = (self.window[0], len(self.lines))
        if self.proc:
            if self.window[1] == self.window[0]:      # none inside: wait for the next one
                t0 = time.perf_counter()
                while len(self.lines) == self.window[1] and time.perf_counter() - t0 < 1.0:
                    time.sleep(0.002)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        a, b = self.window
        inside = self.lines[a:b]
        lines = inside if inside else self.lines[b:b + 1]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(inside), "interval_ms": self.INTERVAL_MS}


def oracle_threads():
    """The host threads the oracle's OpenMP loop uses (all cores unless OMP_NUM_THREADS says otherwise)."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_oracle_sample(sc):
    """Times the FP64 oracle as it stands: brute force over every primitive
    on a bounded pixel sample of the frame, and its own median-split BVH
    (proven equal to brute force) on the full frame.  Returns the cpu_baseline
    object; its value is the BVH mode's full-frame Mrays/s."""
    import oracle as O
    orc = O.OracleScene.from_scene(sc)
    W, H = sc.width, sc.height
    stride = 101             # prime: an even spread of ~20,000 pixels over the frame (10-30 s)
    pix = np.arange(0, W * H, stride)
    t0 = time.perf_counter()
    r = orc.render(sc.camera, W, H, sc.max_depth, mode="brute", pixels=pix)
    dt = time.perf_counter() - t0
    c = r["counts"]
    rays = c["primary"] + c["shadow"] + c["secondary"]
    t0 = time.perf_counter()
    f = orc.render(sc.camera, W, H, sc.max_depth, mode="bvh")
    dtf = time.perf_counter() - t0
    cf = f["counts"]
    rays_f = cf["primary"] + cf["shadow"] + cf["secondary"]
    return {"value": rays_f / dtf / 1e6, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
            "sample": f"the oracle's BVH mode over the full frame ({W * H} px, {rays_f} rays, {dtf:.1f} s)",
            "bvh_full_frame_s": dtf,
            "brute_force": {"value": rays / dt / 1e6, "unit": UNIT,
                            "sample": f"every {stride}th pixel of the frame ({len(pix)} px, {rays} rays, {dt:.1f} s)"}}


def max_over_ranks(x, dist, device="cpu"):
    """The largest of the ranks' values of x (the slowest rank's time); x
    itself on one rank (dist None)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def copy_async(dst, src, st):
    """One cudaMemcpyAsync of src into dst on stream st (pinned host or device
    tensors): a plain copy node when a CUDA graph is being captured."""
    from cuda.bindings import runtime as cudart
    n = src.numel() * src.element_size()
    assert dst.numel() * dst.element_size() == n
    err, = cudart.cudaMemcpyAsync(dst.data_ptr(), src.data_ptr(), n, cudart.cudaMemcpyKind.cudaMemcpyDefault,
                                  st.cuda_stream)
    if err != cudart.cudaError_t.cudaSuccess:
        raise RuntimeError(f"cudaMemcpyAsync: {err}")


def job_throughput(world, rays_per_rank, ms):
    """Whole-job Mrays/s: every rank traces rays_per_rank a step, and the
    job's step lasts as long as its slowest rank's (ms)."""
    return world * rays_per_rank / (ms * 1e3)


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle on the host cores."""
    from paper_1504_03151_b300 import scenes as S
    if rank != 0:
        return
    sc = S.scene_terrain()
    import oracle as O
    orc = O.OracleScene.from_scene(sc)
    W, H = sc.width, sc.height
    # The oracle's BVH mode (the mode of cpu_baseline's value).  A warm-up
    # step on every 97th pixel measures its cost a pixel; the timed steps
    # then take every stride-th pixel (offset by the step), the stride sized
    # so that all of them together take about two minutes: the full frame
    # (stride 1) when K is small enough.
    per_px = 0.0
    for w in range(max(args.warmup, 1)):
        pix = np.arange(w % 97, W * H, 97)
        t0 = time.perf_counter()
        orc.render(sc.camera, W, H, sc.max_depth, mode="bvh", pixels=pix)
        per_px = (time.perf_counter() - t0) / len(pix)
    budget_s = 120.0 / max(args.steps, 1)
    stride = max(1, int(np.ceil(per_px * W * H / budget_s)))
    times, rays, n_px = [], 0, 0
    for k in range(args.steps):
        pix = None if stride == 1 else np.arange(k % stride, W * H, stride)
        t0 = time.perf_counter()
        r = orc.render(sc.camera, W, H, sc.max_depth, mode="bvh", pixels=pix)
        times.append(time.perf_counter() - t0)
        c = r["counts"]
        rays += c["primary"] + c["shadow"] + c["secondary"]
        n_px += W * H if pix is None else len(pix)
    total = sum(times)
    value = rays / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "terrain 1920x1080, 123904 triangles (fBm 256x192 + 20 L3 icospheres), depth 5, "
                               "4 point lights, materials 60/25/15",
                   "sample": f"each step: every {stride}th pixel (offset by the step index), "
                             f"{n_px / args.steps:.0f} px a step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": f"the oracle's BVH mode, every {stride}th pixel a step ({n_px} px, {rays} rays, "
                                   f"{total:.1f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_leg(rtb, S, torch, dev, stream, flush, steps):
    """64 scenes of uneven size (log-uniform 1e3-2e6 triangles, 16.6 M in all)
    and resolution (256^2 .. 1280x720, 36.8 Mpixel), depth 4, in one
    persistent launch; beside it, the same frames as one rt_render_ex each."""
    scs = S.scene_batch()
    D = 4
    scenes = [rtb.Scene(x) for x in scs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for x in scenes:            # first builds allocate the scratch
        x.build()
    torch.cuda.synchronize()
    e0.record(stream)
    for x in scenes:
        x.build()
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    outs = [torch.empty(x.width * x.height * 3, device=dev) for x in scs]
    opts = rtb.make_options(background=scs[0].background)
    b = rtb.Batch(scenes, [x.camera for x in scs], [x.width for x in scs], [x.height for x in scs], D, outs, opts)
    tune, tune_ms = b.autotune()
    st = b.render(stats=True)
    rays = st["primary"] + st["shadow"] + st["secondary"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        b.render()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in ev) / steps
    # the same frames, one launch sequence per frame (warm-up pass allocates their queues)
    for x, sc_, o in zip(scenes, scs, outs):
        rtb.rt_render_ex(x.handle, sc_.camera, sc_.width, sc_.height, D, o, opts)
    torch.cuda.synchronize()
    flush.zero_()
    e0.record(stream)
    for x, sc_, o in zip(scenes, scs, outs):
        rtb.rt_render_ex(x.handle, sc_.camera, sc_.width, sc_.height, D, o, opts)
    e1.record(stream)
    torch.cuda.synchronize()
    per_frame_ms = e0.elapsed_time(e1)
    b.close()
    for x in scenes:
        x.close()
    return {
        "metric": "Mrays/s, 64 scenes in one persistent launch (CUDA graph)", "value": rays / (ms * 1e3),
        "unit": UNIT, "ms_per_render": ms, "rays_per_render": rays, "primary": st["primary"],
        "shadow": st["shadow"], "secondary": st["secondary"],
        "workload": f"{len(scs)} scenes, {sum(x.n_prims for x in scs)} triangles (log-uniform 1e3-2e6), "
                    f"{sum(x.width * x.height for x in scs)} pixels, depth 4, 4 lights",
        "tune": rtb.tune_dict(tune), "autotune_best_ms": tune_ms,
        "per_frame_launches_ms": per_frame_ms, "speedup_vs_per_frame_launches": per_frame_ms / ms,
        "build_all_ms": build_ms, "l2": "flushed between renders",
    }


def scaleup_leg(rtb, S, torch, dev, stream, flush, steps, with_nrc):
    """The scale-up workload: 10,948,608 triangles, four 3840x2160 views,
    depth 8, 8 lights, as one batched launch; then the radiance cache on the
    same views (one network, trained frame after frame) against the plain
    full-depth frames."""
    sc = S.scene_scaleup()
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    scene.build()
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    scene.build()
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    views = S.views_scaleup()
    outs = [torch.empty(W * H * 3, device=dev) for _ in views]
    opts = rtb.make_options(background=sc.background)
    b = rtb.Batch([scene] * 4, views, [W] * 4, [H] * 4, D, outs, opts)
    tune, _ = b.autotune()
    st = b.render(stats=True)
    rays = st["primary"] + st["shadow"] + st["secondary"]
    ts = []
    for k in range(steps):
        flush.zero_()
        e0, e1 = ev(), ev()
        e0.record(stream)
        b.render()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = sum(ts) / len(ts)
    line = {
        "metric": "Mrays/s, 4 views in one persistent launch", "value": rays / (ms * 1e3), "unit": UNIT,
        "ms_per_render": ms, "rays_per_render": rays, "primary": st["primary"], "shadow": st["shadow"],
        "secondary": st["secondary"], "build_ms": build_ms, "tune": rtb.tune_dict(tune),
        "workload": f"{sc.n_prims} triangles (2048x2048-cell terrain + 500 L4 icospheres), 4 views "
                    f"{W}x{H}, depth {D}, {len(sc.lights)} lights",
    }
    if with_nrc:
        # the four views with the cache at depth 2, in one persistent launch
        # (inference and one training step after it), trained online launch
        # after launch; judged against the plain full-depth views above
        full = [o.clone() for o in outs]
        nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=1))
        cached = [torch.empty(W * H * 3, device=dev) for _ in views]
        bn = rtb.Batch([scene] * 4, views, [W] * 4, [H] * 4, D, cached, opts)
        for k in range(32):                      # online training
            bn.render_nrc(nrc, train=True, tune=tune)
        nst = bn.render_nrc(nrc, train=True, tune=tune, stats=True)
        nrays = nst["primary"] + nst["shadow"] + nst["secondary"]
        nms = []
        for k in range(steps):
            flush.zero_()
            e0, e1 = ev(), ev()
            e0.record(stream)
            bn.render_nrc(nrc, train=True, tune=tune)
            e1.record(stream)
            torch.cuda.synchronize()
            nms.append(e0.elapsed_time(e1))
        rel = [float(((x.double() - r.double()) ** 2 / (r.double() ** 2 + 0.01)).mean()) for x, r in zip(cached, full)]
        nrc_ms = sum(nms) / len(nms)
        line["radiance_cache"] = {
            "metric": "Mrays-equivalent/s (full-depth rays of the 4 views per cached launch)",
            "value": rays / (nrc_ms * 1e3), "ms_4_views": nrc_ms, "vs_plain_batch": ms / nrc_ms,
            "relmse_vs_full_depth": rel, "rays_traced_4_views": nrays, "warmup_launches": 32,
            "cache_hits": nst["hits_per_depth"][2],
            "launch": "one persistent launch of the 4 views (rt_batch_render_nrc), the cache's inference over "
                      "their depth-2 hits, one training step (65,536 samples) and Adam",
        }
        bn.close()
        rtb.rt_nrc_destroy(nrc)
    b.close()
    scene.close()
    return line


def passes_leg(rtb, S, torch, dev, stream, flush, steps, with_nrc=True):
    """Progressive passes of the headline terrain with sampled lights (two
    area lights and a glowing sphere besides the 4 point lights), jittered
    camera rays over 4 x 4 strata, depth 5; once with light sampling alone
    and once with the diffuse bounce (Monte-Carlo GI).  Rays per pass are the
    mean of four counted passes."""
    sc = S.scene_terrain_lit()
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc).build()
    acc = torch.empty(W * H * 3, device=dev)
    out = {"metric": "Mrays/s per progressive pass", "unit": UNIT,
           "workload": f"terrain {W}x{H}, {sc.n_prims} primitives, depth {D}, {len(sc.lights)} point lights + "
                       f"{len(sc.area_lights)} area lights + 1 emissive sphere, jittered passes (4x4 strata)",
           "l2": "flushed between passes"}
    for name, flags in (("direct", 0), ("gi", rtb.RT_FLAG_DIFFUSE_BOUNCE)):
        opts = rtb.make_options(background=sc.background, flags=flags)
        counted = [rtb.rt_render_pass(scene.handle, sc.camera, W, H, D, rtb.make_pass(k, 7, 4, True), acc, opts,
                                      stats=True) for k in range(4)]
        rays = sum(c["primary"] + c["shadow"] + c["secondary"] for c in counted) / len(counted)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            rtb.rt_render_pass(scene.handle, sc.camera, W, H, D, rtb.make_pass(4 + k, 7, 4, True), acc, opts)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in ev) / steps
        out[name] = {"value": rays / (ms * 1e3), "ms_per_pass": ms, "rays_per_pass": rays,
                     "shadow_per_pass": sum(c["shadow"] for c in counted) / len(counted),
                     "secondary_per_pass": sum(c["secondary"] for c in counted) / len(counted)}
    if with_nrc:
        # the radiance cache fed by GI paths: passes with the diffuse bounce
        # whose depth-2 hits read the cache, trained online on the GI paths
        # a seeded subset traces to full depth; Mrays-equivalent = the
        # full-depth GI pass's rays / the cached pass's time (with training)
        opts = rtb.make_options(background=sc.background, flags=rtb.RT_FLAG_DIFFUSE_BOUNCE)
        nrc = rtb.rt_nrc_create(scene.handle, rtb.rt_nrc_config_default(seed=1))
        for k in range(64):
            rtb.rt_render_nrc_pass(scene.handle, nrc, sc.camera, W, H, D, rtb.make_pass(k, 7, 4, True), acc, True,
                                   opts)
        nst = rtb.rt_render_nrc_pass(scene.handle, nrc, sc.camera, W, H, D, rtb.make_pass(64, 7, 4, True), acc, True,
                                     opts, stats=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            rtb.rt_render_nrc_pass(scene.handle, nrc, sc.camera, W, H, D, rtb.make_pass(65 + k, 7, 4, True), acc,
                                   True, opts)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in ev) / steps
        # judged on the mean of 8 passes against the mean of the same 8 full-depth passes
        full = torch.empty(W * H * 3, device=dev)
        cached = torch.empty(W * H * 3, device=dev)
        for k in range(8):
            ps = rtb.make_pass(k, 11, 4, True)
            rtb.rt_render_pass(scene.handle, sc.camera, W, H, D, ps, full, opts)
            rtb.rt_render_nrc_pass(scene.handle, nrc, sc.camera, W, H, D, ps, cached, False, opts)
        torch.cuda.synchronize()
        x, r = cached.double(), full.double()
        out["gi_cache"] = {
            "value": out["gi"]["rays_per_pass"] / (ms * 1e3), "ms_per_pass": ms,
            "vs_gi_plain": out["gi"]["ms_per_pass"] / ms,
            "relmse_vs_full_depth_8_passes": float(((x - r) ** 2 / (r ** 2 + 0.01)).mean()),
            "rays_traced_per_pass": nst["primary"] + nst["shadow"] + nst["secondary"],
            "cache_depth": 2, "warmup_passes": 64,
            "metric": "Mrays-equivalent/s (rays of the full-depth GI pass per cached GI pass, with training)",
        }
        rtb.rt_nrc_destroy(nrc)
    scene.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--per-depth", action="store_true", help="queue every depth (no depth-first secondary paths)")
    ap.add_argument("--no-nrc", action="store_true", help="skip the radiance-cache leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-scene batch leg")
    ap.add_argument("--no-scaleup", action="store_true", help="skip the 10.9M-triangle 4K leg")
    ap.add_argument("--no-passes", action="store_true", help="skip the progressive-pass (sampled lights, GI) leg")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the step's calls launched on the stream instead of their captured CUDA graph")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_1504_03151_b300 as rtb
    from paper_1504_03151_b300 import build as rtb_build
    from paper_1504_03151_b300 import scenes as S

    rtb_build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    sc = S.scene_terrain()
    W, H, D = sc.width, sc.height, sc.max_depth
    scene = rtb.Scene(sc)
    h = scene.handle
    tri_bytes = sc.triangles.view(np.uint8).reshape(-1)
    tri_dev = torch.from_numpy(tri_bytes.copy()).to(dev)             # resident input
    tri_pin = torch.from_numpy(tri_bytes.copy()).pin_memory()        # host input for e2e
    out = torch.empty(H * W * 3, device=dev, dtype=torch.float32)
    out_pin = torch.empty(H * W * 3, dtype=torch.float32).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)   # > L2 (126 MB)
    mode = rtb.RT_FLAG_PER_DEPTH_WAVEFRONT if args.per_depth else 0
    opts = rtb.make_options(background=sc.background, flags=mode)
    opts_t = rtb.make_options(background=sc.background, flags=rtb.RT_FLAG_STAGE_TIMING | mode)

    def step(o=None):
        rtb.rt_scene_update(h, None, tri_dev)
        rtb.rt_bvh_build(h)
        rtb.rt_render_ex(h, sc.camera, W, H, D, out, o or opts)

    # rays per frame and algorithmic work (outside the timed region)
    step()
    st = rtb.rt_render_ex(h, sc.camera, W, H, D, out, opts, stats=True)
    rays = st["primary"] + st["shadow"] + st["secondary"]
    work = rtb.rt_render_ex(h, sc.camera, W, H, D, out,
                            rtb.make_options(background=sc.background, flags=rtb.RT_FLAG_COUNT_WORK | mode),
                            stats=True)
    info = rtb.rt_bvh_get_info(h)
    assert rtb.rt_scene_sync(h) == rtb.RT_OK

    for _ in range(max(args.warmup, 3)):
        step(opts_t)                            # the timed step's options: its timing events exist from here on
        rtb.rt_render_stage_times(h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # per-kernel stage times, on steps of their own: reading a step's stage
    # events waits for it, which would leave the device idle while the host
    # enqueues the next step
    trace_ms, shadow_ms = [], []
    for k in range(args.steps):
        flush.zero_()
        step(opts_t)
        _, a, b = rtb.rt_render_stage_times(h)
        trace_ms.append(a)
        shadow_ms.append(b)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the timed steps: enqueued back to back, so that the host stays ahead of
    # the device; each is bracketed by its own event pair on the stream, and
    # the L2 flush between steps lies outside the pairs.  The step's calls
    # are stream-ordered and allocate nothing once the scene has rendered,
    # so they can be captured once into a CUDA graph, as an application
    # rendering frame after frame would: the timed steps replay that graph
    # (the same repack, build and render, every kernel and copy), and the
    # same calls launched one by one on the stream are timed beside them.
    def timed(run):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between steps (not timed)
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            graph.replay()
        torch.cuda.synchronize()
    stream_ms = max_over_ranks(sum(timed(step)) / args.steps, dist, dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms = timed(graph.replay if graph is not None else step)
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dist, dev)
    value = job_throughput(world, rays, ms)        # Mrays/s over all ranks
    # the cached steps below launch on the stream (the cache's Adam step
    # counts frames on the host), so they compare with the plain step launched alike
    stream_value = job_throughput(world, rays, stream_ms)
    assert rtb.rt_scene_sync(h) == rtb.RT_OK

    # end to end through the public API: every step copies the geometry from
    # pinned host memory, builds, renders and copies the image into pinned
    # host memory.  Latency: one frame at a time (rt_scene_update from the
    # host buffer; rt_render_host waits for its copy).  Throughput, the e2e
    # value: frames queued back to back; a step's geometry goes up on an
    # upload stream into one of two device buffers while the previous frame
    # renders (rt_scene_update then copies it on the device), and its image
    # comes back on the scene's copy stream while the next frame renders
    # (rt_render_host_async); L2 flushed between steps; wall clock from the
    # first upload to the last image's arrival (rt_scene_sync)
    e2e_lat, e2e_ms = [], None
    n_e2e = 0 if args.no_e2e else max(3, args.steps)
    for k in range(min(n_e2e, 5)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rtb.rt_scene_update(h, None, tri_pin)
        rtb.rt_bvh_build(h)
        rtb.rt_render_host(h, sc.camera, W, H, D, out_pin, opts)
        e2e_lat.append((time.perf_counter() - t0) * 1e3)
    e2e_lat = sorted(e2e_lat)[len(e2e_lat) // 2] if e2e_lat else None
    if n_e2e:
        out_pins = [out_pin, torch.empty(H * W * 3, dtype=torch.float32).pin_memory()]
        for k in range(2):                      # the second image and the copy stream come into being
            rtb.rt_render_host_async(h, sc.camera, W, H, D, out_pins[k], opts)
        assert rtb.rt_scene_sync(h) == rtb.RT_OK
        if dist:
            dist.barrier()
        up = torch.cuda.Stream(dev)
        stage = [torch.empty_like(tri_dev) for _ in range(2)]
        ev_up = [torch.cuda.Event() for _ in range(2)]        # the upload into stage[j] is done
        ev_used = [torch.cuda.Event() for _ in range(2)]      # rt_scene_update has read stage[j]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            j = k % 2
            up.wait_event(ev_used[j])           # (a no-op until stage[j] has been read once)
            with torch.cuda.stream(up):
                stage[j].copy_(tri_pin, non_blocking=True)
            ev_up[j].record(up)
            flush.zero_()
            stream.wait_event(ev_up[j])
            rtb.rt_scene_update(h, None, stage[j])
            ev_used[j].record(stream)
            rtb.rt_bvh_build(h)
            rtb.rt_render_host_async(h, sc.camera, W, H, D, out_pins[j], opts)
        assert rtb.rt_scene_sync(h) == rtb.RT_OK
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e, dist, dev)
    e2e_stream_ms = e2e_ms
    # The same frames from two captured CUDA graphs, as the timed steps run:
    # graph j repacks the geometry from stage[j], builds, then renders into
    # image[j] while a side branch copies the previous frame's image to the
    # host and uploads the next frame's geometry into stage[1 - j] (forked
    # after the build: copies beside the build slow its latency-bound
    # kernels).  Every step thus moves one frame's upload and one image; the
    # first upload and the last image copy are timed too.  CUDA events on the
    # stream bracket each replay, with the L2 flush between steps outside the
    # pairs, as for the device-resident value; the wall clock over the loop,
    # flushes included, is reported beside it.
    e2e_wall_ms = None
    if n_e2e and graph is not None:
        side = torch.cuda.Stream(dev)
        imgs = [out, torch.empty_like(out)]
        stage = [tri_dev.clone() for _ in range(2)]    # valid geometry from the first read on

        def frame(j):
            rtb.rt_scene_update(h, None, stage[j])
            rtb.rt_bvh_build(h)
            cur = torch.cuda.current_stream()
            side.wait_stream(cur)
            copy_async(out_pins[1 - j], imgs[1 - j], side)
            copy_async(stage[1 - j], tri_pin, side)
            rtb.rt_render_ex(h, sc.camera, W, H, D, imgs[j], opts)
            cur.wait_stream(side)

        for j in (0, 1, 0, 1):                  # buffers and the side stream come into being
            frame(j)
        torch.cuda.synchronize()
        graphs = [torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()]
        for j in range(2):
            with torch.cuda.graph(graphs[j]):
                frame(j)
        torch.cuda.synchronize()
        for k in range(max(args.warmup, 3)):
            flush.zero_()
            graphs[k % 2].replay()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_e2e + 2)]
        t0 = time.perf_counter()
        evs[0][0].record(stream)
        copy_async(stage[0], tri_pin, stream)                 # the first frame's geometry
        evs[0][1].record(stream)
        for k in range(n_e2e):
            flush.zero_()                       # L2 flush between steps (outside the pairs)
            evs[k + 1][0].record(stream)
            graphs[k % 2].replay()
            evs[k + 1][1].record(stream)
        last = (n_e2e - 1) % 2
        evs[-1][0].record(stream)
        copy_async(out_pins[last], imgs[last], stream)        # the last frame's image
        evs[-1][1].record(stream)
        torch.cuda.synchronize()
        e2e_wall_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e, dist, dev)
        e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / n_e2e, dist, dev)
        # the host copies hold the frames rendered (outside the timed region)
        assert torch.equal(out_pins[last], imgs[last].cpu()) and torch.equal(stage[0].cpu(), tri_pin)
    e2e_value = job_throughput(world, rays, e2e_ms) if e2e_ms else None

    # roofline of the two kernel classes (closest hit + shade; any-hit
    # shadow): FP32-issue fraction of the algorithmic operations and L2
    # fraction of the algorithmic bytes, over the classes' stage times in the
    # timed frames (where they overlap each other); beside them the stage
    # times with every kernel run alone (RT_FLAG_SERIAL_STAGES, untimed steps)
    ser_trace, ser_shadow = [], []
    opts_s = rtb.make_options(background=sc.background, flags=rtb.RT_FLAG_STAGE_TIMING | rtb.RT_FLAG_SERIAL_STAGES | mode)
    for k in range(max(args.steps // 2, 3)):
        flush.zero_()
        step(opts_s)
        _, a, b = rtb.rt_render_stage_times(h)
        ser_trace.append(a)
        ser_shadow.append(b)
    l2_probe = {mb: rtb.rt_probe_l2_read(mb << 20, max(1, (40 << 30) // (mb << 20))) for mb in (16, 32, 64)}
    l2_peak = max(l2_probe.values())
    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2032.0)
    alu_peak = 148 * 128 * sm_mhz * 1e6 / 1e12       # FP32 lanes x clock: Tops/s (one op per lane per clock)
    tr = sum(trace_ms) / len(trace_ms)
    sh = sum(shadow_ms) / len(shadow_ms)
    classes = {}
    for c_, name, kms_, sms_, nrays in ((0, "closest_hit", tr, sum(ser_trace) / len(ser_trace),
                                         st["primary"] + st["secondary"]),
                                        (1, "shadow", sh, sum(ser_shadow) / len(ser_shadow), st["shadow"])):
        ops_ = work["box_tests"][c_] * OPS_BOX + work["prim_tests"][c_] * OPS_TRI
        byt_ = work["node_visits"][c_] * BYTES_NODE + work["prim_tests"][c_] * BYTES_TRI + nrays * BYTES_RAY_IO
        tb, tsrc = profiled_traffic(c_)
        classes[name] = {
            "kernel_ms": kms_, "kernel_ms_alone": sms_, "rays": nrays, "alg_ops": ops_, "alg_bytes": byt_,
            "alu_frac": ops_ / (kms_ * 1e-3) / 1e12 / alu_peak,
            "l2_frac": byt_ / (kms_ * 1e-3) / 1e9 / l2_peak,
            "alu_frac_alone": ops_ / (sms_ * 1e-3) / 1e12 / alu_peak,
            "l2_frac_alone": byt_ / (sms_ * 1e-3) / 1e9 / l2_peak,
            "dram_bytes": tb, "dram_source": tsrc,
            "dram_over_alg_bytes": tb / byt_ if tb else None,
        }
        classes[name]["frac"] = max(classes[name]["alu_frac"], classes[name]["l2_frac"])
    cls = 0 if tr >= sh else 1
    cname = "closest_hit" if cls == 0 else "shadow"
    C = classes[cname]
    cls_ms, ops, traffic, traffic_src = C["kernel_ms"], C["alg_ops"], C["dram_bytes"], C["dram_source"]
    achieved = ops / (cls_ms * 1e-3) / 1e12
    l2_bound = C["l2_frac"] > C["alu_frac"]
    # a step: the geometry copy and k_pack (rt_scene_update), the build's
    # kernels and memsets, the frame's counter clear and its kernels
    launches_per_step = 2 + info["build_launches"] + 1 + st["launches"]

    # radiance cache: online training frames, then timed training frames;
    # its Mrays-equivalent = rays the full-depth frame traces / cached step time
    nrc_line = None
    if not args.no_nrc:
        full = torch.empty_like(out)
        rtb.rt_render_ex(h, sc.camera, W, H, D, full, opts)
        nrc = rtb.rt_nrc_create(h, rtb.rt_nrc_config_default(seed=1))
        nrc_out = torch.empty_like(out)

        def nrc_step(stats=False):
            rtb.rt_scene_update(h, None, tri_dev)
            rtb.rt_bvh_build(h)
            return rtb.rt_render_nrc(h, nrc, sc.camera, W, H, D, nrc_out, train=True, options=opts, stats=stats)

        for _ in range(64):
            nrc_step()
        nst = nrc_step(stats=True)
        torch.cuda.synchronize()
        nev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            nev[k][0].record(stream)
            nrc_step()
            nev[k][1].record(stream)
        torch.cuda.synchronize()
        nrc_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in nev) / args.steps, dist, dev)
        # the network's kernels alone, against the tensor-core peak: one training
        # step on 65,536 samples and inference on 2^20 queries (random hits in
        # the scene box; algorithmic FLOPs of the unpadded 96-64-64-64-64-3 MLP)
        gen = torch.Generator(device=dev).manual_seed(5)
        lo_b = torch.tensor(sc.triangles["v0"].min(0), device=dev, dtype=torch.float32)
        hi_b = torch.tensor(sc.triangles["v0"].max(0), device=dev, dtype=torch.float32)

        def random_hits(m):
            p = lo_b + (hi_b - lo_b) * torch.rand(m, 3, device=dev, generator=gen)
            nv = torch.nn.functional.normalize(torch.randn(m, 6, device=dev, generator=gen).view(m, 2, 3), dim=2)
            return torch.cat([p, nv.view(m, 6)], 1).contiguous()

        n_tr, n_inf = 65536, 1 << 20
        pnv_tr, tgt = random_hits(n_tr), torch.rand(n_tr, 3, device=dev, generator=gen) + 0.05
        pnv_inf, inf_out = random_hits(n_inf), torch.empty(n_inf, 3, device=dev)
        kflops = {"train": n_tr * 99456, "infer": n_inf * 37248}   # 2*(fwd 18,624 + dX 12,480 + dW 18,624); 2*18,624
        kms = {}
        for name, fn in (("train", lambda: rtb.rt_nrc_train_step(nrc, h, pnv_tr, tgt, n_tr)),
                         ("infer", lambda: rtb.rt_nrc_infer(nrc, h, pnv_inf, n_inf, inf_out))):
            for _ in range(3):
                fn()
            kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
            for a_, b_ in kev:
                a_.record(stream)
                fn()
                b_.record(stream)
            torch.cuda.synchronize()
            kms[name] = sum(a_.elapsed_time(b_) for a_, b_ in kev) / len(kev)
        pk_n, pk_kind_n = peaks()
        nrc_roof = {name: {"bound": "tensor", "achieved": kflops[name] / (kms[name] * 1e-3) / 1e12,
                           "peak": pk_n["bf16_tflops"], "unit": "TFLOP/s",
                           "frac": kflops[name] / (kms[name] * 1e-3) / 1e12 / pk_n["bf16_tflops"],
                           "ms": kms[name], "flops": kflops[name], "peak_source": f"bf16 burst ({pk_kind_n})"}
                    for name in kms}
        x, r = nrc_out.double(), full.double()
        relmse = float(((x - r) ** 2 / (r ** 2 + 0.01)).mean())
        mse01 = float(((x.clamp(0, 1) - r.clamp(0, 1)) ** 2).mean())
        nrc_value = job_throughput(world, rays, nrc_ms)
        nrc_line = {
            "metric": "Mrays-equivalent/s (full-depth rays per cached step)", "value": nrc_value,
            "ms_per_step": nrc_ms, "vs_plain": nrc_value / stream_value, "relmse_vs_full_depth": relmse,
            "psnr_db": 10 * np.log10(1.0 / max(mse01, 1e-30)), "warmup_frames": 64,
            "train_batch": 65536, "cache_depth": 2,
            "rays_traced_per_step": nst["primary"] + nst["shadow"] + nst["secondary"],
            "cache_hits": nst["hits_per_depth"][2],
            "step": "repack + BVH build + cached frame (inference) + training rays + one Adam step",
            "launch": "on the stream; vs_plain compares with the plain step launched on the stream",
            "kernel_roofline": nrc_roof,
        }
        rtb.rt_nrc_destroy(nrc)

    batch_line = None
    if world == 1 and not args.no_batch:
        batch_line = batch_leg(rtb, S, torch, dev, stream, flush, max(args.steps // 2, 3))
    passes_line = None
    if world == 1 and not args.no_passes:
        passes_line = passes_leg(rtb, S, torch, dev, stream, flush, max(args.steps // 2, 3), not args.no_nrc)
    scaleup_line = None
    if world == 1 and not args.no_scaleup:
        scaleup_line = scaleup_leg(rtb, S, torch, dev, stream, flush, 3, not args.no_nrc)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(sc)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "terrain 1920x1080, 123904 triangles (fBm 256x192 + 20 L3 icospheres), "
                                   "depth 5, 4 point lights, materials 60/25/15",
                       "rays_per_step": rays, "primary": st["primary"], "shadow": st["shadow"],
                       "secondary": st["secondary"], "l2": "flushed between steps (256 MB write)",
                       "step": "repack + BVH build + render", "parallelism": f"replicas x{world}",
                       "launch": ("the step's calls captured once in a CUDA graph, replayed every step"
                                  if graph is not None else "the step's calls launched on the stream"),
                       "stream_launched": {"ms_per_step": stream_ms, "value": stream_value},
                       "bvh": {k: info[k] for k in ("n_nodes", "max_depth", "sah_cost", "sah_cost_lbvh")}},
            "roofline": {"bound": "l2" if l2_bound else "alu",
                         "kernel": "closest-hit+shade" if cls == 0 else "any-hit shadow",
                         "achieved": C["alg_bytes"] / (cls_ms * 1e-3) / 1e9 if l2_bound else achieved,
                         "peak": l2_peak if l2_bound else alu_peak, "unit": "GB/s" if l2_bound else "Tops/s",
                         "frac": C["frac"], "traffic": traffic, "traffic_unit": "bytes per frame",
                         "traffic_source": traffic_src,
                         "alu": {"achieved": achieved, "peak": alu_peak, "unit": "Tops/s", "frac": C["alu_frac"],
                                 "peak_source": f"148 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({pk_kind} clock)"},
                         "l2": {"achieved": C["alg_bytes"] / (cls_ms * 1e-3) / 1e9, "peak": l2_peak, "unit": "GB/s",
                                "frac": C["l2_frac"],
                                "peak_source": "rt_probe_l2_read: streaming L1-bypassing reads of an L2-resident "
                                               "buffer, best of " + ", ".join(f"{m} MB {g:.0f}"
                                                                              for m, g in l2_probe.items())},
                         "kernel_ms": cls_ms, "kernel_ms_alone": C["kernel_ms_alone"], "alg_ops": ops,
                         "alg_bytes": C["alg_bytes"], "dram_over_alg_bytes": C["dram_over_alg_bytes"],
                         "alg_units": "ops: 14 a child-box test, 30 a triangle test; bytes: 128 a node visit, "
                                      "48 a primitive test, 64 a ray (48-B record in, 16-B hit out)",
                         "classes": classes},
            "stage_ms": {"trace": tr, "shadow": sh, "step": ms,
                         "note": "sums of per-kernel times; shadow kernels overlap the next depth's trace"},
            "work": {"node_visits_per_depth": work["node_visits_per_depth"],
                     "max_visits_per_ray_per_depth": work["max_visits_per_depth"],
                     "rays_per_depth": st["rays_per_depth"], "shadow_per_depth": st["shadow_per_depth"]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(tri_bytes.nbytes),
                    "d2h_bytes_per_step": int(H * W * 3 * 4), "ms_per_step": e2e_ms,
                    "steps": n_e2e,
                    "mode": ("two captured CUDA graphs replayed in turn: each repacks and builds from the "
                             "uploaded geometry, then renders while a side branch copies the previous image "
                             "to pinned host memory and uploads the next geometry from it; CUDA events "
                             "around each replay, the first upload and the last image copy; L2 flushed "
                             "between steps, outside the events" if e2e_wall_ms is not None else
                             "frames queued back to back: uploads (pinned host -> device, own stream) and "
                             "image copies (rt_render_host_async) overlap the neighbouring frames; L2 "
                             "flushed between steps; wall clock to the last image on the host"),
                    "wall_ms_per_step_with_l2_flush": e2e_wall_ms,
                    "stream_launched": ({"ms_per_step": e2e_stream_ms,
                                         "value": job_throughput(world, rays, e2e_stream_ms),
                                         "mode": "rt_render_host_async frames queued back to back (uploads on "
                                                 "their own stream); wall clock to the last image on the "
                                                 "host, L2 flushes included"}
                                        if e2e_stream_ms else None),
                    "latency_ms_one_frame": e2e_lat},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if nrc_line:
            line["radiance_cache"] = nrc_line
        if batch_line:
            line["batch"] = batch_line
        if passes_line:
            line["passes"] = passes_line
        if scaleup_line:
            line["scaleup"] = scaleup_line
        print(json.dumps(line), flush=True)
    scene.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
