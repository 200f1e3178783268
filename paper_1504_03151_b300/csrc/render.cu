// render.cu - the wavefront Whitted pipeline: closest-hit + shade kernels
// (the depth-0 one generates its primary rays itself), any-hit shadow
// kernels, warp-aggregated queue pushes, and the ABI entry points.
//
// One frame, per Sec. IV.A of the paper (recursion turned into an
// iteration whose trip count is the depth):
//   depth 0 : camera rays -> closest hit -> shade: shadow rays (Alg. 1, one
//             per point light) to the shadow queue, reflection/refraction
//             rays to the next ray queue, misses / emission to the image
//   shadow  : any hit on (0, dist - eps); unblocked -> add to the image
//   depth d : the same on the queued rays, until max_depth
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "nrc_internal.cuh"
#include "rtb_internal.cuh"
#include "trace_device.cuh"

namespace rtb {

// Device-side counters of one frame (reset at its start).
struct Counters {
  unsigned rays[RT_MAX_DEPTH + 2];        // rays queued for depth d (d >= 1)
  unsigned shadow[RT_MAX_DEPTH + 1];      // shadow rays cast from depth-d hits
  unsigned hits[RT_MAX_DEPTH + 1];
  unsigned fetch_trace[RT_MAX_DEPTH + 1]; // dynamic work fetch
  unsigned fetch_shadow[RT_MAX_DEPTH + 1];
  unsigned max_visits[2][RT_MAX_DEPTH + 1];          // [closest, any][depth], counting runs only
  unsigned infer_count, train_count;                 // radiance-cache records of the frame
  unsigned cache_hits;                               // hits at the cache depth (depth-first frames)
  unsigned long long visits[2][RT_MAX_DEPTH + 1];
  unsigned long long tests[2][RT_MAX_DEPTH + 1];
  unsigned long long boxes[2][RT_MAX_DEPTH + 1];
};

struct FrameParams {
  CamBasis cam;
  int W, H, tiles_x, tiles_y;
  int max_depth;
  float bg_r, bg_g, bg_b;
  float eps_scale;
  float* fb;
  int32_t* aov_prim;
  float* aov_t;
  float4* rayq[2];
  float4* shadowq[2];                     // shadow queue of depth d: shadowq[d & 1]
  unsigned ray_cap, shadow_cap;
  Counters* ctr;
  int path_depth0;          // first depth of the depth-first secondary kernel
  // radiance cache (nrc_depth < 0: off)
  int nrc_depth;
  float* target;            // training targets: pixel ids < 0 route here (slot ~pixel)
  float4* infer_q;          // 4 float4 per record: (p, pixel) (n) (v) (weight)
  float4* train_q;          // 3 float4 per record: (p, slot) (n) (v)
  unsigned infer_cap, train_cap;
  unsigned train_batch;     // wanted training samples; selection probability = batch / rays
  uint32_t seed;
  const unsigned* prev_hits;   // depth-first frames: cache hits of the previous frame (0: take all)
  PassInfo ps;                 // the pass: camera jitter and area-light samples
  unsigned long long* fb_fixed;   // RT_FLAG_DETERMINISTIC: 3 per pixel, 64-bit fixed point (else NULL)
  unsigned* px_rays;              // counting frames: per pixel and depth, closest-hit and shadow rays (else NULL)
  int px_stride;                  // 2 (max_depth + 1)
  int fb_store;                   // 1: the depth-0 kernel stores each pixel's first value (the image is not cleared)
};

// Per-pixel ray counts (counting instances only): cls 0 = a closest-hit ray
// traced at `depth`, cls 1 = a shadow ray cast from a depth-`depth` hit.
// Rays of the radiance cache's training subset (pixel < 0) are not counted.
template <bool kCount>
__device__ __forceinline__ void count_px(const FrameParams& fp, int pixel, int depth, int cls) {
  if (kCount && fp.px_rays != nullptr && pixel >= 0)
    atomicAdd(&fp.px_rays[(size_t)pixel * fp.px_stride + 2 * depth + cls], 1u);
}

constexpr float kFixScale = 4294967296.f;   // 2^32 units of radiance
constexpr float kFixMax = 1073741824.f;     // |contribution| clamp, 2^30: sums stay far inside 64 bits

__device__ __forceinline__ unsigned long long to_fixed(float x) {
  x = x == x ? fminf(fmaxf(x, -kFixMax), kFixMax) : 0.f;
  return (unsigned long long)__float2ll_rn(x * kFixScale);   // two's complement: signed sums wrap right
}

// Adds radiance to a pixel, or to a training target when the ray belongs to
// the radiance cache's training subset (pixel id < 0 -> slot ~pixel).  In a
// deterministic frame the pixel sums are integers, whose order cannot change
// them.
__device__ __forceinline__ void add_fb(const FrameParams& fp, int pixel, f3 c) {
  if (fp.fb_fixed != nullptr && pixel >= 0) {
    unsigned long long* q = fp.fb_fixed + 3 * (size_t)pixel;
    atomicAdd(q, to_fixed(c.x));
    atomicAdd(q + 1, to_fixed(c.y));
    atomicAdd(q + 2, to_fixed(c.z));
    return;
  }
  float* p = pixel >= 0 ? fp.fb + 3 * (size_t)pixel : fp.target + 3 * (size_t)(~pixel);
  atomicAdd(p, c.x);
  atomicAdd(p + 1, c.y);
  atomicAdd(p + 2, c.z);
}

// The first value of a pixel, stored by the depth-0 kernel (every pixel has
// exactly one camera ray, traced before any other kernel of the frame adds).
__device__ __forceinline__ void store_fb(const FrameParams& fp, int pixel, f3 c) {
  float* p = fp.fb + 3 * (size_t)pixel;
  p[0] = c.x;
  p[1] = c.y;
  p[2] = c.z;
}

// The deterministic frame's image: fixed-point sums -> float32.
__global__ void k_fixed_to_float(float* __restrict__ out, const unsigned long long* __restrict__ fixed, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)((double)(long long)fixed[i] * (1.0 / 4294967296.0));
}


template <bool kCount>
__device__ __forceinline__ void flush_work(Counters* ctr, int cls, int depth, WorkCount wc) {
  if (!kCount) return;
  unsigned v = wc.visits, t = wc.tests, m = wc.vmax, b = wc.boxes;
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(kFull, v, o);
    t += __shfl_xor_sync(kFull, t, o);
    b += __shfl_xor_sync(kFull, b, o);
    m = max(m, __shfl_xor_sync(kFull, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&ctr->visits[cls][depth], (unsigned long long)v);
    atomicAdd(&ctr->tests[cls][depth], (unsigned long long)t);
    atomicAdd(&ctr->boxes[cls][depth], (unsigned long long)b);
    atomicMax(&ctr->max_visits[cls][depth], m);
  }
}

// ---------------------------------------------------------------------------
// closest hit + shade (+ primary ray generation at depth 0)
// ---------------------------------------------------------------------------
// Five blocks an SM: with six the closest-hit kernel fits 80 registers and
// spills; the five-block cap (102) holds it without spills, and the wider
// issue of the unspilled code outweighs the sixth block's warps.
#ifndef RTB_TRACE_MIN_BLOCKS
#define RTB_TRACE_MIN_BLOCKS 5
#endif
#ifndef RTB_PATHS_MIN_BLOCKS
#define RTB_PATHS_MIN_BLOCKS 5
#endif

// kPass: the frame has area lights, emissive primitives or jittered camera
// rays (the sampling code is compiled only into these instances, which
// keeps it out of the plain kernels' instruction stream).
template <bool kPrimary, bool kCount, bool kPass>
__global__ void __launch_bounds__(kTraceThreads, RTB_TRACE_MIN_BLOCKS) k_trace(DevScene sc, FrameParams fp, int depth, int cap) {
  __shared__ int s_stack[kStackShared * kTraceThreads];
  int* stack = s_stack + threadIdx.x;
  int lane = threadIdx.x & 31;
  Counters* ctr = fp.ctr;
  unsigned n_items = kPrimary ? (unsigned)(fp.tiles_x * fp.tiles_y * 32) : min(ctr->rays[depth], fp.ray_cap);
  const float4* __restrict__ qin = fp.rayq[depth & 1];
  float4* qout = fp.rayq[(depth + 1) & 1];
  bool spawn = depth < fp.max_depth;
  WorkCount wc = {0u, 0u, 0u, 0u};
  for (;;) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&ctr->fetch_trace[depth], 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= n_items) break;
    unsigned idx = base + lane;
    bool active = idx < n_items;
    f3 o, d, w;
    int pixel = 0;
    uint32_t code = 1u;   // path vertex of the ray's hit
    if (kPrimary) {
      int tile = (int)(idx >> 5);
      int x = (tile % fp.tiles_x) * 8 + (lane & 7);
      int y = (tile / fp.tiles_x) * 4 + (lane >> 3);
      active = active && x < fp.W && y < fp.H;
      x = min(x, fp.W - 1);
      y = min(y, fp.H - 1);
      pixel = y * fp.W + x;
      if (kPass) {
        float px, py;
        pass_pixel_point(fp.ps, pixel, x, y, px, py);
        camera_ray_at(fp.cam, fp.W, fp.H, px, py, o, d);
      } else {
        camera_ray(fp.cam, fp.W, fp.H, x, y, o, d);
      }
      w = mk3(1.f, 1.f, 1.f);
    } else {
      float4 q0 = make_float4(0, 0, 0, 0), q1 = make_float4(0, 0, 1, 0), q2 = make_float4(0, 0, 0, 0);
      if (active) {
        q0 = qin[3 * (size_t)idx];
        q1 = qin[3 * (size_t)idx + 1];
        q2 = qin[3 * (size_t)idx + 2];
      }
      o = xyz(q0);
      pixel = __float_as_int(q0.w);
      d = xyz(q1);
      w = xyz(q2);
      code = __float_as_uint(q2.w);
    }
    if (active) count_px<kCount>(fp, pixel, depth, 0);
    // closest hit
    float t = INFINITY;
    bool fail = false;
    unsigned v0 = wc.visits;
    // camera rays of a tile are coherent: the warp walks together; deeper
    // rays are not, and each lane walks alone (measured: a GI pass 2.10
    // against 2.15 ms, the plain step 1.375 against 1.383 ms)
    int hit = -1;
    if (kPrimary) hit = traverse_warp<false, kCount>(sc, make_ray(o, d), active, 0.0f, t, stack, cap, fail, wc);
    else if (active) hit = traverse<false, kCount>(sc, make_ray(o, d), 0.0f, t, stack, cap, fail, wc);
    if (kCount) wc.vmax = max(wc.vmax, wc.visits - v0);
    if (fail) atomicOr(sc.status, kErrTraversalLimit);
    if (kPrimary && active) {
      if (fp.aov_prim) fp.aov_prim[pixel] = hit >= 0 ? __float_as_int(__ldg(&sc.prims[3 * (size_t)hit + 1]).w) : -1;
      if (fp.aov_t) fp.aov_t[pixel] = hit >= 0 ? t : INFINITY;
    }
    // shading
    bool is_hit = active && hit >= 0;
    const bool first_store = kPrimary && fp.fb_store;
    if (active && hit < 0 && !first_store) add_fb(fp, pixel, w * mk3(fp.bg_r, fp.bg_g, fp.bg_b));
    unsigned hm = __ballot_sync(kFull, is_hit);
    if (lane == 0 && hm) atomicAdd(&ctr->hits[depth], (unsigned)__popc(hm));
    Surface sf;
    sf.kind = RT_MAT_DIELECTRIC;   // no local term, no children unless a hit sets it
    if (is_hit) sf = surface_at(sc, hit, o, d, t, fp.eps_scale);
    // L_e, Eq. 7 (not on a diffuse bounce: its parent sampled the emitters)
    const bool via_bounce = kPass && (code & kCodeBounce) != 0u;
    const uint32_t vcode = kPass ? (code & ~kCodeBounce) : code;
    const bool emits =
        is_hit && !via_bounce && (sf.emission.x != 0.f || sf.emission.y != 0.f || sf.emission.z != 0.f);
    if (first_store) {
      if (active)
        store_fb(fp, pixel, !is_hit ? w * mk3(fp.bg_r, fp.bg_g, fp.bg_b) : (emits ? w * sf.emission : mk3(0.f, 0.f, 0.f)));
    } else if (emits) {
      add_fb(fp, pixel, w * sf.emission);
    }
    if (depth == fp.nrc_depth) {
      // radiance cache: every hit here takes the radiance it reflects from
      // the cache (its own L_e is added above, as at any hit); a seeded
      // subset is also traced on, with unit weight, into a training target
      bool ok;
      unsigned pos = warp_push(&ctr->infer_count, is_hit, fp.infer_cap, ok, sc.status);
      if (ok) {
        float4* q = fp.infer_q + 4 * (size_t)pos;
        q[0] = make_float4(sf.p.x, sf.p.y, sf.p.z, __int_as_float(pixel));
        q[1] = make_float4(sf.n.x, sf.n.y, sf.n.z, 0.f);
        q[2] = make_float4(-d.x, -d.y, -d.z, 0.f);
        q[3] = make_float4(w.x, w.y, w.z, 0.f);
      }
      float u = (float)(hash32(fp.seed ^ hash32((uint32_t)pixel * 0x9E3779B9u ^ __float_as_uint(d.x))) >> 8) *
                (1.0f / 16777216.0f);
      bool sel = is_hit && (float)fp.train_batch > u * (float)n_items;
      unsigned slot = warp_push(&ctr->train_count, sel, fp.train_cap, ok, nullptr);   // a full batch is no error
      sel = sel && slot < fp.train_cap;
      if (sel) {
        float4* q = fp.train_q + 3 * (size_t)slot;
        q[0] = make_float4(sf.p.x, sf.p.y, sf.p.z, __int_as_float((int)slot));
        q[1] = make_float4(sf.n.x, sf.n.y, sf.n.z, 0.f);
        q[2] = make_float4(-d.x, -d.y, -d.z, 0.f);
        w = mk3(1.f, 1.f, 1.f);
        pixel = ~(int)slot;
      }
      is_hit = sel;
    }
    // Alg. 1: one shadow ray per point light where n.l > 0
    bool local = is_hit && sf.kind != RT_MAT_DIELECTRIC && (1.f - sf.rho) > 0.f;
    if (sc.n_lights <= 32) {
      // the warp's rays of every light in one reservation: which lights each
      // lane's hit faces, one atomic for their total, then the records light
      // by light (the same order as one push a light)
      uint32_t faces = 0u;
      unsigned total = 0u;
      for (int li = 0; li < sc.n_lights; ++li) {
        const bool f = local && light_faces(sf, __ldg(&sc.lights[2 * li]));
        faces |= (f ? 1u : 0u) << li;
        total += (unsigned)__popc(__ballot_sync(kFull, f));
      }
      unsigned base = 0u;
      if (total) {
        if ((threadIdx.x & 31) == 0) base = atomicAdd(&ctr->shadow[depth], total);
        base = __shfl_sync(kFull, base, 0);
      }
      const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
      for (int li = 0; li < sc.n_lights && total; ++li) {
        const bool f = (faces >> li) & 1u;
        const unsigned mask = __ballot_sync(kFull, f);
        if (f) {
          f3 contrib = mk3(0, 0, 0), os = mk3(0, 0, 0), sd = mk3(0, 0, 1);
          float tmax = 0.f;
          light_term(sf, d, w, __ldg(&sc.lights[2 * li]), __ldg(&sc.lights[2 * li + 1]), contrib, os, sd, tmax);
          const unsigned pos = base + (unsigned)__popc(mask & lt);
          if (pos < fp.shadow_cap) store_ray(fp.shadowq[depth & 1], pos, os, pixel, sd, tmax, contrib);
          else atomicOr(sc.status, kErrQueueOverflow);
        }
        base += (unsigned)__popc(mask);
      }
    } else {
      for (int li = 0; li < sc.n_lights; ++li) {
        f3 contrib = mk3(0, 0, 0), os = mk3(0, 0, 0), sd = mk3(0, 0, 1);
        float tmax = 0.f;
        bool valid = local && light_term(sf, d, w, __ldg(&sc.lights[2 * li]), __ldg(&sc.lights[2 * li + 1]), contrib,
                                         os, sd, tmax);
        bool ok;
        unsigned pos = warp_push(&ctr->shadow[depth], valid, fp.shadow_cap, ok, sc.status);
        if (ok) store_ray(fp.shadowq[depth & 1], pos, os, pixel, sd, tmax, contrib);
      }
    }
    // area lights, then emissive primitives: one sampled point of each per pass
    for (int li = 0; kPass && li < sc.n_alights + sc.n_emitters; ++li) {
      f3 contrib = mk3(0, 0, 0), os = mk3(0, 0, 0), sd = mk3(0, 0, 1);
      float tmax = 0.f;
      bool valid = false;
      if (local) {
        float a, b;
        pass_sample(fp.ps, pixel, vcode, (uint32_t)li, a, b);
        valid = area_term(sf, d, w, area_point(sc, li, a, b), contrib, os, sd, tmax);
      }
      bool ok;
      unsigned pos = warp_push(&ctr->shadow[depth], valid, fp.shadow_cap, ok, sc.status);
      if (ok) store_ray(fp.shadowq[depth & 1], pos, os, pixel, sd, tmax, contrib);
    }
    // reflection / refraction rays (Fig. 3) or a diffuse bounce, not past the last depth
    Children ch;
    ch.want_r = ch.want_t = ch.bounce = false;
    if (is_hit && spawn) {
      ch = children_of(sf, d, w);
      if (kPass && fp.ps.bounce) add_bounce(ch, sf, w, fp.ps, pixel, vcode);
    }
    {
      bool ok;
      unsigned pos = warp_push(&ctr->rays[depth + 1], ch.want_r, fp.ray_cap, ok, sc.status);
      if (ok) store_ray(qout, pos, ch.or_, pixel, ch.dr, INFINITY, ch.wr, vcode << 1);
      pos = warp_push(&ctr->rays[depth + 1], ch.want_t, fp.ray_cap, ok, sc.status);
      const uint32_t code_t = (vcode << 1) | 1u | (ch.bounce ? kCodeBounce : 0u);
      if (ok) store_ray(qout, pos, ch.ot, pixel, ch.dt, INFINITY, ch.wt, code_t);
    }
  }
  flush_work<kCount>(ctr, 0, depth, wc);
}

// ---------------------------------------------------------------------------
// shadow rays: any hit on (0, tmax); unblocked -> add the light's term
// ---------------------------------------------------------------------------
// Eight blocks an SM: the speculative walk would take 69 registers and leave
// room for seven; at 63 it spills nothing.
template <bool kCount>
__global__ void __launch_bounds__(kTraceThreads, 8) k_shadow(DevScene sc, FrameParams fp, int depth, int cap) {
  __shared__ int s_stack[kStackShared * kTraceThreads];
  int* stack = s_stack + threadIdx.x;
  int lane = threadIdx.x & 31;
  Counters* ctr = fp.ctr;
  unsigned n_items = min(ctr->shadow[depth], fp.shadow_cap);
  WorkCount wc = {0u, 0u, 0u, 0u};
  for (;;) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&ctr->fetch_shadow[depth], 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= n_items) break;
    unsigned idx = base + lane;
    bool part = idx < n_items;
    float4 q0 = make_float4(0, 0, 0, 0), q1 = make_float4(0, 0, 1, 0), q2 = make_float4(0, 0, 0, 0);
    if (part) {
      const float4* q = fp.shadowq[depth & 1] + 3 * (size_t)idx;
      q0 = q[0];
      q1 = q[1];
      q2 = q[2];
    }
    float tmax = q1.w;
    bool fail = false;
    unsigned v0 = wc.visits;
    int h = -1;
    if (part) h = traverse<true, kCount>(sc, make_ray(xyz(q0), xyz(q1)), 0.0f, tmax, stack, cap, fail, wc);
    if (kCount) wc.vmax = max(wc.vmax, wc.visits - v0);
    if (fail) atomicOr(sc.status, kErrTraversalLimit);
    if (part && h < 0 && !fail) add_fb(fp, __float_as_int(q0.w), xyz(q2));
    if (part) count_px<kCount>(fp, __float_as_int(q0.w), depth, 1);
  }
  flush_work<kCount>(ctr, 1, depth, wc);
}

// ---------------------------------------------------------------------------
// secondary rays, depth first: one thread carries a depth-1 ray's whole
// subtree - the paper's recursion-as-iteration (Sec. IV.A) - tracing its
// shadow rays inline.  One launch replaces the per-depth trace and shadow
// launches of depths >= 1, whose few rays would otherwise make every depth
// as slow as its slowest ray.
// ---------------------------------------------------------------------------
template <bool kCount>
__device__ __forceinline__ void count_ray(Counters* ctr, int cls, int depth, unsigned v, unsigned t, unsigned b) {
  if (!kCount) return;
  atomicAdd(&ctr->visits[cls][depth], (unsigned long long)v);
  atomicAdd(&ctr->tests[cls][depth], (unsigned long long)t);
  atomicAdd(&ctr->boxes[cls][depth], (unsigned long long)b);
  atomicMax(&ctr->max_visits[cls][depth], v);
}

constexpr int kWarpPending = 64;   // pending children per warp (shared memory, 12 KB a block)
constexpr int kWavefrontDepths = 1;   // depths 0..1 run as wavefronts (the cache, if any, lies deeper)


template <bool kCount, bool kPass>
__global__ void __launch_bounds__(kTraceThreads, RTB_PATHS_MIN_BLOCKS) k_paths(DevScene sc, FrameParams fp, int cap) {
  __shared__ int s_stack[kStackShared * kTraceThreads];
  __shared__ unsigned s_cnt[3][RT_MAX_DEPTH + 2];   // rays spawned for / shadow rays cast at / hits at depth d
  __shared__ float4 s_pend[kTraceThreads / 32][kWarpPending][3];   // (o, pixel) (d, depth) (w, -)
  __shared__ int s_np[kTraceThreads / 32];
  int* stack = s_stack + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < 3 * (RT_MAX_DEPTH + 2); i += blockDim.x) (&s_cnt[0][0])[i] = 0u;
  if (lane == 0) s_np[warp] = 0;
  __syncthreads();
  Counters* ctr = fp.ctr;
  const int d0 = fp.path_depth0;
  const unsigned n_items = min(ctr->rays[d0], fp.ray_cap);
  const float4* __restrict__ qin = fp.rayq[d0 & 1];
  const f3 bg = mk3(fp.bg_r, fp.bg_g, fp.bg_b);
  // overflow of this lane when the warp's pending stack is full (depth first: <= max depth entries)
  float4 local[RT_MAX_DEPTH][3];
  int nl = 0;
  bool queue_done = false;
  bool have = false;
  WorkCount wc = {0u, 0u, 0u, 0u};
  // A lane's item is a path segment (depth >= 0) or a shadow ray cast from
  // a depth-(~depth) hit (depth < 0; w holds its contribution, tmax its
  // length), so that lanes without a path of their own trace the shadow
  // rays of the others.
  f3 o = mk3(0, 0, 0), d = mk3(0, 0, 1), w = mk3(0, 0, 0);
  int depth = d0, pixel = 0;
  float tmax_item = 0.f;
  uint32_t code = 1u;   // path vertex of a segment's hit (keys the pass's samples)
  // queue rays a warp takes at a time: spread over all warps, so that every
  // warp starts with free lanes for the children and shadow rays it makes
  const unsigned n_warps = gridDim.x * (blockDim.x >> 5);
  const unsigned chunk = max(1u, min(32u, (n_items + n_warps - 1) / n_warps));
  for (;;) {
    // --- refill lanes without a ray: own overflow, warp stack, global queue
    if (!have && nl > 0) {
      --nl;
      o = xyz(local[nl][0]);
      pixel = __float_as_int(local[nl][0].w);
      d = xyz(local[nl][1]);
      depth = __float_as_int(local[nl][1].w);
      w = xyz(local[nl][2]);
      code = __float_as_uint(local[nl][2].w);
      have = true;
    }
    __syncwarp();   // shadow rays pushed by this warp's lanes are visible
    unsigned need = __ballot_sync(kFull, !have);
    int np = s_np[warp];
    if (need && np > 0) {
      int take = min(__popc(need), np);
      int rank = __popc(need & lt);
      if (!have && rank < take) {
        const float4* r = s_pend[warp][np - 1 - rank];
        o = xyz(r[0]);
        pixel = __float_as_int(r[0].w);
        d = xyz(r[1]);
        depth = __float_as_int(r[1].w);
        w = xyz(r[2]);
        tmax_item = r[2].w;              // a shadow ray's length,
        code = __float_as_uint(r[2].w);  // or a segment's path vertex
        have = true;
      }
      __syncwarp();
      if (lane == 0) s_np[warp] = np - take;
      __syncwarp();
      need = __ballot_sync(kFull, !have);
    }
    if (need && !queue_done) {
      unsigned want = min((unsigned)__popc(need), chunk);
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(&ctr->fetch_trace[d0], want);
      base = __shfl_sync(kFull, base, 0);
      unsigned rank = (unsigned)__popc(need & lt);
      unsigned idx = base + rank;
      if (base + want >= n_items) queue_done = true;
      if (!have && rank < want && idx < n_items) {
        float4 q0 = qin[3 * (size_t)idx], q1 = qin[3 * (size_t)idx + 1], q2 = qin[3 * (size_t)idx + 2];
        o = xyz(q0);
        pixel = __float_as_int(q0.w);
        d = xyz(q1);
        w = xyz(q2);
        code = __float_as_uint(q2.w);
        depth = d0;
        have = true;
      }
    }
    if (!__any_sync(kFull, have)) break;   // nothing left for this warp
    // --- one segment per lane: closest hit, shading, shadow rays, children
    Children ch;
    ch.want_r = ch.want_t = ch.bounce = false;
    if (have && depth < 0) {
      bool sfail = false;
      float tm = tmax_item;
      unsigned sv0 = wc.visits, st0 = wc.tests, sb0 = wc.boxes;
      int h = traverse<true, kCount>(sc, make_ray(o, d), 0.0f, tm, stack, cap, sfail, wc);
      count_ray<kCount>(ctr, 1, ~depth, wc.visits - sv0, wc.tests - st0, wc.boxes - sb0);
      count_px<kCount>(fp, pixel, ~depth, 1);
      if (sfail) atomicOr(sc.status, kErrTraversalLimit);
      if (h < 0 && !sfail) add_fb(fp, pixel, w);
    } else if (have) {
      float t = INFINITY;
      bool fail = false;
      unsigned v0 = wc.visits, t0 = wc.tests, b0 = wc.boxes;
      int hit = traverse<false, kCount>(sc, make_ray(o, d), 0.0f, t, stack, cap, fail, wc);
      count_ray<kCount>(ctr, 0, depth, wc.visits - v0, wc.tests - t0, wc.boxes - b0);
      count_px<kCount>(fp, pixel, depth, 0);
      if (fail) atomicOr(sc.status, kErrTraversalLimit);
      bool live = hit >= 0;
      if (!live) add_fb(fp, pixel, w * bg);
      Surface sf;
      if (live) {
        atomicAdd(&s_cnt[2][depth], 1u);
        sf = surface_at(sc, hit, o, d, t, fp.eps_scale);
        // L_e, Eq. 7 (frames with the diffuse bounce run every depth as a
        // wavefront, so no path here is a bounce and every hit adds its L_e)
        if (sf.emission.x != 0.f || sf.emission.y != 0.f || sf.emission.z != 0.f) add_fb(fp, pixel, w * sf.emission);
        if (depth == fp.nrc_depth) {
          // radiance cache (as in k_trace); the selection probability comes
          // from the previous frame's number of cache hits
          atomicAdd(&ctr->cache_hits, 1u);
          unsigned pos = atomicAdd(&ctr->infer_count, 1u);
          if (pos < fp.infer_cap) {
            float4* q = fp.infer_q + 4 * (size_t)pos;
            q[0] = make_float4(sf.p.x, sf.p.y, sf.p.z, __int_as_float(pixel));
            q[1] = make_float4(sf.n.x, sf.n.y, sf.n.z, 0.f);
            q[2] = make_float4(-d.x, -d.y, -d.z, 0.f);
            q[3] = make_float4(w.x, w.y, w.z, 0.f);
          } else {
            atomicOr(sc.status, kErrQueueOverflow);
          }
          unsigned prev = fp.prev_hits ? *fp.prev_hits : 0u;
          float u = (float)(hash32(fp.seed ^ hash32((uint32_t)pixel * 0x9E3779B9u ^ __float_as_uint(d.x))) >> 8) *
                    (1.0f / 16777216.0f);
          bool sel = fp.train_batch > 0 && (prev == 0u || (float)fp.train_batch > u * (float)prev);
          unsigned slot = sel ? atomicAdd(&ctr->train_count, 1u) : 0u;
          if (sel && slot < fp.train_cap) {
            float4* q = fp.train_q + 3 * (size_t)slot;
            q[0] = make_float4(sf.p.x, sf.p.y, sf.p.z, __int_as_float((int)slot));
            q[1] = make_float4(sf.n.x, sf.n.y, sf.n.z, 0.f);
            q[2] = make_float4(-d.x, -d.y, -d.z, 0.f);
            w = mk3(1.f, 1.f, 1.f);
            pixel = ~(int)slot;   // traced on, with unit weight, into the training target
          } else {
            live = false;          // this path ends in the cache
          }
        }
      }
      if (live) {
        if (sf.kind != RT_MAT_DIELECTRIC && (1.f - sf.rho) > 0.f) {
          // point lights, then one sampled point of each area light and emitter
          for (int li = 0; li < sc.n_lights + (kPass ? sc.n_alights + sc.n_emitters : 0); ++li) {
            f3 contrib, os, sd;
            float tmax;
            bool lit;
            if (li < sc.n_lights) {
              lit = light_term(sf, d, w, __ldg(&sc.lights[2 * li]), __ldg(&sc.lights[2 * li + 1]), contrib, os, sd,
                               tmax);
            } else {
              lit = false;
              if constexpr (kPass) {
                float a, b;
                pass_sample(fp.ps, pixel, code, (uint32_t)(li - sc.n_lights), a, b);
                lit = area_term(sf, d, w, area_point(sc, li - sc.n_lights, a, b), contrib, os, sd, tmax);
              }
            }
            if (!lit) continue;
            atomicAdd(&s_cnt[1][depth], 1u);
            // to the warp's pending stack for a free lane; traced here when it is full
            int pos = atomicAdd(&s_np[warp], 1);
            if (pos < kWarpPending) {
              float4* r = s_pend[warp][pos];
              r[0] = make_float4(os.x, os.y, os.z, __int_as_float(pixel));
              r[1] = make_float4(sd.x, sd.y, sd.z, __int_as_float(~depth));
              r[2] = make_float4(contrib.x, contrib.y, contrib.z, tmax);
              continue;
            }
            atomicSub(&s_np[warp], 1);
            bool sfail = false;
            unsigned sv0 = wc.visits, st0 = wc.tests, sb0 = wc.boxes;
            int h = traverse<true, kCount>(sc, make_ray(os, sd), 0.0f, tmax, stack, cap, sfail, wc);
            count_ray<kCount>(ctr, 1, depth, wc.visits - sv0, wc.tests - st0, wc.boxes - sb0);
            count_px<kCount>(fp, pixel, depth, 1);
            if (sfail) atomicOr(sc.status, kErrTraversalLimit);
            if (h < 0 && !sfail) add_fb(fp, pixel, contrib);
          }
        }
        if (depth < fp.max_depth) {
          ch = children_of(sf, d, w);
          if (ch.want_r || ch.want_t) atomicAdd(&s_cnt[0][depth + 1], (unsigned)ch.want_r + (unsigned)ch.want_t);
        }
      }
    }
    // --- a second child goes to the warp's stack (or this lane's overflow)
    bool two = have && ch.want_r && ch.want_t;
    unsigned m2 = __ballot_sync(kFull, two);
    if (m2) {
      __syncwarp();
      int np2 = s_np[warp];
      int room = kWarpPending - np2;
      int rank = __popc(m2 & lt);
      float4 r0 = make_float4(ch.or_.x, ch.or_.y, ch.or_.z, __int_as_float(pixel));
      float4 r1 = make_float4(ch.dr.x, ch.dr.y, ch.dr.z, __int_as_float(depth + 1));
      float4 r2 = make_float4(ch.wr.x, ch.wr.y, ch.wr.z, __uint_as_float(code << 1));
      if (two) {
        if (rank < room) {
          float4* r = s_pend[warp][np2 + rank];
          r[0] = r0;
          r[1] = r1;
          r[2] = r2;
        } else if (nl < RT_MAX_DEPTH) {
          local[nl][0] = r0;
          local[nl][1] = r1;
          local[nl][2] = r2;
          ++nl;
        } else {
          atomicOr(sc.status, kErrQueueOverflow);   // not reachable for depth <= 16
        }
      }
      __syncwarp();
      if (lane == 0) s_np[warp] = np2 + min(__popc(m2), room);
      __syncwarp();
    }
    // --- this lane follows its (other) child, or is free for new work
    if (have) {
      if (ch.want_t) {
        o = ch.ot;
        d = ch.dt;
        w = ch.wt;
        code = (code << 1) | 1u;
        ++depth;
      } else if (ch.want_r) {
        o = ch.or_;
        d = ch.dr;
        w = ch.wr;
        code <<= 1;
        ++depth;
      } else {
        have = false;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= RT_MAX_DEPTH; i += blockDim.x) {
    if (s_cnt[0][i]) atomicAdd(&ctr->rays[i], s_cnt[0][i]);
    if (s_cnt[1][i]) atomicAdd(&ctr->shadow[i], s_cnt[1][i]);
    if (s_cnt[2][i]) atomicAdd(&ctr->hits[i], s_cnt[2][i]);
  }
}

// ---------------------------------------------------------------------------
// plain queries on caller rays
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTraceThreads) k_query(DevScene sc, const float* __restrict__ o,
                                                         const float* __restrict__ d, const float* __restrict__ tmax_in,
                                                         int64_t n, float tmin, int any, int cap,
                                                         int32_t* __restrict__ prim_out, float* __restrict__ t_out,
                                                         uint8_t* __restrict__ occ_out) {
  __shared__ int s_stack[kStackShared * kTraceThreads];
  int* stack = s_stack + threadIdx.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool part = i < n;   // every lane of the warp walks together (traverse_warp)
  int64_t k = part ? i : 0;
  RayInv ri = make_ray(part ? mk3(o[3 * k], o[3 * k + 1], o[3 * k + 2]) : mk3(0, 0, 0),
                       part ? mk3(d[3 * k], d[3 * k + 1], d[3 * k + 2]) : mk3(0, 0, 1));
  bool fail = false;
  WorkCount wc = {0u, 0u, 0u, 0u};
  if (any) {
    float tm = part ? tmax_in[k] : 0.f;
    int h = traverse_warp<true, false>(sc, ri, part, tmin, tm, stack, cap, fail, wc);
    if (part) occ_out[i] = h >= 0 ? 1 : 0;
  } else {
    float t = INFINITY;
    int h = traverse_warp<false, false>(sc, ri, part, tmin, t, stack, cap, fail, wc);
    if (part) {
      prim_out[i] = h >= 0 ? __float_as_int(sc.prims[3 * (size_t)h + 1].w) : -1;
      t_out[i] = h >= 0 ? t : INFINITY;
    }
  }
  if (fail) atomicOr(sc.status, kErrTraversalLimit);
}

__global__ void k_camera_rays(CamBasis cb, int W, int H, float* __restrict__ o, float* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  f3 oo, dd;
  camera_ray(cb, W, H, i % W, i / W, oo, dd);
  o[3 * i] = oo.x;
  o[3 * i + 1] = oo.y;
  o[3 * i + 2] = oo.z;
  d[3 * i] = dd.x;
  d[3 * i + 1] = dd.y;
  d[3 * i + 2] = dd.z;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Every field of a frame's parameters, with the radiance cache off.
static FrameParams frame_defaults() {
  FrameParams fp;
  memset(&fp, 0, sizeof(fp));
  fp.path_depth0 = 1;
  fp.nrc_depth = -1;
  fp.target = nullptr;
  fp.infer_q = fp.train_q = nullptr;
  fp.prev_hits = nullptr;
  fp.ps.strata = 1;   // pass 0 of seed 0, no jitter
  return fp;
}

CamBasis camera_basis(const rt_camera* c, int W, int H) {
  // host FP32 arithmetic, once per frame
  CamBasis cb;
  float fx = c->look_at[0] - c->eye[0], fy = c->look_at[1] - c->eye[1], fz = c->look_at[2] - c->eye[2];
  float fl = 1.0f / std::sqrt(fx * fx + fy * fy + fz * fz);
  fx *= fl;
  fy *= fl;
  fz *= fl;
  float ux = c->up[0], uy = c->up[1], uz = c->up[2];
  float rx = fy * uz - fz * uy, ry = fz * ux - fx * uz, rz = fx * uy - fy * ux;
  float rl = 1.0f / std::sqrt(rx * rx + ry * ry + rz * rz);
  rx *= rl;
  ry *= rl;
  rz *= rl;
  cb.eye = {c->eye[0], c->eye[1], c->eye[2]};
  cb.f = {fx, fy, fz};
  cb.r = {rx, ry, rz};
  cb.u = {ry * fz - rz * fy, rz * fx - rx * fz, rx * fy - ry * fx};
  cb.h = std::tan(0.5f * c->vfov_deg * 3.14159265358979f / 180.0f);
  cb.aspect = (float)W / (float)H;
  return cb;
}

static int g_blocks_per_sm_trace = 0, g_blocks_per_sm_shadow = 0;


using TraceKernel = void (*)(DevScene, FrameParams, int, int);
using PathsKernel = void (*)(DevScene, FrameParams, int);

static TraceKernel trace_kernel(bool primary, bool count, bool pass) {
  if (primary) {
    if (count) return pass ? k_trace<true, true, true> : k_trace<true, true, false>;
    return pass ? k_trace<true, false, true> : k_trace<true, false, false>;
  }
  if (count) return pass ? k_trace<false, true, true> : k_trace<false, true, false>;
  return pass ? k_trace<false, false, true> : k_trace<false, false, false>;
}

static PathsKernel paths_kernel(bool count, bool pass) {
  if (count) return pass ? k_paths<true, true> : k_paths<true, false>;
  return pass ? k_paths<false, true> : k_paths<false, false>;
}

static void occupancy(rt_scene* s) {
  if (s->trace_blocks) return;
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_trace<false, false, false>, kTraceThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_shadow<false>, kTraceThreads, 0);
  int c = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_paths<false, false>, kTraceThreads, 0);
  s->paths_blocks = s->sm_count * std::max(c, 1);
  g_blocks_per_sm_trace = std::max(a, 1);
  g_blocks_per_sm_shadow = std::max(b, 1);
  s->trace_blocks = s->sm_count * g_blocks_per_sm_trace;
  s->shadow_blocks = s->sm_count * g_blocks_per_sm_shadow;
}

// Lazy module loading places a kernel's code when the kernel is first
// used, after whatever was loaded before it.  The frame kernels' speed was
// measured to depend on that placement (the shadow kernel, which runs
// beside the others, by up to 4 %), and so on the sizes of unrelated
// kernels that happened to load first, such as the BVH build's.  The first
// scene created on a device therefore loads them before anything else of
// this library, in a fixed order: the kernels of a plain frame first, then
// their counting and sampling instances.  Of the orders measured on the
// 1080p terrain, this one gave the faster placement (shadow kernel 0.584
// against 0.606 ms in a render loop).
void preload_frame_kernels(int device) {
  static std::mutex mu;
  static std::vector<char> done;
  std::lock_guard<std::mutex> g(mu);
  if (device < 0) return;
  if ((size_t)device >= done.size()) done.resize((size_t)device + 1, 0);
  if (done[device]) return;
  done[device] = 1;
  const void* order[] = {(const void*)k_trace<false, false, false>, (const void*)k_shadow<false>,
                         (const void*)k_paths<false, false>,        (const void*)k_trace<true, false, false>,
                         (const void*)k_trace<true, false, true>,   (const void*)k_trace<false, false, true>,
                         (const void*)k_paths<false, true>,         (const void*)k_trace<true, true, false>,
                         (const void*)k_trace<false, true, false>,  (const void*)k_shadow<true>,
                         (const void*)k_paths<true, false>,         (const void*)k_trace<true, true, true>,
                         (const void*)k_trace<false, true, true>,   (const void*)k_paths<true, true>};
  for (const void* f : order) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) cudaGetLastError();
  }
}

bool finite_cam(const rt_camera* c) {
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(c->eye[i]) || !std::isfinite(c->look_at[i]) || !std::isfinite(c->up[i])) return false;
  if (!std::isfinite(c->vfov_deg) || !(c->vfov_deg > 0.f) || !(c->vfov_deg < 180.f)) return false;
  float fx = c->look_at[0] - c->eye[0], fy = c->look_at[1] - c->eye[1], fz = c->look_at[2] - c->eye[2];
  if (fx == 0.f && fy == 0.f && fz == 0.f) return false;
  float rx = fy * c->up[2] - fz * c->up[1], ry = fz * c->up[0] - fx * c->up[2], rz = fx * c->up[1] - fy * c->up[0];
  return rx != 0.f || ry != 0.f || rz != 0.f;
}

// Timing: event pairs (start, end) recorded around each kernel on the
// stream it runs on; pair 0 brackets the whole frame.  The events are the
// scene's and are reused frame after frame.
static int timing_begin(rt_scene* s, int kind, cudaStream_t st) {
  int slot = s->tcount++;
  while ((size_t)(2 * s->tcount) > s->tev.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    s->tev.push_back(e);
  }
  if ((size_t)s->tcount > s->tkind.size()) s->tkind.resize(s->tcount);
  s->tkind[slot] = kind;
  cudaEventRecord(s->tev[2 * slot], st);
  return slot;
}

static void timing_end(rt_scene* s, int slot, cudaStream_t st) { cudaEventRecord(s->tev[2 * slot + 1], st); }

// Per-kernel times of the last timed frame, summed by kind (waits for the
// frame's end event only).
static rt_status stage_times(rt_scene* s, float* total, float* trace, float* shadow) {
  *total = *trace = *shadow = 0.f;
  if (s->tcount < 1) return set_error(RT_ERR_INVALID_ARG, "no frame was rendered with RT_FLAG_STAGE_TIMING");
  cudaError_t e = cudaEventSynchronize(s->tev[1]);
  if (e != cudaSuccess) return cuda_error(e, "stage times");
  cudaEventElapsedTime(total, s->tev[0], s->tev[1]);
  for (int i = 1; i < s->tcount; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->tev[2 * i], s->tev[2 * i + 1]);
    if (s->tkind[i] == 0) *trace += ms;
    else if (s->tkind[i] == 1) *shadow += ms;
  }
  return RT_OK;
}

// The side stream that runs each depth's shadow kernel while the main
// stream traces the next depth, and the events that order them.
rt_status ensure_side_stream(rt_scene* s) {
  if (s->side) return RT_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
  for (int d = 0; e == cudaSuccess && d <= RT_MAX_DEPTH; ++d) {
    e = cudaEventCreateWithFlags(&s->ev_traced[d], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_shadowed[d], cudaEventDisableTiming);
  }
  return cuda_error(e, "side stream");
}

static rt_status render_impl(rt_scene* s, const rt_camera* cam, int W, int H, int D, float* out,
                             const rt_render_options* opt_in, int32_t* aov_prim, float* aov_t, rt_render_stats* stats,
                             cudaStream_t st, rt_nrc* nrc = nullptr, int train = 0, const rt_pass* pass = nullptr) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_render: scene is NULL");
  if (!cam || !finite_cam(cam)) return set_error(RT_ERR_INVALID_ARG, "rt_render: invalid camera");
  if (W < 1 || H < 1) return set_error(RT_ERR_INVALID_ARG, "rt_render: width and height must be >= 1");
  if ((int64_t)W * H > (int64_t)1 << 30) return set_error(RT_ERR_UNSUPPORTED, "rt_render: image too large");
  if (D < 0 || D > RT_MAX_DEPTH) return set_error(RT_ERR_INVALID_ARG, "rt_render: max_depth outside [0, 16]");
  if (!out) return set_error(RT_ERR_INVALID_ARG, "rt_render: out_rgb is NULL");
  rt_render_options opt;
  rt_render_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (!std::isfinite(opt.background[0]) || !std::isfinite(opt.background[1]) || !std::isfinite(opt.background[2]) ||
      !std::isfinite(opt.eps_scale) || opt.eps_scale < 0.f || opt.queue_capacity < 0 || opt.traversal_cap < 0)
    return set_error(RT_ERR_INVALID_ARG, "rt_render: invalid options");
  const bool deterministic = (opt.flags & RT_FLAG_DETERMINISTIC) != 0;
  if (nrc && deterministic)
    return set_error(RT_ERR_UNSUPPORTED, "rt_render_nrc: the radiance cache does not take RT_FLAG_DETERMINISTIC");
  bool use_bvh = opt.use_bvh != 0;
  if (use_bvh && !s->built) return set_error(RT_ERR_NOT_BUILT, "rt_render: BVH requested before rt_bvh_build");
  occupancy(s);
  // shadow rays per hit: one per point light, area light and emissive primitive
  int64_t lights = std::max<int64_t>(s->n_lights + s->n_alights + s->n_emitters, 1);
  int64_t qcap = opt.queue_capacity > 0 ? opt.queue_capacity : std::max<int64_t>(2 * (int64_t)W * H, 65536);
  int64_t scap = qcap * lights;
  if (qcap > 0x7fffffffLL || scap > 0x7fffffffLL) return set_error(RT_ERR_UNSUPPORTED, "rt_render: queue too large");
  // depth 0 casts up to W*H*lights shadow rays, a deeper depth up to qcap*lights;
  // shadowq[0] serves the even depths, shadowq[1] the odd ones
  int64_t pcap = std::max<int64_t>((int64_t)W * H * lights, scap);
  if (pcap > 0x7fffffffLL) return set_error(RT_ERR_UNSUPPORTED, "rt_render: shadow queue too large");
  rt_status rs;
  if ((rs = ensure(s->rayq[0], (size_t)qcap * 48)) || (rs = ensure(s->rayq[1], (size_t)qcap * 48)) ||
      (rs = ensure(s->shadowq[0], (size_t)pcap * 48)) ||
      (rs = ensure(s->shadowq[1], D > 0 ? (size_t)pcap * 48 : 16)) || (rs = ensure(s->counters, sizeof(Counters))) ||
      (rs = ensure_side_stream(s)))
    return rs;
  s->ray_cap = qcap;
  s->shadow_cap = pcap;
  DevScene sc = dev_scene(s, use_bvh);
  int64_t tcap = opt.traversal_cap > 0 ? opt.traversal_cap : 4 * std::max<int64_t>(s->n_nodes4, 1) + 64;
  int cap = (int)std::min<int64_t>(tcap, 0x7fffffff);
  FrameParams fp = frame_defaults();
  if (pass) {
    fp.ps.seed_lo = (uint32_t)pass->seed;
    fp.ps.seed_hi = (uint32_t)(pass->seed >> 32);
    fp.ps.pass = pass->index;
    fp.ps.strata = pass->strata;
    fp.ps.jitter = pass->jitter != 0;
  }
  fp.ps.bounce = (opt.flags & RT_FLAG_DIFFUSE_BOUNCE) != 0;
  // kernels with the sampling code
  const bool pass_k = s->n_alights > 0 || s->n_emitters > 0 || fp.ps.jitter || fp.ps.bounce;
  fp.cam = camera_basis(cam, W, H);
  fp.W = W;
  fp.H = H;
  fp.tiles_x = (W + 7) / 8;
  fp.tiles_y = (H + 3) / 4;
  fp.max_depth = D;
  fp.bg_r = opt.background[0];
  fp.bg_g = opt.background[1];
  fp.bg_b = opt.background[2];
  fp.eps_scale = opt.eps_scale;
  fp.fb = out;
  fp.aov_prim = aov_prim;
  fp.aov_t = aov_t;
  fp.rayq[0] = (float4*)s->rayq[0].p;
  fp.rayq[1] = (float4*)s->rayq[1].p;
  fp.shadowq[0] = (float4*)s->shadowq[0].p;
  fp.shadowq[1] = (float4*)s->shadowq[1].p;
  fp.ray_cap = (unsigned)qcap;
  fp.shadow_cap = (unsigned)pcap;
  fp.ctr = (Counters*)s->counters.p;
  int T = -1;   // radiance-cache depth of this frame
  if (nrc) {
    NrcFrame nf;
    rs = nrc_frame_buffers(nrc, qcap, train != 0, &nf);
    if (rs) return rs;
    T = nf.depth <= D ? nf.depth : -1;
    fp.nrc_depth = T;
    fp.target = nf.target;
    fp.infer_q = nf.infer_q;
    fp.train_q = nf.train_q;
    fp.infer_cap = nf.infer_cap;
    fp.train_cap = nf.train_cap;
    fp.train_batch = train ? nf.train_batch : 0u;
    fp.seed = nf.seed;
    fp.path_depth0 = T + 1;
    if (T >= 0 && train) cudaMemsetAsync(fp.target, 0, (size_t)nf.train_cap * 12, st);
  }
  bool timing = (opt.flags & RT_FLAG_STAGE_TIMING) != 0;
  bool count = (opt.flags & RT_FLAG_COUNT_WORK) != 0;
  int launches = 0;
  int frame_slot = -1;
  if (timing) {
    s->tcount = 0;
    frame_slot = timing_begin(s, 3, st);
  }
  const size_t n_out = (size_t)W * H * 3;
  if (deterministic) {
    if ((rs = ensure(s->fb_fixed, n_out * sizeof(unsigned long long)))) return rs;
    fp.fb_fixed = (unsigned long long*)s->fb_fixed.p;
    cudaMemsetAsync(fp.fb_fixed, 0, n_out * sizeof(unsigned long long), st);   // out is written at the end
  } else {
    fp.fb_store = 1;   // the depth-0 kernel writes every pixel first: no clear
  }
  cudaMemsetAsync(fp.ctr, 0, sizeof(Counters), st);
  if (count && opt.ray_counts != nullptr) {
    fp.px_rays = opt.ray_counts;
    fp.px_stride = 2 * (D + 1);
    cudaMemsetAsync(fp.px_rays, 0, (size_t)W * H * fp.px_stride * sizeof(unsigned), st);
  }
  bool per_depth = (opt.flags & RT_FLAG_PER_DEPTH_WAVEFRONT) != 0;
  const bool serial = (opt.flags & RT_FLAG_SERIAL_STAGES) != 0;
  // depths 0..last run as wavefronts; the rest run as depth-first paths,
  // which meet the cache at depth T themselves unless it is depth 0.  With
  // the diffuse bounce nearly every hit has a child, every depth is wide,
  // and wavefronts are faster at each of them (measured on the 1080p terrain:
  // 2.2 ms a pass against 3.5 ms depth first); the radiance cache never bounces.
  // Depth 1 (tens of thousands of rays) is a wavefront too and the
  // depth-first kernel takes the tail from depth 2 (measured: 1.37 against
  // 1.38-1.40 ms a step; a wavefront depth 2 as well was slower), unless the
  // cache sits at depth 0 or 1.
  if (fp.ps.bounce) per_depth = true;
  int last = per_depth ? D : (T < 0 || T > kWavefrontDepths ? std::min(D, kWavefrontDepths) : 0);
  bool cache_in_paths = !per_depth && T >= 1;
  if (per_depth || T == 0) fp.path_depth0 = T >= 0 ? T + 1 : 1;
  else fp.path_depth0 = last + 1;
  if (cache_in_paths && fp.nrc_depth >= 0) fp.prev_hits = nrc_prev_hits(nrc);
  // shadow(depth) runs on the side stream, beside trace(depth + 1) (on the
  // main stream after it when the stages are serialised)
  auto launch_shadow = [&](int depth) {
    cudaStream_t sst = serial ? st : s->side;
    cudaStreamWaitEvent(sst, s->ev_traced[depth], 0);
    int slot = timing ? timing_begin(s, 1, sst) : -1;
    if (count) k_shadow<true><<<s->shadow_blocks, kTraceThreads, 0, sst>>>(sc, fp, depth, cap);
    else k_shadow<false><<<s->shadow_blocks, kTraceThreads, 0, sst>>>(sc, fp, depth, cap);
    if (timing) timing_end(s, slot, sst);
    cudaEventRecord(s->ev_shadowed[depth], sst);
    launches += 1;
  };
  for (int depth = 0; depth <= last; ++depth) {
    // trace(depth) fills the shadow buffer that shadow(depth - 2) reads
    if (depth >= 2) cudaStreamWaitEvent(st, s->ev_shadowed[depth - 2], 0);
    int slot = timing ? timing_begin(s, 0, st) : -1;
    if (depth == 0) {
      trace_kernel(true, count, pass_k)<<<s->trace_blocks, kTraceThreads, 0, st>>>(sc, fp, 0, cap);
    } else {
      trace_kernel(false, count, pass_k)<<<s->trace_blocks, kTraceThreads, 0, st>>>(sc, fp, depth, cap);
    }
    if (timing) timing_end(s, slot, st);
    cudaEventRecord(s->ev_traced[depth], st);
    launches += 1;
    launch_shadow(depth);
  }
  bool run_paths = !per_depth && D >= fp.path_depth0 && (T < 0 || cache_in_paths || train);
  if (T >= 0 && !cache_in_paths) {
    // cache lookups of the depth-T hits, beside the training rays' paths
    int slot = timing ? timing_begin(s, 2, s->side) : -1;
    rs = nrc_infer_launch(nrc, fp.infer_q, &fp.ctr->infer_count, fp.infer_cap, out, nullptr, s->status, s->side);
    if (rs) return rs;
    if (timing) timing_end(s, slot, s->side);
    cudaEventRecord(s->ev_shadowed[last], s->side);
    launches += 1;
  }
  if (run_paths) {
    int slot = timing ? timing_begin(s, 0, st) : -1;
    paths_kernel(count, pass_k)<<<s->paths_blocks, kTraceThreads, 0, st>>>(sc, fp, cap);
    if (timing) timing_end(s, slot, st);
    launches += 1;
  }
  if (cache_in_paths) {
    int slot = timing ? timing_begin(s, 2, st) : -1;
    rs = nrc_infer_launch(nrc, fp.infer_q, &fp.ctr->infer_count, fp.infer_cap, out, nullptr, s->status, st);
    if (rs) return rs;
    if (timing) timing_end(s, slot, st);
    nrc_keep_hits(nrc, &fp.ctr->cache_hits, st);
    launches += 2;
  }
  cudaStreamWaitEvent(st, s->ev_shadowed[last], 0);
  if (deterministic) {
    k_fixed_to_float<<<(unsigned)((n_out + 255) / 256), 256, 0, st>>>(out, fp.fb_fixed, n_out);
    launches += 1;
  }
  if (T >= 0 && train) {
    // one Adam step on this frame's targets (complete once both streams joined)
    int slot = timing ? timing_begin(s, 2, st) : -1;
    rs = nrc_train_launch(nrc, fp.train_q, fp.target, &fp.ctr->train_count, fp.train_cap, s->status, st);
    if (rs) return rs;
    if (timing) timing_end(s, slot, st);
    launches += 3;   // training, Adam, BF16 repack
  }
  if (timing) timing_end(s, frame_slot, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "rt_render launch");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    Counters c;
    e = cudaMemcpyAsync(&c, fp.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "rt_render stats");
    stats->primary = (uint64_t)W * H;
    stats->rays_per_depth[0] = stats->primary;
    for (int d = 0; d <= D; ++d) {
      if (d > 0) {
        stats->rays_per_depth[d] = std::min<uint64_t>(c.rays[d], (uint64_t)qcap);
        stats->secondary += stats->rays_per_depth[d];
      }
      stats->shadow_per_depth[d] = std::min<uint64_t>(c.shadow[d], (uint64_t)fp.shadow_cap);
      stats->shadow += stats->shadow_per_depth[d];
      stats->hits_per_depth[d] = c.hits[d];
      for (int k = 0; k < 2; ++k) {
        stats->node_visits[k] += c.visits[k][d];
        stats->prim_tests[k] += c.tests[k][d];
        stats->box_tests[k] += c.boxes[k][d];
        stats->node_visits_per_depth[k][d] = c.visits[k][d];
        stats->max_visits_per_depth[k][d] = c.max_visits[k][d];
      }
    }
    stats->launches = launches;
    if (timing) stage_times(s, &stats->ms_total, &stats->ms_trace, &stats->ms_shadow);
    rt_status sync_st = rt_scene_sync(s, st);
    if (sync_st != RT_OK) return sync_st;
  }
  return RT_OK;
}

}  // namespace rtb

using namespace rtb;

extern "C" {

rt_status rt_render(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth, float* out,
                    void* stream) {
  return render_impl(s, cam, width, height, max_depth, out, nullptr, nullptr, nullptr, nullptr,
                     (cudaStream_t)stream);
}

rt_status rt_render_ex(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth, float* out,
                       const rt_render_options* opt, int32_t* aov_prim, float* aov_t, rt_render_stats* stats,
                       void* stream) {
  return render_impl(s, cam, width, height, max_depth, out, opt, aov_prim, aov_t, stats, (cudaStream_t)stream);
}

rt_status rt_render_host(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth, float* out_host,
                         const rt_render_options* opt, void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_render_host: scene is NULL");
  if (!out_host) return set_error(RT_ERR_INVALID_ARG, "rt_render_host: out_rgb_host is NULL");
  if (width < 1 || height < 1) return set_error(RT_ERR_INVALID_ARG, "rt_render_host: bad size");
  size_t bytes = (size_t)width * height * 3 * sizeof(float);
  rt_status rs = ensure(s->fb_host_stage, bytes);
  if (rs) return rs;
  cudaStream_t st = (cudaStream_t)stream;
  rs = render_impl(s, cam, width, height, max_depth, (float*)s->fb_host_stage.p, opt, nullptr, nullptr, nullptr, st);
  if (rs) return rs;
  cudaError_t e = cudaMemcpyAsync(out_host, s->fb_host_stage.p, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "rt_render_host");
  return RT_OK;
}

static rt_status ensure_copy_stream(rt_scene* s) {
  if (s->copy_stream) return RT_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_issue, cudaEventDisableTiming);
  for (int k = 0; e == cudaSuccess && k < 2; ++k) {
    e = cudaEventCreateWithFlags(&s->ev_rendered[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_copied[k], cudaEventDisableTiming);
  }
  return cuda_error(e, "copy stream");
}

}  // extern "C"

// The pending copy of image p: after its frame (ev_rendered[p]) and, when a
// next frame is being queued on `after`, after the work already queued on
// that stream (the next frame's update and build), so that it runs beside
// the next frame's render.
static rt_status queue_copy(rt_scene* s, cudaStream_t after, bool have_after) {
  const int p = s->copy_pending;
  if (p < 0) return RT_OK;
  cudaError_t e = cudaStreamWaitEvent(s->copy_stream, s->ev_rendered[p], 0);
  if (e == cudaSuccess && have_after) e = cudaEventRecord(s->ev_issue, after);
  if (e == cudaSuccess && have_after) e = cudaStreamWaitEvent(s->copy_stream, s->ev_issue, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->copy_dst, s->fb_stage[p].p, s->copy_bytes, cudaMemcpyDeviceToHost, s->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_copied[p], s->copy_stream);
  s->copy_pending = -1;
  return cuda_error(e, "rt_render_host_async copy");
}

rt_status rtb::issue_pending_copy(rt_scene* s) { return queue_copy(s, nullptr, false); }

extern "C" {

rt_status rt_render_host_async(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                               float* out_host, const rt_render_options* opt, void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_render_host_async: scene is NULL");
  if (!out_host) return set_error(RT_ERR_INVALID_ARG, "rt_render_host_async: out_rgb_host is NULL");
  if (width < 1 || height < 1) return set_error(RT_ERR_INVALID_ARG, "rt_render_host_async: bad size");
  const size_t bytes = (size_t)width * height * 3 * sizeof(float);
  rt_status rs = ensure_copy_stream(s);
  if (rs) return rs;
  const int k = s->stage_next;
  if ((rs = ensure(s->fb_stage[k], bytes))) return rs;
  cudaStream_t st = (cudaStream_t)stream;
  // The previous frame's image goes out now, beside this frame's render:
  // queued right after that frame, the copy ran beside this frame's build,
  // whose latency-bound kernels it slowed by a third (1080p terrain, a
  // step 1.40 against 1.26 ms end to end).
  if ((rs = queue_copy(s, st, true))) return rs;
  // the image this frame renders into was copied out two calls ago: wait for that copy
  cudaError_t e = cudaStreamWaitEvent(st, s->ev_copied[k], 0);
  if (e != cudaSuccess) return cuda_error(e, "rt_render_host_async");
  rs = render_impl(s, cam, width, height, max_depth, (float*)s->fb_stage[k].p, opt, nullptr, nullptr, nullptr, st);
  if (rs) return rs;
  e = cudaEventRecord(s->ev_rendered[k], st);
  if (e != cudaSuccess) return cuda_error(e, "rt_render_host_async");
  s->copy_pending = k;
  s->copy_dst = out_host;
  s->copy_bytes = bytes;
  s->stage_next = k ^ 1;
  return RT_OK;
}

// pass k folded into the running mean: accum += (image - accum) / (k + 1)
__global__ void k_accumulate(float* __restrict__ accum, const float* __restrict__ img, size_t n, int k) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  accum[i] = k == 0 ? img[i] : accum[i] + (img[i] - accum[i]) / (float)(k + 1);
}

}  // extern "C"

// One pass (with or without the radiance cache) folded into the running mean.
static rt_status render_pass_impl(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth,
                                  const rt_pass* pass, float* accum, const rt_render_options* opt,
                                  rt_render_stats* stats, void* stream, rt_nrc* nrc, int train) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_render_pass: scene is NULL");
  if (!pass || !accum) return set_error(RT_ERR_INVALID_ARG, "rt_render_pass: NULL pass or image");
  if (pass->index < 0 || pass->strata < 1 || pass->reserved != 0)
    return set_error(RT_ERR_INVALID_ARG, "rt_render_pass: index < 0, strata < 1 or reserved != 0");
  if (width < 1 || height < 1) return set_error(RT_ERR_INVALID_ARG, "rt_render_pass: bad size");
  size_t n = (size_t)width * height * 3;
  rt_status rs = ensure(s->pass_img, n * sizeof(float));
  if (rs) return rs;
  cudaStream_t st = (cudaStream_t)stream;
  rs = render_impl(s, cam, width, height, max_depth, (float*)s->pass_img.p, opt, nullptr, nullptr, stats, st, nrc,
                   train, pass);
  if (rs) return rs;
  k_accumulate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(accum, (const float*)s->pass_img.p, n, pass->index);
  return cuda_error(cudaGetLastError(), "rt_render_pass");
}

extern "C" {

rt_status rt_render_pass(rt_scene* s, const rt_camera* cam, int width, int height, int max_depth, const rt_pass* pass,
                         float* accum, const rt_render_options* opt, rt_render_stats* stats, void* stream) {
  return render_pass_impl(s, cam, width, height, max_depth, pass, accum, opt, stats, stream, nullptr, 0);
}

rt_status rt_render_nrc_pass(rt_scene* s, rt_nrc* nrc, const rt_camera* cam, int width, int height, int max_depth,
                             const rt_pass* pass, float* accum, int train, const rt_render_options* opt,
                             rt_render_stats* stats, void* stream) {
  if (!nrc) return set_error(RT_ERR_INVALID_ARG, "rt_render_nrc_pass: cache is NULL");
  return render_pass_impl(s, cam, width, height, max_depth, pass, accum, opt, stats, stream, nrc, train);
}

rt_status rt_render_nrc(rt_scene* s, rt_nrc* nrc, const rt_camera* cam, int width, int height, int max_depth,
                        float* out, int train, const rt_render_options* opt, rt_render_stats* stats, void* stream) {
  if (!nrc) return set_error(RT_ERR_INVALID_ARG, "rt_render_nrc: cache is NULL");
  return render_impl(s, cam, width, height, max_depth, out, opt, nullptr, nullptr, stats, (cudaStream_t)stream, nrc,
                     train);
}

rt_status rt_render_stage_times(rt_scene* s, float* ms_total, float* ms_trace, float* ms_shadow) {
  if (!s || !ms_total || !ms_trace || !ms_shadow)
    return set_error(RT_ERR_INVALID_ARG, "rt_render_stage_times: NULL argument");
  return stage_times(s, ms_total, ms_trace, ms_shadow);
}

rt_status rt_camera_rays(const rt_camera* cam, int width, int height, float* o, float* d, void* stream) {
  if (!cam || !finite_cam(cam)) return set_error(RT_ERR_INVALID_ARG, "rt_camera_rays: invalid camera");
  if (width < 1 || height < 1 || !o || !d) return set_error(RT_ERR_INVALID_ARG, "rt_camera_rays: bad argument");
  int n = width * height;
  k_camera_rays<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(camera_basis(cam, width, height), width, height,
                                                                    o, d);
  return cuda_error(cudaGetLastError(), "rt_camera_rays");
}

static rt_status query(rt_scene* s, const float* o, const float* d, const float* tmax, int64_t n, float tmin,
                       int use_bvh, int any, int32_t* prim, float* t, uint8_t* occ, cudaStream_t st) {
  if (!s || !o || !d || n < 0) return set_error(RT_ERR_INVALID_ARG, "rt_trace: bad argument");
  if (any ? (!tmax || !occ) : (!prim || !t)) return set_error(RT_ERR_INVALID_ARG, "rt_trace: NULL output");
  if (use_bvh && !s->built) return set_error(RT_ERR_NOT_BUILT, "rt_trace: BVH requested before rt_bvh_build");
  if (n == 0) return RT_OK;
  DevScene sc = dev_scene(s, use_bvh != 0);
  int cap = (int)std::min<int64_t>(4 * std::max<int64_t>(s->n_nodes4, 1) + 64, 0x7fffffff);
  int64_t blocks = (n + kTraceThreads - 1) / kTraceThreads;
  k_query<<<(unsigned)blocks, kTraceThreads, 0, st>>>(sc, o, d, tmax, n, tmin, any, cap, prim, t, occ);
  return cuda_error(cudaGetLastError(), "rt_trace");
}

rt_status rt_trace_closest(rt_scene* s, const float* o, const float* d, int64_t n, float tmin, int use_bvh,
                           int32_t* prim, float* t, void* stream) {
  return query(s, o, d, nullptr, n, tmin, use_bvh, 0, prim, t, nullptr, (cudaStream_t)stream);
}

rt_status rt_trace_any(rt_scene* s, const float* o, const float* d, const float* tmax, int64_t n, float tmin,
                       int use_bvh, uint8_t* occ, void* stream) {
  return query(s, o, d, tmax, n, tmin, use_bvh, 1, nullptr, nullptr, occ, (cudaStream_t)stream);
}

rt_status rt_scene_destroy(rt_scene* s) {
  if (!s) return RT_OK;
  issue_pending_copy(s);
  cudaDeviceSynchronize();
  release(s->raw_sph);
  release(s->raw_tri);
  release(s->prims_id);
  release(s->prims_leaf);
  release(s->mats);
  release(s->lights);
  release(s->alights);
  release(s->emitters);
  release(s->pass_img);
  release(s->nodes);
  release(s->nodes4);
  release(s->build_tmp);
  release(s->build_info);
  release(s->rayq[0]);
  release(s->rayq[1]);
  release(s->shadowq[0]);
  release(s->shadowq[1]);
  if (s->build_exec) cudaGraphExecDestroy(s->build_exec);
  if (s->build_cap) cudaStreamDestroy(s->build_cap);
  if (s->ev_build_fork) cudaEventDestroy(s->ev_build_fork);
  if (s->ev_build_join) cudaEventDestroy(s->ev_build_join);
  if (s->side) {
    cudaStreamDestroy(s->side);
    for (int d = 0; d <= RT_MAX_DEPTH; ++d) {
      cudaEventDestroy(s->ev_traced[d]);
      cudaEventDestroy(s->ev_shadowed[d]);
    }
  }
  release(s->counters);
  release(s->fb_host_stage);
  release(s->fb_fixed);
  release(s->fb_stage[0]);
  release(s->fb_stage[1]);
  if (s->copy_stream) {
    cudaStreamDestroy(s->copy_stream);
    cudaEventDestroy(s->ev_issue);
    for (int k = 0; k < 2; ++k) {
      cudaEventDestroy(s->ev_rendered[k]);
      cudaEventDestroy(s->ev_copied[k]);
    }
  }
  for (auto e : s->tev) cudaEventDestroy(e);
  if (s->status) cudaFree(s->status);
  delete s;
  return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rt_render_noalloc: the rt_render frame with its ray queues and counters in
// a fixed, file-scope device array instead of memory allocated on demand.
//
// Who needs it: callers that may not allocate device memory while they
// render - a host application or plug-in framework that owns the GPU memory
// budget and forbids cudaMalloc after start-up, or code that runs inside a
// pre-reserved memory pool.  The scene (and its BVH) is still created and
// built beforehand with the ordinary calls.
// ---------------------------------------------------------------------------
namespace rtb {

constexpr int64_t kNoallocMaxPixels = RT_NOALLOC_MAX_PIXELS;
constexpr int64_t kNoallocMaxLights = RT_NOALLOC_MAX_LIGHTS;
constexpr int64_t kNoallocRayCap = 2 * kNoallocMaxPixels;                 // per ray queue
constexpr int64_t kNoallocShadowCap = kNoallocRayCap * kNoallocMaxLights;  // shadow queue
constexpr size_t kNoallocCounterBytes = (sizeof(Counters) + 255) & ~(size_t)255;
constexpr size_t kNoallocBytes = kNoallocCounterBytes + (size_t)(2 * kNoallocRayCap + kNoallocShadowCap) * 48;

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch, looked up once per device.
static void* g_noalloc_addr[64] = {nullptr};

static rt_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "rt_render_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(RT_ERR_UNSUPPORTED, "rt_render_noalloc: device index above 63");
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "rt_render_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return RT_OK;
}

}  // namespace rtb

extern "C" rt_status rt_render_noalloc(rt_scene* s, const rt_camera* cam, int W, int H, int D, float* out,
                                       void* stream) {
  using namespace rtb;
  cudaStream_t st = (cudaStream_t)stream;
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_render_noalloc: scene is NULL");
  if (!cam || !finite_cam(cam)) return set_error(RT_ERR_INVALID_ARG, "rt_render_noalloc: invalid camera");
  if (W < 1 || H < 1) return set_error(RT_ERR_INVALID_ARG, "rt_render_noalloc: width and height must be >= 1");
  if (D < 0 || D > RT_MAX_DEPTH) return set_error(RT_ERR_INVALID_ARG, "rt_render_noalloc: max_depth outside [0, 16]");
  if (!out) return set_error(RT_ERR_INVALID_ARG, "rt_render_noalloc: out_rgb is NULL");
  if ((int64_t)W * H > kNoallocMaxPixels)
    return set_error(RT_ERR_UNSUPPORTED, "rt_render_noalloc: width*height exceeds RT_NOALLOC_MAX_PIXELS (" +
                                             std::to_string(kNoallocMaxPixels) + "); use rt_render");
  // the shadow queue holds one record per ray and light of any kind
  if (s->n_lights + s->n_alights + s->n_emitters > kNoallocMaxLights)
    return set_error(RT_ERR_UNSUPPORTED, "rt_render_noalloc: more than RT_NOALLOC_MAX_LIGHTS (" +
                                             std::to_string(kNoallocMaxLights) +
                                             ") point, area and emissive lights together; use rt_render");
  if (!s->built) return set_error(RT_ERR_NOT_BUILT, "rt_render_noalloc: call rt_bvh_build first");
  void* base = nullptr;
  rt_status rs = noalloc_scratch(&base);
  if (rs) return rs;
  occupancy(s);
  char* p = (char*)base;
  FrameParams fp = frame_defaults();
  fp.cam = camera_basis(cam, W, H);
  fp.W = W;
  fp.H = H;
  fp.tiles_x = (W + 7) / 8;
  fp.tiles_y = (H + 3) / 4;
  fp.max_depth = D;
  fp.bg_r = fp.bg_g = fp.bg_b = 0.1f;
  fp.eps_scale = 1e-4f;
  fp.fb = out;
  fp.aov_prim = nullptr;
  fp.aov_t = nullptr;
  fp.ctr = (Counters*)p;
  fp.rayq[0] = (float4*)(p + kNoallocCounterBytes);
  fp.rayq[1] = fp.rayq[0] + 3 * kNoallocRayCap;
  fp.shadowq[0] = fp.rayq[1] + 3 * kNoallocRayCap;   // its depths run in order on one stream
  fp.shadowq[1] = fp.shadowq[0];
  fp.ray_cap = (unsigned)kNoallocRayCap;
  fp.shadow_cap = (unsigned)kNoallocShadowCap;
  DevScene sc = dev_scene(s, true);
  int cap = (int)std::min<int64_t>(4 * std::max<int64_t>(s->n_nodes4, 1) + 64, 0x7fffffff);
  // the counters must start at zero; the queues are written before they are read
  cudaError_t e = cudaMemsetAsync(fp.ctr, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return cuda_error(e, "rt_render_noalloc memset");
  fp.fb_store = 1;   // the depth-0 kernel writes every pixel first: no clear
  for (int depth = 0; depth <= D; ++depth) {
    const bool pass_k = sc.n_alights + sc.n_emitters > 0;
    trace_kernel(depth == 0, false, pass_k)<<<s->trace_blocks, kTraceThreads, 0, st>>>(sc, fp, depth, cap);
    k_shadow<false><<<s->shadow_blocks, kTraceThreads, 0, st>>>(sc, fp, depth, cap);
  }
  return cuda_error(cudaGetLastError(), "rt_render_noalloc launch");
}
