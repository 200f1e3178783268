// trace_device.cuh - the device side of tracing shared by the frame
// kernels (render.cu) and the batched kernel (batch.cu): 4-wide BVH
// traversal (per lane and per warp), primitive tests, warp-compacted queue
// pushes and the shading of one hit (Eq. 6-12, Alg. 1).
#pragma once

#include <climits>

#include "rtb_internal.cuh"

namespace rtb {

constexpr int kSentinelLink = kEmptyLink;   // popped from an empty stack; never a valid link
constexpr float kSlabUp = 1.0000005f;    // grows a slab's exit distance by > 2 ulps
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// traversal
// ---------------------------------------------------------------------------
struct RayInv {
  f3 o, d, idir, oid;
};

__device__ __forceinline__ RayInv make_ray(f3 o, f3 d) {
  RayInv r;
  r.o = o;
  r.d = d;
  const float tiny = 8.27e-25f;   // 2^-80: keeps 1/d finite
  float dx = fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x);
  float dy = fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y);
  float dz = fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z);
  r.idir = mk3(1.0f / dx, 1.0f / dy, 1.0f / dz);
  r.oid = mk3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
  return r;
}

struct WorkCount {
  unsigned visits, tests, vmax;   // vmax: most node visits of one ray
  unsigned boxes;                 // child boxes tested (non-empty slots of the visited nodes)
};

template <bool kAny>
__device__ __forceinline__ bool test_prim(float4 r0, float4 r1, float4 r2, int k, const RayInv& r, float tmin,
                                          float& tbest, int& best, int& best_id) {
  float t;
  bool h;
  if (__float_as_int(r0.w) == kKindSphere) h = hit_sphere<!kAny>(r.o, r.d, r0, r1, tmin, tbest, t);
  else h = hit_triangle<!kAny>(r.o, r.d, r0, r1, r2, tmin, tbest, t);
  if (h) {
    if (kAny) {
      best = k;
      return true;
    }
    int id = __float_as_int(r1.w);
    if (t < tbest || id < best_id) {
      tbest = t;
      best = k;
      best_id = id;
    }
  }
  return false;
}

// Tests the primitives [start, start+count) in `prims`.  Closest hit:
// nearest t, ties to the lower primitive id; any hit: returns at the first.
// Two records are loaded before either is tested, so a leaf costs one
// memory round trip per pair rather than per primitive.
template <bool kAny, bool kCount>
__device__ __forceinline__ bool leaf_hits(const float4* __restrict__ prims, int start, int count, const RayInv& r,
                                          float tmin, float& tbest, int& best, int& best_id, WorkCount& wc) {
  int k = start, end = start + count;
  for (; k + 1 < end; k += 2) {
    const float4* a = prims + 3 * (size_t)k;
    float4 a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2);
    float4 b0 = __ldg(a + 3), b1 = __ldg(a + 4), b2 = __ldg(a + 5);
    if (kCount) wc.tests += 2;
    if (test_prim<kAny>(a0, a1, a2, k, r, tmin, tbest, best, best_id)) return true;
    if (test_prim<kAny>(b0, b1, b2, k + 1, r, tmin, tbest, best, best_id)) return true;
  }
  if (k < end) {
    const float4* a = prims + 3 * (size_t)k;
    float4 a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2);
    if (kCount) wc.tests++;
    if (test_prim<kAny>(a0, a1, a2, k, r, tmin, tbest, best, best_id)) return true;
  }
  return false;
}

// The shared part of a thread's stack is a column: entry i at stack[i * kStride]
// (kStride = the block's thread count), so that a warp's lanes hit distinct banks.
template <int kStride = kTraceThreads>
__device__ __forceinline__ int pop_stack(const int* stack, const int* deep, int& sp) {
  if (sp == 0) return kSentinelLink;
  --sp;
  return sp < kStackShared ? stack[sp * kStride] : deep[sp - kStackShared];
}

// Three-input FP32 max / min (PTX max.f32 / min.f32 with three sources,
// sm_100 and later); same NaN rule as fmaxf / fminf.  Measured on the 1080p
// terrain step: 0.3 % faster than nested two-input calls.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Entry time of the ray into one child box of a 4-wide node, or +inf when
// it misses: the ordered slab test over the near and far planes (picked by
// the direction's signs), far distance widened by kSlabUp.  A slot with an
// inverted box (lo = +inf, hi = -inf) always misses.
__device__ __forceinline__ float child_entry(float nx, float ny, float nz, float fx, float fy, float fz,
                                             const RayInv& r, float tmin, float tbest) {
  float tn = max3f(fmaf(nx, r.idir.x, -r.oid.x), fmaf(ny, r.idir.y, -r.oid.y),
                   fmaxf(fmaf(nz, r.idir.z, -r.oid.z), tmin));
  float tf = min3f(fmaf(fx, r.idir.x, -r.oid.x), fmaf(fy, r.idir.y, -r.oid.y),
                   fminf(fmaf(fz, r.idir.z, -r.oid.z), tbest)) * kSlabUp;
  return tn <= tf ? tn : INFINITY;
}

__device__ __forceinline__ void order2(float& da, int& la, float& db, int& lb) {
  bool sw = db < da;
  float d = sw ? db : da;
  int l = sw ? lb : la;
  db = sw ? da : db;
  lb = sw ? la : lb;
  da = d;
  la = l;
}

template <int kStride = kTraceThreads>
__device__ __forceinline__ void push_stack(int* stack, int* deep, int& sp, int v) {
  if (sp < kStackShared) stack[sp * kStride] = v;
  else deep[sp - kStackShared] = v;
  ++sp;
}

// One step of the walk at an inner node of the 4-wide tree: tests the four
// child boxes, sorts the children the ray enters by entry distance,
// continues into the nearest and pushes the others (farthest first); pops
// when the ray enters none.  An any-hit walk (kAny) skips the sort: it
// needs no order.  Returns false when the stack would overflow.
template <bool kCount, int kStride = kTraceThreads, bool kAny = false>
__device__ __forceinline__ bool visit_inner(const float4* __restrict__ nodes, int& node, const RayInv& r, int sx,
                                            int sy, int sz, float tmin, float tbest, int* stack, int* deep, int& sp,
                                            WorkCount& wc) {
  const float4* n = nodes + 8 * (size_t)node;
  float4 nx = __ldg(n + sx), fx = __ldg(n + 1 - sx);
  float4 ny = __ldg(n + 2 + sy), fy = __ldg(n + 3 - sy);
  float4 nz = __ldg(n + 4 + sz), fz = __ldg(n + 5 - sz);
  float4 lk = __ldg(n + 6);
  float d0 = child_entry(nx.x, ny.x, nz.x, fx.x, fy.x, fz.x, r, tmin, tbest);
  float d1 = child_entry(nx.y, ny.y, nz.y, fx.y, fy.y, fz.y, r, tmin, tbest);
  float d2 = child_entry(nx.z, ny.z, nz.z, fx.z, fy.z, fz.z, r, tmin, tbest);
  float d3 = child_entry(nx.w, ny.w, nz.w, fx.w, fy.w, fz.w, r, tmin, tbest);
  int l0 = __float_as_int(lk.x), l1 = __float_as_int(lk.y), l2 = __float_as_int(lk.z), l3 = __float_as_int(lk.w);
  if (kCount) {
    wc.visits++;
    wc.boxes += (l0 != kEmptyLink) + (l1 != kEmptyLink) + (l2 != kEmptyLink) + (l3 != kEmptyLink);
  }
  int cnt = (d0 < INFINITY) + (d1 < INFINITY) + (d2 < INFINITY) + (d3 < INFINITY);
  if (cnt == 0) {
    node = pop_stack<kStride>(stack, deep, sp);
  } else if (cnt == 1) {
    node = d0 < INFINITY ? l0 : d1 < INFINITY ? l1 : d2 < INFINITY ? l2 : l3;
  } else if (kAny) {
    // any hit needs no order: push the entered children as they come, go into the last
    if (sp + cnt - 1 > kStackSize) return false;
    int next = kSentinelLink;
    if (d0 < INFINITY) next = l0;
    if (d1 < INFINITY) {
      if (next != kSentinelLink) push_stack<kStride>(stack, deep, sp, next);
      next = l1;
    }
    if (d2 < INFINITY) {
      if (next != kSentinelLink) push_stack<kStride>(stack, deep, sp, next);
      next = l2;
    }
    if (d3 < INFINITY) {
      push_stack<kStride>(stack, deep, sp, next);
      next = l3;
    }
    node = next;
  } else {
    // five compare-exchanges sort four (distance, link) pairs; misses (+inf) go last
    order2(d0, l0, d1, l1);
    order2(d2, l2, d3, l3);
    order2(d0, l0, d2, l2);
    order2(d1, l1, d3, l3);
    order2(d1, l1, d2, l2);
    if (sp + cnt - 1 > kStackSize) return false;
    if (cnt == 4) push_stack<kStride>(stack, deep, sp, l3);
    if (cnt >= 3) push_stack<kStride>(stack, deep, sp, l2);
    push_stack<kStride>(stack, deep, sp, l1);
    node = l0;
  }
  return true;
}

// BVH traversal over the 4-wide tree with a per-thread stack: its first
// kStackShared entries live in shared memory (column `stack[i *
// kTraceThreads]`), deeper ones in local memory, which leaves most of L1 to
// nodes and primitives.  For lanes that walk on their own (the depth-first
// path kernel); traverse_warp below is the form for whole warps.
// Returns the hit record index (leaf order) or -1.  Sets *fail when the
// step cap or the stack depth is exceeded (the ray then counts as a miss).
template <bool kAny, bool kCount, int kStride = kTraceThreads>
__device__ int traverse(const DevScene& sc, const RayInv& r, float tmin, float& tbest, int* stack, int cap,
                        bool& fail, WorkCount& wc) {
  int best = -1, best_id = INT_MAX;
  if (sc.n_prims == 0) return -1;
  if (!sc.use_bvh) {
    leaf_hits<kAny, kCount>(sc.prims, 0, sc.n_prims, r, tmin, tbest, best, best_id, wc);
    return best;
  }
  int sp = 0;
  int node = sc.root;
  int steps = 0;
  int deep[kStackSize - kStackShared > 0 ? kStackSize - kStackShared : 1];   // entries below the shared part
  // rows of the near planes: lo when the direction is positive, else hi
  const int sx = r.idir.x < 0.f, sy = r.idir.y < 0.f, sz = r.idir.z < 0.f;
  // Speculative walk (Aila and Laine 2009): a lane that reaches a leaf
  // keeps it for later and walks on through inner nodes until every lane of
  // the warp holds a leaf, so that the warp's lanes test leaves together
  // instead of one after another.  Any order of the leaves gives the same
  // result (closest hits tie to the lower primitive id).
  int leaf = kSentinelLink;
  for (;;) {
    // inner nodes
    while (node >= 0) {
      if (++steps > cap) {
        fail = true;
        return kAny ? -1 : best;
      }
      if (node >= sc.n_nodes) {
        atomicOr(sc.status, kErrBadTree);
        fail = true;
        return -1;
      }
      if (!visit_inner<kCount, kStride, kAny>(sc.nodes, node, r, sx, sy, sz, tmin, tbest, stack, deep, sp, wc)) {
        fail = true;
        return kAny ? -1 : best;
      }
      if (node < 0 && node != kSentinelLink && leaf == kSentinelLink) {
        leaf = node;
        node = pop_stack<kStride>(stack, deep, sp);
      }
      if (!__any_sync(__activemask(), leaf == kSentinelLink)) break;
    }
    // leaves: the kept one first, then any the walk stands at
    while (leaf != kSentinelLink || (node < 0 && node != kSentinelLink)) {
      int cur;
      if (leaf != kSentinelLink) {
        cur = leaf;
        leaf = kSentinelLink;
      } else {
        cur = node;
        node = pop_stack<kStride>(stack, deep, sp);
      }
      int ls = leaf_start(cur), lc = leaf_count(cur);
      if (ls + lc > sc.n_prims) {
        atomicOr(sc.status, kErrBadTree);
        fail = true;
        return -1;
      }
      if (leaf_hits<kAny, kCount>(sc.prims, ls, lc, r, tmin, tbest, best, best_id, wc)) return best;
      if (node >= 0) break;
    }
    if (node == kSentinelLink && leaf == kSentinelLink) break;
  }
  return best;
}

// The same walk for a whole warp: all 32 lanes call it together, lanes with
// `part` false take no step.  The inner-node and leaf loops run while any
// lane has work of their kind and end in a warp vote, so the warp
// reconverges at every switch between the two instead of running its lanes'
// phases one after another.  Same results and errors as traverse().
template <bool kAny, bool kCount, int kStride = kTraceThreads>
__device__ int traverse_warp(const DevScene& sc, const RayInv& r, bool part, float tmin, float& tbest, int* stack,
                             int cap, bool& fail, WorkCount& wc) {
  int best = -1, best_id = INT_MAX;
  if (sc.n_prims == 0) return -1;
  if (!sc.use_bvh) {
    if (part) leaf_hits<kAny, kCount>(sc.prims, 0, sc.n_prims, r, tmin, tbest, best, best_id, wc);
    return best;
  }
  int sp = 0;
  int node = part ? sc.root : kSentinelLink;
  int steps = 0;
  int deep[kStackSize - kStackShared > 0 ? kStackSize - kStackShared : 1];
  const int sx = r.idir.x < 0.f, sy = r.idir.y < 0.f, sz = r.idir.z < 0.f;
  // Speculative, as traverse(): a lane at a leaf keeps it and takes inner
  // steps with the others until every lane still walking holds a leaf.
  int leaf = kSentinelLink;
  for (;;) {
    while (__any_sync(kFull, node >= 0)) {
      if (node >= 0) {
        if (++steps > cap) {
          fail = true;
          if (kAny) best = -1;
          node = kSentinelLink;
          leaf = kSentinelLink;
        } else if (node >= sc.n_nodes) {
          atomicOr(sc.status, kErrBadTree);
          fail = true;
          best = -1;
          node = kSentinelLink;
          leaf = kSentinelLink;
        } else if (!visit_inner<kCount, kStride, kAny>(sc.nodes, node, r, sx, sy, sz, tmin, tbest, stack, deep, sp,
                                                         wc)) {
          fail = true;
          if (kAny) best = -1;
          node = kSentinelLink;
          leaf = kSentinelLink;
        }
      }
      if (node < 0 && node != kSentinelLink && leaf == kSentinelLink) {
        leaf = node;
        node = pop_stack<kStride>(stack, deep, sp);
      }
      if (!__any_sync(kFull, leaf == kSentinelLink && node >= 0)) break;
    }
    if (!__any_sync(kFull, node != kSentinelLink || leaf != kSentinelLink)) break;
    while (__any_sync(kFull, leaf != kSentinelLink || (node < 0 && node != kSentinelLink))) {
      if (leaf != kSentinelLink || (node < 0 && node != kSentinelLink)) {
        int cur;
        if (leaf != kSentinelLink) {
          cur = leaf;
          leaf = kSentinelLink;
        } else {
          cur = node;
          node = pop_stack<kStride>(stack, deep, sp);
        }
        int ls = leaf_start(cur), lc = leaf_count(cur);
        if (ls + lc > sc.n_prims) {
          atomicOr(sc.status, kErrBadTree);
          fail = true;
          best = -1;
          node = kSentinelLink;
        } else if (leaf_hits<kAny, kCount>(sc.prims, ls, lc, r, tmin, tbest, best, best_id, wc)) {
          node = kSentinelLink;   // any hit: done
        }
      }
    }
  }
  return best;
}


// ---------------------------------------------------------------------------
// warp-aggregated queue push: one atomic per warp per call
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned warp_push(unsigned* counter, bool pred, unsigned cap, bool& ok,
                                              unsigned* status) {
  unsigned mask = __ballot_sync(kFull, pred);
  int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (mask) {
    int leader = __ffs(mask) - 1;
    if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
    base = __shfl_sync(kFull, base, leader);
  }
  unsigned pos = base + (unsigned)__popc(mask & ((1u << lane) - 1u));
  ok = pred && pos < cap;
  if (pred && pos >= cap && status) atomicOr(status, kErrQueueOverflow);
  return pos;
}

// A ray record; `code` is the path vertex the ray leads to (camera ray 1,
// children of vertex c: 2c reflection, 2c + 1 refraction), which keys the
// pass's random numbers there.
__device__ __forceinline__ void store_ray(float4* q, unsigned pos, f3 o, int pixel, f3 d, float tmax, f3 w,
                                          uint32_t code = 0u) {
  float4* p = q + 3 * (size_t)pos;
  p[0] = make_float4(o.x, o.y, o.z, __int_as_float(pixel));
  p[1] = make_float4(d.x, d.y, d.z, tmax);
  p[2] = make_float4(w.x, w.y, w.z, __uint_as_float(code));
}


__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// ---------------------------------------------------------------------------
// passes of a progressive render: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), counted by
// (pixel, pass, path vertex, slot) and keyed by the seed
// ---------------------------------------------------------------------------
struct PassInfo {
  uint32_t seed_lo, seed_hi;
  int pass, strata, jitter;
  int bounce;   // Monte-Carlo GI: one cosine-weighted diffuse bounce per vertex
};

constexpr uint32_t kSlotPixel = 0xFFFFFFFFu;    // the camera jitter's slot (light i uses slot i)
constexpr uint32_t kSlotBounce = 0xFFFFFFFEu;   // the diffuse bounce's slot
// bit 31 of a path-vertex code marks a ray made by a diffuse bounce; the
// other bits number the vertex (1 for the camera ray, 2c and 2c + 1 for the
// children of vertex c; vertex numbers stay below 2^18, so shifting a code
// left drops the mark)
constexpr uint32_t kCodeBounce = 0x80000000u;

__device__ __forceinline__ uint4 philox4x32(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// uniform in [0, 1) from the top 24 bits (exact in FP32)
__device__ __forceinline__ float unit24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// A stratified 2-D sample of the pass for (pixel, path vertex `code`,
// slot): over S x S consecutive passes each cell of an S x S grid is
// visited once, from a first cell fixed per pixel, vertex and slot; the
// point is uniform in its cell.
__device__ __forceinline__ void pass_sample(const PassInfo& ps, int pixel, uint32_t code, uint32_t slot, float& a,
                                            float& b) {
  const uint2 key = make_uint2(ps.seed_lo, ps.seed_hi);
  const uint4 r = philox4x32(make_uint4((uint32_t)pixel, (uint32_t)ps.pass, code, slot), key);
  const uint4 q = philox4x32(make_uint4((uint32_t)pixel, 0xFFFFFFFFu, code, slot), key);
  const uint32_t S = ps.strata > 0 ? (uint32_t)ps.strata : 1u, cells = S * S;
  const uint32_t cell = ((uint32_t)ps.pass % cells + q.x % cells) % cells;
  a = ((float)(cell % S) + unit24(r.x)) / (float)S;
  b = ((float)(cell / S) + unit24(r.y)) / (float)S;
}

// The image point a pass traces pixel (x, y) through.
__device__ __forceinline__ void pass_pixel_point(const PassInfo& ps, int pixel, int x, int y, float& px, float& py) {
  float jx = 0.5f, jy = 0.5f;
  if (ps.jitter) pass_sample(ps, pixel, 0u, kSlotPixel, jx, jy);
  px = (float)x + jx;
  py = (float)y + jy;
}

// ---------------------------------------------------------------------------
// shading of one hit (shared by the wavefront and the per-path kernels)
// ---------------------------------------------------------------------------
struct Surface {
  f3 p, n, albedo, emission;
  float ks, shin, rho, ior, eps;
  int kind;
  bool inside;
};

__device__ __forceinline__ Surface surface_at(const DevScene& sc, int hit, f3 o, f3 d, float t, float eps_scale) {
  Surface sf;
  float4 r0 = __ldg(&sc.prims[3 * (size_t)hit]);
  float4 r1 = __ldg(&sc.prims[3 * (size_t)hit + 1]);
  float4 r2 = __ldg(&sc.prims[3 * (size_t)hit + 2]);
  int mat = __float_as_int(r2.w);
  sf.p = o + d * t;
  f3 ng = geometric_normal(r0, r1, r2, sf.p);
  sf.inside = dot(d, ng) > 0.f;
  sf.n = sf.inside ? ng * -1.f : ng;
  float4 m0 = __ldg(&sc.mats[3 * mat]), m1 = __ldg(&sc.mats[3 * mat + 1]), m2 = __ldg(&sc.mats[3 * mat + 2]);
  sf.albedo = xyz(m0);
  sf.ks = m0.w;
  sf.shin = m1.x;
  sf.ior = m1.z;
  sf.kind = __float_as_int(m1.w);
  sf.rho = sf.kind == RT_MAT_MIRROR ? m1.y : 0.f;
  sf.emission = xyz(m2);
  sf.eps = eps_scale * fmaxf(1.0f, maxabs(sf.p));
  return sf;
}

// The Phong lobe's rv^shininess.  It only scales a shading term (no hit or
// shadow decision depends on it), so the hardware's fast exp2 / log2 path
// (__powf, a few ulps per unit of |shininess log2 rv|) is accurate enough:
// the terrain frame moves by at most 2.4e-7.
__device__ __forceinline__ float spec_pow(float rv, float shin) { return __powf(rv, shin); }

// Alg. 1 for one point light (Eq. 8 with point lights): the term the light
// adds if nothing blocks it, and the shadow ray that decides; false where
// n.l <= 0 (no shadow ray is cast).
// Whether point light L0 lies on the lit side of the hit (n.l > 0): the
// test light_term makes, computed the same way.
__device__ __forceinline__ bool light_faces(const Surface& sf, float4 L0) {
  const f3 l = normalize(xyz(L0) - sf.p);
  return dot(sf.n, l) > 0.f;
}

__device__ __forceinline__ bool light_term(const Surface& sf, f3 d, f3 w, float4 L0, float4 L1, f3& contrib, f3& o_s,
                                           f3& d_s, float& tmax) {
  f3 lp = xyz(L0);
  f3 l = normalize(lp - sf.p);
  float nl = dot(sf.n, l);
  if (!(nl > 0.f)) return false;
  f3 rl = sf.n * (2.f * nl) - l;                  // reflect(-l, n)
  float rv = -dot(rl, d);
  float spec = rv > 0.f ? spec_pow(rv, sf.shin) : 0.f;
  f3 f = sf.albedo * nl + mk3(sf.ks * spec, sf.ks * spec, sf.ks * spec);
  contrib = w * xyz(L1) * f * (1.f - sf.rho);
  o_s = sf.p + sf.n * sf.eps;
  f3 to_l = lp - o_s;
  float dist = sqrtf(dot(to_l, to_l));
  d_s = to_l * (1.f / dist);
  tmax = dist - sf.eps;
  return true;
}

constexpr float kPi = 3.14159265358979f;

// A sampled point y of an area light or of an emissive primitive, with the
// light's normal there, its radiance and area (the sampling density is
// 1 / area).
struct AreaPoint {
  f3 y, ny, L;
  float area;
  bool two_sided;   // triangles emit on both faces
};

// Light slot li (area lights first, then the emissive primitives in id
// order) at the pass's sample (a, b) in [0, 1)^2: a parallelogram at
// corner + a edge_u + b edge_v; a sphere uniformly over its surface
// (z = 1 - 2a, azimuth 2 pi b); a triangle uniformly, (a, b) folded into
// a + b <= 1.
__device__ __forceinline__ AreaPoint area_point(const DevScene& sc, int li, float a, float b) {
  AreaPoint q;
  if (li < sc.n_alights) {
    const float4* rec = sc.alights + 4 * li;
    const float4 A0 = __ldg(rec), A1 = __ldg(rec + 1), A2 = __ldg(rec + 2), A3 = __ldg(rec + 3);
    q.ny = mk3(A1.w, A2.w, A3.w);
    q.y = xyz(A0) + xyz(A1) * a + xyz(A2) * b;
    q.L = xyz(A3);
    q.area = A0.w;
    q.two_sided = false;
    return q;
  }
  const int id = __ldg(&sc.emitters[li - sc.n_alights]);
  const float4 r0 = __ldg(&sc.prims_id[3 * (size_t)id]);
  const float4 r1 = __ldg(&sc.prims_id[3 * (size_t)id + 1]);
  const float4 r2 = __ldg(&sc.prims_id[3 * (size_t)id + 2]);
  q.L = xyz(__ldg(&sc.mats[3 * __float_as_int(r2.w) + 2]));
  if (__float_as_int(r0.w) == kKindSphere) {
    const float z = 1.f - 2.f * a, rxy = sqrtf(fmaxf(0.f, 1.f - z * z));
    float sn, cs;
    sincospif(2.f * b, &sn, &cs);
    q.ny = mk3(rxy * cs, rxy * sn, z);
    q.y = xyz(r0) + q.ny * r1.x;
    q.area = 4.f * kPi * r1.y;
    q.two_sided = false;
  } else {
    if (a + b > 1.f) {
      a = 1.f - a;
      b = 1.f - b;
    }
    const f3 e1 = xyz(r1), e2 = xyz(r2), c = cross(e1, e2);
    const float len = sqrtf(dot(c, c));
    q.y = xyz(r0) + e1 * a + e2 * b;
    q.ny = c * (1.f / len);   // NaN for a degenerate triangle: its term is dropped below
    q.area = 0.5f * len;
    q.two_sided = true;
  }
  return q;
}

// One sampled light point at a hit: the point-light term of light_term
// times A cos(theta_y) / r^2 (Eq. 8 over the light's area, sampled with
// density 1 / A), and the shadow ray to the point; false where n.l <= 0
// or the light faces away (no shadow ray).
__device__ __forceinline__ bool area_term(const Surface& sf, f3 d, f3 w, const AreaPoint& q, f3& contrib, f3& o_s,
                                          f3& d_s, float& tmax) {
  const f3 to = q.y - sf.p;
  const float dist_c = sqrtf(dot(to, to));
  const f3 l = to * (1.f / dist_c);
  const float nll = dot(sf.n, l);
  float cos_y = -dot(l, q.ny);
  if (q.two_sided) cos_y = fabsf(cos_y);
  if (!(nll > 0.f) || !(cos_y > 0.f)) return false;
  f3 rl = sf.n * (2.f * nll) - l;                 // reflect(-l, n)
  float rv = -dot(rl, d);
  float spec = rv > 0.f ? spec_pow(rv, sf.shin) : 0.f;
  f3 f = sf.albedo * nll + mk3(sf.ks * spec, sf.ks * spec, sf.ks * spec);
  const float G = q.area * cos_y / (dist_c * dist_c);
  contrib = w * q.L * f * (G * (1.f - sf.rho));
  o_s = sf.p + sf.n * sf.eps;
  f3 to_l = q.y - o_s;
  float dist = sqrtf(dot(to_l, to_l));
  d_s = to_l * (1.f / dist);
  tmax = dist - sf.eps;
  return true;
}

// Reflection / refraction rays of a hit (Fig. 3): mirror rho -> reflection
// of weight rho; dielectric -> Fresnel-Schlick R reflection and 1-R
// refraction (none on total internal reflection).
struct Children {
  bool want_r, want_t;
  bool bounce;   // the second child is a diffuse bounce, not a refraction
  f3 or_, dr, wr, ot, dt, wt;
};

__device__ __forceinline__ Children children_of(const Surface& sf, f3 d, f3 w) {
  Children c;
  c.want_r = c.want_t = c.bounce = false;
  c.or_ = sf.p + sf.n * sf.eps;
  c.ot = sf.p - sf.n * sf.eps;
  c.dr = c.dt = mk3(0, 0, 1);
  c.wr = c.wt = mk3(0, 0, 0);
  float dn = dot(d, sf.n);
  if (sf.kind != RT_MAT_DIELECTRIC) {
    if (sf.rho > 0.f) {
      c.want_r = true;
      c.dr = normalize(d - sf.n * (2.f * dn));
      c.wr = w * sf.rho;
    }
  } else {
    float n1 = sf.inside ? sf.ior : 1.f, n2 = sf.inside ? 1.f : sf.ior;
    float eta = n1 / n2;
    float ci = -dn;
    float k = 1.f - eta * eta * (1.f - ci * ci);
    float R = 1.f;
    if (k >= 0.f) {
      float ct = sqrtf(k);
      float r0 = (n1 - n2) / (n1 + n2);
      r0 *= r0;
      float cs = n1 <= n2 ? ci : ct;
      float x = 1.f - cs;
      R = r0 + (1.f - r0) * x * x * x * x * x;
      c.want_t = true;
      c.dt = normalize(d * eta + sf.n * (eta * ci - ct));
      c.wt = w * (1.f - R);
    }
    c.want_r = true;
    c.dr = normalize(d - sf.n * (2.f * dn));
    c.wr = w * R;
  }
  return c;
}

// A cosine-weighted direction about the unit normal n for (a, b) in
// [0, 1)^2: Malley's method (the point (sqrt(a), 2 pi b) of the unit disk in
// polar form, lifted onto the hemisphere), in the branch-free orthonormal
// basis of Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT
// 2017), with the sign taken as n.z >= 0.
__device__ __forceinline__ f3 cosine_dir(f3 n, float a, float b) {
  const float sg = n.z >= 0.f ? 1.f : -1.f;
  const float k = -1.f / (sg + n.z);
  const float m = n.x * n.y * k;
  const f3 t1 = mk3(1.f + sg * n.x * n.x * k, sg * m, -sg * n.x);
  const f3 t2 = mk3(m, sg + n.y * n.y * k, -n.y);
  const float r = sqrtf(a);
  float sn, cs;
  sincospif(2.f * b, &sn, &cs);
  return normalize(t1 * (r * cs) + t2 * (r * sn) + n * sqrtf(fmaxf(0.f, 1.f - a)));
}

// Monte-Carlo GI (Eq. 8's hemisphere integral over the Lambert lobe): a
// non-dielectric hit with 1 - rho > 0 and some albedo > 0 sends one
// cosine-weighted ray from the offset point above it, of weight
// pi (1 - rho) albedo (f_r = albedo, as in the light terms, over the
// density cos / pi).  It takes the second child's place, which only a
// dielectric uses otherwise.  vcode: the hit's vertex (without the mark).
__device__ __forceinline__ void add_bounce(Children& c, const Surface& sf, f3 w, const PassInfo& ps, int pixel,
                                           uint32_t vcode) {
  if (sf.kind == RT_MAT_DIELECTRIC || !((1.f - sf.rho) > 0.f) ||
      !(fmaxf(fmaxf(sf.albedo.x, sf.albedo.y), sf.albedo.z) > 0.f))
    return;
  float a, b;
  pass_sample(ps, pixel, vcode, kSlotBounce, a, b);
  c.want_t = true;
  c.bounce = true;
  c.ot = c.or_;
  c.dt = cosine_dir(sf.n, a, b);
  c.wt = w * sf.albedo * (kPi * (1.f - sf.rho));
}

}  // namespace rtb
