// rtb_internal.cuh - device layouts and device functions of the sm_103a
// Whitted tracer.  Included by every .cu of librtb.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rtb.h"

namespace rtb {

// ---------------------------------------------------------------------------
// Tunables
// ---------------------------------------------------------------------------
constexpr int kStackSize = 96;       // traversal stack entries per thread (up to 3 pushes per 4-wide node)
#ifndef RTB_STACK_SHARED
#define RTB_STACK_SHARED 16
#endif
constexpr int kStackShared = RTB_STACK_SHARED;   // of which the top ones live in shared memory; deeper ones in local memory
constexpr int kTraceThreads = 128;   // threads per block of the traversal kernels
constexpr int kMaxLeaf = 8;          // primitives per leaf after SAH collapsing
#ifndef RTB_COST_TRAV
#define RTB_COST_TRAV 1.0f
#endif
constexpr float kCostTrav = RTB_COST_TRAV;   // SAH constants: one node step vs one primitive test
constexpr float kCostIsect = 1.0f;

// Bits of the device status word.
constexpr unsigned kErrQueueOverflow = 1u;
constexpr unsigned kErrTraversalLimit = 2u;
constexpr unsigned kErrBadTree = 4u;      // a link outside the node / primitive arrays
constexpr unsigned kErrBadMaterial = 16u; // rt_scene_update met a material index out of range

// Primitive kinds (row0.w of a primitive record).
constexpr int kKindTriangle = 0;
constexpr int kKindSphere = 1;

// Traversal-stack sentinel: popped from an empty stack.
constexpr int kSentinel = 0x7fffffff;
// Link of an unused slot of a 4-wide node; its box is inverted (lo = +inf,
// hi = -inf), which the ordered slab test never hits.  Equal to the
// traversal's empty-stack value, so that following it can only end a walk.
constexpr int kEmptyLink = (int)0x80000000;

// ---------------------------------------------------------------------------
// Device layouts
//
// Primitive record, 3 x float4 = 48 B, 16-B aligned:
//   triangle: (v0.xyz, kind) (e1.xyz, prim id) (e2.xyz, material)
//   sphere  : (c.xyz,  kind) (r, r*r, 0, prim id) (0, 0, 0, material)
//   (integers stored with __int_as_float)
// Binary BVH node (build output and export format), 4 x float4 = 64 B; the
// two child boxes are stored by axis so that one float4 holds an axis slab
// pair of both children:
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (link0, link1, -, -)
// 4-wide traversal node, 8 x float4 = 128 B (one cache line), one float4 per
// box plane over the four children, so that a ray picks its near and far
// planes by the sign of its direction alone:
//   m0 = lo.x[0..3]  m1 = hi.x[0..3]  m2 = lo.y  m3 = hi.y  m4 = lo.z  m5 = hi.z
//   m6 = (link0..link3)  m7 = unused
// link >= 0: internal node index; link < 0: leaf = ~(start << 3 | count-1)
// over primitive records [start, start+count) in leaf order; kEmptyLink:
// an unused slot.
// Material, 3 x float4: (albedo.rgb, ks) (shininess, reflectivity, ior, kind)
//   (emission.rgb, 0).
// Light, 2 x float4: (position, 0) (intensity, 0).
// Ray record, 3 x float4 = 48 B:
//   (o.xyz, pixel) (d.xyz, tmax) (w.rgb, -)
// ---------------------------------------------------------------------------
__host__ __device__ inline int leaf_link(int start, int count) { return ~((start << 3) | (count - 1)); }
__host__ __device__ inline int leaf_start(int link) { return (~link) >> 3; }
__host__ __device__ inline int leaf_count(int link) { return ((~link) & 7) + 1; }

// Everything a traversal kernel needs, by value.
struct DevScene {
  const float4* prims;      // 3 per primitive, leaf order (BVH) or id order
  const float4* nodes;      // 4-wide nodes, 8 float4 each, one per binary node slot
  const float4* mats;       // 3 per material
  const float4* lights;     // 2 per light
  const float4* alights;    // 4 per area light: (corner, area) (edge_u, n.x) (edge_v, n.y) (radiance, n.z)
  const float4* prims_id;   // 3 per primitive, id order (emitters are looked up here)
  const int* emitters;      // ids of the primitives whose material emits, ascending
  int n_prims;
  int n_lights;
  int n_alights;
  int n_emitters;
  int n_nodes;              // node slots (links are checked against it)
  int root;                 // root node index (-1: no node)
  int use_bvh;
  int traversal_cap;
  unsigned* status;
};

// ---------------------------------------------------------------------------
// Host-side scene
// ---------------------------------------------------------------------------
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  unsigned gen = 0;   // bumped by every allocation (the address alone may repeat)
};

struct GraphCache;

}  // namespace rtb

struct rt_scene {
  int device = 0;
  int64_t n_spheres = 0, n_tris = 0, n_prims = 0, n_mats = 0, n_lights = 0;
  float bbox_lo[3] = {0.f, 0.f, 0.f}, bbox_hi[3] = {1.f, 1.f, 1.f};   // of the input geometry
  // geometry
  rtb::Buf raw_sph, raw_tri;     // raw ABI structs on the device (for repacking)
  rtb::Buf prims_id;             // packed records, primitive-id order
  rtb::Buf prims_leaf;           // packed records, BVH leaf order
  rtb::Buf mats, lights;
  rtb::Buf alights;              // area lights, 4 float4 each
  rtb::Buf pass_img;             // one pass of a progressive render
  int64_t n_alights = 0;
  rtb::Buf emitters;             // int ids of the emissive primitives, ascending
  int64_t n_emitters = 0;
  // BVH
  bool built = false;
  int root = -1;
  int64_t n_nodes_total = 0;     // slots in `nodes` (LBVH internal + top nodes)
  rtb::Buf nodes;
  rtb::Buf nodes4;               // 4-wide traversal layout, indexed like the binary nodes
  int64_t n_nodes4 = 0;
  rtb::Buf build_tmp;            // scratch for the build, carved below
  size_t build_tmp_n = 0;
  rtb::Buf build_info;           // device-side build results (BuildInfo)
  float last_build_ms = 0.f;
  int last_build_launches = 0;
  int lbvh_cut = 0;              // > 0: the LBVH nodes over this many primitives still await their refit
  unsigned bounds_gen = 0;       // build_tmp.gen whose centroid bounds hold their reset value
  // the build's launches captured into a CUDA graph, replayed by the builds
  // that find the same buffers (bvh.cu)
  cudaGraphExec_t build_exec = nullptr;
  cudaStream_t build_cap = nullptr;   // the stream the build is captured on
  unsigned build_key[6] = {0, 0, 0, 0, 0, 0};
  bool build_cap_failed = false;
  int build_root = 0, build_lbvh_cut = 0, build_launches = 0;
  int64_t build_nodes_total = 0, build_nodes4 = 0;
  // the build runs the parts that do not depend on the top rebuild on the
  // side stream (below) beside that rebuild, between these two events
  cudaEvent_t ev_build_fork = nullptr, ev_build_join = nullptr;
  // render
  rtb::Buf rayq[2], shadowq[2], counters, fb_host_stage;
  rtb::Buf fb_fixed;             // RT_FLAG_DETERMINISTIC: the frame's 64-bit fixed-point sums
  // rt_render_host_async: two device images, each copied to the host on the
  // copy stream while the next frame renders into the other
  rtb::Buf fb_stage[2];
  int stage_next = 0;
  // the last frame's copy, queued when the next frame is (or at a sync)
  int copy_pending = -1;         // its image (fb_stage index), or -1
  float* copy_dst = nullptr;
  size_t copy_bytes = 0;
  cudaEvent_t ev_issue = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_rendered[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
  cudaStream_t side = nullptr;   // runs each depth's shadow kernel beside the next depth's trace
  cudaEvent_t ev_traced[RT_MAX_DEPTH + 1], ev_shadowed[RT_MAX_DEPTH + 1];
  int64_t ray_cap = 0, shadow_cap = 0;
  unsigned* status = nullptr;    // device status word
  int sm_count = 0;
  int trace_blocks = 0, shadow_blocks = 0, paths_blocks = 0;
  rtb::GraphCache* graphs = nullptr;
  // stage timing of the last frame rendered with RT_FLAG_STAGE_TIMING
  std::vector<cudaEvent_t> tev;  // reused across frames
  std::vector<int> tkind;        // kind of event pair i: 0 trace, 1 shadow, 3 whole frame
  int tcount = 0;
};

namespace rtb {

// Error reporting helpers (scene.cu).
rt_status set_error(rt_status st, const std::string& msg);
rt_status cuda_error(cudaError_t e, const char* where);
rt_status ensure(Buf& b, size_t bytes);
void release(Buf& b);

// BVH (bvh.cu).
rt_status bvh_build(rt_scene* s, cudaStream_t st);

// The scene's side stream and its per-depth events (render.cu).  The build
// uses it too: a third stream of the scene, measured, made the frame's two
// streams stop overlapping in back-to-back steps (1.34 against 1.20 ms).
rt_status ensure_side_stream(rt_scene* s);

// Queues the copy rt_render_host_async left pending, if any, after the
// frame that rendered it (render.cu).
rt_status issue_pending_copy(rt_scene* s);

// Kernel launch helpers shared by render.cu.
DevScene dev_scene(const rt_scene* s, bool use_bvh);
struct CamBasis;
// Pinhole camera basis of a frame (host FP32 arithmetic) and its validation.
CamBasis camera_basis(const rt_camera* c, int W, int H);
bool finite_cam(const rt_camera* c);
void preload_frame_kernels(int device);   // loads the frame kernels in a fixed order (once per device)

// ---------------------------------------------------------------------------
// Device math
// ---------------------------------------------------------------------------
struct f3 {
  float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 xyz(float4 a) { return {a.x, a.y, a.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ f3 operator*(f3 a, f3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 normalize(f3 a) {
  float inv = 1.0f / sqrtf(dot(a, a));
  return a * inv;
}
__device__ __forceinline__ float maxabs(f3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }
__device__ __forceinline__ float maxc(f3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }

// Pinhole camera basis (vertical FOV, pixel centres at +0.5, row 0 on top).
struct CamBasis {
  f3 eye, f, r, u;
  float h, aspect;
};

// The ray through image point (px, py) in pixel units; the centre of
// pixel (x, y) is (x + 0.5, y + 0.5).
__device__ __forceinline__ void camera_ray_at(const CamBasis& cb, int W, int H, float px, float py, f3& o, f3& d) {
  float sx = (2.0f * px / (float)W - 1.0f) * cb.h * cb.aspect;
  float ty = (1.0f - 2.0f * py / (float)H) * cb.h;
  o = cb.eye;
  d = normalize(cb.f + cb.r * sx + cb.u * ty);
}

__device__ __forceinline__ void camera_ray(const CamBasis& cb, int W, int H, int x, int y, f3& o, f3& d) {
  camera_ray_at(cb, W, H, (float)x + 0.5f, (float)y + 0.5f, o, d);
}

// ---------------------------------------------------------------------------
// Intersection (FP32)
// ---------------------------------------------------------------------------
// Moller-Trumbore without the division for rejected triangles: with
// s = sign(det), u' = s T.P, v' = s d.Q, t' = s e2.Q the hit test
// u >= 0, v >= 0, u + v <= 1, tmin < t < tbest becomes
// u' >= 0, v' >= 0, u' + v' <= |det|, tmin|det| < t' < tbest|det|.
// kUpTo: accept t == tbest too (the caller breaks the tie by primitive id).
template <bool kUpTo>
__device__ __forceinline__ bool hit_triangle(f3 o, f3 d, float4 r0, float4 r1, float4 r2, float tmin,
                                             float tbest, float& t_out) {
  f3 v0 = xyz(r0), e1 = xyz(r1), e2 = xyz(r2);
  f3 P = cross(d, e2);
  float det = dot(e1, P);
  f3 T = o - v0;
  float u = dot(T, P);
  f3 Q = cross(T, e1);
  float v = dot(d, Q);
  float t = dot(e2, Q);
  float adet = fabsf(det);
  float sg = det < 0.0f ? -1.0f : 1.0f;
  u *= sg;
  v *= sg;
  t *= sg;
  bool hit = (det != 0.0f) & (u >= 0.0f) & (v >= 0.0f) & (u + v <= adet) & (t > tmin * adet) &
             (kUpTo ? (t <= tbest * adet) : (t < tbest * adet));
  if (hit) t_out = t / adet;
  return hit;
}

// Ray-sphere, Eq. 9-12, in the form that avoids cancellation: with unit d,
// b' = f.d (f = o - c), disc = r^2 - |f - b' d|^2, c' = f.f - r^2,
// q = -b' - sign(b') sqrt(disc); the roots are c'/q and q.
template <bool kUpTo>
__device__ __forceinline__ bool hit_sphere(f3 o, f3 d, float4 r0, float4 r1, float tmin, float tbest,
                                           float& t_out) {
  f3 c = xyz(r0);
  float rad2 = r1.y;
  f3 f = o - c;
  float b = dot(f, d);
  f3 h = f - d * b;
  float disc = rad2 - dot(h, h);
  if (disc < 0.0f) return false;
  float cc = dot(f, f) - rad2;
  float sq = sqrtf(disc);
  float q = b >= 0.0f ? -b - sq : -b + sq;
  float t0, t1;
  if (q == 0.0f) {
    t0 = t1 = 0.0f;
  } else {
    t0 = cc / q;
    t1 = q;
  }
  if (t0 > t1) {
    float x = t0;
    t0 = t1;
    t1 = x;
  }
  float t = t0 > tmin ? t0 : t1;
  if (t > tmin && (kUpTo ? t <= tbest : t < tbest)) {
    t_out = t;
    return true;
  }
  return false;
}

// Geometric normal at a hit on record (r0, r1, r2), unit length.
__device__ __forceinline__ f3 geometric_normal(float4 r0, float4 r1, float4 r2, f3 p) {
  if (__float_as_int(r0.w) == kKindSphere) return (p - xyz(r0)) * (1.0f / r1.x);
  return normalize(cross(xyz(r1), xyz(r2)));
}

}  // namespace rtb
